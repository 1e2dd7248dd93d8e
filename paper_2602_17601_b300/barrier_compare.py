"""Obstacles as constraints against obstacles as barrier costs, one real-time iteration at a time.

    python -m paper_2602_17601_b300.barrier_compare [--steps 20] [--mu 1e-3] [--delta 5e-3]

The chain of 1000 nodes (K = 3, W = 128, N = 20, nu = 8, 5 spheres of radius 0.02) in two
scenarios: spheres 0.15 from their node at the initial state ("far", the benchmark workload)
and 0.01 from it ("near").  Each runs in the mixed form with the
step replayed as a CUDA graph, stepped repeatedly from its initial state (each step shifts
its own solution into the next linearisation point), once with the linearised sphere rows as
QP constraints and once with them in the cost as relaxed log barriers (gm_constr
barrier_mu / barrier_delta).  Reports device milliseconds per step (CUDA events), ADMM
iterations and status of the last step, and the smallest sphere clearance of the GNN
rollout under the returned inputs.  Prints one JSON line.
"""
from __future__ import annotations


def main(argv=None):
    import argparse
    import json

    import numpy as np
    import torch

    from . import GM_PREC_MIXED, gm_rollout
    from .rti import RTIProblem
    from synth import paper_chain

    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--mu", type=float, default=1e-3)
    ap.add_argument("--delta", type=float, default=5e-3)
    a = ap.parse_args(argv)

    def run(wl, barrier):
        sph = wl.spheres.astype(np.float64)
        prob = RTIProblem.from_workload(wl, precision=GM_PREC_MIXED, graph=True, barrier=barrier)
        x = torch.as_tensor(wl.x0.reshape(-1), dtype=torch.float32, device="cuda")
        U = prob.empty(prob.nU)
        for _ in range(a.warmup):
            prob.step(x, U)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record()
        for _ in range(a.steps):
            prob.step(x, U)
        ev[1].record()
        torch.cuda.synchronize()
        st = prob.read_stats()
        xs = prob.empty(wl.N + 1, wl.M, 6)
        gm_rollout(prob.ctx, x, U, wl.N, xs)
        p = xs.cpu().numpy().astype(np.float64)[1:, :, :3]
        clear = np.linalg.norm(p[:, :, None, :] - sph[None, None, :, :3], axis=-1) - sph[None, None, :, 3]
        out = {"ms_per_step": ev[0].elapsed_time(ev[1]) / a.steps, "admm_iters": st["iters"],
               "status": st["status"], "converged": st["converged"], "min_clearance": float(clear.min()),
               "max_abs_U": float(U.abs().max())}
        prob.close()
        return out

    rep = {"workload": "chain1000_K3_W128_N20_nu8_spheres5", "form": "mixed, graph replay",
           "steps": a.steps, "warmup": a.warmup, "mu": a.mu, "delta": a.delta}
    for name, clear in (("far", 0.15), ("near", 0.01)):
        wl = paper_chain(sphere_clear=clear)
        rep[name] = {"sphere_clearance_at_x0": clear, "constraints": run(wl, None),
                     "barrier": run(wl, (a.mu, a.delta))}
    rep["device"] = torch.cuda.get_device_name()
    print(json.dumps(rep), flush=True)
    return rep


if __name__ == "__main__":
    main()
