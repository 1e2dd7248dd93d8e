"""ADMM against the interior-point method on the condensed QP of one real-time iteration.

    python -m paper_2602_17601_b300.ipm_compare [--reps 5]

Builds the chain of 1000 nodes (K = 3, W = 128, N = 20, nu = 8, 5 spheres), linearises and
condenses at the first step's point (u_hat = 0) in the mixed form, and solves the same QP
with gm_qp_solve (ADMM, adaptive rho) and gm_qp_solve_ipm (Mehrotra predictor-corrector),
both to the workload's tolerance.  Device milliseconds come from CUDA events around each
solve; the IPM synchronises with the host every two iterations, which its time includes.
Prints one JSON line.
"""
from __future__ import annotations


def main(argv=None):
    import argparse
    import json

    import numpy as np
    import torch

    from . import GM_PREC_MIXED
    from .rti import RTIProblem
    from synth import paper_chain

    ap = argparse.ArgumentParser()
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--max-iter", type=int, default=80)
    a = ap.parse_args(argv)
    wl = paper_chain()
    prob = RTIProblem.from_workload(wl, precision=GM_PREC_MIXED)
    x_hat, A, B, c = prob.linearize(wl.x0, np.zeros((wl.N, wl.nu), np.float32))
    H, g, Ct, dt = prob.condense(x_hat, A, B, c)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        out, ms = None, []
        for _ in range(a.reps + 1):
            torch.cuda.synchronize()
            ev[0].record()
            out = fn()
            ev[1].record()
            torch.cuda.synchronize()
            ms.append(ev[0].elapsed_time(ev[1]))
        return out, float(np.median(ms[1:])), prob.read_stats()

    (Ua, _), ms_a, st_a = timed(lambda: prob.qp_solve(H, g, Ct, dt))
    (Ui, _), ms_i, st_i = timed(lambda: prob.qp_solve_ipm(H, g, Ct, dt, max_iter=a.max_iter))
    keep = ("status", "iters", "converged", "r_prim", "r_dual", "kkt_stat", "kkt_prim", "kkt_dual", "kkt_comp")
    rep = {"workload": "chain1000_K3_W128_N20_nu8_spheres5", "n": int(prob.nU), "rows": int(prob.rows_c),
           "tol": wl.tol, "reps": a.reps,
           "admm": {"ms": ms_a, **{k: st_a[k] for k in keep}},
           "ipm": {"ms": ms_i, **{k: st_i[k] for k in keep}},
           "max_abs_U_diff": float((Ua - Ui).abs().max()), "max_abs_U": float(Ua.abs().max()),
           "device": torch.cuda.get_device_name()}
    print(json.dumps(rep), flush=True)
    return rep


if __name__ == "__main__":
    main()
