"""Batched real-time iterations: many independent MPC instances stepped as one CUDA graph.

`Batch` wraps gm_batch_* around a list of RTIProblem instances (any node count,
horizon and input count): the first step runs the instances one after another,
the second captures every instance's step as a child graph of one parent graph,
and later steps replay it with a single launch, the instances' kernels running
side by side.  `cfg4_instances` draws the uneven batch of the cfg4 workload, and
`main` times it against stepping the same instances one after another.  Launch
shapes (ADMM and factor grids, stages per reverse-pass launch) come from the
autotuner (`autotune.py`).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import GM_ERR_INFEASIBLE, STATS_BYTES, Constr, Cost, _check, _lib, _stream


class Batch:
    def __init__(self, problems):
        self.problems = list(problems)
        n = len(self.problems)
        ctxs = (C.c_void_p * n)(*[p.ctx.value if isinstance(p.ctx, C.c_void_p) else p.ctx for p in self.problems])
        h = C.c_void_p()
        _check("gm_batch_create", _lib.gm_batch_create(ctxs, n, C.byref(h)))
        self.h = h
        self._x = (C.c_void_p * n)(*[p._x.data_ptr() for p in self.problems])
        self._U = (C.c_void_p * n)(*[p._U.data_ptr() for p in self.problems])
        self._stats = (C.c_void_p * n)(*[p.stats.data_ptr() for p in self.problems])
        self._costs = (Cost * n)(*[p.cost for p in self.problems])
        self._cons = (Constr * n)(*[p.constr for p in self.problems])

    def __del__(self):
        if getattr(self, "h", None):
            _lib.gm_batch_destroy(self.h)
            self.h = None

    def set_states(self, xs):
        """Copy each instance's measured state into its step buffer (device or host arrays)."""
        for p, x in zip(self.problems, xs):
            p._x.copy_(p.torch.as_tensor(x, dtype=p.torch.float32).reshape(-1), non_blocking=True)

    def step(self, stream=None):
        _check("gm_batch_rti_step", _lib.gm_batch_rti_step(self.h, self._x, self._costs, self._cons, self._U,
                                                           self._stats, _stream(stream)))

    def state(self):
        r, n = C.c_int(), C.c_int()
        _check("gm_batch_state", _lib.gm_batch_state(self.h, C.byref(r), C.byref(n)))
        return r.value, n.value

    def set_lanes(self, lanes):
        """At most this many lanes in the next capture (0: the plan's)."""
        _check("gm_batch_set_lanes", _lib.gm_batch_set_lanes(self.h, int(lanes)))

    def lanes(self):
        n = C.c_int()
        _check("gm_batch_lanes", _lib.gm_batch_lanes(self.h, C.byref(n)))
        return n.value

    def U(self, i):
        return self.problems[i]._U


def cfg4_instances(n=256, first_seed=1000, constrained=True, Ms=(50, 1000), Ns=(10, 15, 20, 30), nus=(4, 8)):
    """The uneven batch: M ~ U[Ms], N from Ns, nu from nus, per-instance seeds first_seed + b for the
    shape draw, state, reference and spheres; the chain-of-1000 GNN weights (seed 0) shared by all
    instances with the same nu; box + 5 spheres (or box only)."""
    from synth import paper_chain
    rng = np.random.default_rng(first_seed)
    out = []
    for b in range(n):
        M = int(rng.integers(Ms[0], Ms[1] + 1))
        N = int(rng.choice(Ns))
        nu = int(rng.choice(nus))
        out.append(paper_chain(seed=first_seed + b, M=M, N=N, nu=nu, w_seed=0,
                               n_spheres=5 if constrained else 0))
    return out


def problems_for(workloads, precision, tuned=None, chunk_mb=256, max_iter=None, warm=False):
    """RTIProblem per workload with the autotuned launch shapes of its bucket (if given; they
    override chunk_mb); warm starts each instance's ADMM from its own shifted previous solution
    (gm_ctx_set_warm)."""
    from .autotune import bucket_of
    from .rti import RTIProblem
    probs = []
    for wl in workloads:
        kw = dict(precision=precision, chunk_mb=chunk_mb, warm=warm)
        if max_iter:
            kw["max_iter"] = max_iter
        if tuned:
            kw.update(tuned.get(bucket_of(wl.M), {}))
        probs.append(RTIProblem.from_workload(wl, **kw))
    return probs


def main(argv=None):
    import argparse
    import json
    import time

    import torch

    from . import GM_PREC_FP32, GM_PREC_MIXED, read_stats
    from .autotune import load_or_tune
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--form", default="mixed", choices=["mixed", "fp32"])
    ap.add_argument("--box-only", action="store_true")
    ap.add_argument("--cache", default=None, help="autotuner JSON cache (default: tuned here, not stored)")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--lanes", type=int, default=0, help="at most this many lanes (0: gm_batch_plan)")
    ap.add_argument("--warm", action="store_true", help="receding-horizon ADMM warm start per instance")
    ap.add_argument("--max-iter", type=int, default=1000,
                    help="ADMM cap: a linearised sphere an instance's rollout drifts into can make its QP "
                         "infeasible, and ADMM then runs to the cap")
    a = ap.parse_args(argv)
    prec = GM_PREC_MIXED if a.form == "mixed" else GM_PREC_FP32
    t0 = time.perf_counter()
    wls = cfg4_instances(a.n, constrained=not a.box_only)
    tuned = None if a.no_tune else load_or_tune(a.cache, prec)
    t_tune = time.perf_counter() - t0
    probs = problems_for(wls, prec, tuned, max_iter=a.max_iter, warm=a.warm)
    t_build = time.perf_counter() - t0 - t_tune
    batch = Batch(probs)
    batch.set_lanes(a.lanes)
    batch.set_states([wl.x0 for wl in wls])
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    # one after another, plain launches
    for p in probs:
        p.reset()
    for p, wl in zip(probs, wls):
        p.step(p._x, p._U)
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(a.steps):
        for p in probs:
            p.step(p._x, p._U)
    ev[1].record()
    torch.cuda.synchronize()
    ms_seq = ev[0].elapsed_time(ev[1]) / a.steps
    # batched: warm-up (plain, then capture), then replays
    for p in probs:
        p.reset()
    batch.step()
    batch.step()
    torch.cuda.synchronize()
    ev[2].record()
    for _ in range(a.steps):
        batch.step()
    ev[3].record()
    torch.cuda.synchronize()
    ms_batch = ev[2].elapsed_time(ev[3]) / a.steps
    st = [read_stats(p.stats) for p in probs]
    rep = {"instances": a.n, "form": a.form, "admm_warm_start": bool(a.warm),
           "constraints": "box" if a.box_only else "box + 5 spheres",
           "M_range": [int(min(w.M for w in wls)), int(max(w.M for w in wls))],
           "N_values": sorted({int(w.N) for w in wls}), "nu_values": sorted({int(w.nu) for w in wls}),
           "steps": a.steps, "sequential_ms_per_batch_step": ms_seq, "batched_ms_per_batch_step": ms_batch,
           "sequential_instance_steps_per_s": a.n * 1000.0 / ms_seq,
           "batched_instance_steps_per_s": a.n * 1000.0 / ms_batch, "speedup": ms_seq / ms_batch,
           "graph": dict(zip(("replayed", "captures"), batch.state())), "lanes": batch.lanes(),
           "converged": int(sum(s["converged"] for s in st)), "status_nonzero": int(sum(s["status"] != 0 for s in st)),
           "infeasible": int(sum(s["status"] == GM_ERR_INFEASIBLE for s in st)),
           "status_counts": {str(k): int(v) for k, v in zip(*np.unique([s["status"] for s in st], return_counts=True))},
           "admm_iters_mean": float(np.mean([s["iters"] for s in st])), "admm_max_iter": a.max_iter,
           "admm_iters_converged_mean": float(np.mean([s["iters"] for s in st if s["converged"]] or [0])),
           "workspace_gb": float(sum(p.workspace.numel() for p in probs) / 2**30),
           "tuned": tuned, "seconds": {"tune": t_tune, "build": t_build},
           "device": torch.cuda.get_device_name()}
    print(json.dumps(rep), flush=True)
    return rep


if __name__ == "__main__":
    main()
