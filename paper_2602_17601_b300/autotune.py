"""Launch-shape autotuner for batched instances.

When many instances share the GPU, each instance's cooperative kernels (the ADMM
iterations and the FP64 factorisation) should take only a slice of the SMs so
that several run side by side; how large a slice pays depends on the instance's
size.  For every node-count bucket the tuner builds a small batch of
representative instances (the cfg4 GNN, N = 20, nu = 8, box + 5 spheres), times
a graph-replayed batch step for each candidate (ADMM grid, factor grid), and
keeps the fastest.  The result is a JSON cache keyed by bucket:

    {"M<=250": {"admm_grid": 16, "factor_grid": 16}, ...}

Timing is on the device (CUDA events around replays, after a capture and a
warm-up replay).
"""
from __future__ import annotations

import json
import os

BUCKETS = (250, 500, 750, 1000)
ADMM_GRIDS = (8, 16, 32, 64)
FACTOR_GRIDS = (8, 16, 32)


def bucket_of(M):
    for b in BUCKETS:
        if M <= b:
            return f"M<={b}"
    return f"M<={BUCKETS[-1]}"


def time_candidate(precision, M, admm_grid, factor_grid, replicas=8, steps=3, seed=77):
    """Device ms of one graph-replayed step of a batch of `replicas` instances of M nodes."""
    import torch

    from synth import paper_chain
    from .batch import Batch
    from .rti import RTIProblem
    probs = []
    for r in range(replicas):
        wl = paper_chain(seed=seed + r, M=M, N=20, nu=8, w_seed=0)
        probs.append(RTIProblem.from_workload(wl, precision=precision, admm_grid=admm_grid,
                                              factor_grid=factor_grid, chunk_mb=256))
        probs[-1]._x.copy_(torch.as_tensor(wl.x0).reshape(-1))
    b = Batch(probs)
    b.step()            # plain launches
    b.step()            # capture + replay
    b.step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        b.step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    del b, probs
    torch.cuda.empty_cache()
    return ms


def tune(precision, replicas=8, log=None):
    best = {}
    for hi in BUCKETS:
        M = max(50, hi - 125)                     # representative size of the bucket
        scores = []
        for ag in ADMM_GRIDS:
            for fg in FACTOR_GRIDS:
                ms = time_candidate(precision, M, ag, fg, replicas)
                scores.append((ms, ag, fg))
                if log:
                    log(f"M={M} admm_grid={ag} factor_grid={fg}: {ms:.3f} ms")
        ms, ag, fg = min(scores)
        best[bucket_of(M)] = {"admm_grid": ag, "factor_grid": fg, "batch_ms": ms, "replicas": replicas}
    return best


def load_or_tune(path, precision, log=None):
    """The cached tuning at path if present (and for this precision), else a fresh one (stored at path)."""
    if path and os.path.exists(path):
        d = json.load(open(path))
        if d.get("precision") == precision:
            return {k: {"admm_grid": v["admm_grid"], "factor_grid": v["factor_grid"]} for k, v in d["buckets"].items()}
    best = tune(precision, log=log)
    if path:
        json.dump({"precision": precision, "buckets": best}, open(path, "w"), indent=1)
    return {k: {"admm_grid": v["admm_grid"], "factor_grid": v["factor_grid"]} for k, v in best.items()}
