"""Launch-shape autotuner for batched instances.

Three launch shapes of an instance's step depend on its size and on the other
instances sharing the GPU:

* the reverse-pass launch shape: how many horizon stages one launch of the
  reverse MLP kernels covers (the device memory budget chunk_mb of the cotangent
  buffers sets it; more stages per launch mean fewer, fuller launches);
* the CTAs of the cooperative ADMM grid and of the FP64 factorisation grid,
  which share the GPU with the other lanes' kernels of a batch.

For every node-count bucket the tuner builds a small batch of representative
instances (the cfg4 GNN, N = 20, nu = 8, box + 5 spheres), times a
graph-replayed batch step for each candidate (chunk_mb, ADMM grid, factor grid),
and keeps the fastest.  The result is a JSON cache keyed by bucket:

    {"M<=250": {"admm_grid": 16, "factor_grid": 16, "chunk_mb": 256}, ...}

Timing is on the device (CUDA events around replays, after a capture and a
warm-up replay).
"""
from __future__ import annotations

import json
import os

BUCKETS = (250, 500, 750, 1000)
ADMM_GRIDS = (16, 32, 64)
FACTOR_GRIDS = (16, 32)
CHUNK_MBS = (64, 256, 1024)


def bucket_of(M):
    for b in BUCKETS:
        if M <= b:
            return f"M<={b}"
    return f"M<={BUCKETS[-1]}"


def time_candidate(precision, M, admm_grid, factor_grid, chunk_mb=256, replicas=8, steps=3, seed=77):
    """Device ms of one graph-replayed step of a batch of `replicas` instances of M nodes."""
    import torch

    from synth import paper_chain
    from .batch import Batch
    from .rti import RTIProblem
    probs = []
    for r in range(replicas):
        wl = paper_chain(seed=seed + r, M=M, N=20, nu=8, w_seed=0)
        probs.append(RTIProblem.from_workload(wl, precision=precision, admm_grid=admm_grid,
                                              factor_grid=factor_grid, chunk_mb=chunk_mb))
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
        for cm in CHUNK_MBS:
            for ag in ADMM_GRIDS:
                for fg in FACTOR_GRIDS:
                    ms = time_candidate(precision, M, ag, fg, cm, replicas)
                    scores.append((ms, ag, fg, cm))
                    if log:
                        log(f"M={M} chunk_mb={cm} admm_grid={ag} factor_grid={fg}: {ms:.3f} ms")
        ms, ag, fg, cm = min(scores)
        best[bucket_of(M)] = {"admm_grid": ag, "factor_grid": fg, "chunk_mb": cm, "batch_ms": ms,
                              "replicas": replicas}
    return best


SHAPE_KEYS = ("admm_grid", "factor_grid", "chunk_mb")


def load_or_tune(path, precision, log=None):
    """The cached tuning at path if present (and for this precision), else a fresh one (stored at path)."""
    if path and os.path.exists(path):
        d = json.load(open(path))
        if d.get("precision") == precision:
            return {k: {s: v[s] for s in SHAPE_KEYS if s in v} for k, v in d["buckets"].items()}
    best = tune(precision, log=log)
    if path:
        json.dump({"precision": precision, "buckets": best}, open(path, "w"), indent=1)
    return {k: {s: v[s] for s in SHAPE_KEYS} for k, v in best.items()}
