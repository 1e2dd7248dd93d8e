"""HBM bandwidth by direction: read-only, write-only and copy streams on this GPU.

    python -m paper_2602_17601_b300.hbm_mix [--gb 4] [--reps 10]

The step's dominant kernel writes three bytes for every one it reads, while the HBM peak
the roofline divides by comes from a copy (one read per write).  This measures what the
memory system gives for each direction alone, with PyTorch's own stream kernels on
buffers far larger than L2 (fill_: write-only; sum: read-only; copy_: one read and one
write per element), timed with CUDA events after a warm-up.  Prints one JSON line.
"""
from __future__ import annotations


def main(argv=None):
    import argparse
    import json

    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--gb", type=float, default=4.0)
    ap.add_argument("--reps", type=int, default=10)
    a = ap.parse_args(argv)
    n = int(a.gb * 1e9) // 4
    x = torch.empty(n, dtype=torch.float32, device="cuda")
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    x.fill_(1.0)
    y.fill_(2.0)
    out = torch.empty(1, dtype=torch.float32, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn, nbytes):
        fn()
        torch.cuda.synchronize()
        ev[0].record()
        for _ in range(a.reps):
            fn()
        ev[1].record()
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / a.reps
        return {"ms": ms, "GB/s": nbytes / (ms * 1e-3) / 1e9}

    rep = {"bytes_per_buffer": 4 * n,
           "write_only": timed(lambda: x.fill_(3.0), 4 * n),
           "read_only": timed(lambda: torch.sum(x, dim=0, out=out), 4 * n),
           "copy": timed(lambda: y.copy_(x), 8 * n),
           "device": torch.cuda.get_device_name()}
    print(json.dumps(rep), flush=True)
    return rep


if __name__ == "__main__":
    main()
