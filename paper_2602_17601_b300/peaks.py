"""Measured FP32 / FP64 FMA peaks and the L2 size of the current device (gm_measure_peaks), and
the HBM rates of read-only, write-only and copy streams over 4 GB (gm_measure_hbm).

These are the roofline denominators of the FP32 kernels (condensing, ADMM) and the FP64
kernels (factorisation, KKT check), beside the separately measured HBM copy and BF16 GEMM peaks; the
one-way stream rates show whether a kernel's read/write mix bounds it below the copy peak.

  python -m paper_2602_17601_b300.peaks [--out FILE]
"""
from __future__ import annotations


def main(argv=None):
    import argparse
    import json

    import torch

    from . import gm_measure_hbm, gm_measure_peaks
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--repeats", type=int, default=5)
    a = ap.parse_args(argv)
    torch.cuda.init()
    runs = [gm_measure_peaks() for _ in range(a.repeats)]
    rep = {"fp32_fma_tflops": max(r["fp32_tflops"] for r in runs),
           "fp64_fma_tflops": max(r["fp64_tflops"] for r in runs),
           "l2_bytes": runs[0]["l2_bytes"], "repeats": a.repeats,
           "how": "independent FMA chains (8 per thread) in 8 CTAs x 256 threads per SM, CUDA events, best of "
                  f"{a.repeats}; L2 from cudaDevAttrL2CacheSize",
           "device": torch.cuda.get_device_name(), "sms": torch.cuda.get_device_properties(0).multi_processor_count}
    buf = torch.empty(4 << 30, dtype=torch.uint8, device="cuda")
    rep.update({f"hbm_{k}": v for k, v in gm_measure_hbm(buf, a.repeats).items()})
    rep["hbm_how"] = ("grid-stride float4 streams (4 CTAs x 512 threads per SM) over two 2 GB halves, streaming "
                      f"cache hints, CUDA events, best of {a.repeats}; GB/s counts bytes read plus written")
    del buf
    print(json.dumps(rep), flush=True)
    if a.out:
        json.dump(rep, open(a.out, "w"), indent=1)
    return rep


if __name__ == "__main__":
    main()
