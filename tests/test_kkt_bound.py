"""The rounding bound behind the FP32 pre-test of the KKT certificate's constraint rows (CPU).

The device tests a row without multiplier in FP32 before any FP64 work.  Lane l of a warp sums
the products C~_rc U_c of its columns c = l, l + 32, ... (at most 8 of them, n <= 256) in
order, then the 32 lane sums meet in five levels of a butterfly (xor 16, 8, 4, 2, 1); s, the sum
of the products' magnitudes, is formed the same way.  The row is cleared when
d32 + 2^-18 s32 + 1e-30 (rounded upwards) < d~_r, which is rigorous only if the FP32 dot lies
within 2^-18 s32 of the exact dot.  This file replays that summation order in float32 (each
product rounded, or fused into the running sum) and checks the bound against the exact dot
(FP64 products of the float32 operands are exact, their sum is accurate to far below the bound)
on random rows, rows built to cancel, and rows of mixed magnitudes.
"""
import numpy as np
import pytest

BOUND = 2.0 ** -18


def lane_sums(prod, fused):
    """Per-lane sequential float32 sums over columns l, l + 32, ... of one row."""
    L = prod.shape[0]
    d = np.zeros(32, np.float32)
    a = np.zeros(32, np.float32)
    for m in range((L + 31) // 32):
        for lane in range(32):
            c = lane + 32 * m
            if c >= L:
                continue
            if fused:
                # fma(x, u, d): the exact product added once, then rounded
                d[lane] = np.float32(np.float64(d[lane]) + prod[c])
            else:
                d[lane] = np.float32(d[lane] + np.float32(prod[c]))
            a[lane] = np.float32(a[lane] + np.abs(np.float32(prod[c])))
    return d, a


def butterfly(v):
    v = v.copy()
    for o in (16, 8, 4, 2, 1):
        v = (v + v[np.arange(32) ^ o]).astype(np.float32)
    return v[0]


def fp32_row(x, u, fused):
    prod = x.astype(np.float64) * u.astype(np.float64)   # exact products of float32 operands
    d, a = lane_sums(prod, fused)
    return butterfly(d), butterfly(a), prod.sum()


def cases(seed):
    rng = np.random.default_rng(seed)
    for L in (8, 31, 32, 33, 96, 160, 256):
        yield rng.standard_normal(L).astype(np.float32), rng.standard_normal(L).astype(np.float32)
        # magnitudes spread over many binades
        x = (rng.standard_normal(L) * 10.0 ** rng.uniform(-6, 6, L)).astype(np.float32)
        yield x, rng.standard_normal(L).astype(np.float32)
        # heavy cancellation: pairs of nearly opposite products
        h = rng.standard_normal(L // 2).astype(np.float32)
        x = np.concatenate([h, -h * np.float32(1 + 1e-6)]).astype(np.float32)
        if x.size < L:
            x = np.append(x, np.float32(1e-3))
        yield x, np.ones(L, np.float32) * np.float32(1.37)


@pytest.mark.parametrize("fused", [False, True], ids=["rounded_products", "fused"])
def test_fp32_row_dot_within_the_bound(fused):
    worst = 0.0
    for seed in range(6):
        for x, u in cases(seed):
            d32, a32, exact = fp32_row(x, u, fused)
            err = abs(float(d32) - exact)
            assert err <= BOUND * float(a32) + 1e-30, (x.size, err, float(a32))
            if a32 > 0:
                worst = max(worst, err / float(a32))
    # the bound is not vacuous: the observed error stays well inside it, but is not zero
    assert 0.0 < worst < BOUND


def test_bound_covers_the_worst_case_order_length():
    # the rounding of each product (when not fused), 8 sequential additions per lane and 5
    # butterfly levels: at most 14 roundings on any product's path, each within 2^-24 of a
    # partial sum bounded by s; 14 * 2^-24 * (1 + 2^-24)^14 is below 2^-18
    u = 2.0 ** -24
    assert 14 * u * (1 + u) ** 14 < BOUND
