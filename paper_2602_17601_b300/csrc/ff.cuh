// Float-float sums: a value kept as an unevaluated pair hi + lo of FP32 numbers, updated with
// error-free transformations (Knuth's TwoSum for sums, the fused multiply-add for the rounding
// error of a product), for sums whose result is small beside their terms (the affine defect
// c = x_{k+1} - A x_k - B u of a linearisation, whose terms are positions of order one).  The
// error of such a sum is about n 2^-48 of the sum of |terms| instead of n 2^-24, with FP32
// operations only.  __fadd_rn / __fmul_rn keep the compiler from contracting or reordering
// the error terms.
#pragma once

namespace gmi {

struct FF {
    float hi = 0.f, lo = 0.f;
};

// s + x, x a float
__device__ __forceinline__ void ff_add(FF& s, float x) {
    const float t = __fadd_rn(s.hi, x);
    const float bp = __fadd_rn(t, -s.hi);
    const float e = __fadd_rn(__fadd_rn(s.hi, -__fadd_rn(t, -bp)), __fadd_rn(x, -bp));
    s.hi = t;
    s.lo = __fadd_rn(s.lo, e);
}

// s + a b (the product's rounding error fma(a, b, -ab) is exact)
__device__ __forceinline__ void ff_add_prod(FF& s, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = fmaf(a, b, -p);
    ff_add(s, p);
    s.lo = __fadd_rn(s.lo, pe);
}

// s + t, both pairs
__device__ __forceinline__ void ff_add_ff(FF& s, const FF& t) {
    ff_add(s, t.hi);
    s.lo = __fadd_rn(s.lo, t.lo);
}

// the warp's sum of every lane's pair, in every lane
__device__ __forceinline__ FF ff_warp_sum(FF s) {
    for (int o = 16; o > 0; o >>= 1) {
        FF t;
        t.hi = __shfl_xor_sync(0xffffffffu, s.hi, o);
        t.lo = __shfl_xor_sync(0xffffffffu, s.lo, o);
        ff_add_ff(s, t);
    }
    return s;
}

__device__ __forceinline__ float ff_value(const FF& s) { return __fadd_rn(s.hi, s.lo); }

}  // namespace gmi
