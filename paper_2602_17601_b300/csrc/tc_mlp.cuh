// Tensor-core (tcgen05) form of the fused 2-layer MLP kernel: BF16 operands,
// FP32 accumulation in tensor memory.  Same Op functors as mlp2_kernel.
//
//   GEMM1  D1[128 x W]    = X[128 x Kin] . B1       (K in chunks of 64)
//   hidden                = relu(D1 + b1) (mask bits saved) or D1 * saved mask
//   GEMM2  D2[128 x Nout] = hid . B2                (K = W in chunks of 64)
//   out(row, n, D2 + b2)
//
// SPLIT = 3 keeps FP32-level accuracy with BF16 tensor cores: every operand
// is stored as hi = bf16(x) and lo = bf16(x - hi), and D = Ah Bh + Ah Bl + Al Bh
// (the Al Bl term is below FP32 rounding).  SPLIT = 1 uses hi only.
//
// Operands are staged in shared memory by the threads in the canonical
// no-swizzle K-major layout of core matrices (8 rows x 16 bytes): element
// (r, k) of a tile with K columns sits at (r/8)*16K + (k/8)*128 + (r%8)*16 +
// (k%8)*2 bytes, so a 16-wide K step of one MMA is 256 bytes further on and
// the descriptor strides are LBO = 128 bytes (next core matrix along K) and
// SBO = 16K bytes (next 8-row group).  One thread issues the MMAs and commits
// them to an mbarrier; every wait is bounded and records GM_ERR_TIMEOUT.
#pragma once

#include <cuda_bf16.h>

namespace gmi {

constexpr int TC_M = 128;        // rows per CTA tile (MMA M)
constexpr int TC_KC = 64;        // K per staged chunk
constexpr int TC_T = 256;        // threads per CTA
constexpr int TC_TMEM_COLS = 512;
constexpr int TC_NB = 256;       // largest product width staged (N of GEMM2)

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ int tc_off(int r, int k, int Kdim) {
    return (r >> 3) * (Kdim * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ unsigned long long tc_desc(unsigned addr, unsigned sbo) {
    unsigned long long d = (unsigned long long)((addr >> 4) & 0x3FFF);
    d |= (unsigned long long)(128u >> 4) << 16;        // LBO: next core matrix along K
    d |= (unsigned long long)((sbo >> 4) & 0x3FFF) << 32;
    d |= 1ull << 46;                                   // descriptor version (tcgen05)
    return d;                                          // no swizzle, base offset 0
}

// kind::f16 instruction descriptor: F32 accumulate, BF16 A and B, both K-major.
__host__ __device__ constexpr unsigned tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(unsigned tmem_d, unsigned long long ad, unsigned long long bd, unsigned idesc,
                                       unsigned acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(void* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ bool tc_wait(void* mbar, unsigned parity, int* status) {
    unsigned done = 0;
    for (long long spin = 0; spin < (1ll << 26) && !done; ++spin) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(parity)
            : "memory");
    }
    if (!done && status) dev_fail(status, GM_ERR_TIMEOUT);
    return done != 0;
}

__device__ __forceinline__ void tc_ld32(unsigned taddr, float* v) {
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ unsigned bf2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<unsigned*>(&h);
}

// 8 values -> BF16 hi part (and lo = bf16(v - hi) for the split form)
template <int SPLIT>
__device__ __forceinline__ void pack8(const float* v, uint4& hi, uint4& lo) {
    hi = make_uint4(bf2(v[0], v[1]), bf2(v[2], v[3]), bf2(v[4], v[5]), bf2(v[6], v[7]));
    if constexpr (SPLIT == 3) {
        float r[8];
        const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&hi);
#pragma unroll
        for (int j = 0; j < 8; ++j) r[j] = v[j] - __bfloat162float(h[j]);
        lo = make_uint4(bf2(r[0], r[1]), bf2(r[2], r[3]), bf2(r[4], r[5]), bf2(r[6], r[7]));
    }
}

// Operand pointers of one launch: K-major BF16 copies [Npad][Kpad] of the two products
// (hi parts, and lo parts for the split form).
struct TcW {
    const __nv_bfloat16* B1;     // [W][K1p]
    const __nv_bfloat16* B2;     // [N2p][W]  (unused in single-product mode)
    const __nv_bfloat16* B1lo;
    const __nv_bfloat16* B2lo;
    int K1p, N2p;
    int* status;
};

template <class Op>
__device__ __forceinline__ void tc_load8(const Op& op, const RowCtx& rc, int k0, float* v) {
    if constexpr (Op::kHasIn8) {
        op.in8(rc, k0, v);
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = (k0 + j < op.kin) ? op.in(rc, k0 + j) : 0.f;
    }
}

template <class Op>
__device__ __forceinline__ void tc_out32(const Op& op, const RowCtx& rc, int c0, const float* v, int nout,
                                         const float* bias) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int n = c0 + 4 * q;
        if constexpr (Op::kHasOut4) {
            if (n + 3 < nout) {
                float4 f = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                if (bias) {
                    f.x += bias[n]; f.y += bias[n + 1]; f.z += bias[n + 2]; f.w += bias[n + 3];
                }
                op.out4(rc, n, f);
                continue;
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (n + j < nout) op.out(rc, n + j, v[4 * q + j] + (bias ? bias[n + j] : 0.f));
    }
}

// Stage rows [0, nrows) x K-chunk [k0, k0 + kc) of a K-major BF16 matrix (row length ld) into smem.
template <int SPLIT>
__device__ __forceinline__ void tc_stage_b(unsigned char* dst_hi, unsigned char* dst_lo, const __nv_bfloat16* hi,
                                           const __nv_bfloat16* lo, int nrows, int ld, int k0, int kc, int tid) {
    const int nv = nrows * (kc / 8);
    for (int v = tid; v < nv; v += TC_T) {
        const int n = v / (kc / 8), kv = v % (kc / 8);
        const long g = (long)n * ld + k0 + kv * 8;
        *reinterpret_cast<uint4*>(dst_hi + tc_off(n, kv * 8, TC_KC)) = *reinterpret_cast<const uint4*>(hi + g);
        if constexpr (SPLIT == 3)
            *reinterpret_cast<uint4*>(dst_lo + tc_off(n, kv * 8, TC_KC)) = *reinterpret_cast<const uint4*>(lo + g);
    }
}

// MMAs of one staged chunk: D (+)= A.B^T, split-product terms for SPLIT = 3.
template <int SPLIT>
__device__ __forceinline__ void tc_issue(unsigned tD, unsigned a_hi, unsigned a_lo, unsigned a_sbo, unsigned b_hi,
                                         unsigned b_lo, int kc, int N, bool first) {
    const unsigned idesc = tc_idesc(TC_M, N);
    for (int kk = 0; kk < kc / 16; ++kk) {
        const unsigned long long ah = tc_desc(a_hi + kk * 256, a_sbo);
        const unsigned long long bh = tc_desc(b_hi + kk * 256, TC_KC * 16);
        tc_mma(tD, ah, bh, idesc, (first && kk == 0) ? 0u : 1u);
        if constexpr (SPLIT == 3) {
            const unsigned long long al = tc_desc(a_lo + kk * 256, a_sbo);
            const unsigned long long bl = tc_desc(b_lo + kk * 256, TC_KC * 16);
            tc_mma(tD, ah, bl, idesc, 1u);
            tc_mma(tD, al, bh, idesc, 1u);
        }
    }
}

template <int W, int SPLIT>
constexpr size_t tc_smem_bytes() {
    // A chunk (hi, lo) + B chunk (hi, lo; up to TC_NB rows) + hidden (hi, lo)
    return (size_t)2 * TC_M * TC_KC * 2 + (size_t)2 * TC_NB * TC_KC * 2 + (size_t)2 * TC_M * W * 2;
}

template <int W, class Op, int SPLIT>
__global__ void __launch_bounds__(TC_T) tc_mlp_kernel(Op op, TcW w) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    unsigned char* sAh = tsm;
    unsigned char* sAl = sAh + TC_M * TC_KC * 2;
    unsigned char* sBh = sAl + TC_M * TC_KC * 2;
    unsigned char* sBl = sBh + TC_NB * TC_KC * 2;
    unsigned char* sHh = sBl + TC_NB * TC_KC * 2;      // hidden, K-major with K = W
    unsigned char* sHl = sHh + TC_M * W * 2;
    __shared__ RowCtx rc[TC_M];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ unsigned tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long row0 = (long)blockIdx.x * TC_M;
    const long rows = op.rows;
    constexpr bool kSingle = (Op::kMode == 2);
    for (int m = tid; m < TC_M; m += TC_T) rc[m] = op.prep(row0 + m < rows ? row0 + m : -1);
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "n"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tmem_base;
    const unsigned tD1 = tmem, tD2 = tmem + W;
    bool ok = true;
    unsigned phase = 0;

    // ---------------- GEMM1 over K chunks
    const int nch = (w.K1p + TC_KC - 1) / TC_KC;
    for (int c = 0; c < nch; ++c) {
        const int k0 = c * TC_KC;
        const int kc = min(TC_KC, w.K1p - k0);        // multiple of 16
        const int nva = TC_M * (kc / 8);
        for (int v = tid; v < nva; v += TC_T) {
            const int m = v / (kc / 8), kv = v % (kc / 8);
            float x[8];
            if (row0 + m < rows) {
                tc_load8(op, rc[m], k0 + kv * 8, x);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) x[j] = 0.f;
            }
            uint4 hi, lo;
            pack8<SPLIT>(x, hi, lo);
            *reinterpret_cast<uint4*>(sAh + tc_off(m, kv * 8, TC_KC)) = hi;
            if constexpr (SPLIT == 3) *reinterpret_cast<uint4*>(sAl + tc_off(m, kv * 8, TC_KC)) = lo;
        }
        tc_stage_b<SPLIT>(sBh, sBl, w.B1, w.B1lo, W, w.K1p, k0, kc, tid);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            tc_issue<SPLIT>(tD1, smem_u32(sAh), smem_u32(sAl), TC_KC * 16, smem_u32(sBh), smem_u32(sBl), kc, W, c == 0);
            tc_commit(&mbar);
        }
        ok = tc_wait(&mbar, phase & 1, w.status) && ok;   // the chunk buffers are free again
        ++phase;
    }
    ok = __syncthreads_and(ok) != 0;           // warp-collective TMEM loads below need a uniform decision
    tc_fence_after();

    // ---------------- hidden layer / single-product epilogue; 32-column blocks alternate
    // between the two warp groups; TMEM lane = tile row
    const int lrow = (warp & 3) * 32 + lane;
    const int chalf = warp >> 2;
    const bool valid = ok && (row0 + lrow < rows);
    const unsigned lane_off = (unsigned)((warp & 3) * 32) << 16;
    if (kSingle) {
        for (int c0 = chalf * 32; c0 < W; c0 += 64) {
            float v[32];
            if (ok) tc_ld32(tD1 + lane_off + (unsigned)c0, v);
            if (valid) tc_out32(op, rc[lrow], c0, v, op.nout, nullptr);
        }
    } else {
        for (int c0 = chalf * 32; c0 < W; c0 += 64) {
            float v[32];
            if (ok) tc_ld32(tD1 + lane_off + (unsigned)c0, v);
            if constexpr (Op::kMode == 0) {
                uint32_t bits = 0;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    float h = v[j] + op.b1[c0 + j];
                    h = h > 0.f ? h : 0.f;
                    bits |= (h > 0.f ? 1u : 0u) << j;
                    v[j] = h;
                }
                if (valid) op.store_mask(rc[lrow], c0 >> 5, bits);
            } else {
                const uint32_t mw = valid ? op.mask_word(rc[lrow], c0 >> 5) : 0u;
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = ((mw >> j) & 1u) ? v[j] : 0.f;
                if constexpr (Op::kStoreHid) {
                    if (valid)
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            op.store_hid4(rc[lrow], c0 + 4 * q,
                                          make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint4 hi, lo;
                pack8<SPLIT>(v + q * 8, hi, lo);
                *reinterpret_cast<uint4*>(sHh + tc_off(lrow, c0 + q * 8, W)) = hi;
                if constexpr (SPLIT == 3) *reinterpret_cast<uint4*>(sHl + tc_off(lrow, c0 + q * 8, W)) = lo;
            }
        }
        // ---------------- GEMM2 over K = W in chunks of 64 (B2 staged chunk by chunk)
        for (int k0 = 0; k0 < W; k0 += TC_KC) {
            const int kc = min(TC_KC, W - k0);
            tc_stage_b<SPLIT>(sBh, sBl, w.B2, w.B2lo, w.N2p, W, k0, kc, tid);
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (tid == 0) {
                // hidden tile: K-major with K = W; the chunk starts k0/8 core matrices along K
                tc_issue<SPLIT>(tD2, smem_u32(sHh) + (k0 / 8) * 128, smem_u32(sHl) + (k0 / 8) * 128, W * 16,
                                smem_u32(sBh), smem_u32(sBl), kc, w.N2p, k0 == 0);
                tc_commit(&mbar);
            }
            ok = tc_wait(&mbar, phase & 1, w.status) && ok;
            ++phase;
        }
        ok = __syncthreads_and(ok) != 0;
        tc_fence_after();
        const bool valid2 = ok && (row0 + lrow < rows);
        for (int c0 = chalf * 32; c0 < w.N2p; c0 += 64) {
            float v[32];
            if (ok) tc_ld32(tD2 + lane_off + (unsigned)c0, v);
            if (valid2) tc_out32(op, rc[lrow], c0, v, op.nout, op.b2);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TC_TMEM_COLS));
}

}  // namespace gmi
