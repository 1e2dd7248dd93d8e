// tcgen05 primitives shared by the tensor-core kernels: shared-memory descriptors of the
// canonical no-swizzle K-major core-matrix layout (element (r, k) of a tile with K columns at
// (r/8)*16K + (k/8)*128 + (r%8)*16 + (k%8)*2 bytes: LBO = 128 bytes to the next core matrix
// along K, SBO = 16K bytes to the next 8-row group), the kind::f16 instruction descriptor,
// MMA issue and commit, bounded mbarrier waits, tensor-memory loads, fences, programmatic
// dependent launch, and the split of FP32 values into BF16 pieces.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace gmi {

constexpr int TC_M = 128;        // rows per CTA tile (MMA M)

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
// Programmatic dependent launch: let the next kernel of the stream start its prologue now,
// and wait until the previous kernel has completed (its writes visible) before reading any
// data it produced.  Both are no-ops for a launch without the programmatic attribute.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ unsigned bf2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<unsigned*>(&h);
}

// 8 values -> P BF16 pieces: piece p = bf16(v - pieces 0..p-1).
template <int P>
__device__ __forceinline__ void pack8(const float* v, uint4* out) {
    float r[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) r[j] = v[j];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        out[p] = make_uint4(bf2(r[0], r[1]), bf2(r[2], r[3]), bf2(r[4], r[5]), bf2(r[6], r[7]));
        if (p + 1 < P) {
            const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&out[p]);
#pragma unroll
            for (int j = 0; j < 8; ++j) r[j] -= __bfloat162float(h[j]);
        }
    }
}

// Thread v of a staging loop handles one 16-byte vector (8 K-elements of one row).
// Rows vary fastest within each 8-row core matrix, so the 8 lanes of a quarter warp
// write one contiguous 128-byte core matrix (no shared-memory bank conflicts).
__device__ __forceinline__ void tc_vec_rc(int v, int kv8, int& r, int& kv) {
    const int rest = v >> 3;
    kv = rest % kv8;
    r = (rest / kv8) * 8 + (v & 7);
}

// MMAs of one staged chunk: D (+)= sum over piece pairs (i, j) with i + j < P of A_i . B_j^T
// (1, 3 or 6 products; the dropped pairs are below the last kept piece's rounding).
template <int P>
__device__ __forceinline__ void tc_issue(unsigned tD, unsigned a0, unsigned a_piece, unsigned a_sbo, unsigned b0,
                                         unsigned b_piece, unsigned b_sbo, int kc, int N, bool first) {
    const unsigned idesc = tc_idesc(TC_M, N);
    bool acc = !first;
    for (int kk = 0; kk < kc / 16; ++kk) {
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const unsigned long long ad = tc_desc(a0 + i * a_piece + kk * 256, a_sbo);
#pragma unroll
            for (int j = 0; i + j < P; ++j) {
                const unsigned long long bd = tc_desc(b0 + j * b_piece + kk * 256, b_sbo);
                tc_mma(tD, ad, bd, idesc, acc ? 1u : 0u);
                acc = true;
            }
        }
    }
}

}  // namespace gmi
