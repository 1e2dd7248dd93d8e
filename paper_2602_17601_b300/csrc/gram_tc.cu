// Tensor-core Gram product  G = sum_r w_r x_r x_r'  over packed stage-major rows (GramRows):
// the H of the condensing (x = rows of Gamma_u, w = Q), rho C~'S^2 C~ of the ADMM set-up, the
// interior-point C~' diag(z/s) C~ and the barrier C~' diag(mu beta'') C~.  A dense contraction
// over 10^5 rows into an n x n result (n = N nu <= 256), so it runs on tcgen05:
//
//   G = Y' Y  with  Y_r = sqrt(w_r) x_r  (or w_r x_r when the weights are given squared),
//
// one operand serving as both A and B.  Y is split into three BF16 pieces (y = y0 + y1 + y2,
// the six products i + j < 3 keep FP32 operand precision, as in the forward MLPs) and
// accumulated in FP32 in tensor memory.  The weights must be >= 0 (a negative one gives NaN).
//
// Each CTA takes K-tiles of 64 rows of one stage (a stage-k row has k nu leading non-zeros),
// tiles blockIdx.x, blockIdx.x + grid, ...; the threads stage a tile into shared memory in the
// K-major core-matrix layout (element (m, k) of the tile: column m of the rows, tile row k),
// double-buffered so that the MMAs of one tile run while the next is staged.  The accumulator
// D0 holds G rows 0..127 (N = all columns), D1 rows 128..255, the latter only for tiles whose
// rows reach column 128.  At the end each CTA writes its partial sum in the [T][T][32 x 32]
// tile layout that gram_reduce_kernel sums over the CTAs.
#include "common.cuh"
#include "kernels.h"
#include "tc_prim.cuh"

namespace gmi {

constexpr int GT_T = 256;            // threads
constexpr int GT_KT = 64;            // rows per K-tile
constexpr int GT_P = 3;              // BF16 pieces

__host__ __device__ constexpr int gt_npad(int n) { return n <= 16 ? 16 : (n + 15) / 16 * 16; }
__host__ __device__ constexpr int gt_mext(int n) { return n > 128 ? 256 : 128; }
__host__ __device__ constexpr size_t gt_piece(int n) { return (size_t)gt_mext(n) * GT_KT * 2; }
__host__ __device__ constexpr size_t gt_smem(int n) { return 2 * GT_P * gt_piece(n); }
static unsigned gt_tmem_cols(int n) {
    if (n > 128) return 512;                           // D0 at column 0, D1 at column 256
    unsigned c = 32;
    while ((int)c < gt_npad(n)) c <<= 1;
    return c;
}

__global__ void __launch_bounds__(GT_T, 1) gram_tc_kernel(GramRows R, int n, float* __restrict__ part,
                                                          unsigned tmem_cols, int* status) {
    extern __shared__ __align__(1024) unsigned char gsm[];
    __shared__ __align__(8) unsigned long long mma_done[2], fin;
    __shared__ unsigned tmem_base;
    __shared__ int d1_used;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int npad = gt_npad(n);
    const size_t piece = gt_piece(n);
    const int tps = (R.rows_per_stage + GT_KT - 1) / GT_KT;       // tiles per stage
    const long ntiles = (long)tps * R.N;
    const int G = gridDim.x;
    const int nt = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / G + 1) : 0;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mma_done[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mma_done[1])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&fin)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        d1_used = 0;
    }
    // rows m >= npad of both buffers stay zero (staging writes m < npad only)
    for (size_t o = (size_t)tid * 16; o < 2 * GT_P * piece; o += (size_t)GT_T * 16)
        *reinterpret_cast<uint4*>(gsm + o) = make_uint4(0u, 0u, 0u, 0u);
    fence_async_smem();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tmem_base;
    const unsigned idesc = tc_idesc(128, npad);
    bool ok = true, acc0 = false, acc1 = false;
    int issued = 0;                                             // tiles whose MMAs were committed
    // item (m, i8) of a tile: column m of tile rows 8 i8 .. 8 i8 + 7, one 16-byte store per
    // piece; the lanes of a warp take consecutive m, so every row read is coalesced.  The
    // rows of tile t + 1 are loaded into registers (and its 64 row weights by threads 0..63)
    // before tile t is converted and stored, so their round trip overlaps the staging and the
    // MMAs of tile t.  The weight factors sqrt(w) (or w) of a tile sit in sw[tile & 1].
    __shared__ float sw[2][GT_KT];
    constexpr int MAXIT = 256 * (GT_KT / 8) / GT_T;
    const int nit = npad * (GT_KT / 8);
    float y[MAXIT][8], yn[MAXIT][8];
    auto tile_of = [&](int t, int& k, int& rb) {
        const long id = blockIdx.x + (long)t * G;
        k = (int)(id / tps) + 1;                               // stage (1-based), rows of length k nu
        rb = (int)(id % tps) * GT_KT;
    };
    auto load = [&](int t, float (&yy)[MAXIT][8]) {
        int k, rb;
        tile_of(t, k, rb);
        const int L = k * R.nu;
        const long base = (long)R.rows_per_stage * R.nu * ((long)k * (k - 1) / 2);
#pragma unroll
        for (int u = 0; u < MAXIT; ++u) {
            const int it = tid + u * GT_T;
            const int m = it % npad, i8 = it / npad;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int r = rb + 8 * i8 + j;
                yy[u][j] = it < nit && r < R.rows_per_stage && m < L ? R.X[base + (long)r * L + m] : 0.f;
            }
        }
    };
    auto weight = [&](int t) {                                 // thread tid < 64: row tid of tile t
        int k, rb;
        tile_of(t, k, rb);
        const int r = rb + tid;
        return R.wts && r < R.rows_per_stage ? R.wts[(long)(k - R.wts_k0) * R.rows_per_stage + r] : 1.f;
    };
    auto factor = [&](float w) { return R.wts_square ? w : sqrtf(w); };
    if (nt > 0) {
        load(0, y);
        if (tid < GT_KT) sw[0][tid] = factor(weight(0));
    }
    for (int t = 0; t < nt; ++t) {
        const int b = t & 1;
        float wnext = 1.f;
        if (t + 1 < nt) {
            if (tid < GT_KT) wnext = weight(t + 1);
            load(t + 1, yn);
        }
        if (t >= 2 && ok) ok = tc_wait(&mma_done[b], ((t - 2) >> 1) & 1, status);   // buffer b free again
        if (!__syncthreads_and(ok)) break;
        int k, rb;
        tile_of(t, k, rb);
        const int L = k * R.nu;
        unsigned char* buf = gsm + (size_t)b * GT_P * piece;
#pragma unroll
        for (int u = 0; u < MAXIT; ++u) {
            const int it = tid + u * GT_T;
            if (it < nit) {
                const int m = it % npad, i8 = it / npad;
                float v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = y[u][j] * sw[b][8 * i8 + j];
                uint4 pc[GT_P];
                pack8<GT_P>(v, pc);
                const int o = tc_off(m, 8 * i8, GT_KT);
#pragma unroll
                for (int p = 0; p < GT_P; ++p) *reinterpret_cast<uint4*>(buf + p * piece + o) = pc[p];
            }
        }
        // sw[b ^ 1] was last read while tile t - 1 was staged, before the barrier above
        if (t + 1 < nt && tid < GT_KT) sw[b ^ 1][tid] = factor(wnext);
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const unsigned a0 = smem_u32(buf);
            const bool use1 = L > 128;
            for (int kk = 0; kk < GT_KT / 16; ++kk)
#pragma unroll
                for (int i = 0; i < GT_P; ++i)
#pragma unroll
                    for (int j = 0; i + j < GT_P; ++j) {
                        const unsigned long long bd = tc_desc(a0 + j * (unsigned)piece + kk * 256, GT_KT * 16);
                        tc_mma(tmem, tc_desc(a0 + i * (unsigned)piece + kk * 256, GT_KT * 16), bd, idesc,
                               acc0 ? 1u : 0u);
                        acc0 = true;
                        if (use1) {
                            tc_mma(tmem + 256, tc_desc(a0 + i * (unsigned)piece + 16 * GT_KT * 16 + kk * 256, GT_KT * 16),
                                   bd, idesc, acc1 ? 1u : 0u);
                            acc1 = true;
                        }
                    }
            tc_commit(&mma_done[b]);
            if (acc1) d1_used = 1;
        }
        ++issued;
#pragma unroll
        for (int u = 0; u < MAXIT; ++u)
#pragma unroll
            for (int j = 0; j < 8; ++j) y[u][j] = yn[u][j];
    }
    // every MMA issued has completed before tensor memory is read and released
    if (tid == 0) tc_commit(&fin);
    bool done = tc_wait(&fin, 0, status);
    tc_fence_after();
    __syncthreads();
    done = __syncthreads_and(done && ok);
    const int T = (n + 31) / 32;
    float* mine = part + (size_t)blockIdx.x * T * T * 1024;
    // warps 0-3: D0 rows 32 w + lane; warps 4-7: D1 rows 128 + 32 (w - 4) + lane
    const int q = warp & 3;
    const int m0 = (warp < 4 ? 0 : 128) + 32 * q;
    if (m0 < n) {
        const int ti = m0 / 32;
        const bool have = done && issued > 0 && (warp < 4 || d1_used);
        const unsigned tD = tmem + (warp < 4 ? 0u : 256u) + ((unsigned)(32 * q) << 16);
        for (int cb = 0; cb < T; ++cb) {
            float v[32];
            if (have) {
                tc_ld32(tD + (unsigned)(32 * cb), v);
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = 0.f;
            }
            float* dst = mine + ((size_t)ti * T + cb) * 1024 + lane * 32;
#pragma unroll
            for (int j = 0; j < 32; j += 4) *reinterpret_cast<float4*>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

bool gram_tc_ok(int n) { return n >= 1 && n <= 256; }

gm_status launch_gram_tc(const GramRows& R, int n, int nsplit, float* part, int* status, cudaStream_t st) {
    const size_t smem = gt_smem(n);
    static size_t set_for = 0;
    if (smem > set_for) {
        GM_CUDA_TRY(cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        set_for = smem;
    }
    gram_tc_kernel<<<nsplit, GT_T, smem, st>>>(R, n, part, gt_tmem_cols(n), status);
    GM_LAUNCH_CHECK();
    return GM_OK;
}

}  // namespace gmi
