// Learned ADMM warm start: a 3-layer MLP (in -> H -> H -> out, ReLU between) mapping pooled
// GNN latents and the reference to a primal input sequence and box duals, with its training
// kernels (MSE loss, backward, Adam).  Inputs and targets are standardised with stored
// means and deviations.  Every product (the forward layers, the weight gradients and the
// propagated gradients) runs on tcgen05 tensor cores with BF16 operands and FP32 accumulation
// in tensor memory; each FP32 operand is split into two BF16 pieces (three products, about 16
// bits), which the weight gradients need to match an FP32 evaluation.
#include <cstring>

#include "ctx.h"
#include "kernels.h"
#include "tc_prim.cuh"

struct gm_ws {
    int n_in = 0, n_hid = 0, n_out = 0, max_batch = 0;
    long n_par = 0;
    long o_W[3], o_b[3];           // parameter offsets
    float *par = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
    float* norm = nullptr;         // [in mean | in std | out mean | out std]
    float *x = nullptr, *a0 = nullptr, *a1 = nullptr, *y = nullptr;   // [B][in], [B][H], [B][H], [B][out]
    float *d0 = nullptr, *d1 = nullptr, *dy = nullptr;                // gradients of a0, a1, y
    float* loss = nullptr;
    int* status = nullptr;         // device word: GM_ERR_TIMEOUT bit when a bounded wait gave up
    int step = 0;                  // Adam step count
};

namespace gmi {
namespace {

constexpr int WG_M = 128, WG_N = 128, WG_KC = 64, WG_T = 256, WG_P = 2;
constexpr size_t WG_SMEM = (size_t)2 * WG_P * WG_M * WG_KC * 2;    // A and B chunks, P pieces each

// C[i][j] (+)= sum_k A(i, k) B(k, j) (+ bias[j]) (ReLU): A(i, k) = A[i sai + k sak],
// B(k, j) = B[k sbk + j sbj], C row-major with ldc.  One CTA per 128 x 128 tile of C: the
// threads stage K chunks of 64 of both operands (any strides, zero past the edges) as P BF16
// pieces in the K-major core-matrix layout, one thread issues the P(P+1)/2 products per 16-wide
// K step into tensor memory, and the epilogue reads its row (TMEM lane) back.
__global__ void __launch_bounds__(WG_T) ws_tc_gemm_kernel(int M, int N, int K, const float* __restrict__ A, long sai,
                                                          long sak, const float* __restrict__ B, long sbk, long sbj,
                                                          float* __restrict__ C, long ldc,
                                                          const float* __restrict__ bias, int relu, int accumulate,
                                                          int* status) {
    extern __shared__ __align__(1024) unsigned char wsg[];
    constexpr int PIECE = WG_M * WG_KC * 2;
    unsigned char* sA = wsg;                      // WG_P pieces of the A chunk [128 rows][64 K]
    unsigned char* sB = wsg + WG_P * PIECE;       // WG_P pieces of the B chunk [128 columns of C][64 K]
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ unsigned tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long i0 = (long)blockIdx.y * WG_M, j0 = (long)blockIdx.x * WG_N;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "n"(WG_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tD = tmem_base;
    bool ok = true;
    const int nch = (K + WG_KC - 1) / WG_KC;
    for (int c = 0; c < nch; ++c) {
        const int k0 = c * WG_KC;
        for (int v = tid; v < WG_M * (WG_KC / 8); v += WG_T) {
            int r, kv;
            tc_vec_rc(v, WG_KC / 8, r, kv);
            float xa[8], xb[8];
            const long i = i0 + r, j = j0 + r;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int k = k0 + kv * 8 + e;
                xa[e] = (i < M && k < K) ? A[i * sai + (long)k * sak] : 0.f;
                xb[e] = (j < N && k < K) ? B[(long)k * sbk + j * sbj] : 0.f;
            }
            uint4 pa[WG_P], pb[WG_P];
            pack8<WG_P>(xa, pa);
            pack8<WG_P>(xb, pb);
            const int o = tc_off(r, kv * 8, WG_KC);
#pragma unroll
            for (int p = 0; p < WG_P; ++p) {
                *reinterpret_cast<uint4*>(sA + p * PIECE + o) = pa[p];
                *reinterpret_cast<uint4*>(sB + p * PIECE + o) = pb[p];
            }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            if (ok) tc_issue<WG_P>(tD, smem_u32(sA), PIECE, WG_KC * 16, smem_u32(sB), PIECE, WG_KC * 16, WG_KC, WG_N, c == 0);
            tc_commit(&mbar);                     // arrives even when nothing was issued
        }
        ok = tc_wait(&mbar, c & 1, status) && ok; // the chunk's products are done: its buffers are free
    }
    ok = __syncthreads_and(ok) != 0;
    tc_fence_after();
    // epilogue: warp w reads the lanes of quadrant w % 4 (one row each), 32-column blocks
    const int q = warp & 3;
    const long i = i0 + q * 32 + lane;
    for (int cb = (warp >> 2) * 32; cb < WG_N; cb += 64) {
        float v[32];
        if (ok) tc_ld32(tD + ((unsigned)(q * 32) << 16) + (unsigned)cb, v);
        if (ok && i < M)
#pragma unroll 4
            for (int jj = 0; jj < 32; ++jj) {
                const long j = j0 + cb + jj;
                if (j >= N) break;
                float val = v[jj];
                if (accumulate) val += C[i * ldc + j];
                if (bias) val += bias[j];
                if (relu) val = fmaxf(val, 0.f);
                C[i * ldc + j] = val;
            }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "n"(WG_N));
}

// x' = (x - mean) / std, row by row
__global__ void ws_normalize_kernel(int B, int n, const float* __restrict__ x, const float* __restrict__ mean,
                                    const float* __restrict__ sd, float* __restrict__ out) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)B * n) return;
    const int j = (int)(t % n);
    out[t] = (x[t] - mean[j]) / sd[j];
}

__global__ void ws_denormalize_kernel(int B, int n, const float* __restrict__ y, const float* __restrict__ mean,
                                      const float* __restrict__ sd, float* __restrict__ out) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)B * n) return;
    const int j = (int)(t % n);
    out[t] = y[t] * sd[j] + mean[j];
}

// MSE on standardised targets: L = sum (y - t')^2 / (B n), dy = 2 (y - t') / (B n)
__global__ void ws_mse_kernel(int B, int n, const float* __restrict__ y, const float* __restrict__ target,
                              const float* __restrict__ mean, const float* __restrict__ sd, float* __restrict__ dy,
                              float* __restrict__ loss) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (t < (long)B * n) {
        const int j = (int)(t % n);
        const float d = y[t] - (target[t] - mean[j]) / sd[j];
        dy[t] = 2.f * d / ((float)B * n);
        l = d * d / ((float)B * n);
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, l);
}

// d *= (a > 0): the ReLU derivative (0 at 0) of the layer whose output is a
__global__ void ws_relu_bwd_kernel(long n, const float* __restrict__ a, float* __restrict__ d) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n && !(a[t] > 0.f)) d[t] = 0.f;
}

// db[j] = sum_i d[i][j]
__global__ void ws_colsum_kernel(int B, int n, const float* __restrict__ d, float* __restrict__ db) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float s = 0.f;
    for (int i = 0; i < B; ++i) s += d[(long)i * n + j];
    db[j] = s;
}

// Adam (Kingma & Ba) with bias correction: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
__global__ void ws_adam_kernel(long n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                               float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float gt = g[t];
    const float mt = b1 * m[t] + (1.f - b1) * gt;
    const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
    m[t] = mt;
    v[t] = vt;
    p[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

// Mean and max over nodes of the final node latents h [M][W] -> feat[0..W) mean, [W..2W) max,
// then the reference positions of stage 1: feat[2W + 3i + a] = x_ref[1][i][a].
__global__ void ws_features_kernel(int M, int W, const float* __restrict__ h, const float* __restrict__ x_ref,
                                   float* __restrict__ feat) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < W) {
        float s = 0.f, mx = -INFINITY;
        for (int i = 0; i < M; ++i) {
            const float v = h[(long)i * W + t];
            s += v;
            mx = fmaxf(mx, v);
        }
        feat[t] = s / (float)M;
        feat[W + t] = mx;
    }
    if (t < 3 * M) feat[2 * W + t] = x_ref[(long)M * 6 + (t / 3) * 6 + t % 3];
}

gm_status gemm(cudaStream_t st, int M, int N, int K, const float* A, long sai, long sak, const float* B, long sbk,
               long sbj, float* C, long ldc, const float* bias, bool relu, bool accumulate, int* status) {
    static bool attr_set = false;
    if (!attr_set) {
        GM_CUDA_TRY(cudaFuncSetAttribute(ws_tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WG_SMEM));
        attr_set = true;
    }
    dim3 grid(cdiv(N, WG_N), cdiv(M, WG_M));
    ws_tc_gemm_kernel<<<grid, WG_T, WG_SMEM, st>>>(M, N, K, A, sai, sak, B, sbk, sbj, C, ldc, bias, relu ? 1 : 0,
                                                   accumulate ? 1 : 0, status);
    GM_LAUNCH_CHECK();
    return GM_OK;
}

// forward on standardised inputs already in w->x: a0, a1, y (standardised outputs)
gm_status ws_fwd(gm_ws* w, int B, cudaStream_t st) {
    const int I = w->n_in, H = w->n_hid, O = w->n_out;
    GM_TRY(gemm(st, B, H, I, w->x, I, 1, w->par + w->o_W[0], H, 1, w->a0, H, w->par + w->o_b[0], true, false, w->status));
    GM_TRY(gemm(st, B, H, H, w->a0, H, 1, w->par + w->o_W[1], H, 1, w->a1, H, w->par + w->o_b[1], true, false, w->status));
    GM_TRY(gemm(st, B, O, H, w->a1, H, 1, w->par + w->o_W[2], O, 1, w->y, O, w->par + w->o_b[2], false, false, w->status));
    return GM_OK;
}

}  // namespace

gm_status ws_features(gm_ctx* c, const float* h, const float* x_ref, float* feat, cudaStream_t st) {
    const int n = std::max(c->W, 3 * c->M);
    ws_features_kernel<<<cdiv(n, 128), 128, 0, st>>>(c->M, c->W, h, x_ref, feat);
    GM_LAUNCH_CHECK();
    return GM_OK;
}

}  // namespace gmi

using namespace gmi;

static long ws_layout(gm_ws* w) {
    const int I = w->n_in, H = w->n_hid, O = w->n_out;
    long o = 0;
    const int din[3] = {I, H, H}, dout[3] = {H, H, O};
    for (int l = 0; l < 3; ++l) {
        w->o_W[l] = o;
        o += (long)din[l] * dout[l];
        w->o_b[l] = o;
        o += dout[l];
    }
    return o;
}

extern "C" {

size_t gm_ws_workspace_size(int n_in, int n_hidden, int n_out, int max_batch) {
    if (n_in <= 0 || n_hidden <= 0 || n_out <= 0 || max_batch <= 0) return 0;
    gm_ws w;
    w.n_in = n_in; w.n_hid = n_hidden; w.n_out = n_out;
    const long P = ws_layout(&w);
    const long B = max_batch;
    const long floats = 4 * P + 2 * (n_in + n_out) + B * (n_in + 4L * n_hidden + 2L * n_out) + 2;
    return (size_t)floats * sizeof(float) + 64 * 256;
}

gm_status gm_ws_create(int n_in, int n_hidden, int n_out, int max_batch, void* workspace, size_t bytes,
                       gm_ws** out) {
    clear_error();
    GM_CHECK_ARG(out && workspace, "NULL argument");
    GM_CHECK_ARG(n_in > 0 && n_hidden > 0 && n_out > 0 && max_batch > 0, "sizes must be positive");
    GM_CHECK_ARG(bytes >= gm_ws_workspace_size(n_in, n_hidden, n_out, max_batch), "workspace too small");
    GM_CHECK_ARG((reinterpret_cast<uintptr_t>(workspace) & 255) == 0, "workspace must be 256-byte aligned");
    gm_ws* w = new gm_ws;
    w->n_in = n_in; w->n_hid = n_hidden; w->n_out = n_out; w->max_batch = max_batch;
    w->n_par = ws_layout(w);
    Carver cv;
    cv.base = static_cast<char*>(workspace);
    const long B = max_batch;
    w->par = cv.take<float>(w->n_par);
    w->grad = cv.take<float>(w->n_par);
    w->m1 = cv.take<float>(w->n_par);
    w->m2 = cv.take<float>(w->n_par);
    w->norm = cv.take<float>(2 * (n_in + n_out));
    w->x = cv.take<float>(B * n_in);
    w->a0 = cv.take<float>(B * n_hidden);
    w->a1 = cv.take<float>(B * n_hidden);
    w->d0 = cv.take<float>(B * n_hidden);
    w->d1 = cv.take<float>(B * n_hidden);
    w->y = cv.take<float>(B * n_out);
    w->dy = cv.take<float>(B * n_out);
    w->loss = cv.take<float>(1);
    w->status = cv.take<int>(1);
    if (cv.off > bytes) {
        delete w;
        set_error("workspace too small");
        return GM_ERR_WORKSPACE;
    }
    *out = w;
    return GM_OK;
}

void gm_ws_destroy(gm_ws* w) { delete w; }

gm_status gm_ws_set_params(gm_ws* w, const float* params, const float* norm, void* stream) {
    clear_error();
    GM_CHECK_ARG(w && params && norm, "NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    GM_CUDA_TRY(cudaMemcpyAsync(w->par, params, sizeof(float) * w->n_par, cudaMemcpyDefault, st));
    GM_CUDA_TRY(cudaMemcpyAsync(w->norm, norm, sizeof(float) * 2 * (w->n_in + w->n_out), cudaMemcpyDefault, st));
    GM_CUDA_TRY(cudaMemsetAsync(w->m1, 0, sizeof(float) * w->n_par, st));
    GM_CUDA_TRY(cudaMemsetAsync(w->m2, 0, sizeof(float) * w->n_par, st));
    GM_CUDA_TRY(cudaMemsetAsync(w->status, 0, sizeof(int), st));
    w->step = 0;
    return GM_OK;
}

gm_status gm_ws_get_params(const gm_ws* w, float* params, float* norm, void* stream) {
    clear_error();
    GM_CHECK_ARG(w && params, "NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    GM_CUDA_TRY(cudaMemcpyAsync(params, w->par, sizeof(float) * w->n_par, cudaMemcpyDefault, st));
    if (norm)
        GM_CUDA_TRY(cudaMemcpyAsync(norm, w->norm, sizeof(float) * 2 * (w->n_in + w->n_out), cudaMemcpyDefault, st));
    return GM_OK;
}

long long gm_ws_param_count(const gm_ws* w) { return w ? (long long)w->n_par : 0; }

gm_status gm_ws_forward(gm_ws* w, const float* feat, int B, float* out, void* stream) {
    clear_error();
    GM_CHECK_ARG(w && feat && out, "NULL argument");
    GM_CHECK_ARG(B > 0 && B <= w->max_batch, "batch %d out of range (max %d)", B, w->max_batch);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int I = w->n_in, O = w->n_out;
    ws_normalize_kernel<<<cdiv((long)B * I, 256), 256, 0, st>>>(B, I, feat, w->norm, w->norm + I, w->x);
    GM_LAUNCH_CHECK();
    GM_TRY(ws_fwd(w, B, st));
    ws_denormalize_kernel<<<cdiv((long)B * O, 256), 256, 0, st>>>(B, O, w->y, w->norm + 2 * I, w->norm + 2 * I + O,
                                                                   out);
    GM_LAUNCH_CHECK();
    return GM_OK;
}

gm_status gm_ws_train_step(gm_ws* w, const float* feat, const float* target, int B, float lr, float beta1,
                           float beta2, float eps, float* loss, void* stream) {
    clear_error();
    GM_CHECK_ARG(w && feat && target, "NULL argument");
    GM_CHECK_ARG(B > 0 && B <= w->max_batch, "batch %d out of range (max %d)", B, w->max_batch);
    GM_CHECK_ARG(lr > 0.f && beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f,
                 "invalid Adam settings");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int I = w->n_in, H = w->n_hid, O = w->n_out;
    ws_normalize_kernel<<<cdiv((long)B * I, 256), 256, 0, st>>>(B, I, feat, w->norm, w->norm + I, w->x);
    GM_LAUNCH_CHECK();
    GM_TRY(ws_fwd(w, B, st));
    GM_CUDA_TRY(cudaMemsetAsync(w->loss, 0, sizeof(float), st));
    ws_mse_kernel<<<cdiv((long)B * O, 256), 256, 0, st>>>(B, O, w->y, target, w->norm + 2 * I, w->norm + 2 * I + O,
                                                           w->dy, w->loss);
    GM_LAUNCH_CHECK();
    float* g = w->grad;
    // layer 2: dW2 = a1' dy, db2 = sum dy, d1 = dy W2' * relu'(a1)
    GM_TRY(gemm(st, H, O, B, w->a1, 1, H, w->dy, O, 1, g + w->o_W[2], O, nullptr, false, false, w->status));
    ws_colsum_kernel<<<cdiv(O, 128), 128, 0, st>>>(B, O, w->dy, g + w->o_b[2]);
    GM_LAUNCH_CHECK();
    GM_TRY(gemm(st, B, H, O, w->dy, O, 1, w->par + w->o_W[2], 1, O, w->d1, H, nullptr, false, false, w->status));
    ws_relu_bwd_kernel<<<cdiv((long)B * H, 256), 256, 0, st>>>((long)B * H, w->a1, w->d1);
    GM_LAUNCH_CHECK();
    // layer 1
    GM_TRY(gemm(st, H, H, B, w->a0, 1, H, w->d1, H, 1, g + w->o_W[1], H, nullptr, false, false, w->status));
    ws_colsum_kernel<<<cdiv(H, 128), 128, 0, st>>>(B, H, w->d1, g + w->o_b[1]);
    GM_LAUNCH_CHECK();
    GM_TRY(gemm(st, B, H, H, w->d1, H, 1, w->par + w->o_W[1], 1, H, w->d0, H, nullptr, false, false, w->status));
    ws_relu_bwd_kernel<<<cdiv((long)B * H, 256), 256, 0, st>>>((long)B * H, w->a0, w->d0);
    GM_LAUNCH_CHECK();
    // layer 0
    GM_TRY(gemm(st, I, H, B, w->x, 1, I, w->d0, H, 1, g + w->o_W[0], H, nullptr, false, false, w->status));
    ws_colsum_kernel<<<cdiv(H, 128), 128, 0, st>>>(B, H, w->d0, g + w->o_b[0]);
    GM_LAUNCH_CHECK();
    ++w->step;
    const float c1 = 1.f - powf(beta1, (float)w->step), c2 = 1.f - powf(beta2, (float)w->step);
    ws_adam_kernel<<<cdiv(w->n_par, 256), 256, 0, st>>>(w->n_par, w->par, g, w->m1, w->m2, lr, beta1, beta2, eps, c1,
                                                         c2);
    GM_LAUNCH_CHECK();
    if (loss) GM_CUDA_TRY(cudaMemcpyAsync(loss, w->loss, sizeof(float), cudaMemcpyDefault, st));
    return GM_OK;
}

gm_status gm_ws_grad(gm_ws* w, float* grad, void* stream) {
    clear_error();
    GM_CHECK_ARG(w && grad, "NULL argument");
    GM_CUDA_TRY(cudaMemcpyAsync(grad, w->grad, sizeof(float) * w->n_par, cudaMemcpyDefault,
                                static_cast<cudaStream_t>(stream)));
    return GM_OK;
}

}  // extern "C"
