// Learned ADMM warm start: a 3-layer MLP (in -> H -> H -> out, ReLU between) mapping pooled
// GNN latents and the reference to a primal input sequence and box duals, with its training
// kernels (MSE loss, backward, Adam).  Inputs and targets are standardised with stored
// means and deviations.  FP32 SIMT: the net is small and its products are 64 x 64 tiles.
#include <cstring>

#include "ctx.h"
#include "kernels.h"

struct gm_ws {
    int n_in = 0, n_hid = 0, n_out = 0, max_batch = 0;
    long n_par = 0;
    long o_W[3], o_b[3];           // parameter offsets
    float *par = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
    float* norm = nullptr;         // [in mean | in std | out mean | out std]
    float *x = nullptr, *a0 = nullptr, *a1 = nullptr, *y = nullptr;   // [B][in], [B][H], [B][H], [B][out]
    float *d0 = nullptr, *d1 = nullptr, *dy = nullptr;                // gradients of a0, a1, y
    float* loss = nullptr;
    int step = 0;                  // Adam step count
};

namespace gmi {
namespace {

constexpr int GT = 64;   // output tile
constexpr int GK = 16;   // K step

// C[i][j] (+)= sum_k A(i, k) B(k, j) (+ bias[j]) (ReLU): A(i, k) = A[i sai + k sak],
// B(k, j) = B[k sbk + j sbj], C row-major with ldc.  256 threads, 4 x 4 outputs each.
__global__ void __launch_bounds__(256) ws_gemm_kernel(int M, int N, int K, const float* __restrict__ A, long sai,
                                                      long sak, const float* __restrict__ B, long sbk, long sbj,
                                                      float* __restrict__ C, long ldc, const float* __restrict__ bias,
                                                      int relu, int accumulate) {
    __shared__ float As[GK][GT + 4];
    __shared__ float Bs[GK][GT + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int i0 = blockIdx.y * GT, j0 = blockIdx.x * GT;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += GK) {
        for (int t = tid; t < GK * GT; t += 256) {
            const int kk = t / GT, ii = t % GT;
            const int i = i0 + ii, j = j0 + ii, k = k0 + kk;
            As[kk][ii] = (i < M && k < K) ? A[(long)i * sai + (long)k * sak] : 0.f;
            Bs[kk][ii] = (j < N && k < K) ? B[(long)k * sbk + (long)j * sbj] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[kk][ty * 4 + q];
                b[q] = Bs[kk][tx * 4 + q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + ty * 4 + p, j = j0 + tx * 4 + q;
            if (i >= M || j >= N) continue;
            float v = acc[p][q];
            if (accumulate) v += C[(long)i * ldc + j];
            if (bias) v += bias[j];
            if (relu) v = fmaxf(v, 0.f);
            C[(long)i * ldc + j] = v;
        }
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
               long sbj, float* C, long ldc, const float* bias, bool relu, bool accumulate) {
    dim3 grid(cdiv(N, GT), cdiv(M, GT));
    ws_gemm_kernel<<<grid, 256, 0, st>>>(M, N, K, A, sai, sak, B, sbk, sbj, C, ldc, bias, relu ? 1 : 0,
                                         accumulate ? 1 : 0);
    GM_LAUNCH_CHECK();
    return GM_OK;
}

// forward on standardised inputs already in w->x: a0, a1, y (standardised outputs)
gm_status ws_fwd(gm_ws* w, int B, cudaStream_t st) {
    const int I = w->n_in, H = w->n_hid, O = w->n_out;
    GM_TRY(gemm(st, B, H, I, w->x, I, 1, w->par + w->o_W[0], H, 1, w->a0, H, w->par + w->o_b[0], true, false));
    GM_TRY(gemm(st, B, H, H, w->a0, H, 1, w->par + w->o_W[1], H, 1, w->a1, H, w->par + w->o_b[1], true, false));
    GM_TRY(gemm(st, B, O, H, w->a1, H, 1, w->par + w->o_W[2], O, 1, w->y, O, w->par + w->o_b[2], false, false));
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
    const long floats = 4 * P + 2 * (n_in + n_out) + B * (n_in + 4L * n_hidden + 2L * n_out) + 1;
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
    GM_TRY(gemm(st, H, O, B, w->a1, 1, H, w->dy, O, 1, g + w->o_W[2], O, nullptr, false, false));
    ws_colsum_kernel<<<cdiv(O, 128), 128, 0, st>>>(B, O, w->dy, g + w->o_b[2]);
    GM_LAUNCH_CHECK();
    GM_TRY(gemm(st, B, H, O, w->dy, O, 1, w->par + w->o_W[2], 1, O, w->d1, H, nullptr, false, false));
    ws_relu_bwd_kernel<<<cdiv((long)B * H, 256), 256, 0, st>>>((long)B * H, w->a1, w->d1);
    GM_LAUNCH_CHECK();
    // layer 1
    GM_TRY(gemm(st, H, H, B, w->a0, 1, H, w->d1, H, 1, g + w->o_W[1], H, nullptr, false, false));
    ws_colsum_kernel<<<cdiv(H, 128), 128, 0, st>>>(B, H, w->d1, g + w->o_b[1]);
    GM_LAUNCH_CHECK();
    GM_TRY(gemm(st, B, H, H, w->d1, H, 1, w->par + w->o_W[1], 1, H, w->d0, H, nullptr, false, false));
    ws_relu_bwd_kernel<<<cdiv((long)B * H, 256), 256, 0, st>>>((long)B * H, w->a0, w->d0);
    GM_LAUNCH_CHECK();
    // layer 0
    GM_TRY(gemm(st, I, H, B, w->x, 1, I, w->d0, H, 1, g + w->o_W[0], H, nullptr, false, false));
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
