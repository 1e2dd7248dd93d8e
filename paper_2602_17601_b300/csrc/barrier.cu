// Barrier-cost obstacle variant (Sec. VI-B: one barrier term per measured node in the cost).
//
// The obstacle rows are the linearised clearances of the constraint form: row r of the
// condensed QP gives s_r(U) = d~_r - C~_r U.  Each row adds mu * beta(s_r) to the cost, beta
// the relaxed logarithmic barrier (Feller and Ebenbauer, IEEE TAC 2017):
//     beta(s) = -ln s                                          s >  delta
//     beta(s) = 1/2 (((s - 2 delta) / delta)^2 - 1) - ln delta  s <= delta
// (convex, twice continuously differentiable, finite inside an obstacle).  Because s_r is
// affine in U, the second-order model at the linearisation point U_hat is exact to second
// order, and folding it into the QP gives
//     H' = H + C~' diag(mu beta''(s^)) C~,
//     g' = g - C~' (mu beta'(s^) + mu beta''(s^) C~ U_hat),     s^ = d~ - C~ U_hat,
// after which the QP keeps only the input box.
//
// Kernels: one warp per row for the row terms (FP64 dot products of the packed row with
// U_hat), the weighted Gram product C~' diag(w) C~ (the tensor-core Gram of the ADMM set-up,
// FP32 operand precision), and a transposed sweep that accumulates C~' v in FP64.
#include "admm.h"
#include "kernels.h"

namespace gmi {

constexpr int BAR_T = 256;

__device__ __forceinline__ void bar_row_geom(long r, int nu, int Mnc, int& L, long& off) {
    const int ks = (int)(r / Mnc);            // stage of the row (0-based): ks + 1 blocks of nu
    L = (ks + 1) * nu;
    off = (long)Mnc * nu * ((long)ks * (ks + 1) / 2) + (r - (long)ks * Mnc) * L;
}

__device__ __forceinline__ double bar_warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// w_r = mu beta''(s^_r) (Gram weight, FP32), v_r = mu beta'(s^_r) + w_r (C~_r U_hat) (FP64)
__global__ void __launch_bounds__(BAR_T) barrier_rows_kernel(long rows, int nu, int Mnc,
                                                             const float* __restrict__ Ct,
                                                             const float* __restrict__ dt,
                                                             const float* __restrict__ U_hat, double mu,
                                                             double delta, float* __restrict__ w,
                                                             double* __restrict__ v) {
    const int lane = threadIdx.x & 31;
    const long warp0 = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long nwarps = ((long)gridDim.x * blockDim.x) >> 5;
    for (long r = warp0; r < rows; r += nwarps) {
        int L;
        long off;
        bar_row_geom(r, nu, Mnc, L, off);
        double a = 0.0;
        for (int c = lane; c < L; c += 32) a += (double)Ct[off + c] * (double)U_hat[c];
        a = bar_warp_sum(a);
        if (lane == 0) {
            const double s = (double)dt[r] - a;
            double b1, b2;
            if (s > delta) {
                b1 = -1.0 / s;
                b2 = 1.0 / (s * s);
            } else {
                b1 = (s - 2.0 * delta) / (delta * delta);
                b2 = 1.0 / (delta * delta);
            }
            w[r] = (float)(mu * b2);
            v[r] = mu * b1 + mu * b2 * a;
        }
    }
}

// acc[c] += sum_r C~_r[c] v_r: per-warp column partials in shared memory ([warps][n]; the
// lanes of a warp own distinct columns), summed over the block's warps, one FP64 atomic
// per column and block.
__global__ void __launch_bounds__(BAR_T) barrier_rowT_kernel(long rows, int nu, int Mnc, int n,
                                                             const float* __restrict__ Ct,
                                                             const double* __restrict__ v,
                                                             double* __restrict__ acc) {
    extern __shared__ double part[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = threadIdx.x; i < nw * n; i += blockDim.x) part[i] = 0.0;
    __syncthreads();
    double* mine = part + (long)wid * n;
    for (long r = (long)blockIdx.x * nw + wid; r < rows; r += (long)gridDim.x * nw) {
        int L;
        long off;
        bar_row_geom(r, nu, Mnc, L, off);
        const double vr = v[r];
        for (int c = lane; c < L; c += 32) mine[c] += (double)Ct[off + c] * vr;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < nw; ++k) s += part[(long)k * n + c];
        if (s != 0.0) atomicAdd(&acc[c], s);
    }
}

// H += G (the weighted Gram), g -= acc
__global__ void barrier_apply_kernel(int n, const float* __restrict__ G, const double* __restrict__ acc,
                                     float* __restrict__ H, float* __restrict__ g) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < (long)n * n) H[t] += G[t];
    if (t < n) g[t] = (float)((double)g[t] - acc[t]);
}

gm_status barrier_fold(gm_ctx* c, const float* Ct, const float* dt, const float* U_hat, float mu, float delta,
                       float* H, float* g, cudaStream_t st) {
    const int n = c->nU;
    const long rows = c->rows_c;
    if (rows == 0) return GM_OK;
    const int Mnc = c->M * c->n_c;
    const int sms = std::max(1, c->num_sms);
    // scratch: FP32 weights in the first interior-point row array, FP64 v in the second,
    // the FP64 column sums in the interior-point vectors
    float* w = reinterpret_cast<float*>(c->d_ipm_rows);
    double* v = c->d_ipm_rows + std::max(1L, rows);
    double* acc = c->d_ipm_vec;
    int nw = BAR_T / 32;
    while (nw > 1 && (size_t)nw * n * sizeof(double) > 48 * 1024) nw >>= 1;
    if ((size_t)nw * n * sizeof(double) > 48 * 1024) {
        set_error("barrier fold: N * nu = %d too large for the transposed sweep", n);
        return GM_ERR_INVALID_ARG;
    }
    GM_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(double) * n, st));
    const int g_dot = (int)std::max(1L, std::min((long)cdiv(rows * 32, (long)BAR_T), 8L * sms));
    barrier_rows_kernel<<<g_dot, BAR_T, 0, st>>>(rows, c->nu, Mnc, Ct, dt, U_hat, (double)mu, (double)delta, w, v);
    GM_LAUNCH_CHECK();
    const int nsplit = gram_split(n, sms, kGramSplitCap, c->gram_tc);
    GramRows R{Ct, Mnc, c->nu, c->N, w, 1, 0};
    GM_TRY(launch_gram(R, n, nsplit, c->d_gram_part, st, c->d_status, c->gram_tc));
    GM_TRY(launch_gram_reduce(n, nsplit, c->d_gram_part, nullptr, 0.f, c->d_G, st));
    const int g_T = (int)std::max(1L, std::min((long)cdiv(rows, (long)nw), 4L * sms));
    barrier_rowT_kernel<<<g_T, nw * 32, (size_t)nw * n * sizeof(double), st>>>(rows, c->nu, Mnc, n, Ct, v, acc);
    GM_LAUNCH_CHECK();
    barrier_apply_kernel<<<cdiv((long)n * n, 256), 256, 0, st>>>(n, c->d_G, acc, H, g);
    GM_LAUNCH_CHECK();
    return GM_OK;
}

}  // namespace gmi

using namespace gmi;

extern "C" gm_status gm_barrier_fold(gm_ctx* ctx, const float* Ct, const float* dt, const float* U_hat, float mu,
                                     float delta, float* H, float* g, void* stream) {
    clear_error();
    GM_CHECK_ARG(ctx && U_hat && H && g, "NULL argument");
    GM_CHECK_ARG(ctx->n_c == 0 || (Ct && dt), "Ct/dt are NULL with n_c = %d", ctx->n_c);
    GM_CHECK_ARG(mu > 0.f && delta > 0.f, "mu and delta must be > 0 (got %g, %g)", (double)mu, (double)delta);
    return barrier_fold(ctx, Ct, dt, U_hat, mu, delta, H, g, static_cast<cudaStream_t>(stream));
}
