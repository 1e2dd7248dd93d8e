// FP64 Cholesky factorisation of the ADMM x-update matrix P = H + rho (I + C~' S^2 C~)
// (Sec. V-B; the paper factors rho I + H once per solve) and the explicit inverse
// P^{-1} = L^{-T} L^{-1} used by the FP32 iterations, in one cooperative launch.
//
// FP64 issues at about 2 FMA per clock per SM on this part, so a one-CTA factorisation
// of n = 160 is held at ~0.5 ms by the pipe alone.  The work is spread over the grid
// in 16 x 16 blocks (the matrix padded with an identity block to np = 16 nb):
//   right-looking blocked Cholesky: per block column k, CTA 0 factors the diagonal
//   block and inverts it (D_k = L_kk^{-1}); the panel L_ik = A_ik D_k^T and the
//   trailing update A_ij -= L_ik L_jk^T run entry-parallel on all CTAs.  CTA 0
//   updates the next diagonal block itself and factors it at once, so a block
//   column costs two grid barriers;
//   X = L^{-1} by block rows: X_ii = D_i, X_ij = -sum_{m=j}^{i-1} (D_i L_im) X_mj;
//   P^{-1}[a][b] = sum_{q >= max(a,b)} X[q][a] X[q][b], stored FP32.
// Items of the thin phases are dealt to CTAs round-robin so that no single SM's FP64
// pipe carries a phase.  Values written by other CTAs are read through L2 (ld.cg).
#include "admm.h"
#include "common.cuh"

namespace gmi {

namespace {

constexpr int FB = 16;            // block size
constexpr int FT = 256;           // threads per CTA

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }

// Factor the FB x FB block S (row-major, lower part valid) in place with all threads of
// the CTA: S <- L_kk, written to L at block (k, k), and rd[j] = 1 / L_kk[j][j].  A
// non-positive pivot sets GM_ERR_NUMERIC and continues with 1.
__device__ void factor_diag(double (*S)[FB + 1], double* rd, int k, int np, double* L, double* Linv, int* status) {
    const int tid = threadIdx.x;
    for (int j = 0; j < FB; ++j) {
        if (tid == 0) {
            double d = S[j][j];
            if (!(d > 0.0)) {
                dev_fail(status, GM_ERR_NUMERIC);
                d = 1.0;
            }
            const double r = rsqrt(d);
            S[j][j] = d * r;
            rd[j] = r;
        }
        __syncthreads();
        if (tid > j && tid < FB) S[tid][j] *= rd[j];
        __syncthreads();
        // rank-1 update of the trailing lower triangle: entry (r, c), j < c <= r
        const int m = FB - 1 - j;
        if (tid < m * (m + 1) / 2) {
            int r = 0, t = tid;
            while (t > r) {
                t -= r + 1;
                ++r;
            }
            const int rr = j + 1 + r, cc = j + 1 + t;
            S[rr][cc] -= S[rr][j] * S[cc][j];
        }
        __syncthreads();
    }
    for (int e = tid; e < FB * FB; e += blockDim.x) {
        const int r = e / FB, c = e % FB;
        L[(long)(k * FB + r) * np + k * FB + c] = c <= r ? S[r][c] : 0.0;
    }
    // the pivot reciprocals, parked on the diagonal of Linv for the panel phase (the
    // diagonal-block inverses overwrite them later)
    if (tid < FB) Linv[(long)(k * FB + tid) * np + k * FB + tid] = rd[tid];
    __syncthreads();
}

}  // namespace

__global__ void __launch_bounds__(FT) factor_kernel(int n, int np, const float* __restrict__ P, double* L,
                                                    double* Linv, float* __restrict__ Pinv, int* status,
                                                    const AdmmState* gate, unsigned* bar, long long max_spins) {
    if (gate && (gate->done || !gate->need_factor)) return;     // uniform over the grid
    __shared__ double S[FB][FB + 1];
    __shared__ double Dm[FB][FB + 1];
    __shared__ double Pr[FB][FB + 1];             // panel rows of the next diagonal block
    __shared__ double rd[FB];
    const int tid = threadIdx.x, G = gridDim.x, b = blockIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int nb = np / FB;
    unsigned phase = 0;
    bool ok = true;
    auto sync = [&]() { ok = grid_barrier(bar, G, ++phase, max_spins, status) && ok; };

    // ---- L <- sym(P), padded with the identity; Linv <- 0
    for (long t = (long)b * FT + tid; t < (long)np * np; t += (long)G * FT) {
        const int r = (int)(t / np), c = (int)(t % np);
        double v = 0.0;
        if (c <= r && r < n) v = 0.5 * ((double)P[(long)r * n + c] + (double)P[(long)c * n + r]);
        else if (r == c) v = 1.0;
        L[t] = v;
        Linv[t] = 0.0;
    }
    sync();
    if (!ok) return;
    if (b == 0) {
        for (int e = tid; e < FB * FB; e += FT) S[e / FB][e % FB] = ldcg(&L[(long)(e / FB) * np + e % FB]);
        __syncthreads();
        factor_diag(S, rd, 0, np, L, Linv, status);
    }
    for (int k = 0; k < nb; ++k) {
        sync();                                  // L_kk and D_k final
        if (!ok) return;
        if (k == nb - 1) break;
        const int k0 = k * FB, r0 = k0 + FB;
        // ---- panel: L_ik = A_ik L_kk^{-T}, row by row (forward substitution, one thread per row)
        if (tid < FB * FB) Dm[tid / FB][tid % FB] = ldcg(&L[(long)(k0 + tid / FB) * np + k0 + tid % FB]);
        if (tid < FB) rd[tid] = ldcg(&Linv[(long)(k0 + tid) * np + k0 + tid]);
        __syncthreads();
        for (int r = r0 + b + G * tid; r < np; r += G * FT) {
            double x[FB];
#pragma unroll
            for (int c = 0; c < FB; ++c) x[c] = ldcg(&L[(long)r * np + k0 + c]);
            // right-looking: once x_c is final it updates all later entries (independent FMAs)
#pragma unroll
            for (int c = 0; c < FB; ++c) {
                x[c] *= rd[c];
#pragma unroll
                for (int q = c + 1; q < FB; ++q) x[q] -= x[c] * Dm[q][c];
            }
#pragma unroll
            for (int c = 0; c < FB; ++c) L[(long)r * np + k0 + c] = x[c];
        }
        sync();
        if (!ok) return;
        // ---- trailing update of the lower triangle below/right of the block
        const int m = np - r0;                    // trailing size
        if (b == 0) {
            // the next diagonal block: its panel rows staged once, updated into shared memory,
            // then factored at once
            if (tid < FB * FB) {
                Pr[tid / FB][tid % FB] = ldcg(&L[(long)(r0 + tid / FB) * np + k0 + tid % FB]);
                S[tid / FB][tid % FB] = ldcg(&L[(long)(r0 + tid / FB) * np + r0 + tid % FB]);
            }
            __syncthreads();
            if (tid < FB * FB) {
                const int r = tid / FB, c = tid % FB;
                if (c <= r) {
                    double v = S[r][c];
#pragma unroll
                    for (int q = 0; q < FB; ++q) v -= Pr[r][q] * Pr[c][q];
                    S[r][c] = v;
                }
            }
            __syncthreads();
            factor_diag(S, rd, k + 1, np, L, Linv, status);
        } else {
            // blocks (i, j), k < j <= i < nb, of the trailing lower triangle other than the next
            // diagonal block, dealt over CTAs 1..G-1: the two 16 x 16 panel blocks staged in shared
            // memory (Dm, Pr), then A_ij -= L_ik L_jk^T entry by entry (256 threads, 16 FMAs each)
            (void)m;
            const int mb = nb - k - 1;                      // trailing block rows
            const int nblk = mb * (mb + 1) / 2;             // lower-triangle blocks, (0, 0) is CTA 0's
            for (int t = b; t < nblk; t += G - 1) {         // t = 0 is the next diagonal block: skipped
                int bi = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
                while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
                while (bi * (bi + 1) / 2 > t) --bi;
                const int bj = t - bi * (bi + 1) / 2;       // bj <= bi
                const int ri = r0 + bi * FB, rj = r0 + bj * FB;
                __syncthreads();                            // the previous block's reads of Dm, Pr are done
                if (tid < FB * FB) {
                    Dm[tid / FB][tid % FB] = ldcg(&L[(long)(ri + tid / FB) * np + k0 + tid % FB]);
                    Pr[tid / FB][tid % FB] = ldcg(&L[(long)(rj + tid / FB) * np + k0 + tid % FB]);
                }
                __syncthreads();
                if (tid < FB * FB) {
                    const int r = tid / FB, c = tid % FB;
                    if (bi != bj || c <= r) {
                        double v = 0.0;
#pragma unroll
                        for (int q = 0; q < FB; ++q) v += Dm[r][q] * Pr[c][q];
                        double* e = &L[(long)(ri + r) * np + rj + c];
                        *e = ldcg(e) - v;                   // last written by another CTA: read through L2
                    }
                }
            }
        }
    }
    // ---- D_i = L_ii^{-1} into the diagonal blocks of Linv (block i on CTA i mod G; column c by
    // forward substitution on thread c)
    for (int i = b; i < nb; i += G) {
        if (tid < FB * FB) S[tid / FB][tid % FB] = ldcg(&L[(long)(i * FB + tid / FB) * np + i * FB + tid % FB]);
        if (tid < FB) rd[tid] = ldcg(&Linv[(long)(i * FB + tid) * np + i * FB + tid]);   // 1 / L_ii[r][r]
        __syncthreads();
        if (tid < FB) {
            const int c = tid;
            double col[FB];
#pragma unroll
            for (int r = 0; r < FB; ++r) {
                double v = (r == c) ? 1.0 : 0.0;
#pragma unroll
                for (int q = 0; q < r; ++q) v -= S[r][q] * col[q];
                col[r] = r < c ? 0.0 : v * rd[r];
            }
#pragma unroll
            for (int r = 0; r < FB; ++r) Linv[(long)(i * FB + r) * np + i * FB + c] = col[r];
        }
        __syncthreads();
    }
    sync();
    if (!ok) return;
    // ---- Lt_im = D_i L_im for m < i, in place in L (one item per block row i and column of L)
    for (int it = b + G * tid; it < (nb * (nb - 1) / 2) * FB; it += G * FT) {
        int i = 1, rem = it;
        while (rem >= i * FB) {
            rem -= i * FB;
            ++i;
        }
        const int col = rem;                      // column in [0, 16 i)
        double Lc[FB];
        for (int s = 0; s < FB; ++s) Lc[s] = ldcg(&L[(long)(i * FB + s) * np + col]);
        for (int r = 0; r < FB; ++r) {
            double v = 0.0;
            for (int s = 0; s <= r; ++s) v += ldcg(&Linv[(long)(i * FB + r) * np + i * FB + s]) * Lc[s];
            L[(long)(i * FB + r) * np + col] = v;
        }
    }
    sync();
    if (!ok) return;
    // ---- X = L^{-1} by block rows (X_ii = D_i already in Linv)
    for (int i = 1; i < nb; ++i) {
        const int ncol = i * FB;                  // columns left of the diagonal block
        for (int t = b + G * tid; t < FB * ncol; t += G * FT) {
            const int r = t / ncol, c = t % ncol;
            const int j0 = (c / FB) * FB;         // first column of block j
            double v = 0.0;
            for (int q = j0; q < i * FB; ++q)
                v -= ldcg(&L[(long)(i * FB + r) * np + q]) * ldcg(&Linv[(long)q * np + c]);
            Linv[(long)(i * FB + r) * np + c] = v;
        }
        sync();
        if (!ok) return;
    }
    // ---- P^{-1} = X' X (lower triangle computed, both halves stored)
    const long ntri = (long)n * (n + 1) / 2;
    for (long t = b + (long)G * tid; t < ntri; t += (long)G * FT) {
        int a = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
        while ((long)(a + 1) * (a + 2) / 2 <= t) ++a;
        while ((long)a * (a + 1) / 2 > t) --a;
        const int c = (int)(t - (long)a * (a + 1) / 2);   // c <= a
        double v = 0.0;
        for (int q = a; q < np; ++q) v += ldcg(&Linv[(long)q * np + a]) * ldcg(&Linv[(long)q * np + c]);
        Pinv[(long)a * n + c] = (float)v;
        Pinv[(long)c * n + a] = (float)v;
    }
}

int factor_pad(int n) { return (n + FB - 1) / FB * FB; }

int factor_grid() {
    static int g = 0;
    if (!g) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        g = sms >= 128 ? 128 : (sms > 2 ? sms : 2);   // the trailing update needs CTAs besides CTA 0
    }
    return g;
}

gm_status factor_pinv(int n, const float* P, double* L, double* Linv, float* Pinv, int* status,
                      const AdmmState* gate, unsigned* bar, long long max_spins, int grid, cudaStream_t st) {
    const int np = factor_pad(n);
    GM_CUDA_TRY(cudaMemsetAsync(bar, 0, sizeof(unsigned), st));
    cudaLaunchConfig_t cfg{};
    // at least 2 CTAs: the trailing update runs on the CTAs other than CTA 0
    cfg.gridDim = dim3(grid > 0 ? std::max(2, std::min(grid, factor_grid())) : factor_grid());
    cfg.blockDim = dim3(FT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    GM_CUDA_TRY(cudaLaunchKernelEx(&cfg, factor_kernel, n, np, P, L, Linv, Pinv, status, gate, bar, max_spins));
    GM_LAUNCH_CHECK();
    return GM_OK;
}

}  // namespace gmi
