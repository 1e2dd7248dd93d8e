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
//   D_k = L_kk^{-1} by column-wise forward substitution on an idle warp of the last CTA
//   while the panel of block column k is solved (CTA 0 does the last block's);
//   X = L^{-1} by columns, one column per CTA at a time, as a blocked forward
//   substitution inside the CTA: x_i = D_i (e_i - sum_{m<i} L_im x_m), no grid barrier;
//   P^{-1}[c][a] = sum_{q >= max(a,c)} X[q][c] X[q][a], row c by the CTA that owns
//   column c, stored FP32 (the sum is the same product sequence for (c, a) and (a, c),
//   so both halves agree bit for bit).
// Items of the thin phases are dealt to CTAs round-robin so that no single SM's FP64
// pipe carries a phase.  Values written by other CTAs are read through L2 (ld.cg).
#include "admm.h"
#include "common.cuh"

namespace gmi {

namespace {

constexpr int FB = 16;            // block size
constexpr int FT = 256;           // threads per CTA: 16 x 16 in the column solve
static_assert(FT == FB * FB, "the column solve maps 16 lanes to each row of a block row");
constexpr size_t kFactorMaxSmem = 160 * 1024;   // the X column in shared memory: np <= 20480

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }

// Factor the FB x FB block S (row-major, lower part valid) in place with the CTA's 256 threads,
// thread (r, c) = (tid / 16, tid % 16) holding entry (r, c) in a register: S <- L_kk, written to
// L at block (k, k), and rd[j] = 1 / L_kk[j][j].  Step j subtracts S_rj S_cj / d_j from every
// trailing entry (one FMA once the pivot's reciprocal is out); the owners of column j + 1 publish
// it for the next step, and the owner of entry (j + 1, j + 1) takes the next pivot at once, so a
// step costs one barrier.  L_rc = S_rc / sqrt(d_c) at the end.  A non-positive pivot sets
// GM_ERR_NUMERIC and continues with 1.
__device__ void factor_diag(double (*S)[FB + 1], double* rd, int k, int np, double* L, double* Linv, int* status) {
    __shared__ double cb[2][FB];      // column j of the working block (not yet scaled), two buffers
    __shared__ double iv[2];          // 1 / d_j
    const int tid = threadIdx.x, rr = tid >> 4, cc = tid & 15;
    const bool low = cc <= rr;
    double v = low ? S[rr][cc] : 0.0;
    auto pivot = [&](int j, int buf) {    // on thread (j, j), whose v is d_j
        if (!(v > 0.0)) {
            dev_fail(status, GM_ERR_NUMERIC);
            v = 1.0;
        }
        const double r = rsqrt(v);
        rd[j] = r;
        iv[buf] = r * r;
    };
    if (cc == 0) cb[0][rr] = v;
    if (tid == 0) pivot(0, 0);
    __syncthreads();
    for (int j = 0; j < FB - 1; ++j) {
        const int buf = j & 1;
        if (low && cc > j) {
            v = fma(-(cb[buf][rr] * cb[buf][cc]), iv[buf], v);
            if (cc == j + 1) {
                cb[buf ^ 1][rr] = v;
                if (rr == j + 1) pivot(j + 1, buf ^ 1);
            }
        }
        __syncthreads();
    }
    if (low) S[rr][cc] = v * rd[cc];
    __syncthreads();
    for (int e = tid; e < FB * FB; e += blockDim.x) {
        const int r = e / FB, c = e % FB;
        L[(long)(k * FB + r) * np + k * FB + c] = c <= r ? S[r][c] : 0.0;
    }
    // the pivot reciprocals, parked on the diagonal of Linv for the panel phase (the
    // diagonal-block inverses overwrite them later)
    if (tid < FB) Linv[(long)(k * FB + tid) * np + k * FB + tid] = rd[tid];
    __syncthreads();
}

// Column c of D_k = L_kk^{-1} (S: L_kk, lower part; rd: its pivot reciprocals) by forward
// substitution, into block (k, k) of Linv.  Entries above the diagonal are stored as exact zeros
// and the diagonal as rd itself, so the parked reciprocals keep their bits.
__device__ void diag_inverse_col(const double (*S)[FB + 1], const double* rd, int k, int np, double* Linv, int c) {
    double col[FB];
#pragma unroll
    for (int r = 0; r < FB; ++r) {
        double v = (r == c) ? 1.0 : 0.0;
#pragma unroll
        for (int q = 0; q < r; ++q) v -= S[r][q] * col[q];
        col[r] = r < c ? 0.0 : v * rd[r];
    }
#pragma unroll
    for (int r = 0; r < FB; ++r) Linv[(long)(k * FB + r) * np + k * FB + c] = col[r];
}

}  // namespace

__global__ void __launch_bounds__(FT, 1) factor_kernel(int n, int np, const float* __restrict__ P, double* L,
                                                    double* Linv, float* __restrict__ Pinv, int* status,
                                                    const AdmmState* gate, unsigned* bar, long long max_spins) {
    if (gate && (gate->done || !gate->need_factor)) return;     // uniform over the grid
    __shared__ double S[FB][FB + 1];
    __shared__ double Dm[FB][FB + 1];
    __shared__ double Pr[FB][FB + 1];             // panel rows of the next diagonal block
    __shared__ double Mm[FB][FB + 1];             // L_kk[q][j] / L_kk[j][j]
    __shared__ double rd[FB];
    __shared__ double rh[FB];                     // right-hand side of one block row of a column solve
    extern __shared__ double xs[];                // [np]: the column of X in hand
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
        if (nb == 1 && tid < FB) diag_inverse_col(S, rd, 0, np, Linv, tid);
    }
    for (int k = 0; k < nb; ++k) {
        sync();                                  // L_kk and D_k final
        if (!ok) return;
        if (k == nb - 1) break;
        const int k0 = k * FB, r0 = k0 + FB;
        // ---- panel: L_ik = A_ik L_kk^{-T}, a row per 16-lane group with lane c holding z_c.  With
        // M[q][j] = L_kk[q][j] / L_kk[j][j], once z_j is final it is broadcast in the group and every
        // later lane takes z_q -= z_j M[q][j] (one FP64 instruction per step for the whole warp:
        // FP64 issue, not lanes, is what a row costs here); x_c = z_c / L_kk[c][c] at the end.
        if (tid < FB * FB) {
            const int q = tid / FB, j = tid % FB;
            const double v = ldcg(&L[(long)(k0 + q) * np + k0 + j]);
            Dm[q][j] = v;
            Mm[q][j] = v * ldcg(&Linv[(long)(k0 + j) * np + k0 + j]);
        }
        if (tid < FB) rd[tid] = ldcg(&Linv[(long)(k0 + tid) * np + k0 + tid]);
        __syncthreads();
        {
            const int g = tid >> 4, c = tid & 15;
            for (int base = r0 + b; base < np; base += G * (FT / FB)) {
                const int r = base + G * g;
                const bool valid = r < np;
                if (__any_sync(0xffffffffu, valid)) {           // uniform over the warp
                    double z = valid ? ldcg(&L[(long)r * np + k0 + c]) : 0.0;
#pragma unroll
                    for (int j = 0; j < FB - 1; ++j) {
                        const double zj = __shfl_sync(0xffffffffu, z, j, FB);
                        if (c > j) z = fma(-zj, Mm[c][j], z);
                    }
                    if (valid) L[(long)r * np + k0 + c] = z * rd[c];
                }
            }
        }
        // D_k on the last CTA's last warp (no panel rows there at this size; its writes to the
        // diagonal of block (k, k) repeat the parked reciprocals bit for bit)
        if (b == G - 1 && tid >= FT - 32 && tid < FT - 32 + FB) diag_inverse_col(Dm, rd, k, np, Linv, tid - (FT - 32));
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
                    double u[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) u[q] = Pr[r][q] * Pr[c][q];
#pragma unroll
                    for (int q = 4; q < FB; ++q) u[q & 3] += Pr[r][q] * Pr[c][q];
                    S[r][c] -= (u[0] + u[1]) + (u[2] + u[3]);
                }
            }
            __syncthreads();
            factor_diag(S, rd, k + 1, np, L, Linv, status);
            if (k + 1 == nb - 1 && tid < FB) diag_inverse_col(S, rd, k + 1, np, Linv, tid);
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
    // ---- X = L^{-1} by columns.  Columns are dealt in a zig-zag (CTA b takes b, then 2G-1-b, ...)
    // so that the long columns (small c) and the short ones pair up.  Column c: for each block
    // row i from c's own, rh = e_c - sum_{m<i} L_im x_m (16 lanes per row, reduced in the half
    // warp), then x_i = D_i rh; X[:, c] is kept in shared memory and written to Linv.
    const int rr = tid >> 4, tt = tid & 15;
    for (int p = 0; p * G < n; ++p) {
        const int c = p * G + ((p & 1) ? G - 1 - b : b);
        if (c >= n) continue;
        const int ic = c / FB;
        for (int i = ic; i < nb; ++i) {
            const int R = i * FB + rr;
            // D_i[rr][tt] (zero above the diagonal): x_i = D_i rh is applied by all 256 threads, a
            // product each and a sum over the 16 lanes of a row, not by 16 threads in one warp
            const double dv = tt <= rr ? ldcg(&Linv[(long)(i * FB + rr) * np + i * FB + tt]) : 0.0;
            double part = 0.0, part1 = 0.0;
            int q = ic * FB + tt;
            for (; q + FB < i * FB; q += 2 * FB) {
                part += ldcg(&L[(long)R * np + q]) * xs[q];
                part1 += ldcg(&L[(long)R * np + q + FB]) * xs[q + FB];
            }
            if (q < i * FB) part += ldcg(&L[(long)R * np + q]) * xs[q];
            part += part1;
#pragma unroll
            for (int o = FB / 2; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (tt == 0) rh[rr] = (R == c ? 1.0 : 0.0) - part;
            __syncthreads();
            double v = dv * rh[tt];
#pragma unroll
            for (int o = FB / 2; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (tt == 0) {
                xs[R] = v;
                Linv[(long)R * np + c] = v;
            }
            __syncthreads();
        }
    }
    sync();
    if (!ok) return;
    // ---- P^{-1} row c = X[:, c]' X for each owned column c (X[q][a] = 0 for q < a)
    for (int p = 0; p * G < n; ++p) {
        const int c = p * G + ((p & 1) ? G - 1 - b : b);
        if (c >= n) continue;
        __syncthreads();                          // the previous row's reads of xs are done
        for (int q = tid; q < n; q += FT) xs[q] = ldcg(&Linv[(long)q * np + c]);
        __syncthreads();
        for (int a = tid; a < n; a += FT) {
            // four partial sums over q from max(a, c): the same sequence for (a, c) and (c, a)
            double u[4] = {0.0, 0.0, 0.0, 0.0};
            int q = a > c ? a : c;
#pragma unroll 2
            for (; q + 3 < n; q += 4) {
#pragma unroll
                for (int s = 0; s < 4; ++s) u[s] += ldcg(&Linv[(long)(q + s) * np + a]) * xs[q + s];
            }
            for (; q < n; ++q) u[0] += ldcg(&Linv[(long)q * np + a]) * xs[q];
            Pinv[(long)c * n + a] = (float)((u[0] + u[1]) + (u[2] + u[3]));
        }
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
    const size_t smem = (size_t)np * sizeof(double);          // one column of X
    if (smem > kFactorMaxSmem) return GM_ERR_INVALID_ARG;
    if (smem > 48 * 1024)
        GM_CUDA_TRY(cudaFuncSetAttribute(factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    GM_CUDA_TRY(cudaMemsetAsync(bar, 0, sizeof(unsigned), st));
    cudaLaunchConfig_t cfg{};
    // at least 2 CTAs: the trailing update runs on the CTAs other than CTA 0
    cfg.gridDim = dim3(grid > 0 ? std::max(2, std::min(grid, factor_grid())) : factor_grid());
    cfg.blockDim = dim3(FT);
    cfg.dynamicSmemBytes = smem;
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
