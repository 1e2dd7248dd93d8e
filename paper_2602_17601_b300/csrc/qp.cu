// The condensed QP (Eq. condensed_matrices) solved by ADMM.
//
//   P = H + rho (I + C~'C~)                     FP32 Gram, FP64 Cholesky + inverse
//   U = P^{-1} (A~'(rho z - y) - g)             every CTA, P^{-1} and H in shared memory
//   a = A~ U, z = clip(a + y/rho, l, h), y += rho (a - z)
//   stop when |a - z|_inf <= tol and |H U + g + A~'y|_inf <= tol
//
// One persistent cooperative kernel runs every iteration: each CTA owns a
// contiguous slice of C~ rows (balanced by non-zeros), keeps its rows' z and y,
// and adds its share of A~'w and A~'y into one of three rotating global
// accumulators; a bounded grid barrier separates iterations.  The box rows
// (A~ = [I; C~]) are evaluated redundantly by every CTA.
//
// Then the FP64 KKT certificate of the returned (U, y).
#include "ctx.h"
#include "kernels.h"

#include <mutex>

namespace gmi {

__global__ void form_p_kernel(int n, const float* __restrict__ H, const float* __restrict__ CtC,
                              float rho, float* __restrict__ P) {
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)n * n) return;
    int i = (int)(t / n), j = (int)(t % n);
    float v = H[t] + (CtC ? rho * CtC[t] : 0.f);
    if (i == j) v += rho;
    P[t] = v;
}

// s_r = 1 / max(|C~_r|_2, 1e-8), one warp per packed row (rows below the floor barely depend on U).
__global__ void row_norm_kernel(long rows, int nu, int Mnc, const float* __restrict__ Ct,
                                float* __restrict__ rs) {
    const long r = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const int ks = (int)(r / Mnc);
    const int L = (ks + 1) * nu;
    const long off = (long)Mnc * nu * ((long)ks * (ks + 1) / 2) + (r - (long)ks * Mnc) * L;
    double s = 0.0;
    for (int c = lane; c < L; c += 32) {
        const double v = Ct[off + c];
        s += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) rs[r] = (float)(1.0 / fmax(sqrt(s), 1e-8));   // floor keeps s_r^2 finite in FP32
}

// Right-looking Cholesky P = L L' in FP64, one CTA; a non-positive pivot sets GM_ERR_NUMERIC.
__global__ void cholesky_kernel(int n, const float* __restrict__ P, double* __restrict__ L,
                                int* status) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (long t = tid; t < (long)n * n; t += nt) {
        int i = (int)(t / n), j = (int)(t % n);
        L[t] = (j <= i) ? 0.5 * ((double)P[t] + (double)P[(long)j * n + i]) : 0.0;
    }
    __syncthreads();
    __shared__ double djj;
    for (int j = 0; j < n; ++j) {
        if (tid == 0) {
            double d = L[(long)j * n + j];
            if (!(d > 0.0)) {
                dev_fail(status, GM_ERR_NUMERIC);
                d = 1.0;
            }
            djj = sqrt(d);
            L[(long)j * n + j] = djj;
        }
        __syncthreads();
        for (int i = j + 1 + tid; i < n; i += nt) L[(long)i * n + j] /= djj;
        __syncthreads();
        const int tx = tid & 31, ty = tid >> 5, ny = nt >> 5;
        for (int i = j + 1 + ty; i < n; i += ny) {
            const double lij = L[(long)i * n + j];
            for (int k = j + 1 + tx; k <= i; k += 32) L[(long)i * n + k] -= lij * L[(long)k * n + j];
        }
        __syncthreads();
    }
}

// Column j of L^{-1} by forward substitution, one warp per column.
__global__ void trinv_kernel(int n, const double* __restrict__ L, double* __restrict__ Linv) {
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    for (int i = lane; i < j; i += 32) Linv[(long)i * n + j] = 0.0;
    for (int i = j; i < n; ++i) {
        double s = 0.0;
        for (int k = j + lane; k < i; k += 32) s += L[(long)i * n + k] * Linv[(long)k * n + j];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const double xi = ((i == j ? 1.0 : 0.0) - s) / L[(long)i * n + i];
        if (lane == 0) Linv[(long)i * n + j] = xi;
        __syncwarp();
    }
}

// P^{-1} = L^{-T} L^{-1}, accumulated in FP64, stored FP32 for the iterations.
__global__ void pinv_kernel(int n, const double* __restrict__ Linv, float* __restrict__ Pinv) {
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)n * n) return;
    int i = (int)(t / n), j = (int)(t % n);
    int k0 = i > j ? i : j;
    double s = 0.0;
    for (int k = k0; k < n; ++k) s += Linv[(long)k * n + i] * Linv[(long)k * n + j];
    Pinv[t] = (float)s;
}

struct AdmmArgs {
    int n, nu, Mnc;
    long rows;
    const float *Ct, *dt, *lo, *hi, *g, *H, *Pinv, *U0, *y0;
    const float* rs;         // per-row scale 1/|C~_r| (nullable: unscaled)
    float *U, *y, *z, *acc;
    unsigned* bar;
    int* status;
    const int* row_begin;
    float rho, tol;
    int max_iter;
    long long max_spins;
    gm_stats* stats;
};

constexpr int ADMM_THREADS = 256;
constexpr int ADMM_MAXC = 8;   // columns per lane: n <= 256

__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
    for (int o = 16; o > 0; o >>= 1) v = nmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <bool SMEM>
__global__ void __launch_bounds__(ADMM_THREADS) admm_kernel(AdmmArgs a) {
    extern __shared__ __align__(16) float sm[];
    const int n = a.n;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int NW = ADMM_THREADS / 32;
    float* base = sm + (SMEM ? 2 * n * n : 0);
    float* su = base;
    float* srhs = su + n;
    float* saty = srhs + n;
    float* zb = saty + n;
    float* yb = zb + n;
    float* red = yb + n;             // [NW][2n]
    float* wmax = red + NW * 2 * n;  // [NW]
    __shared__ float s_rpbox, s_rd;
    const float* Pinv = a.Pinv;
    const float* H = a.H;
    if (SMEM) {
        float* sP = sm;
        float* sH = sm + n * n;
        for (int t = tid; t < n * n; t += ADMM_THREADS) {
            sP[t] = a.Pinv[t];
            sH[t] = a.H[t];
        }
        Pinv = sP;
        H = sH;
    }
    const float rho = a.rho;
    for (int c = tid; c < n; c += ADMM_THREADS) {
        su[c] = a.U0 ? a.U0[c] : 0.f;
        yb[c] = a.y0 ? a.y0[c] : 0.f;
        zb[c] = fminf(fmaxf(su[c], a.lo[c]), a.hi[c]);
    }
    const unsigned G = gridDim.x;
    const long r0 = a.row_begin[blockIdx.x], r1 = a.row_begin[blockIdx.x + 1];
    const int stride = 2 * n + 1;
    __syncthreads();

    // one pass over this CTA's C~ rows; init: z = clip(a), y = y0
    auto row_pass = [&](bool init, float* accw) {
        float pw[ADMM_MAXC], py[ADMM_MAXC];
#pragma unroll
        for (int m = 0; m < ADMM_MAXC; ++m) pw[m] = py[m] = 0.f;
        float rp = 0.f;
        for (long r = r0 + warp; r < r1; r += NW) {
            const int ks = (int)(r / a.Mnc);
            const int wi = (int)(r - (long)ks * a.Mnc);
            const int L = (ks + 1) * a.nu;
            const long off = (long)a.Mnc * a.nu * ((long)ks * (ks + 1) / 2) + (long)wi * L;
            float v[ADMM_MAXC];
            float dot = 0.f;
#pragma unroll
            for (int m = 0; m < ADMM_MAXC; ++m) {
                const int c = lane + 32 * m;
                v[m] = c < L ? a.Ct[off + c] : 0.f;
                if (c < L) dot = fmaf(v[m], su[c], dot);
            }
            // the recurrence runs on the scaled row s_r C~_r <= s_r d~_r
            const float sr = a.rs ? a.rs[r] : 1.f;
            dot = warp_sum(dot) * sr;
            const float d = a.dt[r] * sr;
            float yr, zr;
            if (init) {
                yr = a.y0 ? a.y0[n + r] / sr : 0.f;
                zr = fminf(dot, d);
            } else {
                yr = a.y[n + r];
                zr = fminf(dot + yr / rho, d);
                yr = yr + rho * (dot - zr);
            }
            rp = nmaxf(rp, fabsf(dot - zr));
            if (lane == 0) {
                a.y[n + r] = yr;
                a.z[n + r] = zr;
            }
            const float w = (rho * zr - yr) * sr;
            const float ys = yr * sr;
#pragma unroll
            for (int m = 0; m < ADMM_MAXC; ++m) {
                pw[m] = fmaf(v[m], w, pw[m]);
                py[m] = fmaf(v[m], ys, py[m]);
            }
        }
#pragma unroll
        for (int m = 0; m < ADMM_MAXC; ++m) {
            const int c = lane + 32 * m;
            if (c < n) {
                red[warp * 2 * n + c] = pw[m];
                red[warp * 2 * n + n + c] = py[m];
            }
        }
        rp = warp_max(rp);
        if (lane == 0) wmax[warp] = rp;
        __syncthreads();
        for (int t = tid; t < 2 * n; t += ADMM_THREADS) {
            float s = 0.f;
            for (int w = 0; w < NW; ++w) s += red[w * 2 * n + t];
            if (r1 > r0) atomicAdd(accw + t, s);
        }
        if (tid == 0) {
            float m = 0.f;
            for (int w = 0; w < NW; ++w) m = nmaxf(m, wmax[w]);
            atomicMax(reinterpret_cast<unsigned*>(accw + 2 * n), __float_as_uint(m));
        }
    };

    // pass 0 (initial z, y); accumulator 0 is zeroed by the host
    if (blockIdx.x == 0)
        for (int t = tid; t < stride; t += ADMM_THREADS) a.acc[stride + t] = 0.f;
    row_pass(true, a.acc);
    unsigned phase = 1;
    bool ok = grid_barrier(a.bar, G, phase, a.max_spins, a.status);
    int it_done = 0;
    float rp_last = 0.f, rd_last = 0.f;
    int converged = 0;
    if (ok) {
        for (int it = 1;; ++it) {
            const float* accr = a.acc + ((it - 1) % 3) * stride;
            for (int c = tid; c < n; c += ADMM_THREADS) {
                const float wbox = rho * zb[c] - yb[c];
                srhs[c] = __ldcg(accr + c) + wbox - a.g[c];
                saty[c] = __ldcg(accr + n + c) + yb[c];
            }
            __syncthreads();
            if (it >= 2) {
                // dual residual of the iterate of pass it-1: |H U + g + A~'y|_inf
                float m = 0.f;
                for (int c = warp; c < n; c += NW) {
                    float s = 0.f;
                    for (int j = lane; j < n; j += 32) s = fmaf(H[(long)c * n + j], su[j], s);
                    s = warp_sum(s);
                    m = nmaxf(m, fabsf(s + a.g[c] + saty[c]));
                }
                if (lane == 0) wmax[warp] = m;
                __syncthreads();
                if (tid == 0) {
                    float mm = 0.f;
                    for (int w = 0; w < NW; ++w) mm = nmaxf(mm, wmax[w]);
                    s_rd = mm;
                }
                __syncthreads();
                rp_last = nmaxf(__uint_as_float(__ldcg(reinterpret_cast<const unsigned*>(accr + 2 * n))),
                                s_rpbox);
                rd_last = s_rd;
                converged = (rp_last <= a.tol && rd_last <= a.tol) ? 1 : 0;
                const bool bad = (rp_last != rp_last) || (rd_last != rd_last);
                if (bad && blockIdx.x == 0 && tid == 0) dev_fail(a.status, GM_ERR_NUMERIC);
                if (converged || bad || it - 1 >= a.max_iter) {
                    it_done = it - 1;
                    break;
                }
            }
            // U = P^{-1} rhs
            for (int c = warp; c < n; c += NW) {
                float s = 0.f;
                for (int j = lane; j < n; j += 32) s = fmaf(Pinv[(long)c * n + j], srhs[j], s);
                s = warp_sum(s);
                if (lane == 0) su[c] = s;
            }
            __syncthreads();
            // box rows
            float m = 0.f;
            for (int c = tid; c < n; c += ADMM_THREADS) {
                const float av = su[c];
                const float zn = fminf(fmaxf(av + yb[c] / rho, a.lo[c]), a.hi[c]);
                yb[c] = yb[c] + rho * (av - zn);
                zb[c] = zn;
                m = nmaxf(m, fabsf(av - zn));
            }
            m = warp_max(m);
            if (lane == 0) wmax[warp] = m;
            __syncthreads();
            if (tid == 0) {
                float mm = 0.f;
                for (int w = 0; w < NW; ++w) mm = nmaxf(mm, wmax[w]);
                s_rpbox = mm;
            }
            if (blockIdx.x == 0)
                for (int t = tid; t < stride; t += ADMM_THREADS) a.acc[((it + 1) % 3) * stride + t] = 0.f;
            row_pass(false, a.acc + (it % 3) * stride);
            ++phase;
            if (!grid_barrier(a.bar, G, phase, a.max_spins, a.status)) {
                ok = false;
                break;
            }
        }
    }
    // own rows back to the original scaling: y_r = s_r y'_r, z_r = z'_r / s_r
    if (a.rs)
        for (long r = r0 + tid; r < r1; r += ADMM_THREADS) {
            const float sr = a.rs[r];
            a.y[n + r] *= sr;
            a.z[n + r] /= sr;
        }
    if (blockIdx.x == 0) {
        for (int c = tid; c < n; c += ADMM_THREADS) {
            a.U[c] = su[c];
            a.y[c] = yb[c];
            a.z[c] = zb[c];
        }
        if (tid == 0 && a.stats) {
            a.stats->iters = it_done;
            a.stats->converged = converged;
            a.stats->r_prim = rp_last;
            a.stats->r_dual = rd_last;
            a.stats->polished = 0;
            if (!ok) a.stats->converged = 0;
        }
    }
}

// ---------------------------------------------------------------- FP64 KKT certificate
// kkt[0..n): A~'y (rows part), kkt[n]: max primal violation, kkt[n+1]: max wrong-sign y,
// kkt[n+2]: max complementarity, all over the C~ rows.
__device__ __forceinline__ void atomic_max_pos(double* p, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(v));
}

__global__ void kkt_rows_kernel(int n, int nu, int Mnc, long rows, const float* __restrict__ Ct,
                                const float* __restrict__ dt, const float* __restrict__ U,
                                const float* __restrict__ y, double* kkt) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NW = blockDim.x >> 5;
    extern __shared__ double dsm[];          // [NW][n]
    double part[ADMM_MAXC];
    for (int m = 0; m < ADMM_MAXC; ++m) part[m] = 0.0;
    double prim = 0.0, dual = 0.0, comp = 0.0;
    for (long r = (long)blockIdx.x * NW + warp; r < rows; r += (long)gridDim.x * NW) {
        const int ks = (int)(r / Mnc);
        const int wi = (int)(r - (long)ks * Mnc);
        const int L = (ks + 1) * nu;
        const long off = (long)Mnc * nu * ((long)ks * (ks + 1) / 2) + (long)wi * L;
        const double yr = y[n + r];
        double dot = 0.0;
        for (int m = 0; m < ADMM_MAXC; ++m) {
            const int c = lane + 32 * m;
            if (c < L) {
                const double v = Ct[off + c];
                dot += v * (double)U[c];
                part[m] += v * yr;
            }
        }
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        const double d = dt[r];
        prim = nmax(prim, dot - d);
        dual = nmax(dual, -yr);
        comp = nmax(comp, nmax(yr, 0.0) * fabs(d - dot));
    }
    for (int m = 0; m < ADMM_MAXC; ++m) {
        const int c = lane + 32 * m;
        if (c < n) dsm[warp * n + c] = part[m];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < NW; ++w) s += dsm[w * n + c];
        atomicAdd(kkt + c, s);
    }
    if (lane == 0) {
        atomic_max_pos(kkt + n, nmax(prim, 0.0));
        atomic_max_pos(kkt + n + 1, nmax(dual, 0.0));
        atomic_max_pos(kkt + n + 2, comp);
    }
}

__global__ void kkt_final_kernel(int n, const float* __restrict__ H, const float* __restrict__ g,
                                 const float* __restrict__ lo, const float* __restrict__ hi,
                                 const float* __restrict__ U, const float* __restrict__ y,
                                 const double* __restrict__ kkt, const int* status,
                                 gm_stats* stats) {
    __shared__ double red[4][32];
    double stat = 0.0, prim = 0.0, comp = 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        double s = (double)g[c] + (double)y[c] + kkt[c];
        for (int j = 0; j < n; ++j) s += (double)H[(long)c * n + j] * (double)U[j];
        stat = nmax(stat, fabs(s));
        const double u = U[c], l = lo[c], h = hi[c], yc = y[c];
        prim = nmax(prim, nmax(u - h, l - u));
        comp = nmax(comp, nmax(yc, 0.0) * fabs(h - u));
        comp = nmax(comp, nmax(-yc, 0.0) * fabs(u - l));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        stat = nmax(stat, __shfl_xor_sync(0xffffffffu, stat, o));
        prim = nmax(prim, __shfl_xor_sync(0xffffffffu, prim, o));
        comp = nmax(comp, __shfl_xor_sync(0xffffffffu, comp, o));
    }
    if (lane == 0) {
        red[0][w] = stat;
        red[1][w] = prim;
        red[2][w] = comp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        for (int i = 1; i < nw; ++i) {
            stat = nmax(stat, red[0][i]);
            prim = nmax(prim, red[1][i]);
            comp = nmax(comp, red[2][i]);
        }
        stats->kkt_stat = stat;
        stats->kkt_prim = nmax(nmax(prim, 0.0), kkt[n]);
        stats->kkt_dual = kkt[n + 1];
        stats->kkt_comp = nmax(comp, kkt[n + 2]);
        int st = *status;
        int code = GM_OK;
        if (st & (1 << GM_ERR_TIMEOUT)) code = GM_ERR_TIMEOUT;
        else if (st & (1 << GM_ERR_NUMERIC)) code = GM_ERR_NUMERIC;
        else if (!stats->converged) code = GM_ERR_NOT_CONVERGED;
        if (!(stat == stat)) code = GM_ERR_NUMERIC;
        stats->status = code;
    }
}

static bool admm_smem_mats(int n) {
    // P^{-1} and H resident in shared memory when they fit the 227 KB opt-in limit
    return (size_t)2 * n * n * sizeof(float) + (size_t)(5 * n + (ADMM_THREADS / 32) * 2 * n + 64) * sizeof(float) <=
           226 * 1024;
}

size_t admm_smem_bytes(const gm_ctx* c) {
    const int n = c->nU;
    return (admm_smem_mats(n) ? (size_t)2 * n * n * sizeof(float) : 0) +
           (size_t)(5 * n + (ADMM_THREADS / 32) * 2 * n + ADMM_THREADS / 32) * sizeof(float);
}

const void* admm_kernel_ptr(const gm_ctx* c) {
    return admm_smem_mats(c->nU) ? (const void*)admm_kernel<true> : (const void*)admm_kernel<false>;
}

gm_status qp_solve(gm_ctx* c, const float* H, const float* g, const float* Ct, const float* dt,
                   const float* u_lo, const float* u_hi, const float* warm_U, const float* warm_y,
                   float* U, float* y, gm_stats* stats, cudaStream_t st, cudaEvent_t ev_mid) {
    const int n = c->nU;
    const long rows = c->rows_c;
    float* yv = y ? y : c->d_y;
    GM_CUDA_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(int) * 4, st));
    // P = H + rho (I + C~'C~)
    const float* CtC = nullptr;
    if (rows > 0) {
        const float* rs = nullptr;
        if (c->s.scale_rows) {
            row_norm_kernel<<<cdiv(rows * 32, 256), 256, 0, st>>>(rows, c->nu, c->M * c->n_c, Ct, c->d_rs);
            GM_LAUNCH_CHECK();
            rs = c->d_rs;
        }
        GramRows R{Ct, c->M * c->n_c, c->nu, c->N, rs, 1, 1};
        const int T = (n + 31) / 32;
        const int nsplit = std::max(1, std::min(64, (2 * c->num_sms) / std::max(1, T * (T + 1) / 2)));
        GM_TRY(gram(c, R, nsplit, nullptr, 0.f, c->d_Pinv, st));   // C~'C~ into Pinv (scratch)
        CtC = c->d_Pinv;
    }
    form_p_kernel<<<cdiv((long)n * n, 256), 256, 0, st>>>(n, H, CtC, c->s.rho, c->d_P);
    GM_LAUNCH_CHECK();
    cholesky_kernel<<<1, 1024, 0, st>>>(n, c->d_P, c->d_L, c->d_status);
    GM_LAUNCH_CHECK();
    trinv_kernel<<<cdiv((long)n * 32, 128), 128, 0, st>>>(n, c->d_L, c->d_Linv);
    GM_LAUNCH_CHECK();
    pinv_kernel<<<cdiv((long)n * n, 256), 256, 0, st>>>(n, c->d_Linv, c->d_Pinv);
    GM_LAUNCH_CHECK();
    if (ev_mid) GM_CUDA_TRY(cudaEventRecord(ev_mid, st));
    // ADMM
    GM_CUDA_TRY(cudaMemsetAsync(c->d_bar, 0, sizeof(unsigned) * 4, st));
    GM_CUDA_TRY(cudaMemsetAsync(c->d_acc, 0, sizeof(float) * (2 * n + 1), st));
    AdmmArgs a{};
    a.n = n; a.nu = c->nu; a.Mnc = c->M * c->n_c; a.rows = rows;
    a.Ct = Ct; a.dt = dt; a.lo = u_lo; a.hi = u_hi; a.g = g; a.H = H; a.Pinv = c->d_Pinv;
    a.U0 = warm_U; a.y0 = warm_y;
    a.U = U; a.y = yv; a.z = c->d_z; a.acc = c->d_acc; a.bar = c->d_bar; a.status = c->d_status;
    a.row_begin = c->d_row_begin; a.rho = c->s.rho; a.tol = c->s.tol; a.max_iter = c->s.max_iter;
    a.max_spins = c->s.timeout_spins > 0 ? c->s.timeout_spins : (1LL << 26);
    a.stats = stats;
    a.rs = (rows > 0 && c->s.scale_rows) ? c->d_rs : nullptr;
    const bool smem_mats = admm_smem_mats(n);
    const size_t smem = admm_smem_bytes(c);
    GM_CUDA_TRY(cudaFuncSetAttribute(admm_kernel_ptr(c), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(c->admm_grid);
    cfg.blockDim = dim3(ADMM_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (smem_mats) {
        GM_CUDA_TRY(cudaLaunchKernelEx(&cfg, admm_kernel<true>, a));
    } else {
        GM_CUDA_TRY(cudaLaunchKernelEx(&cfg, admm_kernel<false>, a));
    }
    GM_LAUNCH_CHECK();
    // FP64 KKT certificate of (U, y)
    GM_CUDA_TRY(cudaMemsetAsync(c->d_kkt, 0, sizeof(double) * (n + 4), st));
    if (rows > 0) {
        const int threads = 256;
        kkt_rows_kernel<<<std::max(1, std::min(4 * c->num_sms, cdiv(rows, 8))), threads,
                          (threads / 32) * n * sizeof(double), st>>>(n, c->nu, c->M * c->n_c, rows, Ct,
                                                                    dt, U, yv, c->d_kkt);
        GM_LAUNCH_CHECK();
    }
    kkt_final_kernel<<<1, 256, 0, st>>>(n, H, g, u_lo, u_hi, U, yv, c->d_kkt, c->d_status, stats);
    GM_LAUNCH_CHECK();
    return GM_OK;
}

}  // namespace gmi

// ======================================================================= no-allocation variant
// gm_qp_solve_noalloc keeps every scratch buffer of the solve in this one
// array.  It is part of the library image, so a process that loads the
// library holds it on every GPU it uses until exit, and no call allocates.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GM_NOALLOC_SCRATCH_BYTES];

namespace gmi {

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_addr[256] = {};   // device address of g_noalloc_scratch, per device ordinal
constexpr int kNoAllocGrid = 64;
constexpr int kNoAllocSplit = 8;
}  // namespace

// C~ rows split over `grid` CTAs by non-zeros (one thread; the row count is bounded).
__global__ void noalloc_partition_kernel(long rows, int nu, int Mnc, int grid, int* rb) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double total = 0.0;
    for (long r = 0; r < rows; ++r) total += (double)((r / Mnc) + 1) * nu;
    rb[0] = 0;
    int b = 1;
    double acc = 0.0;
    for (long r = 0; r < rows && b < grid; ++r) {
        acc += (double)((r / Mnc) + 1) * nu;
        while (b < grid && acc >= total * b / grid) rb[b++] = (int)(r + 1);
    }
    for (; b <= grid; ++b) rb[b] = (int)rows;
}

}  // namespace gmi

extern "C" gm_status gm_qp_solve_noalloc(int N, int nu, int Mnc, const gm_settings* s, const float* H,
                                         const float* g, const float* Ct, const float* dt,
                                         const float* u_lo, const float* u_hi, float* U, float* y,
                                         gm_stats* stats, void* stream) {
    using namespace gmi;
    clear_error();
    GM_CHECK_ARG(s && H && g && u_lo && u_hi && U, "NULL argument");
    GM_CHECK_ARG(N >= 1 && nu >= 1 && Mnc >= 0, "need N >= 1, nu >= 1, Mnc >= 0");
    const int n = N * nu;
    const long rows = (long)N * Mnc;
    GM_CHECK_ARG(n <= GM_NOALLOC_MAX_NU, "N * nu = %d exceeds the no-allocation limit %d", n, GM_NOALLOC_MAX_NU);
    GM_CHECK_ARG(rows <= GM_NOALLOC_MAX_ROWS, "N * Mnc = %ld half-space rows exceed the no-allocation limit %d",
                 rows, GM_NOALLOC_MAX_ROWS);
    GM_CHECK_ARG(rows == 0 || (Ct && dt), "Ct/dt are NULL with Mnc = %d", Mnc);
    GM_CHECK_ARG(s->rho > 0.f && s->tol > 0.f && s->max_iter >= 1, "rho, tol must be > 0 and max_iter >= 1");
    int dev = 0;
    GM_CUDA_TRY(cudaGetDevice(&dev));
    GM_CHECK_ARG(dev >= 0 && dev < 256, "device ordinal %d out of range", dev);
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) GM_CUDA_TRY(cudaGetSymbolAddress(&g_noalloc_addr[dev], g_noalloc_scratch));
        base = g_noalloc_addr[dev];
    }
    Carver cv;
    cv.base = static_cast<char*>(base);
    float* P = cv.take<float>((size_t)n * n);
    float* Pinv = cv.take<float>((size_t)n * n);
    double* L = cv.take<double>((size_t)n * n);
    double* Linv = cv.take<double>((size_t)n * n);
    float* z = cv.take<float>(n + rows);
    float* ys = cv.take<float>(n + rows);
    float* rs = cv.take<float>(std::max(rows, 1L));
    float* acc = cv.take<float>(3 * (2 * (size_t)n + 1));
    unsigned* bar = cv.take<unsigned>(4);
    int* status = cv.take<int>(4);
    int* rb = cv.take<int>(kNoAllocGrid + 1);
    double* kkt = cv.take<double>(n + 4);
    gm_stats* st_s = cv.take<gm_stats>(1);
    const int T = (n + 31) / 32;
    float* part = cv.take<float>((size_t)kNoAllocSplit * T * T * 1024);
    if (cv.off > (size_t)GM_NOALLOC_SCRATCH_BYTES) {
        set_error("no-allocation scratch too small (%zu > %d bytes)", cv.off, GM_NOALLOC_SCRATCH_BYTES);
        return GM_ERR_INVALID_ARG;
    }
    float* yv = y ? y : ys;
    gm_stats* stv = stats ? stats : st_s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int sms = 1;
    GM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = rows > 0 ? (int)std::max(1L, std::min<long>(std::min(kNoAllocGrid, sms), rows / 16)) : 1;
    const bool scale = rows > 0 && s->scale_rows;
    GM_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int) * 4, st));
    if (rows > 0) {
        if (scale) {
            row_norm_kernel<<<cdiv(rows * 32, 256), 256, 0, st>>>(rows, nu, Mnc, Ct, rs);
            GM_LAUNCH_CHECK();
        }
        GramRows R{Ct, Mnc, nu, N, scale ? rs : nullptr, 1, 1};
        gram_kernel<<<dim3(T * (T + 1) / 2, kNoAllocSplit), 256, 0, st>>>(R, n, part);
        GM_LAUNCH_CHECK();
        gram_reduce_kernel<<<cdiv((long)n * n, 256), 256, 0, st>>>(n, kNoAllocSplit, part, nullptr, 0.f, Pinv);
        GM_LAUNCH_CHECK();
    }
    form_p_kernel<<<cdiv((long)n * n, 256), 256, 0, st>>>(n, H, rows > 0 ? Pinv : nullptr, s->rho, P);
    GM_LAUNCH_CHECK();
    cholesky_kernel<<<1, 1024, 0, st>>>(n, P, L, status);
    GM_LAUNCH_CHECK();
    trinv_kernel<<<cdiv((long)n * 32, 128), 128, 0, st>>>(n, L, Linv);
    GM_LAUNCH_CHECK();
    pinv_kernel<<<cdiv((long)n * n, 256), 256, 0, st>>>(n, Linv, Pinv);
    GM_LAUNCH_CHECK();
    GM_CUDA_TRY(cudaMemsetAsync(bar, 0, sizeof(unsigned) * 4, st));
    GM_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(float) * (2 * n + 1), st));
    noalloc_partition_kernel<<<1, 32, 0, st>>>(rows, nu, std::max(Mnc, 1), grid, rb);
    GM_LAUNCH_CHECK();
    AdmmArgs a{};
    a.n = n; a.nu = nu; a.Mnc = std::max(Mnc, 1); a.rows = rows;
    a.Ct = Ct; a.dt = dt; a.lo = u_lo; a.hi = u_hi; a.g = g; a.H = H; a.Pinv = Pinv;
    a.U0 = nullptr; a.y0 = nullptr; a.rs = scale ? rs : nullptr;
    a.U = U; a.y = yv; a.z = z; a.acc = acc; a.bar = bar; a.status = status; a.row_begin = rb;
    a.rho = s->rho; a.tol = s->tol; a.max_iter = s->max_iter;
    a.max_spins = s->timeout_spins > 0 ? s->timeout_spins : (1LL << 26);
    a.stats = stv;
    const bool mats = admm_smem_mats(n);
    const size_t smem = (mats ? (size_t)2 * n * n * sizeof(float) : 0) +
                        (size_t)(5 * n + (ADMM_THREADS / 32) * 2 * n + ADMM_THREADS / 32) * sizeof(float);
    const void* fn = mats ? (const void*)admm_kernel<true> : (const void*)admm_kernel<false>;
    GM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(ADMM_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (mats) {
        GM_CUDA_TRY(cudaLaunchKernelEx(&cfg, admm_kernel<true>, a));
    } else {
        GM_CUDA_TRY(cudaLaunchKernelEx(&cfg, admm_kernel<false>, a));
    }
    GM_LAUNCH_CHECK();
    GM_CUDA_TRY(cudaMemsetAsync(kkt, 0, sizeof(double) * (n + 4), st));
    if (rows > 0) {
        const int threads = 256;
        kkt_rows_kernel<<<std::max(1, std::min(4 * sms, cdiv(rows, 8))), threads, (threads / 32) * n * sizeof(double),
                          st>>>(n, nu, std::max(Mnc, 1), rows, Ct, dt, U, yv, kkt);
        GM_LAUNCH_CHECK();
    }
    kkt_final_kernel<<<1, 256, 0, st>>>(n, H, g, u_lo, u_hi, U, yv, kkt, status, stv);
    GM_LAUNCH_CHECK();
    return GM_OK;
}
