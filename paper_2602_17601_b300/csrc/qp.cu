// The condensed QP (Eq. condensed_matrices): set-up, FP64 factorisation, KKT check.
//
//   G = C~' D C~ (D = diag(s^2) with row scales s, or I)   FP32 Gram, once per solve
//   P(rho) = H + rho (I + G)                               FP64 Cholesky, FP64 L^{-1},
//   P^{-1} = L^{-T} L^{-1}                                 stored FP32 for the iterations
//   ADMM iterations with rho adaptation: admm.cu
//   FP64 KKT certificate of the returned (U, y): stationarity |H U + g + A~'y|_inf,
//   bound violation, wrong-sign multipliers, complementarity.
#include "admm.h"
#include "kernels.h"

#include <mutex>

namespace gmi {

// s_r = 1 / max(|C~_r|_2, 1e-8), one warp per packed row (rows below the floor barely depend on U).
__global__ void row_norm_kernel(long rows, int nu, int Mnc, const float* __restrict__ Ct,
                                float* __restrict__ rs) {
    const long r = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const int ks = (int)(r / Mnc);
    const int L = (ks + 1) * nu;
    const long off = (long)Mnc * nu * ((long)ks * (ks + 1) / 2) + (r - (long)ks * Mnc) * L;
    // FP32 sum of squares: the scale only preconditions the rows (any positive value leaves
    // the feasible set and U* unchanged), and FP64 would run on the slow FP64 pipe
    float s = 0.f;
    for (int c = lane; c < L; c += 32) {
        const float v = Ct[off + c];
        s = fmaf(v, v, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) rs[r] = 1.f / fmaxf(sqrtf(s), 1e-8f);   // floor keeps s_r^2 finite in FP32
}

// Row preparation of the ADMM: the row scale and the redundant-row test.  A row that no U in
// the input box can violate, because the box's support in its direction,
//     sup_r = max over lo <= U <= hi of C~_r U = sum_c max(C~_rc hi_c, C~_rc lo_c),
// lies below d~_r by more than kRedundantMargin (|C~_r|_1 max|bound| + |d~_r|), is inactive at
// every feasible U (its multiplier is 0 at the optimum) and does not change the feasible set.
// It gets s_r = 0, which takes it out of C~'S^2 C~ and out of every ADMM pass (keep_r = 0).
// Otherwise s_r = 1 / max(|C~_r|_2, 1e-8) (scale) or 1.  NaN rows are kept.  One warp per row.
__global__ void row_prep_kernel(long rows, int nu, int Mnc, const float* __restrict__ Ct,
                                const float* __restrict__ dt, const float* __restrict__ lo,
                                const float* __restrict__ hi, int scale, float* __restrict__ rs,
                                unsigned char* __restrict__ keep) {
    const long r = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const int ks = (int)(r / Mnc);
    const int L = (ks + 1) * nu;
    const long off = (long)Mnc * nu * ((long)ks * (ks + 1) / 2) + (r - (long)ks * Mnc) * L;
    float ss = 0.f, sup = 0.f, sc = 0.f;
    for (int c = lane; c < L; c += 32) {
        const float v = Ct[off + c];
        ss = fmaf(v, v, ss);
        if (v != 0.f) {
            const float l = lo[c], h = hi[c];
            sup += v > 0.f ? v * h : v * l;
            sc += fabsf(v) * fmaxf(fabsf(l), fabsf(h));
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
        sup += __shfl_xor_sync(0xffffffffu, sup, o);
        sc += __shfl_xor_sync(0xffffffffu, sc, o);
    }
    if (lane == 0) {
        const float d = dt[r];
        const bool redundant = sup < d - kRedundantMargin * (sc + fabsf(d));
        keep[r] = redundant ? 0 : 1;
        rs[r] = redundant ? 0.f : (scale ? 1.f / fmaxf(sqrtf(ss), 1e-8f) : 1.f);
    }
}

// Positions of the kept rows inside their stage (pos, exclusive) and kept rows per stage (cnt):
// one block per stage, blockDim rows at a time with a block-wide scan.
__global__ void keep_scan_kernel(int Mnc, const unsigned char* __restrict__ keep, int* __restrict__ pos,
                                 int* __restrict__ cnt) {
    __shared__ int wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const long base = (long)blockIdx.x * Mnc;
    int carry = 0;
    for (int c0 = 0; c0 < Mnc; c0 += blockDim.x) {
        const int v = c0 + tid < Mnc ? keep[base + c0 + tid] : 0;
        int x = v;                                          // inclusive warp scan
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < warp) before += wsum[w];
            total += wsum[w];
        }
        if (c0 + tid < Mnc) pos[base + c0 + tid] = carry + before + x - v;
        carry += total;
        __syncthreads();
    }
    if (tid == 0) cnt[blockIdx.x] = carry;
}

// ---------------------------------------------------------------- FP64 KKT certificate
// kkt[0..n): A~'y (rows part), kkt[n]: max primal violation, kkt[n+1]: max wrong-sign y,
// kkt[n+2]: max complementarity, all over the C~ rows.
// FP64 runs at about 2 FMA per clock per SM here, so each row is first tested in FP32: with
// s = sum_c |C~_rc U_c| (FP32), the FP32 dot lies within 64 s 2^-24 of the exact one (at most
// 8 sequential FMAs per lane and 5 levels of the lane sum, and s itself within that factor), so a
// row whose FP32 dot plus that bound is below d~_r and whose multiplier is 0 is strictly feasible:
// it adds nothing to any of the four quantities (the primal violation is clamped at 0).  Only
// the other rows take the FP64 evaluation, whose results are therefore unchanged.
constexpr int KKT_MAXC = 8;   // columns per lane: n <= 256

__device__ __forceinline__ void atomic_max_pos(double* p, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(v));
}

__global__ void kkt_rows_kernel(int n, int nu, int Mnc, long rows, const float* __restrict__ Ct,
                                const float* __restrict__ dt, const float* __restrict__ U,
                                const float* __restrict__ y, double* kkt) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NW = blockDim.x >> 5;
    extern __shared__ double dsm[];          // [NW][n]
    double part[KKT_MAXC], ud[KKT_MAXC];
    float uf[KKT_MAXC];                      // U as given, for the FP32 test (no conversions per row)
#pragma unroll
    for (int m = 0; m < KKT_MAXC; ++m) {
        part[m] = 0.0;
        uf[m] = lane + 32 * m < n ? U[lane + 32 * m] : 0.f;
        ud[m] = (double)uf[m];               // converted once
    }
    double prim = 0.0, dual = 0.0, comp = 0.0;
    for (long r = (long)blockIdx.x * NW + warp; r < rows; r += (long)gridDim.x * NW) {
        const int ks = (int)(r / Mnc);
        const int wi = (int)(r - (long)ks * Mnc);
        const int L = (ks + 1) * nu;
        const int nm = (L + 31) >> 5;              // 32-column blocks the row reaches (warp-uniform)
        const long off = (long)Mnc * nu * ((long)ks * (ks + 1) / 2) + (long)wi * L;
        const float yr32 = y[n + r];
        if (yr32 == 0.f) {                         // warp-uniform: the FP32 test of a row without multiplier
            float d32 = 0.f, a32 = 0.f;
#pragma unroll
            for (int m = 0; m < KKT_MAXC; ++m) {
                if (m >= nm) break;
                const int c = lane + 32 * m;
                if (c < L) {
                    const float p = Ct[off + c] * uf[m];
                    d32 += p;
                    a32 += fabsf(p);
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                d32 += __shfl_xor_sync(0xffffffffu, d32, o);
                a32 += __shfl_xor_sync(0xffffffffu, a32, o);
            }
            // d32 + 2^-18 a32 + 1e-30 rounded upwards, so the bound is never below its exact value and
            // the test stays rigorous in FP32 without an FP64 instruction on the path (1e-30: an
            // absolute allowance for products below FP32's normal range)
            if (__fadd_ru(__fmaf_ru(0x1p-18f, a32, d32), 1e-30f) < dt[r]) continue;
        }
        const double yr = (double)yr32;
        double dot = 0.0;
        if (yr != 0.0) {                           // warp-uniform: rows with a multiplier add C~_r' y_r
#pragma unroll
            for (int m = 0; m < KKT_MAXC; ++m) {
                if (m >= nm) break;                // FP64 issue slots only for the row's blocks
                const int c = lane + 32 * m;
                if (c < L) {
                    const double v = Ct[off + c];
                    dot += v * ud[m];
                    part[m] += v * yr;
                }
            }
        } else {
#pragma unroll
            for (int m = 0; m < KKT_MAXC; ++m) {
                if (m >= nm) break;
                const int c = lane + 32 * m;
                if (c < L) dot += (double)Ct[off + c] * ud[m];
            }
        }
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        const double d = dt[r];
        prim = nmax(prim, dot - d);
        dual = nmax(dual, -yr);
        comp = nmax(comp, nmax(yr, 0.0) * fabs(d - dot));
    }
    for (int m = 0; m < KKT_MAXC; ++m) {
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

// Stationarity rows in FP64, in place of kkt[c]: s_c = sum_j H_cj U_j + g_c + y_c + (C~'y)_c, one
// warp per c with the lanes along j.  The FP64 products run on the grid's SMs rather than in one
// block (160 dependent FMAs and 320 conversions per thread there took tens of microseconds).
__global__ void kkt_stat_kernel(int n, const float* __restrict__ H, const float* __restrict__ g,
                                const float* __restrict__ U, const float* __restrict__ y, double* kkt) {
    const int c = blockIdx.x, lane = threadIdx.x;
    double s0 = 0.0, s1 = 0.0;
    int j = lane;
    for (; j + 32 < n; j += 64) {
        s0 += (double)H[(long)c * n + j] * (double)U[j];
        s1 += (double)H[(long)c * n + j + 32] * (double)U[j + 32];
    }
    if (j < n) s0 += (double)H[(long)c * n + j] * (double)U[j];
    double s = s0 + s1;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) kkt[c] = s + ((double)g[c] + (double)y[c] + kkt[c]);
}

__global__ void kkt_final_kernel(int n, const float* __restrict__ H, const float* __restrict__ g,
                                 const float* __restrict__ lo, const float* __restrict__ hi,
                                 const float* __restrict__ U, const float* __restrict__ y,
                                 const double* __restrict__ kkt, const int* status, gm_stats* stats,
                                 AdmmState* S) {
    __shared__ double red[4][32];
    double stat = 0.0, prim = 0.0, comp = 0.0;
    (void)H;
    (void)g;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        stat = nmax(stat, fabs(kkt[c]));         // the stationarity row (kkt_stat_kernel)
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
        int st = status[0] | status[2];
        int code = GM_OK;
        if (st & (1 << GM_ERR_TIMEOUT)) code = GM_ERR_TIMEOUT;
        else if (st & (1 << GM_ERR_NUMERIC)) code = GM_ERR_NUMERIC;
        else if (st & (1 << GM_ERR_INFEASIBLE)) code = GM_ERR_INFEASIBLE;
        else if (!stats->converged) code = GM_ERR_NOT_CONVERGED;
        if (!(stat == stat) && code != GM_ERR_TIMEOUT) code = GM_ERR_NUMERIC;   // a timeout leaves garbage
        // a warm start abandoned for a cold restart that then converged
        if (S && code == GM_OK && S->fell_back) code = GM_STALLED;
        stats->status = code;
        if (S) S->final_status = code;
    }
}

// Row scales, Gram, ADMM rounds and KKT check on the given buffers.
gm_status launch_kkt_final(int n, const float* H, const float* g, const float* lo, const float* hi, const float* U,
                            const float* y, double* kkt, const int* status, gm_stats* stats, AdmmState* S,
                            cudaStream_t st) {
    kkt_stat_kernel<<<n, 32, 0, st>>>(n, H, g, U, y, kkt);
    GM_LAUNCH_CHECK();
    kkt_final_kernel<<<1, 256, 0, st>>>(n, H, g, lo, hi, U, y, kkt, status, stats, S);
    GM_LAUNCH_CHECK();
    return GM_OK;
}

static gm_status solve_with(AdmmPlan& p, int sms, int nsplit, float* gram_part, bool scale, double* kkt) {
    const int n = p.n;
    const long rows = p.rows;
    cudaStream_t st = p.st;
    // status[0..1]: this solve; status[2]: the GNN kernels of the same step (kept)
    GM_CUDA_TRY(cudaMemsetAsync(p.status, 0, sizeof(int) * 2, st));
    if (rows > 0) {
        row_prep_kernel<<<cdiv(rows * 32, 256), 256, 0, st>>>(rows, p.nu, p.Mnc, p.Ct, p.dt, p.lo, p.hi,
                                                              scale ? 1 : 0, const_cast<float*>(p.rs),
                                                              const_cast<unsigned char*>(p.keep));
        GM_LAUNCH_CHECK();
        keep_scan_kernel<<<(unsigned)(rows / p.Mnc), 1024, 0, st>>>(p.Mnc, p.keep, const_cast<int*>(p.kpos),
                                                                    const_cast<int*>(p.kcnt));
        GM_LAUNCH_CHECK();
        // the multipliers of rows the ADMM skips stay 0
        GM_CUDA_TRY(cudaMemsetAsync(p.y + p.n, 0, sizeof(float) * rows, st));
        GramRows R{p.Ct, p.Mnc, p.nu, p.N, p.rs, 1, 1};
        GM_TRY(launch_gram(R, n, nsplit, gram_part, st, p.status, p.gram_tc));
        GM_TRY(launch_gram_reduce(n, nsplit, gram_part, nullptr, 0.f, const_cast<float*>(p.Gram), st));
    }
    GM_TRY(admm_solve(p));
    GM_CUDA_TRY(cudaMemsetAsync(kkt, 0, sizeof(double) * (n + 4), st));
    if (rows > 0) {
        const int threads = 256;
        kkt_rows_kernel<<<std::max(1, std::min(4 * sms, cdiv(rows, 8))), threads, (threads / 32) * n * sizeof(double),
                          st>>>(n, p.nu, p.Mnc, rows, p.Ct, p.dt, p.U, p.y, kkt);
        GM_LAUNCH_CHECK();
    }
    return launch_kkt_final(n, p.H, p.g, p.lo, p.hi, p.U, p.y, kkt, p.status, p.stats, p.S, st);
}

size_t admm_smem_bytes(const gm_ctx* c) { return admm2_smem_bytes(c->nU); }
const void* admm_kernel_ptr(const gm_ctx* c) { return admm2_kernel_ptr(c->nU); }

gm_status qp_solve(gm_ctx* c, const float* H, const float* g, const float* Ct, const float* dt,
                   const float* u_lo, const float* u_hi, const float* warm_U, const float* warm_y,
                   float* U, float* y, gm_stats* stats, cudaStream_t st, cudaEvent_t ev_mid, bool keep_rho) {
    const int n = c->nU;
    const long rows = Ct && dt ? c->rows_c : 0;    // no rows: the box-only QP
    const bool scale = rows > 0 && c->s.scale_rows;
    AdmmPlan p{};
    p.n = n; p.nu = c->nu; p.Mnc = std::max(c->M * c->n_c, 1); p.N = c->N; p.rows = rows;
    p.Ct = Ct; p.dt = dt; p.lo = u_lo; p.hi = u_hi; p.g = g; p.H = H; p.U0 = warm_U; p.y0 = warm_y;
    p.rs = rows > 0 ? c->d_rs : nullptr;
    p.keep = c->d_keep; p.kpos = c->d_kpos; p.kcnt = c->d_kcnt;
    p.Gram = rows > 0 ? c->d_G : nullptr;
    p.U = U; p.y = y ? y : c->d_y; p.z = c->d_z;
    p.P = c->d_P; p.Pinv = c->d_Pinv; p.L = c->d_L; p.Linv = c->d_Linv;
    p.acc = c->d_acc; p.bar = c->d_bar; p.status = c->d_status; p.row_begin = c->d_row_begin;
    p.S = c->d_admm; p.stats = stats;
    p.rho0 = c->s.rho; p.tol = c->s.tol; p.max_iter = c->s.max_iter;
    p.keep_rho = keep_rho;
    p.warm = warm_U != nullptr || warm_y != nullptr;
    p.adapt_every = c->s.adapt_rho ? 25 : 0;
    // a warm start may take kWarmRounds launches before a cold restart takes the usual ones
    p.rounds = (c->s.adapt_rho ? 6 : 1) + (p.warm ? kWarmRounds : 0);
    p.grid = rows > 0 ? c->admm_grid : 1;
    p.factor_grid = c->s.factor_grid;
    p.max_spins = c->s.timeout_spins > 0 ? c->s.timeout_spins : (1LL << 26);
    p.st = st;
    p.ev_mid = ev_mid;
    p.body_st = c->cond_capture ? c->cond_stream : nullptr;
    p.gram_tc = c->gram_tc;
    return solve_with(p, c->num_sms, gram_split(n, c->num_sms, kGramSplitCap, c->gram_tc), c->d_gram_part, scale,
                      c->d_kkt);
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
    float* Gm = cv.take<float>((size_t)n * n);
    double* L = cv.take<double>((size_t)factor_pad(n) * factor_pad(n));
    double* Linv = cv.take<double>((size_t)factor_pad(n) * factor_pad(n));
    float* z = cv.take<float>(n + rows);
    float* ys = cv.take<float>(n + rows);
    float* rs = cv.take<float>(std::max(rows, 1L));
    unsigned char* keep = cv.take<unsigned char>(std::max(rows, 1L));
    int* kpos = cv.take<int>(std::max(rows, 1L));
    int* kcnt = cv.take<int>(N);
    float* acc = cv.take<float>(3 * (size_t)admm_acc_stride(n));
    unsigned* bar = cv.take<unsigned>(4);
    int* status = cv.take<int>(4);
    int* rb = cv.take<int>(kNoAllocGrid + 1);
    double* kkt = cv.take<double>(n + 4);
    gm_stats* st_s = cv.take<gm_stats>(1);
    AdmmState* S = cv.take<AdmmState>(1);
    const int T = (n + 31) / 32;
    float* part = cv.take<float>((size_t)kNoAllocSplit * T * T * 1024);
    if (cv.off > (size_t)GM_NOALLOC_SCRATCH_BYTES) {
        set_error("no-allocation scratch too small (%zu > %d bytes)", cv.off, GM_NOALLOC_SCRATCH_BYTES);
        return GM_ERR_INVALID_ARG;
    }
    int sms = 1;
    GM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const bool scale = rows > 0 && s->scale_rows;
    AdmmPlan p{};
    p.n = n; p.nu = nu; p.Mnc = std::max(Mnc, 1); p.N = N; p.rows = rows;
    p.Ct = Ct; p.dt = dt; p.lo = u_lo; p.hi = u_hi; p.g = g; p.H = H; p.U0 = nullptr; p.y0 = nullptr;
    p.rs = rows > 0 ? rs : nullptr;
    p.keep = keep; p.kpos = kpos; p.kcnt = kcnt;
    p.Gram = rows > 0 ? Gm : nullptr;
    p.U = U; p.y = y ? y : ys; p.z = z;
    p.P = P; p.Pinv = Pinv; p.L = L; p.Linv = Linv;
    p.acc = acc; p.bar = bar; p.status = status; p.row_begin = rb; p.S = S;
    p.stats = stats ? stats : st_s;
    p.rho0 = s->rho; p.tol = s->tol; p.max_iter = s->max_iter;
    p.adapt_every = s->adapt_rho ? 25 : 0;
    p.rounds = s->adapt_rho ? 6 : 1;
    p.grid = rows > 0 ? (int)std::max(1L, std::min<long>(std::min(kNoAllocGrid, sms), rows / 16)) : 1;
    p.max_spins = s->timeout_spins > 0 ? s->timeout_spins : (1LL << 26);
    p.st = static_cast<cudaStream_t>(stream);
    p.ev_mid = nullptr;
    GM_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int) * 4, p.st));
    return solve_with(p, sms, kNoAllocSplit, part, scale, kkt);
}
