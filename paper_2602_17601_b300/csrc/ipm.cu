// Primal-dual interior-point solve of the condensed QP (Eq. condensed_matrices), the solver
// class the paper's controller uses (Sec. VI-A), for comparison with ADMM:
//
//   min 1/2 U'HU + g'U   s.t.   G U <= h,   G = [I; -I; S C~],   h = [hi; -lo; S d~]
//
// (S the row scales 1/|C~_r|).  Mehrotra predictor-corrector on slacks s > 0 and duals
// z > 0 with residuals r_d = H U + g + G'z, r_p = G U + s - h, mu = s'z / m.  Each step
// solves the reduced Newton system
//
//   Phi dU = -r_d - G' S^{-1} (Z r_p - r_c),   Phi = H + G' Z S^{-1} G,
//   ds = -r_p - G dU,   dz = S^{-1} (-r_c - Z ds),
//
// with r_c = s o z (predictor) and s o z + ds_aff o dz_aff - sigma mu (corrector),
// sigma = (mu_aff / mu)^3, and a common step of 0.99 of the largest that keeps s, z > 0.
// Phi is formed with the weighted Gram kernel (C~' diag(w) C~, FP32), factored in FP64
// (factor.cu, which also gives L^{-1}); the two solves per iteration run in FP64 with L^{-1}.
// The run stops when |r_p|_inf, |r_d|_inf and max_i s_i z_i are all <= tol (the largest
// product, not the mean mu: with 10^5 rows a few rows far from complementarity hide in mu).
//
// The iterations are enqueued in chunks without host synchronisation: a device flag set
// on convergence makes the remaining launches of a chunk return at once (the factor kernel
// through the same gate it uses for ADMM), and the host reads the flag between chunks.
#include "admm.h"
#include "kernels.h"

namespace gmi {

// row arrays (double, max(rows, 1) each: slacks of rows with a large scaled bound need FP64)
enum { RA_S = 0, RA_Z, RA_A, RA_DS, RA_DZ, RA_CDU, RA_W };
// vectors (double, n each)
enum { V_U = 0, V_DU, V_RHS, V_S1, V_S2, V_Z1, V_Z2, V_DS1, V_DS2, V_DZ1, V_DZ2, V_RD, V_CTZ, V_CTV, V_Y, V_DIAG };
// scalars (double)
enum {
    SC_MU = 0, SC_SIGMA, SC_ALPHA, SC_SUMSZ, SC_SUMAFF, SC_RP, SC_DONE, SC_ITER, SC_RPN, SC_RDN, SC_ABND,
    SC_BOXAFF, SC_CONV, SC_MAXIT, SC_CMAX
};
static_assert(V_DIAG < kIpmVecArrays && SC_CMAX < kIpmScalars && RA_W < kIpmRowArrays, "IPM workspace");

constexpr int IPM_T = 256;       // threads of the row kernels and of the vector kernel
constexpr int IPM_MAXC = 8;      // columns per lane in the transposed sweep (n <= 256)

struct IpmArgs {
    int n, nu, Mnc;
    long rows;
    const float *H, *g, *Ct, *dt, *lo, *hi, *rs;
    double* rw;           // row arrays [RA_*][R]
    long R;               // row-array stride
    double* v;            // vectors [V_*][n]
    double* sc;           // scalars
    const float* Gram;    // C~' diag(w) C~
    float* Phi;
    const double* Linv;   // [np][np], lower-triangular L^{-1}
    int np;
    AdmmState* gate;      // factor gate (done / need_factor)
    float tol;
};

__device__ __forceinline__ void ipm_row_geom(const IpmArgs& a, long r, int& L, long& off) {
    const int ks = (int)(r / a.Mnc);
    L = (ks + 1) * a.nu;
    off = (long)a.Mnc * a.nu * ((long)ks * (ks + 1) / 2) + (r - (long)ks * a.Mnc) * L;
}
__device__ __forceinline__ void atomic_min_pos(double* p, double v) {   // v >= 0
    atomicMin(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void atomic_max_pos(double* p, double v) {   // v >= 0
    atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ double warp_min(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// largest step t <= inf with x + t dx >= 0 (x > 0)
__device__ __forceinline__ double step_bound(double x, double dx) { return dx < 0.0 ? -x / dx : 1e300; }

// Block reduction of one value per thread into a scalar: op 0 min, 1 max, 2 sum.
template <int OP>
__device__ __forceinline__ void block_reduce_to(double v, double* dst) {
    __shared__ double red[IPM_T / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = OP == 0 ? warp_min(v) : OP == 1 ? warp_max(v) : warp_sum(v);
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = red[0];
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) t = OP == 0 ? fmin(t, red[i]) : OP == 1 ? fmax(t, red[i]) : t + red[i];
        if (OP == 0) atomic_min_pos(dst, t);
        else if (OP == 1) atomic_max_pos(dst, t);
        else atomicAdd(dst, t);
    }
    __syncthreads();
}

// Row dots x_r = S_r C~_r . vec, one warp per row, and what each mode does with them:
//   0 (start): a = S C~ U, s = max(d' - a, 1), z = 1; sums s'z and max |r_p|
//   1 (predictor): ds = -r_p - x, dz = -z - (z/s) ds; step bound
//   2 (corrector): r_c = s z + ds_aff dz_aff - sigma mu, ds = -r_p - x, dz = (-r_c - z ds)/s,
//      x kept for the update of a; step bound
template <int MODE>
__global__ void __launch_bounds__(IPM_T) ipm_rowdot_kernel(IpmArgs a) {
    if (a.sc[SC_DONE] != 0.0) return;
    const int lane = threadIdx.x & 31;
    const long warp0 = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long nwarps = ((long)gridDim.x * blockDim.x) >> 5;
    const double* vec = a.v + (long)(MODE == 0 ? V_U : V_DU) * a.n;
    double* S = a.rw + RA_S * a.R;
    double* Z = a.rw + RA_Z * a.R;
    double* A = a.rw + RA_A * a.R;
    double* DS = a.rw + RA_DS * a.R;
    double* DZ = a.rw + RA_DZ * a.R;
    double* CDU = a.rw + RA_CDU * a.R;
    const double sigma_mu = MODE == 2 ? a.sc[SC_SIGMA] * a.sc[SC_MU] : 0.0;
    double bnd = 1e300, sum = 0.0, rpmax = 0.0, cmax = 0.0;
    for (long r = warp0; r < a.rows; r += nwarps) {
        int L;
        long off;
        ipm_row_geom(a, r, L, off);
        double x = 0.0;
        for (int c = lane; c < L; c += 32) x += (double)a.Ct[off + c] * vec[c];
        x = warp_sum(x) * a.rs[r];
        if (lane == 0) {
            const double dp = (double)a.dt[r] * a.rs[r];
            if (MODE == 0) {
                const double s = fmax(dp - x, 1.0);
                A[r] = x;
                S[r] = s;
                Z[r] = 1.0;
                sum += s;
                cmax = fmax(cmax, s);
                rpmax = fmax(rpmax, fabs(x + s - dp));
            } else {
                const double s = S[r], z = Z[r], rp = (double)A[r] + s - dp;
                const double ds = -rp - x;
                double dz;
                if (MODE == 1) {
                    dz = -z - (z / s) * ds;
                } else {
                    const double rc = s * z + (double)DS[r] * DZ[r] - sigma_mu;
                    dz = (-rc - z * ds) / s;
                    CDU[r] = x;
                }
                DS[r] = ds;
                DZ[r] = dz;
                bnd = fmin(bnd, fmin(step_bound(s, ds), step_bound(z, dz)));
            }
        }
    }
    if (MODE == 0) {
        block_reduce_to<2>(sum, &a.sc[SC_SUMSZ]);
        block_reduce_to<1>(rpmax, &a.sc[SC_RP]);
        block_reduce_to<1>(cmax, &a.sc[SC_CMAX]);
    } else {
        block_reduce_to<0>(bnd, &a.sc[SC_ABND]);
    }
}

// Element-wise row passes: 3 sums (s + alpha ds)(z + alpha dz) for mu_aff; 4 takes the
// step (s, z, a += alpha (ds, dz, x)) and sums s'z and max |r_p| for the next iteration.
template <int MODE>
__global__ void __launch_bounds__(IPM_T) ipm_rowelem_kernel(IpmArgs a) {
    if (a.sc[SC_DONE] != 0.0) return;
    const double alpha = a.sc[SC_ALPHA];
    double* S = a.rw + RA_S * a.R;
    double* Z = a.rw + RA_Z * a.R;
    double* A = a.rw + RA_A * a.R;
    const double* DS = a.rw + RA_DS * a.R;
    const double* DZ = a.rw + RA_DZ * a.R;
    const double* CDU = a.rw + RA_CDU * a.R;
    double sum = 0.0, rpmax = 0.0, cmax = 0.0;
    for (long r = (long)blockIdx.x * blockDim.x + threadIdx.x; r < a.rows; r += (long)gridDim.x * blockDim.x) {
        const double s1 = (double)S[r] + alpha * DS[r], z1 = (double)Z[r] + alpha * DZ[r];
        if (MODE == 3) {
            sum += s1 * z1;
        } else {
            const double a1 = (double)A[r] + alpha * CDU[r];
            S[r] = s1;
            Z[r] = z1;
            A[r] = a1;
            sum += s1 * z1;
            cmax = fmax(cmax, s1 * z1);
            rpmax = fmax(rpmax, fabs(a1 + s1 - (double)a.dt[r] * a.rs[r]));
        }
    }
    block_reduce_to<2>(sum, &a.sc[MODE == 3 ? SC_SUMAFF : SC_SUMSZ]);
    if (MODE == 4) {
        block_reduce_to<1>(rpmax, &a.sc[SC_RP]);
        block_reduce_to<1>(cmax, &a.sc[SC_CMAX]);
    }
}

// Transposed sweep G_rows' v: each lane keeps partial sums for columns lane + 32 m over its
// warp's rows, block-reduced and added to the global vectors.  Mode 0 (predictor):
// C'z -> V_CTZ, C'(w r_p - z) -> V_CTV and the Gram weights w_r S_r^2 (w = z/s); mode 1
// (corrector): C'(w r_p - r_c / s) -> V_CTV.  (C' = S C~.)
template <int MODE>
__global__ void __launch_bounds__(IPM_T) ipm_rowT_kernel(IpmArgs a) {
    if (a.sc[SC_DONE] != 0.0) return;
    extern __shared__ double tsm[];                    // [NW][2][n]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, NW = blockDim.x >> 5;
    const long warp0 = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long nwarps = ((long)gridDim.x * blockDim.x) >> 5;
    const double* S = a.rw + RA_S * a.R;
    const double* Z = a.rw + RA_Z * a.R;
    const double* A = a.rw + RA_A * a.R;
    const double* DS = a.rw + RA_DS * a.R;
    const double* DZ = a.rw + RA_DZ * a.R;
    float* Wt = reinterpret_cast<float*>(a.rw + RA_W * a.R);   // FP32 Gram weights
    const double sigma_mu = MODE == 1 ? a.sc[SC_SIGMA] * a.sc[SC_MU] : 0.0;
    double p1[IPM_MAXC], p2[IPM_MAXC];
#pragma unroll
    for (int m = 0; m < IPM_MAXC; ++m) p1[m] = p2[m] = 0.0;
    for (long r = warp0; r < a.rows; r += nwarps) {
        int L;
        long off;
        ipm_row_geom(a, r, L, off);
        const double rsr = a.rs[r];
        const double s = S[r], z = Z[r], rp = (double)A[r] + s - (double)a.dt[r] * rsr, wr = z / s;
        double v1 = 0.0, v2;
        if (MODE == 0) {
            v1 = z;
            v2 = wr * rp - z;
            if (lane == 0) Wt[r] = (float)(wr * rsr * rsr);
        } else {
            const double rc = s * z + (double)DS[r] * DZ[r] - sigma_mu;
            v2 = wr * rp - rc / s;
        }
#pragma unroll
        for (int m = 0; m < IPM_MAXC; ++m) {
            const int c = lane + 32 * m;
            if (c < L) {
                const double coef = (double)a.Ct[off + c] * rsr;
                if (MODE == 0) p1[m] += coef * v1;
                p2[m] += coef * v2;
            }
        }
    }
#pragma unroll
    for (int m = 0; m < IPM_MAXC; ++m) {
        const int c = lane + 32 * m;
        if (c < a.n) {
            tsm[(w * 2 + 0) * a.n + c] = p1[m];
            tsm[(w * 2 + 1) * a.n + c] = p2[m];
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < a.n; c += blockDim.x) {
        double t1 = 0.0, t2 = 0.0;
        for (int q = 0; q < NW; ++q) {
            t1 += tsm[(q * 2 + 0) * a.n + c];
            t2 += tsm[(q * 2 + 1) * a.n + c];
        }
        if (MODE == 0) atomicAdd(&a.v[(long)V_CTZ * a.n + c], t1);
        atomicAdd(&a.v[(long)V_CTV * a.n + c], t2);
    }
}

// Phi = H + Gram + diag(box weights), FP32 for the FP64 factor kernel.
__global__ void ipm_phi_kernel(IpmArgs a) {
    if (a.sc[SC_DONE] != 0.0) return;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)a.n * a.n) return;
    const int i = (int)(t / a.n), j = (int)(t % a.n);
    double v = (double)a.H[t] + (a.rows > 0 ? (double)a.Gram[t] : 0.0);
    if (i == j) v += a.v[(long)V_DIAG * a.n + i];
    a.Phi[t] = (float)v;
}

// dU = L^{-T} (L^{-1} rhs) in FP64 (one thread per component; sh holds L^{-1} rhs)
__device__ __forceinline__ double ipm_solve(const IpmArgs& a, double rhs_c, double* sh) {
    const int c = threadIdx.x, n = a.n;
    __syncthreads();
    if (c < n) sh[c] = rhs_c;
    __syncthreads();
    double yv = 0.0;
    if (c < n)
        for (int j = 0; j <= c; ++j) yv += a.Linv[(long)c * a.np + j] * sh[j];
    __syncthreads();
    if (c < n) sh[c] = yv;
    __syncthreads();
    double x = 0.0;
    if (c < n)
        for (int i = c; i < n; ++i) x += a.Linv[(long)i * a.np + c] * sh[i];
    return x;
}

// The n-sized part of an iteration, one CTA (thread c = component c).  Stages:
//   0 start: U = clip(0) (box midpoint if 0 lies outside), box slacks max(., 1), duals 1
//   1 residuals r_d, r_p, mu; convergence (sets the done flags); predictor right-hand side
//   2 predictor solve; box predictor steps and their step bound
//   3 predictor step length alpha_aff and the box part of mu_aff
//   4 centring sigma = (mu_aff / mu)^3
//   5 corrector right-hand side and solve; box corrector steps and their step bound
//   6 step length alpha = min(1, 0.99 bound)
//   7 update U and the box slacks and duals
__global__ void __launch_bounds__(IPM_T) ipm_vec_kernel(IpmArgs a, int stage, int max_iter) {
    if (stage != 0 && a.sc[SC_DONE] != 0.0) return;
    __shared__ double sh[IPM_T];
    const int c = threadIdx.x, n = a.n;
    const double m_total = 2.0 * n + (double)a.rows;
    double* V = a.v;
    auto vv = [&](int k) { return V + (long)k * n; };
    const bool act = c < n;
    double lo = 0, hi = 0, U = 0, s1 = 1, s2 = 1, z1 = 1, z2 = 1;
    if (act) {
        lo = a.lo[c];
        hi = a.hi[c];
        if (stage != 0) {
            U = vv(V_U)[c];
            s1 = vv(V_S1)[c];
            s2 = vv(V_S2)[c];
            z1 = vv(V_Z1)[c];
            z2 = vv(V_Z2)[c];
        }
    }
    const double rp1 = U + s1 - hi, rp2 = -U + s2 + lo, w1 = z1 / s1, w2 = z2 / s2;
    if (stage == 0) {
        if (act) {
            const double u0 = (lo <= 0.0 && 0.0 <= hi) ? 0.0 : 0.5 * (lo + hi);
            vv(V_U)[c] = u0;
            vv(V_S1)[c] = fmax(hi - u0, 1.0);
            vv(V_S2)[c] = fmax(u0 - lo, 1.0);
            vv(V_Z1)[c] = 1.0;
            vv(V_Z2)[c] = 1.0;
            vv(V_CTZ)[c] = 0.0;
            vv(V_CTV)[c] = 0.0;
        }
        if (c < kIpmScalars) a.sc[c] = 0.0;
        __syncthreads();
        if (c == 0) {
            a.sc[SC_ABND] = 1e300;
            a.sc[SC_MAXIT] = max_iter;
            a.gate->done = 0;
            a.gate->need_factor = 1;
        }
    } else if (stage == 1) {
        double rd = 0.0, rhs = 0.0;
        if (act) {
            rd = (double)a.g[c] + z1 - z2 + vv(V_CTZ)[c];
            for (int j = 0; j < n; ++j) rd += (double)a.H[(long)c * n + j] * vv(V_U)[j];
            rhs = -rd - ((w1 * rp1 - z1) - (w2 * rp2 - z2)) - vv(V_CTV)[c];
            vv(V_RD)[c] = rd;
            vv(V_RHS)[c] = rhs;
            vv(V_DIAG)[c] = w1 + w2;
        }
        __shared__ double red[4][IPM_T / 32];
        double x0 = act ? fabs(rd) : 0.0, x1 = act ? fmax(fabs(rp1), fabs(rp2)) : 0.0;
        double x2 = act ? s1 * z1 + s2 * z2 : 0.0, x3 = act ? fmax(s1 * z1, s2 * z2) : 0.0;
        x0 = warp_max(x0);
        x1 = warp_max(x1);
        x2 = warp_sum(x2);
        x3 = warp_max(x3);
        if ((c & 31) == 0) {
            red[0][c >> 5] = x0;
            red[1][c >> 5] = x1;
            red[2][c >> 5] = x2;
            red[3][c >> 5] = x3;
        }
        __syncthreads();
        if (c == 0) {
            double rdn = 0.0, rpn = a.sc[SC_RP], box = 0.0, cmax = a.sc[SC_CMAX];
            for (int q = 0; q < IPM_T / 32; ++q) {
                rdn = fmax(rdn, red[0][q]);
                rpn = fmax(rpn, red[1][q]);
                box += red[2][q];
                cmax = fmax(cmax, red[3][q]);
            }
            const double mu = (a.sc[SC_SUMSZ] + box) / m_total;
            a.sc[SC_MU] = mu;
            a.sc[SC_RPN] = rpn;
            a.sc[SC_RDN] = rdn;
            const bool conv = rpn <= a.tol && rdn <= a.tol && cmax <= a.tol;
            const bool bad = !(rpn == rpn) || !(rdn == rdn) || !(mu == mu);
            if (conv || bad || a.sc[SC_ITER] >= max_iter) {
                a.sc[SC_DONE] = 1.0;
                a.sc[SC_CONV] = conv ? 1.0 : 0.0;
                a.gate->done = 1;
            }
            a.sc[SC_ABND] = 1e300;
            a.sc[SC_SUMAFF] = 0.0;
            a.sc[SC_BOXAFF] = 0.0;
        }
    } else if (stage == 2) {
        const double du = ipm_solve(a, act ? vv(V_RHS)[c] : 0.0, sh);
        double bnd = 1e300;
        if (act) {
            const double ds1 = -rp1 - du, ds2 = -rp2 + du;
            const double dz1 = -z1 - w1 * ds1, dz2 = -z2 - w2 * ds2;
            vv(V_DU)[c] = du;
            vv(V_DS1)[c] = ds1;
            vv(V_DS2)[c] = ds2;
            vv(V_DZ1)[c] = dz1;
            vv(V_DZ2)[c] = dz2;
            bnd = fmin(fmin(step_bound(s1, ds1), step_bound(s2, ds2)), fmin(step_bound(z1, dz1), step_bound(z2, dz2)));
        }
        block_reduce_to<0>(bnd, &a.sc[SC_ABND]);
    } else if (stage == 3) {
        const double alpha = fmin(1.0, a.sc[SC_ABND]);
        double t = 0.0;
        if (act)
            t = (s1 + alpha * vv(V_DS1)[c]) * (z1 + alpha * vv(V_DZ1)[c]) +
                (s2 + alpha * vv(V_DS2)[c]) * (z2 + alpha * vv(V_DZ2)[c]);
        block_reduce_to<2>(t, &a.sc[SC_BOXAFF]);
        if (c == 0) a.sc[SC_ALPHA] = alpha;
    } else if (stage == 4) {
        if (act) vv(V_CTV)[c] = 0.0;
        if (c == 0) {
            const double mu = a.sc[SC_MU];
            const double mu_aff = (a.sc[SC_SUMAFF] + a.sc[SC_BOXAFF]) / m_total;
            const double r = mu > 0.0 ? fmin(1.0, fmax(0.0, mu_aff / mu)) : 0.0;
            a.sc[SC_SIGMA] = r * r * r;
            a.sc[SC_ABND] = 1e300;
        }
    } else if (stage == 5) {
        const double smu = a.sc[SC_SIGMA] * a.sc[SC_MU];
        double rc1 = 0.0, rc2 = 0.0, rhs = 0.0;
        if (act) {
            rc1 = s1 * z1 + vv(V_DS1)[c] * vv(V_DZ1)[c] - smu;
            rc2 = s2 * z2 + vv(V_DS2)[c] * vv(V_DZ2)[c] - smu;
            rhs = -vv(V_RD)[c] - ((w1 * rp1 - rc1 / s1) - (w2 * rp2 - rc2 / s2)) - vv(V_CTV)[c];
        }
        const double du = ipm_solve(a, rhs, sh);
        double bnd = 1e300;
        if (act) {
            const double ds1 = -rp1 - du, ds2 = -rp2 + du;
            const double dz1 = (-rc1 - z1 * ds1) / s1, dz2 = (-rc2 - z2 * ds2) / s2;
            vv(V_DU)[c] = du;
            vv(V_DS1)[c] = ds1;
            vv(V_DS2)[c] = ds2;
            vv(V_DZ1)[c] = dz1;
            vv(V_DZ2)[c] = dz2;
            bnd = fmin(fmin(step_bound(s1, ds1), step_bound(s2, ds2)), fmin(step_bound(z1, dz1), step_bound(z2, dz2)));
        }
        block_reduce_to<0>(bnd, &a.sc[SC_ABND]);
    } else if (stage == 6) {
        if (c == 0) {
            a.sc[SC_ALPHA] = fmin(1.0, 0.99 * a.sc[SC_ABND]);
            a.sc[SC_SUMSZ] = 0.0;
            a.sc[SC_RP] = 0.0;
            a.sc[SC_CMAX] = 0.0;
        }
    } else if (stage == 7) {
        const double alpha = a.sc[SC_ALPHA];
        if (act) {
            vv(V_U)[c] = U + alpha * vv(V_DU)[c];
            vv(V_S1)[c] = s1 + alpha * vv(V_DS1)[c];
            vv(V_S2)[c] = s2 + alpha * vv(V_DS2)[c];
            vv(V_Z1)[c] = z1 + alpha * vv(V_DZ1)[c];
            vv(V_Z2)[c] = z2 + alpha * vv(V_DZ2)[c];
            vv(V_CTZ)[c] = 0.0;
            vv(V_CTV)[c] = 0.0;
        }
        if (c == 0) a.sc[SC_ITER] += 1.0;
    }
}

// U, the multipliers (box rows first, then the half-space rows in their original scaling:
// y_r = S_r z_r) and the iteration statistics.
__global__ void ipm_final_kernel(IpmArgs a, float* U, float* y, gm_stats* stats) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = a.n;
    if (t < n) {
        U[t] = (float)a.v[(long)V_U * n + t];
        if (y) y[t] = (float)(a.v[(long)V_Z1 * n + t] - a.v[(long)V_Z2 * n + t]);
    } else if (t < n + a.rows) {
        const long r = t - n;
        if (y) y[t] = (float)(a.rw[RA_Z * a.R + r] * a.rs[r]);
    }
    if (t == 0 && stats) {
        stats->iters = (int)a.sc[SC_ITER];
        stats->converged = a.sc[SC_CONV] != 0.0 ? 1 : 0;
        stats->polished = 0;
        stats->r_prim = (float)a.sc[SC_RPN];
        stats->r_dual = (float)a.sc[SC_RDN];
    }
}

gm_status ipm_solve(gm_ctx* c, const float* H, const float* g, const float* Ct, const float* dt, const float* u_lo,
                    const float* u_hi, int max_iter, float* U, float* y, gm_stats* stats, cudaStream_t st) {
    const int n = c->nU;
    const long rows = c->rows_c;
    const int Mnc = std::max(c->M * c->n_c, 1);
    const int sms = std::max(1, c->num_sms);
    IpmArgs a{};
    a.n = n; a.nu = c->nu; a.Mnc = Mnc; a.rows = rows;
    a.H = H; a.g = g; a.Ct = Ct; a.dt = dt; a.lo = u_lo; a.hi = u_hi; a.rs = c->d_rs;
    a.rw = c->d_ipm_rows; a.R = std::max(1L, rows);
    a.v = c->d_ipm_vec; a.sc = c->d_ipm_vec + (long)kIpmVecArrays * n;
    a.Gram = c->d_G; a.Phi = c->d_P; a.Linv = c->d_Linv; a.np = factor_pad(n);
    a.gate = c->d_admm; a.tol = c->s.tol;
    const long long spins = c->s.timeout_spins > 0 ? c->s.timeout_spins : (1LL << 26);
    GM_CUDA_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(int) * 2, st));
    const int g_dot = (int)std::max(1L, std::min((long)cdiv(rows * 32, (long)IPM_T), 8L * sms));
    const int g_T = (int)std::max(1L, std::min((long)cdiv(rows, (long)(IPM_T / 32)), 4L * sms));
    const int g_el = (int)std::max(1L, std::min((long)cdiv(rows, (long)IPM_T), 8L * sms));
    const size_t smem_T = (size_t)(IPM_T / 32) * 2 * n * sizeof(double);
    const int nsplit = gram_split(n, sms, kGramSplitCap, c->gram_tc);
    auto vec = [&](int stage) {
        ipm_vec_kernel<<<1, IPM_T, 0, st>>>(a, stage, max_iter);
        return cudaGetLastError();
    };
    if (rows > 0) {
        row_norm_kernel<<<cdiv(rows * 32, 256), 256, 0, st>>>(rows, c->nu, Mnc, Ct, c->d_rs);
        GM_LAUNCH_CHECK();
    }
    GM_CUDA_TRY(vec(0));
    if (rows > 0) {
        ipm_rowdot_kernel<0><<<g_dot, IPM_T, 0, st>>>(a);
        GM_LAUNCH_CHECK();
    }
    // chunks of two iterations between reads of the done flag
    constexpr int kChunk = 2;
    double done = 0.0;
    for (int it0 = 0; it0 < max_iter && done == 0.0; it0 += kChunk) {
        for (int it = it0; it < std::min(max_iter, it0 + kChunk); ++it) {
            if (rows > 0) {
                ipm_rowT_kernel<0><<<g_T, IPM_T, smem_T, st>>>(a);
                GM_LAUNCH_CHECK();
            }
            GM_CUDA_TRY(vec(1));
            if (rows > 0) {
                GramRows R{Ct, Mnc, c->nu, c->N, reinterpret_cast<const float*>(a.rw + RA_W * a.R), 1, 0};
                GM_TRY(launch_gram(R, n, nsplit, c->d_gram_part, st, c->d_status, c->gram_tc));
                GM_TRY(launch_gram_reduce(n, nsplit, c->d_gram_part, nullptr, 0.f, c->d_G, st));
            }
            ipm_phi_kernel<<<cdiv((long)n * n, 256), 256, 0, st>>>(a);
            GM_LAUNCH_CHECK();
            GM_TRY(factor_pinv(n, c->d_P, c->d_L, c->d_Linv, c->d_Pinv, c->d_status, c->d_admm, c->d_bar, spins,
                               c->s.factor_grid, st));
            GM_CUDA_TRY(vec(2));
            if (rows > 0) {
                ipm_rowdot_kernel<1><<<g_dot, IPM_T, 0, st>>>(a);
                GM_LAUNCH_CHECK();
            }
            GM_CUDA_TRY(vec(3));
            if (rows > 0) {
                ipm_rowelem_kernel<3><<<g_el, IPM_T, 0, st>>>(a);
                GM_LAUNCH_CHECK();
            }
            GM_CUDA_TRY(vec(4));
            if (rows > 0) {
                ipm_rowT_kernel<1><<<g_T, IPM_T, smem_T, st>>>(a);
                GM_LAUNCH_CHECK();
            }
            GM_CUDA_TRY(vec(5));
            if (rows > 0) {
                ipm_rowdot_kernel<2><<<g_dot, IPM_T, 0, st>>>(a);
                GM_LAUNCH_CHECK();
            }
            GM_CUDA_TRY(vec(6));
            if (rows > 0) {
                ipm_rowelem_kernel<4><<<g_el, IPM_T, 0, st>>>(a);
                GM_LAUNCH_CHECK();
            }
            GM_CUDA_TRY(vec(7));
        }
        GM_CUDA_TRY(cudaMemcpyAsync(&done, a.sc + SC_DONE, sizeof(double), cudaMemcpyDeviceToHost, st));
        GM_CUDA_TRY(cudaStreamSynchronize(st));
    }
    ipm_final_kernel<<<cdiv(n + rows, 256), 256, 0, st>>>(a, U, y ? y : c->d_y, stats);
    GM_LAUNCH_CHECK();
    // FP64 KKT certificate of the returned (U, y), as for ADMM
    const float* yk = y ? y : c->d_y;
    GM_CUDA_TRY(cudaMemsetAsync(c->d_kkt, 0, sizeof(double) * (n + 4), st));
    if (rows > 0) {
        const int threads = 256;
        kkt_rows_kernel<<<std::max(1, std::min(4 * sms, (int)cdiv(rows, 8))), threads,
                          (threads / 32) * n * sizeof(double), st>>>(n, c->nu, Mnc, rows, Ct, dt, U, yk, c->d_kkt);
        GM_LAUNCH_CHECK();
    }
    return launch_kkt_final(n, H, g, u_lo, u_hi, U, yk, c->d_kkt, c->d_status, stats, nullptr, st);
}

}  // namespace gmi

using namespace gmi;

extern "C" gm_status gm_qp_solve_ipm(gm_ctx* ctx, const float* H, const float* g, const float* Ct, const float* dt,
                                     const float* u_lo, const float* u_hi, int max_iter, float* U, float* y,
                                     gm_stats* stats, void* stream) {
    clear_error();
    GM_CHECK_ARG(ctx && H && g && u_lo && u_hi && U, "NULL argument");
    GM_CHECK_ARG(ctx->n_c == 0 || (Ct && dt), "Ct/dt are NULL with n_c = %d", ctx->n_c);
    GM_CHECK_ARG(max_iter >= 1 && max_iter <= 1000, "max_iter must be in [1, 1000] (got %d)", max_iter);
    return ipm_solve(ctx, H, g, Ct, dt, u_lo, u_hi, max_iter, U, y, stats ? stats : ctx->d_stats,
                     static_cast<cudaStream_t>(stream));
}
