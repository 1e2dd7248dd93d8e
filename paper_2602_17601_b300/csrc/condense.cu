// Condensing (Thm. 1 proof): per-node recursion for Gamma_u^i, Gamma_x^i
// (Eq. sparse_gamma_i_u, Eq. sparse_gamma_i_xb), per-node aggregation of H
// and g (Eq. H, Eq. g) and the stacked constraint rows C~^i, d~^i.  FP32.
//
// Gamma_u is kept stage-major and packed: stage k (1..N) holds, for every node
// i and state component a, the k nu non-zero columns of block row k of
// Gamma_u^i.  Stage k reads stage k-1 of the nodes in the K-hop neighbourhood
// of i only, so one stage costs O(M) (Thm. 1).
#include "ctx.h"
#include "ff.cuh"
#include "kernels.h"

namespace gmi {

__global__ void sphere_kernel(int N, int M, int S, const float* __restrict__ x_hat,
                              const float* __restrict__ spheres, float* __restrict__ Cx,
                              float* __restrict__ dx) {
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)N * M * S) return;
    int s = (int)(t % S);
    long ki = t / S;
    int i = (int)(ki % M);
    int k = (int)(ki / M) + 1;                 // stages 1..N
    const float* p = x_hat + ((long)k * M + i) * 6;
    float ox = spheres[s * 4 + 0], oy = spheres[s * 4 + 1], oz = spheres[s * 4 + 2];
    float r = spheres[s * 4 + 3];
    float dxv = p[0] - ox, dyv = p[1] - oy, dzv = p[2] - oz;
    float nrm = sqrtf(dxv * dxv + dyv * dyv + dzv * dzv);
    float nx = 0.f, ny = 0.f, nz = 1.f;
    if (nrm > 0.f) {
        nx = dxv / nrm; ny = dyv / nrm; nz = dzv / nrm;
    }
    // keep p on the far side of the tangent plane: -n'p <= -r - n'o
    Cx[t * 3 + 0] = -nx;
    Cx[t * 3 + 1] = -ny;
    Cx[t * 3 + 2] = -nz;
    dx[t] = -r - (nx * ox + ny * oy + nz * oz);
}

gm_status sphere_halfspaces(gm_ctx* c, const float* x_hat, const float* spheres, int S, float* Cx,
                            float* dx, cudaStream_t st) {
    long n = (long)c->N * c->M * S;
    if (n == 0) return GM_OK;
    sphere_kernel<<<cdiv(n, 256), 256, 0, st>>>(c->N, c->M, S, x_hat, spheres, Cx, dx);
    GM_LAUNCH_CHECK();
    return GM_OK;
}


// Gamma_x is kept as its offset from the rollout, D_k = Gamma_x_k - x_hat_k (D_0 = 0), which
// follows the recursion of Eq. sparse_gamma_i_xb with c substituted:
//   D_{k+1} = sum_j A^{ij}_k D^j_k + e^i_k,   e^i_k = c^i_k - x_hat^i_{k+1} + sum_j A^{ij}_k x_hat^j_k
// (e = -B u_hat in exact arithmetic).  Gamma_x holds absolute positions of order one while the
// quantities that use it (Gamma_x - x_ref, the clearance d - C Gamma_x) are small, so the FP32
// recursion on Gamma_x itself would lose their low bits to cancellation; e is summed in
// float-float pairs and D stays small.  One warp per (stage, node), lanes over the blocks'
// (j, t) columns.
__global__ void defect_kernel(int N, int M, const int* __restrict__ row_ptr, const int* __restrict__ col,
                              long nnzb, const float* __restrict__ A, const float* __restrict__ cvec,
                              const float* __restrict__ x_hat, float* __restrict__ e) {
    const long w = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= (long)N * M) return;
    const int k = (int)(w / M), i = (int)(w % M);
    const float* xk = x_hat + (long)k * M * 6;
    const float* Ak = A + (long)k * nnzb * 36;
    const int b0 = row_ptr[i], nb = row_ptr[i + 1] - b0;
    FF s[6];
    for (int q = lane; q < nb * 6; q += 32) {
        const int b = q / 6, t = q % 6;
        const float x = xk[(long)col[b0 + b] * 6 + t];
        const float* Ab = Ak + (long)(b0 + b) * 36 + t;
#pragma unroll
        for (int a = 0; a < 6; ++a) ff_add_prod(s[a], Ab[a * 6], x);
    }
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        FF t = ff_warp_sum(s[a]);
        if (lane == 0) {
            ff_add(t, cvec[((long)k * M + i) * 6 + a]);
            ff_add(t, -x_hat[((long)(k + 1) * M + i) * 6 + a]);
            e[((long)k * M + i) * 6 + a] = ff_value(t);
        }
    }
}

// Stage k -> k+1 for one node per block:
//   (Gamma_u^i)_{k+1} last block row = [sum_j A^{ij}_k (Gamma_u^j)_k last row , B^i_k]
//   D^i_{k+1}                         =  sum_j A^{ij}_k D^j_k + e^i_k     (see defect_kernel)
__global__ void recursion_kernel(int k, int M, int nu, const int* __restrict__ row_ptr,
                                 const int* __restrict__ col, const float* __restrict__ A,
                                 const float* __restrict__ B, const float* __restrict__ ek,
                                 const float* __restrict__ Gu_k, const float* __restrict__ Gx_k,
                                 float* __restrict__ Gu_k1, float* __restrict__ Gx_k1) {
    extern __shared__ float sA[];
    const int i = blockIdx.x;
    const int b0 = row_ptr[i], nb = row_ptr[i + 1] - b0;
    int* sj = reinterpret_cast<int*>(sA + nb * 36);
    for (int t = threadIdx.x; t < nb * 36; t += blockDim.x) sA[t] = A[(long)b0 * 36 + t];
    for (int t = threadIdx.x; t < nb; t += blockDim.x) sj[t] = col[b0 + t];
    __syncthreads();
    const int Lk = k * nu, Lk1 = (k + 1) * nu;
    for (int cc = threadIdx.x; cc <= Lk1; cc += blockDim.x) {
        float o[6] = {0, 0, 0, 0, 0, 0};
        if (cc < Lk) {
            for (int b = 0; b < nb; ++b) {
                const int j = sj[b];
#pragma unroll
                for (int t = 0; t < 6; ++t) {
                    const float s = Gu_k[((long)j * 6 + t) * Lk + cc];
#pragma unroll
                    for (int a = 0; a < 6; ++a) o[a] = fmaf(sA[b * 36 + a * 6 + t], s, o[a]);
                }
            }
#pragma unroll
            for (int a = 0; a < 6; ++a) Gu_k1[((long)i * 6 + a) * Lk1 + cc] = o[a];
        } else if (cc < Lk1) {
#pragma unroll
            for (int a = 0; a < 6; ++a)
                Gu_k1[((long)i * 6 + a) * Lk1 + cc] = B[((long)i * 6 + a) * nu + (cc - Lk)];
        } else {
#pragma unroll
            for (int a = 0; a < 6; ++a) o[a] = ek[(long)i * 6 + a];
            for (int b = 0; b < nb; ++b) {
                const int j = sj[b];
#pragma unroll
                for (int t = 0; t < 6; ++t) {
                    const float s = Gx_k[(long)j * 6 + t];
#pragma unroll
                    for (int a = 0; a < 6; ++a) o[a] = fmaf(sA[b * 36 + a * 6 + t], s, o[a]);
                }
            }
#pragma unroll
            for (int a = 0; a < 6; ++a) Gx_k1[(long)i * 6 + a] = o[a];
        }
    }
}

// Partial sums of G = sum_r w_r x_r x_r' over one share of every stage's rows: CTA
// (block, sp) computes the 64 x 64 block (I, J), I >= J, over split sp, and stores it as
// the four 32 x 32 tiles (ti, tj) of part[sp] (tiles past the matrix edge are skipped).
// Rows of stage k have length k nu, so stages with k nu <= 64 I add nothing to row block I.
// 16 x 16 threads, 4 x 4 outputs each; 16 rows of both column blocks staged per step.
__global__ void __launch_bounds__(256) gram_kernel(GramRows R, int n, float* __restrict__ part) {
    const int T = (n + 31) / 32;
    int lt = blockIdx.x, I = 0;
    while (lt > I) { lt -= I + 1; ++I; }
    const int J = lt;
    const int nsplit = gridDim.y, sp = blockIdx.y;
    __shared__ __align__(16) float X1[16][64];
    __shared__ __align__(16) float X2[16][64];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    const int c1b = I * 64, c2b = J * 64;
    const int kmin = c1b / R.nu + 1;
    for (int k = kmin; k <= R.N; ++k) {
        const int L = k * R.nu;
        const long base = (long)R.rows_per_stage * R.nu * ((long)k * (k - 1) / 2);
        const int per = (R.rows_per_stage + nsplit - 1) / nsplit;
        const int r0 = sp * per, r1 = min(R.rows_per_stage, r0 + per);
        for (int rb = r0; rb < r1; rb += 16) {
            for (int t = tid; t < 16 * 64; t += 256) {
                const int rr = t >> 6, cc = t & 63;
                const int r = rb + rr;
                float w = 0.f, v1 = 0.f, v2 = 0.f;
                if (r < r1) {
                    w = R.wts ? R.wts[(long)(k - R.wts_k0) * R.rows_per_stage + r] : 1.f;
                    if (R.wts_square) w *= w;
                    const float* xr = R.X + base + (long)r * L;
                    if (c1b + cc < L) v1 = xr[c1b + cc];
                    if (c2b + cc < L) v2 = xr[c2b + cc];
                }
                X1[rr][cc] = v1 * w;
                X2[rr][cc] = v2;
            }
            __syncthreads();
#pragma unroll
            for (int rr = 0; rr < 16; ++rr) {
                const float4 a = *reinterpret_cast<const float4*>(&X1[rr][ty * 4]);
                const float4 b = *reinterpret_cast<const float4*>(&X2[rr][tx * 4]);
                const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c1 = c1b + ty * 4 + i, c2 = c2b + tx * 4 + j;
            const int ti = c1 >> 5, tj = c2 >> 5;
            if (ti < T && tj < T) part[(((long)sp * T + ti) * T + tj) * 1024 + (c1 & 31) * 32 + (c2 & 31)] = acc[i][j];
        }
}

int gram_blocks(int n) {
    const int T64 = (n + 63) / 64;
    return T64 * (T64 + 1) / 2;
}

int gram_split(int n, int sms, int cap, bool tc) {
    if (tc && gram_tc_ok(n)) return std::max(1, std::min(cap, sms));
    return std::max(1, std::min(cap, (2 * sms) / gram_blocks(n)));
}

gm_status launch_gram(const GramRows& R, int n, int nsplit, float* part, cudaStream_t st, int* status, bool tc) {
    if (tc && gram_tc_ok(n)) return launch_gram_tc(R, n, nsplit, part, status, st);
    gram_kernel<<<dim3(gram_blocks(n), nsplit), 256, 0, st>>>(R, n, part);
    GM_LAUNCH_CHECK();
    return GM_OK;
}

// G = the sum of the nsplit partial Grams (tile layout [nsplit][T][T][32 x 32], T = ceil(n/32)), plus
// diag_scale * diag_add on the diagonal.  Only lower-triangle elements are read and each is written
// to both halves, so G is exactly symmetric.  Block (lower tile (ti, tj), row r of the tile): lane l
// takes element (32 ti + r, 32 tj + l); the 8 warps take every 8th share, so each warp load is one
// 128-byte line and about 19 loads per thread are in flight in a few round trips; the 8 partial sums
// meet in shared memory in a fixed order.
__global__ void __launch_bounds__(GR_WARPS * 32) gram_reduce_kernel(int n, int nsplit, const float* __restrict__ part,
                                                                    const float* __restrict__ diag_add,
                                                                    float diag_scale, float* __restrict__ G) {
    __shared__ float red[GR_WARPS][32];
    const int T = (n + 31) / 32;
    const int tile = blockIdx.x / 32, r = blockIdx.x % 32;
    int ti = (int)((sqrtf(8.f * (float)tile + 1.f) - 1.f) * 0.5f);
    while ((ti + 1) * (ti + 2) / 2 <= tile) ++ti;
    while (ti * (ti + 1) / 2 > tile) --ti;
    const int tj = tile - ti * (ti + 1) / 2;                 // tj <= ti
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long base = ((long)ti * T + tj) * 1024 + r * 32 + lane, stride = (long)T * T * 1024;
    float s0 = 0.f, s1 = 0.f;
    int sp = warp;
#pragma unroll 4
    for (; sp + GR_WARPS < nsplit; sp += 2 * GR_WARPS) {
        s0 += part[base + (long)sp * stride];
        s1 += part[base + (long)(sp + GR_WARPS) * stride];
    }
    if (sp < nsplit) s0 += part[base + (long)sp * stride];
    red[warp][lane] = s0 + s1;
    __syncthreads();
    if (warp == 0) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < GR_WARPS; ++w) s += red[w][lane];
        const int a = 32 * ti + r, b = 32 * tj + lane;
        if (a < n && b <= a) {
            if (a == b && diag_add) s += diag_scale * diag_add[a];
            G[(long)a * n + b] = s;
            G[(long)b * n + a] = s;
        }
    }
}

gm_status launch_gram_reduce(int n, int nsplit, const float* part, const float* diag_add, float diag_scale, float* G,
                             cudaStream_t st) {
    const int T = (n + 31) / 32;
    gram_reduce_kernel<<<T * (T + 1) / 2 * 32, GR_WARPS * 32, 0, st>>>(n, nsplit, part, diag_add, diag_scale, G);
    GM_LAUNCH_CHECK();
    return GM_OK;
}

gm_status gram(gm_ctx* c, const GramRows& R, int nsplit, const float* diag_add, float diag_scale,
               float* G, cudaStream_t st) {
    const int n = c->nU;
    GM_TRY(launch_gram(R, n, nsplit, c->d_gram_part, st, c->d_status, c->gram_tc));
    return launch_gram_reduce(n, nsplit, c->d_gram_part, diag_add, diag_scale, G, st);
}

// g = -Rbar u_ref + sum_k sum_{i,a} Gu_k[i,a]^T Q^i_k[a] (Gx_k[i,a] - x_ref_k[i,a]),
// with Gx - x_ref = (x_hat - x_ref) + D (D = Gamma_x - x_hat, see recursion_kernel)
__global__ void grad_kernel(int n, int M, int nu, int N, const float* __restrict__ Gu,
                            const float* __restrict__ Gx, const float* __restrict__ xh,
                            const float* __restrict__ Q, const float* __restrict__ xr,
                            float* __restrict__ part) {
    const int sp = blockIdx.x, nsplit = gridDim.x;
    const int rows = M * 6;
    for (int cc = threadIdx.x; cc < n; cc += blockDim.x) {
        float acc = 0.f;
        const int kmin = cc / nu + 1;
        for (int k = kmin; k <= N; ++k) {
            const int L = k * nu;
            const long base = gu_offset(M, nu, k);
            const int per = (rows + nsplit - 1) / nsplit;
            const int r0 = sp * per, r1 = min(rows, r0 + per);
            for (int r = r0; r < r1; ++r) {
                const long qi = (long)k * rows + r;
                const float w = Q[qi] * ((xh[qi] - xr[qi]) + Gx[qi]);
                if (w != 0.f) acc = fmaf(Gu[base + (long)r * L + cc], w, acc);
            }
        }
        part[(long)sp * n + cc] = acc;
    }
}

// one warp per entry: the lanes stride over the partial sums, then a shuffle tree
__global__ void grad_reduce_kernel(int n, int nsplit, const float* __restrict__ part,
                                   const float* __restrict__ Rd, const float* __restrict__ ur,
                                   float* __restrict__ g) {
    const int cc = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (cc >= n) return;
    float s = 0.f;
    for (int sp = lane; sp < nsplit; sp += 32) s += part[(long)sp * n + cc];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) g[cc] = s - Rd[cc] * ur[cc];
}

// C~ row (k, i, c) = C^{x,i}_k[c] . Gamma_u^i position rows of stage k; d~ = d - C . Gamma_x position
// = (d - C . x_hat position) - C . D position (D = Gamma_x - x_hat).  One warp per (k, i).
__global__ void constraint_kernel(int N, int M, int nu, int n_c, const float* __restrict__ Gu,
                                  const float* __restrict__ Gx, const float* __restrict__ xh,
                                  const float* __restrict__ Cx, const float* __restrict__ dx,
                                  float* __restrict__ Ct, float* __restrict__ dt) {
    const long w = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= (long)N * M) return;
    const int k = (int)(w / M) + 1, i = (int)(w % M);
    const int L = k * nu;
    const float* g0 = Gu + gu_offset(M, nu, k) + (long)i * 6 * L;
    const long cbase = (long)M * n_c * nu * ((long)k * (k - 1) / 2);
    for (int cc = 0; cc < n_c; ++cc) {
        const long crow = (((long)(k - 1) * M + i) * n_c + cc);
        const float a0 = Cx[crow * 3 + 0], a1 = Cx[crow * 3 + 1], a2 = Cx[crow * 3 + 2];
        float* out = Ct + cbase + (long)(i * n_c + cc) * L;
        for (int col = lane; col < L; col += 32)
            out[col] = a0 * g0[col] + a1 * g0[L + col] + a2 * g0[2 * L + col];
        if (lane == 0) {
            const float* gx = Gx + ((long)k * M + i) * 6;
            const float* xp = xh + ((long)k * M + i) * 6;
            dt[crow] = (dx[crow] - (a0 * xp[0] + a1 * xp[1] + a2 * xp[2])) - (a0 * gx[0] + a1 * gx[1] + a2 * gx[2]);
        }
    }
}

gm_status condense(gm_ctx* c, const float* x_hat, const float* A, const float* B, const float* cvec,
                   const gm_cost* cost, const float* Cx, const float* dx, float* H, float* g,
                   float* Ct, float* dt, cudaStream_t st) {
    const int M = c->M, nu = c->nu, N = c->N;
    // Gamma_x stage 0 is the measured state x_hat_0: offset D_0 = 0
    GM_CUDA_TRY(cudaMemsetAsync(c->d_Gx, 0, sizeof(float) * M * 6, st));
    int maxnb = 0;
    for (int i = 0; i < M; ++i) maxnb = std::max(maxnb, c->jac_row_ptr[i + 1] - c->jac_row_ptr[i]);
    const size_t smem = (size_t)maxnb * 36 * sizeof(float) + (size_t)maxnb * sizeof(int);
    {
        const long warps = (long)N * M;
        defect_kernel<<<cdiv(warps * 32, 256), 256, 0, st>>>(N, M, c->dc.nr_ptr_K, c->d_jac_col, c->nnzb, A, cvec,
                                                            x_hat, c->d_defect);
        GM_LAUNCH_CHECK();
    }
    for (int k = 0; k < N; ++k) {
        const float* Guk = k > 0 ? c->d_Gu + gu_offset(M, nu, k) : nullptr;
        recursion_kernel<<<M, 128, smem, st>>>(
            k, M, nu, c->dc.nr_ptr_K, c->d_jac_col, A + (long)k * c->nnzb * 36,
            B + (long)k * M * 6 * nu, c->d_defect + (long)k * M * 6, Guk, c->d_Gx + (long)k * M * 6,
            c->d_Gu + gu_offset(M, nu, k + 1), c->d_Gx + (long)(k + 1) * M * 6);
        GM_LAUNCH_CHECK();
    }
    return condense_tail(c, x_hat, cost, Cx, dx, H, g, Ct, dt, st);
}

gm_status condense_tail(gm_ctx* c, const float* x_hat, const gm_cost* cost, const float* Cx, const float* dx,
                        float* H, float* g, float* Ct, float* dt, cudaStream_t st) {
    const int M = c->M, nu = c->nu, N = c->N;
    // Eq. H: sum of per-node local Hessians + Rbar
    GramRows R{c->d_Gu, M * 6, nu, N, cost->Qdiag, 0, 0};
    GM_TRY(gram(c, R, gram_split(c->nU, c->num_sms, kGramSplitCap, c->gram_tc), cost->Rdiag, 1.f, H, st));
    // Eq. g
    const int gsplit = std::max(1, std::min(4 * c->num_sms, M * 6 / 8));
    grad_kernel<<<gsplit, 256, 0, st>>>(c->nU, M, nu, N, c->d_Gu, c->d_Gx, x_hat, cost->Qdiag, cost->x_ref,
                                       c->d_gram_part);
    GM_LAUNCH_CHECK();
    grad_reduce_kernel<<<cdiv((long)c->nU * 32, 256), 256, 0, st>>>(c->nU, gsplit, c->d_gram_part, cost->Rdiag,
                                                                    cost->u_ref, g);
    GM_LAUNCH_CHECK();
    // stacked constraints
    if (c->n_c > 0) {
        const long warps = (long)N * M;
        constraint_kernel<<<cdiv(warps * 32, 256), 256, 0, st>>>(N, M, nu, c->n_c, c->d_Gu, c->d_Gx, x_hat,
                                                                Cx, dx, Ct, dt);
        GM_LAUNCH_CHECK();
    }
    return GM_OK;
}

}  // namespace gmi
