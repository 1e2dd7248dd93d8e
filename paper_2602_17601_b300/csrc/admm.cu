// ADMM on the condensed QP (Eq. condensed_matrices), with rho adaptation.
//
//   l <= A~ U <= h,  A~ = [I; s .* C~]  (s: optional row scales 1/|C~_r|)
//   U = P(rho)^{-1} (A~'(rho z - y) - g),  P(rho) = H + rho (I + C~' D C~)
//   a = A~ U,  z = clip(a + y/rho, l, h),  y += rho (a - z)
//   r_p = |a - z|_inf,   r_d = |H U + g + A~'y|_inf = rho |A~'(z_prev - z)|_inf
//
// The dual residual uses the identity on the right (it holds for the exact
// U-update; the FP64 KKT check afterwards reports the residual by definition).
//
// Rho adaptation: every adapt_every iterations the ratio of the primal and dual
// residuals, each relative to its scale, gives rho_new = rho sqrt(ratio); a
// change by more than 5x ends the launch with the iterate kept in a device
// state, the next round re-forms and re-factors P(rho_new) in FP64, and the
// next ADMM launch resumes.  A fixed number of rounds is issued; device flags
// make the unneeded ones return at once, so the host never waits.  When the
// step is captured into a graph, rounds after the first sit in nested
// conditional (IF) nodes whose condition a one-thread kernel sets from the
// device state, so the rounds after convergence are not launched at all.
//
// One launch is a persistent cooperative kernel.  Each CTA owns a contiguous
// range of C~ rows, split by cost (16 + row length per row), streams it as
// stage tiles (contiguous rows of one length) into shared memory with
// cp.async double buffering, computes the row dots with lane groups sized to
// the row length, updates z and y, and sums s C~'z and s C~'y by a column
// sweep of the tile.  Block sums go to one of three rotating global
// accumulators; a bounded grid barrier separates iterations.  The box rows
// are evaluated redundantly by every CTA.
#include "admm.h"

#include <type_traits>

namespace gmi {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// wait until at most k (< 4) of this thread's most recent cp.async groups are pending
__device__ __forceinline__ void cp_async_wait_le(int k) {
    if (k <= 0) asm volatile("cp.async.wait_group 0;" ::: "memory");
    else if (k == 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
    else if (k == 2) asm volatile("cp.async.wait_group 2;" ::: "memory");
    else asm volatile("cp.async.wait_group 3;" ::: "memory");
}

__device__ __forceinline__ float wsum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float wmaxf(float v) {
    for (int o = 16; o > 0; o >>= 1) v = nmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// keep_rho: start from the rho the previous solve ended with (a receding-horizon warm start),
// when it is a valid one and that solve succeeded; otherwise rho0.  warm: U0 or y0 are given,
// which turns on the stall test and the cold restart.
__global__ void admm_state_init_kernel(AdmmState* S, float rho0, int keep_rho, int warm) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const float r = S->rho;
        const int prev = S->final_status;
        const bool prev_ok = prev == GM_OK || prev == GM_STALLED;
        S->rho = keep_rho && prev_ok && r >= 1e-6f && r <= 1e6f ? r : rho0;
        S->rho0 = rho0;
        S->need_factor = 1;
        S->done = 0;
        S->started = 0;
        S->iters = 0;
        S->updates = 0;
        S->converged = 0;
        S->rp = S->rd = 0.f;
        S->warm = warm;
        S->cold = 0;
        S->fell_back = 0;
        S->it0 = 0;
        S->stall_ref = -1.f;
    }
}

// P = H + rho (I + G), rho from the state; skipped when no factorisation is due.
__global__ void admm_form_p_kernel(int n, const float* __restrict__ H, const float* __restrict__ G,
                                   const AdmmState* S, float* __restrict__ P) {
    if (S->done || !S->need_factor) return;
    const float rho = S->rho;
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)n * n) return;
    int i = (int)(t / n), j = (int)(t % n);
    float v = H[t] + (G ? rho * G[t] : 0.f);
    if (i == j) v += rho;
    P[t] = v;
}

// Tile of one stage: rows [t0, t0 + tr) of length L, starting at float offset off; live when
// it holds a row that is not redundant (a tile of redundant rows is neither loaded nor passed).
struct Tile {
    long t0, off;
    int tr, L;
    bool live;
};

// Next tile of the row range [r, r1) after a tile ending at row r.
__device__ __forceinline__ Tile next_tile(long r, long r1, int Mnc, int nu, int tile_floats, int tile_rows,
                                          const int* kpos, const int* kcnt) {
    Tile t;
    const int ks = (int)(r / Mnc);
    t.L = (ks + 1) * nu;
    const long stage_end_all = (long)(ks + 1) * Mnc;
    const long stage_end = min(stage_end_all, r1);
    int tr = max(1, tile_floats / t.L);
    tr = min(tr, tile_rows);
    tr = (int)min((long)tr, stage_end - r);
    t.t0 = r;
    t.tr = tr;
    t.off = (long)Mnc * nu * ((long)ks * (ks + 1) / 2) + (r - (long)ks * Mnc) * t.L;
    if (kpos) {
        const long e = r + tr;
        const int p1 = e < stage_end_all ? __ldg(kpos + e) : __ldg(kcnt + ks);
        t.live = p1 > __ldg(kpos + r);
    } else {
        t.live = true;
    }
    return t;
}

// Condition of the IF node around an ADMM round: run it while the solve is not done.
__global__ void admm_round_cond_kernel(const AdmmState* S, cudaGraphConditionalHandle h) {
    cudaGraphSetConditional(h, S->done ? 0u : 1u);
}

template <bool PSMEM>
__global__ void __launch_bounds__(ADMM_T) admm2_kernel(Admm2Args a) {
    extern __shared__ __align__(16) float sm[];
    AdmmState* S = a.S;
    if (S->done) return;                                      // uniform across the grid
    const int n = a.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = ADMM_T / 32;
    // shared layout
    float* sP = sm;                                           // n*n if PSMEM
    float* p = sm + (PSMEM ? n * n : 0);
    float* su = p;          p += n;
    float* srhs = p;        p += n;
    float* zb = p;          p += n;
    float* yb = p;          p += n;
    float* atz = p;         p += n;                           // A~'z of the last pass (box + rows)
    float* aty = p;         p += n;
    float* sdy = p;         p += n;                           // box-row dual step (test iterations)
    float* sacc = p;        p += 3 * n;                       // block sums of s C~'z, s C~'y, s C~'dy
    float* wred = p;        p += 6 * NW;
    p = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15));
    // NB tile buffers: C~ rows staged NB - 1 tiles ahead of the one being processed
    constexpr int NB = PSMEM ? 2 : 3;
    float* tbuf[NB];
    for (int q = 0; q < NB; ++q) {
        tbuf[q] = p;
        p += a.tile_floats;
    }
    float* rstate[NB];                                        // per tile: y, z, d, s (tile_rows each)
    for (int q = 0; q < NB; ++q) {
        rstate[q] = p;
        p += 4 * a.tile_rows;
    }
    float* wz = p;          p += a.tile_rows;                 // s z_r and s y_r of the current tile
    float* wy = p;          p += a.tile_rows;
    float* wd = p;          p += a.tile_rows;                 // s dy_r (test iterations)
    __shared__ float s_misc[8];

    const float* Pinv = a.Pinv;
    if (PSMEM) {
        for (int t = tid; t < n * n; t += ADMM_T) sP[t] = a.Pinv[t];
        Pinv = sP;
    }
    const long r0 = a.row_begin[blockIdx.x], r1 = a.row_begin[blockIdx.x + 1];
    const unsigned G = gridDim.x;
    const int stride = admm_acc_stride(n);
    float rho = S->rho;
    const float inv_rho = 1.f / rho;
    const bool first = !S->started;
    int it = S->iters;
    // the warm inputs, unless a stall or a NaN made this solve restart cold
    const bool cold = S->cold != 0;
    const float* U0 = cold ? nullptr : a.U0;
    const float* y0 = cold ? nullptr : a.y0;
    const bool stall_on = S->warm && !cold;    // the stall test watches warm starts only
    float stall_ref = S->stall_ref;
    const int it0 = S->it0;
    const int updates0 = S->updates;
    for (int c = tid; c < n; c += ADMM_T) {
        if (first) {
            su[c] = U0 ? U0[c] : 0.f;
            yb[c] = y0 ? y0[c] : 0.f;
            // z = clip(U0); a NaN stays NaN (fminf/fmaxf would drop it), so a NaN warm start
            // shows in the first iterate
            zb[c] = su[c] == su[c] ? fminf(fmaxf(su[c], a.lo[c]), a.hi[c]) : su[c];
        } else {
            su[c] = S->u[c];
            zb[c] = S->zb[c];
            yb[c] = S->yb[c];
            atz[c] = S->atz[c];
            aty[c] = S->aty[c];
        }
    }
    __syncthreads();

    // --------------------------------------------------------------- one pass over the CTA's rows
    // init: z = clip(a), y = y0; else the ADMM update.  Adds s C~'z, s C~'y and the maxima
    // (|a - z|, |a|, |z|) into the accumulator accw.  chk (an iteration that tests the
    // infeasibility certificate) also adds s C~'dy, max |dy|, the largest dy of the wrong sign
    // (dy < 0 on a row whose lower bound is -inf) and the support sum d_r max(dy_r, 0).
    auto row_pass = [&](bool init, bool chk, float* accw) {
        const int ns = chk ? 3 * n : 2 * n;
        for (int c = tid; c < ns; c += ADMM_T) sacc[c] = 0.f;
        float rp = 0.f, am = 0.f, zm = 0.f;
        float dym = 0.f, dng = 0.f, dsp = 0.f;
        float pz = 0.f, py = 0.f, pd = 0.f;                    // column-sweep partials
        int cur_L = -1;
        __syncthreads();
        auto issue = [&](const Tile& t, int b) {
            if (!t.live) {                                     // an empty group keeps the count
                cp_async_commit();
                return;
            }
            float* dst = tbuf[b];
            const float* src = a.Ct + t.off;
            const int cnt = t.tr * t.L;
            if (a.vec4) {
                for (int q = tid; q < cnt / 4; q += ADMM_T) cp_async16(dst + 4 * q, src + 4 * q);
            } else {
                for (int q = tid; q < cnt; q += ADMM_T) cp_async4(dst + q, src + q);
            }
            float* rsb = rstate[b];
            for (int i = tid; i < t.tr; i += ADMM_T) {
                const long r = t.t0 + i;
                if (init) {
                    if (y0) cp_async4(rsb + i, y0 + n + r);
                } else {
                    cp_async4(rsb + i, a.y + n + r);
                    cp_async4(rsb + a.tile_rows + i, a.z + n + r);
                }
                cp_async4(rsb + 2 * a.tile_rows + i, a.dt + r);
                if (a.rs) cp_async4(rsb + 3 * a.tile_rows + i, a.rs + r);
            }
            cp_async_commit();
        };
        long rnext = r0;
        Tile q[NB];
        int head = 0, nq = 0;                                  // tiles in flight: slots head .. head+nq-1
        for (int k = 0; k < NB - 1 && rnext < r1; ++k) {
            q[k] = next_tile(rnext, r1, a.Mnc, a.nu, a.tile_floats, a.tile_rows, a.kpos, a.kcnt);
            rnext = q[k].t0 + q[k].tr;
            issue(q[k], k);
            ++nq;
        }
        while (nq > 0) {
            if (rnext < r1 && nq < NB) {
                const int sl = (head + nq) % NB;
                q[sl] = next_tile(rnext, r1, a.Mnc, a.nu, a.tile_floats, a.tile_rows, a.kpos, a.kcnt);
                rnext = q[sl].t0 + q[sl].tr;
                issue(q[sl], sl);
                ++nq;
            }
            cp_async_wait_le(nq - 1);                          // the oldest tile has landed
            __syncthreads();
            const int b = head;
            const Tile cur = q[b];
            if (!cur.live) {                                   // redundant rows only (uniform)
                head = (head + 1) % NB;
                --nq;
                continue;
            }
            const float* T = tbuf[b];
            float* rsb = rstate[b];
            const int L = cur.L, tr = cur.tr;
            // flush the column sweep when the row length changes
            if (L != cur_L) {
                if (cur_L > 0) {
                    const int c = tid % cur_L;
                    if (tid / cur_L < ADMM_T / cur_L) {
                        atomicAdd(&sacc[c], pz);
                        atomicAdd(&sacc[n + c], py);
                        if (chk) atomicAdd(&sacc[2 * n + c], pd);
                    }
                }
                pz = py = pd = 0.f;
                cur_L = L;
            }
            // phase 1: the row dots a_r = C~_r . u, then the row updates (update_row)
            auto update_row = [&](int i, float dot) {
                const float s = a.rs ? rsb[3 * a.tile_rows + i] : 1.f;
                const float av = dot * s;
                const float d = rsb[2 * a.tile_rows + i] * s;
                float yv, zv;
                if (init) {
                    yv = y0 && s > 0.f ? rsb[i] / s : 0.f;          // s = 0: a redundant row
                    zv = fminf(av, d);
                } else {
                    const float yo = rsb[i];
                    zv = fminf(av + yo * inv_rho, d);
                    yv = yo + rho * (av - zv);
                    if (chk) {
                        const float dy = yv - yo;
                        dym = nmaxf(dym, fabsf(dy));
                        if (dy < 0.f) dng = nmaxf(dng, -dy);
                        else if (d < 1e30f) dsp = fmaf(d, dy, dsp);
                        else dng = nmaxf(dng, dy);
                        wd[i] = dy * s;
                    }
                }
                rp = nmaxf(rp, fabsf(av - zv));
                am = nmaxf(am, fabsf(av));
                zm = nmaxf(zm, fabsf(zv));
                rsb[i] = yv;
                rsb[a.tile_rows + i] = zv;
                wz[i] = zv * s;
                wy[i] = yv * s;
            };
            if (L >= 64) {
                // long rows: a warp takes 8 rows at once, lanes along the columns (8 independent
                // accumulators and reductions)
                constexpr int RW = 8;
                for (int i0 = warp * RW; i0 < tr; i0 += NW * RW) {
                    float acc[RW];
#pragma unroll
                    for (int r = 0; r < RW; ++r) acc[r] = 0.f;
                    for (int c = lane; c < L; c += 32) {
                        const float uc = su[c];
#pragma unroll
                        for (int r = 0; r < RW; ++r)
                            if (i0 + r < tr) acc[r] = fmaf(T[(i0 + r) * L + c], uc, acc[r]);
                    }
                    float mine = 0.f;
#pragma unroll
                    for (int r = 0; r < RW; ++r) {
                        const float v = wsum(acc[r]);
                        if (lane == r) mine = v;
                    }
                    if (lane < RW && i0 + lane < tr) update_row(i0 + lane, mine);
                }
            } else {
                // short rows: groups of gs lanes per row
                const int gs = L >= 32 ? 8 : L >= 16 ? 4 : L >= 8 ? 2 : 1;
                const int j = tid & (gs - 1);
                for (int i0 = tid / gs; i0 < ((tr + (ADMM_T / gs) - 1) / (ADMM_T / gs)) * (ADMM_T / gs);
                     i0 += ADMM_T / gs) {
                    const int i = i0;
                    float dot = 0.f;
                    if (i < tr)
                        for (int c = j; c < L; c += gs) dot = fmaf(T[i * L + c], su[c], dot);
                    for (int o = gs >> 1; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
                    if (i < tr && j == 0) update_row(i, dot);
                }
            }
            __syncthreads();
            // write back y, z of the tile; phase 2: column sweep of s C~'z and s C~'y
            for (int i = tid; i < tr; i += ADMM_T) {
                a.y[n + cur.t0 + i] = rsb[i];
                a.z[n + cur.t0 + i] = rsb[a.tile_rows + i];
            }
            auto sweep = [&](auto with_dy) {
                constexpr bool D = decltype(with_dy)::value;
                const int G2 = ADMM_T / L;
                const int c = tid % L, g2 = tid / L;
                if (g2 < G2) {
                    float pz2 = 0.f, py2 = 0.f, pd2 = 0.f;     // a second chain for latency
                    int i = g2;
                    for (; i + G2 < tr; i += 2 * G2) {
                        const float v = T[i * L + c], v2 = T[(i + G2) * L + c];
                        pz = fmaf(v, wz[i], pz);
                        py = fmaf(v, wy[i], py);
                        pz2 = fmaf(v2, wz[i + G2], pz2);
                        py2 = fmaf(v2, wy[i + G2], py2);
                        if (D) {
                            pd = fmaf(v, wd[i], pd);
                            pd2 = fmaf(v2, wd[i + G2], pd2);
                        }
                    }
                    if (i < tr) {
                        const float v = T[i * L + c];
                        pz = fmaf(v, wz[i], pz);
                        py = fmaf(v, wy[i], py);
                        if (D) pd = fmaf(v, wd[i], pd);
                    }
                    pz += pz2;
                    py += py2;
                    if (D) pd += pd2;
                }
            };
            if (chk) sweep(std::true_type{});
            else sweep(std::false_type{});
            __syncthreads();
            head = (head + 1) % NB;
            --nq;
        }
        if (cur_L > 0) {
            const int c = tid % cur_L;
            if (tid / cur_L < ADMM_T / cur_L) {
                atomicAdd(&sacc[c], pz);
                atomicAdd(&sacc[n + c], py);
                if (chk) atomicAdd(&sacc[2 * n + c], pd);
            }
        }
        rp = wmaxf(rp);
        am = wmaxf(am);
        zm = wmaxf(zm);
        if (chk) {
            dym = wmaxf(dym);
            dng = wmaxf(dng);
            dsp = wsum(dsp);
        }
        if (lane == 0) {
            wred[warp] = rp;
            wred[NW + warp] = am;
            wred[2 * NW + warp] = zm;
            wred[3 * NW + warp] = dym;
            wred[4 * NW + warp] = dng;
            wred[5 * NW + warp] = dsp;
        }
        __syncthreads();
        if (r1 > r0)
            for (int c = tid; c < ns; c += ADMM_T) atomicAdd(accw + c, sacc[c]);
        if (tid < (chk ? 5 : 3)) {
            float m = 0.f;
            for (int w = 0; w < NW; ++w) m = nmaxf(m, wred[tid * NW + w]);
            atomicMax(reinterpret_cast<unsigned*>(accw + 3 * n + tid), __float_as_uint(m));
        } else if (chk && tid == 5) {
            float sum = 0.f;
            for (int w = 0; w < NW; ++w) sum += wred[5 * NW + w];
            atomicAdd(accw + 3 * n + 5, sum);
        }
    };

    // read a completed pass: A~'z (box rows added) and the row scalars (max |a - z|, |a|, |z|,
    // |dy|, wrong-sign dy; support sum)
    auto read_pass = [&](const float* accr, float (&v)[6]) {
        for (int c = tid; c < n; c += ADMM_T) {
            srhs[c] = __ldcg(accr + c) + zb[c];               // new A~'z (temporarily in srhs)
        }
        for (int k = 0; k < 5; ++k) v[k] = __uint_as_float(__ldcg(reinterpret_cast<const unsigned*>(accr + 3 * n + k)));
        v[5] = __ldcg(accr + 3 * n + 5);
    };

    unsigned phase = 0;
    int pass = 0;
    bool ok = true, done = false, converged = false, adapt = false, restart = false;
    float rp_last = S->rp, rd_last = S->rd;
    if (first) {
        if (blockIdx.x == 0)
            for (int t = tid; t < stride; t += ADMM_T) a.acc[stride + t] = 0.f;
        row_pass(true, false, a.acc);
        ++phase;
        ok = grid_barrier(a.bar, G, phase, a.max_spins, a.status);
        if (ok) {
            float v[6];
            read_pass(a.acc, v);
            __syncthreads();
            for (int c = tid; c < n; c += ADMM_T) {
                atz[c] = srhs[c];
                aty[c] = __ldcg(a.acc + n + c) + yb[c];
            }
            __syncthreads();
        }
        pass = 1;
    }
    while (ok) {
        // U = P^{-1} (rho A~'z - A~'y - g)
        for (int c = tid; c < n; c += ADMM_T) srhs[c] = rho * atz[c] - aty[c] - a.g[c];
        __syncthreads();
        for (int c = warp; c < n; c += NW) {
            float s = 0.f;
            for (int q = lane; q < n; q += 32) s = fmaf(Pinv[(long)c * n + q], srhs[q], s);
            s = wsum(s);
            if (lane == 0) su[c] = s;
        }
        __syncthreads();
        // this iteration tests the primal-infeasibility certificate (uniform over the grid)
        const bool chk = (it + 1) % kInfeasEvery == 0;
        // box rows
        float rpb = 0.f, amb = 0.f, zmb = 0.f, dyb = 0.f, dnb = 0.f, dsb = 0.f;
        for (int c = tid; c < n; c += ADMM_T) {
            const float av = su[c];
            const float yo = yb[c];
            const float zn = fminf(fmaxf(av + yo / rho, a.lo[c]), a.hi[c]);
            const float yn = yo + rho * (av - zn);
            yb[c] = yn;
            zb[c] = zn;
            rpb = nmaxf(rpb, fabsf(av - zn));
            amb = nmaxf(amb, fabsf(av));
            zmb = nmaxf(zmb, fabsf(zn));
            if (chk) {
                // support of dy over [lo, hi]; an infinite bound takes no dy of its sign
                const float dy = yn - yo;
                sdy[c] = dy;
                dyb = nmaxf(dyb, fabsf(dy));
                if (dy > 0.f) {
                    if (a.hi[c] < 1e30f) dsb = fmaf(a.hi[c], dy, dsb);
                    else dnb = nmaxf(dnb, dy);
                } else if (dy < 0.f) {
                    if (a.lo[c] > -1e30f) dsb = fmaf(a.lo[c], dy, dsb);
                    else dnb = nmaxf(dnb, -dy);
                }
            }
        }
        rpb = wmaxf(rpb);
        amb = wmaxf(amb);
        zmb = wmaxf(zmb);
        if (chk) {
            dyb = wmaxf(dyb);
            dnb = wmaxf(dnb);
            dsb = wsum(dsb);
        }
        if (lane == 0) {
            wred[warp] = rpb;
            wred[NW + warp] = amb;
            wred[2 * NW + warp] = zmb;
            wred[3 * NW + warp] = dyb;
            wred[4 * NW + warp] = dnb;
            wred[5 * NW + warp] = dsb;
        }
        __syncthreads();
        if (tid == 0) {
            float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f, s5 = 0.f;
            for (int w = 0; w < NW; ++w) {
                m0 = nmaxf(m0, wred[w]);
                m1 = nmaxf(m1, wred[NW + w]);
                m2 = nmaxf(m2, wred[2 * NW + w]);
                m3 = nmaxf(m3, wred[3 * NW + w]);
                m4 = nmaxf(m4, wred[4 * NW + w]);
                s5 += wred[5 * NW + w];
            }
            s_misc[0] = m0;
            s_misc[1] = m1;
            s_misc[2] = m2;
            s_misc[3] = m3;
            s_misc[4] = m4;
            s_misc[5] = s5;
        }
        float* accw = a.acc + (pass % 3) * stride;
        if (blockIdx.x == 0)
            for (int t = tid; t < stride; t += ADMM_T) a.acc[((pass + 1) % 3) * stride + t] = 0.f;
        row_pass(false, chk, accw);
        ++phase;
        if (!grid_barrier(a.bar, G, phase, a.max_spins, a.status)) {
            ok = false;
            break;
        }
        ++it;
        float v[6];
        read_pass(accw, v);
        __syncthreads();
        // r_d = rho |A~'z_prev - A~'z|_inf ; new A~'y ; on test iterations |A~'dy|_inf
        float m = 0.f, atd = 0.f;
        for (int c = tid; c < n; c += ADMM_T) {
            m = nmaxf(m, fabsf(srhs[c] - atz[c]));
            atz[c] = srhs[c];
            aty[c] = __ldcg(accw + n + c) + yb[c];
            if (chk) atd = nmaxf(atd, fabsf(__ldcg(accw + 2 * n + c) + sdy[c]));
        }
        m = wmaxf(m);
        if (chk) atd = wmaxf(atd);
        if (lane == 0) {
            wred[3 * NW + warp] = m;
            wred[4 * NW + warp] = atd;
        }
        __syncthreads();
        float mm = 0.f, ad = 0.f;
        for (int w = 0; w < NW; ++w) {
            mm = nmaxf(mm, wred[3 * NW + w]);
            ad = nmaxf(ad, wred[4 * NW + w]);
        }
        const float rp = nmaxf(v[0], s_misc[0]);
        const float rd = rho * mm;
        const float amax = nmaxf(v[1], s_misc[1]);
        const float zmax = nmaxf(v[2], s_misc[2]);
        rp_last = rp;
        rd_last = rd;
        ++pass;
        const bool bad = (rp != rp) || (rd != rd);
        converged = rp <= a.tol && rd <= a.tol;
        // primal infeasibility (Farkas): dy = y - y_prev with |A~'dy| <= eps |dy|, no dy of the
        // sign an infinite bound forbids, and support h'max(dy, 0) + l'min(dy, 0) <= -eps |dy|
        bool infeasible = false;
        if (chk && !converged) {
            const float dmax = nmaxf(v[3], s_misc[3]);
            const float e = kInfeasEps * dmax;
            infeasible = dmax > 0.f && ad <= e && nmaxf(v[4], s_misc[4]) <= e && v[5] + s_misc[5] <= -e;
        }
        if (bad && stall_on) {
            // a NaN warm start: the next launch re-factors P(rho0) and starts cold
            restart = true;
            break;
        }
        if (bad && blockIdx.x == 0 && tid == 0) dev_fail(a.status, GM_ERR_NUMERIC);
        if (infeasible && blockIdx.x == 0 && tid == 0) dev_fail(a.status, GM_ERR_INFEASIBLE);
        if (converged || bad || infeasible || it - it0 >= a.max_iter) {
            done = true;
            break;
        }
        // a warm start may change rho once; a second change waits for the stall test
        const bool may_adapt = !a.last_round && updates0 < kMaxRhoUpdates && !(stall_on && updates0 >= 1);
        if (a.adapt_every > 0 && may_adapt && it % a.adapt_every == 0) {
            // relative residuals: r_p / max(|a|, |z|) against r_d / max(|H U|, |A~'y|, |g|)
            float hu = 0.f, gm = 0.f, ym = 0.f;
            for (int c = warp; c < n; c += NW) {
                float s = 0.f;
                for (int q = lane; q < n; q += 32) s = fmaf(a.H[(long)c * n + q], su[q], s);
                s = wsum(s);
                hu = nmaxf(hu, fabsf(s));
            }
            for (int c = lane; c < n; c += 32) {
                gm = nmaxf(gm, fabsf(a.g[c]));
                ym = nmaxf(ym, fabsf(aty[c]));
            }
            gm = wmaxf(gm);
            ym = wmaxf(ym);
            if (lane == 0) wred[warp] = hu;
            __syncthreads();
            float hm = 0.f;
            for (int w = 0; w < NW; ++w) hm = nmaxf(hm, wred[w]);
            const float ps = fmaxf(fmaxf(amax, zmax), 1e-30f);
            const float ds = fmaxf(fmaxf(hm, fmaxf(ym, gm)), 1e-30f);
            const float ratio = (rp / ps) / fmaxf(rd / ds, 1e-30f);
            float rn = rho * sqrtf(fmaxf(ratio, 0.f));
            rn = fminf(fmaxf(rn, 1e-6f), 1e6f);
            __syncthreads();
            if (rn > 5.f * rho || rn < 0.2f * rho) {
                adapt = true;
                stall_ref = -1.f;                     // the residuals' scale changes: new record
                if (blockIdx.x == 0 && tid == 0) {
                    S->rho = rn;
                    S->updates = S->updates + 1;
                }
                break;
            }
        }
        // stall test of a warm start at iterations where rho did not change (uniform over the
        // grid: every CTA holds the same residuals): max(r_p, r_d) must fall below kStallFactor
        // of its value kStallEvery iterations earlier
        if (stall_on) {
            const float r = fmaxf(rp, rd);
            if (stall_ref < 0.f) {
                stall_ref = r;
            } else if ((it - it0) % kStallEvery == 0) {
                const bool stalled = !(r <= kStallFactor * stall_ref);
                stall_ref = r;
                if (stalled) {
                    // abandon the warm start: the next launch re-factors P(rho0) and starts cold
                    restart = true;
                    break;
                }
            }
        }
    }
    // save the state (CTA 0) / finish
    if (restart) {
        if (blockIdx.x == 0 && tid == 0) {
            S->started = 0;
            S->cold = 1;
            S->fell_back = 1;
            S->rho = S->rho0;
            S->need_factor = 1;
            S->updates = 0;
            S->iters = it;
            S->it0 = it;
            S->converged = 0;
            S->rp = rp_last;
            S->rd = rd_last;
            S->done = 0;
        }
        return;
    }
    if (blockIdx.x == 0) {
        for (int c = tid; c < n; c += ADMM_T) {
            S->u[c] = su[c];
            S->zb[c] = zb[c];
            S->yb[c] = yb[c];
            S->atz[c] = atz[c];
            S->aty[c] = aty[c];
        }
        if (tid == 0) {
            S->iters = it;
            S->started = 1;
            S->rp = rp_last;
            S->rd = rd_last;
            S->converged = converged ? 1 : 0;
            S->need_factor = adapt ? 1 : 0;
            S->done = (done || !ok) ? 1 : 0;
            S->stall_ref = stall_ref;
        }
    }
    if (done || !ok) {
        // rows back to the original scaling: y_r = s_r y'_r, z_r = z'_r / s_r
        if (a.rs)
            for (long r = r0 + tid; r < r1; r += ADMM_T) {
                const float s = a.rs[r];
                a.y[n + r] *= s;
                a.z[n + r] = s > 0.f ? a.z[n + r] / s : 0.f;
            }
        if (blockIdx.x == 0) {
            for (int c = tid; c < n; c += ADMM_T) {
                a.U[c] = su[c];
                a.y[c] = yb[c];
                a.z[c] = zb[c];
            }
            if (tid == 0 && a.stats) {
                a.stats->iters = it;
                a.stats->converged = (converged && ok) ? 1 : 0;
                a.stats->r_prim = rp_last;
                a.stats->r_dual = rd_last;
                a.stats->polished = 0;
            }
        }
    }
}

// C~ rows split over `grid` CTAs by cost 16 + row length: boundary b is the first row
// count whose cumulative cost reaches b/grid of the total (stage-major rows, so the
// cumulative cost is piecewise linear; one thread per boundary).
__global__ void admm_partition_kernel(long rows, int nu, int Mnc, int grid, int* rb) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > grid) return;
    const int N = (int)(rows / Mnc);
    double total = 0.0;
    for (int k = 0; k < N; ++k) total += (double)Mnc * (16.0 + (double)(k + 1) * nu);
    if (b == 0) { rb[0] = 0; return; }
    if (b == grid) { rb[grid] = (int)rows; return; }
    const double target = total * b / grid;
    double cum = 0.0;
    long m = rows;
    for (int k = 0; k < N; ++k) {
        const double per = 16.0 + (double)(k + 1) * nu;
        if (cum + Mnc * per >= target) {
            long j = (long)ceil((target - cum) / per);
            j = j < 1 ? 1 : (j > Mnc ? Mnc : j);
            m = (long)k * Mnc + j;
            break;
        }
        cum += Mnc * per;
    }
    rb[b] = (int)m;
}

static size_t admm2_smem(int n, bool psmem, int tile_floats, int tile_rows) {
    const size_t nb = psmem ? 2 : 3;
    size_t f = (psmem ? (size_t)n * n : 0) + 10 * (size_t)n + 6 * (ADMM_T / 32) + 4 + 4;
    f += nb * (size_t)tile_floats + nb * 4 * (size_t)tile_rows + 3 * (size_t)tile_rows;
    return f * sizeof(float);
}

// Layout: P^{-1} in shared memory with two 8192-float tiles, or P^{-1} read from L2 with three
// larger tiles (the row pass then keeps two tiles in flight).
bool admm2_psmem(int n) {
    return kAdmmPinvShared && admm2_smem(n, true, kAdmmTileFloats, kAdmmTileRows) <= 220 * 1024;
}

static int admm2_tile_floats(int n) { return admm2_psmem(n) ? kAdmmTileFloats : kAdmmTileFloatsL2; }

size_t admm2_smem_bytes(int n) { return admm2_smem(n, admm2_psmem(n), admm2_tile_floats(n), kAdmmTileRows); }

const void* admm2_kernel_ptr(int n) {
    return admm2_psmem(n) ? (const void*)admm2_kernel<true> : (const void*)admm2_kernel<false>;
}

gm_status admm_solve(const AdmmPlan& p) {
    cudaStream_t st = p.st;
    const int n = p.n;
    admm_state_init_kernel<<<1, 32, 0, st>>>(p.S, p.rho0, p.keep_rho ? 1 : 0, p.warm ? 1 : 0);
    GM_LAUNCH_CHECK();
    admm_partition_kernel<<<cdiv(p.grid + 1, 128), 128, 0, st>>>(p.rows, p.nu, std::max(p.Mnc, 1), p.grid,
                                                                 p.row_begin);
    GM_LAUNCH_CHECK();
    Admm2Args a{};
    a.n = n; a.nu = p.nu; a.Mnc = std::max(p.Mnc, 1); a.rows = p.rows;
    a.Ct = p.Ct; a.dt = p.dt; a.lo = p.lo; a.hi = p.hi; a.g = p.g; a.H = p.H; a.Pinv = p.Pinv;
    a.rs = p.rs; a.U0 = p.U0; a.y0 = p.y0; a.U = p.U; a.y = p.y; a.z = p.z; a.acc = p.acc;
    a.kpos = p.rows > 0 ? p.kpos : nullptr; a.kcnt = p.rows > 0 ? p.kcnt : nullptr;
    a.bar = p.bar; a.status = p.status; a.row_begin = p.row_begin; a.S = p.S; a.stats = p.stats;
    a.tol = p.tol; a.max_iter = p.max_iter; a.adapt_every = p.adapt_every; a.max_spins = p.max_spins;
    a.tile_floats = admm2_tile_floats(n);
    a.tile_rows = kAdmmTileRows;
    a.vec4 = (p.nu % 4 == 0) && ((reinterpret_cast<uintptr_t>(p.Ct) & 15) == 0);
    const bool psmem = admm2_psmem(n);
    const size_t smem = admm2_smem_bytes(n);
    GM_CUDA_TRY(cudaFuncSetAttribute(admm2_kernel_ptr(n), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // one round on stream rs: re-form and re-factor P when due, then an ADMM launch
    auto round = [&](int r, cudaStream_t rs) -> gm_status {
        admm_form_p_kernel<<<cdiv((long)n * n, 256), 256, 0, rs>>>(n, p.H, p.Gram, p.S, p.P);
        GM_LAUNCH_CHECK();
        GM_TRY(factor_pinv(n, p.P, p.L, p.Linv, p.Pinv, p.status, p.S, p.bar, p.max_spins, p.factor_grid, rs));
        if (r == 0 && p.ev_mid) GM_CUDA_TRY(cudaEventRecord(p.ev_mid, rs));
        GM_CUDA_TRY(cudaMemsetAsync(p.bar, 0, sizeof(unsigned) * 4, rs));
        GM_CUDA_TRY(cudaMemsetAsync(p.acc, 0, sizeof(float) * admm_acc_stride(n), rs));
        a.last_round = (r == p.rounds - 1) ? 1 : 0;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(p.grid);
        cfg.blockDim = dim3(ADMM_T);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = rs;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (psmem) {
            GM_CUDA_TRY(cudaLaunchKernelEx(&cfg, admm2_kernel<true>, a));
        } else {
            GM_CUDA_TRY(cudaLaunchKernelEx(&cfg, admm2_kernel<false>, a));
        }
        GM_LAUNCH_CHECK();
        return GM_OK;
    };
    bool cond = false;
    if (p.body_st && kAdmmCondRounds) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        GM_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
        cond = cs == cudaStreamCaptureStatusActive;
    }
    // Rounds after the first are nested IF nodes: the body of round r's node holds round r, the
    // condition kernel of round r + 1 and round r + 1's node, so the first false condition skips
    // every later round.  Each body is captured on body_st once the enclosing one is complete.
    cudaStream_t cap = st;                        // the stream whose capture takes the next IF node
    auto add_if = [&](int r) -> gm_status {
        cudaStreamCaptureStatus cs;
        cudaGraph_t g = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        const cudaGraphEdgeData* edges = nullptr;
        size_t nd = 0;
        GM_CUDA_TRY(cudaStreamGetCaptureInfo(cap, &cs, nullptr, &g, nullptr, nullptr, nullptr));
        cudaGraphConditionalHandle h;
        GM_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
        admm_round_cond_kernel<<<1, 1, 0, cap>>>(p.S, h);
        GM_LAUNCH_CHECK();
        GM_CUDA_TRY(cudaStreamGetCaptureInfo(cap, &cs, nullptr, &g, &deps, &edges, &nd));
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeIf;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        GM_CUDA_TRY(cudaGraphAddNode(&node, g, deps, edges, nd, &np));
        GM_CUDA_TRY(cudaStreamUpdateCaptureDependencies(cap, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
        if (cap != st) {                          // the enclosing body is complete
            cudaGraph_t bg = nullptr;
            cap = st;
            GM_CUDA_TRY(cudaStreamEndCapture(p.body_st, &bg));
        }
        GM_CUDA_TRY(cudaStreamBeginCaptureToGraph(p.body_st, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeRelaxed));
        cap = p.body_st;
        return round(r, p.body_st);
    };
    gm_status rs = GM_OK;
    for (int r = 0; r < p.rounds && rs == GM_OK; ++r) rs = (!cond || r == 0) ? round(r, st) : add_if(r);
    if (cap != st) {                              // close the innermost body, also after an error
        cudaGraph_t bg = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(p.body_st, &bg);
        if (rs == GM_OK && ce != cudaSuccess) GM_CUDA_TRY(ce);
    }
    GM_TRY(rs);
    return GM_OK;
}

}  // namespace gmi
