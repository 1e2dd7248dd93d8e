// Tensor-core (tcgen05) form of the fused 2-layer MLP kernel: BF16 operands,
// FP32 accumulation in tensor memory.  Same Op functors as mlp2_kernel.
//
//   GEMM1  D1[128 x W]    = X[128 x Kin] . B1       (K in staged chunks)
//   hidden                = relu(D1 + b1) (mask bits saved) or D1 * saved mask
//   GEMM2  D2[128 x Nout] = hid . B2                (K = W in staged chunks)
//   out(row, n, D2 + b2)
//
// P pieces per operand trade tensor work for accuracy with BF16 tensor cores:
// x = x0 + x1 + ... with x0 = bf16(x), x1 = bf16(x - x0), ..., and
// D = sum over i + j < P of A_i B_j.  P = 1: plain BF16 (8 bits).  P = 2: three
// products, about 16 bits.  P = 3: six products, about 24 bits, i.e. FP32
// operand precision (the dropped pairs lie below the last piece's rounding).
//
// Operands are staged in shared memory by the threads in the canonical
// no-swizzle K-major layout of core matrices (8 rows x 16 bytes): element
// (r, k) of a tile with K columns sits at (r/8)*16K + (k/8)*128 + (r%8)*16 +
// (k%8)*2 bytes, so a 16-wide K step of one MMA is 256 bytes further on and
// the descriptor strides are LBO = 128 bytes (next core matrix along K) and
// SBO = 16K bytes (next 8-row group).  One thread issues the MMAs and commits
// them to an mbarrier; every wait is bounded and records GM_ERR_TIMEOUT.
#pragma once

#include <cuda_bf16.h>

#include "tc_prim.cuh"

namespace gmi {

constexpr int TC_T = 512;        // threads per CTA: four warp groups
constexpr int TC_TMEM_COLS = 256;  // D1, then D2 in the same columns (N <= 256); two CTAs per SM
constexpr int TC_NB = 128;         // rows of the staged B chunk

// Operand pointers of one launch: K-major BF16 copies [Npad][Kpad] of the two products,
// one array per piece (only the first P are read).
struct TcW {
    const __nv_bfloat16* B1[3];  // [W][K1p]
    const __nv_bfloat16* B2[3];  // [N2p][W]  (unused in single-product mode)
    int K1p, N2p;
    int* status;
    // 1: let the next kernel of the stream start its prologue as soon as every CTA of this one
    // has started (programmatic dependent launch), not when each finishes
    int early;
    // single-product form: output columns of the product (0: W; 2W: two halves of W rows of B1,
    // each chunk of B1 holding both halves, written to tensor-memory columns 0.. and W..)
    int N1p;
};

template <class Op>
__device__ __forceinline__ void tc_load8(const Op& op, const RowCtx& rc, int k0, float* v) {
    if constexpr (Op::kHasIn8) {
        op.in8(rc, k0, v);
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = (k0 + j < op.kin) ? op.in(rc, k0 + j) : 0.f;
    }
}

// Output of 32 columns [c0, c0 + 32) of one row: value = product (+ bias), plus the op's
// residual where it has one.  Residual loads are all issued before the first store.
template <class Op>
__device__ __forceinline__ void tc_out32(const Op& op, const RowCtx& rc, int c0, const float* v, int nout,
                                         const float* bias) {
    float4 f[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int n = c0 + 4 * q;
        f[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        if (bias && n + 3 < nout) {
            f[q].x += bias[n]; f[q].y += bias[n + 1]; f[q].z += bias[n + 2]; f[q].w += bias[n + 3];
        }
    }
    if constexpr (Op::kHasOut4 && Op::kHasResid) {
        float4 r[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (c0 + 4 * q + 3 < nout) r[q] = op.resid4(rc, c0 + 4 * q);
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (c0 + 4 * q + 3 < nout) f[q] = add4(f[q], r[q]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int n = c0 + 4 * q;
        if constexpr (Op::kHasOut4) {
            if (n + 3 < nout) {
                op.out4(rc, n, f[q]);
                continue;
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (n + j < nout) op.out(rc, n + j, v[4 * q + j] + (bias ? bias[n + j] : 0.f));
    }
}

// Coalesced output of D [128 x ncols] (TMEM columns from tD) for ops with row-vector
// output (kHasOut4): every warp moves 32-column blocks of its TMEM lane quarter into a padded
// FP32 tile in shared memory; then each warp writes whole rows with its 32 lanes along the
// columns, residual loads of a batch of rows issued before the stores.  Columns go in passes
// of TC_OUT_COLS; the tile needs TC_M x (TC_OUT_COLS + 4) floats.  Called by all threads with
// a uniform ok; contains barriers.
constexpr int TC_OUT_COLS = 128;
constexpr size_t TC_OUT_BYTES = (size_t)TC_M * (TC_OUT_COLS + 4) * 4;

template <class Op>
__device__ __forceinline__ void tc_out_rows(const Op& op, const RowCtx* rc, unsigned char* smem, unsigned tD,
                                            int ncols, const float* bias, long row0, long rows, bool ok) {
    constexpr int TS = TC_OUT_COLS + 4;       // row stride (floats): 16-byte stores of 8 lanes hit distinct banks
    constexpr int NW = TC_T / 32;
    constexpr int RB = 4;                     // rows per batch of loads
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lrow = (warp & 3) * 32 + lane;
    const unsigned lane_off = (unsigned)((warp & 3) * 32) << 16;
    float* T = reinterpret_cast<float*>(smem);
    const int nout = op.nout;
    for (int cb = 0; cb < ncols; cb += TC_OUT_COLS) {
        const int nc = min(TC_OUT_COLS, ncols - cb);
        if (ok) {
            for (int c0 = cb + (warp >> 2) * 32; c0 < cb + nc; c0 += 32 * (TC_T / 128)) {
                float v[32];
                tc_ld32(tD + lane_off + (unsigned)c0, v);
                float* t = T + lrow * TS + (c0 - cb);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    *reinterpret_cast<float4*>(t + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
        }
        __syncthreads();
        if (ok) {
            const int nv = max(0, min(nc, nout - cb)) / 4;     // whole float4 columns of this pass
            for (int rb = warp * RB; rb < TC_M; rb += NW * RB) {
                for (int f = lane; f < nv; f += 32) {
                    const int n = cb + 4 * f;
                    float4 x[RB];
#pragma unroll
                    for (int i = 0; i < RB; ++i) {
                        x[i] = *reinterpret_cast<const float4*>(T + (rb + i) * TS + 4 * f);
                        if (bias) {
                            x[i].x += bias[n]; x[i].y += bias[n + 1]; x[i].z += bias[n + 2]; x[i].w += bias[n + 3];
                        }
                    }
                    if constexpr (Op::kHasResid) {
                        float4 r[RB];
#pragma unroll
                        for (int i = 0; i < RB; ++i)
                            if (row0 + rb + i < rows) r[i] = op.resid4(rc[rb + i], n);
#pragma unroll
                        for (int i = 0; i < RB; ++i)
                            if (row0 + rb + i < rows) x[i] = add4(x[i], r[i]);
                    }
#pragma unroll
                    for (int i = 0; i < RB; ++i)
                        if (row0 + rb + i < rows) op.out4(rc[rb + i], n, x[i]);
                }
                // columns of a ragged nout (not a multiple of 4) element by element
                for (int n = cb + 4 * nv + lane; n < min(cb + nc, nout); n += 32)
                    for (int i = 0; i < RB; ++i)
                        if (row0 + rb + i < rows)
                            op.out(rc[rb + i], n, T[(rb + i) * TS + (n - cb)] + (bias ? bias[n] : 0.f));
            }
        }
        __syncthreads();
    }
}

// Bulk copy (TMA engine) of K chunk [k0, k0 + kc) of the P pieces of a tiled weight operand
// with nrows rows (tc_tile_off layout: the chunk of one piece is one contiguous block) into
// the staging buffer; completion is counted in bytes on mbarrier bar.  One thread calls it.
template <int P>
__device__ __forceinline__ void tc_load_b(unsigned char* dst, int piece_bytes, const __nv_bfloat16* const* src,
                                          int nrows, int k0, int kc, void* bar, long extra = 0) {
    const unsigned bytes = (unsigned)nrows * kc * 2;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes * P)
                 : "memory");
#pragma unroll
    for (int p = 0; p < P; ++p)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(dst + p * piece_bytes)),
            "l"(src[p] + (long)nrows * k0 + extra), "r"(bytes), "r"(smem_u32(bar))
            : "memory");
}

// Stage the A chunk (tile rows x K [k0, k0 + kc)) from the op's input rows, split into P
// pieces.  Full chunks issue every thread's loads before converting and storing.
template <int P, int KC, class Op>
__device__ __forceinline__ void tc_stage_a(const Op& op, const RowCtx* rc, long row0, long rows, unsigned char* sA,
                                           int a_piece, int k0, int kc, int tid) {
    auto put = [&](int m, int kv, const float* x) {
        uint4 pc[P];
        pack8<P>(x, pc);
        const int o = tc_off(m, kv * 8, KC);
#pragma unroll
        for (int p = 0; p < P; ++p) *reinterpret_cast<uint4*>(sA + p * a_piece + o) = pc[p];
    };
    if (kc == KC) {
        constexpr int IT = TC_M * (KC / 8) / TC_T;
        float x[IT][8];
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            int m, kv;
            tc_vec_rc(tid + i * TC_T, KC / 8, m, kv);
            if (row0 + m < rows) {
                tc_load8(op, rc[m], k0 + kv * 8, x[i]);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) x[i][j] = 0.f;
            }
        }
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            int m, kv;
            tc_vec_rc(tid + i * TC_T, KC / 8, m, kv);
            put(m, kv, x[i]);
        }
    } else {
        const int kv8 = kc / 8;
        for (int v = tid; v < TC_M * kv8; v += TC_T) {
            int m, kv;
            tc_vec_rc(v, kv8, m, kv);
            float x[8];
            if (row0 + m < rows) {
                tc_load8(op, rc[m], k0 + kv * 8, x);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) x[j] = 0.f;
            }
            put(m, kv, x);
        }
    }
}

// A full chunk in registers: vectors tid + i TC_T (i < IT) of 8 inputs each.
template <int KC>
struct TcAReg {
    static constexpr int IT = TC_M * (KC / 8) / TC_T;
    float x[IT][8];
};

// Load a full chunk (K [k0, k0 + KC)) of the op's input rows into registers.
template <int KC, class Op>
__device__ __forceinline__ void tc_load_a_full(const Op& op, const RowCtx* rc, long row0, long rows, int k0,
                                               int tid, TcAReg<KC>& a) {
#pragma unroll
    for (int i = 0; i < TcAReg<KC>::IT; ++i) {
        int m, kv;
        tc_vec_rc(tid + i * TC_T, KC / 8, m, kv);
        if (row0 + m < rows) {
            tc_load8(op, rc[m], k0 + kv * 8, a.x[i]);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) a.x[i][j] = 0.f;
        }
    }
}

// Split a register-held chunk into P BF16 pieces in the core-matrix layout.
template <int P, int KC>
__device__ __forceinline__ void tc_store_a_full(unsigned char* sA, int a_piece, int tid, const TcAReg<KC>& a) {
#pragma unroll
    for (int i = 0; i < TcAReg<KC>::IT; ++i) {
        int m, kv;
        tc_vec_rc(tid + i * TC_T, KC / 8, m, kv);
        uint4 pc[P];
        pack8<P>(a.x[i], pc);
        const int o = tc_off(m, kv * 8, KC);
#pragma unroll
        for (int p = 0; p < P; ++p) *reinterpret_cast<uint4*>(sA + p * a_piece + o) = pc[p];
    }
}

// K per staged chunk (the tiled weight layout's chunk width): TC_CHUNK_F for the forward
// (rollout) MLPs, F = true, whose weights are tiled with it; TC_CHUNK for the reverse MLPs.
template <bool F, int P>
__host__ __device__ constexpr int tc_kc() {
    return F ? TC_CHUNK_F : TC_CHUNK;
}
// K per staged chunk of the second product (half a chunk for products wider than TC_NB rows).
template <bool F>
__host__ __device__ inline int tc_kc2(int n2p) {
    return F ? tc_chunk_b2_fwd(n2p) : tc_chunk_b2(n2p);
}

// Shared memory: [A chunk buffers | hidden tile] (the hidden tile reuses the A buffers once
// GEMM1 is done) followed by the B chunk buffers (TC_NB rows x KC; GEMM2 products wider than
// TC_NB stage half-K chunks of the same size).
// Chunk pipeline depth: the A chunk and the weight chunk each get NBUF buffers (chunk g in
// buffer g % NBUF; the weight chunk NBUF - 1 ahead is in flight while chunk c multiplies).
// One buffer everywhere: for the three-piece forward, two full-width buffers (192 KB of shared
// memory, less L1 for its gathered node-row loads) and two or three half-width ones (more
// chunks, each with its barrier and MMA-issue round) all measured slower; the reverse MLPs run
// two CTAs per SM with one buffer.
template <bool F, int P>
__host__ __device__ constexpr int tc_nbuf() {
    return F ? TC_NBUF_F : 1;
}
template <int W, bool F, int P, int NB = tc_nbuf<F, P>()>
__host__ __device__ constexpr size_t tc_region_a() {
    return (size_t)P * ((size_t)NB * TC_M * tc_kc<F, P>() * 2 > (size_t)TC_M * W * 2
                            ? (size_t)NB * TC_M * tc_kc<F, P>() * 2
                            : (size_t)TC_M * W * 2);
}
template <int W, bool F, int P, int NB = tc_nbuf<F, P>()>
__host__ __device__ constexpr size_t tc_smem_bytes() {
    return tc_region_a<W, F, P, NB>() + (size_t)NB * P * TC_NB * tc_kc<F, P>() * 2;
}
// Launch size: at least TC_SMEM_MIN, so that no more than two CTAs share an SM (what two
// TC_TMEM_COLS allocations fill) and the output tile of tc_out_rows fits.
constexpr size_t TC_SMEM_MIN = 100 * 1024;
static_assert(TC_OUT_BYTES <= TC_SMEM_MIN, "output tile must fit the minimum launch size");

// Barrier and pipeline state of a CTA that runs tiles of the tensor-core MLP: the MMA-completion
// and weight-arrival mbarriers of each buffer, their completed phases, and the weight chunks in
// flight.  A CTA that runs several tiles (the persistent rollout) keeps it across tiles.
struct TcTileState {
    unsigned long long* mbar;     // [NBUF] MMA completion (tcgen05.commit)
    unsigned long long* bbar;     // [NBUF] weight chunk arrival (bulk-copy bytes)
    unsigned mph[TC_NBUF_MAX], bphase[TC_NBUF_MAX];   // completed phases
    bool b_pending[TC_NBUF_MAX];
};

// Thread 0: bulk-copy weight chunk g of a tile (g < nch: the K chunks of B1; then the K chunks of
// B2) into buffer g % NBUF.
template <int W, bool F, int P, int NBUF = tc_nbuf<F, P>()>
__device__ __forceinline__ void tc_load_chunk(const TcW& w, unsigned char* sB0, TcTileState& S, int g, int nch,
                                              int kc2, int nh = 1) {
    constexpr int KC = tc_kc<F, P>(), B_BYTES = TC_NB * KC * 2;
    const int b = g % NBUF;
    unsigned char* dst = sB0 + (size_t)b * P * B_BYTES;
    if (nh > 1 && g < nch * nh) {
        // half h of chunk c of a B1 with nh W rows: the chunk's rows are 8-row groups in order,
        // so the half is the contiguous block W kc elements after the chunk's start
        const int c = g % nch, h = g / nch, kc = min(KC, w.K1p - c * KC);
        tc_load_b<P>(dst, B_BYTES, w.B1, W, 0, kc, &S.bbar[b], (long)nh * W * c * KC + (long)h * W * kc);
    } else if (g < nch) {
        tc_load_b<P>(dst, B_BYTES, w.B1, W, g * KC, min(KC, w.K1p - g * KC), &S.bbar[b]);
    } else {
        const int k0 = (g - nch) * kc2;
        tc_load_b<P>(dst, B_BYTES, w.B2, w.N2p, k0, min(kc2, W - k0), &S.bbar[b]);
    }
    S.b_pending[b] = true;
}

// Thread 0: the first weight chunks of a tile (issued early, under the tile's prologue).
template <int W, class Op, int P, int NBUF = tc_nbuf<(Op::kMode == 0), P>()>
__device__ __forceinline__ void tc_tile_prefetch(const TcW& w, unsigned char* tsm, TcTileState& S) {
    constexpr bool F = (Op::kMode == 0);
    constexpr bool kSingle = (Op::kMode == 2);
    const int nch = (w.K1p + tc_kc<F, P>() - 1) / tc_kc<F, P>();
    const int kc2 = tc_kc2<F>(w.N2p);
    const int nh = kSingle && w.N1p > W ? w.N1p / W : 1;
    const int ng = kSingle ? nch * nh : nch + (W + kc2 - 1) / kc2;
    unsigned char* sB0 = tsm + tc_region_a<W, F, P, NBUF>();
    for (int g = 0; g < NBUF && g < ng; ++g) tc_load_chunk<W, F, P, NBUF>(w, sB0, S, g, nch, kc2, nh);
}

// One 128-row tile of the fused MLP (rows row0 ..), run by all TC_T threads of the CTA:
//   GEMM1 over K chunks -> hidden epilogue (bias + ReLU + mask bits, or the saved mask) ->
//   GEMM2 over K chunks -> output epilogue (or the single-product epilogue).
// rc: the tile's row contexts, prepared by the caller (visible after a __syncthreads); tD: the
// CTA's TC_TMEM_COLS tensor-memory columns; the weight chunks of tc_tile_prefetch must have been
// issued.  Returns the CTA-uniform ok (false after a bounded wait gave up).
template <int W, class Op, int P, int NBUF = tc_nbuf<(Op::kMode == 0), P>()>
__device__ __forceinline__ bool tc_mlp_tile(const Op& op, const TcW& w, long row0, unsigned char* tsm,
                                            const RowCtx* rc, unsigned tD, TcTileState& S) {
    constexpr bool F = (Op::kMode == 0);
    constexpr int KC = tc_kc<F, P>();
    constexpr int A_BYTES = TC_M * KC * 2, B_BYTES = TC_NB * KC * 2, H_BYTES = TC_M * W * 2;
    unsigned char* sA = tsm;                          // NBUF x P pieces of the A chunk, K-major with K = KC
    unsigned char* sH = tsm;                          // P pieces of the hidden tile, K = W (after GEMM1)
    unsigned char* sB0 = tsm + tc_region_a<W, F, P, NBUF>();   // NBUF buffers of P pieces of a B chunk (bulk copies)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long rows = op.rows;
    constexpr bool kSingle = (Op::kMode == 2);
    const int nch = (w.K1p + KC - 1) / KC;
    const int kc2 = tc_kc2<F>(w.N2p);
    const int n2 = kSingle ? 0 : (W + kc2 - 1) / kc2;
    const int nh = kSingle && w.N1p > W ? w.N1p / W : 1;   // halves of a wide single product
    const int n1 = nch * nh;                                 // B chunks of GEMM1
    const int ng = n1 + n2;
    bool ok = true;
    // all threads: wait for the MMAs of chunk g (A buffer and B buffer g % NBUF are then free);
    // thread 0 then copies the weight chunk NBUF ahead into the freed B buffer
    auto wait_chunk = [&](int g) {
        const int b = g % NBUF;
        ok = tc_wait(&S.mbar[b], S.mph[b] & 1, w.status) && ok;
        ++S.mph[b];
        if (tid == 0 && ok && g + NBUF < ng && !S.b_pending[b])
            tc_load_chunk<W, F, P, NBUF>(w, sB0, S, g + NBUF, nch, kc2, nh);
    };
    constexpr int CSTEP = 32 * (TC_T / 128);
    const int lrow = (warp & 3) * 32 + lane;
    const int cgrp = warp >> 2;
    // reverse mode: the ReLU mask words of this thread's row and column blocks, fetched under GEMM1
    constexpr int NMW = (W + CSTEP - 1) / CSTEP;
    uint32_t mwv[NMW];
    if constexpr (Op::kMode == 1) {
#pragma unroll
        for (int q = 0; q < NMW; ++q) {
            const int c0 = cgrp * 32 + q * CSTEP;
            mwv[q] = (c0 < W && row0 + lrow < rows) ? op.mask_word(rc[lrow], c0 >> 5) : 0u;
        }
    }

    // thread 0: wait for the staged B chunk, issue the chunk's MMAs, commit them to mbar (the
    // commit arrives even when nothing was issued, so the other threads never wait in vain)
    auto issue = [&](int g, unsigned a0, unsigned a_piece, unsigned a_sbo, unsigned b_sbo, int kc, int N, bool first,
                     unsigned dcol = 0) {
        const int b = g % NBUF;
        bool okb = false;
        if (S.b_pending[b]) {
            okb = tc_wait(&S.bbar[b], S.bphase[b] & 1, w.status);
            if (okb) {
                ++S.bphase[b];
                S.b_pending[b] = false;
            }
        }
        if (okb)
            tc_issue<P>(tD + dcol, a0, a_piece, a_sbo, smem_u32(sB0 + (size_t)b * P * B_BYTES), B_BYTES, b_sbo, kc, N,
                        first);
        tc_commit(&S.mbar[b]);
        return okb;
    };

    // ---------------- GEMM1 over K chunks; a full chunk's inputs are loaded into registers one
    // chunk ahead, under the previous chunk's MMAs (not for the gather-sum inputs of the
    // single-product form, whose variable-length loops measured slower that way)
    constexpr bool kAhead = !kSingle;
    TcAReg<KC> xa;
    if (kAhead && nch > 0 && KC <= w.K1p) tc_load_a_full<KC>(op, rc, row0, rows, 0, tid, xa);
    // Chunk c goes into A buffer c % NBUF, whose previous chunk (c - NBUF) was waited for at the
    // end of iteration c - 1; chunk c's MMAs then run while chunk c + 1 is staged.
    if (kSingle && nh > 1) {
        // a wide single product (K1p = W, N = nh W): the whole input tile staged once in the
        // K-major layout of the hidden tile, then its K chunks for each N half of W columns
        tc_stage_a<P, W>(op, rc, row0, rows, sH, H_BYTES, 0, W, tid);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        for (int g1 = 0; g1 < n1; ++g1) {
            const int c = g1 % nch, h = g1 / nch;
            const int k0 = c * KC, kc = min(KC, w.K1p - k0);
            if (tid == 0)
                ok = issue(g1, smem_u32(sH) + (k0 / 8) * 128, H_BYTES, W * 16, kc * 16, kc, W, c == 0,
                           (unsigned)(h * W)) && ok;
            if (g1 - NBUF + 1 >= 0) wait_chunk(g1 - NBUF + 1);
        }
    } else {
    for (int c = 0; c < nch; ++c) {
        const int k0 = c * KC;
        const int kc = min(KC, w.K1p - k0);        // multiple of 16
        unsigned char* sAc = sA + (size_t)(c % NBUF) * P * A_BYTES;
        if (kAhead && kc == KC) tc_store_a_full<P, KC>(sAc, A_BYTES, tid, xa);
        else tc_stage_a<P, KC>(op, rc, row0, rows, sAc, A_BYTES, k0, kc, tid);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) ok = issue(c, smem_u32(sAc), A_BYTES, KC * 16, kc * 16, kc, W, c == 0) && ok;
        if (kAhead && k0 + 2 * KC <= w.K1p) tc_load_a_full<KC>(op, rc, row0, rows, k0 + KC, tid, xa);
        // the chunk NBUF - 1 back has finished: its buffers take chunk c + 1 (A) and the weight
        // chunk NBUF ahead of it (for the last GEMM1 chunks, the first GEMM2 chunks)
        if (c - NBUF + 1 >= 0) wait_chunk(c - NBUF + 1);
    }
    }
    for (int g = max(0, n1 - NBUF + 1); g < n1; ++g) wait_chunk(g);   // GEMM1 complete
    ok = __syncthreads_and(ok) != 0;           // warp-collective TMEM loads below need a uniform decision
    tc_fence_after();

    // ---------------- hidden layer / single-product epilogue; 32-column blocks rotate
    // over the warp groups; TMEM lane = tile row (warp w reads lanes 32 (w % 4) ..)
    const bool valid = ok && (row0 + lrow < rows);
    const unsigned lane_off = (unsigned)((warp & 3) * 32) << 16;
    if (kSingle) {
        if constexpr (Op::kHasOut4) {
            tc_out_rows(op, rc, tsm, tD, W * nh, nullptr, row0, rows, ok);
        } else {
            for (int c0 = cgrp * 32; c0 < W; c0 += CSTEP) {
                float v[32];
                if (ok) tc_ld32(tD + lane_off + (unsigned)c0, v);
                if (valid) tc_out32(op, rc[lrow], c0, v, op.nout, nullptr);
            }
        }
    } else {
        for (int c0 = cgrp * 32; c0 < W; c0 += CSTEP) {
            float v[32];
            if (ok) tc_ld32(tD + lane_off + (unsigned)c0, v);
            if constexpr (Op::kMode == 0) {
                uint32_t bits = 0;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    float h = v[j] + op.b1[c0 + j];
                    h = h > 0.f ? h : 0.f;
                    bits |= (h > 0.f ? 1u : 0u) << j;
                    v[j] = h;
                }
                if (valid) op.store_mask(rc[lrow], c0 >> 5, bits);
            } else {
                const uint32_t mw = valid ? mwv[(c0 - cgrp * 32) / CSTEP] : 0u;
                if constexpr (Op::kHidAdd) {
                    if (valid) op.hid_add(rc[lrow], c0, v);     // terms of the first layer added per row
                }
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = ((mw >> j) & 1u) ? v[j] : 0.f;
                if constexpr (Op::kStoreHid) {
                    if (valid)
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            op.store_hid4(rc[lrow], c0 + 4 * q,
                                          make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint4 pc[P];
                pack8<P>(v + q * 8, pc);
                const int o = tc_off(lrow, c0 + q * 8, W);
#pragma unroll
                for (int p = 0; p < P; ++p) *reinterpret_cast<uint4*>(sH + p * H_BYTES + o) = pc[p];
            }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();                       // sH complete; every warp's TMEM reads of D1 are done
        tc_fence_after();
        // ---------------- GEMM2 over K = W in chunks of kc2 (B2 chunks by bulk copy)
        for (int k0 = 0; k0 < W; k0 += kc2) {
            const int kc = min(kc2, W - k0);
            // hidden tile: K-major with K = W; the chunk starts k0/8 core matrices along K
            const int g = nch + k0 / kc2;
            if (tid == 0) ok = issue(g, smem_u32(sH) + (k0 / 8) * 128, H_BYTES, W * 16, kc * 16, kc, w.N2p, k0 == 0) && ok;
            if (g - NBUF + 1 >= nch) wait_chunk(g - NBUF + 1);
        }
        for (int g = max(nch, ng - NBUF + 1); g < ng; ++g) wait_chunk(g);   // GEMM2 complete
        ok = __syncthreads_and(ok) != 0;
        tc_fence_after();
        if constexpr (Op::kHasOut4) {
            tc_out_rows(op, rc, tsm, tD, w.N2p, op.b2, row0, rows, ok);   // A/H and B buffers are free
        } else {
            const bool valid2 = ok && (row0 + lrow < rows);
            for (int c0 = cgrp * 32; c0 < w.N2p; c0 += CSTEP) {
                float v[32];
                if (ok) tc_ld32(tD + lane_off + (unsigned)c0, v);
                if (valid2) tc_out32(op, rc[lrow], c0, v, op.nout, op.b2);
            }
        }
    }
    return ok;
}

// Set-up of a CTA that runs tensor-core MLP tiles: barrier init (thread 0) and the tensor-memory
// allocation (warp 0); tc_cta_teardown waits for weight copies still in flight and frees it.
template <bool F, int P, int NBUF = tc_nbuf<F, P>()>
__device__ __forceinline__ void tc_cta_init(TcTileState& S, unsigned long long* mbar, unsigned long long* bbar) {
    S.mbar = mbar;
    S.bbar = bbar;
    for (int b = 0; b < TC_NBUF_MAX; ++b) {
        S.mph[b] = 0;
        S.bphase[b] = 0;
        S.b_pending[b] = false;
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int b = 0; b < NBUF; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bbar[b])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
}
__device__ __forceinline__ void tc_tmem_alloc(unsigned* tmem_base) {
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_base)),
                     "n"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
}
template <bool F, int P, int NBUF = tc_nbuf<F, P>()>
__device__ __forceinline__ void tc_cta_teardown(TcTileState& S, unsigned tmem_base) {
    // a bulk copy whose wait gave up may still be landing: wait (bounded) before the CTA exits
    if (threadIdx.x == 0)
#pragma unroll
        for (int b = 0; b < NBUF; ++b)
            if (S.b_pending[b]) tc_wait(&S.bbar[b], S.bphase[b] & 1, nullptr);
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "n"(TC_TMEM_COLS));
}

// One tile per CTA (tile blockIdx.x).
template <int W, class Op, int P, int NB = tc_nbuf<(Op::kMode == 0), P>()>
__global__ void __launch_bounds__(TC_T) tc_mlp_kernel(Op op, TcW w) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ RowCtx rc[TC_M];
    constexpr bool F = (Op::kMode == 0);
    __shared__ __align__(8) unsigned long long mbar[NB];   // MMA completion per buffer (tcgen05.commit)
    __shared__ __align__(8) unsigned long long bbar[NB];   // B chunk arrival (bulk-copy bytes)
    __shared__ unsigned tmem_base;
    TcTileState S;
    tc_cta_init<F, P, NB>(S, mbar, bbar);
    const long row0 = (long)blockIdx.x * TC_M;
    const long rows = op.rows;
    if (threadIdx.x == 0) tc_tile_prefetch<W, Op, P, NB>(w, tsm, S);      // first chunks, under the prologue
    // the prologue reads only weights and the static row indices (op.prep): it overlaps the
    // previous kernel's tail under programmatic dependent launch
    for (int m = threadIdx.x; m < TC_M; m += TC_T) rc[m] = op.prep(row0 + m < rows ? row0 + m : -1);
    tc_tmem_alloc(&tmem_base);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    pdl_wait();
    if (w.early) pdl_launch_dependents();
    tc_mlp_tile<W, Op, P, NB>(op, w, row0, tsm, rc, tmem_base, S);
    // this CTA's work is done: the next kernel may start its prologue (triggered at the end, not
    // the start, so that early CTAs of the next kernel do not hold SMs for this kernel's
    // whole duration when many instances run side by side)
    pdl_launch_dependents();
    tc_cta_teardown<F, P, NB>(S, tmem_base);
}

// Two MLPs in sequence on the same 128 rows (tile blockIdx.x), where the second reads only what
// the first wrote for those rows (row-local): one launch instead of two.  The first tile's
// output stores become visible to the CTA's threads at the barrier between the two; the second
// tile's weight chunks are copied once the first tile's buffers are free.  Both ops run in
// reverse (mask) mode with the same rows.
template <int W, class Op1, class Op2, int P, int NB = tc_nbuf<false, P>()>
__global__ void __launch_bounds__(TC_T) tc_mlp_seq_kernel(Op1 op1, TcW w1, Op2 op2, TcW w2) {
    static_assert(Op1::kMode == 1 && (Op2::kMode == 1 || Op2::kMode == 2),
                  "sequenced MLP tiles run in reverse (or single-product) mode");
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ RowCtx rc[TC_M];
    __shared__ __align__(8) unsigned long long mbar[NB];
    __shared__ __align__(8) unsigned long long bbar[NB];
    __shared__ unsigned tmem_base;
    TcTileState S;
    tc_cta_init<false, P, NB>(S, mbar, bbar);
    const long row0 = (long)blockIdx.x * TC_M;
    if (threadIdx.x == 0) tc_tile_prefetch<W, Op1, P, NB>(w1, tsm, S);
    for (int m = threadIdx.x; m < TC_M; m += TC_T) rc[m] = op1.prep(row0 + m < op1.rows ? row0 + m : -1);
    tc_tmem_alloc(&tmem_base);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    pdl_wait();
    bool ok = tc_mlp_tile<W, Op1, P, NB>(op1, w1, row0, tsm, rc, tmem_base, S);
    // the first tile's stores and its reads of shared and tensor memory are complete
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0 && ok) tc_tile_prefetch<W, Op2, P, NB>(w2, tsm, S);
    for (int m = threadIdx.x; m < TC_M; m += TC_T) rc[m] = op2.prep(row0 + m < op2.rows ? row0 + m : -1);
    __syncthreads();
    if (ok) tc_mlp_tile<W, Op2, P, NB>(op2, w2, row0, tsm, rc, tmem_base, S);
    pdl_launch_dependents();
    tc_cta_teardown<false, P, NB>(S, tmem_base);
}

}  // namespace gmi
