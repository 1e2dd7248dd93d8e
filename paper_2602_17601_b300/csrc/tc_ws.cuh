// Warp-specialised persistent form of a reverse two-layer MLP (W = 128, two BF16 pieces):
// the edge-update reverse step (stored hidden cotangent, residual output, 128 outputs) and
// the edge- and node-encoder reverse steps (no stored hidden, no residual, a few outputs;
// their input rows arrive whole by bulk copy into a landing tile, Op::kWsLand).
//
// Per 128-row tile:  D1  = A . B1^T            (A: the row cotangents, K = 128)
//                    H   = mask . D1           (ReLU mask of the forward pass; stored as FP32
//                                               when Op::kWsHid)
//                    out = D2 = [A . I +] H . B2^T   (N2p = 128, or 16 / 32 columns)
// With Op::kWsResid the residual (out = A + H B2^T) is added by the tensor cores: D2 starts as the BF16 pieces
// of A times a 16 x 16 identity block (a_hi + a_lo, within 2^-18 |a| of the FP32 input), so
// the output epilogue loads nothing.
//
// One CTA per SM walks the tiles blockIdx.x, blockIdx.x + grid, ...  Both weight operands
// stay in shared memory for the whole launch (bulk-copied once).  Four roles overlap
// consecutive tiles:
//   warp 0 (one thread)  issues the tcgen05 MMAs; GEMM1 of tile t + 1 is issued before
//                        GEMM2 of tile t;
//   warps 1-11           producer: row contexts (one tile ahead), A loads (the two input
//                        rows of each vector issued together), BF16 split into the A buffer;
//   warps 12-19          hidden epilogue: D1 -> mask -> the stored hidden (FP32), and the
//                        BF16 pieces of H written back into D1's own tensor-memory columns
//                        (two BF16 per 32-bit column), where GEMM2 reads its A operand;
//   warps 20-27          output epilogue: D2 (two warps per lane quadrant, 64 columns each).
// Tensor memory holds two tile slots of 256 columns ([D1 | H] and D2).  A lives in shared
// memory only until GEMM1 and the identity product have read it, so the producer stages the
// next tile while the hidden epilogue and GEMM2 of this one run.  Both epilogues write whole
// 128-byte row segments (an in-register transpose within groups of 8 lanes): stores of
// 32-byte pieces of many rows measured 1.4x slower for the whole kernel.
//
// Row contexts live in a ring of four slots (filled and released through their own
// barriers), so the producer runs up to four tiles ahead of the epilogues, and every role
// reads them through a barrier the producer arrives on, not through an MMA commit.
//
// Hand-offs are mbarriers (each waited with a bound; a wait that gives up records
// GM_ERR_TIMEOUT and its role stops); role-internal decisions are made uniform with
// barrier.red so that no named barrier or warp-collective instruction is skipped by part
// of a group.  Every barrier is waited on by at most one phase ahead of its producer (the
// dependency chain of the roles guarantees it), so parity waits cannot alias.
#pragma once

namespace gmi {

constexpr int WS_W = 128;                  // hidden width = K of both products = output width
constexpr int WS_P = 2;                    // BF16 pieces of each operand
constexpr int WS_T = 896;                  // threads: 28 warps
constexpr int WS_PROD0 = 1, WS_NPROD = 11; // producer warps 1..11
constexpr int WS_HID0 = 12, WS_NHID = 8;   // hidden-epilogue warps 12..19
constexpr int WS_OUT0 = 20, WS_NOUT = 8;   // output-epilogue warps 20..27
constexpr int WS_PIECE = TC_M * WS_W * 2;  // bytes of one BF16 piece of a 128 x 128 operand
constexpr int WS_NRC = 4;                  // row-context slots
constexpr int WS_LROW = WS_W + 4;          // landing-tile row pitch (floats): 512 bytes + 16 of pad
constexpr int WS_N2_LAND = 16;             // GEMM2 width of the landing form

// Shared-memory layout of one op: [B1 | B2 | A | landing tile | row contexts | identity].
// Ops with kWsLand (one contiguous 512-byte input row per tile row, GEMM2 of 16 columns) keep
// a small B2 and an FP32 landing tile that per-row bulk copies fill one tile ahead.
template <class Op>
struct WsLayout {
    static constexpr bool kLand = Op::kWsLand;
    static constexpr size_t b2_piece = kLand ? (size_t)WS_N2_LAND * WS_W * 2 : (size_t)WS_PIECE;
    static constexpr size_t off_b1 = 0;
    static constexpr size_t off_b2 = off_b1 + (size_t)WS_P * WS_PIECE;
    static constexpr size_t off_a = off_b2 + (size_t)WS_P * b2_piece;
    static constexpr size_t off_land = off_a + (size_t)WS_P * WS_PIECE;
    static constexpr size_t off_rc = off_land + (kLand ? (size_t)TC_M * WS_LROW * 4 : 0);
    static constexpr size_t off_id = off_rc + (size_t)WS_NRC * TC_M * sizeof(RowCtx);   // 16 x 16 identity
    static constexpr size_t smem = off_id + 16 * 16 * 2;
    static_assert(smem <= 226 * 1024, "warp-specialised MLP exceeds the shared memory of one CTA");
};

__device__ __forceinline__ bool ws_bar_and(int id, int n, bool p) {
    unsigned r;
    asm volatile(
        "{\n.reg .pred q, s;\nsetp.ne.u32 q, %1, 0;\nbarrier.red.and.pred s, %2, %3, q;\nselp.u32 %0, 1, 0, s;\n}\n"
        : "=r"(r)
        : "r"((unsigned)p), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void ws_bar_sync(int id, int n) { asm volatile("barrier.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void ws_arrive(void* mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}
// Bounded mbarrier wait: gives up after about 2 s of device time (%globaltimer), records
// GM_ERR_TIMEOUT in status (nullable) and returns false.
__device__ __forceinline__ bool ws_wait(void* mbar, unsigned parity, int* status) {
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (unsigned it = 0;; ++it) {
        unsigned done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 255) == 255) {
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t - t0 > 2000000000ull) break;
        }
    }
    if (status) dev_fail(status, GM_ERR_TIMEOUT);
    return false;
}
// 16 consecutive 32-bit tensor-memory columns of this thread's lane <- w[0..15]
__device__ __forceinline__ void ws_st16(unsigned taddr, const unsigned* w) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7]), "r"(w[8]), "r"(w[9]),
        "r"(w[10]), "r"(w[11]), "r"(w[12]), "r"(w[13]), "r"(w[14]), "r"(w[15])
        : "memory");
}
// MMA with the A operand in tensor memory (M = 128 lanes, K = 16 as 8 packed columns)
__device__ __forceinline__ void ws_mma_ta(unsigned tmem_d, unsigned tmem_a, unsigned long long bd, unsigned idesc,
                                          unsigned acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
        "r"(tmem_a), "l"(bd), "r"(idesc), "r"(acc));
}
// Write this warp's 32 rows x 32 columns (v[0..31] of the lane's row) as whole 128-byte row
// segments: an 8 x 8 transpose of float4 blocks inside each group of 8 lanes (three
// xor-shuffle stages) leaves lane j with chunk (j & 7) of rows (j & ~7) + g, g = 0..7, so
// each of the eight stores covers four rows x 128 contiguous bytes.
// store(row_in_warp, col, float4).
template <class F>
__device__ __forceinline__ void ws_rows32(int lane, const float* v, F&& store) {
    float4 x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
#pragma unroll
    for (int m = 1; m < 8; m <<= 1) {
        const bool up = (lane & m) != 0;
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            if (p & m) continue;
            const float4 snd = up ? x[p] : x[p | m];
            float4 rcv;
            rcv.x = __shfl_xor_sync(0xffffffffu, snd.x, m);
            rcv.y = __shfl_xor_sync(0xffffffffu, snd.y, m);
            rcv.z = __shfl_xor_sync(0xffffffffu, snd.z, m);
            rcv.w = __shfl_xor_sync(0xffffffffu, snd.w, m);
            if (up) x[p] = rcv;
            else x[p | m] = rcv;
        }
    }
#pragma unroll
    for (int g = 0; g < 8; ++g) store((lane & ~7) + g, 4 * (lane & 7), x[g]);
}

template <class Op>
__global__ void __launch_bounds__(WS_T, 1) tc_ws_bwd_kernel(Op op, TcW w) {
    extern __shared__ __align__(1024) unsigned char wsm[];
    using LY = WsLayout<Op>;
    unsigned char* sB1 = wsm + LY::off_b1;
    unsigned char* sB2 = wsm + LY::off_b2;
    unsigned char* sA = wsm + LY::off_a;
    float* sL = reinterpret_cast<float*>(wsm + LY::off_land);          // [TC_M][WS_LROW] (kWsLand)
    RowCtx* rcs = reinterpret_cast<RowCtx*>(wsm + LY::off_rc);          // [WS_NRC][TC_M]
    __nv_bfloat16* sI = reinterpret_cast<__nv_bfloat16*>(wsm + LY::off_id);
    __shared__ __align__(8) unsigned long long bbar, a_full, a_free, fin, land_full;
    __shared__ __align__(8) unsigned long long d1_full[2], h_full[2], d2_full[2], out_free[2];
    __shared__ __align__(8) unsigned long long rc_full[WS_NRC], rc_free[WS_NRC];
    __shared__ unsigned tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long rows = op.rows;
    const long ntiles = (rows + TC_M - 1) / TC_M;
    const long G = gridDim.x;
    const int nt = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / G + 1) : 0;
    if (tid == 0) {
        auto init = [](unsigned long long* b, unsigned n) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(n));
        };
        init(&bbar, 1); init(&a_full, 32 * WS_NPROD); init(&a_free, 1); init(&fin, 1); init(&land_full, 1);
        for (int k = 0; k < 2; ++k) {
            init(&d1_full[k], 1);
            init(&h_full[k], 32 * WS_NHID);
            init(&d2_full[k], 1);
            init(&out_free[k], 32 * WS_NOUT);
        }
        for (int k = 0; k < WS_NRC; ++k) {
            init(&rc_full[k], TC_M);
            init(&rc_free[k], 32 * (WS_NHID + WS_NOUT));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // identity block, K-major core-matrix layout (K = 16): element (n, k) at tc_off(n, k, 16)
    for (int t = tid; t < 256; t += WS_T) {
        const int n = t >> 4, k = t & 15;
        sI[tc_off(n, k, 16) / 2] = __float2bfloat16(n == k ? 1.f : 0.f);
    }
    fence_async_smem();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    pdl_wait();                  // before any read of data an earlier kernel produced
    if (w.early) pdl_launch_dependents();
    const unsigned tmem = tmem_base;
    auto tile_row0 = [&](int i) { return (blockIdx.x + (long)i * G) * TC_M; };

    if (warp == 0) {
        // ------------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            bool ok = true;
            bool b_pending = true;
            {
                const unsigned bytes = (unsigned)WS_PIECE, bytes2 = (unsigned)w.N2p * WS_W * 2;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bbar)),
                             "r"(WS_P * (bytes + bytes2)) : "memory");
#pragma unroll
                for (int p = 0; p < WS_P; ++p) {
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            smem_u32(sB1 + p * WS_PIECE)), "l"(w.B1[p]), "r"(bytes), "r"(smem_u32(&bbar)) : "memory");
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            smem_u32(sB2 + p * LY::b2_piece)), "l"(w.B2[p]), "r"(bytes2), "r"(smem_u32(&bbar)) : "memory");
                }
            }
            if (nt > 0) {
                ok = ws_wait(&bbar, 0, w.status);
                b_pending = !ok;
            }
            // weight chunks (K 64) lie 16 KB apart with SBO = 64 * 16; A uses K = 128
            const unsigned a0 = smem_u32(sA), b10 = smem_u32(sB1), b20 = smem_u32(sB2);
            const unsigned long long bdI = tc_desc(smem_u32(sI), 16 * 16);
            auto ready = [](unsigned long long* b, unsigned parity) {
                unsigned done;
                asm volatile(
                    "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                    : "=r"(done)
                    : "r"(smem_u32(b)), "r"(parity)
                    : "memory");
                return done != 0;
            };
            // GEMM1 of tile i into D1 of its slot, then D2 = A . I (residual); frees the A buffer
            auto gemm1 = [&](int i) {
                const int s = i & 1;
                const unsigned tD1 = tmem + (unsigned)(s * 256), tD2 = tD1 + 128;
                tc_fence_after();
                for (int j = 0; j < 2; ++j)
                    tc_issue<WS_P>(tD1, a0 + j * 1024, WS_PIECE, WS_W * 16, b10 + j * (WS_W * 64 * 2), WS_PIECE,
                                   64 * 16, 64, WS_W, j == 0);
                if constexpr (Op::kWsResid)
                    for (int j = 0; j < WS_W / 16; ++j)
#pragma unroll
                        for (int p = 0; p < WS_P; ++p)
                            tc_mma(tD2 + (unsigned)(16 * j), tc_desc(a0 + p * WS_PIECE + j * 256, WS_W * 16), bdI,
                                   tc_idesc(TC_M, 16), p > 0 ? 1u : 0u);
                tc_commit(&a_free);
                tc_commit(&d1_full[s]);
            };
            // GEMM2 of tile i: D2 (+)= H . B2^T with H's pieces in tensor memory (K-block kk of
            // piece q at column 16 kk + 8 q of the slot); B2 chunks (K 64) are N2p x 64 apart
            auto gemm2 = [&](int i) {
                const int s = i & 1;
                const unsigned tH = tmem + (unsigned)(s * 256), tD2 = tH + 128;
                tc_fence_after();
                const unsigned idesc = tc_idesc(TC_M, w.N2p);
                bool acc = Op::kWsResid;
                for (int kk = 0; kk < WS_W / 16; ++kk) {
                    const unsigned boff = (unsigned)((kk >> 2) * (w.N2p * 64 * 2) + (kk & 3) * 256);
#pragma unroll
                    for (int qa = 0; qa < WS_P; ++qa)
#pragma unroll
                        for (int qb = 0; qa + qb < WS_P; ++qb) {
                            ws_mma_ta(tD2, tH + (unsigned)(16 * kk + 8 * qa),
                                      tc_desc(b20 + qb * (unsigned)LY::b2_piece + boff, 64 * 16), idesc, acc ? 1u : 0u);
                            acc = true;
                        }
                }
                tc_commit(&d2_full[s]);
            };
            // tile i's GEMM2 and tile i + 1's GEMM1, in whichever order their inputs arrive
            // (GEMM1 of tile i + 2, which overwrites H of tile i, is issued after GEMM2 of tile i)
            if (ok && nt > 0) ok = ws_wait(&a_full, 0, w.status);
            if (ok && nt > 0) gemm1(0);
            for (int i = 0; i < nt && ok; ++i) {
                bool g1 = i + 1 >= nt, g2 = false;
                unsigned long long t0;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
                for (unsigned it = 0; !(g1 && g2); ++it) {
                    if (!g2 && ready(&h_full[i & 1], (i >> 1) & 1)) {
                        gemm2(i);
                        g2 = true;
                        continue;
                    }
                    const int n = i + 1;
                    if (!g1 && (n < 2 || ready(&out_free[n & 1], ((n >> 1) - 1) & 1)) && ready(&a_full, n & 1)) {
                        gemm1(n);
                        g1 = true;
                        continue;
                    }
                    if ((it & 255) == 255) {
                        unsigned long long t;
                        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
                        if (t - t0 > 2000000000ull) {
                            dev_fail(w.status, GM_ERR_TIMEOUT);
                            ok = false;
                            break;
                        }
                    }
                }
            }
            // every MMA issued so far has completed before tensor memory is released
            tc_commit(&fin);
            ws_wait(&fin, 0, nullptr);
            if (b_pending) ws_wait(&bbar, 0, nullptr);
        }
        __syncwarp();
    } else if (warp < WS_HID0) {
        // ------------------------------------------------------------------ producer
        constexpr int NP = 32 * WS_NPROD;
        constexpr int NV = TC_M * (WS_W / 8);          // 8-float vectors of one A tile
        constexpr int NVT = (NV + NP - 1) / NP;        // per thread
        constexpr int H1 = NVT / 2;
        const int ptid = tid - 32 * WS_PROD0;
        // row contexts of tile i: threads 0..127 of the group write one row each and arrive
        auto prep = [&](int i) {
            RowCtx* rc = rcs + (i % WS_NRC) * TC_M;
            const long row0 = tile_row0(i);
            if (ptid < TC_M) {
                rc[ptid] = op.prep(row0 + ptid < rows ? row0 + ptid : -1);
                ws_arrive(&rc_full[i % WS_NRC]);
            }
        };
        bool ok = true;
        if (nt > 0) prep(0);
        if constexpr (LY::kLand) {
            // Landing form: thread m < 128 bulk-copies tile row m (512 bytes) into the padded
            // landing tile, the byte count registered on land_full by thread 0; the group then
            // splits the landed tile into the A buffer.  The next tile's rows are copied as soon
            // as this one has been read, so they land while this tile's MMAs and epilogues run.
            int issued = 0, landed = 0;
            auto issue_rows = [&](int i) {
                const long row0 = tile_row0(i);
                const int vr = (int)min((long)TC_M, rows - row0);
                if (ptid == 0)
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&land_full)),
                                 "r"((unsigned)vr * WS_W * 4) : "memory");
                if (ptid < vr) {
                    const RowCtx* rc = rcs + (i % WS_NRC) * TC_M;
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            smem_u32(sL + ptid * WS_LROW)), "l"(op.land_row(rc[ptid])), "r"((unsigned)WS_W * 4),
                        "r"(smem_u32(&land_full)) : "memory");
                }
                ++issued;
            };
            if (nt > 0) issue_rows(0);                  // thread m reads only its own row's context
            for (int i = 0; i < nt; ++i) {
                const long row0 = tile_row0(i);
                ok = ws_wait(&land_full, i & 1, w.status) && ok;
                if (ok) ++landed;
                if (i >= 1) ok = ws_wait(&a_free, (i - 1) & 1, w.status) && ok;   // GEMM1 of the last tile done
                if (!ws_bar_and(1, NP, ok)) break;
#pragma unroll
                for (int j = 0; j < NVT; ++j) {
                    const int v = ptid + j * NP;
                    if (v < NV) {
                        int m, kv;
                        tc_vec_rc(v, WS_W / 8, m, kv);
                        float x8[8];
                        if (row0 + m < rows) {
                            const float4 u0 = *reinterpret_cast<const float4*>(sL + m * WS_LROW + kv * 8);
                            const float4 u1 = *reinterpret_cast<const float4*>(sL + m * WS_LROW + kv * 8 + 4);
                            x8[0] = u0.x; x8[1] = u0.y; x8[2] = u0.z; x8[3] = u0.w;
                            x8[4] = u1.x; x8[5] = u1.y; x8[6] = u1.z; x8[7] = u1.w;
                        } else {
#pragma unroll
                            for (int e = 0; e < 8; ++e) x8[e] = 0.f;
                        }
                        uint4 pc[WS_P];
                        pack8<WS_P>(x8, pc);
                        const int o = tc_off(m, kv * 8, WS_W);
#pragma unroll
                        for (int p = 0; p < WS_P; ++p) *reinterpret_cast<uint4*>(sA + p * WS_PIECE + o) = pc[p];
                    }
                }
                fence_async_smem();
                ws_bar_sync(4, NP);                    // the landing tile has been read by every thread
                ws_arrive(&a_full);
                const int in = i + 1;
                if (in < nt) {
                    if (in >= WS_NRC) ok = ws_wait(&rc_free[in % WS_NRC], ((in / WS_NRC) - 1) & 1, w.status) && ok;
                    if (!ws_bar_and(1, NP, ok)) break;
                    prep(in);
                    issue_rows(in);
                }
            }
            // copies still landing after a failed wait finish before the CTA exits
            while (landed < issued) {
                ws_wait(&land_full, landed & 1, nullptr);
                ++landed;
            }
        } else {
        for (int i = 0; i < nt; ++i) {
            const long row0 = tile_row0(i);
            const RowCtx* rc = rcs + (i % WS_NRC) * TC_M;
            ok = ws_wait(&rc_full[i % WS_NRC], (i / WS_NRC) & 1, w.status) && ok;
            float4 xa[NVT][2], xb[NVT][2];
            auto load = [&](int j) {
                const int v = ptid + j * NP;
                int m = 0, kv = 0;
                if (v < NV) tc_vec_rc(v, WS_W / 8, m, kv);
                if (ok && v < NV && row0 + m < rows) {
                    op.in8_pair(rc[m], kv * 8, xa[j], xb[j]);
                } else {
                    xa[j][0] = xa[j][1] = xb[j][0] = xb[j][1] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            };
            auto store = [&](int j) {
                const int v = ptid + j * NP;
                if (v >= NV) return;
                int m, kv;
                tc_vec_rc(v, WS_W / 8, m, kv);
                const float4 u0 = add4(xa[j][0], xb[j][0]), u1 = add4(xa[j][1], xb[j][1]);
                const float x8[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
                uint4 pc[WS_P];
                pack8<WS_P>(x8, pc);
                const int o = tc_off(m, kv * 8, WS_W);
#pragma unroll
                for (int p = 0; p < WS_P; ++p) *reinterpret_cast<uint4*>(sA + p * WS_PIECE + o) = pc[p];
            };
#pragma unroll
            for (int j = 0; j < H1; ++j) load(j);
            if (i >= 1) ok = ws_wait(&a_free, (i - 1) & 1, w.status) && ok;   // GEMM1 of the last tile done
            if (!ws_bar_and(1, NP, ok)) break;
#pragma unroll
            for (int j = 0; j < H1; ++j) store(j);
#pragma unroll
            for (int j = H1; j < NVT; ++j) load(j);
            // row contexts of the next tile, under the second half's loads (its slot was last
            // used WS_NRC tiles ago)
            const int in = i + 1;
            if (in < nt) {
                if (in >= WS_NRC) ok = ws_wait(&rc_free[in % WS_NRC], ((in / WS_NRC) - 1) & 1, w.status) && ok;
                if (!ws_bar_and(1, NP, ok)) break;
                prep(in);
            }
#pragma unroll
            for (int j = H1; j < NVT; ++j) store(j);
            fence_async_smem();
            ws_arrive(&a_full);
        }
        }
    } else if (warp < WS_OUT0) {
        // ------------------------------------------------------------------ hidden epilogue
        const int q = warp & 3, hh = (warp - WS_HID0) >> 2;   // lane quadrant, column half
        const int lrow = q * 32 + lane;
        const unsigned lane_off = (unsigned)(q * 32) << 16;
        bool ok = true;
        for (int i = 0; i < nt; ++i) {
            const int s = i & 1;
            const long row0 = tile_row0(i);
            const bool valid = row0 + lrow < rows;
            const RowCtx* rc = rcs + (i % WS_NRC) * TC_M;
            ok = ws_wait(&rc_full[i % WS_NRC], (i / WS_NRC) & 1, w.status) && ok;
            if (!ws_bar_and(2, 32 * WS_NHID, ok)) break;
            uint32_t mw[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) mw[k] = valid ? op.mask_word(rc[lrow], 2 * hh + k) : 0u;
            ok = ws_wait(&d1_full[s], (i >> 1) & 1, w.status) && ok;
            if (!ws_bar_and(2, 32 * WS_NHID, ok)) break;
            tc_fence_after();
            const unsigned tD1 = tmem + (unsigned)(s * 256) + lane_off;
#pragma unroll 1
            for (int blk = 0; blk < 2; ++blk) {
                const int c32 = 64 * hh + 32 * blk;
                float v[32];
                tc_ld32(tD1 + (unsigned)c32, v);
                if constexpr (Op::kHidAdd) {
                    if (valid) op.hid_add(rc[lrow], c32, v);     // per-row terms of the first layer
                }
                const uint32_t bits = mw[blk];
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = ((bits >> j) & 1u) ? v[j] : 0.f;
                // H in place: K-block of 16 -> piece 0 in its first 8 columns, piece 1 in the next 8
#pragma unroll
                for (int kb = 0; kb < 2; ++kb) {
                    uint4 pa[WS_P], pb[WS_P];
                    pack8<WS_P>(v + 16 * kb, pa);
                    pack8<WS_P>(v + 16 * kb + 8, pb);
                    const unsigned wd[16] = {pa[0].x, pa[0].y, pa[0].z, pa[0].w, pb[0].x, pb[0].y, pb[0].z, pb[0].w,
                                             pa[1].x, pa[1].y, pa[1].z, pa[1].w, pb[1].x, pb[1].y, pb[1].z, pb[1].w};
                    ws_st16(tD1 + (unsigned)(c32 + 16 * kb), wd);
                }
                // stored hidden (FP32, masked D1)
                if constexpr (Op::kWsHid)
                    ws_rows32(lane, v, [&](int r, int c, float4 x) {
                        const int grow = q * 32 + r;
                        if (row0 + grow < rows) op.store_hid4(rc[grow], c32 + c, x);
                    });
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            ws_arrive(&h_full[s]);
            ws_arrive(&rc_free[i % WS_NRC]);
        }
    } else {
        // ------------------------------------------------------------------ output epilogue
        const int q = warp & 3, half = (warp - WS_OUT0) >> 2;   // lane quadrant, column half
        const unsigned lane_off = (unsigned)(q * 32) << 16;
        bool ok = true;
        for (int i = 0; i < nt; ++i) {
            const int s = i & 1;
            const long row0 = tile_row0(i);
            const RowCtx* rc = rcs + (i % WS_NRC) * TC_M;
            ok = ws_wait(&rc_full[i % WS_NRC], (i / WS_NRC) & 1, w.status) && ok;
            ok = ws_wait(&d2_full[s], (i >> 1) & 1, w.status) && ok;
            if (!ws_bar_and(3, 32 * WS_NOUT, ok)) break;
            tc_fence_after();
            const unsigned tD2 = tmem + (unsigned)(s * 256) + 128 + lane_off;
            bool wide = false;
            if constexpr (Op::kHasOut4) wide = w.N2p == WS_W;
            if (wide) {
                if constexpr (Op::kHasOut4) {
#pragma unroll 1
                    for (int c32 = 64 * half; c32 < 64 * half + 64; c32 += 32) {
                        float v[32];
                        tc_ld32(tD2 + (unsigned)c32, v);
                        ws_rows32(lane, v, [&](int r, int c, float4 x) {
                            const int grow = q * 32 + r;
                            if (row0 + grow < rows) op.out4(rc[grow], c32 + c, x);
                        });
                    }
                }
            } else if (half == 0) {
                // a few outputs per row (N2p <= 32): one lane per row, op.nout values
                float v[32];
                tc_ld32(tD2, v);
                const int lrow = q * 32 + lane;
                if (row0 + lrow < rows)
#pragma unroll
                    for (int n = 0; n < 32; ++n)
                        if (n < op.nout) op.out(rc[lrow], n, v[n]);
            }
            tc_fence_before();
            ws_arrive(&out_free[s]);
            ws_arrive(&rc_free[i % WS_NRC]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    pdl_launch_dependents();     // all tiles of this CTA done: the next kernel may start its prologue
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

}  // namespace gmi
