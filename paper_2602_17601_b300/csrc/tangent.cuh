// Matrix-free condensing: the sensitivities S_k = d x_k / d U (the block rows of Gamma_u) pushed
// through the GNN by forward-mode products, one tangent per input column, instead of forming the
// local Jacobians A_k and running the recursion of Eq. sparse_gamma_i_u (Thm. 1 proof):
//
//   S_{k+1}[:, t] = dF/dx(x_hat_k, u_hat_k) S_k[:, t] + dF/du(x_hat_k, u_hat_k) e_t   (t in stage k)
//
// Each tangent runs through the stage's MLPs as their linearisation at the rollout: the same
// weights, no biases, the hidden layer multiplied by the ReLU mask the rollout stored
// (Eq. linearized_dynamics), and the residual connections carried.  Column t = i nu + a is zero
// for k <= i and, for k > i, outside the nodes that act_node[a] reaches in K (k - i) edges; within
// stage k its tangent gains one hop per message-passing layer.  The rows of a launch are, tangent
// by tangent, the nodes (edges) of that support in the per-actuator hop order of the context's
// tables (struct Tangents), so every gather of the previous layer is a position in that order
// compared with the previous support's size.  Gamma_x follows from the rollout: the prediction
// Gamma_u U + Gamma_x reproduces x_hat at U = u_hat, so D_k = Gamma_x_k - x_hat_k = -S_k u_hat.
//
// Included by gnn.cu (uses its launch helpers and ReLU-mask layout).
#pragma once

namespace gmi {

// Edge rows of a layer from which its first layer runs on per-node projections (NodeProjTan +
// EdgeMpTan) instead of whole per edge row (EdgeMpTanK3).  With the projections as one wide
// product in the node update's launch, the last tangent stage of the closed-loop step at the
// chain of 1000 ends 6.15 ms into it from 30k rows, 6.18 from 60k, 6.22 from 100k.
constexpr long kTanSplitRows = 30000;   // gm_settings.tan_split_rows = 0

// Whether each tangent kernel lets the next one of the stage start its prologue (weight chunks,
// row contexts, tensor-memory allocation) as soon as all of its own CTAs have started.  Off: the
// waiting CTAs hold SMs that the rollout of later stages needs (closed-loop step at the chain of
// 1000: 7.69 ms off, 8.52 ms on; 8.31 ms with the rollout's kernels early as well).
constexpr bool kTanPdlEarly = false;
static TcW tan_w(TcW w) {
    w.early = kTanPdlEarly ? 1 : 0;
    return w;
}

// Row -> (tangent, position in its support) of one (stage, layer) launch.  The ops read each
// row's context from the launch's slice of the context's tables (struct Tangents: one 16-byte
// load); off, find and the order tables remain for the counts and the message sum.
struct TanBase : BwdBase {
    static constexpr bool kTangent = true;
    const int4* ctx;         // row contexts of this launch, [rows]
    const int* off;          // [T + 1] row offsets of the tangents in this launch
    int T, nu, K, k, M, E, Rmax;
    const int *norder, *npos, *ncnt, *eorder, *epos, *ecnt;
    const uint32_t* mlmask;  // the rollout's ReLU mask of this MLP at stage k: [units][W/32]
    __device__ int find(long r) const {
        int lo = 0, hi = T;                  // off[lo] <= r < off[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (off[mid] <= r) lo = mid;
            else hi = mid;
        }
        return lo;
    }
    __device__ int node_count(int a, int R) const { return R < 0 ? 0 : ncnt[a * (Rmax + 1) + min(R, Rmax)]; }
    __device__ int edge_count(int a, int R) const { return R < 0 ? 0 : ecnt[a * (Rmax + 1) + min(R, Rmax)]; }
    // row of (tangent t, node n) in a node layer with offsets poff and radius R, or -1 outside
    __device__ int node_row(const int* poff, int t, int a, int n, int R) const {
        const int p = npos[a * M + n];
        return p < node_count(a, R) ? poff[t] + p : -1;
    }
    __device__ int edge_row(const int* poff, int t, int a, int q, int R) const {
        const int p = epos[a * E + q];
        return p < edge_count(a, R) ? poff[t] + p : -1;
    }
    __device__ uint32_t mask_word(const RowCtx& x, int wd) const { return mlmask[(long)x.d * wwords + wd]; }
};

// Node encoder: input [dx (6) | m u (nu)] of node n: dx = S_k[n][:, t] (i < k), du = e_a at
// act_node[a] (i = k).  RowCtx: a row, b node, c tangent, d node (mask), e 1 if i < k, f the input
// index 6 + a carrying the unit tangent at the actuated node (i = k), else -1.
struct NodeEncTan : TanBase {
    const float* Sk;         // Gamma_u block row k (k >= 1), row length L = k nu
    const int* act;
    float* th;
    __device__ RowCtx prep(long r) const {
        RowCtx x{0, 0, 0, 0, 0, -1};
        if (r < 0) return x;
        const int4 v = __ldg(ctx + r);               // {-, t, n, i < k}
        const int a = v.y % nu;
        x.a = (int)r; x.b = v.z; x.c = v.y; x.d = v.z; x.e = v.w;
        x.f = (v.w == 0 && act[a] == v.z) ? 6 + a : -1;
        return x;
    }
    __device__ float in(const RowCtx& x, int kk) const {
        if (kk < 6) return x.e ? Sk[((long)x.b * 6 + kk) * (k * nu) + x.c] : 0.f;
        return kk == x.f ? 1.f : 0.f;
    }
    __device__ void out(const RowCtx& x, int n, float v) const { th[(long)x.a * W + n] = v; }
    static constexpr bool kHasOut4 = true;
    __device__ void out4(const RowCtx& x, int n, float4 v) const { st4(th + (long)x.a * W + n, v); }
};

// Edge encoder (edges j -> i, input x_i - x_j): rows only for tangents with i < k.
// RowCtx: a row, b dst, c src, d edge (mask), e tangent.
struct EdgeEncTan : TanBase {
    const float* Sk;
    const int *src, *dst;
    float* te;
    __device__ RowCtx prep(long r) const {
        RowCtx x{0, 0, 0, 0, 0, 0};
        if (r < 0) return x;
        const int4 v = __ldg(ctx + r);               // {dst, src, q, t}
        x.a = (int)r; x.b = v.x; x.c = v.y; x.d = v.z; x.e = v.w;
        return x;
    }
    __device__ float in(const RowCtx& x, int kk) const {
        if (kk >= 6) return 0.f;
        const long L = (long)k * nu;
        return Sk[((long)x.b * 6 + kk) * L + x.e] - Sk[((long)x.c * 6 + kk) * L + x.e];
    }
    __device__ void out(const RowCtx& x, int n, float v) const { te[(long)x.a * W + n] = v; }
    static constexpr bool kHasOut4 = true;
    __device__ void out4(const RowCtx& x, int n, float4 v) const { st4(te + (long)x.a * W + n, v); }
};

// Edge update of layer l with the whole first layer per edge row:
// te_l = te_{l-1} + J [th_{l-1}(dst) | th_{l-1}(src) | te_{l-1}] (K = 3W).  Used where a layer has
// few edge rows (early stages), where one launch costs less than the projections' extra launch.
// RowCtx: a row, b th row of dst, c th row of src, d edge (mask), e te row of the edge (-1: 0).
struct EdgeMpTanK3 : TanBase {
    const int *src, *dst;
    const int *noff_prev, *eoff_prev;
    int Rn_prev_base, Re_prev_base;
    const float *th_prev, *te_prev;
    float* te;
    __device__ RowCtx prep(long r) const {
        RowCtx x{0, -1, -1, 0, -1, 0};
        if (r < 0) return x;
        const int4 v = __ldg(ctx + r);               // {dst row, src row, q, previous edge row}
        x.a = (int)r; x.b = v.x; x.c = v.y; x.d = v.z; x.e = v.w;
        return x;
    }
    __device__ float in(const RowCtx& x, int kk) const {
        if (kk < W) return x.b >= 0 ? th_prev[(long)x.b * W + kk] : 0.f;
        if (kk < 2 * W) return x.c >= 0 ? th_prev[(long)x.c * W + kk - W] : 0.f;
        return x.e >= 0 ? te_prev[(long)x.e * W + kk - 2 * W] : 0.f;
    }
    __device__ void out(const RowCtx& x, int n, float v) const {
        te[(long)x.a * W + n] = (x.e >= 0 ? te_prev[(long)x.e * W + n] : 0.f) + v;
    }
    static constexpr bool kHasIn8 = true, kHasOut4 = true, kHasResid = true;
    __device__ void in8(const RowCtx& x, int k0, float* v) const {
        const int row = k0 < W ? x.b : (k0 < 2 * W ? x.c : x.e);
        const float* base = k0 < 2 * W ? th_prev : te_prev;
        if (row >= 0) {
            ld8(base + (long)row * W + (k0 % W), v);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = 0.f;
        }
    }
    __device__ float4 resid4(const RowCtx& x, int n) const {
        return x.e >= 0 ? ld4(te_prev + (long)x.e * W + n) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __device__ void out4(const RowCtx& x, int n, float4 v) const { st4(te + (long)x.a * W + n, v); }
};

// The node blocks of an edge update's first layer, per node row of layer l - 1:
// P = th_{l-1} [W_a | W_b] (2W columns), so that an edge row's first layer is P[dst][:W] +
// P[src][W:] + te W_c.  Run as the tensor-core MLP with an identity first product and an all-ones
// mask (GEMM1 only re-splits th into the operand pieces of GEMM2, N = 2W).
// RowCtx: a row (also the row of P).
struct NodeProjTan : TanBase {
    const float* th_prev;
    float* P;
    __device__ RowCtx prep(long r) const { return RowCtx{r < 0 ? 0 : (int)r, 0, 0, 0, 0, 0}; }
    __device__ float in(const RowCtx& x, int kk) const { return th_prev[(long)x.a * W + kk]; }
    __device__ uint32_t mask_word(const RowCtx&, int) const { return 0xFFFFFFFFu; }
    __device__ void out(const RowCtx& x, int n, float v) const { P[(long)x.a * 2 * W + n] = v; }
    static constexpr bool kHasIn8 = true, kHasOut4 = true;
    __device__ void in8(const RowCtx& x, int k0, float* v) const { ld8(th_prev + (long)x.a * W + k0, v); }
    __device__ void out4(const RowCtx& x, int n, float4 v) const { st4(P + (long)x.a * 2 * W + n, v); }
};

// The same projections as one product on the tensor cores: P = th_{l-1} [W_a | W_b] with the
// operand's 2W rows taken as two halves of W (TcW::N1p = 2W).
struct NodeProjTan1 : NodeProjTan {
    static constexpr int kMode = 2;
};

// Edge update of layer l: te_l = te_{l-1} + W2' (mask . (P[dst][:W] + P[src][W:] + te_{l-1} W_c)),
// the node blocks of the first layer taken from the projections P of the node layer l - 1.
// RowCtx: a row, b P row of dst (-1: 0), c P row of src (-1: 0), d edge (mask), e te row of the
// edge in the previous edge layer (-1: 0).
struct EdgeMpTan : TanBase {
    static constexpr bool kHidAdd = true;
    static constexpr bool kWsResid = true;    // warp-specialised kernel: te_{l-1} added by the tensor cores
    const int *src, *dst;
    const int *noff_prev, *eoff_prev;   // offsets of the node layer l - 1 and the edge layer l - 1
    int Rn_prev_base, Re_prev_base;     // radius of those layers minus K (k - i)
    const float *P, *te_prev;
    float* te;
    __device__ RowCtx prep(long r) const {
        RowCtx x{0, -1, -1, 0, -1, 0};
        if (r < 0) return x;
        // {dst row, src row, q, previous edge row}; the edge encoder has no rows for the tangents
        // of stage k (their x tangent is zero)
        const int4 v = __ldg(ctx + r);
        x.a = (int)r; x.b = v.x; x.c = v.y; x.d = v.z; x.e = v.w;
        return x;
    }
    __device__ float in(const RowCtx& x, int kk) const { return x.e >= 0 ? te_prev[(long)x.e * W + kk] : 0.f; }
    __device__ float hid_val(const RowCtx& x, int n) const {
        return (x.b >= 0 ? P[(long)x.b * 2 * W + n] : 0.f) + (x.c >= 0 ? P[(long)x.c * 2 * W + W + n] : 0.f);
    }
    // 32 hidden columns [c0, c0 + 32): both projected rows loaded before the adds
    __device__ void hid_add(const RowCtx& x, int c0, float* v) const {
        float4 pa[8], pb[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            pa[q] = ldg4_if(P + (long)(x.b >= 0 ? x.b : 0) * 2 * W + c0 + 4 * q, x.b >= 0);
            pb[q] = ldg4_if(P + (long)(x.c >= 0 ? x.c : 0) * 2 * W + W + c0 + 4 * q, x.c >= 0);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            v[4 * q] += pa[q].x + pb[q].x; v[4 * q + 1] += pa[q].y + pb[q].y;
            v[4 * q + 2] += pa[q].z + pb[q].z; v[4 * q + 3] += pa[q].w + pb[q].w;
        }
    }
    __device__ void out(const RowCtx& x, int n, float v) const {
        te[(long)x.a * W + n] = (x.e >= 0 ? te_prev[(long)x.e * W + n] : 0.f) + v;
    }
    static constexpr bool kHasIn8 = true, kHasOut4 = true, kHasResid = true;
    __device__ void in8(const RowCtx& x, int k0, float* v) const {
        if (x.e >= 0) {
            ld8(te_prev + (long)x.e * W + k0, v);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = 0.f;
        }
    }
    __device__ float4 resid4(const RowCtx& x, int n) const {
        return x.e >= 0 ? ld4(te_prev + (long)x.e * W + n) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __device__ void out4(const RowCtx& x, int n, float4 v) const { st4(te + (long)x.a * W + n, v); }
    // warp-specialised kernel: the A row is te_{l-1} (zero where the edge had no tangent)
    __device__ void in8_pair(const RowCtx& x, int k0, float4* a, float4* b) const {
        const float* pa = te_prev + (long)(x.e >= 0 ? x.e : 0) * W + k0;
        a[0] = ldg4_if(pa, x.e >= 0);
        a[1] = ldg4_if(pa + 4, x.e >= 0);
        b[0] = b[1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
};

// Node update of layer l: th_l = th_{l-1} + J [th_{l-1} | tagg_l].  RowCtx: a row (also the
// row of tagg_l, same layer), b th row of the node in layer l - 1 (-1: 0), d node (mask).
struct NodeMpTan : TanBase {
    const int* noff_prev;
    int Rn_prev_base;
    const float *th_prev, *tagg;
    float* th;
    __device__ RowCtx prep(long r) const {
        RowCtx x{0, -1, 0, 0, 0, 0};
        if (r < 0) return x;
        const int4 v = __ldg(ctx + r);               // {previous row, t, n, -}
        x.a = (int)r; x.b = v.x; x.d = v.z;
        return x;
    }
    __device__ float in(const RowCtx& x, int kk) const {
        if (kk < W) return x.b >= 0 ? th_prev[(long)x.b * W + kk] : 0.f;
        return tagg[(long)x.a * W + kk - W];
    }
    __device__ void out(const RowCtx& x, int n, float v) const {
        th[(long)x.a * W + n] = (x.b >= 0 ? th_prev[(long)x.b * W + n] : 0.f) + v;
    }
    static constexpr bool kHasIn8 = true, kHasOut4 = true, kHasResid = true;
    __device__ void in8(const RowCtx& x, int k0, float* v) const {
        if (k0 >= W) {
            ld8(tagg + (long)x.a * W + k0 - W, v);
        } else if (x.b >= 0) {
            ld8(th_prev + (long)x.b * W + k0, v);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = 0.f;
        }
    }
    __device__ float4 resid4(const RowCtx& x, int n) const {
        return x.b >= 0 ? ld4(th_prev + (long)x.b * W + n) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __device__ void out4(const RowCtx& x, int n, float4 v) const { st4(th + (long)x.a * W + n, v); }
};

// Decoder and Euler update (semi-implicit, Eq. forward_dynamics): dv' = J th_K, v' = dv_x + dv',
// p' = dp_x + dt v', written to Gamma_u block row k + 1.  RowCtx: a row, b node, c tangent,
// d node (mask), e 1 if i < k (the tangent has an x part).
struct DecTan : TanBase {
    const float* Sk;         // block row k (k >= 1), row length k nu
    float* Sk1;              // block row k + 1, row length (k + 1) nu
    const float* th;
    float dt;
    __device__ RowCtx prep(long r) const {
        RowCtx x{0, 0, 0, 0, 0, 0};
        if (r < 0) return x;
        const int4 v = __ldg(ctx + r);               // {-, t, n, i < k}
        x.a = (int)r; x.b = v.z; x.c = v.y; x.d = v.z; x.e = v.w;
        return x;
    }
    __device__ float in(const RowCtx& x, int kk) const { return th[(long)x.a * W + kk]; }
    static constexpr bool kHasIn8 = true;
    __device__ void in8(const RowCtx& x, int k0, float* v) const { ld8(th + (long)x.a * W + k0, v); }
    __device__ void out(const RowCtx& x, int n, float dv) const {
        const long L = (long)k * nu, L1 = (long)(k + 1) * nu;
        const float vx = x.e ? Sk[((long)x.b * 6 + 3 + n) * L + x.c] : 0.f;
        const float px = x.e ? Sk[((long)x.b * 6 + n) * L + x.c] : 0.f;
        const float v1 = vx + dv;
        Sk1[((long)x.b * 6 + 3 + n) * L1 + x.c] = v1;
        Sk1[((long)x.b * 6 + n) * L1 + x.c] = px + dt * v1;
    }
};

// Message sum of layer l for every node row (tangent t, node n): the sum of the edge rows of its
// in-edges within the edge layer's support (the context's list, in edge order).  One warp per
// row, four columns per lane; up to eight edge rows are loaded at once.
__global__ void tan_agg_kernel(long rows, int W, const int* __restrict__ aptr, const int* __restrict__ alist,
                               const float* __restrict__ te, float* __restrict__ tagg, int early) {
    const long r = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    pdl_wait();                  // launched with programmatic serialization: the edge update is done
    if (early) pdl_launch_dependents();
    if (r >= rows) {
        pdl_launch_dependents();
        return;
    }
    const int j0 = __ldg(aptr + r), j1 = __ldg(aptr + r + 1);
    for (int c0 = lane * 4; c0 < W; c0 += 128) {
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int jb = j0; jb < j1; jb += 8) {
            int idx[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) idx[u] = jb + u < j1 ? __ldg(alist + jb + u) : -1;
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = idx[u] >= 0 ? ld4(te + (long)idx[u] * W + c0) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (idx[u] >= 0) s = add4(s, v[u]);
        }
        st4(tagg + r * W + c0, s);
    }
    pdl_launch_dependents();
}

// D_k = Gamma_x_k - x_hat_k = -S_k u_hat for k = 1..N (D_0 = 0), one warp per (k, node, component).
__global__ void tan_offset_kernel(int N, int M, int nu, const float* __restrict__ Gu,
                                  const float* __restrict__ u_hat, float* __restrict__ D) {
    const long w = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= (long)N * M * 6) return;
    const int k = (int)(w / ((long)M * 6)) + 1;
    const long ia = w % ((long)M * 6);
    const int L = k * nu;
    const float* row = Gu + gu_offset(M, nu, k) + ia * L;
    float s = 0.f;
    for (int t = lane; t < L; t += 32) s = fmaf(row[t], u_hat[t], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) D[(long)k * M * 6 + ia] = -s;
}

template <class Op>
static void fill_tan(Op& op, const gm_ctx* c, const MlpOff& m, int k, int layer_off, bool edge, const uint32_t* mask) {
    const Tangents& T = c->tan;
    const int L = c->N * c->nu + 1;
    const int* offs = edge ? c->dtan.eoff : c->dtan.noff;
    op.off = offs + (long)(k * (c->K + 1) + layer_off) * L;
    op.ctx = (edge ? c->dtan.ectx : c->dtan.nctx) +
             (edge ? T.ebase : T.nbase)[(size_t)k * (c->K + 1) + layer_off];
    const std::vector<int>& hoff = edge ? T.eoff : T.noff;
    const int Tk = (k + 1) * c->nu;
    op.rows = hoff[(size_t)(k * (c->K + 1) + layer_off) * L + Tk];
    op.T = Tk; op.nu = c->nu; op.K = c->K; op.k = k; op.M = c->M; op.E = c->E; op.Rmax = T.Rmax;
    op.norder = c->dtan.norder; op.npos = c->dtan.npos; op.ncnt = c->dtan.ncnt;
    op.eorder = c->dtan.eorder; op.epos = c->dtan.epos; op.ecnt = c->dtan.ecnt;
    op.kin = m.in;
    op.nout = m.out;
    op.B1 = c->d_wts + m.W1;          // the forward orientation: the tangent map is the linearised forward MLP
    op.B2 = c->d_wts + m.W2;
    op.mlmask = mask;
    op.wwords = c->W / 32;
    op.W = c->W;
    op.R = 0;
}

static long tan_rows(const gm_ctx* c, int k, int layer, bool edge) {
    const int L = c->N * c->nu + 1;
    const std::vector<int>& hoff = edge ? c->tan.eoff : c->tan.noff;
    return hoff[(size_t)(k * (c->K + 1) + layer) * L + (k + 1) * c->nu];
}

// Tangent pass of stage k: S_{k+1} from S_k and the rollout's ReLU masks of stage k.
static gm_status tangent_stage(gm_ctx* c, int k, cudaStream_t st) {
    const int M = c->M, K = c->K, N = c->N, nu = c->nu, W = c->W;
    const int L = N * nu + 1;
    float* th[2] = {c->d_thA, c->d_thB};
    float* te[2] = {c->d_teA, c->d_teB};
    const float* Sk = k > 0 ? c->d_Gu + gu_offset(M, nu, k) : nullptr;
    float* Sk1 = c->d_Gu + gu_offset(M, nu, k + 1);
    // the two encoders read only S_k: the edge encoder's tangents run on a side stream beside the
    // node encoder's (a fork and a join of events, graph branches when captured)
    const bool edges = k > 0 && c->E > 0;
    const bool fork = edges && c->tan_side;
    if (fork) {
        GM_CUDA_TRY(cudaEventRecord(c->ev_tfork, st));
        GM_CUDA_TRY(cudaStreamWaitEvent(c->tan_side, c->ev_tfork, 0));
    }
    if (edges) {   // edge encoder (edge layer 0): tangents of earlier stages only
        EdgeEncTan op{};
        fill_tan(op, c, c->mlp[1], k, 0, true, edge_mask(c, k, 0));
        op.Sk = Sk; op.src = c->d_src; op.dst = c->d_dst; op.te = te[0];
        GM_TRY(launch_mlp(c, op, tan_w(tc_fwd(c, c->mlp[1])), fork ? c->tan_side : st, !fork));
    }
    if (fork) GM_CUDA_TRY(cudaEventRecord(c->ev_tjoin, c->tan_side));
    // The projections of an edge layer's node blocks (NodeProjTan, layers of kTanSplitRows edge
    // rows or more) and the decoder are row-local on the node rows the node encoder or the node
    // update just wrote: each runs in the same launch as its producer (tc_mlp_seq_kernel).
    const long split = c->s.tan_split_rows > 0 ? c->s.tan_split_rows : kTanSplitRows;
    auto projected = [&](int l) { return c->E > 0 && l <= K && tan_rows(c, k, l, true) >= split; };
    // P of edge layer l from node layer l - 1 after the launch of op (with tw): one product on the
    // tensor cores, the identity-first-layer MLP in the FP32 form
    auto with_proj = [&](int l, const auto& op, const TcW& tw) -> gm_status {
        const MlpOff& m = c->mlp[2 + 2 * (l - 1)];
        auto fill = [&](NodeProjTan& pj) {
            fill_tan(pj, c, m, k, l - 1, false, nullptr);
            pj.kin = W; pj.nout = 2 * W;
            pj.B1 = c->d_wts + m.eye; pj.B2 = c->d_wts + m.Pab;
            pj.th_prev = th[(l - 1) & 1]; pj.P = c->d_tproj;
        };
        if (c->s.precision == GM_PREC_FP32) {
            NodeProjTan pj{};
            fill(pj);
            return launch_mlp_seq(c, op, tw, pj, tan_w(tc_w(c, m.eyek, m.pabk, W, 2 * W)), st);
        }
        NodeProjTan1 pj{};
        fill(pj);
        TcW tp = tan_w(tc_w(c, m.pabk1, -1, W, 0));
        tp.N1p = 2 * W;
        return launch_mlp_seq(c, op, tw, pj, tp, st);
    };
    {   // node encoder (node layer 0)
        NodeEncTan op{};
        fill_tan(op, c, c->mlp[0], k, 0, false, node_mask(c, k, 0));
        op.Sk = Sk; op.act = c->d_act; op.th = th[0];
        const TcW tw = tan_w(tc_fwd(c, c->mlp[0]));
        if (projected(1)) {
            GM_TRY(with_proj(1, op, tw));
        } else {
            GM_TRY(launch_mlp(c, op, tw, st));
        }
    }
    if (fork) GM_CUDA_TRY(cudaStreamWaitEvent(st, c->ev_tjoin, 0));
    for (int l = 1; l <= K; ++l) {
        const int* noff_prev = c->dtan.noff + (long)(k * (K + 1) + l - 1) * L;
        const int* eoff_prev = c->dtan.eoff + (long)(k * (K + 1) + l - 1) * L;
        if (c->E > 0) {
            const MlpOff& m = c->mlp[2 + 2 * (l - 1)];
            const long erows = tan_rows(c, k, l, true);
            const double ep = (double)tan_rows(c, k, l - 1, true), np = (double)tan_rows(c, k, l - 1, false);
            int kt = -1;
            if (projected(l)) {
                // the edge rows with the e-block of the first layer alone (K = W); the node blocks
                // came with the launch that wrote node layer l - 1
                EdgeMpTan em{};
                fill_tan(em, c, m, k, l, true, edge_mask(c, k, l));
                em.kin = W;
                em.B1 = c->d_wts + m.W1 + (long)2 * W * W;   // the e-block of W1, [W][hid]
                em.src = c->d_src; em.dst = c->d_dst;
                em.noff_prev = noff_prev; em.eoff_prev = eoff_prev;
                em.Rn_prev_base = l - 1;
                em.Re_prev_base = l == 1 ? -1 : l - 2;   // -1: the encoder's layer (none for i = k)
                em.P = c->d_tproj; em.te_prev = te[(l - 1) & 1]; em.te = te[l & 1];
                // timed: 4W bytes per edge row written and per carried edge row read, 8W per
                // projected node row, W/8 per edge mask; one product of 2 (W W + W W) FLOPs per row
                if (c->ktiming)
                    kt = kev_begin(c, 4.0 * W * (erows + ep) + 8.0 * W * np + (double)c->E * W / 8.0,
                                   4.0 * W * W * erows, (int)cdiv(erows, TC_M), st);
                const TcW tw = tan_w(tc_w(c, m.fck, m.fk2, W, m.out_p));
                if (c->s.precision == GM_PREC_MIXED && W == WS_W && tw.N2p == WS_W) {
                    GM_TRY(launch_ws_bwd(c, em, tw, st));     // warp-specialised persistent form
                } else {
                    GM_TRY(launch_mlp(c, em, tw, st));
                }
            } else if (erows > 0) {
                EdgeMpTanK3 em{};
                fill_tan(em, c, m, k, l, true, edge_mask(c, k, l));
                em.src = c->d_src; em.dst = c->d_dst;
                em.noff_prev = noff_prev; em.eoff_prev = eoff_prev;
                em.Rn_prev_base = l - 1;
                em.Re_prev_base = l == 1 ? -1 : l - 2;
                em.th_prev = th[(l - 1) & 1]; em.te_prev = te[(l - 1) & 1]; em.te = te[l & 1];
                // timed: 4W bytes per edge row written, per carried edge row and per node row of
                // the previous layer read, W/8 per edge mask; one product of 2 (3W W + W W) FLOPs
                if (c->ktiming)
                    kt = kev_begin(c, 4.0 * W * (erows + ep + np) + (double)c->E * W / 8.0, 8.0 * W * W * erows,
                                   (int)cdiv(erows, TC_M), st);
                GM_TRY(launch_mlp(c, em, tan_w(tc_fwd(c, m)), st));
            }
            if (kt >= 0) GM_CUDA_TRY(record_kev(c->kev[kt][1], st));
        }
        const long nrows = tan_rows(c, k, l, false);
        if (nrows > 0) {
            if (c->E > 0) {
                GM_CUDA_TRY(launch_pdl(c->pdl, tan_agg_kernel, dim3((unsigned)cdiv(nrows * 32, 256)), dim3(256), 0, st,
                                       nrows, W, (const int*)(c->dtan.aptr + c->tan.nbase[(size_t)k * (K + 1) + l]),
                                       (const int*)c->dtan.alist, (const float*)te[l & 1], c->d_tagg,
                                       kTanPdlEarly ? 1 : 0));
            } else {
                GM_CUDA_TRY(cudaMemsetAsync(c->d_tagg, 0, sizeof(float) * nrows * W, st));
            }
        }
        NodeMpTan nm{};
        fill_tan(nm, c, c->mlp[3 + 2 * (l - 1)], k, l, false, node_mask(c, k, l));
        nm.noff_prev = noff_prev; nm.Rn_prev_base = l - 1;
        nm.th_prev = th[(l - 1) & 1]; nm.tagg = c->d_tagg; nm.th = th[l & 1];
        const TcW tn = tan_w(tc_fwd(c, c->mlp[3 + 2 * (l - 1)]));
        if (l == K) {   // the decoder and the Euler update into S_{k+1}
            DecTan de{};
            fill_tan(de, c, c->mlp[2 + 2 * K], k, K, false, node_mask(c, k, K + 1));
            de.Sk = Sk; de.Sk1 = Sk1; de.th = th[K & 1]; de.dt = c->dt;
            GM_TRY(launch_mlp_seq(c, nm, tn, de, tan_w(tc_fwd(c, c->mlp[2 + 2 * K])), st));
        } else if (projected(l + 1)) {
            GM_TRY(with_proj(l + 1, nm, tn));
        } else {
            GM_TRY(launch_mlp(c, nm, tn, st));
        }
    }
    return GM_OK;   // (K >= 1: the decoder ran with the last node update)
}

static gm_status tangent_offset(gm_ctx* c, const float* u_hat, cudaStream_t st) {
    const int M = c->M, N = c->N;
    GM_CUDA_TRY(cudaMemsetAsync(c->d_Gx, 0, sizeof(float) * M * 6, st));
    const long warps = (long)N * M * 6;
    tan_offset_kernel<<<cdiv(warps * 32, 256), 256, 0, st>>>(N, M, c->nu, c->d_Gu, u_hat, c->d_Gx);
    GM_LAUNCH_CHECK();
    return GM_OK;
}

static gm_status check_mf(const gm_ctx* c) {
    if (c->s.condensing != 1 || !c->dtan.noff) {
        set_error("matrix-free condensing needs a context created with gm_settings.condensing = 1");
        return GM_ERR_INVALID_ARG;
    }
    return GM_OK;
}

// Gamma_u block rows 1..N to zero before the tangent pass (DecTan writes only its supports).
static gm_status tangent_clear(gm_ctx* c, cudaStream_t st) {
    const long n = gu_offset(c->M, c->nu, c->N + 1) - gu_offset(c->M, c->nu, 1);
    GM_CUDA_TRY(cudaMemsetAsync(c->d_Gu + gu_offset(c->M, c->nu, 1), 0, sizeof(float) * n, st));
    return GM_OK;
}

gm_status gnn_sensitivities(gm_ctx* c, const float* u_hat, cudaStream_t st) {
    GM_TRY(check_mf(c));
    GM_TRY(tangent_clear(c, st));
    for (int k = 0; k < c->N; ++k) GM_TRY(tangent_stage(c, k, st));
    return tangent_offset(c, u_hat, st);
}

// Rollout and sensitivities overlapped: the rollout runs on the context's high-priority stream,
// forked from st, and records an event after each stage; the tangent pass of stage k waits for it
// on st (it reads only stage k's ReLU masks and S_k) and runs beside the rollout of later stages.
gm_status gnn_rollout_sensitivities(gm_ctx* c, const float* x0, const float* u_hat, float* x_hat,
                                    cudaStream_t st) {
    GM_TRY(check_mf(c));
    const int M = c->M, N = c->N;
    if (!c->roll_stream || (int)c->ev_tan.size() < N) {
        GM_TRY(gnn_rollout(c, x0, u_hat, x_hat, st));
        return gnn_sensitivities(c, u_hat, st);
    }
    cudaStream_t rs = c->roll_stream;
    // the tangent pass on its own highest-priority stream when the context has one
    cudaStream_t ts = c->tan_stream ? c->tan_stream : st;
    GM_CUDA_TRY(cudaEventRecord(c->ev_roll, st));
    GM_CUDA_TRY(cudaStreamWaitEvent(rs, c->ev_roll, 0));
    if (ts != st) GM_CUDA_TRY(cudaStreamWaitEvent(ts, c->ev_roll, 0));
    const bool tl = c->stiming && (int)c->sev.size() >= 2 * N + 1;
    if (tl) GM_CUDA_TRY(record_kev(c->sev[0], rs));
    if (x_hat != x0) GM_CUDA_TRY(cudaMemcpyAsync(x_hat, x0, sizeof(float) * M * 6, cudaMemcpyDeviceToDevice, rs));
    GM_TRY(tangent_clear(c, ts));
    for (int k = 0; k < N; ++k) {
        GM_TRY(forward_stage(c, k, x_hat + (long)k * M * 6, u_hat + (long)k * c->nu, x_hat + (long)(k + 1) * M * 6,
                             rs));
        GM_CUDA_TRY(cudaEventRecord(c->ev_tan[k], rs));
        if (tl) GM_CUDA_TRY(record_kev(c->sev[1 + k], rs));
        GM_CUDA_TRY(cudaStreamWaitEvent(ts, c->ev_tan[k], 0));
        GM_TRY(tangent_stage(c, k, ts));
        if (tl) GM_CUDA_TRY(record_kev(c->sev[1 + N + k], ts));
    }
    GM_TRY(tangent_offset(c, u_hat, ts));
    if (ts != st) {   // join: the tangent pass (which waited for the whole rollout) into st
        GM_CUDA_TRY(cudaEventRecord(c->ev_tan_done, ts));
        GM_CUDA_TRY(cudaStreamWaitEvent(st, c->ev_tan_done, 0));
    }
    return GM_OK;
}

}  // namespace gmi
