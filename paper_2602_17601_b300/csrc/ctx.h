// Internal state of graphs, GNN models and contexts, shared by the .cu files.
#pragma once

#include <vector>

#include "common.cuh"

struct gm_graph {
    int M = 0, E = 0, nu = 0;
    std::vector<int> src, dst;      // edges sorted by (dst, src)
    std::vector<int> in_ptr;        // [M+1] CSR by destination
    std::vector<int> act_node;      // [nu]
};

struct gm_gnn {
    gm_gnn_desc d{};
    std::vector<float> blob;
};

struct gm_ctx;

// A batch of contexts stepped as one CUDA graph (gm_batch_rti_step).
struct gm_batch {
    std::vector<gm_ctx*> ctx;
    int lanes = 1;                 // independent chains of instance steps in the batch graph
    int lanes_req = 0;             // lanes asked for by gm_batch_set_lanes (0: gm_batch_plan)
    cudaGraphExec_t exec = nullptr;
    std::vector<uintptr_t> key;
    int eager = 0, captures = 0;
    bool replayed = false;
};

namespace gmi {

struct AdmmState;

// One 2-layer MLP as stored on the device (offsets into the weight array).
struct MlpOff {
    int in = 0, hid = 0, out = 0;
    long W1 = 0, b1 = 0, W2 = 0, b2 = 0;   // forward: W1 [in][hid], W2 [hid][out]
    long W2t = 0;                           // backward GEMM1 operand: W2^T [out][hid]
    long W1t = 0;                           // backward GEMM2 operand: W1^T [hid][in]
    // edge-update MLPs only: the split of W1 by input block [h_dst | h_src | e]
    long Wc = 0;                            // [hid][W]:  Wc[j][n]  = W1[2W + n][j]
    long Bab = 0;                           // [2W][W]:   Bab[j][n] = W1[n][j], Bab[W+j][n] = W1[W+n][j]
    // BF16 K-major copies for the tensor-core kernels ([N rows][K], K and N padded to 16)
    int in_p = 0, out_p = 0;                // in, out rounded up to a multiple of 16
    long fk1 = 0, fk2 = 0;                  // forward:  W1^T [hid][in_p], W2^T [out_p][hid]
    long bk1 = 0, bk2 = 0;                  // reverse:  W2 [hid][out_p],   W1 [in_p][hid]
    long wck = 0, babk = 0;                 // edge MLPs: Wc^T [W][W], Bab^T [W][2W]
    // edge MLPs, matrix-free tangents: the e-block of W1 and the node blocks [W_a | W_b] apart
    long Pab = 0;                           // FP32 [W][2W]: Pab[k][n] = W1[k][n], Pab[k][W+n] = W1[W+k][n]
    long eye = 0;                           // FP32 identity [W][W]
    long fck = 0, pabk = 0, eyek = 0;       // BF16: W1 e-block^T [W][W], Pab^T [2W][W], identity [W][W]
    long pabk1 = 0;                         // BF16: Pab^T [2W][W] in chunks of TC_CHUNK (one product)
};

// Rows of the reverse-mode cones (one seed = one output node s, 3 cotangent
// channels for dv^s).  Level r holds the pairs (s, n) with n reaching s in at
// most r edges (NR_r), and the edges into those nodes (ER_r).
struct Cones {
    int K = 0;
    std::vector<std::vector<int>> nr_node, nr_seed, nr_ptr, nr_prev;  // r = 0..K
    std::vector<std::vector<int>> er_edge, er_dstrow, er_srcrow, er_prev;  // r = 0..K-1
    std::vector<std::vector<int>> er_dst_ptr;              // [|NR_r|+1] rows of ER_r per NR_r row
    std::vector<std::vector<int>> er_src_ptr, er_src_list; // CSR: NR_{r+1} row -> ER_r rows
    // encoder level: ER_{K-1} rows grouped by the NR_K row of their dst
    std::vector<int> enc_dst_ptr, enc_dst_list;            // CSR: NR_K row -> ER_{K-1} rows
    std::vector<int> b_row;                                // [M][nu] NR_K row of (s, act_node[a]) or -1
};

// Device copies of the cone arrays.
struct DCones {
    int* nr_node[8];
    int* nr_prev[8];
    int* er_edge[8];
    int* er_dstrow[8];
    int* er_prev[8];
    int* er_dst_ptr[8];
    int* er_src_ptr[8];
    int* er_src_list[8];
    int* enc_dst_ptr;
    int* enc_dst_list;
    int* nr_ptr_K;       // per-seed offsets of NR_K = Jacobian pattern row_ptr
    int* b_row;
    int nr_count[8];
    int er_count[8];
};

// Matrix-free condensing (gm_settings.condensing = 1): the supports of the forward-mode
// sensitivity columns.  Column t = i nu + a (input a of stage i) is non-zero at stage k > i on the
// nodes that act_node[a] reaches in K (k - i) edges, and inside stage k its tangent grows by one
// hop per message-passing layer.  Nodes (edges) are ordered per actuator by hop distance (by the
// smaller hop distance of their two ends), so the support of radius R is a prefix of that order.
struct Tangents {
    int Rmax = 0;                                  // largest radius used: K N
    std::vector<int> norder, npos, ncnt;           // [nu][M], [nu][M], [nu][Rmax + 1]
    std::vector<int> eorder, epos, ecnt;           // [nu][E], [nu][E], [nu][Rmax + 1]
    // rows of each (stage k, layer l = 0..K) launch: tangent t's rows are off[t] .. off[t + 1];
    // node layer l has radius K (k - i) + l; edge layer 0 (encoder) K (k - i) for i < k and
    // none for i = k; edge layer l >= 1 K (k - i) + l - 1
    std::vector<int> noff, eoff;                   // [N][K + 1][N nu + 1]
    long max_nrows = 0, max_erows = 0;
    // Row contexts of every launch, 4 ints per row, launch (k, l) from row nbase / ebase[k (K + 1) + l]:
    //   node row (t, n):  {row of n in node layer l - 1 (-1: outside it or l = 0), t, n, 1 if i < k}
    //   edge row (t, q), layer 0:  {dst q, src q, q, t}
    //   edge row (t, q), layer l >= 1:  {row of dst q, row of src q in node layer l - 1,
    //                                    q, row of q in edge layer l - 1}   (-1: outside)
    // They depend only on the graph, K and N, so they are built once per context.
    std::vector<int> nctx, ectx;
    std::vector<long> nbase, ebase;                // [N (K + 1)]
    // message sums: node row g (index into nctx / 4) sums the edge rows alist[aptr[g] .. aptr[g + 1])
    // of the same stage and layer, its in-edges within that edge layer's support, in edge order
    std::vector<int> aptr, alist;
};
struct DTangents {
    int *norder = nullptr, *npos = nullptr, *ncnt = nullptr;
    int *eorder = nullptr, *epos = nullptr, *ecnt = nullptr;
    int *noff = nullptr, *eoff = nullptr;
    int4 *nctx = nullptr, *ectx = nullptr;         // row contexts (struct Tangents)
    int *aptr = nullptr, *alist = nullptr;         // message-sum lists (struct Tangents)
};

}  // namespace gmi

struct gm_ctx {
    gm_settings s{};
    int M = 0, E = 0, nu = 0, K = 0, W = 0, N = 0, nU = 0, n_c = 0;
    float dt = 0.f;
    long rows_c = 0;          // N * M * n_c
    long ct_len = 0;          // packed C~ length
    int num_sms = 0;
    bool pdl = true;             // programmatic dependent launch of the MLP kernels (off in a batch)
    bool warm = false;           // ADMM of gm_rti_step starts from the shifted previous (U, y)
    bool gram_tc = true;         // tensor-core Gram products (off in a batch: their one-CTA-per-SM
                                 // grids starve the cooperative grids of the other lanes)
    int stage_chunk = 1;      // stages per reverse-pass launch group

    // host copies
    gm_graph graph;
    std::vector<float> wts_host;
    // BF16 pieces of the tensor-core weight operands: p0 = bf16(x), p1 = bf16(x - p0), p2 = bf16(x - p0 - p1)
    std::vector<uint16_t> wbp_host[3];
    std::vector<int> jac_row_ptr, jac_col;
    gmi::Cones cones;
    gmi::Tangents tan;           // matrix-free condensing only
    std::vector<gmi::MlpOff> mlp;   // blob order: ne, ee, (em, nm) x K, dec
    int nnzb = 0;

    // device pointers carved from the workspace
    char* ws = nullptr;
    size_t ws_bytes = 0;
    int *d_src = nullptr, *d_dst = nullptr, *d_in_ptr = nullptr, *d_act = nullptr;
    int *d_jac_col = nullptr;
    float* d_wts = nullptr;
    uint16_t* d_wbp[3] = {nullptr, nullptr, nullptr};
    gmi::DCones dc{};
    gmi::DTangents dtan{};
    float *d_thA = nullptr, *d_thB = nullptr, *d_tagg = nullptr;   // forward-mode node tangents
    float *d_teA = nullptr, *d_teB = nullptr;                      // forward-mode edge tangents
    float* d_tproj = nullptr;    // node tangents projected by the edge MLP's node blocks [rows][2W]
    // rollout
    float *d_h = nullptr, *d_e = nullptr, *d_agg = nullptr;
    float* d_yw = nullptr;       // shifted previous multipliers (ADMM warm start) [nU + rows]
    uint32_t *d_mask_node = nullptr, *d_mask_edge = nullptr;   // [N][layers][units][W/32]
    // reverse pass (per stage chunk)
    float *d_dhA = nullptr, *d_dhB = nullptr, *d_dacc = nullptr, *d_dagg = nullptr;
    float *d_deA = nullptr, *d_deB = nullptr, *d_ehid = nullptr;
    float *d_dxn = nullptr, *d_dd = nullptr;
    // step state
    float *d_u_hat = nullptr, *d_x_hat = nullptr, *d_A = nullptr, *d_B = nullptr, *d_c = nullptr;
    float *d_Cx = nullptr, *d_dx = nullptr;
    float *d_Gu = nullptr, *d_Gx = nullptr;
    float* d_defect = nullptr;   // condensing: e_k = c_k - x_hat_{k+1} + A_k x_hat_k  [N][M][6]
    float *d_H = nullptr, *d_g = nullptr, *d_Ct = nullptr, *d_dt = nullptr;
    float *d_U = nullptr, *d_y = nullptr, *d_z = nullptr, *d_rs = nullptr;
    unsigned char* d_keep = nullptr;   // ADMM: 0 for redundant half-space rows
    int *d_kpos = nullptr, *d_kcnt = nullptr;   // kept-row positions per stage, kept rows per stage
    float *d_gram_part = nullptr;
    double *d_L = nullptr, *d_Linv = nullptr;
    float *d_P = nullptr, *d_Pinv = nullptr, *d_G = nullptr;
    gmi::AdmmState* d_admm = nullptr;
    float *d_acc = nullptr;      // ADMM reduction buffers [3][admm_acc_stride(nU)]
    double* d_ipm_rows = nullptr; // interior-point row arrays [kIpmRowArrays][max(rows, 1)]
    double* d_ipm_vec = nullptr; // interior-point vectors [kIpmVecArrays][nU] + scalars
    unsigned* d_bar = nullptr;   // grid barrier counters
    int* d_status = nullptr;     // device status word(s)
    int* d_row_begin = nullptr;  // ADMM row partition [grid+1]
    double* d_kkt = nullptr;     // KKT accumulators
    double* d_pol = nullptr;     // polish scratch (FP64)
    int* d_pol_idx = nullptr;
    float* d_U_pol = nullptr;
    float* d_y_pol = nullptr;
    gm_stats* d_stats = nullptr; // internal stats when the caller passes none
    int admm_grid = 0;
    // phase timing of gm_rti_step (events on the caller's stream)
    bool timing = false;
    std::vector<std::array<cudaEvent_t, 6>> events;
    // CUDA-graph replay of gm_rti_step
    bool graph_on = false, graph_failed = false, graph_replayed = false;
    int graph_eager = 0, graph_captures = 0;
    std::vector<uintptr_t> graph_key;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t cond_stream = nullptr;   // bodies of the ADMM rounds' IF nodes while a step is captured
    bool cond_capture = false;            // the capture in progress may use IF nodes (whole-step capture)
    // the edge encoder of a rollout stage runs on this stream beside the node encoder
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // the rollout runs on this high-priority stream while the reverse pass of the stages it has
    // finished runs on the caller's stream (ev_stage[c]: the stages of reverse chunk c are rolled out)
    cudaStream_t roll_stream = nullptr;
    int ws_grid = 0;             // CTAs of the persistent reverse kernels (0: one per SM)
    cudaEvent_t ev_roll = nullptr;
    std::vector<cudaEvent_t> ev_stage;
    std::vector<cudaEvent_t> ev_tan;   // matrix-free: stage k of the rollout is done (tangent pass of k may start)
    cudaStream_t tan_stream = nullptr;  // matrix-free: the tangent pass (highest priority)
    cudaEvent_t ev_tan_done = nullptr;
    cudaStream_t tan_side = nullptr;    // matrix-free: the edge-encoder tangents beside the node encoder's
    cudaEvent_t ev_tfork = nullptr, ev_tjoin = nullptr;
    // launch timing of the reverse edge-update MLP (events around each launch of the last step)
    bool ktiming = false;
    int kev_n = 0;
    std::vector<std::array<cudaEvent_t, 2>> kev;
    std::vector<double> kev_bytes, kev_flops;
    std::vector<int> kev_ctas;   // CTAs of each timed launch (fewer than the SMs while the rollout runs beside it)
    // stage timeline of the overlapped rollout and tangent pass: sev[0] where both start,
    // sev[1 + k] after rollout stage k, sev[1 + N + k] after tangent stage k (timing events)
    bool stiming = false;
    std::vector<cudaEvent_t> sev;

    ~gm_ctx() {
        for (auto& e : kev)
            for (auto ev : e) cudaEventDestroy(ev);
        for (auto ev : sev) cudaEventDestroy(ev);
        for (auto& e : events)
            for (auto ev : e) cudaEventDestroy(ev);
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (cond_stream) cudaStreamDestroy(cond_stream);
        if (side_stream) cudaStreamDestroy(side_stream);
        if (roll_stream) cudaStreamDestroy(roll_stream);
        if (tan_stream) cudaStreamDestroy(tan_stream);
        if (tan_side) cudaStreamDestroy(tan_side);
        if (ev_tfork) cudaEventDestroy(ev_tfork);
        if (ev_tjoin) cudaEventDestroy(ev_tjoin);
        if (ev_tan_done) cudaEventDestroy(ev_tan_done);
        if (ev_roll) cudaEventDestroy(ev_roll);
        for (auto ev : ev_stage) cudaEventDestroy(ev);
        for (auto ev : ev_tan) cudaEventDestroy(ev);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
    }
};
