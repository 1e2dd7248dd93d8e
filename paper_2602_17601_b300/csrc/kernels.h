// Launchers shared between the .cu files of the library (internal).
#pragma once

#include "ctx.h"

namespace gmi {

// Tensor-core weight operands ([N rows][K] K-major BF16, three pieces) are stored tiled so that
// one bulk copy moves one K chunk of one piece: K in chunks of kc columns (the last chunk may be
// narrower), each chunk an N x kc block of 8 x 8 core matrices with element (n, k) at
// (n/8)*8*kc + (k/8)*64 + (n%8)*8 + k%8.  kc = 64, except 32 for second-product operands
// wider than 128 rows, whose chunks must still fit the 128 x 64 staging buffer.
constexpr int TC_CHUNK = 64;
inline __host__ __device__ int tc_chunk_b2(int rows) { return rows > 128 ? TC_CHUNK / 2 : TC_CHUNK; }
// forward (rollout) MLPs: K chunk width and weight/A buffers.  Measured on the chain of 1000
// (rollout phase): 64 / 1: 3.35 ms; 64 / 2: 4.07 ms; 32 / 2: 4.25 ms; 32 / 3: 4.47 ms
constexpr int TC_CHUNK_F = 64;
constexpr int TC_NBUF_F = 1;
constexpr int TC_NBUF_MAX = 2;   // buffers the tile state tracks
constexpr int TC_NBUF_SMALL = 2; // reverse-mode launches of at most one tile per SM (mixed form, W = 128)
static_assert(TC_NBUF_F <= TC_NBUF_MAX, "forward chunk buffers exceed the tile state");
inline __host__ __device__ int tc_chunk_b2_fwd(int rows) { return rows > 128 ? TC_CHUNK_F / 2 : TC_CHUNK_F; }
inline __host__ __device__ long tc_tile_off(int n, int k, int kc) {
    return (long)(n >> 3) * 8 * kc + (k >> 3) * 64 + (n & 7) * 8 + (k & 7);
}

// gnn.cu
gm_status gnn_rollout(gm_ctx* c, const float* x0, const float* u_hat, float* x_hat, cudaStream_t st);
gm_status gnn_rollout_steps(gm_ctx* c, const float* x0, const float* u_hat, float* x_hat, int n_steps,
                            cudaStream_t st);
gm_status gnn_jacobians(gm_ctx* c, const float* x_hat, const float* u_hat, float* A, float* B,
                        float* cvec, cudaStream_t st);
// rollout and Jacobians with the reverse pass of each stage chunk overlapping the rollout of
// the later stages (rollout on the context's high-priority stream, joined back into st)
gm_status gnn_linearize(gm_ctx* c, const float* x0, const float* u_hat, float* x_hat, float* A, float* B,
                        float* cvec, cudaStream_t st);

// condense.cu
// Packed stage-major rows (a stage-k row has k nu leading non-zeros) for Gram products.
struct GramRows {
    const float* X;         // packed rows
    int rows_per_stage;     // rows of one stage (M*6 or M*n_c)
    int nu, N;
    const float* wts;       // weights, index (k - wts_k0) * rows_per_stage + r (nullable: 1)
    int wts_k0 = 0;         // first stage the weight array covers
    int wts_square = 0;     // use w*w instead of w
};
gm_status gram(gm_ctx* c, const GramRows& R, int nsplit, const float* diag_add, float diag_scale,
               float* G, cudaStream_t st);
__global__ void gram_kernel(GramRows R, int n, float* __restrict__ part);
// Partial Gram sums over nsplit row shares into part [nsplit][T][T][32 x 32] (T = ceil(n/32));
// gram_split picks nsplit (at most cap): one share per SM for the tensor-core form (tc and
// n <= 256, gram_tc.cu), about two CTAs per SM for the FP32 SIMT kernel otherwise.  A
// context's partial buffer holds kGramSplitCap shares.  launch_gram takes the same tc.
// Final node latents of stage 0 into c->d_h; their pooled features (warm start, ws.cu).
gm_status gnn_latents(gm_ctx* c, const float* x0, const float* u0, cudaStream_t st);
gm_status ws_features(gm_ctx* c, const float* h, const float* x_ref, float* feat, cudaStream_t st);
int gram_blocks(int n);
constexpr int kGramSplitCap = 160;
int gram_split(int n, int sms, int cap, bool tc);
gm_status launch_gram(const GramRows& R, int n, int nsplit, float* part, cudaStream_t st, int* status, bool tc);
bool gram_tc_ok(int n);
gm_status launch_gram_tc(const GramRows& R, int n, int nsplit, float* part, int* status, cudaStream_t st);
// qp.cu: row scales 1/|C~_r| and the FP64 KKT certificate of (U, y)
__global__ void row_norm_kernel(long rows, int nu, int Mnc, const float* __restrict__ Ct, float* __restrict__ rs);
__global__ void kkt_rows_kernel(int n, int nu, int Mnc, long rows, const float* __restrict__ Ct,
                                const float* __restrict__ dt, const float* __restrict__ U,
                                const float* __restrict__ y, double* kkt);
// The FP64 stationarity rows (one warp per row, in place of kkt[0..n)), then the certificate's maxima
// and the final status into stats (S nullable: records the final status, GM_STALLED).
gm_status launch_kkt_final(int n, const float* H, const float* g, const float* lo, const float* hi, const float* U,
                           const float* y, double* kkt, const int* status, gm_stats* stats, AdmmState* S,
                           cudaStream_t st);
// barrier.cu: relaxed log-barrier obstacle rows folded into H and g
gm_status barrier_fold(gm_ctx* c, const float* Ct, const float* dt, const float* U_hat, float mu, float delta,
                       float* H, float* g, cudaStream_t st);
// ipm.cu: interior-point solve of the condensed QP
gm_status ipm_solve(gm_ctx* c, const float* H, const float* g, const float* Ct, const float* dt, const float* u_lo,
                    const float* u_hi, int max_iter, float* U, float* y, gm_stats* stats, cudaStream_t st);
// G = the sum of nsplit partial Grams (launch_gram's tile layout) + diag_scale * diag_add on the
// diagonal (diag_add nullable); G is written in full and exactly symmetric.
constexpr int GR_WARPS = 8;
gm_status launch_gram_reduce(int n, int nsplit, const float* part, const float* diag_add, float diag_scale, float* G,
                             cudaStream_t st);
gm_status sphere_halfspaces(gm_ctx* c, const float* x_hat, const float* spheres, int S, float* Cx,
                            float* dx, cudaStream_t st);
gm_status condense(gm_ctx* c, const float* x_hat, const float* A, const float* B, const float* cvec,
                   const gm_cost* cost, const float* Cx, const float* dx, float* H, float* g,
                   float* Ct, float* dt, cudaStream_t st);
// H, g, C~, d~ from Gamma_u (c->d_Gu) and the offset form of Gamma_x (c->d_Gx) as they stand
gm_status condense_tail(gm_ctx* c, const float* x_hat, const gm_cost* cost, const float* Cx, const float* dx,
                        float* H, float* g, float* Ct, float* dt, cudaStream_t st);
// Gamma_u block row k (k >= 1) of node i, component a, column t: d_Gu[gu_offset(M, nu, k) + (i 6 + a) k nu + t]
__host__ __device__ inline long gu_offset(int M, int nu, int k) {
    return (long)M * 6 * nu * ((long)k * (k - 1) / 2);
}
// gnn.cu (matrix-free condensing): Gamma_u stages 1..N and the offset D_k = Gamma_x_k - x_hat_k
// from forward-mode products along the rollout (its ReLU masks in c); needs gm_settings.condensing = 1
gm_status gnn_sensitivities(gm_ctx* c, const float* u_hat, cudaStream_t st);
// the rollout (x_hat) and the sensitivities, the tangent pass of each stage beside the rollout of
// the later stages
gm_status gnn_rollout_sensitivities(gm_ctx* c, const float* x0, const float* u_hat, float* x_hat,
                                    cudaStream_t st);

// qp.cu
// ev_mid (nullable) is recorded between the set-up (P, Cholesky, inverse) and the iterations;
// keep_rho starts from the rho the previous solve on c ended with.
gm_status qp_solve(gm_ctx* c, const float* H, const float* g, const float* Ct, const float* dt,
                   const float* u_lo, const float* u_hi, const float* warm_U, const float* warm_y,
                   float* U, float* y, gm_stats* stats, cudaStream_t st, cudaEvent_t ev_mid = nullptr,
                   bool keep_rho = false);

size_t admm_smem_bytes(const gm_ctx* c);
const void* admm_kernel_ptr(const gm_ctx* c);

// small device utilities (api.cu)
gm_status shift_inputs(gm_ctx* c, const float* U, float* u_hat, cudaStream_t st);
gm_status shift_duals(gm_ctx* c, const float* y, float* yw, cudaStream_t st);

}  // namespace gmi
