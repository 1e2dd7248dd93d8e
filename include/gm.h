/*
 * gm.h — C ABI of the B300 (sm_103a) GNN-MPC real-time-iteration library.
 *
 * One real-time iteration (Algorithm 1, one pass of its outer loop) of
 * Graph Neural MPC: roll the GNN dynamics model out along the horizon,
 * linearise it (Eq. linearized_dynamics), condense the states out with the
 * per-node recursion of the Thm. 1 proof (Eq. sparse_gamma_i_xb,
 * Eq. sparse_gamma_i_u, Eq. H, Eq. g and the stacked constraints), and solve
 * the dense condensed QP (Eq. condensed_matrices) with ADMM.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns a gm_status.  On failure gm_last_error() returns
 *   a message for the calling thread; outputs are then unspecified.
 * - Handles are opaque.  gm_graph and gm_gnn live in host memory only.
 *   gm_ctx lives in host memory and in a caller-provided device workspace;
 *   the library itself never allocates device memory.
 * - Array arguments of the compute calls are DEVICE pointers (float32 unless
 *   noted), read or written in stream order on the given stream
 *   (cudaStream_t passed as void*; NULL = legacy default stream).  Inputs
 *   are only read during the call's kernels; outputs are caller-owned and
 *   must not alias inputs.  The calls are asynchronous: results are valid
 *   once the stream has reached them.
 * - Indices are 0-based int32.  Node states are x^i = (p^i, v^i) in R^6
 *   (position then velocity, Sec. V-A "Model").
 * - Errors: GM_ERR_INVALID_ARG for bad sizes / NULL pointers / workspace too
 *   small, GM_ERR_CUDA when a CUDA call fails (message holds the CUDA
 *   error string).  There is no CPU fallback: without a CUDA device every
 *   compute call returns GM_ERR_CUDA.
 */
#ifndef GM_H
#define GM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int gm_status;
#define GM_OK                 0
#define GM_ERR_INVALID_ARG    1
#define GM_ERR_CUDA           2
#define GM_ERR_WORKSPACE      3   /* workspace missing, too small or misaligned */
#define GM_ERR_NOT_CONVERGED  4   /* ADMM hit max_iter; U holds the last iterate */
#define GM_STALLED            5   /* warm-started ADMM stalled; cold restart used */
#define GM_ERR_TIMEOUT        6   /* a bounded device-side wait gave up */
#define GM_ERR_NUMERIC        7   /* NaN/Inf or a non-positive pivot */
#define GM_ERR_INFEASIBLE     8   /* ADMM found a certificate that no U satisfies the constraints */

/* Precision forms of the step. */
#define GM_PREC_FP32   0   /* every GNN, Jacobian, condensing and ADMM op in FP32 (SIMT);
                              Cholesky of rho I + H (+ rho C~'C~) and the KKT check in FP64 */
#define GM_PREC_MIXED  1   /* GNN MLPs and Jacobian products on tcgen05 tensor cores with
                              split BF16 operands (x = hi + lo, three products, FP32
                              accumulate: about FP32 accuracy); the rest as GM_PREC_FP32 */
#define GM_PREC_BF16   2   /* as GM_PREC_MIXED with one BF16 product (hi parts only):
                              about 1e-2 relative error in the Jacobians */

typedef struct gm_graph gm_graph;
typedef struct gm_gnn gm_gnn;
typedef struct gm_ctx gm_ctx;

/* Thread-local message of the last failing call ("" if none). */
const char* gm_last_error(void);
/* Library version string. */
const char* gm_version(void);

/* ------------------------------------------------------------------------
 * gm_graph_create — the interaction graph G = (V, E) (Sec. III-A) with the
 * actuator attachment.
 *   M          number of nodes (subsystems), M >= 1
 *   E          number of directed edges, E >= 0
 *   src, dst   HOST int32 [E]: edge k carries node src[k]'s state to node
 *              dst[k] (e^{ij} with j = src, i = dst; N_i = { j : (j -> i) }).
 *              Self-loops and duplicates are rejected (GM_ERR_INVALID_ARG).
 *   nu         number of inputs, nu >= 1
 *   act_node   HOST int32 [nu]: input a enters the node update of node
 *              act_node[a] (node input [x^i, m^i * u], m^i one-hot).
 * The arrays are copied; the caller keeps ownership.
 * ---------------------------------------------------------------------- */
gm_status gm_graph_create(int M, int E, const int32_t* src, const int32_t* dst,
                          int nu, const int32_t* act_node, gm_graph** out);
void gm_graph_destroy(gm_graph* g);

/* ------------------------------------------------------------------------
 * gm_gnn_load — the GNN dynamics model (Sec. V-A "Model", Eq. forward_dynamics)
 * in encode-process-decode form with K message-passing steps:
 *   h^0_i = MLP_ne([x^i, m^i u]),  e^0_ij = MLP_ee(x^i - x^j),
 *   e^l_ij = e^{l-1}_ij + MLP_el([h^{l-1}_i, h^{l-1}_j, e^{l-1}_ij]),
 *   h^l_i  = h^{l-1}_i + MLP_nl([h^{l-1}_i, sum_{j->i} e^l_ij]),
 *   dv^i = MLP_d(h^K_i),  v+ = v + dv,  p+ = p + dt v+.
 * Every MLP is Linear-ReLU-Linear with hidden width W; ReLU'(0) = 0.
 *   desc.K >= 1, desc.W in {32, 64, 128}, desc.nu >= 1, desc.dt > 0.
 *   blob   HOST float32 [n]: MLPs in the order node encoder (6+nu->W->W),
 *          edge encoder (6->W->W), then per step edge update (3W->W->W) and
 *          node update (2W->W->W), then decoder (W->W->3); inside each MLP
 *          W1 [in][W] row-major, b1 [W], W2 [W][out] row-major, b2 [out].
 *          n must equal that total (GM_ERR_INVALID_ARG otherwise).
 * ---------------------------------------------------------------------- */
typedef struct {
    int K;
    int W;
    int nu;
    float dt;
} gm_gnn_desc;

gm_status gm_gnn_load(const gm_gnn_desc* desc, const float* blob, size_t n,
                      gm_gnn** out);
void gm_gnn_destroy(gm_gnn* m);

/* ------------------------------------------------------------------------
 * Settings of a context.
 *   N          horizon (>= 1)
 *   n_c        position half-spaces per node and stage (stages 1..N), >= 0
 *   precision  GM_PREC_FP32 or GM_PREC_MIXED
 *   rho        ADMM penalty (fixed, > 0)
 *   tol        ADMM stop: |A~U - z|_inf <= tol and dual residual <= tol
 *   max_iter   ADMM iteration cap (>= 1)
 *   polish     1: after ADMM, re-solve the equality QP on the guessed active
 *              set in FP64 and keep it if its KKT certificate is better
 *   timeout_spins  cap on every device-side spin-wait (0 = default)
 *   scale_rows 1: ADMM runs on the half-space rows divided by their 2-norms
 *              (same feasible set and U*; multipliers are returned for the
 *              original rows).  Rows of C~ can be many orders of magnitude
 *              smaller than 1, and unscaled fixed-rho ADMM stalls on them.
 *   adapt_rho  1: every 25 iterations compare the primal and dual residuals,
 *              each relative to its scale, and re-factor P with
 *              rho sqrt(ratio) (clamped to [1e-6, 1e6]) when that changes rho
 *              by more than 5x, at most 5 times per solve; 0: fixed rho.
 *   admm_grid    CTAs of the cooperative ADMM kernel (0: one per resident slot
 *                on every SM); smaller grids let batched instances run side by side
 *   factor_grid  CTAs of the cooperative FP64 factor kernel (0: 128)
 *   chunk_mb     device memory budget of the reverse-pass cotangent buffers in
 *                MB (0: 16384, and at most a quarter of the horizon per chunk);
 *                fewer stages per launch group when smaller.  gm_linearize and
 *                gm_rti_step run the rollout on a high-priority internal stream
 *                and the reverse pass of each chunk as soon as its stages are
 *                rolled out, beside the rollout of the later stages (with at
 *                most SMs - ceil(E/128) CTAs per persistent reverse launch until
 *                the rollout ends)
 *   condensing   0: local Jacobians A_k, B_k, c_k by the reverse pass and the
 *                recursion of Thm. 1 (Eq. sparse_gamma_i_u); 1: matrix-free: the
 *                sensitivities d x_k / d U pushed through the GNN by forward-mode
 *                products, one tangent per input column on its support (the
 *                nodes the column's actuator reaches in K (k - i) edges), no A_k
 *                formed; the same H, g, C~, d~ up to rounding.  Used by
 *                gm_rti_step and gm_condense_matrix_free.
 *   tan_split_rows  matrix-free condensing: the tangent edge rows of a message-
 *                passing layer from which its first layer runs on per-node
 *                projections of its two node blocks (one product per node row,
 *                K = W per edge row) instead of whole (K = 3W per edge row);
 *                0: 30000; 1: every layer.  >= 0.
 * ---------------------------------------------------------------------- */
typedef struct {
    int N;
    int n_c;
    int precision;
    float rho;
    float tol;
    int max_iter;
    int polish;
    int timeout_spins;
    int scale_rows;
    int adapt_rho;
    int admm_grid;
    int factor_grid;
    int chunk_mb;
    int condensing;
    int tan_split_rows;
} gm_settings;

/* Per-solve statistics, written to DEVICE memory by the QP calls. */
typedef struct {
    int32_t status;       /* gm_status of the solve */
    int32_t iters;        /* ADMM iterations (U updates) */
    int32_t converged;    /* 1 if both ADMM residuals reached tol */
    int32_t polished;     /* 1 if the polished solution was kept */
    float r_prim;         /* last ADMM primal residual |A~U - z|_inf */
    float r_dual;         /* last ADMM dual residual */
    double kkt_stat;      /* FP64 |H U + g + A~'y|_inf of the returned (U, y) */
    double kkt_prim;      /* FP64 max bound violation of A~U */
    double kkt_dual;      /* FP64 wrong-sign multiplier magnitude */
    double kkt_comp;      /* FP64 max |y_r| * slack_r */
} gm_stats;

/* ------------------------------------------------------------------------
 * gm_ctx_workspace_size / gm_ctx_create — a context binds a graph, a GNN and
 * settings, and owns (inside the caller's device workspace) the device copy
 * of both, the Jacobian sparsity pattern, every intermediate of the step and
 * the linearisation inputs u_hat carried between steps (Algorithm 1).
 *   workspace  DEVICE pointer, 256-byte aligned, >= the reported size; the
 *              caller keeps ownership and frees it after gm_ctx_destroy.
 *   stream     stream on which the static data is uploaded.
 * gm_ctx_create copies graph and GNN; they may be destroyed afterwards.
 * ---------------------------------------------------------------------- */
gm_status gm_ctx_workspace_size(const gm_graph* g, const gm_gnn* m,
                                const gm_settings* s, size_t* bytes);
gm_status gm_ctx_create(const gm_graph* g, const gm_gnn* m, const gm_settings* s,
                        void* workspace, size_t bytes, void* stream, gm_ctx** out);
void gm_ctx_destroy(gm_ctx* ctx);

/* ------------------------------------------------------------------------
 * gm_jac_pattern — block sparsity of A_k (Assumption 1 with a K-step GNN):
 * block row i holds A^{ij} for every j with a directed path of at most K
 * edges into i (including i), columns ascending.  HOST arrays owned by the
 * context: row_ptr [M+1], col [nnzb].
 * ---------------------------------------------------------------------- */
gm_status gm_jac_pattern(const gm_ctx* ctx, int* nnzb, const int32_t** row_ptr,
                         const int32_t** col);

/* ------------------------------------------------------------------------
 * gm_rollout — the GNN dynamics alone (Eq. forward_dynamics): x_out[0] = x0,
 * x_out[k+1] = F(x_out[k], u[k]) for k < n_steps (1 <= n_steps <= N); the
 * plant of a closed loop that uses the model itself, or a prediction.
 *   x0 [M][6], u [n_steps][nu], x_out [n_steps+1][M][6] (out; may alias x0
 *   at its first block).  Shares the context's scratch with the other calls.
 * ---------------------------------------------------------------------- */
gm_status gm_rollout(gm_ctx* ctx, const float* x0, const float* u, int n_steps, float* x_out, void* stream);

/* ------------------------------------------------------------------------
 * gm_linearize — rollout and local Jacobians (Eq. forward_dynamics,
 * Eq. linearized_dynamics; Algorithm 1 "Linearize GNN dynamics").
 *   x0     [M][6]                measured state x~(t)
 *   u_hat  [N][nu]               linearisation inputs
 *   x_hat  [N+1][M][6]   (out)   x_hat_0 = x0, x_hat_{k+1} = F(x_hat_k, u_hat_k)
 *   A      [N][nnzb][6][6] (out) A^{ij}_k = d f^i / d x^j at (x_hat_k, u_hat_k),
 *                                blocks in gm_jac_pattern order, row-major 6x6
 *   B      [N][M][6][nu]   (out) B^i_k = d f^i / d u_k
 *   c      [N][M][6]       (out) c^i_k = x_hat^i_{k+1} - sum_j A^{ij}_k x_hat^j_k - B^i_k u_hat_k
 * Any of A, B, c may be NULL to skip writing it.
 * ---------------------------------------------------------------------- */
gm_status gm_linearize(gm_ctx* ctx, const float* x0, const float* u_hat, float* x_hat,
                       float* A, float* B, float* c, void* stream);

/* Cost of Eq. linear_gnn_mpc_ocp_explicit (diagonal Q^i_k, R_k). */
typedef struct {
    const float* Qdiag;   /* [N+1][M][6]  diagonal of Q^i_k, >= 0 */
    const float* Rdiag;   /* [N][nu]      diagonal of R_k, > 0 */
    const float* x_ref;   /* [N+1][M][6]  x^{i,r}_k */
    const float* u_ref;   /* [N][nu]      u^r_k */
} gm_cost;

/* Constraints: input box U_k and node-position half-spaces X^i_k. */
typedef struct {
    const float* u_lo;    /* [N][nu] */
    const float* u_hi;    /* [N][nu], u_lo <= u_hi */
    const float* Cx;      /* [N][M][n_c][3]  C^{x,i}_k acting on p^i_k, stages k = 1..N (nullable if n_c = 0) */
    const float* dx;      /* [N][M][n_c]     d^{x,i}_k */
    int n_spheres;        /* > 0: ignore Cx/dx and linearise these spheres at x_hat instead
                             (requires n_c == n_spheres) */
    const float* spheres; /* [n_spheres][4]  centre xyz, radius */
    float barrier_mu;     /* > 0: gm_rti_step puts the state rows (spheres or Cx/dx) into the
                             cost as relaxed log barriers of weight barrier_mu (gm_barrier_fold)
                             instead of constraints; 0: constraints */
    float barrier_delta;  /* relaxation point of the barrier (> 0 when barrier_mu > 0) */
} gm_constr;

/* ------------------------------------------------------------------------
 * gm_condense — the condensed QP (Eq. condensed_matrices) by the per-node
 * recursion (Eq. sparse_gamma_i_xb, Eq. sparse_gamma_i_u) and per-node
 * aggregation (Eq. H, Eq. g, stacked C~ / d~), in the convention
 *     min 1/2 U'HU + g'U   s.t.  u_lo <= U <= u_hi,  C~ U <= d~
 * with H = Gu' Qbar Gu + Rbar and g = Gu' Qbar (Gx - x_ref) - Rbar u_ref
 * (one half of the paper's objective; same minimiser).
 *   x_hat, A, B, c   as produced by gm_linearize (A in gm_jac_pattern order)
 *   H   [nU][nU]  (out) nU = N nu, row-major, symmetric
 *   g   [nU]      (out)
 *   Ct  (out) packed stage-major rows: stage k = 1..N holds M n_c rows of
 *             length k nu (row (k, i, c) at float offset
 *             M n_c nu k(k-1)/2 + (i n_c + c) k nu); total M n_c nu N(N+1)/2.
 *             Columns >= k nu of a stage-k row are zero and not stored.
 *   dt  [N][M][n_c]  (out)
 * Ct and dt may be NULL when n_c == 0.
 * ---------------------------------------------------------------------- */
gm_status gm_condense(gm_ctx* ctx, const float* x_hat, const float* A, const float* B,
                      const float* c, const gm_cost* cost, const gm_constr* cons,
                      float* H, float* g, float* Ct, float* dt, void* stream);

/* ------------------------------------------------------------------------
 * gm_condense_matrix_free — the condensed QP of gm_condense without local
 * Jacobians (needs a context created with gm_settings.condensing = 1): the
 * rollout x_hat from x0 along u_hat (Eq. forward_dynamics), then the
 * sensitivities Gamma_u = d x / d U by forward-mode products through the GNN
 * at the rollout, one tangent per input column restricted to the nodes its
 * actuator reaches (the product A_k S_k + B_k E_k of Eq. sparse_gamma_i_u as one
 * directional derivative of the stage map), Gamma_x = x_hat - Gamma_u u_hat,
 * and H, g, C~, d~ as gm_condense (spheres of cons linearised at x_hat).
 *   x0 [M][6], u_hat [N][nu]; x_hat [N+1][M][6] (out); H, g, Ct, dt as gm_condense.
 * GM_ERR_INVALID_ARG on a context created with condensing = 0.
 * ---------------------------------------------------------------------- */
gm_status gm_condense_matrix_free(gm_ctx* ctx, const float* x0, const float* u_hat, const gm_cost* cost,
                                  const gm_constr* cons, float* x_hat, float* H, float* g, float* Ct, float* dt,
                                  void* stream);

/* ------------------------------------------------------------------------
 * gm_qp_solve — ADMM on the condensed QP (no relaxation):
 *   P = H + rho (I + C~'S^2 C~) (S the row scaling when settings.scale_rows),
 *   factored in FP64 (Cholesky) once, and again after each adaptive rho
 *   update (settings.adapt_rho: every 25 iterations, at most 5 updates);
 *   per iteration U = P^{-1}(A~'(rho z - y) - g), a = A~U,
 *   z = clip(a + y/rho, l, h), y += rho (a - z), with A~ = [I; C~],
 *   l = [u_lo; -inf], h = [u_hi; d~]; stop when |a - z|_inf <= tol and the
 *   dual residual |H U + g + A~'y|_inf <= tol.  Then optional FP64 polish and
 *   the FP64 KKT certificate into stats.
 *   Every 10th iteration tests the primal-infeasibility certificate of
 *   Banjac et al. (2019) on the dual step dy = y - y_prev (scaled rows):
 *   |A~'dy|_inf <= 1e-4 |dy|_inf, dy >= -1e-4 |dy|_inf on rows whose lower
 *   bound is -inf (and dy <= 1e-4 |dy|_inf where the upper bound is +inf),
 *   and h'max(dy, 0) + l'min(dy, 0) <= -1e-4 |dy|_inf over the finite
 *   bounds; when it holds no U satisfies the constraints, ADMM stops and
 *   stats->status is GM_ERR_INFEASIBLE (U holds the last iterate).
 *   H, g, Ct, dt, u_lo, u_hi  as from gm_condense / gm_constr; Ct = dt = NULL
 *     solves the box-only QP (the barrier variant) even when n_c > 0
 *   warm_U [nU], warm_y [nU + N M n_c]  nullable warm start (U^0, y^0).  A
 *     warm-started solve watches its residual: when max(r_p, r_d) has not
 *     fallen below half of its value 25 iterations earlier (a stall), or an
 *     iterate turns NaN, it drops the warm start and restarts cold (U^0 = 0,
 *     y^0 = 0, rho = settings.rho, P re-factored) inside the same call; a
 *     restart that converges reports stats->status = GM_STALLED, and
 *     stats->iters counts both parts.  A warm start may change rho once.
 *   U [nU] (out), y [nU + N M n_c] (out, nullable)  multipliers, box rows first
 *   stats  DEVICE gm_stats* (out, nullable)
 * Returns GM_OK even when ADMM did not converge; stats->status says so.
 * ---------------------------------------------------------------------- */
gm_status gm_qp_solve(gm_ctx* ctx, const float* H, const float* g, const float* Ct,
                      const float* dt, const float* u_lo, const float* u_hi,
                      const float* warm_U, const float* warm_y, float* U, float* y,
                      gm_stats* stats, void* stream);

/* ------------------------------------------------------------------------
 * gm_barrier_fold — barrier-cost obstacle variant (Sec. VI-B: one barrier
 *   term per node and obstacle in the cost; the paper gives no formula).
 *   Row r of the condensed constraints gives the clearance
 *   s_r(U) = d~_r - C~_r U (for spheres: the distance to the sphere along
 *   the normal at the rollout).  Each row adds mu beta(s_r) to the cost,
 *   beta the relaxed logarithmic barrier of Feller and Ebenbauer (2017):
 *   -ln s for s > delta, 1/2 (((s - 2 delta)/delta)^2 - 1) - ln delta
 *   below (convex, twice continuously differentiable, finite for s <= 0).
 *   s_r is affine in U, so the second-order model at U_hat is exact to second
 *   order; this call folds it into the QP in place:
 *     H <- H + C~' diag(mu beta''(s^)) C~
 *     g <- g - C~' (mu beta'(s^) + mu beta''(s^) C~ U_hat),  s^ = d~ - C~ U_hat
 *   after which gm_qp_solve with Ct = dt = NULL solves the box-only QP: one
 *   Newton step on the barrier-augmented cost under the input box.
 *   Ct, dt   DEVICE, as from gm_condense (n_c > 0; with n_c = 0 nothing changes)
 *   U_hat    DEVICE [nU] the linearisation point (the shifted previous solution)
 *   mu > 0, delta > 0, else GM_ERR_INVALID_ARG
 *   H [nU][nU], g [nU]  DEVICE, updated in place
 *   Uses the context's interior-point scratch (not concurrently with
 *   gm_qp_solve_ipm on the same context).  FP64 row terms and C~' v, FP32
 *   weighted Gram (as for rho C~'C~ in gm_qp_solve).
 * ---------------------------------------------------------------------- */
gm_status gm_barrier_fold(gm_ctx* ctx, const float* Ct, const float* dt, const float* U_hat,
                          float mu, float delta, float* H, float* g, void* stream);

/* ------------------------------------------------------------------------
 * gm_qp_solve_ipm — the same QP by a primal-dual interior-point method (the
 *   solver class of the paper's controller, Sec. VI-A), for comparison with
 *   ADMM: Mehrotra predictor-corrector on G U <= h with G = [I; -I; S C~],
 *   h = [u_hi; -u_lo; S d~] (S the row scales 1/|C~_r|), slacks s > 0 and
 *   duals z > 0.  Each iteration forms Phi = H + G'diag(z/s)G (FP32 Gram),
 *   factors it in FP64 and solves the predictor and corrector systems in
 *   FP64.  Stops when |G U + s - h|_inf, |H U + g + G'z|_inf and max_i s_i z_i
 *   are all <= settings.tol, or after max_iter iterations (1..1000).
 *   Arguments as gm_qp_solve (no warm start); y [nU + N M n_c] (out, nullable)
 *   receives z_hi - z_lo for the box rows and S z for the half-space rows.
 *   stats: iters, converged, r_prim = |r_p|_inf, r_dual = |r_d|_inf of the
 *   last iterate, and the FP64 KKT certificate of (U, y).  The host reads a
 *   device flag every two iterations (stream synchronisation), so this call
 *   cannot be captured into a CUDA graph.
 * Returns GM_OK even when it did not converge; stats->status says so.
 * ---------------------------------------------------------------------- */
gm_status gm_qp_solve_ipm(gm_ctx* ctx, const float* H, const float* g, const float* Ct,
                          const float* dt, const float* u_lo, const float* u_hi, int max_iter,
                          float* U, float* y, gm_stats* stats, void* stream);

/* ------------------------------------------------------------------------
 * gm_rti_step — one iteration of Algorithm 1 on the device:
 *   u_hat <- context trajectory (zero after gm_ctx_create / gm_ctx_reset,
 *            else the shifted previous solution (U*_1..U*_{N-1}, U*_{N-1}));
 *   x_hat <- rollout of x_meas; linearise; (spheres -> half-spaces at x_hat);
 *   condense; ADMM (+ polish, KKT certificate); store U* for the next shift.
 *   x_meas [M][6]      measured state x~(t)
 *   U      [N][nu]     (out) U*
 *   u0     [nu]        (out, nullable) first input to apply
 *   stats  DEVICE gm_stats* (out, nullable)
 * ---------------------------------------------------------------------- */
gm_status gm_rti_step(gm_ctx* ctx, const float* x_meas, const gm_cost* cost,
                      const gm_constr* cons, float* U, float* u0, gm_stats* stats,
                      void* stream);

/* Reset the carried linearisation inputs u_hat to zero (Algorithm 1 "Initialize"). */
gm_status gm_ctx_reset(gm_ctx* ctx, void* stream);

/* ------------------------------------------------------------------------
 * Measurement helpers (no counterpart in the paper's method; they report on
 * the calls above).
 * ---------------------------------------------------------------------- */

/* Sizes and algorithmic work of one step of this context (host, no GPU work).
 * flops_* count 2 x the multiply-adds of the products the kernels perform
 * (the reverse-mode Jacobian counts the cone rows it actually processes);
 * bytes_* count the bytes a pass must move at least once. */
typedef struct {
    int M, E, nu, K, W, N, n_c, nU;
    int nnzb;                     /* blocks of the Jacobian pattern */
    long long rows_c;             /* half-space rows of C~ */
    long long cone_node_rows;     /* (seed, node) rows over all reverse levels */
    long long cone_edge_rows;     /* (seed, edge) rows over all reverse levels */
    double flops_rollout;         /* per step: N GNN forwards */
    double flops_jacobian;        /* per step: reverse pass over all stages */
    double flops_condense;        /* per step: recursion + H + g + C~ */
    double flops_qp_setup;        /* per step: C~'C~, Cholesky, inverse */
    double flops_admm_iter;       /* per ADMM iteration */
    double bytes_admm_iter;       /* per ADMM iteration: C~, d~, z, y */
    size_t workspace_bytes;
    int stage_chunk;              /* stages per reverse-pass launch group */
    int admm_grid;                /* CTAs of the persistent ADMM kernel */
} gm_info;

gm_status gm_ctx_info(const gm_ctx* ctx, gm_info* out);

/* Phase timing: when on, gm_rti_step records CUDA events on its stream at the
 * boundaries of rollout, Jacobians, condensing, QP set-up (C~'C~, Cholesky,
 * inverse) and ADMM + KKT check.  gm_ctx_phase_ms waits for the recorded
 * events, writes the summed milliseconds of the 5 phases and the number of
 * recorded steps, and clears the record. */
gm_status gm_ctx_set_timing(gm_ctx* ctx, int on);
gm_status gm_ctx_phase_ms(gm_ctx* ctx, float* ms5, int* steps);

/* Arithmetic peaks of the current device for the roofline of the FP32 and FP64
 * kernels: FP32 and FP64 fused multiply-add throughput (TFLOP/s, 2 flops per
 * FMA) of independent FMA chains in every lane of 8 CTAs of 256 threads per
 * SM, timed with CUDA events on stream (which the call synchronises), and the
 * L2 size in bytes (cudaDevAttrL2CacheSize). */
gm_status gm_measure_peaks(double* fp32_tflops, double* fp64_tflops, long long* l2_bytes, void* stream);

/* HBM rates of three streams over a caller-owned device buffer buf of bytes
 * (16-byte aligned, at least 64 MB; use well above the L2 size): read-only
 * (the first half), write-only (the second half) and copy (first half to
 * second), 16-byte accesses, CUDA events on stream (which the call
 * synchronises), best of repeats after one warm-up; GB/s counts the bytes read
 * plus written.  The buffer is overwritten with zeros.  For the roofline of
 * kernels whose traffic is mostly reads or mostly writes, beside the copy peak. */
gm_status gm_measure_hbm(void* buf, size_t bytes, int repeats, double* read_gbs, double* write_gbs,
                         double* copy_gbs, void* stream);

/* Number of CUDA kernels this library has launched in this process. */
unsigned long long gm_launch_count(void);

/* CUDA-graph replay of gm_rti_step (no paper counterpart: a launch-overhead
 * measure for the real-time loop).  When on, the first gm_rti_step runs as
 * usual; the next one is captured once into a CUDA graph (on an internal
 * stream) and every later call replays that graph on the caller's stream.
 * The graph bakes in every pointer and scalar of the call (x_meas, cost,
 * constraints, U, u0, stats, settings); a call that changes any of them is
 * captured anew.  Phase timing (gm_ctx_set_timing) runs the steps eagerly.
 * In the graph, the ADMM rounds after the first (rho adaptation, warm-start
 * restart) sit in nested conditional nodes that the device enables only while
 * the solve is not done, so a step that converges early launches none of
 * them; the eager step issues every round (the unneeded ones return at once).
 * If the capture fails the context falls back to eager steps and
 * gm_ctx_graph_state reports 0.  gm_ctx_graph_state: 1 when the last step
 * replayed a graph, 0 otherwise; captures counts the captures so far. */
gm_status gm_ctx_set_graph(gm_ctx* ctx, int on);

/* Receding-horizon warm start of gm_rti_step's ADMM (Algorithm 1 shifts the
 * solution into the next linearisation point; with on != 0 the QP solve
 * starts from it too): U^0 = u_hat (the previous U* shifted by one stage,
 * last stage repeated) and y^0 = the previous multipliers shifted alike, box
 * rows and half-space rows stage by stage, and rho starts where the previous
 * solve's adaptation left it.  After gm_ctx_reset all three are back to the
 * cold start (zeros, settings.rho).  Off by default.  The solve still runs to
 * settings.tol, so the optimum is the same; only the iteration count changes.
 * A stalled warm start restarts cold inside the step (gm_qp_solve, GM_STALLED).
 * After a step whose solve did not succeed (status other than GM_OK and
 * GM_STALLED) the next step starts its duals at zero and rho at settings.rho;
 * after GM_ERR_NUMERIC or GM_ERR_TIMEOUT, u_hat goes back to zero too
 * (Algorithm 1's initial trajectory), with or without the warm start. */
gm_status gm_ctx_set_warm(gm_ctx* ctx, int on);

/* Cap on the device-side spin-waits (grid barriers of the cooperative ADMM and
 * FP64 factor kernels) of this context's later calls, in polls; 0 restores the
 * default (2^26).  A wait that runs out makes its kernel record GM_ERR_TIMEOUT
 * in stats->status and return; the context stays usable.  spins < 0 is
 * GM_ERR_INVALID_ARG.  (No paper counterpart: failure detection.) */
gm_status gm_ctx_set_timeout_spins(gm_ctx* ctx, int spins);

/* Batched real-time iterations (no paper counterpart: many independent MPC
 * instances on one GPU).  A batch holds n contexts of any sizes (node count,
 * horizon, inputs, GNN); gm_batch_rti_step runs gm_rti_step on every instance
 * i with (x_meas[i], costs[i], cons[i], U[i], stats[i]).  The first call runs
 * the instances one after another with plain launches; the next captures
 * every instance's step as two child graphs of one parent graph: the part
 * without cooperative kernels (rollout, Jacobians, condensing) in up to 16
 * lanes planned by gm_batch_plan on cost (M * N * (1 + nU/64)), and the QP part
 * (set-up, the cooperative FP64 factorisation and ADMM grids, KKT check), which
 * follows the instance's first part and runs in one chain with the other
 * instances' QP parts, so that at most one cooperative grid is on the GPU at a
 * time.  Every later call with the same arguments replays that graph with a
 * single launch on the stream, the lanes running side by side.  Changing any
 * argument captures anew.  x_meas, U, stats: host arrays of n device pointers
 * (stats may be NULL); costs, cons: host arrays of n structs.  Contexts of a
 * batch must not be stepped elsewhere while the batch runs.  gm_batch_state:
 * as gm_ctx_graph_state. */
typedef struct gm_batch gm_batch;
gm_status gm_batch_create(gm_ctx* const* ctxs, int n, gm_batch** out);
void gm_batch_destroy(gm_batch* b);
gm_status gm_batch_rti_step(gm_batch* b, const float* const* x_meas, const gm_cost* costs, const gm_constr* cons,
                            float* const* U, gm_stats* const* stats, void* stream);
gm_status gm_batch_state(const gm_batch* b, int* replayed, int* captures);
/* Lanes of the last captured batch graph (1 before the first capture). */
gm_status gm_batch_lanes(const gm_batch* b, int* lanes);
/* At most this many lanes for the first parts in the next captured batch graph
 * (instance i in lane i mod lanes when fewer than gm_batch_plan's); 0 (the
 * default) keeps the plan.  lanes = 1 runs the instances one after another
 * inside one graph launch. */
gm_status gm_batch_set_lanes(gm_batch* b, int lanes);

/* Host-only lane plan for n instance steps that each run cooperative grids
 * of up to width[i] CTAs (one CTA per SM assumed) and cost cost[i] (any
 * unit).  Instances of one lane run one after another; lanes run side by
 * side.  The plan groups the widths into classes (each instance goes to the
 * narrowest class at least as wide as it; the narrowest classes merge into
 * wider ones until one lane per class fits in sms, and a width above sms
 * counts as sms), gives each class one lane and then adds lanes, one at a
 * time, to the class with the largest cost per lane while the sum of all
 * lanes' class widths stays <= sms and the class has more instances than
 * lanes; inside a class the costliest instance goes first to the least
 * loaded lane.  So at most one grid per lane runs at a time and the widths
 * of the running grids sum to <= sms.  Writes lane[i] in [0, *n_lanes).
 * width[i] >= 1 and cost[i] >= 0, else GM_ERR_INVALID_ARG; n == 0 gives 0 lanes. */
gm_status gm_batch_plan(int n, const int* width, const double* cost, int sms, int* lane, int* n_lanes);
gm_status gm_ctx_graph_state(const gm_ctx* ctx, int* replayed, int* captures);

/* Launch timing of the dominant kernel: the reverse edge-update MLP (one launch per
 * message-passing level and stage chunk; Eq. linearized_dynamics), or on a context with
 * gm_settings.condensing = 1 the tangent edge-update MLP (one launch per stage and
 * message-passing layer; Eq. sparse_gamma_i_u by forward-mode products).  When on,
 * gm_rti_step records a CUDA event pair around each of these launches (inside
 * the captured graph in graph mode) and notes each launch's algorithmic DRAM
 * bytes (rows x 4W for the hidden and carry outputs, 4W per carried input row
 * and per distinct aggregate row, W/8 per distinct edge mask) and FLOPs
 * (4 W^2 per row, one product).  gm_ctx_kernel_stats waits for the last
 * recorded step and returns its launch count, summed milliseconds, bytes and
 * FLOPs (all zero before the first recorded step). */
gm_status gm_ctx_set_kernel_timing(gm_ctx* ctx, int on);
gm_status gm_ctx_kernel_stats(gm_ctx* ctx, int* launches, double* ms, double* bytes, double* flops);
/* Launch i (0 <= i < the launches of gm_ctx_kernel_stats) of the last recorded step: its
 * milliseconds, algorithmic bytes and CTAs (one per SM; fewer than the SMs for a launch that
 * ran beside the rollout of later stages: gm_settings chunk_mb).  GM_ERR_INVALID_ARG for
 * an index out of range. */
gm_status gm_ctx_kernel_launch(gm_ctx* ctx, int i, double* ms, double* bytes, int* ctas);

/* Stage timeline of matrix-free condensing (gm_settings.condensing = 1; GM_ERR_INVALID_ARG
 * on another context).  When on, gm_rti_step records a timing event where the rollout and the
 * tangent pass start, one after each rollout stage and one after each tangent stage (inside
 * the captured graph in graph mode).  gm_ctx_stage_times waits for the last recorded step and
 * writes, for k = 0..N-1, the milliseconds from the start to the end of rollout stage k
 * (roll_ms[k]) and of tangent stage k (tan_ms[k]); caller-owned host arrays of N floats.
 * GM_ERR_INVALID_ARG while timing is off. */
gm_status gm_ctx_set_stage_timing(gm_ctx* ctx, int on);
gm_status gm_ctx_stage_times(gm_ctx* ctx, float* roll_ms, float* tan_ms);

/* ------------------------------------------------------------------------
 * Learned ADMM warm start (no paper counterpart; an added systems pattern).
 * A 3-layer MLP  in -> H -> H -> out  (Linear-ReLU-Linear-ReLU-Linear) maps
 * the features of an MPC instance to a primal input sequence and box duals
 * (out = 2 nU: U^0 then y^0), which warm-start gm_qp_solve.  Cold-start
 * ADMM stays the fallback: it runs whenever the warm-started solve does not
 * converge.  Features (gm_ws_features, [2W + 3M]): the mean and the max over
 * nodes of the final node latents h^K of stage 0 at (x_meas, the context's
 * current u_hat[0]; zeros after gm_ctx_reset), then the stage-1 reference
 * positions x_ref[1][i][0..2].  Inputs and outputs are standardised with
 * stored means and deviations (norm = [in mean | in std | out mean | out std]).
 * Parameters are packed [W0 (in x H) | b0 | W1 (H x H) | b1 | W2 (H x out) | b2],
 * each W row-major [fan-in][fan-out].  All arrays are device pointers on the
 * given stream (params/norm may be host pointers in set/get).
 *   gm_ws_workspace_size / gm_ws_create: caller-owned workspace (256-byte
 *     aligned) holding parameters, gradients, Adam moments and activations for
 *     batches up to max_batch; the library allocates nothing.
 *   gm_ws_set_params: parameters and normalisation; resets Adam.
 *   gm_ws_forward: out [B][n_out] for feat [B][n_in].
 *   gm_ws_train_step: one Adam step (bias-corrected) on the mean squared error
 *     of the standardised outputs against target [B][n_out]; loss (device
 *     float, nullable) receives that loss before the step.
 *   gm_ws_grad: the gradient of the last train step (packed like params).
 * ---------------------------------------------------------------------- */
typedef struct gm_ws gm_ws;
size_t gm_ws_workspace_size(int n_in, int n_hidden, int n_out, int max_batch);
gm_status gm_ws_create(int n_in, int n_hidden, int n_out, int max_batch, void* workspace, size_t bytes,
                       gm_ws** out);
void gm_ws_destroy(gm_ws* w);
long long gm_ws_param_count(const gm_ws* w);
gm_status gm_ws_set_params(gm_ws* w, const float* params, const float* norm, void* stream);
gm_status gm_ws_get_params(const gm_ws* w, float* params, float* norm, void* stream);
gm_status gm_ws_forward(gm_ws* w, const float* feat, int B, float* out, void* stream);
gm_status gm_ws_train_step(gm_ws* w, const float* feat, const float* target, int B, float lr, float beta1,
                           float beta2, float eps, float* loss, void* stream);
gm_status gm_ws_grad(gm_ws* w, float* grad, void* stream);
gm_status gm_ws_features(gm_ctx* ctx, const float* x_meas, const float* x_ref, float* feat, void* stream);

/* ------------------------------------------------------------------------
 * gm_qp_solve_noalloc — the ADMM solve of gm_qp_solve for callers that
 * cannot allocate device memory at all.  The paper has no counterpart: it
 * exists for hosts such as a real-time control loop that must not call
 * cudaMalloc once running (an allocation can synchronise the device and has
 * no latency bound), or a plug-in living inside another runtime that owns
 * the whole device-memory budget and hands out no workspace.  Such a caller
 * cannot create a gm_ctx (its workspace is caller-allocated device memory),
 * so this call needs no context.
 *
 * All scratch (P and its factors, ADMM z / y / row scales, reduction buffers,
 * barrier counters, KKT accumulators) lives in one fixed array of
 * GM_NOALLOC_SCRATCH_BYTES inside the library, held by every GPU that loads
 * it until the process exits.  The call allocates nothing.
 *   Limits: N * nu <= GM_NOALLOC_MAX_NU, N * Mnc <= GM_NOALLOC_MAX_ROWS;
 *           larger problems are rejected with GM_ERR_INVALID_ARG.
 *   N, nu, Mnc  horizon, inputs, half-space rows per stage (M * n_c)
 *   s           rho, tol, max_iter, scale_rows, timeout_spins are used
 *   H, g, Ct, dt, u_lo, u_hi, U, y, stats   as for gm_qp_solve (device
 *           pointers; Ct/dt NULL when Mnc == 0; y and stats nullable)
 * The first call on a device looks up the array's device address on that
 * device (the device must be current).  That first call is also when CUDA
 * loads the library's kernel modules onto the device (lazy loading), which
 * reserves their device memory, the array included, and may synchronise the
 * device: a caller that must not allocate once running makes one call at
 * initialisation, before any stream capture; later calls allocate nothing.  Every call uses the same array and leaves the last
 * call's contents in it (the call clears what must start at zero): calls
 * whose kernels overlap on the GPU (other streams, other host threads) race
 * and give wrong results; serialise them.
 * ---------------------------------------------------------------------- */
#define GM_NOALLOC_MAX_NU 64
#define GM_NOALLOC_MAX_ROWS 8192
#define GM_NOALLOC_SCRATCH_BYTES (512 * 1024)
gm_status gm_qp_solve_noalloc(int N, int nu, int Mnc, const gm_settings* s, const float* H,
                              const float* g, const float* Ct, const float* dt,
                              const float* u_lo, const float* u_hi, float* U, float* y,
                              gm_stats* stats, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GM_H */
