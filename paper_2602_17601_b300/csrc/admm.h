// ADMM solve of the condensed QP: device state, kernel arguments, launcher (internal).
#pragma once

#include "ctx.h"

namespace gmi {

constexpr int ADMM_T = 512;             // threads per CTA of the persistent kernel
constexpr int kAdmmTileFloats = 8192;   // C~ floats per shared-memory tile (x2 buffers, P^{-1} in smem)
constexpr int kAdmmTileFloatsL2 = 12288; // C~ floats per tile (x3 buffers, P^{-1} from L2)
constexpr bool kAdmmPinvShared = false;  // keep P^{-1} in shared memory when it fits
constexpr int kAdmmTileRows = 512;      // rows per tile at most
constexpr int kAdmmMaxN = 256;          // N nu
constexpr int kInfeasEvery = 10;        // iterations between primal-infeasibility tests
constexpr float kInfeasEps = 1e-4f;     // relative tolerance of the infeasibility certificate
constexpr int kStallEvery = 25;         // warm-started solves: iterations between stall tests
constexpr float kStallFactor = 0.5f;    // a stall: max(r_p, r_d) not below this fraction of its
                                        // value kStallEvery iterations earlier
constexpr bool kAdmmCondRounds = true;     // IF nodes around rounds after the first under capture
constexpr int kWarmRounds = 2;          // launches a warm-started solve may use (one rho update)
constexpr int kMaxRhoUpdates = 5;       // rho changes per start (warm or cold)
constexpr float kRedundantMargin = 1e-4f; // relative margin of the redundant-row test (qp.cu)

// Floats of one rotating accumulator: sums of s C~'z, s C~'y, s C~'dy ([3n]) and 8 scalars
// (max |a - z|, |a|, |z|, |dy|, wrong-sign dy; sum of the bound support of dy).
__host__ __device__ inline int admm_acc_stride(int n) { return 3 * n + 8; }

// Iterate and control flags kept on the device between the launches of one solve.
struct AdmmState {
    float rho;
    int need_factor;   // P(rho) must be formed and factored before the next launch
    int done;          // converged, iteration cap reached, or failed
    int started;       // initial pass done
    int iters;
    int updates;       // rho changes so far
    int converged;
    float rp, rd;
    float rho0;        // the settings' rho (the cold restart starts from it)
    int warm;          // this solve started from warm inputs: the stall test is on
    int cold;          // the warm start was abandoned: U0, y0 are ignored from now on
    int fell_back;     // the cold restart ran (reported as GM_STALLED when it converged)
    int it0;           // iteration count when the current start (warm or cold) began
    float stall_ref;   // max(r_p, r_d) at the last stall test (< 0: not yet taken)
    int final_status;  // gm_status of the last finished solve (next step's warm start reads it)
    float u[kAdmmMaxN], zb[kAdmmMaxN], yb[kAdmmMaxN], atz[kAdmmMaxN], aty[kAdmmMaxN];
};

struct Admm2Args {
    int n, nu, Mnc;
    long rows;
    const float *Ct, *dt, *lo, *hi, *g, *H, *Pinv, *rs, *U0, *y0;
    const int *kpos, *kcnt;   // kept-row positions per stage and counts (nullable: no skipping)
    float *U, *y, *z, *acc;
    unsigned* bar;
    int* status;
    const int* row_begin;
    AdmmState* S;
    gm_stats* stats;
    float tol;
    int max_iter, adapt_every, last_round, tile_floats, tile_rows;
    long long max_spins;
    bool vec4;
};

// Everything one solve needs; scratch pointers come from a context workspace or
// from the library-held scratch of gm_qp_solve_noalloc.
struct AdmmPlan {
    int n, nu, Mnc, N;
    long rows;
    const float *Ct, *dt, *lo, *hi, *g, *H, *U0, *y0;
    const float* rs;       // row scales (0: a redundant row) or nullptr when there are no rows
    const unsigned char* keep;   // [rows] 0 for redundant rows
    const int *kpos, *kcnt;      // [rows] position among the stage's kept rows, [N] kept per stage
    const float* Gram;     // C~' D C~ or nullptr when there are no half-space rows
    bool gram_tc = true;   // form it with the tensor-core Gram (gram_tc.cu)
    bool keep_rho = false; // start from the previous solve's final rho (warm start)
    bool warm = false;     // U0 or y0 given: stall test, cold restart on a stall or a NaN
    float *U, *y, *z;      // y, z: [n + rows]
    float *P, *Pinv;       // [n n]
    double *L, *Linv;      // [factor_pad(n)^2]
    float* acc;            // [3 admm_acc_stride(n)]
    unsigned* bar;         // [4]
    int* status;           // [4]
    int* row_begin;        // [grid + 1]
    AdmmState* S;
    gm_stats* stats;
    float rho0, tol;
    int max_iter, adapt_every, rounds, grid;
    int factor_grid;       // CTAs of the factor kernel (0: default)
    long long max_spins;
    cudaStream_t st;
    cudaEvent_t ev_mid;    // recorded after the first factorisation (nullable)
    // while st is being captured into a graph: rounds after the first go into conditional (IF)
    // nodes whose bodies are captured on this stream, so rounds after convergence are skipped
    // (nullable: every round is launched)
    cudaStream_t body_st;
};

gm_status admm_solve(const AdmmPlan& p);

// Interior-point solve of the same QP (ipm.cu): workspace sizes of its row and vector arrays.
constexpr int kIpmRowArrays = 7;
constexpr int kIpmVecArrays = 16;
constexpr int kIpmScalars = 32;
size_t admm2_smem_bytes(int n);
const void* admm2_kernel_ptr(int n);

// FP64 Cholesky of P and P^{-1} = L^{-T} L^{-1} (stored FP32) in one cooperative launch
// (factor.cu); gate (nullable) skips it when no factorisation is due.  L and Linv hold
// factor_pad(n)^2 doubles; bar[0] is used (and reset) as the grid barrier counter.
int factor_pad(int n);
int factor_grid();            // default CTAs of the factor kernel (cooperative)
gm_status factor_pinv(int n, const float* P, double* L, double* Linv, float* Pinv, int* status,
                      const AdmmState* gate, unsigned* bar, long long max_spins, int grid, cudaStream_t st);

}  // namespace gmi
