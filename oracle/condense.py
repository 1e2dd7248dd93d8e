"""Condensing of the linearised OCP into a QP in the inputs, FP64 (oracle; test infrastructure only).

Conventions (readings of the paper, stated once here):

* The QP is  min 1/2 U^T H U + g^T U  s.t.  lo <= U <= hi,  C~ U <= d~  with
      H = Gu^T Qbar Gu + Rbar,
      g = Gu^T Qbar (Gx - x_ref) - Rbar u_ref.
  This is exactly one half of the tracking cost of Eq. linear_gnn_mpc_ocp_explicit,
  so the minimiser is the paper's.  (Eq. condensed_matrices writes the
  objective without the 1/2; with its linear term q = -2 Q x_ref the two agree
  up to that overall factor.)
* Gu has (N+1) block rows (x_0 included, its row is zero) and N nu columns;
  Gx has (N+1) n_x entries.
* Q^i_k is diagonal (6 entries per node and stage, stages 0..N); R_k diagonal.
* State constraints act on node positions: C^{x,i}_k [n_c, 3], d^{x,i}_k [n_c],
  for stages k = 1..N (x_0 is fixed by Eq. ocp_initial_state).
* C~ rows are stored stage-major (k, i, c).  The paper stacks them per node
  (i, k, c); the two differ by a row permutation only.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------------
# Textbook dense condensing (Sec. III-B, Eq. condensed_matrices)
# ----------------------------------------------------------------------------------

def transition(A, k, m):
    """Phi(k, m) = A_{k-1} ... A_m  (identity when k == m)."""
    nx = A.shape[1]
    P = np.eye(nx)
    for t in range(m, k):
        P = A[t] @ P
    return P


def gamma_dense(A, B, c, x0):
    """Gu [(N+1) nx, N nu] and Gx [(N+1) nx] with x = Gu u + Gx, written out as products.

    Block (k, l) of Gu is Phi(k, l+1) B_l for l < k; block k of Gx is
    Phi(k, 0) x0 + sum_{l<k} Phi(k, l+1) c_l.
    """
    N, nx, nu = B.shape
    Gu = np.zeros(((N + 1) * nx, N * nu))
    Gx = np.zeros((N + 1) * nx)
    for k in range(N + 1):
        Gx[k * nx:(k + 1) * nx] = transition(A, k, 0) @ x0
        for l in range(k):
            P = transition(A, k, l + 1)
            Gu[k * nx:(k + 1) * nx, l * nu:(l + 1) * nu] = P @ B[l]
            Gx[k * nx:(k + 1) * nx] += P @ c[l]
    return Gu, Gx


def position_selector(M):
    """S [3M, 6M] picking the position part of every node state."""
    S = np.zeros((3 * M, 6 * M))
    for i in range(M):
        S[3 * i:3 * i + 3, 6 * i:6 * i + 3] = np.eye(3)
    return S


def condense_dense(A, B, c, x0, Qdiag, Rdiag, x_ref, u_ref, Cx, dx):
    """H, g, C~ (stage-major rows), d~ by Eq. condensed_matrices with dense matrices.

    A [N, nx, nx], B [N, nx, nu], c [N, nx], x0 [nx], Qdiag [N+1, nx],
    Rdiag [N, nu], x_ref [N+1, nx], u_ref [N, nu], Cx [N, M, n_c, 3],
    dx [N, M, n_c] (stages 1..N).
    """
    N, nx, nu = B.shape
    M = nx // 6
    Gu, Gx = gamma_dense(A, B, c, x0)
    Qbar = np.diag(np.asarray(Qdiag, np.float64).reshape(-1))
    Rbar = np.diag(np.asarray(Rdiag, np.float64).reshape(-1))
    xr = np.asarray(x_ref, np.float64).reshape(-1)
    ur = np.asarray(u_ref, np.float64).reshape(-1)
    H = Gu.T @ Qbar @ Gu + Rbar
    g = Gu.T @ Qbar @ (Gx - xr) - Rbar @ ur
    n_c = Cx.shape[2] if Cx is not None else 0
    if n_c == 0:
        return H, g, np.zeros((0, N * nu)), np.zeros(0), Gu, Gx
    # block-diagonal C_x over stages 1..N acting on positions
    Sel = position_selector(M)
    rows = N * M * n_c
    Cbar = np.zeros((rows, (N + 1) * nx))
    dbar = np.zeros(rows)
    for k in range(1, N + 1):
        Ck = np.zeros((M * n_c, 3 * M))
        for i in range(M):
            Ck[i * n_c:(i + 1) * n_c, 3 * i:3 * i + 3] = Cx[k - 1, i]
        r0 = (k - 1) * M * n_c
        Cbar[r0:r0 + M * n_c, k * nx:(k + 1) * nx] = Ck @ Sel
        dbar[r0:r0 + M * n_c] = np.asarray(dx[k - 1], np.float64).reshape(-1)
    Ct = Cbar @ Gu
    dt = dbar - Cbar @ Gx
    return H, g, Ct, dt, Gu, Gx


# ----------------------------------------------------------------------------------
# Per-node recursion (Thm. 1 proof: Eq. sparse_gamma_i_xb, Eq. sparse_gamma_i_u,
# Eq. H, Eq. g and the per-node constraint stacking)
# ----------------------------------------------------------------------------------

def blocks_from_dense(A, B, c, neighbourhoods):
    """Per stage and node: (Ñ_i, [A^{ij} for j in Ñ_i], B^i, c^i) from dense A, B, c."""
    N = B.shape[0]
    out = []
    for n in range(N):
        per = []
        for i, nb in enumerate(neighbourhoods):
            Ablk = np.stack([A[n, 6 * i:6 * i + 6, 6 * j:6 * j + 6] for j in nb])
            per.append((list(nb), Ablk, B[n, 6 * i:6 * i + 6], c[n, 6 * i:6 * i + 6]))
        out.append(per)
    return out


class MacCounter:
    """Counts the multiply-adds the recursion performs on non-zero columns (Thm. 1)."""

    def __init__(self):
        self.macs = 0


def condense_recursive(blocks, x0, Qdiag, Rdiag, x_ref, u_ref, Cx, dx, counter=None):
    """H, g, C~ (stage-major rows), d~ by the per-node recursion of the Thm. 1 proof.

    blocks[n][i] = (Ñ_i, A-blocks [|Ñ_i|, 6, 6], B^i_n [6, nu], c^i_n [6]).
    Each node keeps its own block rows (Gamma_u^i)_n and (Gamma_x^i)_n; the
    next block row only reads the last block row of the nodes in Ñ_i.
    """
    N = len(blocks)
    M = len(blocks[0])
    nu = blocks[0][0][2].shape[1]
    nU = N * nu
    x0 = np.asarray(x0, np.float64).reshape(M, 6)
    Qd = np.asarray(Qdiag, np.float64).reshape(N + 1, M, 6)
    xr = np.asarray(x_ref, np.float64).reshape(N + 1, M, 6)
    Rd = np.asarray(Rdiag, np.float64).reshape(N, nu)
    ur = np.asarray(u_ref, np.float64).reshape(N, nu)
    cnt = counter if counter is not None else MacCounter()

    # (Gamma_u^i)_n as a list of block rows, each 6 x nU (columns >= n*nu are zero)
    Gu = [[np.zeros((6, nU))] for _ in range(M)]
    Gx = [[x0[i].copy()] for i in range(M)]
    for n in range(N):
        for i in range(M):
            nb, Ablk, Bi, ci = blocks[n][i]
            row_u = np.zeros((6, nU))
            row_x = np.array(ci, dtype=np.float64)
            for b, j in enumerate(nb):
                last_u = Gu[j][n]            # E_n (Gamma_u^j)_n: last block row
                last_x = Gx[j][n]
                row_u[:, :n * nu] += Ablk[b] @ last_u[:, :n * nu]
                row_x += Ablk[b] @ last_x
                cnt.macs += 36 * (n * nu + 1)
            row_u[:, n * nu:(n + 1) * nu] = Bi
            Gu[i].append(row_u)
            Gx[i].append(row_x)

    # Eq. H and Eq. g: per-node contributions, summed, plus the input terms
    H = np.diag(Rd.reshape(-1)).copy()
    g = -(Rd * ur).reshape(-1)
    for i in range(M):
        for k in range(N + 1):
            Q = Qd[k, i]
            cols = k * nu
            Sk = Gu[i][k][:, :cols]
            H[:cols, :cols] += Sk.T @ (Q[:, None] * Sk)
            qbar = -Q * xr[k, i]
            g[:cols] += Sk.T @ (Q * Gx[i][k] + qbar)
            cnt.macs += 6 * cols * cols + 6 * cols
    # constraint rows, per node, then laid out stage-major (k, i, c)
    n_c = Cx.shape[2] if Cx is not None else 0
    Ct = np.zeros((N * M * n_c, nU))
    dt = np.zeros(N * M * n_c)
    for i in range(M):
        for k in range(1, N + 1):
            C = np.asarray(Cx[k - 1, i], np.float64)          # [n_c, 3]
            r0 = ((k - 1) * M + i) * n_c
            Ct[r0:r0 + n_c] = C @ Gu[i][k][:3]
            dt[r0:r0 + n_c] = np.asarray(dx[k - 1, i], np.float64) - C @ Gx[i][k][:3]
            cnt.macs += n_c * 3 * (k * nu + 1)
    Gu_full = np.concatenate([np.concatenate(Gu[i], 0)[None] for i in range(M)], 0)
    Gx_full = np.stack([np.stack(Gx[i]) for i in range(M)])   # [M, N+1, 6]
    return H, g, Ct, dt, Gu_full, Gx_full


def sphere_halfspaces(x_hat, spheres):
    """Linearise sphere obstacles at the rollout positions, stages 1..N.

    For node position p^ and sphere (o, r): n = (p^ - o)/|p^ - o|, the row
    -n^T p <= -r - n^T o keeps p on the far side of the tangent plane.  A node
    exactly at the centre uses n = +z.  Returns Cx [N, M, S, 3], dx [N, M, S].
    """
    x_hat = np.asarray(x_hat, np.float64)
    Np1, M, _ = x_hat.shape
    S = spheres.shape[0]
    Cx = np.zeros((Np1 - 1, M, S, 3))
    dx = np.zeros((Np1 - 1, M, S))
    for k in range(1, Np1):
        for s in range(S):
            o = np.asarray(spheres[s, :3], np.float64)
            r = float(spheres[s, 3])
            diff = x_hat[k, :, :3] - o
            nrm = np.sqrt((diff * diff).sum(1))
            n = np.where(nrm[:, None] > 0, diff / np.where(nrm > 0, nrm, 1.0)[:, None],
                         np.array([0.0, 0.0, 1.0]))
            Cx[k - 1, :, s] = -n
            dx[k - 1, :, s] = -r - n @ o
    return Cx, dx
