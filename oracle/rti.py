"""One real-time iteration of GNN-MPC (Algorithm 1, one pass of its outer loop), FP64.

Oracle; test infrastructure only.  Steps, in the order of Algorithm 1:

1. linearisation trajectory: u_hat = shifted previous solution (zero at start),
   x_hat = GNN rollout of the measured state under u_hat;
2. linearise: A^{ij}_k, B^i_k, c^i_k at (x_hat_k, u_hat_k) (Eq. linearized_dynamics);
3. condense per node and aggregate (Thm. 1 proof); sphere obstacles are first
   linearised to position half-spaces at x_hat;
4. solve the QP (exact optimum, or the ADMM recurrence);
5. shift: next u_hat = (U*_1, ..., U*_{N-1}, U*_{N-1}).
"""
from __future__ import annotations

import numpy as np

from . import barrier as br
from . import condense as cd
from . import gnn as gm
from . import qp


def model_of(wl, activation="relu"):
    gnn = gm.GNN(wl.blob, wl.K, wl.W, wl.nu, wl.dt, activation=activation)
    g = gm.Graph(wl.M, wl.src, wl.dst, wl.nu, wl.act_node)
    return gnn, g


def shift(U):
    """Alg. 1 "update lin. trajectory": drop u_0, repeat the last input."""
    U = np.asarray(U, np.float64)
    return np.concatenate([U[1:], U[-1:]], axis=0)


def linearize_dense(gnn, g, x_hat, u_hat):
    """A [N, nx, nx], B [N, nx, nu], c [N, nx] at every stage of the trajectory."""
    N = u_hat.shape[0]
    As, Bs, cs = [], [], []
    for k in range(N):
        A, B, c, _ = gm.jacobian_dense(gnn, g, x_hat[k], u_hat[k])
        As.append(A); Bs.append(B); cs.append(c)
    return np.stack(As), np.stack(Bs), np.stack(cs)


def rti_step(wl, u_hat=None, activation="relu", solver="exact", condensing="recursive",
             return_all=False, scale_rows=True, adapt_every=25, barrier=None):
    """One RTI step on workload wl.  Returns U* [N, nu] (and intermediates).

    barrier = (mu, delta): the obstacle rows enter the cost as relaxed log barriers
    (``oracle.barrier``, Sec. VI-B) instead of constraints; the QP keeps the box only.
    """
    gnn, g = model_of(wl, activation)
    u_hat = np.zeros((wl.N, wl.nu)) if u_hat is None else np.asarray(u_hat, np.float64)
    x_hat = gm.rollout(gnn, g, wl.x0, u_hat)
    A, B, c = linearize_dense(gnn, g, x_hat, u_hat)
    if wl.spheres.shape[0] > 0:
        Cx, dx = cd.sphere_halfspaces(x_hat, wl.spheres.astype(np.float64))
    else:
        Cx = dx = None
    x0 = np.asarray(wl.x0, np.float64).reshape(-1)
    if condensing == "recursive":
        nbh = [g.in_ball(i, gnn.K) for i in range(wl.M)]
        blocks = cd.blocks_from_dense(A, B, c, nbh)
        H, gv, Ct, dt, _, _ = cd.condense_recursive(
            blocks, x0, wl.Qdiag, wl.Rdiag, wl.x_ref, wl.u_ref,
            Cx if Cx is not None else np.zeros((wl.N, wl.M, 0, 3)),
            dx if dx is not None else np.zeros((wl.N, wl.M, 0)))
    else:
        H, gv, Ct, dt, _, _ = cd.condense_dense(
            A, B, c, x0, wl.Qdiag.reshape(wl.N + 1, -1), wl.Rdiag,
            wl.x_ref.reshape(wl.N + 1, -1), wl.u_ref,
            Cx if Cx is not None else np.zeros((wl.N, wl.M, 0, 3)),
            dx if dx is not None else np.zeros((wl.N, wl.M, 0)))
    lo = wl.u_lo.reshape(-1).astype(np.float64)
    hi = wl.u_hi.reshape(-1).astype(np.float64)
    if barrier is not None:
        H, gv = br.barrier_fold(H, gv, Ct, dt, u_hat.reshape(-1), barrier[0], barrier[1])
        Ct, dt = np.zeros((0, H.shape[0])), np.zeros(0)
    if solver == "exact":
        U, y, info = qp.solve_exact(H, gv, lo, hi, Ct, dt)
    else:
        U, z, y, it, rp, rd, ok = qp.admm(H, gv, lo, hi, Ct, dt, rho=wl.rho, tol=wl.tol,
                                          max_iter=wl.max_iter, scale_rows=scale_rows,
                                          adapt_every=adapt_every)
        info = dict(iters=it, r_p=rp, r_d=rd, converged=ok)
    U = U.reshape(wl.N, wl.nu)
    if not return_all:
        return U
    return dict(U=U, y=y, info=info, x_hat=x_hat, u_hat=u_hat, A=A, B=B, c=c, H=H, g=gv,
                Ct=Ct, dt=dt, Cx=Cx, dx=dx)
