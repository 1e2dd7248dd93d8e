"""A context plus its device-resident problem data, around the C entry points.

RTIProblem allocates (with torch) the workspace and the device copies of the
cost and constraint arrays, creates the graph / GNN / context handles, and
exposes one method per C call.  It holds no arithmetic of the method.
"""
from __future__ import annotations

import numpy as np

from . import (GM_PREC_FP32, STATS_BYTES, gm_barrier_fold, gm_condense, gm_condense_matrix_free, gm_ctx_create,
               gm_ctx_destroy, gm_ctx_graph_state,
               gm_ctx_set_warm,
               gm_ctx_reset, gm_ctx_set_graph, gm_ctx_workspace_size, gm_gnn_destroy, gm_gnn_load, gm_graph_create, gm_graph_destroy,
               gm_jac_pattern, gm_linearize, gm_qp_solve, gm_qp_solve_ipm, gm_rti_step, make_constr, make_cost,
               make_settings, read_stats)


class RTIProblem:
    """Device state for one MPC instance.

    Arguments mirror the paper's problem statement: graph (M, src, dst), inputs
    (nu, act_node), GNN (K, W, dt, weight blob), horizon N, cost (Qdiag, Rdiag,
    x_ref, u_ref), input box (u_lo, u_hi) and either explicit position
    half-spaces (Cx, dx) or spheres linearised at the rollout.  barrier = (mu, delta)
    makes step() put those rows into the cost as relaxed log barriers (gm_barrier_fold).
    warm=True starts each step's ADMM from the shifted previous solution (gm_ctx_set_warm).
    condensing=1 builds the condensed QP matrix-free (forward-mode sensitivities, no A_k);
    tan_split_rows sets where its edge updates switch to per-node projections (0: the default).
    """

    def __init__(self, M, src, dst, nu, act_node, K, W, dt, blob, N, Qdiag, Rdiag, x_ref, u_ref, u_lo,
                 u_hi, Cx=None, dx=None, spheres=None, rho=0.1, tol=1e-6, max_iter=4000,
                 precision=GM_PREC_FP32, polish=0, timeout_spins=0, scale_rows=1, adapt_rho=1,
                 graph=False, admm_grid=0, factor_grid=0, chunk_mb=0, barrier=None, warm=False, condensing=0,
                 tan_split_rows=0, device="cuda"):
        import torch
        self.torch = torch
        self.M, self.nu, self.N, self.K, self.W = int(M), int(nu), int(N), int(K), int(W)
        self.nU = self.N * self.nu
        f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device=device)  # noqa: E731
        self.spheres = None if spheres is None or len(spheres) == 0 else f32(spheres)
        if self.spheres is not None:
            n_c = int(self.spheres.shape[0])
            self.Cx = self.dx = None
        elif Cx is not None:
            n_c = int(np.asarray(Cx).shape[2])
            self.Cx, self.dx = f32(Cx), f32(dx)
        else:
            n_c = 0
            self.Cx = self.dx = None
        self.n_c = n_c
        self.rows_c = self.N * self.M * n_c
        self.ct_len = self.M * n_c * self.nu * self.N * (self.N + 1) // 2
        self.graph = gm_graph_create(M, src, dst, nu, act_node)
        self.gnn = gm_gnn_load(K, W, nu, dt, blob)
        self.settings = make_settings(N, n_c, precision, rho, tol, max_iter, polish, timeout_spins,
                                      scale_rows, adapt_rho, admm_grid, factor_grid, chunk_mb, condensing,
                                      tan_split_rows)
        nbytes = gm_ctx_workspace_size(self.graph, self.gnn, self.settings)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.ctx = gm_ctx_create(self.graph, self.gnn, self.settings, self.workspace)
        self.Qdiag, self.Rdiag, self.x_ref, self.u_ref = f32(Qdiag), f32(Rdiag), f32(x_ref), f32(u_ref)
        self.u_lo, self.u_hi = f32(u_lo), f32(u_hi)
        self.cost = make_cost(self.Qdiag, self.Rdiag, self.x_ref, self.u_ref)
        self.constr = make_constr(self.u_lo, self.u_hi, self.Cx, self.dx, self.spheres, barrier)
        self.row_ptr, self.col = gm_jac_pattern(self.ctx, self.M)
        self.nnzb = int(self.col.size)
        self.stats = torch.zeros(STATS_BYTES, dtype=torch.uint8, device=device)
        # fixed step buffers, so that a captured step (graph=True) keeps its pointers
        self._x = torch.zeros(self.M * 6, dtype=torch.float32, device=device)
        self._U = torch.zeros(self.nU, dtype=torch.float32, device=device)
        if graph:
            gm_ctx_set_graph(self.ctx, 1)
        if warm:
            gm_ctx_set_warm(self.ctx, 1)

    @classmethod
    def from_workload(cls, wl, **kw):
        """Build from any object with the workload attributes (see synth.Workload)."""
        args = dict(rho=wl.rho, tol=wl.tol, max_iter=wl.max_iter)
        args.update(kw)
        return cls(wl.M, wl.src, wl.dst, wl.nu, wl.act_node, wl.K, wl.W, wl.dt, wl.blob, wl.N, wl.Qdiag,
                   wl.Rdiag, wl.x_ref, wl.u_ref, wl.u_lo, wl.u_hi, spheres=wl.spheres, **args)

    def close(self):
        if getattr(self, "ctx", None):
            gm_ctx_destroy(self.ctx)
            gm_gnn_destroy(self.gnn)
            gm_graph_destroy(self.graph)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty(self, *shape):
        return self.torch.empty(*shape, dtype=self.torch.float32, device=self.Qdiag.device)

    def linearize(self, x0, u_hat):
        t = self.torch
        x0 = t.as_tensor(x0, dtype=t.float32, device=self.Qdiag.device).contiguous()
        u_hat = t.as_tensor(u_hat, dtype=t.float32, device=self.Qdiag.device).contiguous()
        x_hat = self.empty(self.N + 1, self.M, 6)
        A = self.empty(self.N, self.nnzb, 6, 6)
        B = self.empty(self.N, self.M, 6, self.nu)
        c = self.empty(self.N, self.M, 6)
        gm_linearize(self.ctx, x0, u_hat, x_hat, A, B, c)
        return x_hat, A, B, c

    def condense(self, x_hat, A, B, c):
        H = self.empty(self.nU, self.nU)
        g = self.empty(self.nU)
        Ct = self.empty(max(self.ct_len, 1))
        dt = self.empty(max(self.rows_c, 1))
        gm_condense(self.ctx, x_hat, A, B, c, self.cost, self.constr, H, g,
                    Ct if self.n_c else None, dt if self.n_c else None)
        return H, g, Ct[:self.ct_len], dt[:self.rows_c]

    def condense_matrix_free(self, x0, u_hat):
        """(x_hat, H, g, C~, d~) without local Jacobians (a context built with condensing=1)."""
        t = self.torch
        x0 = t.as_tensor(x0, dtype=t.float32, device=self.Qdiag.device).contiguous()
        u_hat = t.as_tensor(u_hat, dtype=t.float32, device=self.Qdiag.device).contiguous()
        x_hat = self.empty(self.N + 1, self.M, 6)
        H = self.empty(self.nU, self.nU)
        g = self.empty(self.nU)
        Ct = self.empty(max(self.ct_len, 1))
        dt = self.empty(max(self.rows_c, 1))
        gm_condense_matrix_free(self.ctx, x0, u_hat, self.cost, self.constr, x_hat, H, g,
                                Ct if self.n_c else None, dt if self.n_c else None)
        return x_hat, H, g, Ct[:self.ct_len], dt[:self.rows_c]

    def qp_solve(self, H, g, Ct=None, dt=None, warm_U=None, warm_y=None, box_only=False):
        """ADMM on the condensed QP; box_only drops the half-space rows (barrier variant)."""
        U = self.empty(self.nU)
        y = self.empty(self.nU + self.rows_c)
        rows = self.n_c and not box_only
        gm_qp_solve(self.ctx, H, g, Ct if rows else None, dt if rows else None, self.u_lo,
                    self.u_hi, U, y, self.stats, warm_U, warm_y)
        return U, y

    def barrier_fold(self, H, g, Ct, dt, U_hat, mu, delta):
        """H, g with the relaxed log-barrier model of the rows folded in (in place; returned)."""
        t = self.torch
        U_hat = t.as_tensor(U_hat, dtype=t.float32, device=self.Qdiag.device).reshape(-1).contiguous()
        gm_barrier_fold(self.ctx, Ct, dt, U_hat, mu, delta, H, g)
        return H, g

    def qp_solve_ipm(self, H, g, Ct=None, dt=None, max_iter=60):
        """The same QP by the interior-point method (gm_qp_solve_ipm)."""
        U = self.empty(self.nU)
        y = self.empty(self.nU + self.rows_c)
        gm_qp_solve_ipm(self.ctx, H, g, Ct if self.n_c else None, dt if self.n_c else None, self.u_lo,
                        self.u_hi, U, y, self.stats, max_iter)
        return U, y

    def step(self, x_meas, U=None, u0=None):
        """One RTI step from measured state x_meas [M*6].  Without U the result lands in a
        buffer of this object that the next step overwrites."""
        t = self.torch
        self._x.copy_(t.as_tensor(x_meas, dtype=t.float32).reshape(-1), non_blocking=True)
        U = self._U if U is None else U
        gm_rti_step(self.ctx, self._x, self.cost, self.constr, U, u0, self.stats)
        return U

    def graph_state(self):
        """(1 if the last step replayed a CUDA graph, number of captures)."""
        return gm_ctx_graph_state(self.ctx)

    def reset(self):
        gm_ctx_reset(self.ctx)

    def read_stats(self):
        return read_stats(self.stats)
