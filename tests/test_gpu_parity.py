"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.  Needs a GPU.

Tolerances: see gpu_helpers (REL = 2e-4 of the quantity's max-abs, derived
from FP32 accumulation over the GNN's layer chain).  Solver outputs are
compared with the oracle running the same ADMM recurrence to the same
tolerance, and with the exact optimum through the KKT certificate.
"""
import numpy as np
import pytest

from gpu_helpers import (REL, blocks_to_dense, dense_to_blocks, dense_to_packed_ct, max_rel_err,
                         ocd, ogm, oqp, oracle_linearize, orti, packed_to_dense_ct)
from synth import paper_chain, random_instance, small_chain

pytestmark = pytest.mark.gpu


def _cases():
    return {
        "chain10": lambda: small_chain(),
        "rand_directed": lambda: random_instance(3, M=13, N=4, nu=3, K=2, W=32, reach=3, p=0.6,
                                                 directed=True),
        "rand_sym_W64_K3": lambda: random_instance(8, M=17, N=3, nu=2, K=3, W=64, reach=2, p=0.7),
        "edgeless": lambda: random_instance(4, M=5, N=3, nu=2, K=1, W=32, reach=1, p=0.0),
        "chain40_W128": lambda: paper_chain(M=40, N=5, nu=4, n_spheres=0),
    }


def _degenerate_cases():
    """Smallest shapes the method admits: one node with no edges and a one-stage horizon, a
    one-stage horizon on a graph, several inputs sharing an actuator node."""
    return {
        "M1_N1_nu1_sphere": lambda: random_instance(5, M=1, N=1, nu=1, K=1, W=32, reach=1, p=0.0,
                                                    n_spheres=1),
        "rand6_N1": lambda: random_instance(6, M=6, N=1, nu=2, K=2, W=32, reach=2, p=0.8),
        "M3_nu5_shared_nodes": lambda: random_instance(7, M=3, N=3, nu=5, K=2, W=32, reach=2, p=1.0),
    }


def _u_hat(wl, seed=0):
    return np.random.default_rng(seed).uniform(-0.5, 0.5, (wl.N, wl.nu)).astype(np.float32)


@pytest.mark.parametrize("case", list(_cases()) + list(_degenerate_cases()))
def test_linearize_parity(lib, case):
    """x_hat (Eq. forward_dynamics) and A, B, c (Eq. linearized_dynamics) against the oracle."""
    wl = {**_cases(), **_degenerate_cases()}[case]()
    u_hat = _u_hat(wl)
    prob = lib.RTIProblem.from_workload(wl)
    x_hat, A, B, c = (t.cpu().numpy().astype(np.float64) for t in prob.linearize(wl.x0, u_hat))
    xo, Ao, Bo, co = oracle_linearize(wl, u_hat.astype(np.float64))
    assert max_rel_err(x_hat, xo) <= REL
    for k in range(wl.N):
        # the oracle's dense A vanishes outside the K-hop block pattern the library uses
        assert np.array_equal(blocks_to_dense(dense_to_blocks(Ao[k], prob.row_ptr, prob.col, wl.M),
                                              prob.row_ptr, prob.col, wl.M), Ao[k])
        Ag = blocks_to_dense(A[k], prob.row_ptr, prob.col, wl.M)
        # scale: the learned part of A, d dv / dx (the Euler identity part is exact in both)
        V = Ao[k].reshape(wl.M, 6, wl.M, 6)[:, 3:].copy()
        for i in range(wl.M):
            V[i, :, i, 3:] -= np.eye(3)
        Jscale = np.abs(V).max()
        assert max_rel_err(Ag, Ao[k], scale=max(Jscale, 1e-3)) <= REL, (case, k)
        assert max_rel_err(B[k].reshape(-1, wl.nu), Bo[k]) <= REL, (case, k)
        assert max_rel_err(c[k].reshape(-1), co[k]) <= REL, (case, k)


def _halfspaces(wl, n_c, seed):
    rng = np.random.default_rng(seed)
    n = rng.normal(0, 1, (wl.N, wl.M, n_c, 3))
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    d = rng.uniform(0.5, 2.0, (wl.N, wl.M, n_c))
    return n.astype(np.float32), d.astype(np.float32)


@pytest.mark.parametrize("mode", ["halfspaces", "spheres"])
def test_condense_parity(lib, mode):
    """H, g, C~, d~ by the per-node recursion (Thm. 1 proof) against the oracle on the same A, B, c."""
    wl = small_chain()
    u_hat = _u_hat(wl, 1)
    xo, Ao, Bo, co = oracle_linearize(wl, u_hat.astype(np.float64))
    if mode == "halfspaces":
        Cx, dx = _halfspaces(wl, 3, 2)
        prob = lib.RTIProblem(wl.M, wl.src, wl.dst, wl.nu, wl.act_node, wl.K, wl.W, wl.dt, wl.blob, wl.N,
                              wl.Qdiag, wl.Rdiag, wl.x_ref, wl.u_ref, wl.u_lo, wl.u_hi, Cx=Cx, dx=dx)
    else:
        wl.spheres = np.array([[0.0, 0.05, -0.3, 0.02], [0.02, -0.04, -0.7, 0.03]], np.float32)
        prob = lib.RTIProblem.from_workload(wl)
    torch = prob.torch
    f32 = lambda a: np.asarray(a, np.float32)  # noqa: E731
    x_hat32, A32, B32, c32 = f32(xo), f32(Ao), f32(Bo), f32(co)
    Ablk = np.stack([dense_to_blocks(A32[k], prob.row_ptr, prob.col, wl.M) for k in range(wl.N)])
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")  # noqa: E731
    H, g, Ct, dt = (t.cpu().numpy().astype(np.float64) for t in prob.condense(
        dev(x_hat32), dev(Ablk), dev(B32.reshape(wl.N, wl.M, 6, wl.nu)), dev(c32.reshape(wl.N, wl.M, 6))))
    x64 = x_hat32.astype(np.float64)
    if mode == "spheres":
        Cx, dx = ocd.sphere_halfspaces(x64, wl.spheres.astype(np.float64))
    nbh = [list(prob.col[prob.row_ptr[i]:prob.row_ptr[i + 1]]) for i in range(wl.M)]
    blocks = ocd.blocks_from_dense(A32.astype(np.float64), B32.astype(np.float64),
                                   c32.astype(np.float64), nbh)
    Ho, go, Cto, dto, _, _ = ocd.condense_recursive(blocks, x64[0].reshape(-1), wl.Qdiag, wl.Rdiag,
                                                    wl.x_ref, wl.u_ref, np.asarray(Cx, np.float64),
                                                    np.asarray(dx, np.float64))
    R = np.diag(wl.Rdiag.reshape(-1).astype(np.float64))
    assert max_rel_err(H - R, Ho - R) <= REL
    assert max_rel_err(g, go) <= REL
    n_c = Cx.shape[2]
    assert max_rel_err(Ct, dense_to_packed_ct(Cto, wl.N, wl.M, n_c, wl.nu)) <= REL
    assert max_rel_err(dt, dto) <= REL


@pytest.mark.parametrize("constrained", [False, True])
def test_qp_parity(lib, constrained):
    """ADMM on the GPU against the oracle's ADMM recurrence and the exact optimum."""
    wl = small_chain()
    u_hat = _u_hat(wl, 3)
    xo, Ao, Bo, co = oracle_linearize(wl, u_hat.astype(np.float64))
    gnn, gr = orti.model_of(wl)
    nbh = [gr.in_ball(i, wl.K) for i in range(wl.M)]
    if constrained:
        # half-spaces through the nominal positions: some rows active at the optimum
        rng = np.random.default_rng(5)
        n = rng.normal(0, 1, (wl.N, wl.M, 2, 3))
        n /= np.linalg.norm(n, axis=-1, keepdims=True)
        p = xo[1:, :, None, :3]
        dx = (np.einsum("kics,kics->kic", n, np.broadcast_to(p, n.shape)) + 1e-4).astype(np.float32)
        Cx = n.astype(np.float32)
    else:
        Cx = np.zeros((wl.N, wl.M, 0, 3), np.float32)
        dx = np.zeros((wl.N, wl.M, 0), np.float32)
    blocks = ocd.blocks_from_dense(Ao, Bo, co, nbh)
    H, g, Ct, dt, _, _ = ocd.condense_recursive(blocks, xo[0].reshape(-1), wl.Qdiag, wl.Rdiag, wl.x_ref,
                                                wl.u_ref, Cx.astype(np.float64), dx.astype(np.float64))
    H32, g32, Ct32, dt32 = (np.asarray(a, np.float32) for a in (H, g, Ct, dt))
    H64, g64, Ct64, dt64 = (a.astype(np.float64) for a in (H32, g32, Ct32, dt32))
    lo = wl.u_lo.reshape(-1).astype(np.float64)
    hi = wl.u_hi.reshape(-1).astype(np.float64)
    Ua, za, ya, it_o, rp_o, rd_o, ok_o = oqp.admm(H64, g64, lo, hi, Ct64 if Cx.shape[2] else None,
                                                  dt64 if Cx.shape[2] else None, rho=wl.rho, tol=wl.tol,
                                                  max_iter=wl.max_iter, scale_rows=True, adapt_every=25)
    Ux, yx, _ = oqp.solve_exact(H64, g64, lo, hi, Ct64 if Cx.shape[2] else None,
                                dt64 if Cx.shape[2] else None)
    n_c = Cx.shape[2]
    prob = lib.RTIProblem(wl.M, wl.src, wl.dst, wl.nu, wl.act_node, wl.K, wl.W, wl.dt, wl.blob, wl.N,
                          wl.Qdiag, wl.Rdiag, wl.x_ref, wl.u_ref, wl.u_lo, wl.u_hi,
                          Cx=Cx if n_c else None, dx=dx if n_c else None, rho=wl.rho, tol=wl.tol,
                          max_iter=wl.max_iter)
    torch = prob.torch
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")  # noqa: E731
    U, y = prob.qp_solve(dev(H32), dev(g32), dev(dense_to_packed_ct(Ct32, wl.N, wl.M, n_c, wl.nu))
                         if n_c else None, dev(dt32) if n_c else None)
    st = prob.read_stats()
    U = U.cpu().numpy().astype(np.float64)
    y = y.cpu().numpy().astype(np.float64)
    assert st["converged"] == 1 and ok_o
    # same recurrence, same stopping rule: iteration counts agree up to FP32 rounding near tol
    assert abs(st["iters"] - it_o) <= max(3, 0.05 * it_o), (st["iters"], it_o)
    # iterates of the same recurrence agree to the accuracy ADMM has reached
    assert np.abs(U - Ua).max() <= 10 * wl.tol / wl.rho, np.abs(U - Ua).max()
    # and the FP64 KKT certificate the library reports matches one recomputed here
    At, l, h = oqp.stack_rows(lo, hi, Ct64 if n_c else None, dt64 if n_c else None)
    cert = oqp.kkt_certificate(H64, g64, At, l, h, U, y)
    assert abs(st["kkt_stat"] - cert["stationarity"]) <= 1e-6 * max(1.0, cert["stationarity"]) + 1e-9
    assert st["kkt_prim"] <= 10 * wl.tol
    # the row parts of the certificate (the library tests most rows in FP32 with a rounding bound
    # first) equal the FP64 evaluation here on the same FP32 rows (H64, Ct64 are the FP32 data)
    for key, ck in (("kkt_prim", "primal"), ("kkt_comp", "complementarity"), ("kkt_dual", "dual")):
        assert abs(st[key] - cert[ck]) <= 1e-9 * max(1.0, abs(cert[ck])) + 1e-12, (key, st[key], cert[ck])
    # distance to the exact optimum is bounded by the dual residual / lambda_min(H)
    lam = np.linalg.eigvalsh(H64).min()
    assert np.abs(U - Ux).max() <= 2 * max(st["r_dual"], st["kkt_stat"]) / lam + 1e-5


def test_rti_step_matches_oracle_two_steps(lib):
    """Two real-time iterations (Alg. 1) end to end: U against the oracle's ADMM and exact U*."""
    wl = small_chain()
    prob = lib.RTIProblem.from_workload(wl)
    u_prev = None
    for step in range(2):
        U = prob.step(wl.x0).cpu().numpy().astype(np.float64).reshape(wl.N, wl.nu)
        st = prob.read_stats()
        uh = None if u_prev is None else orti.shift(u_prev)
        ro = orti.rti_step(wl, u_hat=uh, solver="admm", return_all=True)
        rx = orti.rti_step(wl, u_hat=uh, solver="exact", return_all=True)
        assert st["converged"] == 1
        assert np.abs(U - ro["U"]).max() <= 10 * wl.tol / wl.rho, (step, np.abs(U - ro["U"]).max())
        lam = np.linalg.eigvalsh(rx["H"]).min()
        assert np.abs(U - rx["U"]).max() <= 2 * max(st["r_dual"], st["kkt_stat"]) / lam + 1e-5
        u_prev = ro["U"]


@pytest.mark.parametrize("case", list(_degenerate_cases()))
def test_rti_step_degenerate_shapes(lib, case):
    """One real-time iteration on the smallest shapes: U against the oracle's exact optimum."""
    wl = _degenerate_cases()[case]()
    prob = lib.RTIProblem.from_workload(wl)
    U = prob.step(wl.x0).cpu().numpy().astype(np.float64).reshape(wl.N, wl.nu)
    st = prob.read_stats()
    rx = orti.rti_step(wl, solver="exact", return_all=True)
    assert st["status"] == 0 and st["converged"] == 1, st
    lam = np.linalg.eigvalsh(rx["H"]).min()
    assert np.abs(U - rx["U"]).max() <= 2 * max(st["r_dual"], st["kkt_stat"]) / lam + 1e-5, case


def _simulate_blocks(A, B, c, x0, U, row_ptr, col, M):
    """x_{k+1} = A_k x_k + B_k u_k + c_k with block-sparse A (FP64 on the CPU)."""
    xs = [x0.reshape(M, 6)]
    for k in range(A.shape[0]):
        xk = xs[-1]
        prod = np.einsum("qab,qb->qa", A[k], xk[col])
        ax = np.add.reduceat(prod, row_ptr[:-1], axis=0)
        xs.append(ax + np.einsum("iau,u->ia", B[k], U[k]) + c[k])
    return np.stack(xs)


def test_paper_scale_sampled_and_properties(lib):
    """Chain of 1000, K=3, W=128, N=20, 5 spheres: full rollout and sampled Jacobian rows
    against the oracle; condensing and QP checked by identities that hold at any size."""
    wl = paper_chain()
    prob = lib.RTIProblem.from_workload(wl)
    u_hat = _u_hat(wl, 7) * 0.2
    x_hat, A, B, c = prob.linearize(wl.x0, u_hat)
    xh = x_hat.cpu().numpy().astype(np.float64)
    gnn, gr = orti.model_of(wl)
    xo = ogm.rollout(gnn, gr, wl.x0, u_hat.astype(np.float64))
    assert max_rel_err(xh, xo) <= REL
    An, Bn, cn = (t.cpu().numpy().astype(np.float64) for t in (A, B, c))
    rng = np.random.default_rng(0)
    for (k, i) in [(0, 0), (0, 500), (7, 62), (13, 999), (19, 437), (10, int(rng.integers(0, 1000)))]:
        ball, Ablk, Bi, fi = ogm.local_jacobian_rows(gnn, gr, xo[k], u_hat[k].astype(np.float64), i)
        q0, q1 = prob.row_ptr[i], prob.row_ptr[i + 1]
        assert list(prob.col[q0:q1]) == ball
        scale = max(np.abs(Ablk[:, 3:]).max(), 1e-3)
        assert max_rel_err(An[k, q0:q1], Ablk, scale=scale) <= REL, (k, i)
        assert max_rel_err(Bn[k, i], Bi, scale=max(np.abs(Bi).max(), 1e-6)) <= REL, (k, i)
    # condensing: the QP objective equals half the tracking cost of the simulated linear system
    H, g, Ct, dt = prob.condense(x_hat, A, B, c)
    Hn, gn, Ctn, dtn = (t.cpu().numpy().astype(np.float64) for t in (H, g, Ct, dt))
    assert np.allclose(Hn, Hn.T, atol=1e-6 * np.abs(Hn).max())
    Qd = wl.Qdiag.astype(np.float64)
    consts = []
    for s in range(3):
        U = rng.uniform(-1, 1, (wl.N, wl.nu))
        xs = _simulate_blocks(An, Bn, cn, xh[0], U, prob.row_ptr, prob.col, wl.M)
        cost = 0.5 * (np.sum(Qd * (xs - wl.x_ref) ** 2) + np.sum(wl.Rdiag * (U - wl.u_ref) ** 2))
        u = U.reshape(-1)
        consts.append(cost - (0.5 * u @ Hn @ u + gn @ u))
        # constraint rows: C~ U - d~ == C_x p(U) - d_x, spheres linearised at x_hat
        Cx, dx = ocd.sphere_halfspaces(xh, wl.spheres.astype(np.float64))
        lhs = packed_to_dense_ct(Ctn, wl.N, wl.M, Cx.shape[2], wl.nu) @ u - dtn
        rhs = (np.einsum("kics,kis->kic", Cx, xs[1:, :, :3]) - dx).reshape(-1)
        assert np.abs(lhs - rhs).max() <= REL * max(1.0, np.abs(rhs).max())
    scale = max(abs(c_) for c_ in consts)
    assert np.ptp(consts) <= REL * max(scale, 1.0)
    # QP: the FP64 certificate of the returned solution
    U, y = prob.qp_solve(H, g, Ct, dt)
    st = prob.read_stats()
    assert st["status"] == 0 and st["converged"] == 1, st
    assert st["kkt_prim"] <= 10 * wl.tol and st["kkt_dual"] <= 10 * wl.tol
    Un = U.cpu().numpy()
    assert np.all(Un >= wl.u_lo.reshape(-1) - 1e-6) and np.all(Un <= wl.u_hi.reshape(-1) + 1e-6)


def test_rti_step_paper_scale_runs(lib):
    """The whole step at paper scale: converged, finite, feasible, and the shift is applied."""
    wl = paper_chain()
    prob = lib.RTIProblem.from_workload(wl)
    U1 = prob.step(wl.x0).cpu().numpy()
    st = prob.read_stats()
    assert st["status"] == 0 and st["converged"] == 1, st
    assert np.all(np.isfinite(U1))
    U2 = prob.step(wl.x0).cpu().numpy()
    assert np.all(np.isfinite(U2))
    prob.reset()
    U3 = prob.step(wl.x0).cpu().numpy()
    # reset restores the zero linearisation inputs (ADMM sums in atomic order: not bitwise)
    assert np.abs(U1 - U3).max() <= 10 * wl.tol / wl.rho
