"""The interior-point solve of the condensed QP (gm_qp_solve_ipm) against the exact optimum.  Needs a GPU.

The oracle's optimum U* is the definition (solve_exact: an FP64 interior-point
method to a tight KKT residual, then the equality-constrained solve on its
active set; pinned to brute force and to the uncondensed QP in
test_oracle_qp).  The device IPM stops when its primal and dual residuals and
its complementarity gap are below tol, so its U must satisfy the FP64 KKT
certificate to about tol and lie within the distance that certificate allows
from U*.  The same QPs are solved by ADMM for comparison.
"""
import numpy as np
import pytest

from gpu_helpers import dense_to_packed_ct, ocd, oqp, oracle_linearize, orti
from synth import small_chain

pytestmark = pytest.mark.gpu


def _qp(constrained, offset=1e-4, seed=5):
    wl = small_chain()
    u_hat = np.random.default_rng(3).uniform(-0.5, 0.5, (wl.N, wl.nu))
    xo, Ao, Bo, co = oracle_linearize(wl, u_hat)
    gnn, gr = orti.model_of(wl)
    nbh = [gr.in_ball(i, wl.K) for i in range(wl.M)]
    if constrained:
        rng = np.random.default_rng(seed)
        n = rng.normal(0, 1, (wl.N, wl.M, 2, 3))
        n /= np.linalg.norm(n, axis=-1, keepdims=True)
        p = xo[1:, :, None, :3]
        dx = np.einsum("kics,kics->kic", n, np.broadcast_to(p, n.shape)) + offset
    else:
        n = np.zeros((wl.N, wl.M, 0, 3))
        dx = np.zeros((wl.N, wl.M, 0))
    H, g, Ct, dt, _, _ = ocd.condense_recursive(ocd.blocks_from_dense(Ao, Bo, co, nbh), xo[0].reshape(-1),
                                                wl.Qdiag, wl.Rdiag, wl.x_ref, wl.u_ref, n, dx)
    return wl, n.astype(np.float32), dx.astype(np.float32), [np.asarray(a, np.float32) for a in (H, g, Ct, dt)]


@pytest.mark.parametrize("constrained", [False, True])
def test_ipm_reaches_the_exact_optimum(lib, constrained):
    wl, Cx, dx, (H, g, Ct, dt) = _qp(constrained)
    n_c = Cx.shape[2]
    H64, g64, Ct64, dt64 = (a.astype(np.float64) for a in (H, g, Ct, dt))
    lo = wl.u_lo.reshape(-1).astype(np.float64)
    hi = wl.u_hi.reshape(-1).astype(np.float64)
    Ux, yx, _ = oqp.solve_exact(H64, g64, lo, hi, Ct64 if n_c else None, dt64 if n_c else None)
    prob = lib.RTIProblem(wl.M, wl.src, wl.dst, wl.nu, wl.act_node, wl.K, wl.W, wl.dt, wl.blob, wl.N,
                          wl.Qdiag, wl.Rdiag, wl.x_ref, wl.u_ref, wl.u_lo, wl.u_hi,
                          Cx=Cx if n_c else None, dx=dx if n_c else None, rho=wl.rho, tol=wl.tol,
                          max_iter=wl.max_iter)
    torch = prob.torch
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")  # noqa: E731
    Ctp = dev(dense_to_packed_ct(Ct, wl.N, wl.M, n_c, wl.nu)) if n_c else None
    U, y = prob.qp_solve_ipm(dev(H), dev(g), Ctp, dev(dt) if n_c else None)
    st = prob.read_stats()
    U = U.cpu().numpy().astype(np.float64)
    y = y.cpu().numpy().astype(np.float64)
    assert st["status"] == lib.GM_OK and st["converged"] == 1, st
    assert st["iters"] <= 40, st
    assert st["r_prim"] <= wl.tol and st["r_dual"] <= wl.tol, st
    # the FP64 certificate the library reports matches one recomputed here, and is near tol
    At, l, h = oqp.stack_rows(lo, hi, Ct64 if n_c else None, dt64 if n_c else None)
    cert = oqp.kkt_certificate(H64, g64, At, l, h, U, y)
    assert abs(st["kkt_stat"] - cert["stationarity"]) <= 1e-6 * max(1.0, cert["stationarity"]) + 1e-9
    assert max(cert.values()) <= 100 * wl.tol, cert
    # distance to U*: H is strongly convex, so |U - U*| <= (stationarity + complementarity terms) / lambda_min
    lam = np.linalg.eigvalsh(H64).min()
    bound = 2 * (cert["stationarity"] + np.sqrt(cert["complementarity"] + cert["primal"])) / lam + 1e-5
    assert np.abs(U - Ux).max() <= bound, (np.abs(U - Ux).max(), bound)
    # and ADMM on the same QP lands on the same optimum
    Ua, _ = prob.qp_solve(dev(H), dev(g), Ctp, dev(dt) if n_c else None)
    sta = prob.read_stats()
    assert sta["converged"] == 1
    assert np.abs(Ua.cpu().numpy() - Ux).max() <= 2 * max(sta["r_dual"], sta["kkt_stat"]) / lam + 1e-5


def test_ipm_iteration_cap_is_reported(lib):
    """One iteration cannot converge: the call returns GM_OK and stats says GM_ERR_NOT_CONVERGED."""
    wl, Cx, dx, (H, g, Ct, dt) = _qp(True)
    prob = lib.RTIProblem(wl.M, wl.src, wl.dst, wl.nu, wl.act_node, wl.K, wl.W, wl.dt, wl.blob, wl.N,
                          wl.Qdiag, wl.Rdiag, wl.x_ref, wl.u_ref, wl.u_lo, wl.u_hi, Cx=Cx, dx=dx,
                          rho=wl.rho, tol=wl.tol, max_iter=wl.max_iter)
    torch = prob.torch
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")  # noqa: E731
    prob.qp_solve_ipm(dev(H), dev(g), dev(dense_to_packed_ct(Ct, wl.N, wl.M, 2, wl.nu)), dev(dt), max_iter=1)
    st = prob.read_stats()
    assert st["status"] == lib.GM_ERR_NOT_CONVERGED and st["converged"] == 0 and st["iters"] == 1, st
