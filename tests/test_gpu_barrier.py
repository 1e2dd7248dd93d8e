"""Barrier-cost obstacle variant (gm_barrier_fold, barrier RTI step) against the oracle.  Needs a GPU.

The oracle (oracle.barrier) folds the relaxed log barrier of every obstacle row into H and
g in FP64; it is pinned in test_oracle_barrier.  Here the device fold takes the same FP32
inputs and must match element by element within the FP32 rounding of its Gram sum; the
barrier RTI step must reach the oracle's exact optimum of the folded box-only QP.
"""
import numpy as np
import pytest

from gpu_helpers import dense_to_packed_ct, ocd, oracle_linearize, orti, packed_to_dense_ct
from oracle import barrier as obr
from synth import paper_chain, small_chain

pytestmark = pytest.mark.gpu


def _fold_bounds(H, g, Ct, dt, U_hat, mu, delta):
    """Element-wise error allowance of an FP32 fold: 1e-5 of the magnitude sums it adds up."""
    a = Ct @ U_hat
    _, b1, b2 = obr.relaxed_log_barrier(dt - a, delta)
    absH = np.abs(H) + np.abs(Ct).T @ (mu * b2[:, None] * np.abs(Ct))
    absg = np.abs(g) + np.abs(Ct).T @ np.abs(mu * b1 + mu * b2 * a)
    return 1e-5 * absH + 1e-6, 1e-5 * absg + 1e-6


@pytest.mark.parametrize("clearance", [(1e-3, 2e-2), (-4e-3, 2e-2)])
def test_barrier_fold_matches_oracle(lib, clearance):
    """Rows at clearances drawn from a range around delta (negative: inside an obstacle)."""
    wl = small_chain()
    u_hat = np.random.default_rng(3).uniform(-0.5, 0.5, (wl.N, wl.nu))
    xo, Ao, Bo, co = oracle_linearize(wl, u_hat)
    gnn, gr = orti.model_of(wl)
    nbh = [gr.in_ball(i, wl.K) for i in range(wl.M)]
    rng = np.random.default_rng(11)
    n = rng.normal(0, 1, (wl.N, wl.M, 2, 3))
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    p = xo[1:, :, None, :3]
    dx = np.einsum("kics,kics->kic", n, np.broadcast_to(p, n.shape)) + rng.uniform(*clearance, n.shape[:3])
    H, g, Ct, dt, _, _ = ocd.condense_recursive(ocd.blocks_from_dense(Ao, Bo, co, nbh), xo[0].reshape(-1),
                                                wl.Qdiag, wl.Rdiag, wl.x_ref, wl.u_ref, n, dx)
    H, g, Ct, dt = (np.asarray(a, np.float32).astype(np.float64) for a in (H, g, Ct, dt))
    U_hat = u_hat.reshape(-1).astype(np.float32).astype(np.float64)
    mu, delta = 1e-3, 5e-3
    s = dt - Ct @ U_hat
    assert (s > delta).any() and (s <= delta).any()       # both branches of the barrier
    assert (s < 0).any() == (clearance[0] < 0)
    Hx, gx = obr.barrier_fold(H, g, Ct, dt, U_hat, mu, delta)
    prob = lib.RTIProblem(wl.M, wl.src, wl.dst, wl.nu, wl.act_node, wl.K, wl.W, wl.dt, wl.blob, wl.N,
                          wl.Qdiag, wl.Rdiag, wl.x_ref, wl.u_ref, wl.u_lo, wl.u_hi,
                          Cx=n.astype(np.float32), dx=dx.astype(np.float32), rho=wl.rho, tol=wl.tol,
                          max_iter=wl.max_iter)
    torch = prob.torch
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")  # noqa: E731
    Hd, gd = dev(H), dev(g)
    prob.barrier_fold(Hd, gd, dev(dense_to_packed_ct(Ct, wl.N, wl.M, 2, wl.nu)), dev(dt), U_hat, mu, delta)
    bH, bg = _fold_bounds(H, g, Ct, dt, U_hat, mu, delta)
    dH = np.abs(Hd.cpu().numpy() - Hx)
    dg = np.abs(gd.cpu().numpy() - gx)
    assert (dH <= bH).all(), (dH.max(), np.unravel_index((dH / bH).argmax(), dH.shape))
    assert (dg <= bg).all(), (dg.max(), (dg / bg).max())
    # the box-only solve of the folded QP reaches the oracle's optimum
    U, _ = prob.qp_solve(Hd, gd, box_only=True)
    st = prob.read_stats()
    assert st["status"] == 0 and st["converged"] == 1, st
    lo, hi = wl.u_lo.reshape(-1).astype(np.float64), wl.u_hi.reshape(-1).astype(np.float64)
    Ux = orti.qp.solve_exact(Hx, gx, lo, hi)[0]
    lam = np.linalg.eigvalsh(Hx).min()
    assert np.abs(U.cpu().numpy() - Ux).max() <= 2 * max(st["r_dual"], st["kkt_stat"]) / lam + 1e-4


def test_barrier_rti_steps_match_oracle(lib):
    """Two barrier RTI steps (Alg. 1 with the obstacle rows in the cost) against the oracle."""
    wl = small_chain(n_spheres=3)
    mu, delta = 1e-3, 5e-3
    prob = lib.RTIProblem.from_workload(wl, barrier=(mu, delta))
    u_prev = None
    for step in range(2):
        U = prob.step(wl.x0).cpu().numpy().astype(np.float64).reshape(wl.N, wl.nu)
        st = prob.read_stats()
        uh = None if u_prev is None else orti.shift(u_prev)
        rb = orti.rti_step(wl, u_hat=uh, solver="exact", barrier=(mu, delta), return_all=True)
        assert st["status"] == 0 and st["converged"] == 1, st
        lam = np.linalg.eigvalsh(rb["H"]).min()
        err = np.abs(U - rb["U"]).max()
        assert err <= 2 * max(st["r_dual"], st["kkt_stat"]) / lam + 1e-4, (step, err)
        if step == 0:
            # the barrier changes the answer: the plain QP without the obstacle terms differs
            rc = orti.rti_step(wl, u_hat=uh, solver="exact", barrier=(1e-12, delta), return_all=True)
            assert np.abs(rb["U"] - rc["U"]).max() > 10 * (err + 1e-4)
        u_prev = rb["U"]


def test_barrier_fold_paper_scale(lib):
    """Chain of 1000, N=20, 5 spheres: the device fold of the device-condensed QP against the
    FP64 fold of the same FP32 arrays, every element, and a converged barrier RTI step."""
    wl = paper_chain()
    mu, delta = 1e-3, 5e-3
    prob = lib.RTIProblem.from_workload(wl)
    u_hat = np.random.default_rng(7).uniform(-0.2, 0.2, (wl.N, wl.nu)).astype(np.float32)
    x_hat, A, B, c = prob.linearize(wl.x0, u_hat)
    H, g, Ct, dt = prob.condense(x_hat, A, B, c)
    H64, g64, dt64 = (t.cpu().numpy().astype(np.float64) for t in (H, g, dt))
    Ct64 = packed_to_dense_ct(Ct.cpu().numpy(), wl.N, wl.M, prob.n_c, wl.nu).astype(np.float64)
    U_hat = u_hat.reshape(-1).astype(np.float64)
    Hx, gx = obr.barrier_fold(H64, g64, Ct64, dt64, U_hat, mu, delta)
    prob.barrier_fold(H, g, Ct, dt, U_hat, mu, delta)
    bH, bg = _fold_bounds(H64, g64, Ct64, dt64, U_hat, mu, delta)
    dH = np.abs(H.cpu().numpy() - Hx)
    dg = np.abs(g.cpu().numpy() - gx)
    assert (dH <= bH).all(), dH.max()
    assert (dg <= bg).all(), dg.max()
    prob.close()
    pb = lib.RTIProblem.from_workload(wl, barrier=(mu, delta))
    U = pb.step(wl.x0).cpu().numpy()
    st = pb.read_stats()
    assert st["status"] == 0 and st["converged"] == 1, st
    assert np.isfinite(U).all() and (np.abs(U) <= 1 + 1e-6).all()
