"""Pins of the oracle's QP solvers against brute force, the uncondensed QP and closed forms.  No GPU."""
import numpy as np
import pytest

from oracle import condense as cd
from oracle import qp
from oracle import rti
from synth import small_chain

from test_oracle_condense import random_ltv


def random_qp(n, m, seed, active=True):
    rng = np.random.default_rng(seed)
    L = rng.normal(0, 1, (n, n))
    H = L @ L.T + 0.1 * np.eye(n)
    g = rng.normal(0, 3.0 if active else 0.1, n)
    lo = -np.ones(n)
    hi = np.ones(n)
    C = rng.normal(0, 1, (m, n))
    d = rng.uniform(-0.2, 0.5, m) if active else np.full(m, 100.0)
    return H, g, lo, hi, C, d


@pytest.mark.parametrize("seed", range(6))
def test_exact_solution_equals_brute_force_active_sets(seed):
    H, g, lo, hi, C, d = random_qp(4, 3, seed)
    U, y, info = qp.solve_exact(H, g, lo, hi, C, d)
    bf = qp.brute_force(H, g, lo, hi, C, d)
    assert bf is not None
    assert np.abs(U - bf[0]).max() <= 1e-10
    At, l, h = qp.stack_rows(lo, hi, C, d)
    cert = qp.kkt_certificate(H, g, At, l, h, U, y)
    assert max(cert.values()) <= 1e-9, cert


def test_unconstrained_closed_form():
    """Loose bounds: the optimum is U = -H^{-1} g."""
    H, g, lo, hi, C, d = random_qp(6, 4, 1, active=False)
    U, _, _ = qp.solve_exact(H, g, lo * 1e3, hi * 1e3, C, d)
    assert np.allclose(U, np.linalg.solve(H, -g), atol=1e-11)


@pytest.mark.parametrize("seed", [0, 3])
def test_condensed_equals_uncondensed_qp(seed):
    """The condensed QP's U* equals the (x, u) QP's U* with the dynamics as equalities (Sec. III-B)."""
    M, N, nu = 2, 3, 2
    A, B, c, x0, Qd, Rd, xr, ur, Cx, dx, nbh = random_ltv(M, N, nu, 1, seed, n_c=1, scale=0.3)
    B *= 0.5
    dx = dx + 2.0            # mostly loose half-spaces, some active
    lo = -0.5 * np.ones((N, nu))
    hi = 0.5 * np.ones((N, nu))
    blocks = cd.blocks_from_dense(A, B, c, nbh)
    H, g, Ct, dt, _, _ = cd.condense_recursive(blocks, x0, Qd, Rd, xr, ur, Cx, dx)
    U, y, _ = qp.solve_exact(H, g, lo.reshape(-1), hi.reshape(-1), Ct, dt)
    Uu = qp.uncondensed(A, B, c, x0, Qd, Rd, xr, ur, lo, hi, Cx, dx)
    assert Uu is not None
    assert np.abs(U - Uu.reshape(-1)).max() <= 1e-10
    # the instance must exercise at least one active inequality
    At, l, h = qp.stack_rows(lo.reshape(-1), hi.reshape(-1), Ct, dt)
    assert np.any(np.abs(At @ U - h) < 1e-9) or np.any(np.abs(At @ U - l) < 1e-9)


@pytest.mark.parametrize("seed", range(4))
def test_admm_converges_to_the_optimum(seed):
    """The ADMM recurrence (fixed rho) reaches U* when run to a tight residual."""
    H, g, lo, hi, C, d = random_qp(8, 6, 10 + seed)
    U, y, _ = qp.solve_exact(H, g, lo, hi, C, d)
    Ua, z, ya, it, rp, rd, ok = qp.admm(H, g, lo, hi, C, d, rho=1.0, tol=1e-11, max_iter=200000)
    assert ok
    assert np.abs(Ua - U).max() <= 1e-8


def test_admm_dual_residual_identity():
    """With an exact U-update, H U + g + A~'y = rho A~'(z_prev - z) at every iteration."""
    H, g, lo, hi, C, d = random_qp(5, 4, 21)
    At, l, h = qp.stack_rows(lo, hi, C, d)
    rho = 0.7
    P = H + rho * At.T @ At
    U = np.zeros(5)
    y = np.zeros(At.shape[0])
    z = np.clip(At @ U, l, h)
    for _ in range(30):
        z_prev = z
        U = np.linalg.solve(P, At.T @ (rho * z - y) - g)
        a = At @ U
        z = np.clip(a + y / rho, l, h)
        y = y + rho * (a - z)
        assert np.allclose(H @ U + g + At.T @ y, rho * At.T @ (z_prev - z), atol=1e-11)
    # and the oracle's recurrence produces the same iterates
    Ua, *_ = qp.admm(H, g, lo, hi, C, d, rho=rho, tol=0.0, max_iter=30)
    assert np.allclose(Ua, U, atol=1e-12)


def test_row_scaled_admm_reaches_the_same_optimum():
    """Dividing half-space rows by their norms changes neither the feasible set nor U*.

    Rows are given norms from 1e-7 to 1e2; the scaled recurrence reaches the
    exact optimum and returns multipliers certified for the original rows.
    """
    H, g, lo, hi, C, d = random_qp(8, 6, 41)
    f = np.array([1e-7, 1e-4, 1e-2, 1.0, 10.0, 100.0])
    C, d = C * f[:, None], d * f
    U, y, _ = qp.solve_exact(H, g, lo, hi, C, d)
    Ua, za, ya, it, rp, rd, ok = qp.admm(H, g, lo, hi, C, d, rho=1.0, tol=1e-11, max_iter=200000,
                                         scale_rows=True)
    assert ok and np.abs(Ua - U).max() <= 1e-8
    At, l, h = qp.stack_rows(lo, hi, C, d)
    cert = qp.kkt_certificate(H, g, At, l, h, Ua, ya)
    assert cert["stationarity"] <= 1e-9 and cert["dual"] <= 1e-12


@pytest.mark.parametrize("seed", range(3))
def test_adaptive_rho_admm_reaches_the_optimum(seed):
    """Re-factoring with an adapted rho keeps the fixed point: the same U* is reached."""
    H, g, lo, hi, C, d = random_qp(8, 6, 50 + seed)
    f = np.array([1e-5, 1e-3, 1.0, 1.0, 30.0, 1e2])
    C, d = C * f[:, None], d * f
    U, y, _ = qp.solve_exact(H, g, lo, hi, C, d)
    Ua, za, ya, it, rp, rd, ok = qp.admm(H, g, lo, hi, C, d, rho=0.1, tol=1e-11, max_iter=100000,
                                         scale_rows=True, adapt_every=25)
    assert ok and np.abs(Ua - U).max() <= 1e-8


def test_polish_recovers_the_optimum_from_a_loose_admm_iterate():
    H, g, lo, hi, C, d = random_qp(8, 6, 31)
    U, _, _ = qp.solve_exact(H, g, lo, hi, C, d)
    Ua, z, ya, it, rp, rd, ok = qp.admm(H, g, lo, hi, C, d, rho=1.0, tol=1e-4, max_iter=100000)
    assert ok and np.abs(Ua - U).max() > 1e-9
    Up, yp, accepted = qp.polish(H, g, lo, hi, C, d, Ua, z, ya)
    assert accepted
    assert np.abs(Up - U).max() <= 1e-10


def test_small_chain_optimum_certificate():
    """Chain of 10 (N=10, nu=4): the oracle's U* carries an FP64 KKT certificate."""
    wl = small_chain()
    r = rti.rti_step(wl, return_all=True)
    At, l, h = qp.stack_rows(wl.u_lo.reshape(-1).astype(float), wl.u_hi.reshape(-1).astype(float),
                             r["Ct"] if r["Ct"].size else None, r["dt"] if r["dt"].size else None)
    cert = qp.kkt_certificate(r["H"], r["g"], At, l, h, r["U"].reshape(-1), r["y"])
    assert max(cert.values()) <= 1e-12


# ------------------------------------------------------------------ primal infeasibility
def _box_row_conflict(n=3):
    """|U_i| <= 1 and U_0 <= -2: infeasible; the Farkas direction is -1 on the lower bound of
    box row 0 and +1 on the half-space row (A~'v = 0, support 1 - 2 = -1)."""
    lo, hi = -np.ones(n), np.ones(n)
    C = np.zeros((1, n))
    C[0, 0] = 1.0
    return lo, hi, C, np.array([-2.0])


def test_certificate_by_farkas_on_a_hand_made_direction():
    lo, hi, C, d = _box_row_conflict()
    At, l, h = qp.stack_rows(lo, hi, C, d)
    v = np.array([-1.0, 0.0, 0.0, 1.0])
    assert qp.primal_infeasible(At, l, h, v)
    assert qp.primal_infeasible(At, l, h, 7.5 * v)              # scale-free
    assert not qp.primal_infeasible(At, l, h, -v)               # -v: dy < 0 on a row with l = -inf
    assert not qp.primal_infeasible(At, l, h, v + np.array([0, 0.1, 0, 0]))   # A~'v != 0
    assert not qp.primal_infeasible(At, l, h, np.zeros(4))
    # the same direction with a feasible bound d = -0.5: support 1 - 0.5 > 0
    At2, l2, h2 = qp.stack_rows(lo, hi, C, np.array([-0.5]))
    assert not qp.primal_infeasible(At2, l2, h2, v)


@pytest.mark.parametrize("scale_rows", [False, True])
def test_admm_stops_on_a_constructed_infeasible_qp(scale_rows):
    """ADMM's dual step converges to the Farkas direction (up to scale) and the run stops."""
    lo, hi, C, d = _box_row_conflict()
    H, g = np.diag([1.0, 2.0, 3.0]), np.array([0.3, -0.2, 0.1])
    *_, ok, info = qp.admm(H, g, lo, hi, C * 4.0, d * 4.0, rho=0.1, tol=1e-8, max_iter=5000,
                           scale_rows=scale_rows, adapt_every=25, return_info=True)
    assert not ok and info["infeasible"]
    v = info["dy"] / np.abs(info["dy"]).max()
    # original rows: box row 0 gets -1 and the half-space row (C scaled by 4) gets +1/4
    assert np.abs(v / v[0] * -1 - np.array([-1.0, 0.0, 0.0, 0.25])).max() <= 1e-3, v


def _lp_margin(lo, hi, C, d):
    """t* = min t over lo <= U <= hi, C U <= d + t (scipy's HiGHS): the set is feasible iff t* <= 0."""
    from scipy.optimize import linprog
    n, m = lo.size, C.shape[0]
    res = linprog(np.r_[np.zeros(n), 1.0], A_ub=np.hstack([C, -np.ones((m, 1))]), b_ub=d,
                  bounds=[(a, b) for a, b in zip(lo, hi)] + [(None, None)], method="highs")
    assert res.status == 0
    return res.fun


@pytest.mark.parametrize("seed", range(16))
def test_infeasibility_verdict_matches_linear_programming(seed):
    """On random box + half-space sets, ADMM flags infeasibility exactly when an LP says the
    set is empty (sets within 0.05 of the boundary are skipped)."""
    rng = np.random.default_rng(100 + seed)
    n, m = 5, 8
    H, g, lo, hi, C, _ = random_qp(n, m, 200 + seed)
    d = rng.uniform(-2.0, 1.0, m)
    t = _lp_margin(lo, hi, C, d)
    if abs(t) < 0.05:
        pytest.skip(f"margin {t:.3f} too close to the boundary")
    *_, ok, info = qp.admm(H, g, lo, hi, C, d, rho=0.1, tol=1e-7, max_iter=20000, scale_rows=True,
                           adapt_every=25, return_info=True)
    if t > 0:
        assert info["infeasible"] and not ok
        At, l, h = qp.stack_rows(lo, hi, C, d)
        assert qp.primal_infeasible(At, l, h, info["dy"], eps=1e-3)
    else:
        assert ok and not info["infeasible"]


def stall_qp(seed=5):
    """A QP with the condensed stage structure (N = 4 stages, 2 inputs, 3 half-spaces per
    stage acting on the inputs up to their stage) whose feasible set has active rows."""
    N, NU, MNC = 4, 2, 3
    rng = np.random.default_rng(seed)
    n, m = N * NU, N * MNC
    L = rng.normal(0, 1, (n, n))
    H = L @ L.T + 0.1 * np.eye(n)
    g = rng.normal(0, 3.0, n)
    C = rng.normal(0, 1, (m, n))
    for k in range(N):
        C[k * MNC:(k + 1) * MNC, (k + 1) * NU:] = 0.0
    d = rng.uniform(0.2, 1.5, m)
    kw = dict(rho=0.1, tol=1e-6, max_iter=20000, scale_rows=True, adapt_every=25)
    return H, g, -np.ones(n), np.ones(n), C, d, kw


def stall_warm_duals(n, m, seed=5, scale=1e4):
    """A deliberately bad warm start: half-space duals of size 1e4."""
    y0 = np.zeros(n + m)
    y0[n:] = np.random.default_rng(seed).normal(0.0, 1.0, m) * scale
    return y0


def test_stalled_warm_start_restarts_as_the_cold_solve():
    """Duals 1e4 off: without the stall rule the recurrence does not reach tol in 20000
    iterations; with it the warm start is dropped at a stall test, and since that test falls
    on a multiple of the adaptation period the restarted run takes exactly the cold solve's
    iterates (same U to rounding, count = restart iteration + cold count)."""
    H, g, lo, hi, C, d, kw = stall_qp()
    n = H.shape[0]
    y0 = stall_warm_duals(n, C.shape[0])
    w = qp.admm(H, g, lo, hi, C, d, U0=np.zeros(n), y0=y0, stall_every=25, return_info=True, **kw)
    c = qp.admm(H, g, lo, hi, C, d, **kw)
    assert w[7]["restarted"] and w[6] and c[6]
    assert (w[3] - c[3]) % 25 == 0 and w[3] > c[3]          # the restart came at a stall test
    assert np.abs(w[0] - c[0]).max() <= 1e-12
    nr = qp.admm(H, g, lo, hi, C, d, U0=np.zeros(n), y0=y0, **kw)
    assert not nr[6] and nr[3] == kw["max_iter"]


def test_good_warm_start_is_kept_and_a_nan_one_restarts_at_once():
    H, g, lo, hi, C, d, kw = stall_qp()
    n = H.shape[0]
    Ue, ye, _ = qp.solve_exact(H, g, lo, hi, C, d)
    w = qp.admm(H, g, lo, hi, C, d, U0=Ue, y0=ye, stall_every=25, return_info=True, **kw)
    assert w[6] and not w[7]["restarted"] and w[3] <= 3
    U0 = np.zeros(n)
    U0[3] = np.nan
    w = qp.admm(H, g, lo, hi, C, d, U0=U0, stall_every=25, return_info=True, **kw)
    assert w[6] and w[7]["restarted"] and np.isfinite(w[0]).all()
    assert np.abs(w[0] - Ue).max() <= 10 * kw["tol"] / kw["rho"]


def test_redundant_rows_cannot_be_violated_and_dropping_them_keeps_the_optimum():
    """The redundant-row test against sampling: no U in the box (vertices included) violates a
    row it drops; the ADMM with and without the drop reaches the exact optimum of the full QP,
    with zero multipliers on the dropped rows and a valid KKT certificate."""
    rng = np.random.default_rng(2)
    H, g, lo, hi, C, d = random_qp(6, 40, 4)
    d = d + rng.uniform(0.0, 4.0, d.size)               # a mix of redundant and binding rows
    red = qp.redundant_rows(C, d, lo, hi)
    assert 0 < red.sum() < red.size
    Us = rng.uniform(lo, hi, (20000, lo.size))
    Us = np.vstack([Us, np.where(rng.random((2000, lo.size)) < 0.5, lo, hi)])
    assert (Us @ C[red].T <= d[red]).all()
    # the support is attained at a vertex: a row just above the margin is kept
    sup = np.maximum(C * hi, C * lo).sum(1)
    assert not qp.redundant_rows(C, sup + 1e-9, lo, hi).any()
    Ue, ye, _ = qp.solve_exact(H, g, lo, hi, C, d)
    assert np.abs(ye[lo.size:][red]).max() <= 1e-9
    for drop in (True, False):
        U, z, y, it, rp, rd, ok = qp.admm(H, g, lo, hi, C, d, rho=0.1, tol=1e-9, max_iter=20000,
                                          scale_rows=True, adapt_every=25, drop_redundant=drop)
        assert ok and np.abs(U - Ue).max() <= 1e-6, (drop, np.abs(U - Ue).max())
        if drop:
            assert (y[lo.size:][red] == 0).all()
        At, l, h = qp.stack_rows(lo, hi, C, d)
        cert = qp.kkt_certificate(H, g, At, l, h, U, y)
        assert max(cert.values()) <= 1e-6, cert
