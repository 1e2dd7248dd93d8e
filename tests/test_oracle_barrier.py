"""Pins of the barrier-cost obstacle oracle (oracle.barrier, Sec. VI-B) to things other than itself.

* the relaxed barrier is -ln s above delta, and its slope and curvature are those of its
  own values (central differences), continuous across delta;
* the folded QP is the second-order Taylor model of the barrier-augmented cost at U_hat:
  its gradient and Hessian there match central differences of that cost;
* Newton steps on the fold converge to the minimiser of the barrier-augmented cost found
  by an independent solver (scipy BFGS on the cost's values);
* as mu -> 0 with the box kept, the barrier minimiser approaches the constrained optimum
  of the same QP (solve_exact), the central-path property of the log barrier.
"""
import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import barrier as br
from oracle import qp as oqp


def _qp(seed, n=6, rows=10, feasible=True):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, n))
    H = X @ X.T + 0.5 * np.eye(n)
    g = rng.normal(size=n)
    Ct = rng.normal(size=(rows, n))
    U_hat = rng.uniform(-0.3, 0.3, n)
    s = rng.uniform(0.05, 1.0, rows) if feasible else rng.uniform(-0.2, 1.0, rows)
    dt = Ct @ U_hat + s
    return H, g, Ct, dt, U_hat


def test_relaxed_barrier_values_slope_curvature():
    delta = 0.05
    s = np.concatenate([np.linspace(-0.3, 0.049, 23), np.linspace(0.0501, 2.0, 31)])
    b0, b1, b2 = br.relaxed_log_barrier(s, delta)
    above = s > delta
    assert np.array_equal(b0[above], -np.log(s[above]))
    h = 1e-5
    f = lambda x: br.relaxed_log_barrier(x, delta)[0]   # noqa: E731
    np.testing.assert_allclose(b1, (f(s + h) - f(s - h)) / (2 * h), rtol=1e-6, atol=1e-6)
    h2 = 1e-4
    np.testing.assert_allclose(b2, (f(s + h2) - 2 * f(s) + f(s - h2)) / h2 ** 2, rtol=1e-4)
    assert (b2 > 0).all()
    # value, slope and curvature agree across s = delta
    lo = br.relaxed_log_barrier(np.array([delta * (1 - 1e-9)]), delta)
    hi = br.relaxed_log_barrier(np.array([delta * (1 + 1e-9)]), delta)
    for a, b in zip(lo, hi):
        assert abs(a[0] - b[0]) <= 1e-6 * max(1.0, abs(b[0]))
    # finite inside an obstacle
    assert np.isfinite(br.relaxed_log_barrier(np.array([-1.0]), delta)).all()


@pytest.mark.parametrize("feasible", [True, False])
def test_fold_is_the_second_order_model(feasible):
    mu, delta = 0.05, 0.1
    H, g, Ct, dt, U_hat = _qp(1 if feasible else 2, feasible=feasible)
    Hb, gb = br.barrier_fold(H, g, Ct, dt, U_hat, mu, delta)
    phi = lambda U: br.barrier_objective(H, g, Ct, dt, U, mu, delta)   # noqa: E731
    n = len(U_hat)
    E = np.eye(n)
    h = 1e-5
    grad = np.array([(phi(U_hat + h * E[i]) - phi(U_hat - h * E[i])) / (2 * h) for i in range(n)])
    np.testing.assert_allclose(Hb @ U_hat + gb, grad, rtol=1e-6, atol=1e-6)
    h = 1e-4
    hess = np.array([[(phi(U_hat + h * (E[i] + E[j])) - phi(U_hat + h * (E[i] - E[j]))
                       - phi(U_hat - h * (E[i] - E[j])) + phi(U_hat - h * (E[i] + E[j]))) / (4 * h * h)
                      for j in range(n)] for i in range(n)])
    np.testing.assert_allclose(Hb, hess, rtol=1e-4, atol=1e-4)
    assert np.allclose(Hb, Hb.T) and np.linalg.eigvalsh(Hb).min() > 0


def _newton(H, g, Ct, dt, U0, mu, delta, lo=None, hi=None, iters=60):
    """Sequential QPs on the fold with a backtracking line search on the barrier cost."""
    phi = lambda U: br.barrier_objective(H, g, Ct, dt, U, mu, delta)   # noqa: E731
    U = U0.copy()
    for _ in range(iters):
        Hb, gb = br.barrier_fold(H, g, Ct, dt, U, mu, delta)
        if lo is None:
            V = np.linalg.solve(Hb, -gb)
        else:
            V = oqp.solve_exact(Hb, gb, lo, hi)[0]
        step = V - U
        if np.abs(step).max() < 1e-13:
            break
        t, f0 = 1.0, phi(U)
        while phi(U + t * step) > f0 and t > 1e-12:
            t *= 0.5
        U = U + t * step
    return U


def test_newton_on_the_fold_reaches_the_barrier_minimum():
    mu, delta = 0.05, 0.1
    H, g, Ct, dt, U_hat = _qp(3, feasible=False)
    U = _newton(H, g, Ct, dt, U_hat, mu, delta)
    ref = minimize(lambda V: br.barrier_objective(H, g, Ct, dt, V, mu, delta), U_hat, method="BFGS",
                   options=dict(gtol=1e-10, maxiter=2000))
    np.testing.assert_allclose(U, ref.x, atol=1e-5)
    n = len(U)
    h = 1e-6
    phi = lambda V: br.barrier_objective(H, g, Ct, dt, V, mu, delta)   # noqa: E731
    grad = np.array([(phi(U + h * np.eye(n)[i]) - phi(U - h * np.eye(n)[i])) / (2 * h) for i in range(n)])
    assert np.abs(grad).max() < 1e-6


def test_barrier_minimiser_approaches_the_constrained_optimum():
    H, g, Ct, dt, U0 = _qp(4, n=5, rows=8)
    g = 3.0 * g                       # pull the optimum against some rows
    lo, hi = -np.ones(5), np.ones(5)
    U_star, _, _ = oqp.solve_exact(H, g, lo, hi, Ct, dt)
    assert (dt - Ct @ U0 > 0).all() and (np.abs(U0) < 1).all()
    assert (dt - Ct @ U_star).min() < 1e-9          # some rows are active at the optimum
    errs = []
    for mu in (1e-2, 1e-3, 1e-4, 1e-5):
        U = _newton(H, g, Ct, dt, U0, mu, 1e-9, lo, hi, iters=200)
        assert (dt - Ct @ U > 0).all()
        errs.append(np.abs(U - U_star).max())
        U0 = U
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-3, errs
