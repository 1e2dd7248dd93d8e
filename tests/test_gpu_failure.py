"""Failure paths of the device solve, in the forms that fault no GPU (needs a GPU).

* A bounded wait that runs out: every grid barrier of the cooperative ADMM and FP64
  factor kernels is capped at one poll (gm_ctx_set_timeout_spins), so the kernels give
  up, record GM_ERR_TIMEOUT and return; the same context then solves normally.
* A NaN in the measured state (host-side input): the step ends with GM_ERR_NUMERIC, and
  the next step of the same warm-started context starts from Algorithm 1's initial
  trajectory and converges to the oracle's optimum.
* A warm start that stalls (dual start 1e4 off, host-side input) or is NaN: the solve
  drops it and restarts cold inside the call (GM_STALLED), like the oracle's ADMM with the
  same stall rule, and returns the cold solve's U.
"""
import numpy as np
import pytest

from gpu_helpers import oqp, orti
from synth import small_chain

pytestmark = pytest.mark.gpu


def _spheres_chain():
    # two spheres placed clear of the rollout: a feasible QP with 200 half-space rows, so the
    # ADMM runs as a multi-CTA cooperative grid
    return small_chain(tol=1e-4, n_spheres=2, sphere_clear=0.15)


def _qp(prob, wl):
    """The condensed QP of wl's first step (u_hat = 0), on the device."""
    t = prob.torch
    x = t.as_tensor(np.asarray(wl.x0, np.float32).reshape(-1), device="cuda")
    zeros_u = t.zeros(prob.N, prob.nu, dtype=t.float32, device="cuda")
    x_hat, A, B, c = prob.linearize(x, zeros_u)
    return prob.condense(x_hat, A, B, c)


def test_grid_barrier_timeout_is_reported_and_the_context_recovers(lib):
    wl = _spheres_chain()
    prob = lib.RTIProblem.from_workload(wl)
    H, g, Ct, dt = _qp(prob, wl)
    lib.gm_ctx_set_timeout_spins(prob.ctx, 1)
    prob.qp_solve(H, g, Ct, dt)
    st = prob.read_stats()
    assert st["status"] == lib.GM_ERR_TIMEOUT, st
    lib.gm_ctx_set_timeout_spins(prob.ctx, 0)
    U, _ = prob.qp_solve(H, g, Ct, dt)
    st = prob.read_stats()
    assert st["status"] == lib.GM_OK and st["converged"] == 1, st
    Hd, gd, Cd, dd = (np.asarray(a.cpu().numpy(), np.float64) for a in (H, g, Ct, dt))
    from gpu_helpers import packed_to_dense_ct
    C = packed_to_dense_ct(Cd, wl.N, wl.M, 2, wl.nu)
    Ue, _, _ = oqp.solve_exact(Hd, gd, wl.u_lo.reshape(-1), wl.u_hi.reshape(-1), C, dd)
    assert np.abs(U.cpu().numpy() - Ue).max() <= 10 * wl.tol / wl.rho


@pytest.mark.parametrize("mixed_graph", [False, True])
def test_nan_state_reports_numeric_and_the_next_step_recovers(lib, mixed_graph):
    wl = small_chain()
    kw = dict(precision=lib.GM_PREC_MIXED, graph=True) if mixed_graph else {}
    prob = lib.RTIProblem.from_workload(wl, warm=True, **kw)
    x_good = np.asarray(wl.x0, np.float32).reshape(-1)
    prob.step(x_good)                                 # a good step first: the warm start is armed
    assert prob.read_stats()["status"] == lib.GM_OK
    x_bad = x_good.copy()
    x_bad[7] = np.nan
    prob.step(x_bad)
    st = prob.read_stats()
    assert st["status"] == lib.GM_ERR_NUMERIC, st
    # after the failed step u_hat is back at zero: the next step is a fresh step of the oracle
    U = prob.step(x_good).cpu().numpy().astype(np.float64).reshape(wl.N, wl.nu)
    st = prob.read_stats()
    assert st["status"] in (lib.GM_OK, lib.GM_STALLED) and st["converged"] == 1, st
    ref = orti.rti_step(wl, solver="exact")
    assert np.isfinite(U).all()
    assert np.abs(U - ref).max() <= 10 * wl.tol / wl.rho + 1e-4, np.abs(U - ref).max()


def _stall_problem(lib):
    """A context sized for the staged test QP (N = 4, nu = 2, 3 half-space rows per stage:
    three nodes with one row each); the QP itself is passed to gm_qp_solve."""
    from synth import random_instance
    wl = random_instance(0, M=3, N=4, nu=2, K=1, W=32)
    prob = lib.RTIProblem(wl.M, wl.src, wl.dst, wl.nu, wl.act_node, wl.K, wl.W, wl.dt, wl.blob, wl.N,
                          wl.Qdiag, wl.Rdiag, wl.x_ref, wl.u_ref, wl.u_lo, wl.u_hi,
                          Cx=np.zeros((4, 3, 1, 3), np.float32), dx=np.ones((4, 3, 1), np.float32),
                          rho=0.1, tol=1e-6, max_iter=20000)
    return prob


def _dev_qp(prob, H, g, C, d):
    from gpu_helpers import dense_to_packed_ct
    t = prob.torch
    dev = lambda a: t.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")  # noqa: E731
    H32, g32, C32, d32 = (np.asarray(a, np.float32) for a in (H, g, C, d))
    return (dev(H32), dev(g32), dev(dense_to_packed_ct(C32, 4, 3, 1, 2)), dev(d32),
            tuple(a.astype(np.float64) for a in (H32, g32, C32, d32)))


def test_stalled_warm_start_restarts_cold_like_the_oracle(lib):
    """Half-space duals 1e4 off: the oracle's ADMM without the stall rule does not reach tol
    in 20000 iterations; with the rule both the oracle and the device drop the warm start at a
    stall test and restart cold (GM_STALLED), and return the cold solve's U."""
    from test_oracle_qp import stall_qp, stall_warm_duals
    H, g, lo, hi, C, d, kw = stall_qp()
    prob = _stall_problem(lib)
    Hd, gd, Ctd, dtd, (H64, g64, C64, d64) = _dev_qp(prob, H, g, C, d)
    n = H.shape[0]
    y0 = stall_warm_duals(n, C.shape[0])
    ref = oqp.admm(H64, g64, lo, hi, C64, d64, U0=np.zeros(n), y0=y0, stall_every=25, return_info=True, **kw)
    cold = oqp.admm(H64, g64, lo, hi, C64, d64, **kw)
    assert ref[7]["restarted"] and ref[6]
    t = prob.torch
    U, _ = prob.qp_solve(Hd, gd, Ctd, dtd, warm_U=t.zeros(n, device="cuda"),
                         warm_y=t.as_tensor(y0, dtype=t.float32, device="cuda"))
    st = prob.read_stats()
    assert st["status"] == lib.GM_STALLED and st["converged"] == 1, st
    # the same stall test drops the warm start; the cold part takes the cold solve's count
    # (FP32 against FP64: within a few iterations)
    assert abs(st["iters"] - ref[3]) <= max(3, 0.05 * ref[3]), (st["iters"], ref[3])
    Ue, _, _ = oqp.solve_exact(H64, g64, lo, hi, C64, d64)
    Ud = U.cpu().numpy()
    assert np.abs(Ud - Ue).max() <= 1e-4 and np.abs(Ud - cold[0]).max() <= 1e-4


def test_nan_warm_start_restarts_cold_and_a_good_one_does_not(lib):
    from test_oracle_qp import stall_qp
    H, g, lo, hi, C, d, kw = stall_qp()
    prob = _stall_problem(lib)
    Hd, gd, Ctd, dtd, (H64, g64, C64, d64) = _dev_qp(prob, H, g, C, d)
    Ue, ye, _ = oqp.solve_exact(H64, g64, lo, hi, C64, d64)
    t = prob.torch
    n = H.shape[0]
    # NaN in U0: the first iterate is NaN, the solve restarts cold at once
    U0 = t.zeros(n, device="cuda")
    U0[3] = float("nan")
    U, _ = prob.qp_solve(Hd, gd, Ctd, dtd, warm_U=U0, warm_y=None)
    st = prob.read_stats()
    assert st["status"] == lib.GM_STALLED and st["converged"] == 1, st
    assert np.abs(U.cpu().numpy() - Ue).max() <= 1e-4
    # the exact optimum as the warm start: no restart, few iterations
    U, _ = prob.qp_solve(Hd, gd, Ctd, dtd, warm_U=t.as_tensor(Ue, dtype=t.float32, device="cuda"),
                         warm_y=t.as_tensor(ye, dtype=t.float32, device="cuda"))
    st2 = prob.read_stats()
    assert st2["status"] == lib.GM_OK and st2["converged"] == 1, st2
    assert st2["iters"] < st["iters"]


def test_redundant_rows_are_skipped_with_zero_multipliers(lib):
    """Rows that no input in the box can violate (the oracle's test, FP64) get multiplier 0
    from the device solve, which agrees with the oracle's ADMM that drops the same rows."""
    from test_oracle_qp import stall_qp
    H, g, lo, hi, C, d, kw = stall_qp(seed=2)
    d = d + np.random.default_rng(3).uniform(0.0, 3.0, d.size)
    prob = _stall_problem(lib)
    Hd, gd, Ctd, dtd, (H64, g64, C64, d64) = _dev_qp(prob, H, g, C, d)
    red = oqp.redundant_rows(C64, d64, lo, hi)
    assert 0 < red.sum() < red.size, red
    U, y = prob.qp_solve(Hd, gd, Ctd, dtd)
    st = prob.read_stats()
    assert st["status"] == lib.GM_OK and st["converged"] == 1, st
    y = y.cpu().numpy()
    n = H.shape[0]
    assert (y[n:][red] == 0).all()
    ref = oqp.admm(H64, g64, lo, hi, C64, d64, **kw)
    assert abs(st["iters"] - ref[3]) <= max(3, 0.05 * ref[3]), (st["iters"], ref[3])
    assert np.abs(U.cpu().numpy() - ref[0]).max() <= 1e-4
