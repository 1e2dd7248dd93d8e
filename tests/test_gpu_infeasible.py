"""Primal-infeasibility detection of the device ADMM against an LP verdict and the oracle.  Needs a GPU.

Every 10th ADMM iteration tests the dual step dy = y - y_prev as a Farkas
certificate (Banjac et al., 2019): when no U meets the constraints, dy
converges to a direction with A~'dy = 0 and negative support over [l, h].
The device solve must then stop with status GM_ERR_INFEASIBLE, on feasible
sets it must not fire.  Which sets are empty is decided by scipy's LP solver
(sets within 0.05 of the boundary are skipped), so the verdict does not rest
on either ADMM.
"""
import numpy as np
import pytest

from gpu_helpers import dense_to_packed_ct, oqp
from synth import small_chain

pytestmark = pytest.mark.gpu

N, NU, MNC = 4, 2, 3


def _lp_margin(lo, hi, C, d):
    from scipy.optimize import linprog
    n, m = lo.size, C.shape[0]
    res = linprog(np.r_[np.zeros(n), 1.0], A_ub=np.hstack([C, -np.ones((m, 1))]), b_ub=d,
                  bounds=[(a, b) for a, b in zip(lo, hi)] + [(None, None)], method="highs")
    assert res.status == 0
    return res.fun


def _staged_qp(seed):
    """Random QP with the condensed structure: stage k's rows act on U_0 .. U_k."""
    rng = np.random.default_rng(seed)
    n, m = N * NU, N * MNC
    L = rng.normal(0, 1, (n, n))
    H = (L @ L.T + 0.1 * np.eye(n)).astype(np.float32)
    g = rng.normal(0, 3.0, n).astype(np.float32)
    C = rng.normal(0, 1, (m, n))
    for k in range(N):
        C[k * MNC:(k + 1) * MNC, (k + 1) * NU:] = 0.0
    C = C.astype(np.float32)
    d = rng.uniform(-1.0, 1.5, m).astype(np.float32)
    return H, g, C, d


@pytest.mark.parametrize("seed", range(12))
def test_noalloc_solve_flags_exactly_the_empty_sets(lib, seed):
    import torch
    H, g, C, d = _staged_qp(300 + seed)
    lo, hi = -np.ones(N * NU, np.float32), np.ones(N * NU, np.float32)
    t = _lp_margin(lo.astype(np.float64), hi.astype(np.float64), C.astype(np.float64), d.astype(np.float64))
    if abs(t) < 0.05:
        pytest.skip(f"margin {t:.3f} too close to the boundary")
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")  # noqa: E731
    s = lib.make_settings(N, 1, rho=0.1, tol=1e-6, max_iter=20000)
    U = torch.zeros(N * NU, device="cuda")
    y = torch.zeros(N * NU + N * MNC, device="cuda")
    stats = torch.zeros(lib.STATS_BYTES, dtype=torch.uint8, device="cuda")
    lib.gm_qp_solve_noalloc(N, NU, MNC, s, dev(H), dev(g), dev(dense_to_packed_ct(C, N, MNC, 1, NU)), dev(d),
                            dev(lo), dev(hi), U, y, stats)
    st = lib.read_stats(stats)
    *_, it_o, _, _, ok_o, info = oqp.admm(H.astype(np.float64), g.astype(np.float64), lo.astype(np.float64),
                                         hi.astype(np.float64), C.astype(np.float64), d.astype(np.float64),
                                         rho=0.1, tol=1e-6, max_iter=20000, scale_rows=True, adapt_every=25,
                                         return_info=True)
    if t > 0:
        assert info["infeasible"]
        assert st["status"] == lib.GM_ERR_INFEASIBLE and st["converged"] == 0, st
        # tested on every 10th iteration only, and within a few tests of the FP64 recurrence
        assert st["iters"] % 10 == 0 and st["iters"] <= 2 * it_o + 100, (st["iters"], it_o)
    else:
        assert ok_o and st["status"] == lib.GM_OK and st["converged"] == 1, st


def test_rti_step_reports_contradicting_half_spaces(lib):
    """A whole RTI step whose position half-spaces contradict at the actuated node in the last
    stage (n'p <= n'p0 - 1 and -n'p <= -n'p0 - 1, so 0 <= -2 for their sum): the step ends with
    GM_ERR_INFEASIBLE, and the next step, with both half-spaces relaxed, converges again."""
    wl = small_chain()
    rng = np.random.default_rng(9)
    nrm = rng.normal(0, 1, (wl.N, wl.M, 2, 3))
    nrm /= np.linalg.norm(nrm, axis=-1, keepdims=True)
    dx = np.full((wl.N, wl.M, 2), 1e3)
    i, k = int(wl.act_node[0]), wl.N - 1
    nrm[k, i, 1] = -nrm[k, i, 0]
    p0 = np.asarray(wl.x0, np.float64).reshape(wl.M, 6)[i, :3]
    dx[k, i, 0] = nrm[k, i, 0] @ p0 - 1.0
    dx[k, i, 1] = -nrm[k, i, 0] @ p0 - 1.0
    prob = lib.RTIProblem(wl.M, wl.src, wl.dst, wl.nu, wl.act_node, wl.K, wl.W, wl.dt, wl.blob, wl.N,
                          wl.Qdiag, wl.Rdiag, wl.x_ref, wl.u_ref, wl.u_lo, wl.u_hi,
                          Cx=nrm.astype(np.float32), dx=dx.astype(np.float32), rho=wl.rho, tol=wl.tol,
                          max_iter=wl.max_iter)
    prob.step(wl.x0)
    st = prob.read_stats()
    assert st["status"] == lib.GM_ERR_INFEASIBLE and st["iters"] < wl.max_iter, st
    dx[k, i, :] = 1e3
    prob.dx.copy_(prob.torch.as_tensor(dx.astype(np.float32)))    # the constraint set points at prob.dx
    prob.step(wl.x0)
    st = prob.read_stats()
    assert st["status"] == lib.GM_OK and st["converged"] == 1, st
