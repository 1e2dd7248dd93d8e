"""Matrix-free condensing on the device (gm_condense_matrix_free; gm_settings.condensing = 1):
the sensitivities pushed through the GNN by forward-mode products on their supports, against the
oracle's forward-mode condensing (itself pinned to the textbook condensing of explicit Jacobians
in test_oracle_matrix_free) and against the device's Jacobian path.  Needs a GPU."""
import numpy as np
import pytest

from gpu_helpers import REL, dense_to_packed_ct, max_rel_err, ocd, orti
from oracle import gnn as ogm
from oracle import matrix_free as omf
from synth import paper_chain, random_instance, small_chain

pytestmark = pytest.mark.gpu

SPHERES = np.array([[0.0, 0.05, -0.3, 0.02], [0.02, -0.04, -0.7, 0.03]], np.float32)


def _u(wl, seed):
    return np.random.default_rng(seed).uniform(-0.3, 0.3, (wl.N, wl.nu)).astype(np.float32)


def _oracle(wl, u):
    gnn, gr = orti.model_of(wl)
    u64 = u.astype(np.float64)
    xo = ogm.rollout(gnn, gr, wl.x0, u64)
    if wl.spheres.shape[0]:
        Cx, dx = ocd.sphere_halfspaces(xo, wl.spheres.astype(np.float64))
    else:
        Cx = dx = None
    out = omf.condense_matrix_free(gnn, gr, wl.x0, u64, wl.Qdiag.reshape(wl.N + 1, -1), wl.Rdiag, wl.x_ref,
                                   wl.u_ref, Cx, dx)
    return xo, out


@pytest.mark.parametrize("case", ["chain10", "random", "random_box"])
def test_matrix_free_parity_with_the_oracle(lib, case):
    """FP32 form: x_hat, H, g, C~, d~ element by element against the FP64 oracle, and against the
    device's Jacobian path on the same context kind (same rollout, same ReLU masks): there the two
    condensing algorithms differ only in FP32 summation order.  H is stored in FP32 with R = 0.01 I
    on its diagonal, so the bound on H adds that storage rounding where the Gram part is far
    below it."""
    if case == "chain10":
        wl = small_chain()
        wl.spheres = SPHERES
    elif case == "random":
        wl = random_instance(11, M=9, N=5, nu=3, K=2, W=32)
        wl.spheres = SPHERES
    else:
        wl = random_instance(12, M=12, N=6, nu=2, K=1, W=32)
    u = _u(wl, 1)
    prob = lib.RTIProblem.from_workload(wl, condensing=1)
    x_hat, H, g, Ct, dt = (t.cpu().numpy().astype(np.float64) for t in prob.condense_matrix_free(wl.x0, u))
    xo, (Ho, go, Cto, dto, _, _) = _oracle(wl, u)
    assert max_rel_err(x_hat, xo) <= 1e-5
    R = np.diag(wl.Rdiag.reshape(-1).astype(np.float64))
    # REL of the Gram part's scale, plus the FP32 rounding of H itself (R on the diagonal)
    assert np.abs(H - Ho).max() <= REL * np.abs(Ho - R).max() + 4 * 2.0 ** -24 * np.abs(Ho).max()
    assert max_rel_err(g, go) <= REL
    jp = lib.RTIProblem.from_workload(wl)
    xj, A, B, c = jp.linearize(wl.x0, u)
    H_j, g_j, Ct_j, dt_j = (t.cpu().numpy().astype(np.float64) for t in jp.condense(xj, A, B, c))
    assert max_rel_err(H - R, H_j - R) <= 1e-5 and max_rel_err(g, g_j) <= 1e-5
    if wl.spheres.shape[0]:
        assert max_rel_err(Ct, Ct_j) <= 1e-5 and max_rel_err(dt, dt_j) <= 1e-5
        n_c = wl.spheres.shape[0]
        assert max_rel_err(Ct, dense_to_packed_ct(Cto, wl.N, wl.M, n_c, wl.nu)) <= REL
        assert max_rel_err(dt, dto) <= REL


def test_matrix_free_rejected_on_a_jacobian_context(lib):
    from paper_2602_17601_b300 import GMError
    wl = small_chain()
    prob = lib.RTIProblem.from_workload(wl)
    with pytest.raises(GMError):
        prob.condense_matrix_free(wl.x0, _u(wl, 2))


def test_matrix_free_step_matches_the_oracle(lib):
    """One RTI step (gm_rti_step) on a matrix-free context against the oracle's step with the
    exact QP optimum, within the solver's tolerance bound."""
    wl = small_chain(tol=1e-7, n_spheres=2, sphere_clear=0.15)
    prob = lib.RTIProblem.from_workload(wl, condensing=1)
    U = prob.step(wl.x0).cpu().numpy().astype(np.float64).reshape(wl.N, wl.nu)
    st = prob.read_stats()
    assert st["converged"] == 1, st
    ref = orti.rti_step(wl, solver="exact")
    assert np.abs(U - ref).max() <= 10 * wl.tol / wl.rho + 1e-4, np.abs(U - ref).max()


def test_matrix_free_against_the_jacobian_path_mixed_form(lib):
    """The chosen (mixed) form on a 300-node chain with the paper's GNN (K = 3, W = 128), N = 10:
    H, g, C~, d~ of the two condensing paths agree within the mixed form's accuracy (each
    differs from FP64 by up to about 1e-3 of its scale near ReLU kinks), and their RTI steps
    (graph replay, warm start, three closed-loop steps) agree within the ADMM bound."""
    from paper_2602_17601_b300 import GM_PREC_MIXED
    wl = paper_chain(seed=6, M=300, N=10, nu=8)
    u = _u(wl, 4)
    mf = lib.RTIProblem.from_workload(wl, precision=GM_PREC_MIXED, condensing=1)
    jp = lib.RTIProblem.from_workload(wl, precision=GM_PREC_MIXED)
    x_m, H_m, g_m, Ct_m, dt_m = (t.cpu().numpy().astype(np.float64) for t in mf.condense_matrix_free(wl.x0, u))
    xj, A, B, c = jp.linearize(wl.x0, u)
    H_j, g_j, Ct_j, dt_j = (t.cpu().numpy().astype(np.float64) for t in jp.condense(xj, A, B, c))
    assert np.array_equal(x_m, xj.cpu().numpy())
    R = np.diag(wl.Rdiag.reshape(-1).astype(np.float64))
    assert max_rel_err(H_m - R, H_j - R) <= 2e-3
    assert max_rel_err(g_m, g_j) <= 2e-3
    assert max_rel_err(Ct_m, Ct_j) <= 2e-3
    assert max_rel_err(dt_m, dt_j, scale=np.abs(x_m).max()) <= 2e-3
    steps = {}
    for name, cond in (("mf", 1), ("jac", 0)):
        p = lib.RTIProblem.from_workload(wl, precision=GM_PREC_MIXED, condensing=cond, graph=True, warm=True)
        x = np.asarray(wl.x0, np.float32).reshape(-1)
        out = []
        for _ in range(3):
            out.append(p.step(x).cpu().numpy().copy())
            assert p.read_stats()["converged"] == 1
        steps[name] = out
    for a, b in zip(steps["mf"], steps["jac"]):
        assert np.abs(a - b).max() <= 2e-2 * max(np.abs(b).max(), 1e-3), np.abs(a - b).max()


def test_matrix_free_barrier_step_matches_the_jacobian_path(lib):
    """The barrier-cost variant (sphere rows folded into H and g, box-only QP) on a matrix-free
    context against the same step on a Jacobian context."""
    wl = small_chain(tol=1e-7, n_spheres=2, sphere_clear=0.15)
    out = {}
    for cond in (0, 1):
        p = lib.RTIProblem.from_workload(wl, condensing=cond, barrier=(1e-3, 5e-3))
        out[cond] = p.step(wl.x0).cpu().numpy().astype(np.float64)
        assert p.read_stats()["converged"] == 1
    assert np.abs(out[1] - out[0]).max() <= 10 * wl.tol / wl.rho + 1e-5, np.abs(out[1] - out[0]).max()


def test_matrix_free_contexts_in_a_batch(lib):
    """Matrix-free contexts stepped as one batch (gm_batch_*: plain launches, then the captured
    graph) give each instance the U of its own single-instance steps."""
    from paper_2602_17601_b300.batch import Batch
    wls = [small_chain(), random_instance(7, M=8, N=6, nu=3, K=2, W=32),
           paper_chain(seed=3, M=40, N=5, nu=2, K=2, W=32, w_seed=0, n_spheres=2)]
    alone = []
    for wl in wls:
        p = lib.RTIProblem.from_workload(wl, condensing=1, admm_grid=8, factor_grid=16)
        alone.append([p.step(wl.x0).cpu().numpy().copy() for _ in range(3)])
    probs = [lib.RTIProblem.from_workload(wl, condensing=1, admm_grid=8, factor_grid=16) for wl in wls]
    b = Batch(probs)
    b.set_states([wl.x0 for wl in wls])
    for k in range(3):
        b.step()
        for i, (wl, p) in enumerate(zip(wls, probs)):
            assert p.read_stats()["converged"] == 1, (k, i)
            U = p._U.cpu().numpy()
            assert np.abs(U - alone[i][k]).max() <= 10 * wl.tol / wl.rho, (k, i, np.abs(U - alone[i][k]).max())


def test_stage_timeline(lib):
    """gm_ctx_stage_times on a graph-replayed matrix-free step: every tangent stage ends after
    the rollout stage it reads and after the tangent stage before it; rejected while off and on a
    Jacobian context."""
    from paper_2602_17601_b300 import GMError
    import paper_2602_17601_b300 as gm
    wl = small_chain()
    p = lib.RTIProblem.from_workload(wl, condensing=1, graph=True)
    with pytest.raises(GMError):
        gm.gm_ctx_stage_times(p.ctx, wl.N)
    gm.gm_ctx_set_stage_timing(p.ctx, True)
    for _ in range(2):
        p.step(wl.x0)
    roll, tan = gm.gm_ctx_stage_times(p.ctx, wl.N)
    assert all(t >= r for r, t in zip(roll, tan))
    assert all(b >= a for a, b in zip(tan, tan[1:])) and all(b >= a for a, b in zip(roll, roll[1:]))
    assert roll[0] > 0
    jp = lib.RTIProblem.from_workload(wl)
    with pytest.raises(GMError):
        gm.gm_ctx_set_stage_timing(jp.ctx, True)
