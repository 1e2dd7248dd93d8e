"""Matrix-free condensing in the oracle (no GPU): the forward-mode sensitivities against the
textbook condensing of explicit Jacobians, and the support of each sensitivity column."""
import numpy as np

from oracle import condense as cd
from oracle import gnn as gm
from oracle import matrix_free as mf
from oracle import rti as orti
from synth import random_instance, small_chain


def _case(wl, seed=1):
    gnn, g = orti.model_of(wl)
    U = np.random.default_rng(seed).uniform(-0.3, 0.3, (wl.N, wl.nu))
    return gnn, g, U


def test_matrix_free_equals_condensing_of_explicit_jacobians():
    """H, g, C~, d~, Gamma_u, Gamma_x from forward-mode sensitivities against Eq. condensed_matrices
    written out with the dense A_k, B_k, c_k of every stage (products of transition matrices)."""
    wl = small_chain(n_spheres=2, sphere_clear=0.15)
    gnn, g, U = _case(wl)
    x_hat = gm.rollout(gnn, g, wl.x0, U)
    A, B, c = orti.linearize_dense(gnn, g, x_hat, U)
    Cx, dx = cd.sphere_halfspaces(x_hat, wl.spheres.astype(np.float64))
    x0 = np.asarray(wl.x0, np.float64).reshape(-1)
    Q = wl.Qdiag.reshape(wl.N + 1, -1)
    ref = cd.condense_dense(A, B, c, x0, Q, wl.Rdiag, wl.x_ref, wl.u_ref, Cx, dx)
    got = mf.condense_matrix_free(gnn, g, wl.x0, U, Q, wl.Rdiag, wl.x_ref, wl.u_ref, Cx, dx)
    for a, b, name in zip(got, ref, ("H", "g", "Ct", "dt", "Gu", "Gx")):
        assert a.shape == b.shape, name
        assert np.abs(a - b).max() <= 1e-10 * max(1.0, np.abs(b).max()), (name, np.abs(a - b).max())


def test_matrix_free_on_a_random_graph():
    wl = random_instance(4, M=7, N=4, nu=2, K=2, W=32)
    gnn, g, U = _case(wl, seed=2)
    x_hat = gm.rollout(gnn, g, wl.x0, U)
    A, B, c = orti.linearize_dense(gnn, g, x_hat, U)
    Gu, Gx = cd.gamma_dense(A, B, c, np.asarray(wl.x0, np.float64).reshape(-1))
    x_mf, S = mf.sensitivities(gnn, g, wl.x0, U)
    assert np.array_equal(x_mf, x_hat)
    nx = 6 * wl.M
    assert np.abs(S.reshape((wl.N + 1) * nx, -1) - Gu).max() <= 1e-11 * np.abs(Gu).max()
    # the affine part reproduces the rollout at U_hat
    assert np.abs(Gu @ U.reshape(-1) + Gx - x_hat.reshape(-1)).max() <= 1e-11


def test_sensitivity_columns_vanish_outside_their_reach():
    """Column (i, a) of S_k is zero for k <= i and outside the nodes act_node[a] reaches in
    K (k - i) edges, and non-zero somewhere on the last hop ring (the bound is attained)."""
    wl = small_chain()
    gnn, g, U = _case(wl, seed=3)
    _, S = mf.sensitivities(gnn, g, wl.x0, U)
    K, nu = wl.K, wl.nu
    attained = 0
    for k in range(wl.N + 1):
        for i in range(wl.N):
            for a in range(nu):
                col = S[k][:, :, i * nu + a]
                if k <= i:
                    assert not col.any(), (k, i, a)
                    continue
                inside = set(mf.downstream_ball(g, int(wl.act_node[a]), K * (k - i)))
                outside = [n for n in range(wl.M) if n not in inside]
                assert not col[outside].any(), (k, i, a)
                ring = set(inside) - set(mf.downstream_ball(g, int(wl.act_node[a]), K * (k - i) - 1))
                attained += bool(np.abs(col[sorted(ring)]).max() > 0) if ring else 0
    assert attained > 0


def test_tangent_row_count_of_a_line_graph():
    """Closed form on a directed line 0 -> 1 -> ... -> M-1, one actuator at node 0, K = 1, N = 2:
    stage 0, column (0, 0): layers reach 0 and 1 hops (1 + 2 nodes, 1 + 2 edges with an endpoint
    inside); stage 1: column (0, 0) at 1 and 2 hops (2 + 3 nodes, 2 + 3 edges), column (1, 0)
    at 0 and 1 hops (1 + 2 nodes, 1 + 2 edges)."""
    g = gm.Graph(8, list(range(7)), list(range(1, 8)), 1, [0])
    nr, er = mf.tangent_rows(g, K=1, N=2, nu=1)
    assert (nr, er) == (1 + 2 + 2 + 3 + 1 + 2, 1 + 2 + 2 + 3 + 1 + 2)
