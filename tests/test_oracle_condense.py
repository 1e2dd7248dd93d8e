"""Pins of the oracle's condensing (Sec. III-B and the Thm. 1 proof).  No GPU."""
import numpy as np
import pytest

from oracle import condense as cd
from oracle import gnn as gm
from oracle import rti
from synth import small_chain, chain_edges


def random_ltv(M, N, nu, reach, seed, n_c=2, scale=0.3):
    """Random LTV system whose A^{ij} vanish beyond `reach` chain positions."""
    rng = np.random.default_rng(seed)
    nx = 6 * M
    A = np.zeros((N, nx, nx))
    for k in range(N):
        for i in range(M):
            for j in range(max(0, i - reach), min(M, i + reach + 1)):
                A[k, 6 * i:6 * i + 6, 6 * j:6 * j + 6] = rng.normal(0, scale, (6, 6))
    B = rng.normal(0, 1.0, (N, nx, nu))
    c = rng.normal(0, 0.1, (N, nx))
    x0 = rng.normal(0, 1, nx)
    Qd = rng.uniform(0.5, 2.0, (N + 1, nx))
    Rd = rng.uniform(0.01, 0.1, (N, nu))
    xr = rng.normal(0, 1, (N + 1, nx))
    ur = rng.normal(0, 0.1, (N, nu))
    Cx = rng.normal(0, 1, (N, M, n_c, 3))
    dx = rng.normal(0, 1, (N, M, n_c))
    nbh = [list(range(max(0, i - reach), min(M, i + reach + 1))) for i in range(M)]
    return A, B, c, x0, Qd, Rd, xr, ur, Cx, dx, nbh


def simulate(A, B, c, x0, U):
    """Eq. ocp_dynamics: x_{k+1} = A_k x_k + B_k u_k + c_k, x_0 given."""
    xs = [x0]
    for k in range(B.shape[0]):
        xs.append(A[k] @ xs[-1] + B[k] @ U[k] + c[k])
    return np.stack(xs)


def paper_cost(xs, U, Qd, Rd, xr, ur):
    """Eq. linear_gnn_mpc_ocp_explicit's objective, evaluated on a trajectory."""
    return float(np.sum(Qd * (xs - xr) ** 2) + np.sum(Rd * (U - ur) ** 2))


@pytest.mark.parametrize("seed", [0, 1])
def test_recursion_equals_textbook_condensing(seed):
    M, N, nu = 5, 4, 2
    A, B, c, x0, Qd, Rd, xr, ur, Cx, dx, nbh = random_ltv(M, N, nu, 1, seed)
    H1, g1, C1, d1, Gu1, Gx1 = cd.condense_dense(A, B, c, x0, Qd, Rd, xr, ur, Cx, dx)
    blocks = cd.blocks_from_dense(A, B, c, nbh)
    H2, g2, C2, d2, Gu2, Gx2 = cd.condense_recursive(blocks, x0, Qd, Rd, xr, ur, Cx, dx)
    for a, b in ((H1, H2), (g1, g2), (C1, C2), (d1, d2)):
        assert np.allclose(a, b, rtol=1e-12, atol=1e-10 * max(1.0, np.abs(a).max()))
    # Gamma per node (paper layout) against the dense Gamma rows of that node
    for i in range(M):
        for k in range(N + 1):
            assert np.allclose(Gu2[i, 6 * k:6 * k + 6], Gu1[k * 6 * M + 6 * i:k * 6 * M + 6 * i + 6],
                               atol=1e-10 * max(1.0, np.abs(Gu1).max()))
            assert np.allclose(Gx2[i, k], Gx1[k * 6 * M + 6 * i:k * 6 * M + 6 * i + 6],
                               atol=1e-10 * max(1.0, np.abs(Gx1).max()))


def test_single_stage_worked_case():
    """N = 1: Gamma_u^i = [0; B^i_0], Gamma_x^i = [x^i_0; sum_j A^{ij}_0 x^j_0 + c^i_0] (Thm. 1 proof)."""
    M, N, nu = 4, 1, 3
    A, B, c, x0, Qd, Rd, xr, ur, Cx, dx, nbh = random_ltv(M, N, nu, 1, 5)
    blocks = cd.blocks_from_dense(A, B, c, nbh)
    _, _, _, _, Gu, Gx = cd.condense_recursive(blocks, x0, Qd, Rd, xr, ur, Cx, dx)
    for i in range(M):
        assert np.all(Gu[i, :6] == 0.0)
        assert np.array_equal(Gu[i, 6:12], B[0, 6 * i:6 * i + 6])
        assert np.array_equal(Gx[i, 0], x0[6 * i:6 * i + 6])
        expect = c[0, 6 * i:6 * i + 6].copy()
        for j in nbh[i]:
            expect += A[0, 6 * i:6 * i + 6, 6 * j:6 * j + 6] @ x0[6 * j:6 * j + 6]
        assert np.allclose(Gx[i, 1], expect, atol=1e-14)


def test_gamma_reproduces_simulation_cost_and_constraints():
    """x = Gu U + Gx, the QP objective and C~ U - d~ all match a direct simulation.

    For random input sequences U: the trajectory of Eq. ocp_dynamics equals
    Gu U + Gx; (1/2) * (paper cost) - (1/2 U'HU + g'U) is the same constant for
    every U (catches a factor 2, a sign or a dropped term in H or g); and
    C~ U - d~ equals C_x x(U) - d_x row by row.
    """
    M, N, nu = 4, 5, 2
    A, B, c, x0, Qd, Rd, xr, ur, Cx, dx, nbh = random_ltv(M, N, nu, 1, 7)
    blocks = cd.blocks_from_dense(A, B, c, nbh)
    H, g, Ct, dt, _, _ = cd.condense_recursive(blocks, x0, Qd, Rd, xr, ur, Cx, dx)
    _, _, _, _, Gu, Gx = cd.condense_dense(A, B, c, x0, Qd, Rd, xr, ur, Cx, dx)
    rng = np.random.default_rng(3)
    consts = []
    for _ in range(4):
        U = rng.normal(0, 1, (N, nu))
        xs = simulate(A, B, c, x0, U)
        assert np.allclose(xs.reshape(-1), Gu @ U.reshape(-1) + Gx, atol=1e-9)
        u = U.reshape(-1)
        consts.append(0.5 * paper_cost(xs, U, Qd, Rd, xr, ur) - (0.5 * u @ H @ u + g @ u))
        lhs = Ct @ u - dt
        rhs = []
        for k in range(1, N + 1):
            for i in range(M):
                for s in range(Cx.shape[2]):
                    rhs.append(Cx[k - 1, i, s] @ xs[k, 6 * i:6 * i + 3] - dx[k - 1, i, s])
        assert np.allclose(lhs, rhs, atol=1e-9)
    assert np.ptp(consts) <= 1e-9 * max(1.0, abs(consts[0]))


def test_disconnected_graph_hessian_is_sum_of_single_node_problems():
    """E = 0: H - Rbar and g - rbar are sums of independent single-node contributions (Eq. H, Eq. g)."""
    M, N, nu = 3, 3, 2
    A, B, c, x0, Qd, Rd, xr, ur, Cx, dx, _ = random_ltv(M, N, nu, 0, 11)
    nbh = [[i] for i in range(M)]
    H, g, _, _, _, _ = cd.condense_recursive(cd.blocks_from_dense(A, B, c, nbh), x0, Qd, Rd,
                                             xr, ur, Cx, dx)
    Hsum = np.diag(Rd.reshape(-1)).copy()
    gsum = -(Rd * ur).reshape(-1)
    for i in range(M):
        s = slice(6 * i, 6 * i + 6)
        Ai, Bi, ci = A[:, s, s], B[:, s], c[:, s]
        Hi, gi, _, _, _, _ = cd.condense_dense(Ai, Bi, ci, x0[s], Qd[:, s], np.zeros_like(Rd),
                                              xr[:, s], ur, None, None)
        Hsum += Hi
        gsum += gi
    assert np.allclose(H, Hsum, atol=1e-10) and np.allclose(g, gsum, atol=1e-10)


def test_condensing_flops_linear_in_nodes():
    """Thm. 1: for fixed n_x-bar, n_u, N and neighbourhood size the work is O(M).

    The recursion counts its multiply-adds; the log-log slope over M must be 1.
    """
    N, nu, reach = 4, 2, 2
    Ms = [20, 40, 80, 160]
    macs = []
    rng = np.random.default_rng(0)
    for M in Ms:
        nbh = [list(range(max(0, i - reach), min(M, i + reach + 1))) for i in range(M)]
        blocks = []
        for k in range(N):
            blocks.append([(nb, rng.normal(0, 0.1, (len(nb), 6, 6)), rng.normal(0, 1, (6, nu)),
                            rng.normal(0, 1, 6)) for nb in nbh])
        cnt = cd.MacCounter()
        cd.condense_recursive(blocks, np.zeros(6 * M), np.ones((N + 1, 6 * M)),
                              np.ones((N, nu)), np.zeros((N + 1, 6 * M)), np.zeros((N, nu)),
                              np.zeros((N, M, 1, 3)), np.zeros((N, M, 1)), counter=cnt)
        macs.append(cnt.macs)
    slope = np.polyfit(np.log(Ms), np.log(macs), 1)[0]
    assert abs(slope - 1.0) <= 0.1, (slope, macs)


def test_sphere_halfspace_slack_is_distance_minus_radius():
    """At the linearisation point the half-space slack equals |p^ - o| - r (outside => >= 0)."""
    rng = np.random.default_rng(4)
    x_hat = rng.normal(0, 1, (4, 5, 6))
    spheres = np.array([[0.1, 0.2, -0.3, 0.5], [1.0, -1.0, 0.0, 0.2]])
    Cx, dx = cd.sphere_halfspaces(x_hat, spheres)
    for k in range(1, 4):
        for i in range(5):
            for s in range(2):
                p = x_hat[k, i, :3]
                slack = dx[k - 1, i, s] - Cx[k - 1, i, s] @ p
                dist = np.linalg.norm(p - spheres[s, :3]) - spheres[s, 3]
                assert abs(slack - dist) <= 1e-12
                # and every point of the sphere satisfies the constraint with equality at most
                n = -Cx[k - 1, i, s]
                closest = spheres[s, :3] + spheres[s, 3] * n
                assert Cx[k - 1, i, s] @ closest <= dx[k - 1, i, s] + 1e-12


def test_gnn_condensing_recursion_equals_textbook():
    """The same equality on the GNN's own Jacobians along its rollout (chain of 10)."""
    wl = small_chain()
    r1 = rti.rti_step(wl, return_all=True, condensing="recursive")
    r2 = rti.rti_step(wl, return_all=True, condensing="dense")
    assert np.allclose(r1["H"], r2["H"], atol=1e-14)
    assert np.allclose(r1["g"], r2["g"], atol=1e-14)
    assert np.allclose(r1["U"], r2["U"], atol=1e-10)
