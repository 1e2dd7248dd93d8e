"""Pins of the oracle's GNN dynamics and Jacobians against what the paper and mathematics fix.

No GPU.  Each test checks the FP64 oracle against something other than itself:
finite differences, a closed form, an invariance, or a hand-worked example.
"""
import numpy as np
import pytest

from oracle import gnn as gm
from synth import small_chain, random_instance, make_workload


def _model(wl, activation="relu"):
    return (gm.GNN(wl.blob, wl.K, wl.W, wl.nu, wl.dt, activation=activation),
            gm.Graph(wl.M, wl.src, wl.dst, wl.nu, wl.act_node))


def _fd_jacobian(gnn, g, x, u, h=1e-6):
    """Central differences of F over every state and input coordinate."""
    x = np.asarray(x, np.float64)
    u = np.asarray(u, np.float64)
    nx = x.size
    cols = []
    for t in range(nx + u.size):
        xp, xm, up, um = x.copy(), x.copy(), u.copy(), u.copy()
        if t < nx:
            xp.reshape(-1)[t] += h
            xm.reshape(-1)[t] -= h
        else:
            up[t - nx] += h
            um[t - nx] -= h
        cols.append((gm.step(gnn, g, xp, up) - gm.step(gnn, g, xm, um)).reshape(-1) / (2 * h))
    J = np.stack(cols, 1)
    return J[:, :nx], J[:, nx:]


@pytest.mark.parametrize("case", ["chain10", "rand_directed"])
def test_jacobian_matches_central_differences(case):
    """A = dF/dx, B = dF/du (Eq. linearized_dynamics) against FP64 central differences."""
    if case == "chain10":
        wl = small_chain()
    else:
        wl = random_instance(3, M=7, N=3, nu=3, K=2, W=16, reach=2, directed=True)
    gnn, g = _model(wl)
    rng = np.random.default_rng(1)
    x = wl.x0.astype(np.float64)
    # sample points away from ReLU kinks so that F is smooth within the FD stencil
    x0 = x
    for _ in range(200):
        u = rng.uniform(-1, 1, wl.nu)
        x = x0 + rng.normal(0.0, 1e-2, x0.shape)
        if gm.preactivations_min_abs(gnn, g, x, u) > 1e-4:
            break
    assert gm.preactivations_min_abs(gnn, g, x, u) > 1e-4
    A, B, c, x1 = gm.jacobian_dense(gnn, g, x, u)
    Afd, Bfd = _fd_jacobian(gnn, g, x, u)
    scale = max(np.abs(A).max(), 1.0)
    assert np.abs(A - Afd).max() <= 1e-7 * scale
    assert np.abs(B - Bfd).max() <= 1e-7 * max(np.abs(B).max(), 1e-3)
    # c is the linearisation offset: F(x,u) = A x + B u + c at the point itself
    assert np.allclose(A @ x.reshape(-1) + B @ u + c, x1.reshape(-1), rtol=0, atol=1e-13)


def test_jacobian_block_sparsity_is_k_hop():
    """A^{ij} is exactly zero unless j reaches i in at most K edges (Assumption 1, K-step GNN)."""
    wl = random_instance(5, M=12, N=2, nu=2, K=2, W=8, reach=2, p=0.5, directed=True)
    gnn, g = _model(wl)
    A, _, _, _ = gm.jacobian_dense(gnn, g, wl.x0, np.array([0.3, -0.2]))
    nonzero_somewhere = 0
    for i in range(wl.M):
        ball = set(g.in_ball(i, wl.K))
        for j in range(wl.M):
            blk = A[6 * i:6 * i + 6, 6 * j:6 * j + 6]
            if j not in ball:
                assert np.all(blk == 0.0), (i, j)
            elif j != i:
                nonzero_somewhere += int(np.any(blk != 0.0))
    assert nonzero_somewhere > 0


def test_edge_direction():
    """Edge j -> i carries information from j to i only (Sec. III-A neighbourhood N_i)."""
    src, dst = np.array([0], np.int32), np.array([1], np.int32)
    wl = make_workload("pair", 2, src, dst, 1, [0], 1, 8, 2, 4)
    gnn, g = _model(wl)
    A, B, _, _ = gm.jacobian_dense(gnn, g, wl.x0, np.array([0.5]))
    assert np.all(A[0:6, 6:12] == 0.0)           # node 0 does not see node 1
    assert np.abs(A[9:12, 0:6]).max() > 0.0      # node 1's velocity sees node 0
    assert np.abs(B[6:12]).max() > 0.0           # actuator at node 0 reaches node 1


def test_local_subgraph_rows_equal_full_graph_rows():
    """Differentiating one subsystem on its K-hop subgraph gives the same rows (Sec. V-A)."""
    wl = random_instance(7, M=9, N=2, nu=2, K=2, W=8, reach=2, p=0.6)
    gnn, g = _model(wl)
    u = np.array([0.2, -0.7])
    A, B, c, x1 = gm.jacobian_dense(gnn, g, wl.x0, u)
    for i in (0, 4, 8):
        ball, Ablk, Bi, fi = gm.local_jacobian_rows(gnn, g, wl.x0, u, i)
        for b, j in enumerate(ball):
            assert np.allclose(Ablk[b], A[6 * i:6 * i + 6, 6 * j:6 * j + 6], atol=1e-14)
        assert np.allclose(Bi, B[6 * i:6 * i + 6], atol=1e-14)
        assert np.allclose(fi, x1[i], atol=1e-14)


def test_semi_implicit_euler_structure():
    """p+ = p + dt v+ and the position rows of A are [I, dt I] + dt * velocity rows (Eq. forward_dynamics)."""
    wl = small_chain()
    gnn, g = _model(wl)
    x = wl.x0.astype(np.float64)
    u = np.array([0.1, 0.2, -0.3, 0.4])
    x1 = gm.step(gnn, g, x, u)
    assert np.array_equal(x1[:, :3], x[:, :3] + wl.dt * x1[:, 3:])
    A, B, _, _ = gm.jacobian_dense(gnn, g, x, u)
    M = wl.M
    for i in range(M):
        vel = A[6 * i + 3:6 * i + 6]
        pos = A[6 * i:6 * i + 3]
        expect = wl.dt * vel.copy()
        expect[:, 6 * i:6 * i + 3] += np.eye(3)
        assert np.allclose(pos, expect, atol=1e-15)
    # zero decoder: the model is a pure double integrator with dv = decoder bias only
    gnn.dec = (gnn.dec[0], gnn.dec[1], np.zeros_like(gnn.dec[2]), np.zeros(3))
    x1 = gm.step(gnn, g, x, u)
    assert np.array_equal(x1[:, 3:], x[:, 3:])
    assert np.allclose(x1[:, :3], x[:, :3] + wl.dt * x[:, 3:], atol=0)


def test_sum_aggregation():
    """Duplicating every edge doubles the aggregated message (sum, not mean, Sec. V-A).

    So the doubled graph with the aggregate's input weights halved is the
    original model, while the doubled graph with unchanged weights is not.
    """
    wl = small_chain()
    gnn, g = _model(wl)
    x = wl.x0.astype(np.float64)
    u = np.array([0.3, -0.1, 0.2, 0.5])
    g2 = gm.Graph(wl.M, np.concatenate([wl.src, wl.src]), np.concatenate([wl.dst, wl.dst]),
                  wl.nu, wl.act_node)
    half = gm.GNN(wl.blob, wl.K, wl.W, wl.nu, wl.dt)
    for l in range(wl.K):
        W1, b1, W2, b2 = half.node_mp[l]
        W1 = W1.copy()
        W1[wl.W:] *= 0.5                        # rows fed by sum_j e_ij
        half.node_mp[l] = (W1, b1, W2, b2)
    assert np.allclose(gm.step(half, g2, x, u), gm.step(gnn, g, x, u), atol=1e-13)
    assert not np.allclose(gm.step(gnn, g2, x, u), gm.step(gnn, g, x, u), atol=1e-6)


def test_relative_edge_feature_translation():
    """e^{ij} = x^i - x^j: a rigid shift of all positions only shifts the positions out.

    With the node encoder blind to positions, the model depends on positions only
    through the relative edge features, so F(x + t) = F(x) + (t, 0).
    """
    wl = small_chain()
    gnn, g = _model(wl)
    W1, b1, W2, b2 = gnn.node_enc
    W1 = W1.copy()
    W1[:3] = 0.0
    gnn.node_enc = (W1, b1, W2, b2)
    x = wl.x0.astype(np.float64)
    u = np.array([0.1, -0.4, 0.3, 0.2])
    t = np.array([0.7, -0.3, 1.1])
    xs = x.copy()
    xs[:, :3] += t
    d = gm.step(gnn, g, xs, u) - gm.step(gnn, g, x, u)
    assert np.allclose(d[:, :3], t[None], atol=1e-13)
    assert np.allclose(d[:, 3:], 0.0, atol=1e-13)


def test_permutation_equivariance():
    """Relabelling the nodes permutes the outputs (message passing, Sec. III-A)."""
    wl = random_instance(11, M=8, N=2, nu=2, K=2, W=8)
    gnn, g = _model(wl)
    perm = np.random.default_rng(0).permutation(wl.M)
    inv = np.argsort(perm)                       # new label of old node n is inv[n]
    gp = gm.Graph(wl.M, inv[wl.src], inv[wl.dst], wl.nu, inv[wl.act_node])
    x = wl.x0.astype(np.float64)
    u = np.array([0.5, -0.5])
    y = gm.step(gnn, g, x, u)
    yp = gm.step(gnn, gp, x[perm], u)
    assert np.allclose(yp, y[perm], atol=1e-14)


def test_identity_activation_is_affine_with_closed_form():
    """Identity activations make F affine; its Jacobians are products of weight matrices.

    For a graph without edges the velocity rows of A and B are, per node,
        [W1 W2]_ne  *  prod_l (I + [W1 W2]_nl restricted to the h input)  *  [W1 W2]_d
    (row-vector convention), the same for every node and every state.
    """
    src = np.zeros(0, np.int32)
    wl = make_workload("iso", 3, src, src, 2, [0, 2], 2, 6, 2, 9)
    gnn, g = _model(wl, activation="identity")
    Lne = gnn.node_enc[0] @ gnn.node_enc[2]                 # (6+nu) x W
    chain = np.eye(wl.W)
    for l in range(wl.K):
        Ln = gnn.node_mp[l][0] @ gnn.node_mp[l][2]          # 2W x W
        chain = chain @ (np.eye(wl.W) + Ln[:wl.W])
    Ld = gnn.dec[0] @ gnn.dec[2]                            # W x 3
    T = Lne @ chain @ Ld                                    # (6+nu) x 3
    for xs in (wl.x0, wl.x0 * 3.0 + 0.5):
        A, B, _, _ = gm.jacobian_dense(gnn, g, xs, np.array([0.2, 0.9]))
        for i in range(3):
            assert np.allclose(A[6 * i + 3:6 * i + 6, 6 * i:6 * i + 6], np.eye(6)[3:] + T[:6].T,
                               atol=1e-12)
        assert np.allclose(B[3:6, 0], T[6], atol=1e-12)     # actuator 0 at node 0
        assert np.allclose(B[15:18, 1], T[7], atol=1e-12)   # actuator 1 at node 2
        assert np.all(B[9:12] == 0.0)


def test_identity_activation_affine_on_graph():
    """With identity activations F(x,u) = A x + B u + c exactly, A and B state-independent."""
    wl = small_chain()
    gnn, g = _model(wl, activation="identity")
    rng = np.random.default_rng(2)
    x1, u1 = rng.normal(size=(wl.M, 6)), rng.normal(size=wl.nu)
    x2, u2 = rng.normal(size=(wl.M, 6)), rng.normal(size=wl.nu)
    A1, B1, c1, _ = gm.jacobian_dense(gnn, g, x1, u1)
    A2, B2, c2, _ = gm.jacobian_dense(gnn, g, x2, u2)
    assert np.allclose(A1, A2, atol=1e-12) and np.allclose(B1, B2, atol=1e-12)
    assert np.allclose(c1, c2, atol=1e-11)
    # F evaluated directly at a third point agrees with the affine model
    x3, u3 = rng.normal(size=(wl.M, 6)), rng.normal(size=wl.nu)
    assert np.allclose(gm.step(gnn, g, x3, u3).reshape(-1), A1 @ x3.reshape(-1) + B1 @ u3 + c1,
                       atol=1e-11)


def test_hand_worked_two_node_example():
    """W = 1, K = 1, one edge 0 -> 1, one actuator at node 1: every number by hand.

    Node input [x (6), m*u (1)]; all MLPs Linear(.,1)-ReLU-Linear(1,.).
    """
    K, W, nu = 1, 1, 1
    # weights chosen by hand (blob order: node enc, edge enc, edge mp, node mp, decoder)
    ne = dict(W1=[0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 1.0], b1=[0.05], W2=[2.0], b2=[-0.1])
    ee = dict(W1=[1.0, -1.0, 0.5, 0.0, 0.0, 2.0], b1=[0.1], W2=[0.5], b2=[0.2])
    em = dict(W1=[1.0, -2.0, 3.0], b1=[0.3], W2=[-1.0], b2=[0.4])
    nm = dict(W1=[0.5, 1.5], b1=[-0.2], W2=[0.7], b2=[0.1])
    de = dict(W1=[2.0], b1=[0.5], W2=[0.1, -0.2, 0.3], b2=[0.01, 0.02, 0.03])
    blob = []
    for p in (ne, ee, em, nm, de):
        for key in ("W1", "b1", "W2", "b2"):
            blob += p[key]
    blob = np.array(blob)
    gnn = gm.GNN(blob, K, W, nu, 0.1)
    g = gm.Graph(2, [0], [1], nu, [1])
    x = np.array([[0.0, 0.0, 0.0, 0.0, 0.0, 0.0],
                  [0.1, -0.2, 0.3, 0.5, 0.0, -0.5]])
    u = np.array([0.8])
    relu = lambda v: max(v, 0.0)  # noqa: E731
    # node encoder
    z0 = 0.05                                     # node 0: all zero inputs, no actuator
    h0 = 2.0 * relu(z0) - 0.1                     # 0.0
    z1 = 0.1 * 0.1 + 0.2 * -0.2 + 0.3 * 0.3 + 0.4 * 0.5 + 0.6 * -0.5 + 1.0 * 0.8 + 0.05
    h1 = 2.0 * relu(z1) - 0.1
    # edge 0 -> 1: e = x1 - x0
    d = x[1] - x[0]
    ze = 1.0 * d[0] - 1.0 * d[1] + 0.5 * d[2] + 2.0 * d[5] + 0.1
    e = 0.5 * relu(ze) + 0.2
    # message passing: e' = e + MLP([h_dst, h_src, e]) with dst = 1, src = 0
    zm = 1.0 * h1 - 2.0 * h0 + 3.0 * e + 0.3
    e = e + (-1.0 * relu(zm) + 0.4)
    # node update: node 1 aggregates e, node 0 aggregates nothing
    zn1 = 0.5 * h1 + 1.5 * e - 0.2
    h1 = h1 + 0.7 * relu(zn1) + 0.1
    zn0 = 0.5 * h0 + 0.0 - 0.2
    h0 = h0 + 0.7 * relu(zn0) + 0.1
    # decoder
    dv1 = np.array([0.1, -0.2, 0.3]) * relu(2.0 * h1 + 0.5) + np.array([0.01, 0.02, 0.03])
    dv0 = np.array([0.1, -0.2, 0.3]) * relu(2.0 * h0 + 0.5) + np.array([0.01, 0.02, 0.03])
    v1 = x[1, 3:] + dv1
    v0 = x[0, 3:] + dv0
    expect = np.array([np.concatenate([x[0, :3] + 0.1 * v0, v0]),
                       np.concatenate([x[1, :3] + 0.1 * v1, v1])])
    assert np.allclose(gm.step(gnn, g, x, u), expect, atol=1e-15)
