"""GNN dynamics model and its exact Jacobians, FP64 (oracle; test infrastructure only).

Model (Sec. V-A "Model", Eq. forward_dynamics, generalised to an
encode-process-decode interaction network):

    node input   [x^i, m^i * u]           (m^i: one-hot actuator mask of node i)
    h^0_i      = MLP_ne([x^i, m^i * u])
    e^0_ij     = MLP_ee(x^i - x^j)        (edge j -> i, relative state, Sec. V-A)
    for l = 1..K:
        e^l_ij = e^{l-1}_ij + MLP_el([h^{l-1}_i, h^{l-1}_j, e^{l-1}_ij])
        h^l_i  = h^{l-1}_i + MLP_nl([h^{l-1}_i, sum_{j -> i} e^l_ij])   (sum aggregation)
    dv^i       = MLP_d(h^K_i)                                            (velocity increment)
    v^i_{k+1}  = v^i_k + dv^i ;  p^i_{k+1} = p^i_k + dt * v^i_{k+1}     (Eq. forward_dynamics)

Every MLP is Linear -> ReLU -> Linear.  The ReLU derivative at 0 is taken as 0
(footnote to Sec. V-A "Linearization").

Jacobians (Eq. linearized_dynamics): A^{ij}_k = d f^i / d x^j, B^i_k = d f^i / d u,
c^i_k = f^i - sum_j A^{ij} x^j - B^i u, computed by propagating tangent
vectors through every layer (forward-mode chain rule), one tangent per input
coordinate.  ``local_jacobian_rows`` differentiates one subsystem's dynamics on
its own K-hop subgraph, as the paper describes ("each subsystem's local
dynamics independently").
"""
from __future__ import annotations

from collections import deque

import numpy as np


def _mlp_shapes(K, W, nu):
    shapes = [(6 + nu, W, W), (6, W, W)]
    for _ in range(K):
        shapes += [(3 * W, W, W), (2 * W, W, W)]
    shapes.append((W, W, 3))
    return shapes


def parse_blob(blob, K, W, nu):
    """Split the flat weight blob into (W1, b1, W2, b2) float64 tuples, blob order."""
    blob = np.asarray(blob, dtype=np.float64)
    out, off = [], 0
    for (i, h, o) in _mlp_shapes(K, W, nu):
        W1 = blob[off:off + i * h].reshape(i, h); off += i * h
        b1 = blob[off:off + h]; off += h
        W2 = blob[off:off + h * o].reshape(h, o); off += h * o
        b2 = blob[off:off + o]; off += o
        out.append((W1, b1, W2, b2))
    assert off == blob.size, "blob size does not match (K, W, nu)"
    return out


class GNN:
    """Weights plus hyper-parameters of the encode-process-decode model."""

    def __init__(self, blob, K, W, nu, dt, activation="relu"):
        self.K, self.W, self.nu, self.dt = K, W, nu, float(dt)
        self.activation = activation
        mlps = parse_blob(blob, K, W, nu)
        self.node_enc = mlps[0]
        self.edge_enc = mlps[1]
        self.edge_mp = [mlps[2 + 2 * l] for l in range(K)]
        self.node_mp = [mlps[3 + 2 * l] for l in range(K)]
        self.dec = mlps[2 + 2 * K]

    def mask(self, a):
        if self.activation == "identity":
            return np.ones_like(a, dtype=bool)
        return a > 0.0


class Graph:
    """Directed edges j -> i stored as (src=j, dst=i); nu actuators at act_node."""

    def __init__(self, M, src, dst, nu, act_node):
        self.M = int(M)
        self.src = np.asarray(src, dtype=np.int64)
        self.dst = np.asarray(dst, dtype=np.int64)
        self.nu = int(nu)
        # act_node[a] = -1 marks an actuator outside this (sub)graph
        self.act_node = np.asarray(act_node, dtype=np.int64)

    @property
    def E(self):
        return self.src.size

    def actuator_mask(self):
        """m [M, nu]: m[i, a] = 1 if actuator a is attached at node i."""
        m = np.zeros((self.M, self.nu))
        for a, n in enumerate(self.act_node):
            if n >= 0:
                m[n, a] = 1.0
        return m

    def in_ball(self, i, R):
        """Nodes with a directed path of at most R edges into node i (incl. i)."""
        preds = [[] for _ in range(self.M)]
        for j, t in zip(self.src, self.dst):
            preds[t].append(j)
        dist = {int(i): 0}
        q = deque([int(i)])
        while q:
            n = q.popleft()
            if dist[n] == R:
                continue
            for j in preds[n]:
                j = int(j)
                if j not in dist:
                    dist[j] = dist[n] + 1
                    q.append(j)
        return sorted(dist)


def _mlp(gnn, p, z):
    """Linear -> ReLU -> Linear on the rows of z; also returns the ReLU mask."""
    W1, b1, W2, b2 = p
    a = z @ W1 + b1
    m = gnn.mask(a)
    return np.where(m, a, 0.0) @ W2 + b2, m


def _mlp_tangent(p, m, tz):
    """Tangent of the MLP output for tangent tz [T, rows, in] at the point with mask m."""
    W1, _, W2, _ = p
    return (np.where(m[None], tz @ W1, 0.0)) @ W2


def step(gnn, g, x, u):
    """One application of the GNN dynamics: x_{k+1} = F(x_k, u_k), x [M, 6], u [nu]."""
    return step_jvp(gnn, g, x, u, None, None)[0]


def step_jvp(gnn, g, x, u, tx, tu):
    """F(x, u) and its directional derivatives along T tangents (tx [T,M,6], tu [T,nu])."""
    x = np.asarray(x, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    has_t = tx is not None
    m_act = g.actuator_mask()
    src, dst = g.src, g.dst

    z = np.concatenate([x, m_act * u[None, :]], axis=1)
    h, mk = _mlp(gnn, gnn.node_enc, z)
    if has_t:
        tz = np.concatenate([tx, m_act[None] * tu[:, None, :]], axis=2)
        th = _mlp_tangent(gnn.node_enc, mk, tz)

    d = x[dst] - x[src]
    e, mk = _mlp(gnn, gnn.edge_enc, d)
    if has_t:
        te = _mlp_tangent(gnn.edge_enc, mk, tx[:, dst] - tx[:, src])

    for l in range(gnn.K):
        ze = np.concatenate([h[dst], h[src], e], axis=1)
        de, mk = _mlp(gnn, gnn.edge_mp[l], ze)
        if has_t:
            tze = np.concatenate([th[:, dst], th[:, src], te], axis=2)
            te = te + _mlp_tangent(gnn.edge_mp[l], mk, tze)
        e = e + de
        agg = np.zeros_like(h)
        np.add.at(agg, dst, e)
        if has_t:
            tagg = np.zeros_like(th)
            np.add.at(tagg, (slice(None), dst), te)
        zn = np.concatenate([h, agg], axis=1)
        dh, mk = _mlp(gnn, gnn.node_mp[l], zn)
        if has_t:
            th = th + _mlp_tangent(gnn.node_mp[l], mk, np.concatenate([th, tagg], axis=2))
        h = h + dh

    dv, mk = _mlp(gnn, gnn.dec, h)
    v1 = x[:, 3:] + dv
    p1 = x[:, :3] + gnn.dt * v1
    x1 = np.concatenate([p1, v1], axis=1)
    if not has_t:
        return x1, None
    tdv = _mlp_tangent(gnn.dec, mk, th)
    tv1 = tx[:, :, 3:] + tdv
    tp1 = tx[:, :, :3] + gnn.dt * tv1
    return x1, np.concatenate([tp1, tv1], axis=2)


def rollout(gnn, g, x0, U):
    """x_hat[0] = x0, x_hat[k+1] = F(x_hat[k], U[k]) for k < N.  Returns [N+1, M, 6]."""
    N = U.shape[0]
    xs = [np.asarray(x0, dtype=np.float64)]
    for k in range(N):
        xs.append(step(gnn, g, xs[-1], U[k]))
    return np.stack(xs)


def jacobian_dense(gnn, g, x, u):
    """Full A = dF/dx [6M, 6M], B = dF/du [6M, nu], c = F - A x - B u (exact, all columns)."""
    M, nu = g.M, g.nu
    nx = 6 * M
    T = nx + nu
    tx = np.zeros((T, M, 6))
    tx[np.arange(nx), np.arange(nx) // 6, np.arange(nx) % 6] = 1.0
    tu = np.zeros((T, nu))
    tu[nx + np.arange(nu), np.arange(nu)] = 1.0
    x1, t1 = step_jvp(gnn, g, x, u, tx, tu)
    cols = t1.reshape(T, nx)           # row t = derivative along input coordinate t
    A = cols[:nx].T.copy()
    B = cols[nx:].T.copy()
    c = x1.reshape(-1) - A @ np.asarray(x, np.float64).reshape(-1) - B @ np.asarray(u, np.float64)
    return A, B, c, x1


def local_jacobian_rows(gnn, g, x, u, i):
    """Rows of node i only, differentiated on node i's K-hop subgraph.

    Returns (ball, Ablk [len(ball), 6, 6], Bi [6, nu], f_i [6]) with Ablk[b] = A^{i, ball[b]}.
    The subgraph holds every node within K hops of i and every edge between
    them, which is everything f^i depends on.
    """
    ball = g.in_ball(i, gnn.K)
    loc = {n: b for b, n in enumerate(ball)}
    keep = [k for k in range(g.E) if int(g.src[k]) in loc and int(g.dst[k]) in loc]
    src = np.array([loc[int(g.src[k])] for k in keep], dtype=np.int64)
    dst = np.array([loc[int(g.dst[k])] for k in keep], dtype=np.int64)
    # actuators outside the ball cannot reach node i
    act = np.array([loc.get(int(n), -1) for n in g.act_node])
    sub = Graph(len(ball), src, dst, g.nu, act)
    xs = np.asarray(x, np.float64)[ball]
    nb = len(ball)
    T = 6 * nb + g.nu
    tx = np.zeros((T, nb, 6))
    tx[np.arange(6 * nb), np.arange(6 * nb) // 6, np.arange(6 * nb) % 6] = 1.0
    tu = np.zeros((T, g.nu))
    tu[6 * nb + np.arange(g.nu), np.arange(g.nu)] = 1.0
    x1, t1 = step_jvp(gnn, sub, xs, u, tx, tu)
    bi = loc[int(i)]
    rows = t1[:, bi, :]                 # [T, 6]: derivative of f^i along each input
    Ablk = rows[:6 * nb].reshape(nb, 6, 6).transpose(0, 2, 1).copy()
    Bi = rows[6 * nb:].T.copy()
    return ball, Ablk, Bi, x1[bi]


def preactivations_min_abs(gnn, g, x, u):
    """Smallest |pre-activation| over every ReLU of F(x, u) (distance to a kink)."""
    x = np.asarray(x, np.float64)
    u = np.asarray(u, np.float64)
    src, dst = g.src, g.dst
    mins = []

    def mlp(p, z):
        W1, b1, W2, b2 = p
        a = z @ W1 + b1
        mins.append(np.abs(a).min() if a.size else np.inf)
        return np.maximum(a, 0.0) @ W2 + b2

    h = mlp(gnn.node_enc, np.concatenate([x, g.actuator_mask() * u[None]], 1))
    e = mlp(gnn.edge_enc, x[dst] - x[src])
    for l in range(gnn.K):
        e = e + mlp(gnn.edge_mp[l], np.concatenate([h[dst], h[src], e], 1))
        agg = np.zeros_like(h)
        np.add.at(agg, dst, e)
        h = h + mlp(gnn.node_mp[l], np.concatenate([h, agg], 1))
    mlp(gnn.dec, h)
    return float(min(mins))
