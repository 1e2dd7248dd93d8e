"""Matrix-free condensing, FP64 (oracle; test infrastructure only).

The condensed QP needs the sensitivities S_k = d x_k / d U, the block rows of Gamma_u.  The
Thm. 1 proof builds them with the recursion of Eq. sparse_gamma_i_u, S_{k+1} = A_k S_k + B_k E_k,
from the explicit local Jacobians A_k, B_k.  Here the product A_k S_k + B_k E_k is taken as one
directional derivative of the stage map F(x, u) of Eq. forward_dynamics, so A_k is never
formed:

    S_0 = 0
    S_{k+1}[:, t] = dF/dx(x_hat_k, u_hat_k) S_k[:, t] + dF/du(x_hat_k, u_hat_k) [t in stage k]

for every column t = (stage i, input a), with one tangent per column that can be non-zero at
stage k (the k nu columns of the earlier stages plus the nu new ones).  Column (i, a) vanishes
for k <= i, and for k > i outside the nodes that act_node[a] reaches in K (k - i) edges: one
stage moves an influence K message-passing hops along the edges (source to destination).

The affine part follows from the rollout: the linearised prediction x = Gamma_u U + Gamma_x
reproduces x_hat at U = U_hat, so Gamma_x = x_hat - Gamma_u U_hat.  H, g, C~, d~ are then formed
exactly as in ``condense.condense_dense`` (Eq. condensed_matrices).
"""
from __future__ import annotations

from collections import deque

import numpy as np

from . import condense as cd
from . import gnn as gm


def downstream_ball(g, a, R):
    """Nodes that node a reaches along directed edges (source -> destination) in at most R edges."""
    out = [[] for _ in range(g.M)]
    for s, d in zip(g.src, g.dst):
        out[int(s)].append(int(d))
    dist = {int(a): 0}
    q = deque([int(a)])
    while q:
        v = q.popleft()
        if dist[v] == R:
            continue
        for w in out[v]:
            if w not in dist:
                dist[w] = dist[v] + 1
                q.append(w)
    return sorted(dist)


def sensitivities(gnn, g, x0, U_hat):
    """Rollout x_hat [N+1, M, 6] and S [N+1, M, 6, N nu] (S[k] = d x_k / d U) by forward-mode
    products through the GNN, one tangent per input column (columns of later stages are 0)."""
    U_hat = np.asarray(U_hat, np.float64)
    N, nu = U_hat.shape
    M = g.M
    nU = N * nu
    x = np.asarray(x0, np.float64).reshape(M, 6)
    xs = [x]
    S = np.zeros((N + 1, M, 6, nU))
    for k in range(N):
        T = (k + 1) * nu                              # columns that can be non-zero after stage k
        tx = np.moveaxis(S[k][:, :, :T], 2, 0)        # [T, M, 6]
        tu = np.zeros((T, nu))
        tu[k * nu + np.arange(nu), np.arange(nu)] = 1.0
        x1, t1 = gm.step_jvp(gnn, g, x, U_hat[k], tx, tu)
        S[k + 1][:, :, :T] = np.moveaxis(t1, 0, 2)
        x = x1
        xs.append(x)
    return np.stack(xs), S


def condense_matrix_free(gnn, g, x0, U_hat, Qdiag, Rdiag, x_ref, u_ref, Cx, dx):
    """H, g, C~ (stage-major rows), d~, Gamma_u, Gamma_x of Eq. condensed_matrices from the
    forward-mode sensitivities; same conventions and layout as condense.condense_dense."""
    U_hat = np.asarray(U_hat, np.float64)
    N, nu = U_hat.shape
    M = g.M
    nx = 6 * M
    x_hat, S = sensitivities(gnn, g, x0, U_hat)
    Gu = S.reshape(N + 1, nx, N * nu).reshape((N + 1) * nx, N * nu)
    Gx = x_hat.reshape(-1) - Gu @ U_hat.reshape(-1)
    Qbar = np.diag(np.asarray(Qdiag, np.float64).reshape(-1))
    Rbar = np.diag(np.asarray(Rdiag, np.float64).reshape(-1))
    xr = np.asarray(x_ref, np.float64).reshape(-1)
    ur = np.asarray(u_ref, np.float64).reshape(-1)
    H = Gu.T @ Qbar @ Gu + Rbar
    gv = Gu.T @ Qbar @ (Gx - xr) - Rbar @ ur
    n_c = Cx.shape[2] if Cx is not None else 0
    if n_c == 0:
        return H, gv, np.zeros((0, N * nu)), np.zeros(0), Gu, Gx
    Sel = cd.position_selector(M)
    rows = N * M * n_c
    Cbar = np.zeros((rows, (N + 1) * nx))
    dbar = np.zeros(rows)
    for k in range(1, N + 1):
        Ck = np.zeros((M * n_c, 3 * M))
        for i in range(M):
            Ck[i * n_c:(i + 1) * n_c, 3 * i:3 * i + 3] = Cx[k - 1, i]
        r0 = (k - 1) * M * n_c
        Cbar[r0:r0 + M * n_c, k * nx:(k + 1) * nx] = Ck @ Sel
        dbar[r0:r0 + M * n_c] = np.asarray(dx[k - 1], np.float64).reshape(-1)
    return H, gv, Cbar @ Gu, dbar - Cbar @ Gx, Gu, Gx


def tangent_rows(g, K, N, nu):
    """MLP rows that a forward-mode pass restricted to the non-zero tangents evaluates per RTI
    step: for every stage k and column (i, a) with i <= k, at layer l = 0..K the nodes within
    r = K (k - i) + l hops of act_node[a] and the edges with an endpoint among them (an edge's
    tangent is non-zero once an endpoint's is).  Counting only.  Returns (node_rows, edge_rows)."""
    out = [[] for _ in range(g.M)]
    for s, d in zip(g.src, g.dst):
        out[int(s)].append(int(d))
    src, dst = np.asarray(g.src), np.asarray(g.dst)
    dists = []
    for a in range(nu):
        dist = np.full(g.M, np.iinfo(np.int64).max)
        dist[int(g.act_node[a])] = 0
        q = deque([int(g.act_node[a])])
        while q:
            v = q.popleft()
            for w in out[v]:
                if dist[w] > dist[v] + 1:
                    dist[w] = dist[v] + 1
                    q.append(w)
        dists.append(dist)
    node_rows = edge_rows = 0
    for k in range(N):
        for i in range(k + 1):
            for a in range(nu):
                for layer in range(K + 1):
                    r = K * (k - i) + layer
                    node_rows += int((dists[a] <= r).sum())
                    edge_rows += int(((dists[a][src] <= r) | (dists[a][dst] <= r)).sum())
    return node_rows, edge_rows


if __name__ == "__main__":
    import sys
    sys.path.insert(0, __import__("os").path.dirname(__import__("os").path.dirname(__import__("os").path.abspath(__file__))))
    from synth import paper_chain
    wl = paper_chain()
    g = gm.Graph(wl.M, wl.src, wl.dst, wl.nu, wl.act_node)
    nr, er = tangent_rows(g, wl.K, wl.N, wl.nu)
    print({"workload": "chain1000_K3_W128_N20_nu8", "tangent_node_rows": nr, "tangent_edge_rows": er,
           "dense_node_rows": wl.N * (wl.N + 1) // 2 * wl.nu * (wl.K + 1) * wl.M,
           "dense_edge_rows": wl.N * (wl.N + 1) // 2 * wl.nu * (wl.K + 1) * len(wl.src)})
