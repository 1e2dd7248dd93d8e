"""Training loss of the GNN dynamics model and its gradient, FP64 (oracle; test infrastructure only).

Sec. V-A "Training": the model is fitted on transitions (x_t, u_t, x_{t+1}) by minimising
the mean squared prediction error weighted by O, plus an L2 penalty on the parameters,
with Adam.  Readings (the paper gives the loss, not these details):

* O is diagonal with one weight per state component (p, v), shared by all nodes:
  ||r||^2_O = sum_i sum_a O_a r_{i,a}^2;
* theta is the whole weight blob (weights and biases of every MLP), so
  lambda ||theta||^2 covers both;
* the mean is over the transitions of the batch:
      L(theta) = 1/B sum_b ||x_{t+1,b} - F_theta(x_{t,b}, u_{t,b})||^2_O + lambda ||theta||^2;
* Adam is the published update (Kingma and Ba, 2015) with bias correction; the
  learning-rate schedule on patience is left to the caller.

The gradient is reverse-mode through one application of F (oracle.gnn.step), written out
layer by layer: decoder, the K message-passing levels in reverse (node update, sum
aggregation, edge update, residual paths), then both encoders.  It returns the gradient in
blob order, so it can be compared with any flat parameter vector.
"""
from __future__ import annotations

import numpy as np

from . import gnn as og


def _forward_cache(gnn, g, x, u):
    """F(x, u) with every layer input and ReLU mask kept for the reverse pass."""
    x = np.asarray(x, np.float64)
    u = np.asarray(u, np.float64)
    src, dst = g.src, g.dst
    c = {}
    z = np.concatenate([x, g.actuator_mask() * u[None, :]], axis=1)
    h, m = og._mlp(gnn, gnn.node_enc, z)
    c["ne"] = (z, m)
    d = x[dst] - x[src]
    e, m = og._mlp(gnn, gnn.edge_enc, d)
    c["ee"] = (d, m)
    c["levels"] = []
    for lvl in range(gnn.K):
        ze = np.concatenate([h[dst], h[src], e], axis=1)
        de, me = og._mlp(gnn, gnn.edge_mp[lvl], ze)
        e = e + de
        agg = np.zeros_like(h)
        np.add.at(agg, dst, e)
        zn = np.concatenate([h, agg], axis=1)
        dh, mn = og._mlp(gnn, gnn.node_mp[lvl], zn)
        c["levels"].append((ze, me, zn, mn))
        h = h + dh
    dv, m = og._mlp(gnn, gnn.dec, h)
    c["dec"] = (h, m)
    v1 = x[:, 3:] + dv
    x1 = np.concatenate([x[:, :3] + gnn.dt * v1, v1], axis=1)
    return x1, c


def _mlp_back(p, z, m, dy):
    """Cotangents of Linear -> ReLU -> Linear: (dW1, db1, dW2, db2), dz for output cotangent dy."""
    W1, _, W2, _ = p
    a = np.where(m, z @ W1 + p[1], 0.0)
    dW2 = a.T @ dy
    db2 = dy.sum(axis=0)
    da = np.where(m, dy @ W2.T, 0.0)
    dW1 = z.T @ da
    db1 = da.sum(axis=0)
    return (dW1, db1, dW2, db2), da @ W1.T


def step_vjp(gnn, g, x, u, dx1):
    """Gradient of <dx1, F(x, u)> with respect to every MLP's (W1, b1, W2, b2), blob order."""
    _, c = _forward_cache(gnn, g, x, u)
    src, dst = g.src, g.dst
    K, W = gnn.K, gnn.W
    grads = [None] * (3 + 2 * K)
    # x1 = [p + dt v1, v1], v1 = v + dv
    dv1 = dx1[:, 3:] + gnn.dt * dx1[:, :3]
    hK, m = c["dec"]
    grads[2 + 2 * K], dh = _mlp_back(gnn.dec, hK, m, dv1)
    de = np.zeros((src.size, W))
    for lvl in reversed(range(K)):
        ze, me, zn, mn = c["levels"][lvl]
        # h_{l+1} = h_l + MLP_n([h_l, agg_l]), agg_l = sum over in-edges of e_{l+1}
        grads[3 + 2 * lvl], dzn = _mlp_back(gnn.node_mp[lvl], zn, mn, dh)
        dh = dh + dzn[:, :W]
        de = de + dzn[:, W:][dst]
        # e_{l+1} = e_l + MLP_e([h_l[dst], h_l[src], e_l])
        grads[2 + 2 * lvl], dze = _mlp_back(gnn.edge_mp[lvl], ze, me, de)
        np.add.at(dh, dst, dze[:, :W])
        np.add.at(dh, src, dze[:, W:2 * W])
        de = de + dze[:, 2 * W:]
    z, m = c["ne"]
    grads[0], _ = _mlp_back(gnn.node_enc, z, m, dh)
    d, m = c["ee"]
    grads[1], _ = _mlp_back(gnn.edge_enc, d, m, de)
    return grads


def flatten(grads):
    """Per-MLP (W1, b1, W2, b2) in blob order -> one flat vector."""
    return np.concatenate([np.concatenate([a.reshape(-1) for a in gr]) for gr in grads])


def loss(blob, K, W, nu, dt, g, X, U, Xn, O, lam):
    """L(theta) of the module docstring; X, Xn [B, M, 6], U [B, nu], O [6]."""
    gnn = og.GNN(blob, K, W, nu, dt)
    O = np.asarray(O, np.float64)
    err = 0.0
    for x, u, xn in zip(X, U, Xn):
        r = np.asarray(xn, np.float64) - og.step(gnn, g, x, u)
        err += float((O[None, :] * r * r).sum())
    th = np.asarray(blob, np.float64)
    return err / len(X) + lam * float(th @ th)


def loss_grad(blob, K, W, nu, dt, g, X, U, Xn, O, lam):
    """(L, dL/dtheta) with the gradient in blob order."""
    gnn = og.GNN(blob, K, W, nu, dt)
    O = np.asarray(O, np.float64)
    th = np.asarray(blob, np.float64)
    B = len(X)
    L = lam * float(th @ th)
    grad = 2.0 * lam * th
    for x, u, xn in zip(X, U, Xn):
        x1 = og.step(gnn, g, x, u)
        r = np.asarray(xn, np.float64) - x1
        L += float((O[None, :] * r * r).sum()) / B
        grad = grad + flatten(step_vjp(gnn, g, x, u, -2.0 * O[None, :] * r / B))
    return L, grad


def adam_step(theta, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015); t counts from 1.  Returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
