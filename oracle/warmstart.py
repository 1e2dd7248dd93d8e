"""Learned ADMM warm start, FP64 (oracle; test infrastructure only).

The warm start is an addition to the paper's method (not in the paper): a
3-layer MLP  in -> H -> H -> out  with ReLU between layers maps the features
of an MPC instance to a primal input sequence U^0 and box duals y^0.

* ``features``  mean and max over nodes of the final node latents h^K of
  stage 0 (the GNN of Sec. V-A evaluated at (x, u)), then the stage-1
  reference positions.
* ``forward`` / ``loss_and_grad``  the MLP on standardised inputs, the mean
  squared error of the standardised outputs, and its gradient by the chain
  rule written out layer by layer (ReLU derivative 0 at 0).
* ``adam_step``  Adam (Kingma and Ba, 2015) with bias correction.

Parameters are packed [W0 (in x H) | b0 | W1 (H x H) | b1 | W2 (H x out) | b2],
each W with rows = fan-in.
"""
from __future__ import annotations

import numpy as np


def layout(n_in, n_hid, n_out):
    """[(W offset, W shape, b offset, b size)] of the packed parameter vector, and its length."""
    out, o = [], 0
    for din, dout in ((n_in, n_hid), (n_hid, n_hid), (n_hid, n_out)):
        out.append((o, (din, dout), o + din * dout, dout))
        o += din * dout + dout
    return out, o


def unpack(theta, n_in, n_hid, n_out):
    lay, _ = layout(n_in, n_hid, n_out)
    return [(theta[ow:ow + s[0] * s[1]].reshape(s), theta[ob:ob + nb]) for ow, s, ob, nb in lay]


def node_latents(gnn, g, x, u):
    """h^K [M, W]: the encoder and K message-passing steps of the GNN at (x, u)."""
    x = np.asarray(x, np.float64)
    u = np.asarray(u, np.float64)

    def mlp(p, z):
        W1, b1, W2, b2 = p
        return np.maximum(z @ W1 + b1, 0.0) @ W2 + b2

    h = mlp(gnn.node_enc, np.concatenate([x, g.actuator_mask() * u[None]], axis=1))
    e = mlp(gnn.edge_enc, x[g.dst] - x[g.src])
    for l in range(gnn.K):
        e = e + mlp(gnn.edge_mp[l], np.concatenate([h[g.dst], h[g.src], e], axis=1))
        agg = np.zeros_like(h)
        np.add.at(agg, g.dst, e)
        h = h + mlp(gnn.node_mp[l], np.concatenate([h, agg], axis=1))
    return h


def features(gnn, g, x, u, x_ref):
    """[mean_i h^K_i, max_i h^K_i, x_ref[1][i][0..2] for all i]."""
    h = node_latents(gnn, g, x, u)
    M = h.shape[0]
    ref = np.asarray(x_ref, np.float64).reshape(-1, M, 6)[1, :, :3].reshape(-1)
    return np.concatenate([h.mean(axis=0), h.max(axis=0), ref])


def forward(theta, xs, dims):
    """Standardised outputs y [B, out] and the activations (x, a0, a1) for standardised inputs xs."""
    (W0, b0), (W1, b1), (W2, b2) = unpack(theta, *dims)
    a0 = np.maximum(xs @ W0 + b0, 0.0)
    a1 = np.maximum(a0 @ W1 + b1, 0.0)
    return a1 @ W2 + b2, (xs, a0, a1)


def standardise(v, mean, sd):
    return (np.asarray(v, np.float64) - mean) / sd


def loss_and_grad(theta, xs, ts, dims):
    """L = mean over batch and outputs of (y - t)^2 on standardised data, and dL/dtheta."""
    (W0, b0), (W1, b1), (W2, b2) = unpack(theta, *dims)
    y, (x, a0, a1) = forward(theta, xs, dims)
    B, n_out = y.shape
    r = y - ts
    L = float((r * r).sum() / (B * n_out))
    dy = 2.0 * r / (B * n_out)
    gW2, gb2 = a1.T @ dy, dy.sum(axis=0)
    d1 = (dy @ W2.T) * (a1 > 0)
    gW1, gb1 = a0.T @ d1, d1.sum(axis=0)
    d0 = (d1 @ W1.T) * (a0 > 0)
    gW0, gb0 = x.T @ d0, d0.sum(axis=0)
    grad = np.concatenate([gW0.ravel(), gb0, gW1.ravel(), gb1, gW2.ravel(), gb2])
    return L, grad


def adam_step(theta, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step at step count t (1-based); returns new (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def init_params(dims, seed):
    """He-normal weights, zero biases (the random numbers are the generator's, passed in)."""
    rng = np.random.default_rng(seed)
    lay, n = layout(*dims)
    theta = np.zeros(n)
    for ow, (din, dout), _, _ in lay:
        theta[ow:ow + din * dout] = rng.normal(0.0, np.sqrt(2.0 / din), din * dout)
    return theta


