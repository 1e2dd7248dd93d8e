"""Pins of the warm-start oracle (CPU): the MLP gradient against central
differences of the FP64 loss, the all-active linear regime, the first Adam step
and invariances of the pooled GNN-latent features."""
import numpy as np

from oracle import rti as orti
from oracle import warmstart as ows
from synth import random_instance, small_chain

DIMS = (7, 9, 5)


def _kink_free_batch(theta, rng, B=6, margin=1e-3):
    """Standardised inputs whose pre-activations all keep a margin from 0 (FD is smooth there)."""
    (W0, b0), (W1, b1), _ = ows.unpack(theta, *DIMS)
    for _ in range(200):
        xs = rng.normal(0, 1, (B, DIMS[0]))
        z0 = xs @ W0 + b0
        z1 = np.maximum(z0, 0) @ W1 + b1
        if np.abs(z0).min() > margin and np.abs(z1).min() > margin:
            return xs
    raise AssertionError("no kink-free batch")


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = ows.init_params(DIMS, 1) + rng.normal(0, 0.05, ows.layout(*DIMS)[1])
    xs = _kink_free_batch(theta, rng)
    ts = rng.normal(0, 1, (xs.shape[0], DIMS[2]))
    L, g = ows.loss_and_grad(theta, xs, ts, DIMS)
    h = 1e-6
    fd = np.empty_like(theta)
    for i in range(theta.size):
        e = np.zeros_like(theta)
        e[i] = h
        fd[i] = (ows.loss_and_grad(theta + e, xs, ts, DIMS)[0] - ows.loss_and_grad(theta - e, xs, ts, DIMS)[0]) / (2 * h)
    assert np.abs(fd - g).max() <= 1e-7 * max(1.0, np.abs(g).max()), np.abs(fd - g).max()
    assert L > 0


def test_all_active_mlp_is_the_product_of_its_matrices():
    # with every pre-activation positive the ReLUs pass through: y = x W0 W1 W2 + const
    rng = np.random.default_rng(2)
    lay, n = ows.layout(*DIMS)
    theta = rng.uniform(0.1, 0.5, n)                    # positive weights and biases
    xs = rng.uniform(0.0, 1.0, (4, DIMS[0]))            # positive inputs: all units active
    (W0, b0), (W1, b1), (W2, b2) = ows.unpack(theta, *DIMS)
    y, _ = ows.forward(theta, xs, DIMS)
    expect = xs @ (W0 @ W1 @ W2) + (b0 @ W1 @ W2 + b1 @ W2 + b2)
    assert np.allclose(y, expect, rtol=1e-13, atol=1e-13)


def test_first_adam_step_moves_against_the_gradient_sign():
    rng = np.random.default_rng(3)
    theta = rng.normal(0, 1, 50)
    g = rng.normal(0, 1, 50)
    lr = 1e-3
    new, m, v = ows.adam_step(theta, g, np.zeros(50), np.zeros(50), 1, lr)
    step = theta - new
    # bias-corrected first step: lr |g| / (|g| + eps) against sign(g), i.e. lr up to eps
    assert np.all(np.sign(step) == np.sign(g))
    assert np.allclose(np.abs(step), lr, rtol=1e-6)


def test_adam_minimises_a_convex_quadratic():
    rng = np.random.default_rng(4)
    A = rng.normal(0, 1, (8, 8))
    Q = A @ A.T + np.eye(8)
    b = rng.normal(0, 1, 8)
    x_star = np.linalg.solve(Q, b)
    x, m, v = np.zeros(8), np.zeros(8), np.zeros(8)
    for t in range(1, 3001):
        x, m, v = ows.adam_step(x, Q @ x - b, m, v, t, 0.05)
    assert np.abs(x - x_star).max() < 1e-3


def test_pooled_features_are_permutation_invariant_and_carry_the_reference():
    wl = random_instance(5, M=9, N=3, nu=2, K=2, W=16, reach=2, p=0.7)
    gnn, g = orti.model_of(wl)
    rng = np.random.default_rng(5)
    x = np.asarray(wl.x0, np.float64).reshape(wl.M, 6)
    u = rng.uniform(-0.5, 0.5, wl.nu)
    f = ows.features(gnn, g, x, u, wl.x_ref)
    # relabel the nodes: pooled latents unchanged, reference block permuted accordingly
    perm = rng.permutation(wl.M)
    inv = np.argsort(perm)
    src, dst = inv[g.src], inv[g.dst]
    wl2 = random_instance(5, M=9, N=3, nu=2, K=2, W=16, reach=2, p=0.7)
    wl2.src, wl2.dst, wl2.act_node = src.astype(np.int32), dst.astype(np.int32), inv[wl.act_node].astype(np.int32)
    gnn2, g2 = orti.model_of(wl2)
    xr = np.asarray(wl.x_ref, np.float64).reshape(-1, wl.M, 6)[:, perm]
    f2 = ows.features(gnn2, g2, x[perm], u, xr)
    W = gnn.W
    assert np.allclose(f2[:2 * W], f[:2 * W], atol=1e-12)
    assert np.allclose(f2[2 * W:].reshape(wl.M, 3), f[2 * W:].reshape(wl.M, 3)[perm], atol=0)
    assert np.allclose(f[2 * W:].reshape(wl.M, 3), xr[1, inv][:, :3], atol=0)


def test_pooled_mean_equals_max_when_all_latents_are_equal():
    # an edgeless graph of identical nodes (no actuator input): every h^K_i is the same
    wl = small_chain()
    gnn, g = orti.model_of(wl)
    g.src = g.src[:0]
    g.dst = g.dst[:0]
    x = np.tile(np.asarray(wl.x0, np.float64).reshape(wl.M, 6)[:1], (wl.M, 1))
    f = ows.features(gnn, g, x, np.zeros(wl.nu), wl.x_ref)
    W = gnn.W
    assert np.allclose(f[:W], f[W:2 * W], atol=1e-14)
