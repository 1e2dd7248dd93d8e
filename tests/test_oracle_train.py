"""Pins of the training-loss oracle (oracle.train, Sec. V-A "Training") to things other than itself.

* the reverse-mode gradient of the loss against central finite differences of the loss
  itself, on sampled parameters of every MLP, at a point kept away from ReLU kinks;
* targets equal to the model's own predictions: the data term vanishes, so the gradient
  is exactly 2 lambda theta;
* the loss with O = 0 is lambda ||theta||^2 (a closed form);
* Adam against its update written out for two steps on a scalar, and a few Adam steps
  lowering the loss of a small model.
"""
import numpy as np

from oracle import gnn as og
from oracle import rti as orti
from oracle import train as otr
from synth import random_instance


def _setup(seed=0, B=3, w_scale="0.5"):
    # at weight scale 0.5 every path through the graph moves the loss visibly (at 0.1 the
    # source-node path of the edge updates changes the gradient by 1e-8 only)
    wl = random_instance(seed, M=5, N=2, nu=2, K=2, W=4, reach=2, p=0.8, directed=True, w_scale=w_scale)
    gnn, g = orti.model_of(wl)
    rng = np.random.default_rng(100 + seed)
    x0 = np.asarray(wl.x0, np.float64).reshape(wl.M, 6)
    X = np.stack([x0 + rng.normal(0, 0.02, x0.shape) for _ in range(B)])
    U = rng.uniform(-1, 1, (B, wl.nu))
    Xn = np.stack([og.step(gnn, g, X[b], U[b]) + rng.normal(0, 0.01, x0.shape) for b in range(B)])
    O = np.array([1.0, 1.0, 1.0, 0.5, 0.5, 0.5])
    return wl, g, X, U, Xn, O


def _min_preact(wl, g, X, U, blob):
    gnn = og.GNN(blob, wl.K, wl.W, wl.nu, wl.dt)
    return min(og.preactivations_min_abs(gnn, g, X[b], U[b]) for b in range(len(X)))


def test_gradient_matches_finite_differences():
    lam = 1e-3
    for seed in range(6):                       # the first instance whose ReLUs keep a margin
        wl, g, X, U, Xn, O = _setup(seed)
        blob = np.asarray(wl.blob, np.float64)
        if _min_preact(wl, g, X, U, blob) > 1e-4:     # FD steps of 1e-6 move none across a kink
            break
    else:
        raise AssertionError("no kink-free instance among the seeds")
    args = (wl.K, wl.W, wl.nu, wl.dt, g, X, U, Xn, O, lam)
    L, grad = otr.loss_grad(blob, *args)
    assert abs(L - otr.loss(blob, *args)) <= 1e-12 * max(1.0, abs(L))
    h = 1e-6
    for i in range(blob.size):                  # every parameter of every MLP
        e = np.zeros_like(blob)
        e[i] = h
        fd = (otr.loss(blob + e, *args) - otr.loss(blob - e, *args)) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (i, fd, grad[i])


def test_zero_residual_leaves_only_the_penalty():
    wl, g, X, U, _, O = _setup(1)
    gnn, _ = orti.model_of(wl)
    Xn = np.stack([og.step(gnn, g, X[b], U[b]) for b in range(len(X))])
    blob = np.asarray(wl.blob, np.float64)
    lam = 0.05
    L, grad = otr.loss_grad(blob, wl.K, wl.W, wl.nu, wl.dt, g, X, U, Xn, O, lam)
    np.testing.assert_allclose(grad, 2 * lam * blob, rtol=0, atol=1e-12)
    assert abs(L - lam * blob @ blob) <= 1e-12
    # O = 0: the loss is the penalty alone for any data
    _, _, _, _, Xr, _ = _setup(2)
    L0 = otr.loss(blob, wl.K, wl.W, wl.nu, wl.dt, g, X, U, Xr[:len(X)], np.zeros(6), lam)
    assert abs(L0 - lam * blob @ blob) <= 1e-12


def test_adam_update_and_descent():
    # two steps on f(t) = t^2 from t = 1 with lr 0.1, written out
    t, m, v = np.array([1.0]), np.zeros(1), np.zeros(1)
    t1, m1, v1 = otr.adam_step(t, 2 * t, m, v, 1, lr=0.1)
    g1 = 2.0
    mh, vh = 0.1 * g1 / (1 - 0.9), 0.001 * g1 * g1 / (1 - 0.999)
    assert np.isclose(t1[0], 1.0 - 0.1 * mh / (np.sqrt(vh) + 1e-8))
    t2, _, _ = otr.adam_step(t1, 2 * t1, m1, v1, 2, lr=0.1)
    g2 = 2 * t1[0]
    m2, v2 = 0.9 * 0.1 * g1 + 0.1 * g2, 0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2
    assert np.isclose(t2[0], t1[0] - 0.1 * (m2 / (1 - 0.81)) / (np.sqrt(v2 / (1 - 0.999 ** 2)) + 1e-8))
    # a few Adam steps on the model lower the loss
    wl, g, X, U, Xn, O = _setup(3, w_scale="0.1")
    th = np.asarray(wl.blob, np.float64)
    args = (wl.K, wl.W, wl.nu, wl.dt, g, X, U, Xn, O, 1e-4)
    L0 = otr.loss(th, *args)
    m, v = np.zeros_like(th), np.zeros_like(th)
    for k in range(1, 21):
        _, grad = otr.loss_grad(th, *args)
        th, m, v = otr.adam_step(th, grad, m, v, k, lr=5e-3)
    assert otr.loss(th, *args) < 0.9 * L0
