"""The learned warm start's kernels (features, MLP forward, MSE backward, Adam) against the
FP64 oracle, and the generate / fit / evaluate pipeline on a small case.  Needs a GPU.

Tolerances: the net's products run on tensor cores with each FP32 operand split into two
BF16 pieces (about 16 bits) and FP32 accumulation, over lengths <= 512 and three layers:
2e-4 of each quantity's max-abs for features, outputs and gradients; Adam's first steps move
parameters by about lr, compared to 1e-6 absolute at lr = 1e-4 (the update's FP32 rounding).
"""
import numpy as np
import pytest

from gpu_helpers import max_rel_err, orti
from oracle import warmstart as ows
from synth import small_chain

pytestmark = pytest.mark.gpu

REL = 2e-4


def _net(lib, dims, B):
    from paper_2602_17601_b300.warmstart import WarmStartNet
    return WarmStartNet(dims[0], dims[2], n_hidden=dims[1], max_batch=B)


def test_features_match_oracle(lib):
    from paper_2602_17601_b300.warmstart import features, features_size
    wl = small_chain()
    prob = lib.RTIProblem.from_workload(wl)
    torch = prob.torch
    rng = np.random.default_rng(0)
    for s in range(3):
        x = (np.asarray(wl.x0, np.float64).reshape(wl.M, 6) + rng.normal(0, 0.02, (wl.M, 6))).astype(np.float32)
        x_dev = torch.as_tensor(x.reshape(-1), device="cuda")
        prob.reset()
        f = features(prob, x_dev, prob.x_ref, torch.empty(features_size(prob), device="cuda")).cpu().numpy()
        gnn, g = orti.model_of(wl)
        fo = ows.features(gnn, g, x.astype(np.float64), np.zeros(wl.nu), wl.x_ref)
        assert f.shape == fo.shape
        assert max_rel_err(f, fo) <= REL, max_rel_err(f, fo)


def _norm(rng, dims):
    return (rng.normal(0, 0.3, dims[0]), rng.uniform(0.5, 2.0, dims[0]), rng.normal(0, 0.3, dims[2]),
            rng.uniform(0.5, 2.0, dims[2]))


def test_forward_matches_oracle(lib):
    import torch
    dims, B = (94, 512, 80), 37
    rng = np.random.default_rng(1)
    theta = ows.init_params(dims, 3) + rng.normal(0, 0.01, ows.layout(*dims)[1])
    im, isd, om, osd = _norm(rng, dims)
    net = _net(lib, dims, 64)
    net.set_params(theta, np.concatenate([im, isd, om, osd]))
    x = rng.normal(0, 1, (B, dims[0]))
    out = net.forward(torch.as_tensor(x.astype(np.float32), device="cuda")).cpu().numpy()
    ys, _ = ows.forward(theta, ows.standardise(x, im, isd), dims)
    assert max_rel_err(out, ys * osd + om) <= REL


def test_train_step_matches_oracle_gradient_and_adam(lib):
    import torch
    dims, B = (30, 64, 12), 48
    rng = np.random.default_rng(2)
    theta = ows.init_params(dims, 4)
    im, isd, om, osd = _norm(rng, dims)
    net = _net(lib, dims, 64)
    net.set_params(theta, np.concatenate([im, isd, om, osd]))
    x = rng.normal(0, 1, (B, dims[0]))
    t = rng.normal(0, 1, (B, dims[2]))
    lr = 1e-4
    loss = net.train_step(torch.as_tensor(x.astype(np.float32), device="cuda"),
                          torch.as_tensor(t.astype(np.float32), device="cuda"), lr)
    g = net.grad().cpu().numpy()
    p, _ = net.get_params()
    L, go = ows.loss_and_grad(theta, ows.standardise(x, im, isd), ows.standardise(t, om, osd), dims)
    assert abs(float(loss.item()) - L) <= REL * L
    assert max_rel_err(g, go) <= REL, max_rel_err(g, go)
    po, _, _ = ows.adam_step(theta, go, np.zeros_like(theta), np.zeros_like(theta), 1, lr)
    # entries whose gradient is tiny flip sign under FP32 rounding; compare where |g| is resolved
    sel = np.abs(go) > 1e-3 * np.abs(go).max()
    assert np.abs(p - po)[sel].max() <= 1e-6


def test_training_reduces_the_loss(lib):
    import torch
    dims, B = (16, 64, 8), 128
    rng = np.random.default_rng(3)
    Wt = rng.normal(0, 1, (dims[0], dims[2]))
    x = rng.normal(0, 1, (4096, dims[0])).astype(np.float32)
    y = (0.25 * x @ Wt).astype(np.float32)        # a linear map: well within a ReLU MLP's reach
    X, Y = torch.as_tensor(x, device="cuda"), torch.as_tensor(y, device="cuda")
    from paper_2602_17601_b300.warmstart import fit
    net = _net(lib, dims, B)
    hist = fit(net, X, Y, epochs=15, batch=B, lr=3e-3)
    assert hist[-1] < 0.1 * hist[0], hist


def test_pipeline_small(lib):
    """generate -> fit -> evaluate on cfg1 shapes: every solve converges and the warm-started
    (or fallen-back) U agrees with the cold U to the solver tolerance."""
    from paper_2602_17601_b300 import warmstart as W
    wl = small_chain(tol=1e-4)
    prob = lib.RTIProblem.from_workload(wl)
    inst = []
    for s in range(260):
        w = small_chain(seed=10**6 + s, w_seed=0)
        inst.append((w.x0, w.x_ref))
    feat, target, iters = W.generate(prob, inst[:200])
    assert np.isfinite(feat.cpu().numpy()).all() and np.isfinite(target.cpu().numpy()).all()
    net = W.WarmStartNet(feat.shape[1], target.shape[1], n_hidden=128, max_batch=64)
    W.fit(net, feat, target, epochs=20, batch=32, lr=1e-3)
    rows = W.evaluate(prob, net, inst[200:])
    s = W.summarise(rows)
    assert s["all_converged"], s
    # both solves stop at residual tol (inf-norm); H >= Rbar = min(R) I, so each U lies within
    # sqrt(nU) tol / min(R) of U* in the 2-norm, and the two within twice that
    nU = wl.N * wl.nu
    assert s["max_du"] <= 2 * np.sqrt(nU) * wl.tol / float(np.min(wl.Rdiag)), s


def test_trained_warm_start_halves_the_admm_iterations(lib):
    """What the trained net gains over cold ADMM: 3000 cold solves of chain-of-10 instances
    (state and reference from seeds 1e6 + s) train the 94 -> 512 -> 512 -> 80 net on the
    device; on 300 held-out instances the warm-started solves (the library's own cold restart
    as the fallback on a stall) take at most half the cold solves' mean iterations, every solve
    converges to the same tolerance, and the two U agree within the solver's own bound."""
    from paper_2602_17601_b300 import warmstart as W
    wl = small_chain(tol=1e-4)
    prob = lib.RTIProblem.from_workload(wl)
    inst = W.cfg5_instances(3300)
    feat, target, _ = W.generate(prob, inst[:3000])
    net = W.WarmStartNet(feat.shape[1], target.shape[1], n_hidden=512, max_batch=256)
    hist = W.fit(net, feat, target, epochs=40, batch=256, lr=1e-3)
    assert hist[-1] < 0.5 * hist[0], hist
    s = W.summarise(W.evaluate(prob, net, inst[3000:]))
    print(f"warm start, chain of 10, 3000 training solves: held-out ADMM iterations cold "
          f"{s['cold_iters_mean']:.2f}, warm {s['warm_iters_mean']:.2f} (medians {s['cold_iters_median']:.0f}, "
          f"{s['warm_iters_median']:.0f}), cold restarts {s['fallbacks']}, max |U_warm - U_cold| {s['max_du']:.2e}")
    assert s["all_converged"], s
    assert s["warm_iters_mean"] <= 0.5 * s["cold_iters_mean"], s
    nU = wl.N * wl.nu
    assert s["max_du"] <= 2 * np.sqrt(nU) * wl.tol / float(np.min(wl.Rdiag)), s
