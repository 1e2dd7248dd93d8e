"""Learned ADMM warm start (an addition to the paper's method), around the gm_ws_* C calls.

A 3-layer MLP maps pooled GNN latents and the reference of an MPC instance to a
primal input sequence U^0 and box duals y^0 that warm-start the condensed-QP
ADMM.  Cold-start ADMM remains the fallback (the library restarts a stalled
warm-started solve cold, `solve_with_fallback`) and the arbiter of the net's error.  Everything numeric runs in the library's kernels:

* features       gm_ws_features (stage-0 GNN latents, mean/max pooled, + reference)
* inference      gm_ws_forward
* training       gm_ws_train_step (forward, MSE, backward, Adam)

This module only allocates device memory (torch), moves arguments and drives
the loops: dataset generation by cold solves, minibatch training, and the
held-out warm-versus-cold evaluation.
"""
from __future__ import annotations

import ctypes as C
import time

import numpy as np

from . import STATS_BYTES, _check, _lib, _ptr, _stream, read_stats


def features_size(prob):
    return 2 * prob.W + 3 * prob.M


class WarmStartNet:
    """The MLP in a caller-owned (torch) device workspace."""

    def __init__(self, n_in, n_out, n_hidden=512, max_batch=1024, device="cuda"):
        import torch
        self.torch = torch
        self.n_in, self.n_hid, self.n_out, self.max_batch = int(n_in), int(n_hidden), int(n_out), int(max_batch)
        nbytes = _lib.gm_ws_workspace_size(self.n_in, self.n_hid, self.n_out, self.max_batch)
        if nbytes == 0:
            raise ValueError("invalid warm-start net sizes")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = self.workspace.data_ptr()
        off = (-base) % 256
        h = C.c_void_p()
        _check("gm_ws_create", _lib.gm_ws_create(self.n_in, self.n_hid, self.n_out, self.max_batch,
                                                 C.c_void_p(base + off), nbytes, C.byref(h)))
        self.h = h
        self.n_par = int(_lib.gm_ws_param_count(h))
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)

    def __del__(self):
        if getattr(self, "h", None):
            _lib.gm_ws_destroy(self.h)
            self.h = None

    def init_params(self, seed, in_mean, in_std, out_mean, out_std):
        """He-normal weights (seeded numpy), zero biases, and the standardisation."""
        rng = np.random.default_rng(seed)
        parts = []
        for din, dout in ((self.n_in, self.n_hid), (self.n_hid, self.n_hid), (self.n_hid, self.n_out)):
            parts.append(rng.normal(0.0, np.sqrt(2.0 / din), din * dout))
            parts.append(np.zeros(dout))
        self.set_params(np.concatenate(parts), np.concatenate([in_mean, in_std, out_mean, out_std]))

    def set_params(self, params, norm):
        t = self.torch
        p = t.as_tensor(np.asarray(params, np.float32), device=self.workspace.device).contiguous()
        n = t.as_tensor(np.asarray(norm, np.float32), device=self.workspace.device).contiguous()
        _check("gm_ws_set_params", _lib.gm_ws_set_params(self.h, _ptr(p), _ptr(n), _stream(None)))
        t.cuda.current_stream().synchronize()

    def get_params(self):
        t = self.torch
        p = t.empty(self.n_par, dtype=t.float32, device=self.workspace.device)
        n = t.empty(2 * (self.n_in + self.n_out), dtype=t.float32, device=self.workspace.device)
        _check("gm_ws_get_params", _lib.gm_ws_get_params(self.h, _ptr(p), _ptr(n), _stream(None)))
        return p.cpu().numpy(), n.cpu().numpy()

    def forward(self, feat, out=None):
        B = int(feat.shape[0])
        out = self.torch.empty(B, self.n_out, dtype=self.torch.float32, device=feat.device) if out is None else out
        _check("gm_ws_forward", _lib.gm_ws_forward(self.h, _ptr(feat), B, _ptr(out), _stream(None)))
        return out

    def train_step(self, feat, target, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        """One Adam step; returns the (device) loss of the batch before the step."""
        B = int(feat.shape[0])
        _check("gm_ws_train_step", _lib.gm_ws_train_step(self.h, _ptr(feat), _ptr(target), B, lr, beta1, beta2,
                                                         eps, _ptr(self.loss), _stream(None)))
        return self.loss

    def grad(self):
        g = self.torch.empty(self.n_par, dtype=self.torch.float32, device=self.workspace.device)
        _check("gm_ws_grad", _lib.gm_ws_grad(self.h, _ptr(g), _stream(None)))
        return g


def features(prob, x_meas, x_ref, out):
    """Warm-start features of (x_meas, x_ref) at the context's current u_hat into out [2W + 3M]."""
    _check("gm_ws_features", _lib.gm_ws_features(prob.ctx, _ptr(x_meas), _ptr(x_ref), _ptr(out), _stream(None)))
    return out


def generate(prob, instances, tol=None):
    """Features and cold-solve targets [U*, box duals] for a list of (x0, x_ref) arrays.

    Each instance is linearised at u_hat = 0 (a cold start), condensed and solved by
    cold ADMM.  Returns device tensors feat [n, F], target [n, 2 nU] and the host
    iteration counts of the cold solves."""
    t = prob.torch
    n, F, nU = len(instances), features_size(prob), prob.nU
    feat = t.empty(n, F, dtype=t.float32, device="cuda")
    target = t.empty(n, 2 * nU, dtype=t.float32, device="cuda")
    stats = t.empty(n, STATS_BYTES, dtype=t.uint8, device="cuda")
    x_dev = t.empty(prob.M * 6, dtype=t.float32, device="cuda")
    zeros_u = t.zeros(prob.N, prob.nu, dtype=t.float32, device="cuda")
    y = t.empty(nU + prob.rows_c, dtype=t.float32, device="cuda")
    for i, (x0, x_ref) in enumerate(instances):
        x_dev.copy_(t.as_tensor(np.asarray(x0, np.float32).reshape(-1)))
        prob.x_ref.copy_(t.as_tensor(np.asarray(x_ref, np.float32)).reshape(prob.x_ref.shape))
        prob.reset()
        features(prob, x_dev, prob.x_ref, feat[i])
        x_hat, A, B, c = prob.linearize(x_dev, zeros_u)
        H, g, Ct, dt = prob.condense(x_hat, A, B, c)
        U = target[i, :nU]
        from . import gm_qp_solve
        gm_qp_solve(prob.ctx, H, g, Ct if prob.n_c else None, dt if prob.n_c else None, prob.u_lo, prob.u_hi,
                    U, y, stats[i], None, None)
        target[i, nU:].copy_(y[:nU])
    t.cuda.synchronize()
    iters = np.array([read_stats(stats[i])["iters"] for i in range(n)])
    return feat, target, iters


def fit(net, feat, target, epochs=30, batch=256, lr=1e-3, seed=0, log=None):
    """Minibatch Adam on (feat, target); the standardisation comes from the training set."""
    t = net.torch
    fm, fs = feat.mean(0), feat.std(0).clamp_min(1e-6)
    tm, ts = target.mean(0), target.std(0).clamp_min(1e-6)
    net.init_params(seed, fm.cpu().numpy(), fs.cpu().numpy(), tm.cpu().numpy(), ts.cpu().numpy())
    n = feat.shape[0]
    g = t.Generator(device="cpu").manual_seed(seed)
    history = []
    for ep in range(epochs):
        perm = t.randperm(n, generator=g).to(feat.device)
        lr_ep = lr * 0.5 * (1.0 + np.cos(np.pi * ep / epochs))       # cosine schedule
        tot = t.zeros(1, device=feat.device)
        steps = 0
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch]
            tot += net.train_step(feat[idx].contiguous(), target[idx].contiguous(), lr_ep)
            steps += 1
        history.append(float(tot.item()) / max(steps, 1))
        if log:
            log(f"epoch {ep}: loss {history[-1]:.5f}")
    return history


def solve_with_fallback(prob, H, g, Ct, dt, warm, stats):
    """Warm-started ADMM from warm = [U0, box duals].  The library itself restarts the solve
    cold when the warm start stalls (max(r_p, r_d) not halved over 25 iterations) or turns
    NaN, and then reports GM_STALLED.  Returns (U, cold_fallback_used)."""
    from . import GM_STALLED, gm_qp_solve
    t = prob.torch
    nU = prob.nU
    U = t.empty(nU, dtype=t.float32, device="cuda")
    y0 = t.zeros(nU + prob.rows_c, dtype=t.float32, device="cuda")
    y0[:nU].copy_(warm[nU:])
    gm_qp_solve(prob.ctx, H, g, Ct if prob.n_c else None, dt if prob.n_c else None, prob.u_lo, prob.u_hi, U,
                None, stats, warm[:nU].contiguous(), y0)
    return U, read_stats(stats)["status"] == GM_STALLED


def evaluate(prob, net, instances):
    """Held-out comparison at the context's tolerance on the same H, g: iterations and device
    time of cold ADMM against features + net inference + warm-started ADMM (including the
    cold restart the library makes when the warm start stalls)."""
    from . import GM_STALLED, gm_qp_solve
    t = prob.torch
    nU, F = prob.nU, features_size(prob)
    feat = t.empty(F, dtype=t.float32, device="cuda")
    sc_t = t.empty(STATS_BYTES, dtype=t.uint8, device="cuda")
    sw_t = t.empty(STATS_BYTES, dtype=t.uint8, device="cuda")
    x_dev = t.empty(prob.M * 6, dtype=t.float32, device="cuda")
    zeros_u = t.zeros(prob.N, prob.nu, dtype=t.float32, device="cuda")
    y0 = t.zeros(nU + prob.rows_c, dtype=t.float32, device="cuda")
    Uc = t.empty(nU, dtype=t.float32, device="cuda")
    Uw = t.empty(nU, dtype=t.float32, device="cuda")
    ev = [t.cuda.Event(enable_timing=True) for _ in range(5)]
    ct = lambda: Ct if prob.n_c else None  # noqa: E731
    dtt = lambda: dt if prob.n_c else None  # noqa: E731
    rows = []
    for x0, x_ref in instances:
        x_dev.copy_(t.as_tensor(np.asarray(x0, np.float32).reshape(-1)))
        prob.x_ref.copy_(t.as_tensor(np.asarray(x_ref, np.float32)).reshape(prob.x_ref.shape))
        prob.reset()
        x_hat, A, B, c = prob.linearize(x_dev, zeros_u)
        H, g, Ct, dt = prob.condense(x_hat, A, B, c)
        ev[0].record()
        gm_qp_solve(prob.ctx, H, g, ct(), dtt(), prob.u_lo, prob.u_hi, Uc, None, sc_t, None, None)
        ev[1].record()
        prob.reset()
        ev[2].record()
        features(prob, x_dev, prob.x_ref, feat)
        warm = net.forward(feat.view(1, F)).view(-1)
        y0[:nU].copy_(warm[nU:])
        ev[3].record()
        gm_qp_solve(prob.ctx, H, g, ct(), dtt(), prob.u_lo, prob.u_hi, Uw, None, sw_t, warm[:nU].contiguous(), y0)
        ev[4].record()
        t.cuda.synchronize()
        sc, sw = read_stats(sc_t), read_stats(sw_t)
        # a stalled warm start was restarted cold inside the solve (its time and iterations
        # are part of the warm solve's)
        fell_back = sw["status"] == GM_STALLED
        net_ms, solve_ms = ev[2].elapsed_time(ev[3]), ev[3].elapsed_time(ev[4])
        rows.append(dict(cold_iters=sc["iters"], warm_iters=sw["iters"], cold_ms=ev[0].elapsed_time(ev[1]),
                         warm_ms=net_ms + solve_ms, net_ms=net_ms, warm_solve_ms=solve_ms,
                         fallback=fell_back, du=float((Uw - Uc).abs().max().item()),
                         pred_err=float((warm[:nU] - Uc).abs().max().item()),
                         cold_ok=sc["converged"], warm_ok=sw["converged"]))
    return rows


def summarise(rows):
    f = lambda k: np.array([r[k] for r in rows], dtype=float)  # noqa: E731
    return {"instances": len(rows),
            "cold_iters_mean": float(f("cold_iters").mean()), "warm_iters_mean": float(f("warm_iters").mean()),
            "cold_iters_median": float(np.median(f("cold_iters"))),
            "warm_iters_median": float(np.median(f("warm_iters"))),
            "cold_ms_mean": float(f("cold_ms").mean()), "warm_ms_mean": float(f("warm_ms").mean()),
            "warm_net_ms_mean": float(f("net_ms").mean()), "warm_solve_ms_mean": float(f("warm_solve_ms").mean()),
            "fallbacks": int(f("fallback").sum()), "max_du": float(f("du").max()),
            "pred_err_mean": float(f("pred_err").mean()),
            "all_converged": bool(f("cold_ok").all() and f("warm_ok").all())}


def timed(fn):
    t0 = time.perf_counter()
    out = fn()
    return out, time.perf_counter() - t0


def cfg5_instances(n, first_seed=10**6, **kw):
    """(x0, x_ref) of n chain-of-10 instances: seeds first_seed + s for the state and the
    reference, the GNN and graph of seed 0 (the chain of 10 workload)."""
    from synth import small_chain
    out = []
    for s in range(n):
        w = small_chain(seed=first_seed + s, w_seed=0, **kw)
        out.append((w.x0, w.x_ref))
    return out


def main(argv=None):
    """Train and evaluate the warm start on chain-of-10 instances (90/10 split); print a JSON report."""
    import argparse
    import json

    import torch

    from synth import small_chain
    from .rti import RTIProblem
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=100000)
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--hidden", type=int, default=512)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--eval", type=int, default=2000, help="held-out instances timed (of the 10%%)")
    a = ap.parse_args(argv)
    wl = small_chain(tol=a.tol)
    prob = RTIProblem.from_workload(wl)
    inst, t_inst = timed(lambda: cfg5_instances(a.n))
    n_train = int(0.9 * a.n)
    (feat, target, iters), t_gen = timed(lambda: generate(prob, inst[:n_train]))
    net = WarmStartNet(feat.shape[1], target.shape[1], n_hidden=a.hidden, max_batch=max(a.batch, 1))
    hist, t_fit = timed(lambda: fit(net, feat, target, epochs=a.epochs, batch=a.batch, lr=a.lr))
    held = inst[n_train:][:a.eval]
    rows, t_eval = timed(lambda: evaluate(prob, net, held))
    rep = {"workload": "chain10_K2_W32_N10_nu4 (GNN of seed 0; state and reference from seeds 1e6 + s)",
           "tol": a.tol, "instances": a.n, "train": n_train, "held_out_timed": len(held),
           "net": f"{feat.shape[1]} -> {a.hidden} -> {a.hidden} -> {target.shape[1]}",
           "epochs": a.epochs, "batch": a.batch, "lr": a.lr,
           "train_cold_iters_mean": float(iters.mean()), "loss_first_last": [hist[0], hist[-1]],
           "held_out": summarise(rows),
           "seconds": {"instances": t_inst, "generate": t_gen, "fit": t_fit, "evaluate": t_eval},
           "device": torch.cuda.get_device_name()}
    print(json.dumps(rep), flush=True)
    return rep


if __name__ == "__main__":
    main()
