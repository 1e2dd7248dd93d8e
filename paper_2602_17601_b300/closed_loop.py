"""Closed-loop receding horizon (the outer loop of Algorithm 1) with the GNN itself as the plant.

Each step t: the reference window x_ref[t .. t+N] (shifted by one stage per step when a
reference trajectory is given), one real-time iteration at the measured state (gm_rti_step:
rollout along the shifted previous solution, Jacobians, condensing, ADMM), the first input
applied to the plant x_{t+1} = F(x_t, u_t) (gm_rollout, one stage).  This module only moves
buffers; every step of the method runs in the library.
"""
from __future__ import annotations

import numpy as np

from . import gm_rollout, read_stats


def run(prob, x0, steps, ref_traj=None):
    """Closed loop for `steps` steps from x0 [M*6].  ref_traj: optional [steps + N + 1][M][6]
    reference trajectory (else the problem's fixed reference).  Returns (states [steps+1][M][6],
    inputs [steps][nu], per-step stats)."""
    t = prob.torch
    M, N, nu = prob.M, prob.N, prob.nu
    x = t.as_tensor(np.asarray(x0, np.float32).reshape(-1), device="cuda").clone()
    nxt = t.empty(2, M * 6, dtype=t.float32, device="cuda")
    u0 = t.empty(1, nu, dtype=t.float32, device="cuda")
    if ref_traj is not None:
        ref = t.as_tensor(np.asarray(ref_traj, np.float32), device="cuda")
        assert ref.shape[0] >= steps + N + 1, "the reference must cover steps + N + 1 stages"
    states, inputs, stats = [x.clone()], [], []
    prob.reset()
    for k in range(steps):
        if ref_traj is not None:
            prob.x_ref.copy_(ref[k:k + N + 1].reshape(prob.x_ref.shape))
        U = prob.step(x)
        u0.copy_(U[:nu].view(1, nu))
        stats.append(read_stats(prob.stats))
        gm_rollout(prob.ctx, x, u0, 1, nxt)
        x.copy_(nxt[1])
        states.append(x.clone())
        inputs.append(u0.view(-1).clone())
    S = t.stack(states).view(steps + 1, M, 6).cpu().numpy()
    Uin = t.stack(inputs).cpu().numpy()
    return S, Uin, stats


def tracking_cost(states, x_ref, Qdiag):
    """sum over steps of (x_t - x_ref)' Q (x_t - x_ref) with the stage-1 reference and weights."""
    M = states.shape[1]
    d = states - np.asarray(x_ref, np.float64).reshape(-1, M, 6)[1][None]
    q = np.asarray(Qdiag, np.float64).reshape(-1, M, 6)[1][None]
    return float((q * d * d).sum())
