"""Closed-loop receding horizon with the GNN as the plant (outer loop of Algorithm 1) against the
oracle's closed loop (exact QP optimum each step, FP64 plant).  Needs a GPU.

Both loops linearise at the shifted previous solution and apply the first input to the same GNN.
The GPU's U differs from the exact optimum by the ADMM tolerance and FP32 rounding, so the
trajectories separate slowly; over 6 steps at tol 1e-6 they stay within 1e-4 of each other."""
import numpy as np
import pytest

from gpu_helpers import ogm, orti
from synth import small_chain

pytestmark = pytest.mark.gpu


def _oracle_loop(wl, steps):
    gnn, g = orti.model_of(wl)
    x = np.asarray(wl.x0, np.float64).reshape(wl.M, 6)
    xs, us, u_prev = [x.copy()], [], None
    for _ in range(steps):
        w = wl
        w.x0 = x.astype(np.float32).reshape(np.asarray(wl.x0).shape)
        uh = None if u_prev is None else orti.shift(u_prev)
        r = orti.rti_step(w, u_hat=uh, solver="exact", return_all=True)
        u_prev = r["U"]
        u0 = r["U"][0]
        x = ogm.step(gnn, g, x, u0)
        xs.append(x.copy())
        us.append(u0)
    return np.stack(xs), np.stack(us)


def test_closed_loop_matches_oracle(lib):
    from paper_2602_17601_b300 import closed_loop
    wl = small_chain()
    x0 = np.asarray(wl.x0, np.float64).copy()
    prob = lib.RTIProblem.from_workload(wl)
    S, U, stats = closed_loop.run(prob, x0, 6)
    assert all(s["converged"] == 1 for s in stats)
    So, Uo = _oracle_loop(small_chain(), 6)
    assert np.abs(U - Uo).max() <= 1e-4, np.abs(U - Uo).max()
    assert np.abs(S - So).max() <= 1e-4, np.abs(S - So).max()


def test_warm_started_closed_loop_matches_oracle_in_fewer_iterations(lib):
    """The receding-horizon warm start (gm_ctx_set_warm: each step's ADMM starts from the
    shifted previous U*, y*) follows the oracle's closed loop as closely as cold starts do,
    and needs fewer ADMM iterations once the loop runs."""
    from paper_2602_17601_b300 import closed_loop
    wl = small_chain()
    x0 = np.asarray(wl.x0, np.float64).copy()
    S, U, st_w = closed_loop.run(lib.RTIProblem.from_workload(wl, warm=True), x0, 6)
    _, _, st_c = closed_loop.run(lib.RTIProblem.from_workload(small_chain()), x0, 6)
    assert all(s["converged"] == 1 for s in st_w)
    So, Uo = _oracle_loop(small_chain(), 6)
    assert np.abs(U - Uo).max() <= 1e-4, np.abs(U - Uo).max()
    assert np.abs(S - So).max() <= 1e-4, np.abs(S - So).max()
    assert st_w[0]["iters"] == st_c[0]["iters"]                 # the first step starts cold
    warm_its = sum(s["iters"] for s in st_w[1:])
    cold_its = sum(s["iters"] for s in st_c[1:])
    print(f"closed loop, steps 2-6: ADMM iterations warm {warm_its}, cold {cold_its}")
    assert warm_its < cold_its, (warm_its, cold_its)


def test_rollout_matches_oracle_step(lib):
    from paper_2602_17601_b300 import gm_rollout
    wl = small_chain()
    prob = lib.RTIProblem.from_workload(wl)
    torch = prob.torch
    rng = np.random.default_rng(0)
    u = rng.uniform(-0.5, 0.5, (3, wl.nu)).astype(np.float32)
    out = torch.empty(4, wl.M * 6, device="cuda")
    gm_rollout(prob.ctx, torch.as_tensor(wl.x0, device="cuda"), torch.as_tensor(u, device="cuda"), 3, out)
    gnn, g = orti.model_of(wl)
    xo = ogm.rollout(gnn, g, wl.x0, u.astype(np.float64))
    assert np.abs(out.cpu().numpy().reshape(4, wl.M, 6) - xo).max() <= 2e-4 * np.abs(xo).max()
