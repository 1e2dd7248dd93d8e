"""CUDA-graph replay of gm_rti_step (gm_ctx_set_graph) against eager steps.  Needs a GPU.

The graph runs the same kernels in the same order, so the receding-horizon
sequence (Alg. 1: shifted warm trajectory carried from step to step) must match
the eager one up to the order of floating-point atomics in the ADMM reductions.
"""
import numpy as np
import pytest

from synth import paper_chain, small_chain

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make", [small_chain, lambda: paper_chain(M=40, N=5, nu=4)], ids=["chain10", "chain40"])
def test_graph_steps_match_eager(lib, make):
    wl = make()
    runs = {}
    for graph in (False, True):
        prob = lib.RTIProblem.from_workload(wl, graph=graph)
        Us = []
        for _ in range(4):
            Us.append(prob.step(wl.x0).cpu().numpy().astype(np.float64))
            assert prob.read_stats()["converged"] == 1
        runs[graph] = (Us, prob.graph_state())
    (eager, _), (graphed, (replayed, captures)) = runs[False], runs[True]
    assert captures == 1 and replayed == 1
    for k, (a, b) in enumerate(zip(eager, graphed)):
        assert np.abs(a - b).max() <= 10 * wl.tol / wl.rho, (k, np.abs(a - b).max())


def test_graph_recaptures_when_a_pointer_changes(lib):
    wl = small_chain()
    prob = lib.RTIProblem.from_workload(wl, graph=True)
    torch = prob.torch
    for _ in range(3):
        prob.step(wl.x0)
    assert prob.graph_state() == (1, 1)
    U2 = torch.full((prob.nU,), float("nan"), device="cuda")   # a new output pointer: captured anew
    prob.step(wl.x0, U=U2)
    assert prob.graph_state() == (1, 2)
    assert np.isfinite(U2.cpu().numpy()).all() and prob.read_stats()["converged"] == 1
    prob.step(wl.x0, U=U2)
    assert prob.graph_state() == (1, 2)


def test_graph_replay_runs_rounds_after_a_rho_update(lib):
    """Cold solves from a small rho change rho after 25 iterations and need the ADMM rounds after
    the first.  In the captured step those rounds sit in nested conditional nodes that the device
    enables while the solve is not done, so the replayed steps (each from its own measured state)
    must still run them, converge and reach the eager solutions.  Measured states far apart and
    tight input bounds (no spheres) keep box constraints active in every step."""
    wl = paper_chain(M=40, N=5, nu=4, u_bound=0.02, n_spheres=0)
    x0 = np.asarray(wl.x0, np.float32).reshape(-1)
    rng = np.random.default_rng(5)
    states = [x0 + np.float32(0.3 * (-1) ** k) * np.abs(rng.standard_normal(x0.shape)).astype(np.float32)
              for k in range(4)]
    runs = {}
    for graph in (False, True):
        prob = lib.RTIProblem.from_workload(wl, graph=graph, warm=False, rho=1e-3)
        out = []
        for x in states:
            U = prob.step(x).cpu().numpy().astype(np.float64)
            st = prob.read_stats()
            assert st["converged"] == 1, (graph, len(out), st)
            out.append((U, st["iters"]))
        runs[graph] = (out, prob.graph_state())
    (eager, _), (graphed, (replayed, captures)) = runs[False], runs[True]
    assert captures == 1 and replayed == 1
    iters = [it for _, it in eager]
    assert max(iters[1:]) > 25, iters              # the replayed steps went past the first rho check
    for k, ((a, _), (b, _)) in enumerate(zip(eager, graphed)):
        assert np.abs(a - b).max() <= 10 * wl.tol / wl.rho, (k, np.abs(a - b).max())
