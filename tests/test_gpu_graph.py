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
