"""Batched real-time iterations (gm_batch_*) against stepping each instance alone.  Needs a GPU.

Instances of different node counts, horizons and input counts; each batched step (plain
launches first, then one captured graph) must give every instance the U of its own
single-instance step sequence, up to the order of floating-point atomics in the ADMM
reductions (10 tol / rho)."""
import numpy as np
import pytest

from synth import paper_chain, small_chain

pytestmark = pytest.mark.gpu


def _workloads():
    return [small_chain(), paper_chain(seed=3, M=60, N=10, nu=4, w_seed=0),
            paper_chain(seed=4, M=90, N=15, nu=8, w_seed=0), small_chain(seed=5)]


def test_batch_matches_single_instances(lib):
    from paper_2602_17601_b300.batch import Batch
    wls = _workloads()
    alone = []
    for wl in wls:
        p = lib.RTIProblem.from_workload(wl, admm_grid=8, factor_grid=16, chunk_mb=64)
        alone.append([p.step(wl.x0).cpu().numpy().copy() for _ in range(4)])
    probs = [lib.RTIProblem.from_workload(wl, admm_grid=8, factor_grid=16, chunk_mb=64) for wl in wls]
    b = Batch(probs)
    b.set_states([wl.x0 for wl in wls])
    for k in range(4):
        b.step()
        for i, (wl, p) in enumerate(zip(wls, probs)):
            U = p._U.cpu().numpy()
            assert p.read_stats()["converged"] == 1, (k, i)
            assert np.abs(U - alone[i][k]).max() <= 10 * wl.tol / wl.rho, (k, i, np.abs(U - alone[i][k]).max())
    assert b.state() == (1, 1)


def test_batch_rejects_a_repeated_context(lib):
    from paper_2602_17601_b300 import GMError
    from paper_2602_17601_b300.batch import Batch
    p = lib.RTIProblem.from_workload(small_chain())
    with pytest.raises(GMError):
        Batch([p, p])


def test_batch_matches_the_oracle_per_instance(lib):
    """Four small instances of different node counts, horizons and input counts stepped as one
    batch (plain launches, then the captured graph with its QP chain): the first batched step of
    each instance against the oracle's RTI step (exact QP optimum) on that instance, within the
    solver's tolerance bound; the second against the oracle's step from the shifted solution."""
    from oracle import rti as orti
    from paper_2602_17601_b300.batch import Batch
    from synth import random_instance
    wls = [small_chain(tol=1e-7), random_instance(7, M=8, N=6, nu=3, K=2, W=32, tol=1e-7),
           paper_chain(seed=3, M=12, N=5, nu=2, K=2, W=32, w_seed=0, tol=1e-7, n_spheres=2),
           random_instance(9, M=14, N=8, nu=2, K=1, W=64, tol=1e-7, n_spheres=1)]
    probs = [lib.RTIProblem.from_workload(wl, admm_grid=8, factor_grid=16, chunk_mb=64) for wl in wls]
    b = Batch(probs)
    b.set_states([wl.x0 for wl in wls])
    prev = [None] * len(wls)
    for k in range(2):
        b.step()
        for i, (wl, p) in enumerate(zip(wls, probs)):
            U = p._U.cpu().numpy().astype(np.float64).reshape(wl.N, wl.nu)
            st = p.read_stats()
            assert st["converged"] == 1 and st["status"] == lib.GM_OK, (k, i, st)
            ref = orti.rti_step(wl, u_hat=None if prev[i] is None else orti.shift(prev[i]), solver="exact",
                                return_all=True)
            lam = np.linalg.eigvalsh(ref["H"]).min()
            bound = 2 * max(st["r_dual"], st["kkt_stat"]) / lam + 2e-4 * max(np.abs(ref["U"]).max(), 1e-3)
            assert np.abs(U - ref["U"]).max() <= bound, (k, i, np.abs(U - ref["U"]).max(), bound)
            prev[i] = U
    assert b.state()[0] == 1
