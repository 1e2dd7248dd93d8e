"""The C-ABI library loads, exports every entry point of include/gm.h, and validates
its arguments on the host.  No GPU: only host-side calls (no compute)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "gm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gm_[a-z_]+)\s*\(", src)))


def test_library_exports_every_header_function():
    import paper_2602_17601_b300 as gm
    lib = ctypes.CDLL(gm.LIB_PATH)
    names = header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(gm.HEADER_FUNCTIONS) <= set(names)


def test_graph_and_gnn_validation():
    import paper_2602_17601_b300 as gm
    from synth import small_chain
    wl = small_chain()
    g = gm.gm_graph_create(wl.M, wl.src, wl.dst, wl.nu, wl.act_node)
    m = gm.gm_gnn_load(wl.K, wl.W, wl.nu, wl.dt, wl.blob)
    s = gm.make_settings(wl.N)
    assert gm.gm_ctx_workspace_size(g, m, s) > 0
    bad = [
        lambda: gm.gm_graph_create(3, [0, 1], [1, 1], 1, [0]),        # self-loop
        lambda: gm.gm_graph_create(3, [0, 0], [1, 1], 1, [0]),        # duplicate
        lambda: gm.gm_graph_create(3, [0], [3], 1, [0]),              # out of range
        lambda: gm.gm_graph_create(3, [0], [1], 1, [5]),              # actuator out of range
        lambda: gm.gm_gnn_load(wl.K, wl.W, wl.nu, wl.dt, wl.blob[:-1]),   # wrong size
        lambda: gm.gm_gnn_load(wl.K, 48, wl.nu, wl.dt, wl.blob),          # unsupported width
        lambda: gm.gm_ctx_workspace_size(g, m, gm.make_settings(0)),      # N = 0
        lambda: gm.gm_ctx_workspace_size(g, m, gm.make_settings(wl.N, condensing=2)),        # no such path
        lambda: gm.gm_ctx_workspace_size(g, m, gm.make_settings(wl.N, condensing=1, tan_split_rows=-1)),
        lambda: gm.gm_ctx_workspace_size(g, gm.gm_gnn_load(wl.K, wl.W, 3, wl.dt,
                                                           np.zeros(_blob(wl.K, wl.W, 3), np.float32)), s),
    ]
    for f in bad:
        with pytest.raises(gm.GMError) as e:
            f()
        assert e.value.code == gm.GM_ERR_INVALID_ARG
    nan_blob = wl.blob.copy()
    nan_blob[3] = np.nan
    with pytest.raises(gm.GMError):
        gm.gm_gnn_load(wl.K, wl.W, wl.nu, wl.dt, nan_blob)
    gm.gm_gnn_destroy(m)
    gm.gm_graph_destroy(g)


def _blob(K, W, nu):
    from synth import gnn_blob_size
    return gnn_blob_size(K, W, nu)


def test_workspace_grows_linearly_in_nodes():
    """Thm. 1: memory O(M) for fixed n_x-bar, n_u, N and neighbourhood size."""
    import paper_2602_17601_b300 as gm
    from synth import paper_chain
    sizes = []
    Ms = [200, 400, 800]
    for M in Ms:
        wl = paper_chain(M=M, N=5, nu=4)
        g = gm.gm_graph_create(wl.M, wl.src, wl.dst, wl.nu, wl.act_node)
        m = gm.gm_gnn_load(wl.K, wl.W, wl.nu, wl.dt, wl.blob)
        sizes.append(gm.gm_ctx_workspace_size(g, m, gm.make_settings(wl.N, 5)))
    slope = np.polyfit(np.log(Ms), np.log(sizes), 1)[0]
    assert abs(slope - 1.0) < 0.1, (sizes, slope)


def test_no_cuda_device_fails_loudly():
    """Without a CUDA device the compute path raises; there is no CPU fallback."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import paper_2602_17601_b300 as gm
    from synth import small_chain
    with pytest.raises(Exception):
        gm.RTIProblem.from_workload(small_chain())


def _check_plan(gm, width, cost, sms):
    lane, n = gm.gm_batch_plan(width, cost, sms)
    w = np.minimum(np.asarray(width), sms)
    assert n >= 1 and lane.min() >= 0 and lane.max() < n and len(np.unique(lane)) == n
    # the widest grid of every lane, summed over the lanes, fits on the SMs
    lane_w = np.array([w[lane == l].max() for l in range(n)])
    assert lane_w.sum() <= sms, (lane_w, sms)
    return lane, n


def test_batch_plan_lanes_fit_and_balance():
    import paper_2602_17601_b300 as gm
    rng = np.random.default_rng(0)
    # one width: SMs // width lanes, and the costs spread within the LPT bound
    cost = rng.uniform(1, 10, 200)
    lane, n = _check_plan(gm, [32] * 200, cost, 148)
    assert n == 4
    loads = np.array([cost[lane == l].sum() for l in range(n)])
    assert loads.max() <= cost.sum() / n + cost.max()      # greedy list-scheduling bound
    # two widths: a lane of the wide class plus lanes of the narrow one, more than 148 // 32
    width = [32] * 20 + [16] * 100
    lane, n = _check_plan(gm, width, np.ones(120), 148)
    assert n > 4
    # a width above the SMs counts as the SMs: one lane
    lane, n = _check_plan(gm, [200, 8, 8], [1, 1, 1], 148)
    assert n == 1
    # fewer instances than lanes: one lane each
    lane, n = _check_plan(gm, [8, 8, 8], [3, 2, 1], 148)
    assert n == 3
    # random widths and costs
    for seed in range(20):
        r = np.random.default_rng(seed)
        k = int(r.integers(1, 60))
        _check_plan(gm, r.choice([2, 8, 16, 32, 64, 128], k), r.uniform(0, 5, k), int(r.integers(1, 200)))
    assert gm.gm_batch_plan([], [], 148)[1] == 0
    with pytest.raises(gm.GMError):
        gm.gm_batch_plan([0], [1.0], 148)
    with pytest.raises(gm.GMError):
        gm.gm_batch_plan([4], [-1.0], 148)


def test_null_handles_are_rejected_on_the_host():
    """Entry points taking a handle validate it before any CUDA call (GM_ERR_INVALID_ARG = 1)."""
    import paper_2602_17601_b300 as gm
    lib = ctypes.CDLL(gm.LIB_PATH)
    lib.gm_ctx_set_warm.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.gm_ctx_set_graph.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.gm_batch_set_lanes.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.gm_barrier_fold.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_float] * 2 + [ctypes.c_void_p] * 3
    lib.gm_qp_solve_ipm.argtypes = [ctypes.c_void_p] * 7 + [ctypes.c_int] + [ctypes.c_void_p] * 4
    assert lib.gm_ctx_set_warm(None, 1) == 1
    assert lib.gm_ctx_set_graph(None, 1) == 1
    assert lib.gm_batch_set_lanes(None, 2) == 1
    assert lib.gm_barrier_fold(None, None, None, None, 1e-3, 5e-3, None, None, None) == 1
    assert lib.gm_qp_solve_ipm(None, None, None, None, None, None, None, 10, None, None, None, None) == 1
    lib.gm_last_error.restype = ctypes.c_char_p
    assert b"NULL" in lib.gm_last_error()
