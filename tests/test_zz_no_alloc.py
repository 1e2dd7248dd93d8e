"""gm_qp_solve_noalloc: the QP solve for callers that cannot allocate device memory.

Such callers (a real-time control loop that must not call cudaMalloc once it
runs, or a plug-in whose host runtime owns all device memory) cannot create a
context, whose workspace is caller-allocated.  The no-allocation entry point
keeps its scratch in one array inside the library.  This test calls it twice
in a row through the C ABI and checks both results against gm_qp_solve on the
same QP, within the solver tolerance used by the other QP tests (10 tol / rho).
It lives in its own file, collected last, and also passes run alone.
"""
import numpy as np
import pytest

from gpu_helpers import dense_to_packed_ct, ocd, oracle_linearize, orti
from synth import small_chain

pytestmark = pytest.mark.gpu


def _constrained_qp():
    """The chain-of-10 QP with two half-spaces per node and stage through the nominal positions."""
    wl = small_chain()
    u_hat = np.random.default_rng(3).uniform(-0.5, 0.5, (wl.N, wl.nu))
    xo, Ao, Bo, co = oracle_linearize(wl, u_hat)
    gnn, gr = orti.model_of(wl)
    nbh = [gr.in_ball(i, wl.K) for i in range(wl.M)]
    rng = np.random.default_rng(5)
    n = rng.normal(0, 1, (wl.N, wl.M, 2, 3))
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    p = xo[1:, :, None, :3]
    dx = np.einsum("kics,kics->kic", n, np.broadcast_to(p, n.shape)) + 1e-4
    H, g, Ct, dt, _, _ = ocd.condense_recursive(ocd.blocks_from_dense(Ao, Bo, co, nbh), xo[0].reshape(-1),
                                                wl.Qdiag, wl.Rdiag, wl.x_ref, wl.u_ref, n, dx)
    return wl, n.astype(np.float32), dx.astype(np.float32), H, g, Ct, dt


def test_noalloc_solve_matches_context_solve_twice(lib):
    import torch
    wl, Cx, dx, H, g, Ct, dt = _constrained_qp()
    n_c = Cx.shape[2]
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")  # noqa: E731
    H_d, g_d = dev(H), dev(g)
    Ct_d, dt_d = dev(dense_to_packed_ct(Ct, wl.N, wl.M, n_c, wl.nu)), dev(dt)
    lo, hi = dev(wl.u_lo.reshape(-1)), dev(wl.u_hi.reshape(-1))
    # the existing entry point, through a context
    prob = lib.RTIProblem(wl.M, wl.src, wl.dst, wl.nu, wl.act_node, wl.K, wl.W, wl.dt, wl.blob, wl.N,
                          wl.Qdiag, wl.Rdiag, wl.x_ref, wl.u_ref, wl.u_lo, wl.u_hi, Cx=Cx, dx=dx,
                          rho=wl.rho, tol=wl.tol, max_iter=wl.max_iter)
    U_ref, y_ref = prob.qp_solve(H_d, g_d, Ct_d, dt_d)
    st_ref = prob.read_stats()
    U_ref = U_ref.cpu().numpy()
    assert st_ref["converged"] == 1
    # the no-allocation entry point, two calls in a row on the same scratch
    s = lib.make_settings(wl.N, n_c, rho=wl.rho, tol=wl.tol, max_iter=wl.max_iter)
    nU, rows = wl.N * wl.nu, wl.N * wl.M * n_c
    for call in range(2):
        U = torch.full((nU,), float("nan"), device="cuda")
        y = torch.full((nU + rows,), float("nan"), device="cuda")
        stats = torch.zeros(lib.STATS_BYTES, dtype=torch.uint8, device="cuda")
        lib.gm_qp_solve_noalloc(wl.N, wl.nu, wl.M * n_c, s, H_d, g_d, Ct_d, dt_d, lo, hi, U, y, stats)
        st = lib.read_stats(stats)
        Un = U.cpu().numpy()
        assert st["status"] == lib.GM_OK and st["converged"] == 1, (call, st)
        assert abs(st["iters"] - st_ref["iters"]) <= max(3, 0.05 * st_ref["iters"]), (call, st, st_ref)
        assert np.abs(Un - U_ref).max() <= 10 * wl.tol / wl.rho, (call, np.abs(Un - U_ref).max())
        assert np.all(np.isfinite(y.cpu().numpy()))


def test_noalloc_rejects_sizes_beyond_its_limit(lib):
    import torch
    s = lib.make_settings(9, 0)
    z = torch.zeros(1, device="cuda")
    with pytest.raises(lib.GMError) as e:      # N * nu = 72 > 64
        lib.gm_qp_solve_noalloc(9, 8, 0, s, z, z, None, None, z, z, z)
    assert e.value.code == lib.GM_ERR_INVALID_ARG
    with pytest.raises(lib.GMError) as e:      # 8 * 1100 = 8800 rows > 8192
        lib.gm_qp_solve_noalloc(8, 4, 1100, s, z, z, z, z, z, z, z)
    assert e.value.code == lib.GM_ERR_INVALID_ARG


_FRESH = r"""
import sys, ctypes
sys.path.insert(0, sys.argv[1])
import numpy as np
import torch
import paper_2602_17601_b300 as gm
torch.cuda.init()
N, nu, Mnc = 4, 2, 3
rng = np.random.default_rng(0)
L = rng.normal(0, 1, (N * nu, N * nu))
H = (L @ L.T + 0.1 * np.eye(N * nu)).astype(np.float32)
g = rng.normal(0, 1, N * nu).astype(np.float32)
Ct = rng.normal(0, 1, Mnc * nu * N * (N + 1) // 2).astype(np.float32)
dt = np.full(N * Mnc, 1.0, np.float32)
dev = lambda a: torch.as_tensor(a, device="cuda")
H_d, g_d, Ct_d, dt_d = dev(H), dev(g), dev(Ct), dev(dt)
lo, hi = dev(-np.ones(N * nu, np.float32)), dev(np.ones(N * nu, np.float32))
U = torch.empty(N * nu, device="cuda")
stats = torch.zeros(gm.STATS_BYTES, dtype=torch.uint8, device="cuda")
s = gm.make_settings(N, 1, rho=0.1, tol=1e-6, max_iter=4000)
torch.cuda.synchronize()
gm.gm_qp_solve_noalloc(N, nu, Mnc, s, H_d, g_d, Ct_d, dt_d, lo, hi, U, None, stats)   # first call: loads the modules
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
for _ in range(2):
    gm.gm_qp_solve_noalloc(N, nu, Mnc, s, H_d, g_d, Ct_d, dt_d, lo, hi, U, None, stats)
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
st = gm.read_stats(stats)
print(free0, free1, st["status"], st["converged"])
"""


def test_noalloc_later_calls_leave_free_device_memory_unchanged(lib, tmp_path):
    """In a fresh process whose only library call is the no-allocation solve: after the first
    call (which loads the library's modules onto the device), two more calls leave the device's
    free memory (cudaMemGetInfo) unchanged."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "fresh_noalloc.py"
    script.write_text(_FRESH)
    r = subprocess.run([sys.executable, str(script), root], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    free0, free1, status, conv = (int(v) for v in r.stdout.split()[-4:])
    assert status == lib.GM_OK and conv == 1, r.stdout
    assert free1 == free0, (free0, free1)
