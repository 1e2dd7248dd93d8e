"""GNN-MPC real-time iteration on B300 (sm_103a) — Python binding of the C ABI.

The functions here carry the names of the C entry points in include/gm.h and
only marshal arguments: every step of the method runs in the CUDA kernels of
libgm.so.  torch supplies device memory (tensors) and streams.  There is no
CPU fallback: without the library, or without a CUDA device, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgm.so")

GM_OK = 0
GM_ERR_INVALID_ARG = 1
GM_ERR_CUDA = 2
GM_ERR_WORKSPACE = 3
GM_ERR_NOT_CONVERGED = 4
GM_STALLED = 5
GM_ERR_TIMEOUT = 6
GM_ERR_NUMERIC = 7
GM_ERR_INFEASIBLE = 8
GM_PREC_FP32 = 0
GM_PREC_MIXED = 1
GM_PREC_BF16 = 2

STATUS_NAMES = {0: "GM_OK", 1: "GM_ERR_INVALID_ARG", 2: "GM_ERR_CUDA", 3: "GM_ERR_WORKSPACE",
                4: "GM_ERR_NOT_CONVERGED", 5: "GM_STALLED", 6: "GM_ERR_TIMEOUT", 7: "GM_ERR_NUMERIC",
                8: "GM_ERR_INFEASIBLE"}


class GnnDesc(C.Structure):
    _fields_ = [("K", C.c_int), ("W", C.c_int), ("nu", C.c_int), ("dt", C.c_float)]


class Settings(C.Structure):
    _fields_ = [("N", C.c_int), ("n_c", C.c_int), ("precision", C.c_int), ("rho", C.c_float),
                ("tol", C.c_float), ("max_iter", C.c_int), ("polish", C.c_int),
                ("timeout_spins", C.c_int), ("scale_rows", C.c_int), ("adapt_rho", C.c_int),
                ("admm_grid", C.c_int), ("factor_grid", C.c_int), ("chunk_mb", C.c_int),
                ("condensing", C.c_int), ("tan_split_rows", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("converged", C.c_int32),
                ("polished", C.c_int32), ("r_prim", C.c_float), ("r_dual", C.c_float),
                ("kkt_stat", C.c_double), ("kkt_prim", C.c_double), ("kkt_dual", C.c_double),
                ("kkt_comp", C.c_double)]


class Cost(C.Structure):
    _fields_ = [("Qdiag", C.c_void_p), ("Rdiag", C.c_void_p), ("x_ref", C.c_void_p),
                ("u_ref", C.c_void_p)]


class Constr(C.Structure):
    _fields_ = [("u_lo", C.c_void_p), ("u_hi", C.c_void_p), ("Cx", C.c_void_p),
                ("dx", C.c_void_p), ("n_spheres", C.c_int), ("spheres", C.c_void_p),
                ("barrier_mu", C.c_float), ("barrier_delta", C.c_float)]


class Info(C.Structure):
    _fields_ = [("M", C.c_int), ("E", C.c_int), ("nu", C.c_int), ("K", C.c_int), ("W", C.c_int),
                ("N", C.c_int), ("n_c", C.c_int), ("nU", C.c_int), ("nnzb", C.c_int),
                ("rows_c", C.c_longlong), ("cone_node_rows", C.c_longlong),
                ("cone_edge_rows", C.c_longlong), ("flops_rollout", C.c_double),
                ("flops_jacobian", C.c_double), ("flops_condense", C.c_double),
                ("flops_qp_setup", C.c_double), ("flops_admm_iter", C.c_double),
                ("bytes_admm_iter", C.c_double), ("workspace_bytes", C.c_size_t),
                ("stage_chunk", C.c_int), ("admm_grid", C.c_int)]


PHASES = ("rollout", "jacobian", "condense", "qp_setup", "admm_kkt")
STATS_BYTES = C.sizeof(Stats)


class GMError(RuntimeError):
    def __init__(self, fn, code, msg):
        super().__init__(f"{fn} -> {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libgm.so not built at {LIB_PATH}: run `python -m paper_2602_17601_b300.build`")
    lib = C.CDLL(LIB_PATH)
    vp, i32p = C.c_void_p, C.POINTER(C.c_int32)
    sig = {
        "gm_last_error": ([], C.c_char_p),
        "gm_version": ([], C.c_char_p),
        "gm_graph_create": ([C.c_int, C.c_int, i32p, i32p, C.c_int, i32p, C.POINTER(vp)], C.c_int),
        "gm_graph_destroy": ([vp], None),
        "gm_gnn_load": ([C.POINTER(GnnDesc), C.POINTER(C.c_float), C.c_size_t, C.POINTER(vp)], C.c_int),
        "gm_gnn_destroy": ([vp], None),
        "gm_ctx_workspace_size": ([vp, vp, C.POINTER(Settings), C.POINTER(C.c_size_t)], C.c_int),
        "gm_ctx_create": ([vp, vp, C.POINTER(Settings), vp, C.c_size_t, vp, C.POINTER(vp)], C.c_int),
        "gm_ctx_destroy": ([vp], None),
        "gm_jac_pattern": ([vp, C.POINTER(C.c_int), C.POINTER(i32p), C.POINTER(i32p)], C.c_int),
        "gm_linearize": ([vp, vp, vp, vp, vp, vp, vp, vp], C.c_int),
        "gm_condense_matrix_free": ([vp, vp, vp, C.POINTER(Cost), C.POINTER(Constr), vp, vp, vp, vp, vp, vp],
                                    C.c_int),
        "gm_condense": ([vp, vp, vp, vp, vp, C.POINTER(Cost), C.POINTER(Constr), vp, vp, vp, vp, vp],
                        C.c_int),
        "gm_qp_solve": ([vp] * 12 + [vp], C.c_int),
        "gm_qp_solve_ipm": ([vp] * 7 + [C.c_int] + [vp] * 4, C.c_int),
        "gm_rti_step": ([vp, vp, C.POINTER(Cost), C.POINTER(Constr), vp, vp, vp, vp], C.c_int),
        "gm_ctx_reset": ([vp, vp], C.c_int),
        "gm_ctx_info": ([vp, C.POINTER(Info)], C.c_int),
        "gm_ctx_set_timing": ([vp, C.c_int], C.c_int),
        "gm_ctx_phase_ms": ([vp, C.POINTER(C.c_float), C.POINTER(C.c_int)], C.c_int),
        "gm_launch_count": ([], C.c_ulonglong),
        "gm_ctx_set_graph": ([vp, C.c_int], C.c_int),
        "gm_ctx_graph_state": ([vp, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
        "gm_ctx_set_kernel_timing": ([vp, C.c_int], C.c_int),
        "gm_ws_workspace_size": ([C.c_int] * 4, C.c_size_t),
        "gm_ws_create": ([C.c_int] * 4 + [vp, C.c_size_t, C.POINTER(vp)], C.c_int),
        "gm_ws_destroy": ([vp], None),
        "gm_ws_param_count": ([vp], C.c_longlong),
        "gm_ws_set_params": ([vp, vp, vp, vp], C.c_int),
        "gm_ws_get_params": ([vp, vp, vp, vp], C.c_int),
        "gm_ws_forward": ([vp, vp, C.c_int, vp, vp], C.c_int),
        "gm_ws_train_step": ([vp, vp, vp, C.c_int] + [C.c_float] * 4 + [vp, vp], C.c_int),
        "gm_ws_grad": ([vp, vp, vp], C.c_int),
        "gm_ws_features": ([vp, vp, vp, vp, vp], C.c_int),
        "gm_batch_create": ([C.POINTER(vp), C.c_int, C.POINTER(vp)], C.c_int),
        "gm_rollout": ([vp, vp, vp, C.c_int, vp, vp], C.c_int),
        "gm_batch_destroy": ([vp], None),
        "gm_batch_rti_step": ([vp, C.POINTER(vp), vp, vp, C.POINTER(vp), C.POINTER(vp), vp], C.c_int),
        "gm_batch_state": ([vp, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
        "gm_batch_lanes": ([vp, C.POINTER(C.c_int)], C.c_int),
        "gm_ctx_set_warm": ([vp, C.c_int], C.c_int),
        "gm_ctx_set_timeout_spins": ([vp, C.c_int], C.c_int),
        "gm_measure_peaks": ([C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_longlong), vp], C.c_int),
        "gm_measure_hbm": ([vp, C.c_size_t, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                            C.POINTER(C.c_double), vp], C.c_int),
        "gm_batch_set_lanes": ([vp, C.c_int], C.c_int),
        "gm_batch_plan": ([C.c_int, vp, vp, C.c_int, vp, C.POINTER(C.c_int)], C.c_int),
        "gm_barrier_fold": ([vp, vp, vp, vp, C.c_float, C.c_float, vp, vp, vp], C.c_int),
        "gm_ctx_kernel_stats": ([vp, C.POINTER(C.c_int)] + [C.POINTER(C.c_double)] * 3, C.c_int),
        "gm_ctx_kernel_launch": ([vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int)],
                                 C.c_int),
        "gm_ctx_set_stage_timing": ([vp, C.c_int], C.c_int),
        "gm_ctx_stage_times": ([vp, vp, vp], C.c_int),
        "gm_qp_solve_noalloc": ([C.c_int, C.c_int, C.c_int, C.POINTER(Settings)] + [vp] * 10, C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()
HEADER_FUNCTIONS = ("gm_last_error", "gm_version", "gm_graph_create", "gm_graph_destroy",
                    "gm_gnn_load", "gm_gnn_destroy", "gm_ctx_workspace_size", "gm_ctx_create",
                    "gm_ctx_destroy", "gm_jac_pattern", "gm_linearize", "gm_condense", "gm_condense_matrix_free",
                    "gm_qp_solve", "gm_qp_solve_ipm", "gm_rti_step", "gm_ctx_reset", "gm_ctx_info",
                    "gm_ctx_set_timing", "gm_ctx_phase_ms", "gm_launch_count", "gm_qp_solve_noalloc",
                    "gm_ctx_set_graph", "gm_ctx_graph_state", "gm_ctx_set_kernel_timing",
                    "gm_ctx_kernel_stats", "gm_ctx_kernel_launch", "gm_ctx_set_stage_timing", "gm_ctx_stage_times",
                    "gm_ws_workspace_size", "gm_ws_create", "gm_ws_destroy",
                    "gm_ws_param_count", "gm_ws_set_params", "gm_ws_get_params", "gm_ws_forward",
                    "gm_ws_train_step", "gm_ws_grad", "gm_ws_features", "gm_batch_create",
                    "gm_batch_destroy", "gm_batch_rti_step", "gm_batch_state", "gm_batch_lanes", "gm_batch_set_lanes", "gm_batch_plan", "gm_ctx_set_warm", "gm_barrier_fold", "gm_ctx_set_timeout_spins", "gm_measure_peaks", "gm_measure_hbm",
                    "gm_rollout")

GM_NOALLOC_MAX_NU = 64
GM_NOALLOC_MAX_ROWS = 8192


def gm_qp_solve_noalloc(N, nu, Mnc, settings, H, g, Ct, dt, u_lo, u_hi, U, y=None, stats=None, stream=None):
    """ADMM solve of gm_qp_solve with no context and no device allocation (library-held scratch).

    For callers that must not allocate device memory; sizes are capped at
    N*nu <= GM_NOALLOC_MAX_NU and N*Mnc <= GM_NOALLOC_MAX_ROWS.  Calls must not
    overlap on the GPU: they share one scratch array.
    """
    _check("gm_qp_solve_noalloc",
           _lib.gm_qp_solve_noalloc(int(N), int(nu), int(Mnc), C.byref(settings), _ptr(H), _ptr(g), _ptr(Ct),
                                    _ptr(dt), _ptr(u_lo), _ptr(u_hi), _ptr(U), _ptr(y), _ptr(stats),
                                    _stream(stream)))


def gm_ctx_info(ctx):
    out = Info()
    _check("gm_ctx_info", _lib.gm_ctx_info(ctx, C.byref(out)))
    return {f: getattr(out, f) for f, _ in Info._fields_}


def gm_ctx_set_timing(ctx, on):
    _check("gm_ctx_set_timing", _lib.gm_ctx_set_timing(ctx, int(bool(on))))


def gm_ctx_phase_ms(ctx):
    """(dict phase -> summed ms, number of recorded steps); waits for the events."""
    ms = (C.c_float * 5)()
    n = C.c_int()
    _check("gm_ctx_phase_ms", _lib.gm_ctx_phase_ms(ctx, ms, C.byref(n)))
    return dict(zip(PHASES, list(ms))), n.value


def gm_launch_count():
    return int(_lib.gm_launch_count())


def gm_batch_plan(width, cost, sms):
    """Lane plan for batched instance steps (host only): (lane per instance, number of lanes)."""
    w = np.ascontiguousarray(width, np.int32)
    c = np.ascontiguousarray(cost, np.float64)
    lane = np.zeros(len(w), np.int32)
    n = C.c_int()
    _check("gm_batch_plan", _lib.gm_batch_plan(len(w), w.ctypes.data, c.ctypes.data, int(sms),
                                                lane.ctypes.data, C.byref(n)))
    return lane, n.value


def gm_ctx_set_warm(ctx, on):
    _check("gm_ctx_set_warm", _lib.gm_ctx_set_warm(ctx, int(bool(on))))


def gm_measure_peaks(stream=None):
    """Measured FP32 and FP64 FMA peaks (TFLOP/s) and the L2 size (bytes) of the current device."""
    f32, f64, l2 = C.c_double(), C.c_double(), C.c_longlong()
    _check("gm_measure_peaks", _lib.gm_measure_peaks(C.byref(f32), C.byref(f64), C.byref(l2), _stream(stream)))
    return {"fp32_tflops": f32.value, "fp64_tflops": f64.value, "l2_bytes": int(l2.value)}


def gm_measure_hbm(buf, repeats=5, stream=None):
    """HBM GB/s of read-only, write-only and copy streams over the device tensor buf (overwritten)."""
    r, w, c = C.c_double(), C.c_double(), C.c_double()
    _check("gm_measure_hbm", _lib.gm_measure_hbm(C.c_void_p(buf.data_ptr()), buf.numel() * buf.element_size(),
                                                 int(repeats), C.byref(r), C.byref(w), C.byref(c), _stream(stream)))
    return {"read_gbs": r.value, "write_gbs": w.value, "copy_gbs": c.value}


def gm_ctx_set_timeout_spins(ctx, spins):
    _check("gm_ctx_set_timeout_spins", _lib.gm_ctx_set_timeout_spins(ctx, int(spins)))


def gm_ctx_set_graph(ctx, on):
    _check("gm_ctx_set_graph", _lib.gm_ctx_set_graph(ctx, int(bool(on))))


def gm_ctx_set_kernel_timing(ctx, on):
    _check("gm_ctx_set_kernel_timing", _lib.gm_ctx_set_kernel_timing(ctx, int(bool(on))))


def gm_ctx_kernel_stats(ctx):
    """Last recorded step's reverse edge-MLP launches: dict(launches, ms, bytes, flops)."""
    n = C.c_int()
    ms, by, fl = C.c_double(), C.c_double(), C.c_double()
    _check("gm_ctx_kernel_stats", _lib.gm_ctx_kernel_stats(ctx, C.byref(n), C.byref(ms), C.byref(by), C.byref(fl)))
    return dict(launches=n.value, ms=ms.value, bytes=by.value, flops=fl.value)


def gm_ctx_kernel_launch(ctx, i):
    """Launch i of the last recorded step's reverse edge-MLP launches: dict(ms, bytes, ctas)."""
    ms, by, n = C.c_double(), C.c_double(), C.c_int()
    _check("gm_ctx_kernel_launch", _lib.gm_ctx_kernel_launch(ctx, int(i), C.byref(ms), C.byref(by), C.byref(n)))
    return dict(ms=ms.value, bytes=by.value, ctas=n.value)


def gm_ctx_set_stage_timing(ctx, on):
    _check("gm_ctx_set_stage_timing", _lib.gm_ctx_set_stage_timing(ctx, 1 if on else 0))


def gm_ctx_stage_times(ctx, N):
    """Last recorded step's stage timeline (matrix-free contexts): (roll_ms[N], tan_ms[N]),
    milliseconds from the start of the rollout to the end of each rollout and tangent stage."""
    roll = (C.c_float * N)()
    tan = (C.c_float * N)()
    _check("gm_ctx_stage_times", _lib.gm_ctx_stage_times(ctx, roll, tan))
    return list(roll), list(tan)


def gm_ctx_graph_state(ctx):
    """(1 if the last gm_rti_step replayed a CUDA graph else 0, captures so far)."""
    r, n = C.c_int(), C.c_int()
    _check("gm_ctx_graph_state", _lib.gm_ctx_graph_state(ctx, C.byref(r), C.byref(n)))
    return r.value, n.value


def lib():
    return _lib


def _check(fn, code):
    if code != GM_OK:
        raise GMError(fn, code, _lib.gm_last_error().decode())


def _ptr(t):
    """Device pointer of a torch tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def gm_last_error():
    return _lib.gm_last_error().decode()


def gm_version():
    return _lib.gm_version().decode()


def gm_graph_create(M, src, dst, nu, act_node):
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    act = np.ascontiguousarray(act_node, np.int32)
    out = C.c_void_p()
    i32p = C.POINTER(C.c_int32)
    _check("gm_graph_create",
           _lib.gm_graph_create(int(M), int(src.size), src.ctypes.data_as(i32p), dst.ctypes.data_as(i32p),
                                int(nu), act.ctypes.data_as(i32p), C.byref(out)))
    return out


def gm_graph_destroy(g):
    _lib.gm_graph_destroy(g)


def gm_gnn_load(K, W, nu, dt, blob):
    blob = np.ascontiguousarray(blob, np.float32)
    d = GnnDesc(int(K), int(W), int(nu), float(dt))
    out = C.c_void_p()
    _check("gm_gnn_load", _lib.gm_gnn_load(C.byref(d), blob.ctypes.data_as(C.POINTER(C.c_float)),
                                           blob.size, C.byref(out)))
    return out


def gm_gnn_destroy(m):
    _lib.gm_gnn_destroy(m)


def make_settings(N, n_c=0, precision=GM_PREC_FP32, rho=0.1, tol=1e-6, max_iter=4000, polish=0,
                  timeout_spins=0, scale_rows=1, adapt_rho=1, admm_grid=0, factor_grid=0, chunk_mb=0,
                  condensing=0, tan_split_rows=0):
    return Settings(int(N), int(n_c), int(precision), float(rho), float(tol), int(max_iter), int(polish),
                    int(timeout_spins), int(scale_rows), int(adapt_rho), int(admm_grid), int(factor_grid),
                    int(chunk_mb), int(condensing), int(tan_split_rows))


def gm_ctx_workspace_size(graph, gnn, settings):
    n = C.c_size_t()
    _check("gm_ctx_workspace_size", _lib.gm_ctx_workspace_size(graph, gnn, C.byref(settings), C.byref(n)))
    return n.value


def gm_ctx_create(graph, gnn, settings, workspace, stream=None):
    out = C.c_void_p()
    _check("gm_ctx_create", _lib.gm_ctx_create(graph, gnn, C.byref(settings), _ptr(workspace),
                                               workspace.numel() * workspace.element_size(),
                                               _stream(stream), C.byref(out)))
    return out


def gm_ctx_destroy(ctx):
    _lib.gm_ctx_destroy(ctx)


def gm_ctx_reset(ctx, stream=None):
    _check("gm_ctx_reset", _lib.gm_ctx_reset(ctx, _stream(stream)))


def gm_jac_pattern(ctx, M):
    """(row_ptr [M+1], col [nnzb]) of the block pattern of A_k (M = number of nodes)."""
    nnzb = C.c_int()
    rp = C.POINTER(C.c_int32)()
    col = C.POINTER(C.c_int32)()
    _check("gm_jac_pattern", _lib.gm_jac_pattern(ctx, C.byref(nnzb), C.byref(rp), C.byref(col)))
    row_ptr = np.ctypeslib.as_array(rp, shape=(M + 1,)).copy()
    return row_ptr, np.ctypeslib.as_array(col, shape=(nnzb.value,)).copy()


def gm_linearize(ctx, x0, u_hat, x_hat, A=None, B=None, c=None, stream=None):
    _check("gm_linearize", _lib.gm_linearize(ctx, _ptr(x0), _ptr(u_hat), _ptr(x_hat), _ptr(A), _ptr(B),
                                             _ptr(c), _stream(stream)))


def gm_rollout(ctx, x0, u, n_steps, x_out, stream=None):
    _check("gm_rollout", _lib.gm_rollout(ctx, _ptr(x0), _ptr(u), int(n_steps), _ptr(x_out), _stream(stream)))


def make_cost(Qdiag, Rdiag, x_ref, u_ref):
    return Cost(_ptr(Qdiag), _ptr(Rdiag), _ptr(x_ref), _ptr(u_ref))


def make_constr(u_lo, u_hi, Cx=None, dx=None, spheres=None, barrier=None):
    """barrier = (mu, delta): the state rows enter the cost as relaxed log barriers."""
    ns = 0 if spheres is None else int(spheres.shape[0])
    mu, delta = (0.0, 0.0) if barrier is None else (float(barrier[0]), float(barrier[1]))
    return Constr(_ptr(u_lo), _ptr(u_hi), _ptr(Cx), _ptr(dx), ns, _ptr(spheres), mu, delta)


def gm_barrier_fold(ctx, Ct, dt, U_hat, mu, delta, H, g, stream=None):
    _check("gm_barrier_fold", _lib.gm_barrier_fold(ctx, _ptr(Ct), _ptr(dt), _ptr(U_hat), float(mu), float(delta),
                                                   _ptr(H), _ptr(g), _stream(stream)))


def gm_condense(ctx, x_hat, A, B, c, cost, constr, H, g, Ct=None, dt=None, stream=None):
    _check("gm_condense", _lib.gm_condense(ctx, _ptr(x_hat), _ptr(A), _ptr(B), _ptr(c), C.byref(cost),
                                           C.byref(constr), _ptr(H), _ptr(g), _ptr(Ct), _ptr(dt),
                                           _stream(stream)))


def gm_condense_matrix_free(ctx, x0, u_hat, cost, constr, x_hat, H, g, Ct=None, dt=None, stream=None):
    _check("gm_condense_matrix_free", _lib.gm_condense_matrix_free(
        ctx, _ptr(x0), _ptr(u_hat), C.byref(cost), C.byref(constr), _ptr(x_hat), _ptr(H), _ptr(g), _ptr(Ct),
        _ptr(dt), _stream(stream)))


def gm_qp_solve_ipm(ctx, H, g, Ct, dt, u_lo, u_hi, U, y=None, stats=None, max_iter=60, stream=None):
    _check("gm_qp_solve_ipm", _lib.gm_qp_solve_ipm(ctx, _ptr(H), _ptr(g), _ptr(Ct), _ptr(dt), _ptr(u_lo),
                                                   _ptr(u_hi), int(max_iter), _ptr(U), _ptr(y), _ptr(stats),
                                                   _stream(stream)))


def gm_qp_solve(ctx, H, g, Ct, dt, u_lo, u_hi, U, y=None, stats=None, warm_U=None, warm_y=None,
                stream=None):
    _check("gm_qp_solve", _lib.gm_qp_solve(ctx, _ptr(H), _ptr(g), _ptr(Ct), _ptr(dt), _ptr(u_lo),
                                           _ptr(u_hi), _ptr(warm_U), _ptr(warm_y), _ptr(U), _ptr(y),
                                           _ptr(stats), _stream(stream)))


def gm_rti_step(ctx, x_meas, cost, constr, U, u0=None, stats=None, stream=None):
    _check("gm_rti_step", _lib.gm_rti_step(ctx, _ptr(x_meas), C.byref(cost), C.byref(constr), _ptr(U),
                                           _ptr(u0), _ptr(stats), _stream(stream)))


def read_stats(stats_tensor):
    """gm_stats from a device buffer of STATS_BYTES bytes (synchronises on copy)."""
    raw = stats_tensor.cpu().numpy().tobytes()
    s = Stats.from_buffer_copy(raw[:STATS_BYTES])
    return {f: getattr(s, f) for f, _ in Stats._fields_}


from .rti import RTIProblem  # noqa: E402,F401
