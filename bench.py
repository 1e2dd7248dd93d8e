#!/usr/bin/env python
"""RTI MPC steps/s of the GNN-MPC real-time iteration on B300.

Workload (synthetic, seeded; stands in for the paper's MuJoCo trunk, Sec. VI-B
"Scalability"): chain of 1000 nodes with edges to +-1..+-3 neighbours, state 6
per node, encode-process-decode GNN with 3 message-passing steps and width-128
MLPs, 8 actuators, horizon N = 20, input box |u| <= 1, 5 sphere obstacles
linearised to half-spaces on every node and stage (100k rows), ADMM rho = 0.1
to residual 1e-4.

One step = one gm_rti_step (rollout, sensitivities, condensing, QP set-up, ADMM,
FP64 KKT check) on device-resident inputs; `e2e` adds the host->device copy of
the measured state and the device->host copy of U* each step.  The measured
states are distinct: before timing, the controller runs the closed loop
(Algorithm 1's outer loop) with the GNN itself as the plant, and timed step i
uses the loop's state i, so every step linearises, condenses and warm-starts
as in a receding-horizon run.  The same form with cold ADMM is timed on the
same states beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--form mixed|bf16|fp32] [--condensing matrix-free|jacobian] [--no-graph]
                  [--no-plain] [--workload chain1000|chain200|chain10]
  python bench.py --compare ipm       # ADMM against the interior-point solve on the step's QP
  python bench.py --compare barrier   # obstacles as QP rows against obstacles as barrier costs
  python bench.py --compare matrix-free  # cost estimate of forward-mode condensing from row counts

The comparisons print their own JSON line (not the metric line above).

The chosen form (default): matrix-free condensing (the sensitivities pushed through
the GNN by forward-mode products on their supports, the tangent pass of each stage
beside the rollout of the later stages), GNN MLPs and their tangent products on
tcgen05 tensor cores with split-BF16 operands (forward rollout three pieces,
tangents two), FP32 condensing and ADMM, FP64 Cholesky and KKT check, the whole
step replayed as a CUDA graph.  `--condensing jacobian` runs the Jacobian path
(reverse pass over cones, Thm. 1 recursion) instead.  The same run times the
plain GPU form (FP32 everywhere, eager launches, cold ADMM, Jacobian path) on the
same inputs to the same ADMM residual and reports the speedup.

Multi-GPU: one process per GPU (torchrun); every rank runs its own MPC
instance (the path does not shard inside an instance: replicas), value = all
instances' steps / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RTI MPC steps/s at 1000 nodes, N=20 (chosen vs plain GPU form, same residual)"


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--form", default="mixed", choices=["fp32", "mixed", "bf16"])
    p.add_argument("--no-graph", action="store_true", help="eager launches instead of CUDA-graph replay")
    p.add_argument("--no-warm", action="store_true", help="cold ADMM every step (no receding-horizon warm start)")
    p.add_argument("--no-plain", action="store_true", help="skip the plain FP32 comparison run")
    p.add_argument("--workload", default="chain1000", choices=["chain1000", "chain200", "chain10"],
                   help="chain200: the chain-of-1000 configuration on 200 nodes (a small case for "
                        "counter captures of the same kernels)")
    p.add_argument("--condensing", default="matrix-free", choices=["jacobian", "matrix-free"],
                   help="jacobian: local Jacobians by the reverse pass and the Thm. 1 recursion; matrix-free: "
                        "forward-mode sensitivities (gm_settings.condensing = 1)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--compare", default=None, choices=["ipm", "barrier", "matrix-free"],
                   help="ipm: gm_qp_solve against gm_qp_solve_ipm on the chain-of-1000 step's QP; barrier: "
                        "sphere rows as constraints against relaxed log barriers, spheres far and near")
    p.add_argument("--reps", type=int, default=5, help="--compare ipm: timed solves (median)")
    p.add_argument("--time-oracle-step", default=None, choices=list(FULL_STEP_WORKLOADS),
                   help=argparse.SUPPRESS)   # child process of full_oracle_steps
    p.add_argument("--mu", type=float, default=1e-3, help="--compare barrier: barrier weight")
    p.add_argument("--delta", type=float, default=5e-3, help="--compare barrier: relaxation threshold")
    return p.parse_args(argv)


def workload(name):
    from synth import paper_chain, small_chain
    if name == "chain1000":
        return paper_chain()
    if name == "chain200":
        return paper_chain(M=200)
    return small_chain()


def config_of(wl, form, extra=None):
    cfg = {"workload": f"{wl.name}_K{wl.K}_W{wl.W}_N{wl.N}_nu{wl.nu}_spheres{wl.spheres.shape[0]}",
           "M": wl.M, "E": wl.E, "N": wl.N, "nu": wl.nu, "K": wl.K, "W": wl.W,
           "n_spheres": int(wl.spheres.shape[0]), "rho": wl.rho, "tol": wl.tol, "form": form}
    if extra:
        cfg.update(extra)
    return cfg


# ------------------------------------------------------------------ clocks during the timed region
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ oracle timing (CPU)
def oracle_sample_seconds(wl, n_jac=4, m_reduced=50, seed=0):
    """Seconds of one RTI step of the FP64 oracle on wl, extrapolated from a bounded sample.

    Sample: one rollout stage (x N), n_jac local Jacobian rows (x N M / n_jac),
    condensing + ADMM on a chain of m_reduced nodes with the same horizon, inputs
    and neighbourhood radius (x M / m_reduced, linear in M by Thm. 1).
    """
    import numpy as np

    from oracle import condense as ocd
    from oracle import gnn as ogm
    from oracle import qp as oqp
    from oracle import rti as orti
    gnn, g = orti.model_of(wl)
    u = np.zeros(wl.nu)
    t0 = time.perf_counter()
    x1 = ogm.step(gnn, g, wl.x0, u)
    t_roll = (time.perf_counter() - t0) * wl.N
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    for _ in range(n_jac):
        ogm.local_jacobian_rows(gnn, g, x1, u, int(rng.integers(0, wl.M)))
    t_jac = (time.perf_counter() - t0) / n_jac * wl.M * wl.N
    # condensing + QP on a reduced chain with cfg-like random blocks
    M = m_reduced
    R = max(1, (len(g.in_ball(wl.M // 2, wl.K)) - 1) // 2)
    nbh = [list(range(max(0, i - R), min(M, i + R + 1))) for i in range(M)]
    blocks = [[(nb, rng.normal(0, 0.05, (len(nb), 6, 6)), rng.normal(0, 0.01, (6, wl.nu)),
                rng.normal(0, 0.01, 6)) for nb in nbh] for _ in range(wl.N)]
    S = wl.spheres.shape[0]
    Cx = rng.normal(0, 1, (wl.N, M, S, 3))
    Cx /= np.linalg.norm(Cx, axis=-1, keepdims=True)
    dx = np.full((wl.N, M, S), 1.0)
    t0 = time.perf_counter()
    H, gv, Ct, dt, _, _ = ocd.condense_recursive(blocks, rng.normal(0, 0.01, 6 * M),
                                                 np.ones((wl.N + 1, M * 6)), wl.Rdiag,
                                                 np.zeros((wl.N + 1, M * 6)), wl.u_ref, Cx, dx)
    oqp.admm(H, gv, wl.u_lo.reshape(-1), wl.u_hi.reshape(-1), Ct, dt, rho=wl.rho, tol=wl.tol,
             max_iter=wl.max_iter, scale_rows=True)
    t_cq = (time.perf_counter() - t0) * wl.M / M
    return t_roll + t_jac + t_cq, dict(rollout=t_roll, jacobian=t_jac, condense_qp=t_cq)


def cpu_cores():
    """Host threads the oracle's BLAS may use: the thread-count variables if set, else the cores
    this process may run on."""
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        v = os.environ.get(var, "")
        if v.isdigit() and int(v) > 0:
            return int(v)
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


SAMPLE_DESC = ("one GNN stage x N, {n_jac} sampled local Jacobian rows x N*M/{n_jac}, condensing + ADMM on a "
               "50-node chain with the same N, nu, radius and spheres x M/50; extrapolated to one step")


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


FULL_STEP_WORKLOADS = ("chain10_K2_W32_N10_nu4", "chain50_K3_W128_N20_nu8_spheres5")


def time_full_oracle_step(name, reps):
    """Seconds per full RTI step of the FP64 oracle on one of FULL_STEP_WORKLOADS (run in a child
    process, so that its BLAS thread count follows the child's environment)."""
    from oracle import rti as orti
    from synth import paper_chain, small_chain
    wl = small_chain() if name.startswith("chain10_") else paper_chain(M=50)
    t0 = time.perf_counter()
    for _ in range(reps):
        orti.rti_step(wl, solver="admm")
    return (time.perf_counter() - t0) / reps


def full_oracle_steps():
    """Measured (not extrapolated) full RTI steps of the FP64 oracle (oracle.rti.rti_step with its
    ADMM, the method's own solver): the chain of 10 (K=2, W=32, N=10) and a chain of 50 with the
    paper-scale GNN and horizon (K=3, W=128, N=20, nu=8, 5 spheres), each with all host cores and
    with one BLAS thread (a child process per leg with the thread-count variables set)."""
    out = {}
    one = {v: "1" for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for name, reps in zip(FULL_STEP_WORKLOADS, (10, 1)):
        ent = {}
        for mode, extra in (("all_cores", {}), ("one_thread", one)):
            env = dict(os.environ, **extra)
            r = subprocess.run([sys.executable, os.path.abspath(__file__), "--time-oracle-step", name,
                                "--reps", str(reps)], env=env, capture_output=True, text=True, timeout=900)
            if r.returncode != 0:
                raise RuntimeError(f"oracle step timing failed ({name}, {mode}):\n{r.stderr[-2000:]}")
            rep = json.loads(r.stdout.strip().splitlines()[-1])
            sec = rep["seconds_per_step"]
            ent[mode] = {"seconds_per_step": sec, "steps_per_s": 1.0 / sec, "steps_timed": reps,
                         "threads": rep["threads"]}
        out[name] = ent
    return out


def cpu_baseline(wl, n_jac=24):
    """The oracle on the host cores: the bench workload's step extrapolated from a bounded
    sample (its own key), and measured full steps at two smaller workloads."""
    secs, parts = oracle_sample_seconds(wl, n_jac=n_jac)
    return {"value": 1.0 / secs, "unit": "steps/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": SAMPLE_DESC.format(n_jac=n_jac),
            "value_is": f"extrapolated: {wl.name} step from the sample above",
            "extrapolated": {"workload": wl.name, "seconds_per_step": secs, "parts_s": parts},
            "measured_full_steps": full_oracle_steps(),
            "nproc": os.cpu_count(), "cpu_model": cpu_model()}


def run_reference(args):
    """The oracle as it stands on the host cores.  One reference step is one bounded sample of
    the workload's step (oracle_sample_seconds), so the run ends within minutes: ms_per_step is
    the measured wall time of a sample, and value is the full step's rate extrapolated from the
    samples (the sample's share of the full step's work is fixed)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload(args.workload)
    for _ in range(args.warmup):
        oracle_sample_seconds(wl)
    secs, walls = [], []
    t_wall = time.perf_counter()
    for s in range(args.steps):
        t0 = time.perf_counter()
        t, _ = oracle_sample_seconds(wl, seed=s)
        walls.append(time.perf_counter() - t0)
        secs.append(t)
    wall = time.perf_counter() - t_wall
    sample_ms = 1000.0 * statistics.mean(walls)
    full_ms = 1000.0 * statistics.mean(secs)
    value = 1000.0 / full_ms
    full = full_oracle_steps()
    out = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": sample_ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)", "impl": "reference",
           "config": config_of(wl, "fp64-oracle"),
           "step_is": "one bounded sample of the workload's step (ms_per_step: its measured wall time); "
                      "value: the full step's rate extrapolated from the samples",
           "extrapolated_full_step_ms": full_ms,
           "cpu_baseline": {"value": value, "unit": "steps/s", "cores": cpu_cores(), "kind": "oracle",
                            "sample": SAMPLE_DESC.format(n_jac=4), "measured_full_steps": full,
                            "nproc": os.cpu_count(), "cpu_model": cpu_model()},
           "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "wall_s": wall}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ our arm
KERNEL_TC = ("tc_ws_bwd_kernel<EdgeMpBwd> (reverse edge-update MLP, warp-specialised persistent, "
             "split-BF16 tcgen05)")
KERNEL_FP32 = "mlp2_kernel<128, EdgeMpBwd> (reverse edge-update MLP, FP32 SIMT)"
KERNEL_TAN = ("EdgeMpTan: tangent edge update of matrix-free condensing, tc_ws_bwd_kernel<EdgeMpTan> "
              "(warp-specialised persistent, projected first layer) on layers of 30k edge rows or more, "
              "tc_mlp_kernel<128, EdgeMpTanK3, 2> below; split-BF16 tcgen05")
KERNEL_TAN_FP32 = "mlp2_kernel<128, EdgeMpTan> (tangent edge-update MLP of matrix-free condensing, FP32 SIMT)"
TRAFFIC_SOURCES = ("paper_2602_17601_b300/csrc/tc_prim.cuh", "paper_2602_17601_b300/csrc/tc_mlp.cuh", "paper_2602_17601_b300/csrc/tc_ws.cuh",
                   "paper_2602_17601_b300/csrc/gnn.cu", "paper_2602_17601_b300/csrc/tangent.cuh")


def sources_sha256():
    h = hashlib.sha256()
    for rel in TRAFFIC_SOURCES:
        h.update(open(os.path.join(ROOT, rel), "rb").read())
    return h.hexdigest()


def kernel_traffic(form):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, if the
    kernel sources are unchanged since it was taken (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        ent = json.load(open(path)).get(form)
        if not ent or ent.get("sources_sha256") != sources_sha256():
            return None
        return ent["dram_bytes_per_launch"]
    except Exception:
        return None


def timed_steps(torch, prob, X, U, first, steps, stream):
    """Device time per step of `steps` RTI steps at the measured states X[first + i]."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(steps):
        prob.step(X[first + i], U)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def closed_loop_states(prob, wl, n):
    """Measured states of an n-step closed loop (Algorithm 1's outer loop): this problem's
    controller drives the GNN itself as the plant from wl.x0 (gm_rollout applies u_0).
    Returns the states [n][M*6] on the device and the per-step solve statistics."""
    import torch

    from paper_2602_17601_b300 import closed_loop
    S, _, stats = closed_loop.run(prob, wl.x0, n)
    X = torch.as_tensor(S[:n].reshape(n, -1), dtype=torch.float32, device="cuda").contiguous()
    return X, stats


def mean_iters(stats):
    return float(statistics.mean(s["iters"] for s in stats)) if stats else None


def run_ours(args):
    import torch

    import paper_2602_17601_b300 as gm
    from paper_2602_17601_b300.replicas import Replicas
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    reps = Replicas("nccl", device="cuda")
    world = reps.world
    wl = workload(args.workload)
    precs = {"fp32": gm.GM_PREC_FP32, "mixed": gm.GM_PREC_MIXED, "bf16": gm.GM_PREC_BF16}
    graph = not args.no_graph
    warm = not args.no_warm
    cond = 1 if args.condensing == "matrix-free" else 0
    prob = gm.RTIProblem.from_workload(wl, precision=precs[args.form], graph=graph, warm=warm, condensing=cond)
    stream = torch.cuda.current_stream()
    U = prob.empty(prob.nU)
    warmup = max(args.warmup, 3)
    n_states = warmup + args.steps
    barrier = reps.barrier
    max_over_ranks = reps.max_over_ranks

    # ---- one eager step counts the kernels of a step (a fresh context's first step is eager)
    l0 = gm.gm_launch_count()
    prob.step(wl.x0, U)
    torch.cuda.synchronize()
    kernels_per_step = gm.gm_launch_count() - l0

    # ---- distinct measured states: the closed loop of this controller with the GNN as the plant,
    # run once before timing; the timed steps then step through the same states in order, so each
    # step's linearisation point, QP and warm start are those of a receding-horizon run
    X, loop_stats = closed_loop_states(prob, wl, n_states)
    timed_stats = loop_stats[warmup:]

    # ---- the chosen form on device-resident states (graph replay from the second step on)
    prob.reset()
    for i in range(warmup):
        prob.step(X[i], U)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    ms = timed_steps(torch, prob, X, U, warmup, args.steps, stream)
    barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    replayed, captures = prob.graph_state()
    st = prob.read_stats()
    ms = max_over_ranks(ms)

    # ---- end to end through the public API: each step's state from pinned host memory in, U* out
    X_host = X.cpu().pin_memory()
    x_dev = torch.empty_like(X[0])
    U_host = torch.empty(prob.nU, dtype=torch.float32).pin_memory()
    prob.reset()
    for i in range(warmup):
        x_dev.copy_(X_host[i], non_blocking=True)
        prob.step(x_dev, U)
        U_host.copy_(U, non_blocking=True)
    torch.cuda.synchronize()
    barrier()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for i in range(warmup, n_states):
        x_dev.copy_(X_host[i], non_blocking=True)
        prob.step(x_dev, U)
        U_host.copy_(U, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e2.elapsed_time(e3) / args.steps)

    # ---- the dominant kernel's launches: the same timed steps again with an event pair around each
    # of its launches (kept out of the headline pass, whose step the event records would lengthen);
    # every step's launches are read back after the step
    gm.gm_ctx_set_kernel_timing(prob.ctx, True)
    prob.reset()
    for i in range(warmup):
        prob.step(X[i], U)
    klaunch = []                                            # per step: its timed launches
    kst = {"launches": 0, "ms": 0.0, "bytes": 0.0, "flops": 0.0}
    for i in range(warmup, n_states):
        prob.step(X[i], U)
        s_ = gm.gm_ctx_kernel_stats(prob.ctx)
        klaunch.append([gm.gm_ctx_kernel_launch(prob.ctx, j) for j in range(s_["launches"])])
        for key in kst:
            kst[key] += s_[key]
    k_steps = max(n_states - warmup, 1)
    kst = {key: v / k_steps for key, v in kst.items()}      # per step
    gm.gm_ctx_set_kernel_timing(prob.ctx, False)

    # ---- stage timeline of the overlapped rollout and tangent pass (matrix-free): when each
    # rollout stage and each tangent stage ends, from where both start, mean over the same states
    timeline = None
    if cond:
        gm.gm_ctx_set_stage_timing(prob.ctx, True)
        prob.reset()
        for i in range(warmup):
            prob.step(X[i], U)
        acc_r, acc_t = [0.0] * wl.N, [0.0] * wl.N
        for i in range(warmup, n_states):
            prob.step(X[i], U)
            r_, t_ = gm.gm_ctx_stage_times(prob.ctx, wl.N)
            acc_r = [a + b for a, b in zip(acc_r, r_)]
            acc_t = [a + b for a, b in zip(acc_t, t_)]
        gm.gm_ctx_set_stage_timing(prob.ctx, False)
        timeline = {"rollout_stage_end_ms": [round(v / k_steps, 4) for v in acc_r],
                    "tangent_stage_end_ms": [round(v / k_steps, 4) for v in acc_t]}

    # ---- per-phase breakdown (events at phase boundaries force eager steps: not timed above)
    gm.gm_ctx_set_timing(prob.ctx, True)
    gm.gm_ctx_phase_ms(prob.ctx)
    prob.reset()
    for i in range(warmup):
        prob.step(X[i], U)
    gm.gm_ctx_phase_ms(prob.ctx)
    for i in range(warmup, min(warmup + 3, n_states)):
        prob.step(X[i], U)
    phases, nrec = gm.gm_ctx_phase_ms(prob.ctx)
    gm.gm_ctx_set_timing(prob.ctx, False)
    per_phase = {("sensitivities" if cond and k == "jacobian" else k): v / max(nrec, 1) for k, v in phases.items()}

    # ---- the same form with cold ADMM every step, on the same states
    cold = None
    if warm:
        del prob
        torch.cuda.empty_cache()
        pc = gm.RTIProblem.from_workload(wl, precision=precs[args.form], graph=graph, warm=False, condensing=cond)
        pc.reset()
        for i in range(warmup):
            pc.step(X[i], U)
        torch.cuda.synchronize()
        barrier()
        ms_c = max_over_ranks(timed_steps(torch, pc, X, U, warmup, args.steps, stream))
        cstats = []
        for i in range(warmup, n_states):              # untimed pass: iterations of each step
            pc.step(X[i], U)
            cstats.append(pc.read_stats())
        cold = {"form": "same form, cold ADMM every step", "value": reps.steps_per_s(ms_c), "unit": "steps/s",
                "ms_per_step": ms_c, "admm_iters_mean": mean_iters(cstats),
                "statuses": sorted({s["status"] for s in cstats})}
        del pc
    else:
        del prob

    # ---- the plain GPU form: FP32 everywhere, eager launches, cold ADMM, same states and residual
    plain = None
    if not args.no_plain and args.form != "fp32":
        torch.cuda.empty_cache()
        pp = gm.RTIProblem.from_workload(wl, precision=gm.GM_PREC_FP32, graph=False)
        pp.reset()
        for i in range(warmup):
            pp.step(X[i], U)
        torch.cuda.synchronize()
        barrier()
        ms_p = max_over_ranks(timed_steps(torch, pp, X, U, warmup, args.steps, stream))
        sp = pp.read_stats()
        plain = {"form": "fp32, eager launches, cold ADMM, local Jacobians and the Thm. 1 recursion",
                 "value": reps.steps_per_s(ms_p), "unit": "steps/s",
                 "ms_per_step": ms_p, "admm_iters_last_step": sp["iters"], "kkt_stat_last_step": sp["kkt_stat"],
                 "r_dual_last_step": sp["r_dual"], "status_last_step": sp["status"]}
        del pp

    if not reps.leader:
        reps.close()
        return

    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    hbm_peak = peaks.get("hbm_gbs")
    peak_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if hbm_peak else "fallback 6400 GB/s"
    hbm_peak = hbm_peak or 6400.0
    k_ms = kst["ms"]
    achieved = kst["bytes"] / (k_ms * 1e-3) / 1e9 if k_ms > 0 else 0.0
    products = {"mixed": 3, "bf16": 1, "fp32": 1}[args.form]
    if cond:
        kname = KERNEL_TAN_FP32 if args.form == "fp32" else KERNEL_TAN.replace(", 2>", ", 1>" if args.form == "bf16" else ", 2>")
    else:
        kname = KERNEL_FP32 if args.form == "fp32" else KERNEL_TC.replace(", 2>", ", 1>" if args.form == "bf16" else ", 2>")
    roof = {"kernel": kname,
            "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak, "peak_source": peak_src,
            "traffic": kernel_traffic(args.form + ("-matrix-free" if cond else "")),
            "launches_per_step": kst["launches"], "ms_per_step": k_ms,
            "algorithmic_bytes_per_launch": kst["bytes"] / max(kst["launches"], 1),
            "avg_launch_ms": k_ms / max(kst["launches"], 1),
            "tensor_tflops": kst["flops"] * products / (k_ms * 1e-3) / 1e12 if k_ms > 0 else 0.0,
            "tensor_peak_tflops": peaks.get("bf16_tflops_sustained"),
            "share_of_step": k_ms / ms,
            "phase_ms": per_phase}
    if timeline is not None:
        roof["stage_timeline"] = timeline
    # the launches that had the whole GPU (after the rollout): the kernel's own rate; the earlier
    # launches share the SMs and HBM with the rollout of later stages.  Jacobian path: the last
    # chunk's (the launches with every SM); matrix-free: the last stage's K launches
    full, rest = [], []
    for step_l in klaunch:
        if not step_l:
            continue
        if cond:
            f_ = step_l[-wl.K:] if len(step_l) > wl.K else []
        else:
            top = max(x["ctas"] for x in step_l)
            f_ = [L for L in step_l if L["ctas"] >= top]
        full += f_
        rest += step_l[:len(step_l) - len(f_)] if cond else [L for L in step_l if L not in f_]
    f_ms, f_by = sum(L["ms"] for L in full), sum(L["bytes"] for L in full)
    if f_ms > 0 and rest:
        roof["beside_rollout"] = {"launches_per_step": len(rest) / k_steps,
                                  "ctas": [min(L["ctas"] for L in rest), max(L["ctas"] for L in rest)]}
        roof["alone"] = {"launches_per_step": len(full) / k_steps, "ctas": max(L["ctas"] for L in full),
                         "ms_per_step": f_ms / k_steps,
                         "achieved": f_by / (f_ms * 1e-3) / 1e9, "frac": f_by / (f_ms * 1e-3) / 1e9 / hbm_peak}
    out = {"metric": METRIC, "value": reps.steps_per_s(ms), "unit": "steps/s", "n_gpus": world,
           "steps": args.steps, "warmup": warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": {"fp32": "f32", "mixed": "bf16x3/f32", "bf16": "bf16/f32"}[args.form] + " (f64 Cholesky, KKT)",
           "data": "synthetic (seeded)",
           "config": config_of(wl, args.form, {
               "condensing": args.condensing,
               "graph_replay": bool(replayed), "graph_captures": captures,
               "admm_warm_start": "shifted previous U*, y* (receding horizon)" if warm else "cold",
               "states": f"closed-loop trajectory: {n_states} distinct measured states, the GNN as the plant "
                         "driven by this controller (computed before timing; timed step i uses state i)",
               "parallelism": f"replicas{world}",
               "l2": ("inputs larger than L2: the step streams ~9 GB of tangent rows" if cond else
                      "inputs larger than L2: the step streams ~2 GB of Jacobian/condensing buffers"),
               "admm_iters_mean": mean_iters(timed_stats),
               "admm_iters_per_step": [s["iters"] for s in timed_stats],
               "admm_iters_source": "the closed-loop pass that produced the states (same states, same warm starts)",
               "statuses": sorted({s["status"] for s in timed_stats}),
               "admm_iters_last_step": st["iters"], "kkt_stat_last_step": st["kkt_stat"],
               "r_dual_last_step": st["r_dual"], "status_last_step": st["status"]}),
           "clocks": clocks,
           "e2e": {"value": reps.steps_per_s(ms_e2e), "unit": "steps/s",
                   "h2d_bytes_per_step": int(wl.x0.nbytes), "d2h_bytes_per_step": int(prob_nU(wl) * 4)},
           "gpu_launches": int(kernels_per_step * args.steps),
           "roofline": roof,
           "context": "paper: 100 Hz closed loop up to 1000 nodes, N=20 on RTX 4090 + Ryzen 9 7950X3D "
                      "with its own (unstated-size) trunk GNN; not this workload"}
    if cold is not None:
        out["cold_admm_form"] = cold
    if plain is not None:
        out["plain_gpu_form"] = plain
        out["speedup_vs_plain"] = plain["ms_per_step"] / ms
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl)
    print(json.dumps(out), flush=True)
    reps.close()


def prob_nU(wl):
    return wl.N * wl.nu


def compare_ipm(args):
    """ADMM (gm_qp_solve, adaptive rho) against the interior-point method (gm_qp_solve_ipm,
    Mehrotra predictor-corrector) on the condensed QP of the chain of 1000 nodes at the first
    step's point (u_hat = 0), mixed form, both to the workload's tolerance.  Device ms from CUDA
    events around each call (the IPM's host reads of its done flag included), median of reps
    after one warm-up."""
    import numpy as np
    import torch

    import paper_2602_17601_b300 as gm
    wl = workload("chain1000")
    prob = gm.RTIProblem.from_workload(wl, precision=gm.GM_PREC_MIXED)
    x_hat, A, B, c = prob.linearize(wl.x0, np.zeros((wl.N, wl.nu), np.float32))
    H, g, Ct, dt = prob.condense(x_hat, A, B, c)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        out, ms = None, []
        for _ in range(args.reps + 1):
            torch.cuda.synchronize()
            ev[0].record()
            out = fn()
            ev[1].record()
            torch.cuda.synchronize()
            ms.append(ev[0].elapsed_time(ev[1]))
        return out, float(np.median(ms[1:])), prob.read_stats()

    (Ua, _), ms_a, st_a = timed(lambda: prob.qp_solve(H, g, Ct, dt))
    (Ui, _), ms_i, st_i = timed(lambda: prob.qp_solve_ipm(H, g, Ct, dt, max_iter=80))
    keep = ("status", "iters", "converged", "r_prim", "r_dual", "kkt_stat", "kkt_prim", "kkt_dual", "kkt_comp")
    print(json.dumps({"compare": "ipm", "workload": "chain1000_K3_W128_N20_nu8_spheres5", "n": int(prob.nU),
                      "rows": int(prob.rows_c), "tol": wl.tol, "reps": args.reps,
                      "admm": {"ms": ms_a, **{k: st_a[k] for k in keep}},
                      "ipm": {"ms": ms_i, **{k: st_i[k] for k in keep}},
                      "max_abs_U_diff": float((Ua - Ui).abs().max()), "max_abs_U": float(Ua.abs().max()),
                      "device": torch.cuda.get_device_name()}), flush=True)


def compare_barrier(args):
    """The chain of 1000 nodes with its 5 spheres (radius 0.02) 0.15 ("far", the benchmark
    workload) and 0.01 ("near") from their nodes at the initial state, each stepped from that
    state (the step's own solution shifted into the next linearisation point), mixed form, graph
    replay: sphere rows as QP constraints against relaxed log barriers in the cost (gm_constr
    barrier_mu / barrier_delta).  Device ms per step (CUDA events over args.steps steps after
    args.warmup), the last step's ADMM iterations and status, and the smallest sphere clearance
    of the GNN rollout under the returned inputs."""
    import numpy as np
    import torch

    import paper_2602_17601_b300 as gm
    from synth import paper_chain

    def run(wl, barrier):
        sph = wl.spheres.astype(np.float64)
        prob = gm.RTIProblem.from_workload(wl, precision=gm.GM_PREC_MIXED, graph=True, barrier=barrier)
        x = torch.as_tensor(wl.x0.reshape(-1), dtype=torch.float32, device="cuda")
        U = prob.empty(prob.nU)
        for _ in range(args.warmup):
            prob.step(x, U)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record()
        for _ in range(args.steps):
            prob.step(x, U)
        ev[1].record()
        torch.cuda.synchronize()
        st = prob.read_stats()
        xs = prob.empty(wl.N + 1, wl.M, 6)
        gm.gm_rollout(prob.ctx, x, U, wl.N, xs)
        p = xs.cpu().numpy().astype(np.float64)[1:, :, :3]
        clear = np.linalg.norm(p[:, :, None, :] - sph[None, None, :, :3], axis=-1) - sph[None, None, :, 3]
        out = {"ms_per_step": ev[0].elapsed_time(ev[1]) / args.steps, "admm_iters": st["iters"],
               "status": st["status"], "converged": st["converged"], "min_clearance": float(clear.min()),
               "max_abs_U": float(U.abs().max())}
        prob.close()
        return out

    rep = {"compare": "barrier", "workload": "chain1000_K3_W128_N20_nu8_spheres5", "form": "mixed, graph replay",
           "steps": args.steps, "warmup": args.warmup, "mu": args.mu, "delta": args.delta}
    for name, clear in (("far", 0.15), ("near", 0.01)):
        wl = paper_chain(sphere_clear=clear)
        rep[name] = {"sphere_clearance_at_x0": clear, "constraints": run(wl, None),
                     "barrier": run(wl, (args.mu, args.delta))}
    rep["device"] = torch.cuda.get_device_name()
    print(json.dumps(rep), flush=True)


def tangent_row_counts(wl):
    """MLP rows of a forward-mode (matrix-free) condensing pass restricted to non-zero tangents:
    for every stage k, input column (i <= k, a) and layer l = 0..K, the nodes within
    K (k - i) + l hops of actuator a along the edges and the edges with an endpoint among them."""
    import collections

    import numpy as np
    out = collections.defaultdict(list)
    for s_, d_ in zip(wl.src, wl.dst):
        out[int(s_)].append(int(d_))
    src, dst = np.asarray(wl.src), np.asarray(wl.dst)
    nodes = edges = 0
    for a in range(wl.nu):
        hop = np.full(wl.M, 1 << 30)
        hop[int(wl.act_node[a])] = 0
        q = collections.deque([int(wl.act_node[a])])
        while q:
            v = q.popleft()
            for w in out[v]:
                if hop[w] > hop[v] + 1:
                    hop[w] = hop[v] + 1
                    q.append(w)
        for k in range(wl.N):
            for i in range(k + 1):
                for layer in range(wl.K + 1):
                    r = wl.K * (k - i) + layer
                    nodes += int((hop <= r).sum())
                    edges += int(((hop[src] <= r) | (hop[dst] <= r)).sum())
    return nodes, edges


def reverse_row_counts(wl):
    """MLP rows of the reverse pass over cones: 3 channels x N stages x (the (seed, node) pairs
    within r hops upstream for r = 0..K, and the edges into the nodes of levels 0..K-1)."""
    import collections

    import numpy as np
    inn = collections.defaultdict(list)
    for s_, d_ in zip(wl.src, wl.dst):
        inn[int(d_)].append(int(s_))
    indeg = np.bincount(np.asarray(wl.dst), minlength=wl.M)
    nodes = edges = 0
    for s0 in range(wl.M):
        hop = {s0: 0}
        q = collections.deque([s0])
        while q:
            v = q.popleft()
            if hop[v] == wl.K:
                continue
            for w in inn[v]:
                if w not in hop:
                    hop[w] = hop[v] + 1
                    q.append(w)
        h = np.array(list(hop.values()))
        deg = np.array([indeg[n] for n in hop])
        for r in range(wl.K + 1):
            nodes += int((h <= r).sum())
            if r < wl.K:
                edges += int(deg[h <= r].sum())
    return 3 * wl.N * nodes, 3 * wl.N * edges


def compare_matrix_free(args):
    """Cost of matrix-free condensing (sensitivities S_k pushed through the GNN by forward-mode
    products, no A_k) on the chain of 1000, from measurements of this library's kernels: the
    tangent rows it evaluates (graph counting) times the per-row time of the forward MLP kernels
    at full occupancy (the rollout of a 16000-node chain with the same GNN, CUDA events), beside
    the measured rollout, reverse pass and condensing of the chosen form (phase timing).  A
    tangent row is a forward MLP row without bias and ReLU evaluation (the masks are the
    rollout's), so the forward kernels' per-row time is its cost."""
    import numpy as np
    import torch

    import paper_2602_17601_b300 as gm
    from synth import paper_chain
    wl = workload("chain1000")
    t_nodes, t_edges = tangent_row_counts(wl)
    big = paper_chain(M=16000, n_spheres=0)
    pb = gm.RTIProblem.from_workload(big, precision=gm.GM_PREC_MIXED)
    x0 = torch.as_tensor(big.x0.reshape(-1), dtype=torch.float32, device="cuda")
    U = torch.zeros(big.N, big.nu, dtype=torch.float32, device="cuda")
    xs = torch.empty(big.N + 1, big.M, 6, dtype=torch.float32, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for _ in range(3):
        gm.gm_rollout(pb.ctx, x0, U, big.N, xs)
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(args.reps):
        gm.gm_rollout(pb.ctx, x0, U, big.N, xs)
    ev[1].record()
    torch.cuda.synchronize()
    ms_big = ev[0].elapsed_time(ev[1]) / args.reps
    E_big = len(big.src)
    f_nodes = big.N * big.M * (big.K + 2)           # node encoder, K node updates, decoder
    f_edges = big.N * E_big * (big.K + 1)           # edge encoder, K edge updates
    us_per_row = ms_big * 1e3 / (f_nodes + f_edges)
    pb.close()
    del pb
    torch.cuda.empty_cache()
    prob = gm.RTIProblem.from_workload(wl, precision=gm.GM_PREC_MIXED)
    gm.gm_ctx_set_timing(prob.ctx, 1)
    x = torch.as_tensor(wl.x0.reshape(-1), dtype=torch.float32, device="cuda")
    for _ in range(3):
        prob.step(x)
    torch.cuda.synchronize()
    phase, n = gm.gm_ctx_phase_ms(prob.ctx)
    r_nodes, r_edges = reverse_row_counts(wl)
    est = us_per_row * (t_nodes + t_edges) / 1e3
    print(json.dumps({
        "compare": "matrix-free", "workload": "chain1000_K3_W128_N20_nu8",
        "tangent_rows": {"node": t_nodes, "edge": t_edges},
        "reverse_rows": {"node": r_nodes, "edge": r_edges},
        "forward_kernels_at_full_occupancy": {"workload": "chain16000_K3_W128_N20_nu8 rollout", "ms": ms_big,
                                              "mlp_rows": f_nodes + f_edges, "us_per_row": us_per_row},
        "tangent_pass_ms_estimate": est,
        "chosen_form_phase_ms": {k: v / max(n, 1) for k, v in phase.items()},
        "device": torch.cuda.get_device_name()}), flush=True)


def main():
    args = parse()
    if args.time_oracle_step:
        print(json.dumps({"seconds_per_step": time_full_oracle_step(args.time_oracle_step, args.reps),
                          "threads": cpu_cores()}), flush=True)
    elif args.compare == "ipm":
        compare_ipm(args)
    elif args.compare == "barrier":
        compare_barrier(args)
    elif args.compare == "matrix-free":
        compare_matrix_free(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
