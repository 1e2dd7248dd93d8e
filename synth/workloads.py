"""Seeded synthetic inputs shaped like the paper's trunk workloads.

The paper's simulated trunk (Sec. VI-A) and its trained weights are not
available, so every input is drawn here from a fixed seed:

* graph: a chain of M nodes (the trunk's segments) whose edges join nodes up to
  a few positions apart, or a random local graph of bounded degree
  (Assumption 2);
* GNN weights: encode-process-decode MLPs with Gaussian entries;
* state: a hanging chain (positions along -z) plus small noise, velocities
  small noise;
* cost / bounds: position tracking (Q on positions), R on inputs, input box;
* obstacles: spheres placed beside randomly chosen nodes.

Everything is returned as float32 (int32 for indices) so that the oracle and
the CUDA path read bit-identical values; the oracle widens them to float64.

GNN weight blob format (flat float32, read independently by the oracle and by
the C library): the MLPs in the order
    node encoder  (6 + nu -> W -> W)
    edge encoder  (6      -> W -> W)
    for l in 1..K: edge update (3W -> W -> W), node update (2W -> W -> W)
    decoder       (W      -> W -> 3)
and, inside each MLP, W1 [in][hid] row-major, b1 [hid], W2 [hid][out]
row-major, b2 [out].
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np


def gnn_layer_shapes(K: int, W: int, nu: int):
    """(in, hidden, out) of every 2-layer MLP of the blob, in blob order."""
    shapes = [(6 + nu, W, W), (6, W, W)]
    for _ in range(K):
        shapes.append((3 * W, W, W))
        shapes.append((2 * W, W, W))
    shapes.append((W, W, 3))
    return shapes


def gnn_blob_size(K: int, W: int, nu: int) -> int:
    return sum(i * h + h + h * o + o for (i, h, o) in gnn_layer_shapes(K, W, nu))


def make_gnn_blob(K: int, W: int, nu: int, seed: int, scale="0.1") -> np.ndarray:
    """Gaussian weights and biases.

    scale "0.1" draws every entry from N(0, 0.1^2).  scale "fan_in:s" draws the
    entries of a matrix with fan-in n from N(0, s^2 / n) and biases from
    N(0, (0.1 s)^2).
    """
    rng = np.random.default_rng(seed)
    parts = []
    for (i, h, o) in gnn_layer_shapes(K, W, nu):
        for (rows, cols) in ((i, h), (h, o)):
            if scale.startswith("fan_in:"):
                s = float(scale.split(":")[1])
                w = rng.normal(0.0, s / np.sqrt(rows), size=(rows, cols))
                b = rng.normal(0.0, 0.1 * s, size=(cols,))
            else:
                s = float(scale)
                w = rng.normal(0.0, s, size=(rows, cols))
                b = rng.normal(0.0, s, size=(cols,))
            parts.append(w.reshape(-1))
            parts.append(b)
    blob = np.concatenate(parts).astype(np.float32)
    assert blob.size == gnn_blob_size(K, W, nu)
    return blob


def chain_edges(M: int, offsets):
    """Directed edges j -> i for every pair with |i - j| in offsets.

    Returned sorted by destination, then source.  (src, dst) int32 arrays.
    """
    src, dst = [], []
    for i in range(M):
        nbrs = []
        for o in offsets:
            if i - o >= 0:
                nbrs.append(i - o)
            if i + o < M:
                nbrs.append(i + o)
        for j in sorted(nbrs):
            src.append(j)
            dst.append(i)
    return np.asarray(src, np.int32), np.asarray(dst, np.int32)


def random_local_edges(M: int, reach: int, p: float, seed: int, directed=False,
                       max_in_degree: Optional[int] = None):
    """Random local graph: j -> i kept with probability p for 0 < |i-j| <= reach.

    Bounded in-degree (Assumption 2).  Not necessarily symmetric when
    directed=True.  Returned in a shuffled order to exercise the sorting done
    by the consumers.
    """
    rng = np.random.default_rng(seed)
    pairs = set()
    for i in range(M):
        for j in range(max(0, i - reach), min(M, i + reach + 1)):
            if j == i:
                continue
            if directed:
                if rng.random() < p:
                    pairs.add((j, i))
            elif j < i and rng.random() < p:
                pairs.add((j, i))
                pairs.add((i, j))
    pairs = sorted(pairs)
    if max_in_degree is not None:
        kept, indeg = [], np.zeros(M, int)
        for (j, i) in pairs:
            if indeg[i] < max_in_degree:
                kept.append((j, i))
                indeg[i] += 1
        pairs = kept
    order = rng.permutation(len(pairs)) if pairs else np.zeros(0, int)
    src = np.asarray([pairs[k][0] for k in order], np.int32)
    dst = np.asarray([pairs[k][1] for k in order], np.int32)
    return src, dst


@dataclass
class Workload:
    """One MPC instance: graph, GNN, horizon, cost, bounds, obstacles, solver settings."""
    name: str
    M: int
    src: np.ndarray
    dst: np.ndarray
    nu: int
    act_node: np.ndarray
    K: int
    W: int
    dt: float
    blob: np.ndarray
    N: int
    x0: np.ndarray          # [M, 6]     measured state x~(t)
    u_hat: np.ndarray       # [N, nu]    linearisation inputs (Alg. 1 starts at 0)
    Qdiag: np.ndarray       # [N+1, M, 6]
    Rdiag: np.ndarray       # [N, nu]
    x_ref: np.ndarray       # [N+1, M, 6]
    u_ref: np.ndarray       # [N, nu]
    u_lo: np.ndarray        # [N, nu]
    u_hi: np.ndarray        # [N, nu]
    spheres: np.ndarray     # [S, 4]  centre xyz, radius (S may be 0)
    rho: float = 0.1
    tol: float = 1e-6
    max_iter: int = 4000
    meta: dict = field(default_factory=dict)

    @property
    def E(self) -> int:
        return int(self.src.size)

    @property
    def nU(self) -> int:
        return self.N * self.nu


def make_workload(name, M, src, dst, nu, act_node, K, W, N, seed, *,
                  dt=0.01, w_scale="0.1", w_seed=None, spacing=None,
                  pos_noise=None, vel_noise=0.01, ref_noise=0.05,
                  q_pos=1.0, q_vel=0.0, r_u=0.01, u_bound=1.0,
                  n_spheres=0, sphere_r=0.02, sphere_clear=0.01,
                  rho=0.1, tol=1e-6, max_iter=4000) -> Workload:
    rng = np.random.default_rng(seed)
    spacing = (1.0 / M) if spacing is None else spacing
    pos_noise = 0.1 * spacing if pos_noise is None else pos_noise
    rest = np.zeros((M, 3))
    rest[:, 2] = -spacing * np.arange(M)
    x0 = np.zeros((M, 6))
    x0[:, :3] = rest + rng.normal(0.0, pos_noise, size=(M, 3))
    x0[:, 3:] = rng.normal(0.0, vel_noise, size=(M, 3))
    # reference: per-node position set-point, constant over the horizon
    pref = rest + rng.normal(0.0, ref_noise, size=(M, 3))
    x_ref = np.zeros((N + 1, M, 6))
    x_ref[:, :, :3] = pref[None]
    Qdiag = np.zeros((N + 1, M, 6))
    Qdiag[:, :, :3] = q_pos
    Qdiag[:, :, 3:] = q_vel
    Rdiag = np.full((N, nu), r_u)
    u_ref = np.zeros((N, nu))
    u_lo = np.full((N, nu), -u_bound)
    u_hi = np.full((N, nu), u_bound)
    spheres = np.zeros((n_spheres, 4))
    for s in range(n_spheres):
        n = int(rng.integers(0, M))
        phi = rng.uniform(0, 2 * np.pi)
        d = np.array([np.cos(phi), np.sin(phi), 0.0])
        spheres[s, :3] = x0[n, :3] + (sphere_r + sphere_clear) * d
        spheres[s, 3] = sphere_r
    blob = make_gnn_blob(K, W, nu, seed if w_seed is None else w_seed, w_scale)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)  # noqa: E731
    return Workload(
        name=name, M=M, src=np.ascontiguousarray(src, np.int32),
        dst=np.ascontiguousarray(dst, np.int32), nu=nu,
        act_node=np.ascontiguousarray(act_node, np.int32), K=K, W=W, dt=dt,
        blob=blob, N=N, x0=f32(x0), u_hat=f32(np.zeros((N, nu))),
        Qdiag=f32(Qdiag), Rdiag=f32(Rdiag), x_ref=f32(x_ref), u_ref=f32(u_ref),
        u_lo=f32(u_lo), u_hi=f32(u_hi), spheres=f32(spheres), rho=rho, tol=tol,
        max_iter=max_iter,
        meta=dict(seed=seed, w_scale=w_scale, spacing=spacing))


def even_actuators(M: int, nu: int) -> np.ndarray:
    """nu actuator nodes spread evenly along a chain: floor((2a+1) M / (2 nu))."""
    return np.asarray([((2 * a + 1) * M) // (2 * nu) for a in range(nu)], np.int32)


def small_chain(seed=0, **kw) -> Workload:
    """Chain of 10 nodes, edges to +-1 and +-2, K=2, W=32, nu=4 at nodes 3,5,7,9, N=10."""
    src, dst = chain_edges(10, (1, 2))
    args = dict(dt=0.01, w_scale="0.1", rho=0.1, tol=1e-6)
    args.update(kw)
    return make_workload("chain10", 10, src, dst, 4, [3, 5, 7, 9], 2, 32, 10, seed,
                         **args)


PAPER_W_SCALE = "fan_in:0.5"


def paper_chain(seed=0, M=1000, N=20, nu=8, K=3, W=128, n_spheres=5, **kw) -> Workload:
    """Trunk-like chain: M nodes, edges to +-1..+-3, K=3, W=128, nu actuators, N=20, 5 spheres."""
    src, dst = chain_edges(M, (1, 2, 3))
    args = dict(dt=0.01, w_scale=PAPER_W_SCALE, rho=0.1, tol=1e-4,
                n_spheres=n_spheres, sphere_clear=0.15)
    args.update(kw)
    return make_workload(f"chain{M}", M, src, dst, nu, even_actuators(M, nu), K, W,
                         N, seed, **args)


def random_instance(seed, M, N, nu, K=2, W=16, reach=2, p=0.7, directed=False,
                    n_spheres=0, **kw) -> Workload:
    """Irregular local graph with uneven neighbourhoods, random actuator nodes."""
    rng = np.random.default_rng(10_000 + seed)
    src, dst = random_local_edges(M, reach, p, seed, directed=directed)
    act = np.sort(rng.choice(M, size=nu, replace=nu > M)).astype(np.int32)
    args = dict(dt=0.01, w_scale="0.1", rho=0.1, tol=1e-6, n_spheres=n_spheres)
    args.update(kw)
    return make_workload(f"rand{M}", M, src, dst, nu, act, K, W, N, seed, **args)


CONFIGS = {
    "chain10": small_chain,
    "chain1000": paper_chain,
}
