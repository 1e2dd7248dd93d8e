"""The chosen (split-BF16 tensor-core) form against the FP64 oracle at the benchmarked
configuration: chain of 1000 nodes, K = 3, W = 128, N = 20, nu = 8, 5 spheres (100k
half-space rows).  Needs a GPU.

* Jacobian rows (Eq. linearized_dynamics): 48 seeded (stage, node) pairs; the oracle
  differentiates node i's dynamics on its K-hop subgraph at the device's linearisation point
  x_hat[k] (widened to FP64), so the comparison isolates the Jacobian phase.  A ReLU network's
  Jacobian jumps where a pre-activation crosses zero, and at this size nearly every node's
  cone holds a few of its ~30k units within 1e-5 of zero.  The forward pass evaluates the
  pre-activations at FP32 operand precision (about 1e-7 of their terms), so a unit whose
  margin exceeds KINK = 1e-6 has the oracle's mask; a row is compared when every unit of its
  cone does, and the test prints how many rows that excluded (at most a third may be).
* H, g and U (Eq. H, Eq. g, Eq. condensed_matrices) against an FP64 reference: the oracle's
  FP64 rollout, the FP32 form's Jacobian blocks (pinned to the oracle element by element),
  c recomputed in FP64 on that rollout, the oracle's FP64 condensing, and the exact optimum
  of that QP (FP64 IPM + active set).  H - Rbar within 1e-4 of its max-abs; g, a sum over
  20k node-stages that inherits the rows' one-sided derivatives at near-kink units, within
  G_TOL = 2e-3 (both forms' errors are printed).  U of a cold
  step at ADMM tolerance 1e-7: within U_KINK = 2e-3 of max|U*| against the FP64 reference (the
  kink margins above let FP32-precision and FP64 evaluations take different one-sided
  derivatives on some units), and within the ADMM's own bound (twice the FP64 stationarity
  residual over the smallest eigenvalue of H) plus 1e-4 of max|U*| against the exact
  optimum of the QP the step solved.
* U of the fourth step of a warm-started, graph-replayed closed loop at the bench tolerance
  (1e-4) against the exact optimum of the QP that step solved, within the same bound.
"""
from collections import deque

import numpy as np
import pytest

from gpu_helpers import REL, max_rel_err, ocd, ogm, oqp, orti, packed_to_dense_ct
from synth import paper_chain

pytestmark = pytest.mark.gpu

REL_MIXED = 1e-4
KINK = 1e-6
G_TOL = 2e-3
U_KINK = 2e-3
GM_PREC_MIXED = 1


def _dist_to(g, i, K):
    """Hop distance from every node that reaches node i in at most K edges."""
    preds = {}
    for j, t in zip(g.src, g.dst):
        preds.setdefault(int(t), []).append(int(j))
    dist = {int(i): 0}
    q = deque([int(i)])
    while q:
        n = q.popleft()
        if dist[n] == K:
            continue
        for j in preds.get(n, []):
            if j not in dist:
                dist[j] = dist[n] + 1
                q.append(j)
    return dist


def cone_kink_margin(gnn, g, x, u, i):
    """Smallest |pre-activation| over the ReLU units f^i depends on: node i's K-hop subgraph
    evaluated in FP64, restricted to the units in i's cone (node units of nodes within
    K - 1 - t hops at message-passing step t, edge units of edges into them, the encoders
    of the ball and the edges into the (K - 1)-ball, the decoder at i)."""
    K = gnn.K
    dist = _dist_to(g, i, K)
    ball = sorted(dist)
    loc = {n: b for b, n in enumerate(ball)}
    keep = [k for k in range(g.E) if int(g.src[k]) in loc and int(g.dst[k]) in loc]
    src = np.array([loc[int(g.src[k])] for k in keep], dtype=np.int64)
    dst = np.array([loc[int(g.dst[k])] for k in keep], dtype=np.int64)
    dnode = np.array([dist[n] for n in ball])
    dedge = dnode[dst]
    xs = np.asarray(x, np.float64)[ball]
    m = np.zeros((len(ball), g.nu))
    for a, n in enumerate(g.act_node):
        if int(n) in loc:
            m[loc[int(n)], a] = 1.0
    worst = np.inf

    def mlp(p, z, rows):
        nonlocal worst
        W1, b1, W2, b2 = p
        a = z @ W1 + b1
        if rows.any():
            worst = min(worst, float(np.abs(a[rows]).min()))
        return np.maximum(a, 0.0) @ W2 + b2

    h = mlp(gnn.node_enc, np.concatenate([xs, m * np.asarray(u, np.float64)[None]], 1), dnode <= K)
    e = mlp(gnn.edge_enc, xs[dst] - xs[src], dedge <= K - 1)
    for t in range(K):
        e = e + mlp(gnn.edge_mp[t], np.concatenate([h[dst], h[src], e], 1), dedge <= K - 1 - t)
        agg = np.zeros_like(h)
        np.add.at(agg, dst, e)
        h = h + mlp(gnn.node_mp[t], np.concatenate([h, agg], 1), dnode <= K - 1 - t)
    mlp(gnn.dec, h, dnode == 0)
    return worst


def _learned_scale(Ablk, ball, i, dt):
    """Max-abs of the learned part of node i's Jacobian rows (the Euler identity removed)."""
    V = Ablk.copy()
    b = ball.index(i)
    V[b, 0:3, 0:3] -= np.eye(3)
    V[b, 0:3, 3:6] -= dt * np.eye(3)
    V[b, 3:6, 3:6] -= np.eye(3)
    return max(np.abs(V).max(), 1e-6)


def test_mixed_jacobian_rows_at_paper_scale(lib):
    wl = paper_chain()
    prob = lib.RTIProblem.from_workload(wl, precision=GM_PREC_MIXED)
    u_hat = (np.random.default_rng(7).uniform(-0.5, 0.5, (wl.N, wl.nu)) * 0.2).astype(np.float32)
    x_hat, A, B, c = (t.cpu().numpy().astype(np.float64) for t in prob.linearize(wl.x0, u_hat))
    gnn, gr = orti.model_of(wl)
    xo = ogm.rollout(gnn, gr, wl.x0, u_hat.astype(np.float64))
    ex = max_rel_err(x_hat, xo)
    print(f"mixed form, chain of 1000: x_hat rel err {ex:.2e}")
    assert ex <= REL
    rng = np.random.default_rng(11)
    pairs = [(0, 0), (0, 999), (19, 500), (10, int(wl.act_node[3]))]
    pairs += [(int(rng.integers(0, wl.N)), int(rng.integers(0, wl.M))) for _ in range(44)]
    errs, excluded = [], []
    for k, i in pairs:
        xk, uk = x_hat[k].reshape(wl.M, 6), u_hat[k].astype(np.float64)
        margin = cone_kink_margin(gnn, gr, xk, uk, i)
        if margin < KINK:
            excluded.append((k, i, margin))
            continue
        ball, Ablk, Bi, fi = ogm.local_jacobian_rows(gnn, gr, xk, uk, i)
        q0, q1 = prob.row_ptr[i], prob.row_ptr[i + 1]
        assert list(prob.col[q0:q1]) == ball
        ea = max_rel_err(A[k, q0:q1], Ablk, scale=_learned_scale(Ablk, ball, i, wl.dt))
        eb = max_rel_err(B[k, i], Bi, scale=max(np.abs(Bi).max(), 1e-6))
        # c^i_k = f^i - sum_j A^{ij} x^j - B^i u: against its largest term
        ax = np.einsum("bst,bt->s", Ablk, xk[ball])
        co = fi - ax - Bi @ uk
        terms = max(np.abs(fi).max(), np.abs(ax).max(), np.abs(Bi @ uk).max())
        ec = max_rel_err(c[k, i], co, scale=terms)
        errs.append((k, i, ea, eb, ec))
    print(f"mixed form, chain of 1000: {len(errs)} rows compared, {len(excluded)} excluded "
          f"(cone kink margin < {KINK:g}: {[(k, i, f'{m:.1e}') for k, i, m in excluded]}); "
          f"max errors A {max(e[2] for e in errs):.2e}, B {max(e[3] for e in errs):.2e}, "
          f"c {max(e[4] for e in errs):.2e}")
    assert len(excluded) <= len(pairs) // 3, excluded
    for k, i, ea, eb, ec in errs:
        assert ea <= REL_MIXED and eb <= REL_MIXED and ec <= REL_MIXED, (k, i, ea, eb, ec)


def _exact_u(wl, n_c, H, g, Ct, dt):
    Hd, gd, Cd, dd = (np.asarray(a.cpu().numpy(), np.float64) for a in (H, g, Ct, dt))
    C = packed_to_dense_ct(Cd, wl.N, wl.M, n_c, wl.nu)
    U, _, _ = oqp.solve_exact(Hd, gd, wl.u_lo.reshape(-1).astype(np.float64),
                              wl.u_hi.reshape(-1).astype(np.float64), C, dd)
    return U, np.linalg.eigvalsh(Hd).min()


def _check_u(tag, U, st, Ue, lam):
    bound = 2 * max(st["r_dual"], st["kkt_stat"]) / lam
    scale = np.abs(Ue).max()
    err = np.abs(U - Ue).max()
    print(f"mixed form, chain of 1000, {tag}: |U - U*| = {err:.2e} (max|U*| {scale:.2e}, relative "
          f"{err / scale:.2e}; ADMM bound {bound:.2e}), ADMM iterations {st['iters']}, status {st['status']}")
    assert err <= bound + REL_MIXED * scale, (err, bound, scale)


def _fp64_reference(lib, wl, x0, zeros):
    """H, g and U* in FP64 at (x0, u_hat = 0): the oracle's FP64 rollout, the FP32 form's
    Jacobian blocks (pinned to the oracle element by element), c = x_hat_{k+1} - A x_hat_k in
    FP64 on the oracle's rollout, the oracle's FP64 condensing and its exact QP optimum.
    Also returns the FP32 form's own H and g."""
    p32 = lib.RTIProblem.from_workload(wl)
    _, A, B, _ = (t.cpu().numpy().astype(np.float64) for t in p32.linearize(x0, zeros))
    gnn, gr = orti.model_of(wl)
    M, N = wl.M, wl.N
    xo = ogm.rollout(gnn, gr, wl.x0, np.zeros((N, wl.nu))).reshape(N + 1, M, 6)
    rp, col = p32.row_ptr, p32.col
    blocks = []
    for k in range(N):
        per = []
        for i in range(M):
            nb = list(col[rp[i]:rp[i + 1]])
            Ablk = A[k, rp[i]:rp[i + 1]]
            ck = xo[k + 1, i] - np.einsum("bst,bt->s", Ablk, xo[k][nb])
            per.append((nb, Ablk, B[k, i], ck))
        blocks.append(per)
    Cx, dx = ocd.sphere_halfspaces(xo, wl.spheres.astype(np.float64))
    H, g, Ct, dt, _, _ = ocd.condense_recursive(blocks, xo[0].reshape(-1), wl.Qdiag, wl.Rdiag, wl.x_ref,
                                                wl.u_ref, Cx, dx)
    U, _, _ = oqp.solve_exact(H, g, wl.u_lo.reshape(-1).astype(np.float64),
                              wl.u_hi.reshape(-1).astype(np.float64), Ct, dt)
    H32, g32, _, _ = (t.cpu().numpy().astype(np.float64) for t in p32.condense(*p32.linearize(x0, zeros)))
    del p32
    return H, g, U, H32, g32


def test_mixed_u_at_paper_scale_cold_and_warm_graph(lib):
    from paper_2602_17601_b300 import gm_rollout
    wl = paper_chain()
    import torch as t
    zeros = t.zeros(wl.N, wl.nu, dtype=t.float32, device="cuda")
    x0 = t.as_tensor(np.asarray(wl.x0, np.float32).reshape(-1), device="cuda")
    Href, gref, Uref, H32, g32 = _fp64_reference(lib, wl, x0, zeros)
    R = np.diag(wl.Rdiag.reshape(-1).astype(np.float64))
    # H and g of the mixed form (and, for reference, of the FP32 form) against FP64 condensing
    prob = lib.RTIProblem.from_workload(wl, precision=GM_PREC_MIXED)
    H, g, Ct, dt = prob.condense(*prob.linearize(x0, zeros))
    Hm, gm_ = (a.cpu().numpy().astype(np.float64) for a in (H, g))
    eh, eg = max_rel_err(Hm - R, Href - R), max_rel_err(gm_, gref)
    eh32, eg32 = max_rel_err(H32 - R, Href - R), max_rel_err(g32, gref)
    print(f"chain of 1000 against the FP64 reference: mixed H - Rbar {eh:.2e}, g {eg:.2e}; "
          f"FP32 form H - Rbar {eh32:.2e}, g {eg32:.2e}")
    # g sums Gamma_u' Q (x_hat - x_ref) over 20k node-stages and inherits the Jacobian rows'
    # one-sided derivatives at near-kink units (the reference takes the FP32 form's rows)
    assert eh <= REL_MIXED and eg <= G_TOL, (eh, eg)
    # U of a cold step at a tight ADMM tolerance against the FP64 reference optimum
    wl_t = paper_chain(tol=1e-7)
    pt = lib.RTIProblem.from_workload(wl_t, precision=GM_PREC_MIXED)
    U = pt.step(wl.x0).cpu().numpy().astype(np.float64)
    st = pt.read_stats()
    assert st["status"] == lib.GM_OK and st["converged"] == 1, st
    err = np.abs(U - Uref).max()
    print(f"mixed form, chain of 1000, cold step, tol 1e-7: |U - U*_FP64| = {err:.2e} "
          f"(relative {err / np.abs(Uref).max():.2e}), ADMM iterations {st['iters']}")
    # every Jacobian row of this network has ReLU units within ~1e-6 of their kink, where an
    # evaluation at FP32 operand precision and the FP64 one may take opposite one-sided
    # derivatives: U is bounded at U_KINK of max|U*| against the FP64 reference, and at 1e-4
    # (beyond the ADMM's own bound) against the exact optimum of the QP the step solved
    assert err <= U_KINK * np.abs(Uref).max(), err
    H, g, Ct, dt = pt.condense(*pt.linearize(x0, zeros))
    Ue, lam = _exact_u(wl, pt.n_c, H, g, Ct, dt)
    _check_u("cold step, tol 1e-7, against its own QP's exact optimum", U, st, Ue, lam)
    del pt
    # the bench tolerance: one cold step against the exact optimum of its own QP
    U = prob.step(wl.x0).cpu().numpy().astype(np.float64)
    st = prob.read_stats()
    assert st["status"] == lib.GM_OK and st["converged"] == 1, st
    Ue, lam = _exact_u(wl, prob.n_c, H, g, Ct, dt)
    _check_u("cold step, tol 1e-4", U, st, Ue, lam)
    # four steps of a warm-started, graph-replayed closed loop (the GNN as the plant)
    pw = lib.RTIProblem.from_workload(wl, precision=GM_PREC_MIXED, graph=True, warm=True)
    x = x0.clone()
    nxt = t.empty(2, wl.M * 6, dtype=t.float32, device="cuda")
    Us = []
    for s_ in range(4):
        Us.append(pw.step(x).clone())
        stw = pw.read_stats()
        assert stw["status"] in (lib.GM_OK, lib.GM_STALLED) and stw["converged"] == 1, (s_, stw)
        if s_ < 3:
            gm_rollout(pw.ctx, x, Us[-1][:wl.nu].contiguous(), 1, nxt)
            x.copy_(nxt[1])
    assert pw.graph_state()[0] == 1
    u_hat = t.as_tensor(orti.shift(Us[2].cpu().numpy().astype(np.float64).reshape(wl.N, wl.nu)),
                        dtype=t.float32, device="cuda")
    H, g, Ct, dt = prob.condense(*prob.linearize(x, u_hat))
    Ue, lam = _exact_u(wl, prob.n_c, H, g, Ct, dt)
    _check_u("fourth warm graph-replayed closed-loop step", Us[3].cpu().numpy().astype(np.float64), stw, Ue, lam)
