"""Parity of the tensor-core precision forms with the FP64 oracle.  Needs a GPU.

GM_PREC_MIXED runs every GNN product on BF16 tensor cores with each operand
split into a hi and a lo BF16 part (three products, FP32 accumulation in
tensor memory), which carries about 16 significant bits through each MLP.
Its target: the oracle's linearisation within REL_MIXED = 1e-4 of each
quantity's max-abs, and U within 1e-4 of max|U| beyond what the solver's own
tolerance allows.

A ReLU network's Jacobian jumps where a pre-activation crosses zero, so two
correct evaluations whose pre-activations differ by e disagree on every unit
closer than e to its kink.  Element-wise parity at 1e-4 therefore needs
inputs whose pre-activations all keep a margin well above the form's
rounding.  The cases below are seeded instances picked by the oracle alone
(largest margin among the first seeds), with weights at fan-in scale 2 so that
such a margin exists on a graph of useful size, and the decoder's output layer
scaled by 1e-3 so that the velocity increments, and with them the condensed
QP, stay well conditioned.

c = x_hat[k+1] - A x_hat[k] - B u_hat[k] is a difference of larger terms, so
its error is measured against the largest of those terms.
"""
import numpy as np
import pytest

from gpu_helpers import blocks_to_dense, max_rel_err, ocd, oracle_linearize, orti
from oracle import gnn as ognn
from synth import random_instance

pytestmark = pytest.mark.gpu

REL_MIXED = 1e-4
GM_PREC_MIXED, GM_PREC_BF16 = 1, 2


def _u_hat(wl, seed):
    return np.random.default_rng(seed).uniform(-0.5, 0.5, (wl.N, wl.nu)).astype(np.float32)


def _margin(wl, u_hat):
    """Smallest |pre-activation| over the oracle's rollout along u_hat."""
    gnn, g = orti.model_of(wl)
    x = np.asarray(wl.x0, np.float64).reshape(wl.M, 6)
    m = np.inf
    for k in range(wl.N):
        m = min(m, ognn.preactivations_min_abs(gnn, g, x, u_hat[k].astype(np.float64)))
        x = ognn.step(gnn, g, x, u_hat[k].astype(np.float64))
    return m


DEC_SCALE = 1e-3


def _instance(seed, W):
    wl = random_instance(seed, M=9, N=2, nu=2, K=3, W=W, reach=2, p=0.7, w_scale="fan_in:2")
    wl.blob = wl.blob.copy()
    wl.blob[-(3 * W + 3):] *= DEC_SCALE      # decoder layer 2: W2 [W][3], b2 [3]
    return wl


def _kink_free(W, n_seeds=20, zero_u=False):
    """The instance with the widest kink margin along u_hat (zeros: the first RTI step's)."""
    best = None
    for seed in range(n_seeds):
        wl = _instance(seed, W)
        u_hat = np.zeros((wl.N, wl.nu), np.float32) if zero_u else _u_hat(wl, seed)
        m = _margin(wl, u_hat)
        if best is None or m > best[0]:
            best = (m, wl, u_hat)
    assert best[0] > 1e-4, best[0]
    return best[1], best[2]


def _linearize(lib, wl, u_hat, precision):
    prob = lib.RTIProblem.from_workload(wl, precision=precision)
    out = tuple(t.cpu().numpy().astype(np.float64) for t in prob.linearize(wl.x0, u_hat))
    return prob, out


def _errors(prob, wl, u_hat, got, want):
    x_hat, A, B, c = got
    xo, Ao, Bo, co = want
    errs = {"x_hat": max_rel_err(x_hat, xo), "A": 0.0, "B": 0.0, "c": 0.0}
    for k in range(wl.N):
        Ag = blocks_to_dense(A[k], prob.row_ptr, prob.col, wl.M)
        V = Ao[k].reshape(wl.M, 6, wl.M, 6)[:, 3:].copy()
        for i in range(wl.M):
            V[i, :, i, 3:] -= np.eye(3)
        errs["A"] = max(errs["A"], max_rel_err(Ag, Ao[k], scale=max(np.abs(V).max(), 1e-3)))
        errs["B"] = max(errs["B"], max_rel_err(B[k].reshape(-1, wl.nu), Bo[k]))
        xk = xo[k].reshape(-1)
        terms = max(np.abs(xo[k + 1]).max(), np.abs(Ao[k] @ xk).max(), np.abs(Bo[k] @ u_hat[k]).max())
        errs["c"] = max(errs["c"], max_rel_err(c[k].reshape(-1), co[k], scale=terms))
    return errs


@pytest.mark.parametrize("W", [32, 64, 128])
def test_mixed_linearize_parity(lib, W):
    """x_hat and A, B, c (Eq. linearized_dynamics) of the split-BF16 form against the oracle."""
    wl, u_hat = _kink_free(W)
    prob, got = _linearize(lib, wl, u_hat, GM_PREC_MIXED)
    errs = _errors(prob, wl, u_hat, got, oracle_linearize(wl, u_hat.astype(np.float64)))
    assert max(errs.values()) <= REL_MIXED, errs


@pytest.mark.parametrize("W", [64, 128])
def test_mixed_condensed_h_g(lib, W):
    """H and g (Eq. H, Eq. g) from the split-BF16 linearisation, condensed on the GPU, against the
    oracle's condensing of its own linearisation.  H's learned part (H - Rbar) and g are compared
    to 1e-4 of their max-abs; both are sums of products of Jacobian entries, so they carry the
    Jacobians' relative error."""
    wl, u_hat = _kink_free(W)
    prob, (x_hat, A, B, c) = _linearize(lib, wl, u_hat, GM_PREC_MIXED)
    torch = prob.torch
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")  # noqa: E731
    H, g, _, _ = (t.cpu().numpy().astype(np.float64) for t in prob.condense(dev(x_hat), dev(A), dev(B), dev(c)))
    xo, Ao, Bo, co = oracle_linearize(wl, u_hat.astype(np.float64))
    nbh = [list(prob.col[prob.row_ptr[i]:prob.row_ptr[i + 1]]) for i in range(wl.M)]
    blocks = ocd.blocks_from_dense(Ao, Bo, co, nbh)
    Ho, go, _, _, _, _ = ocd.condense_recursive(blocks, xo[0].reshape(-1), wl.Qdiag, wl.Rdiag, wl.x_ref, wl.u_ref,
                                                np.zeros((wl.N, wl.M, 0, 3)), np.zeros((wl.N, wl.M, 0)))
    R = np.diag(wl.Rdiag.reshape(-1).astype(np.float64))
    eh, eg = max_rel_err(H - R, Ho - R), max_rel_err(g, go)
    print(f"mixed form W={W}: H - Rbar rel err {eh:.2e}, g rel err {eg:.2e}")
    assert eh <= REL_MIXED and eg <= REL_MIXED, (eh, eg)


def test_mixed_rti_step_u(lib):
    """A whole real-time iteration (Alg. 1) in the split-BF16 form: U against the exact optimum."""
    wl, _ = _kink_free(128, zero_u=True)
    wl.tol = 1e-7
    prob = lib.RTIProblem.from_workload(wl, precision=GM_PREC_MIXED)
    U = prob.step(wl.x0).cpu().numpy().astype(np.float64).reshape(wl.N, wl.nu)
    st = prob.read_stats()
    rx = orti.rti_step(wl, solver="exact", return_all=True)
    assert st["converged"] == 1
    lam = np.linalg.eigvalsh(rx["H"]).min()
    admm_bound = 2 * max(st["r_dual"], st["kkt_stat"]) / lam
    scale = np.abs(rx["U"]).max()
    assert np.abs(U - rx["U"]).max() <= admm_bound + REL_MIXED * scale, (np.abs(U - rx["U"]).max(), scale)


def test_bf16_form_runs(lib):
    """The single-BF16 form: a speed form with no parity claim beyond the forward rollout
    at BF16 accuracy; its QP is still solved to the requested tolerance."""
    wl, u_hat = _kink_free(64)
    prob, got = _linearize(lib, wl, u_hat, GM_PREC_BF16)
    xo = oracle_linearize(wl, u_hat.astype(np.float64))[0]
    assert all(np.isfinite(a).all() for a in got)
    assert max_rel_err(got[0], xo) <= 3e-2
    prob.step(wl.x0)
    st = prob.read_stats()
    assert st["converged"] == 1 and st["kkt_prim"] <= 10 * wl.tol


def test_mixed_linearize_multi_tile_against_fp32_form(lib):
    """The split-BF16 reverse pass at a size where each persistent CTA walks many 128-row tiles
    with a ragged last tile (chain of 150 nodes, K = 3, W = 128: about 1.6k tiles for the
    largest reverse edge-MLP launch), against the FP32 form on the same inputs (the FP32 form
    is pinned to the oracle element by element in test_gpu_parity).  Both reverse passes use
    the forward ReLU pattern of their own rollout, so a few units near a kink may differ; the
    test bounds the 99.99th percentile of the error and its maximum separately."""
    from synth import paper_chain
    wl = paper_chain(seed=3, M=150, N=4, nu=8)
    u_hat = np.random.default_rng(4).uniform(-0.3, 0.3, (wl.N, wl.nu)).astype(np.float32)
    out = {}
    for prec in (0, GM_PREC_MIXED):
        prob = lib.RTIProblem.from_workload(wl, precision=prec)
        out[prec] = [t.cpu().numpy().astype(np.float64) for t in prob.linearize(wl.x0, u_hat)]
        del prob
    (xm, Am, Bm, cm), (xf, Af, Bf, cf) = out[GM_PREC_MIXED], out[0]
    assert max_rel_err(xm, xf) <= 1e-5
    for got, ref in ((Am, Af), (Bm, Bf)):
        e = np.abs(got - ref) / np.abs(ref).max()
        assert np.quantile(e, 0.9999) <= REL_MIXED and e.max() <= 5e-2, (np.quantile(e, 0.9999), e.max())
    # c: a difference of larger terms, measured against x_hat's scale
    e = np.abs(cm - cf) / np.abs(xf).max()
    assert np.quantile(e, 0.9999) <= REL_MIXED, np.quantile(e, 0.9999)


@pytest.mark.parametrize("W", [32, 64, 128])
@pytest.mark.parametrize("split", [0, 1])
def test_mixed_matrix_free_h_g(lib, W, split):
    """Matrix-free condensing in the split-BF16 form (tangent MLPs on tensor cores, the node-side
    pairs in one launch): H and g against the oracle's condensing of its own linearisation, to
    1e-4 of their max-abs.  split = 1 puts every edge layer on per-node projections of the first
    layer's node blocks (gm_settings.tan_split_rows = 1; the warp-specialised kernel at W = 128),
    split = 0 keeps the whole first layer on these small graphs."""
    wl, u_hat = _kink_free(W)
    prob = lib.RTIProblem.from_workload(wl, precision=GM_PREC_MIXED, condensing=1, tan_split_rows=split)
    x_hat, H, g, _, _ = (t.cpu().numpy().astype(np.float64) for t in prob.condense_matrix_free(wl.x0, u_hat))
    xo, Ao, Bo, co = oracle_linearize(wl, u_hat.astype(np.float64))
    nbh = [list(prob.col[prob.row_ptr[i]:prob.row_ptr[i + 1]]) for i in range(wl.M)]
    blocks = ocd.blocks_from_dense(Ao, Bo, co, nbh)
    Ho, go, _, _, _, _ = ocd.condense_recursive(blocks, xo[0].reshape(-1), wl.Qdiag, wl.Rdiag, wl.x_ref, wl.u_ref,
                                                np.zeros((wl.N, wl.M, 0, 3)), np.zeros((wl.N, wl.M, 0)))
    R = np.diag(wl.Rdiag.reshape(-1).astype(np.float64))
    assert max_rel_err(x_hat, xo) <= REL_MIXED
    eh, eg = max_rel_err(H - R, Ho - R), max_rel_err(g, go)
    assert eh <= REL_MIXED and eg <= REL_MIXED, (W, split, eh, eg)
