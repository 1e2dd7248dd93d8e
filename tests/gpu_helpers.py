"""Shared helpers of the GPU parity tests (oracle on one side, the C-ABI library on the other).

Tolerances.  The CUDA path computes in FP32 and the oracle in FP64.  Each
GNN layer is a chain of dot products of length <= 3W = 384 whose rounding
error is about sqrt(n) * 2^-24 ~ 1.2e-6 relative on average (n * 2^-24 ~ 2.3e-5
worst case); a rollout/Jacobian passes through about 5 + 2K such layers per
stage and N stages.  We therefore bound the max-abs error of every floating
output by REL * (max-abs of the quantity) with REL = 2e-4, which leaves a
margin of 10x over the expected accumulation but catches any wrong term, sign
or index (those produce O(1) relative errors).
"""
import numpy as np

from oracle import condense as ocd
from oracle import gnn as ogm
from oracle import qp as oqp
from oracle import rti as orti

REL = 2e-4


def max_rel_err(got, ref, scale=None):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    s = np.abs(ref).max() if scale is None else scale
    s = max(s, 1e-30)
    return float(np.abs(got - ref).max() / s) if ref.size else 0.0


def blocks_to_dense(Ablk, row_ptr, col, M):
    """[nnzb, 6, 6] blocks in pattern order -> dense [6M, 6M]."""
    A = np.zeros((6 * M, 6 * M))
    for i in range(M):
        for q in range(row_ptr[i], row_ptr[i + 1]):
            j = col[q]
            A[6 * i:6 * i + 6, 6 * j:6 * j + 6] = Ablk[q]
    return A


def dense_to_blocks(A, row_ptr, col, M):
    out = np.zeros((col.size, 6, 6))
    for i in range(M):
        for q in range(row_ptr[i], row_ptr[i + 1]):
            j = col[q]
            out[q] = A[6 * i:6 * i + 6, 6 * j:6 * j + 6]
    return out


def oracle_linearize(wl, u_hat):
    gnn, g = orti.model_of(wl)
    x_hat = ogm.rollout(gnn, g, wl.x0, u_hat)
    A, B, c = orti.linearize_dense(gnn, g, x_hat, u_hat)
    return x_hat, A, B, c


def packed_to_dense_ct(Ct, N, M, n_c, nu):
    """Packed stage-major C~ (rows of length k nu) -> dense [N M n_c, N nu]."""
    rows = N * M * n_c
    D = np.zeros((rows, N * nu))
    off = 0
    for k in range(1, N + 1):
        L = k * nu
        for w in range(M * n_c):
            D[(k - 1) * M * n_c + w, :L] = Ct[off:off + L]
            off += L
    return D


def dense_to_packed_ct(D, N, M, n_c, nu):
    out = []
    for k in range(1, N + 1):
        L = k * nu
        for w in range(M * n_c):
            out.append(D[(k - 1) * M * n_c + w, :L])
    return np.concatenate(out) if out else np.zeros(0)


__all__ = ["REL", "max_rel_err", "blocks_to_dense", "dense_to_blocks", "oracle_linearize",
           "packed_to_dense_ct", "dense_to_packed_ct", "ocd", "ogm", "oqp", "orti"]
