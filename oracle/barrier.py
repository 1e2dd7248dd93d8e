"""Barrier-cost obstacle variant of the condensed QP, FP64 (oracle; test infrastructure only).

Sec. VI-B avoids obstacles with one barrier term per measured node in the
cost, and gives no formula.  Reading used here:

* the obstacle rows are the same linearised sphere clearances the constraint
  form uses (``condense.sphere_halfspaces``): for node i, stage k and sphere
  (o, r) the clearance is s = n^T (p - o) - r with n the unit normal at the
  rollout point, and in the condensed variables s(U) = d~_r - C~_r U;
* each row adds mu * beta(s) to the (halved) cost, beta the relaxed
  logarithmic barrier of Feller and Ebenbauer (IEEE TAC 2017, after Hauser and
  Saccon 2006):

      beta(s) = -ln s                                   s >  delta
      beta(s) = 1/2 (((s - 2 delta) / delta)^2 - 1) - ln delta    s <= delta

  which is convex and twice continuously differentiable (value, slope and
  curvature agree at s = delta) and finite for s <= 0, so a rollout that has
  entered an obstacle still gives a well-defined step;
* an RTI step takes the second-order model of the barrier at the
  linearisation point U_hat (the shifted previous solution).  Because s is
  affine in U, the model is the exact second-order Taylor expansion, and the
  step is one Newton step on  1/2 U'HU + g'U + mu sum_r beta(s_r(U))  under the
  input box:

      H' = H + C~' diag(mu beta''(s^)) C~
      g' = g - C~' (mu beta'(s^) + mu beta''(s^) C~ U_hat),    s^ = d~ - C~ U_hat.

  The QP keeps the input box and has no half-space rows.
"""
from __future__ import annotations

import numpy as np


def relaxed_log_barrier(s, delta):
    """beta(s), beta'(s), beta''(s) of the relaxed logarithmic barrier (element-wise)."""
    s = np.asarray(s, np.float64)
    inner = s > delta
    ss = np.where(inner, s, 1.0)
    t = (s - 2.0 * delta) / delta
    b0 = np.where(inner, -np.log(ss), 0.5 * (t * t - 1.0) - np.log(delta))
    b1 = np.where(inner, -1.0 / ss, (s - 2.0 * delta) / (delta * delta))
    b2 = np.where(inner, 1.0 / (ss * ss), 1.0 / (delta * delta))
    return b0, b1, b2


def barrier_objective(H, g, Ct, dt, U, mu, delta):
    """The barrier-augmented condensed cost 1/2 U'HU + g'U + mu sum_r beta(d~_r - C~_r U)."""
    U = np.asarray(U, np.float64)
    s = np.asarray(dt, np.float64) - np.asarray(Ct, np.float64) @ U
    return 0.5 * U @ H @ U + g @ U + mu * relaxed_log_barrier(s, delta)[0].sum()


def barrier_fold(H, g, Ct, dt, U_hat, mu, delta):
    """H', g' of the second-order barrier model at U_hat (module docstring)."""
    Ct = np.asarray(Ct, np.float64)
    U_hat = np.asarray(U_hat, np.float64).reshape(-1)
    a = Ct @ U_hat
    _, b1, b2 = relaxed_log_barrier(np.asarray(dt, np.float64) - a, delta)
    Hb = np.asarray(H, np.float64) + Ct.T @ (mu * b2[:, None] * Ct)
    gb = np.asarray(g, np.float64) - Ct.T @ (mu * b1 + mu * b2 * a)
    return Hb, gb
