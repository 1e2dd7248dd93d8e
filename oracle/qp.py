"""The condensed QP and the solvers used to check the method, FP64 (oracle; test infrastructure only).

QP (Sec. III-B, Eq. condensed_matrices, with the 1/2 convention of
``oracle.condense``):

    min 1/2 U^T H U + g^T U   s.t.   lo <= U <= hi,   C U <= d.

Written with A~ = [I; C], l = [lo; -inf], h = [hi; d] as  l <= A~ U <= h.
H is positive definite because Rbar is (R = 0.01 I), so the optimal U is unique;
the multipliers may not be when the active rows are linearly dependent (LICQ,
Sec. I).

Contents:
* ``kkt_certificate``   stationarity, feasibility, dual signs, complementarity;
* ``solve_exact``       the definition of the optimum: a primal-dual interior
                        point method to a tight KKT residual, then the equality-
                        constrained solve on the active set it identifies;
* ``admm``              the ADMM recurrence the GPU path runs (fixed rho,
                        no relaxation, no scaling);
* ``primal_infeasible`` the certificate ADMM's dual step gives when no U
                        satisfies the constraints;
* ``polish``            equality-constrained re-solve on the active set guessed
                        from an ADMM iterate;
* ``brute_force``       every active set, for tiny problems;
* ``uncondensed``       the QP in (x, u) with the dynamics as equalities
                        (Eq. ocp_dynamics), for tiny problems.
"""
from __future__ import annotations

import itertools

import numpy as np


def stack_rows(lo, hi, C, d):
    """A~ = [I; C], l = [lo; -inf], h = [hi; d]."""
    n = lo.size
    C = np.zeros((0, n)) if C is None else np.asarray(C, np.float64)
    d = np.zeros(0) if d is None else np.asarray(d, np.float64)
    At = np.vstack([np.eye(n), C])
    l = np.concatenate([np.asarray(lo, np.float64), np.full(C.shape[0], -np.inf)])
    h = np.concatenate([np.asarray(hi, np.float64), d])
    return At, l, h


def kkt_certificate(H, g, At, l, h, U, y):
    """Residuals of the KKT conditions of min 1/2 U'HU + g'U s.t. l <= A~U <= h.

    y_r > 0 pushes against the upper bound, y_r < 0 against the lower bound.
    """
    a = At @ U
    stat = np.abs(H @ U + g + At.T @ y).max() if U.size else 0.0
    prim = max(0.0, np.max(a - h, initial=0.0), np.max(l - a, initial=0.0))
    # a row without an upper bound may not push up (y <= 0), without a lower bound not down
    dual = max(np.max(np.where(np.isinf(h), np.maximum(y, 0.0), 0.0), initial=0.0),
               np.max(np.where(np.isinf(l), np.maximum(-y, 0.0), 0.0), initial=0.0))
    up = np.maximum(y, 0.0) * np.abs(np.where(np.isinf(h), 0.0, h - a))
    lo_ = np.maximum(-y, 0.0) * np.abs(np.where(np.isinf(l), 0.0, a - l))
    comp = max(np.max(up, initial=0.0), np.max(lo_, initial=0.0))
    return dict(stationarity=float(stat), primal=float(prim), dual=float(dual),
                complementarity=float(comp))


def _ineq_form(At, l, h):
    """G U <= hh with one row per finite bound (upper rows +a, lower rows -a)."""
    rows, rhs, owner, sign = [], [], [], []
    for r in range(At.shape[0]):
        if np.isfinite(h[r]):
            rows.append(At[r]); rhs.append(h[r]); owner.append(r); sign.append(1.0)
        if np.isfinite(l[r]):
            rows.append(-At[r]); rhs.append(-l[r]); owner.append(r); sign.append(-1.0)
    n = At.shape[1]
    G = np.array(rows) if rows else np.zeros((0, n))
    return G, np.array(rhs), np.array(owner, int), np.array(sign)


def ipm(H, g, G, hh, tol=1e-13, max_iter=200):
    """Mehrotra predictor-corrector primal-dual interior point for min 1/2x'Hx+g'x, Gx<=hh."""
    n, m = H.shape[0], G.shape[0]
    x = np.zeros(n)
    if m == 0:
        return np.linalg.solve(H, -g), np.zeros(0), np.zeros(0), 0
    s = np.maximum(hh - G @ x, 1.0)
    z = np.ones(m)
    scale = max(1.0, np.abs(g).max(), np.abs(hh).max())
    for it in range(max_iter):
        rd = H @ x + g + G.T @ z
        rp = G @ x + s - hh
        mu = s @ z / m
        if max(np.abs(rd).max(), np.abs(rp).max()) <= tol * scale and mu <= tol * scale:
            return x, s, z, it

        def solve(rc):
            Wd = z / s
            Kmat = H + G.T @ (Wd[:, None] * G)
            rhs = -rd - G.T @ (Wd * rp - rc / s)
            dx = np.linalg.solve(Kmat, rhs)
            dz = Wd * (G @ dx + rp) - rc / s
            ds = -(rc + s * dz) / z
            return dx, ds, dz

        def step_len(v, dv):
            neg = dv < 0
            return min(1.0, np.min(-v[neg] / dv[neg], initial=np.inf))

        try:
            dxa, dsa, dza = solve(s * z)
        except np.linalg.LinAlgError:
            return x, s, z, it            # the Newton matrix lost rank at a converged point
        aa = min(step_len(s, dsa), step_len(z, dza))
        mu_aff = (s + aa * dsa) @ (z + aa * dza) / m
        sigma = (mu_aff / mu) ** 3
        dx, ds, dz = solve(s * z + dsa * dza - sigma * mu)
        a = 0.99 * min(step_len(s, ds), step_len(z, dz))
        x, s, z = x + a * dx, s + a * ds, z + a * dz
    return x, s, z, max_iter


def equality_solve(H, g, At, l, h, upper, lower):
    """Minimise 1/2U'HU+g'U with the rows in `upper` held at h and `lower` at l.

    Returns (U, y) with y the full multiplier vector (zero off the active set),
    or None if the KKT matrix is singular.
    """
    n = H.shape[0]
    act = list(upper) + list(lower)
    if not act:
        return np.linalg.solve(H, -g), np.zeros(At.shape[0])
    Ga = At[act]
    ba = np.concatenate([h[list(upper)], l[list(lower)]])
    K = np.block([[H, Ga.T], [Ga, np.zeros((len(act), len(act)))]])
    rhs = np.concatenate([-g, ba])
    try:
        sol = np.linalg.solve(K, rhs)
    except np.linalg.LinAlgError:
        return None
    if not np.all(np.isfinite(sol)):
        return None
    U = sol[:n]
    y = np.zeros(At.shape[0])
    y[act] = sol[n:]
    return U, y


def solve_exact(H, g, lo, hi, C=None, d=None):
    """The optimum U* of the condensed QP and one valid multiplier vector.

    Interior point to a tight residual, then the active set it identifies
    (multiplier larger than slack) is re-solved as an equality QP; the re-solve
    is kept when its KKT certificate is at least as good.
    """
    H = np.asarray(H, np.float64)
    g = np.asarray(g, np.float64)
    At, l, h = stack_rows(np.asarray(lo, np.float64), np.asarray(hi, np.float64), C, d)
    G, hh, owner, sign = _ineq_form(At, l, h)
    x, s, z, it = ipm(H, g, G, hh)
    y = np.zeros(At.shape[0])
    np.add.at(y, owner, sign * z)
    best = (x, y)
    cert = kkt_certificate(H, g, At, l, h, x, y)
    best_err = max(cert.values())
    act = z > s
    upper = sorted({int(owner[k]) for k in np.nonzero(act & (sign > 0))[0]})
    lower = sorted({int(owner[k]) for k in np.nonzero(act & (sign < 0))[0]})
    res = equality_solve(H, g, At, l, h, upper, lower)
    if res is not None:
        c2 = kkt_certificate(H, g, At, l, h, *res)
        if max(c2.values()) <= best_err:
            best = res
            best_err = max(c2.values())
    return best[0], best[1], dict(ipm_iters=it, kkt=best_err)


ROW_NORM_FLOOR = 1e-8
REDUNDANT_MARGIN = 1e-4    # relative safety margin of the redundant-row test
INFEAS_EVERY = 10          # ADMM iterations between infeasibility tests
STALL_FACTOR = 0.5         # warm start stalls when max(r_p, r_d) is not below this fraction
                           # of its value stall_every iterations earlier
INFEAS_EPS = 1e-4          # relative tolerance of the certificate


def primal_infeasible(At, l, h, dy, eps=INFEAS_EPS):
    """True when dy certifies that no U satisfies l <= A~U <= h, up to eps.

    Farkas' lemma: the set is empty iff some v has A~'v = 0 and support
    sup_{l <= s <= h} v's = h'max(v, 0) + l'min(v, 0) < 0; a component of v
    whose sign meets an infinite bound makes the support +inf.  For ADMM,
    Banjac, Goulart, Stellato and Boyd (2019, "Infeasibility detection in the
    alternating direction method of multipliers for convex optimization")
    show that the dual step dy = y^k - y^(k-1) converges to such a v when the
    constraints are infeasible.  The relative test (eps scales |dy|_inf):
        |A~'dy|_inf <= eps |dy|_inf,
        dy_r >= -eps |dy|_inf where l_r = -inf,  dy_r <= eps |dy|_inf where h_r = +inf,
        sum over finite bounds of h_r max(dy_r, 0) + l_r min(dy_r, 0) <= -eps |dy|_inf.
    """
    dy = np.asarray(dy, np.float64)
    dmax = np.abs(dy).max(initial=0.0)
    if dmax == 0.0:
        return False
    e = eps * dmax
    up, dn = np.maximum(dy, 0.0), np.minimum(dy, 0.0)
    hfin, lfin = np.isfinite(h), np.isfinite(l)
    wrong = max(np.max(up[~hfin], initial=0.0), np.max(-dn[~lfin], initial=0.0))
    support = float(np.sum(h[hfin] * up[hfin]) + np.sum(l[lfin] * dn[lfin]))
    return bool(np.abs(At.T @ dy).max() <= e and wrong <= e and support <= -e)


def redundant_rows(C, d, lo, hi, margin=None):
    """Rows that no U in the input box can violate: the box's support in the row's direction,
    max over lo <= U <= hi of C_r U = sum_c max(C_rc hi_c, C_rc lo_c), lies below d_r by more
    than margin (|C_r|_1 max|bound| + |d_r|).  Such a row is inactive at every feasible U (its
    multiplier is 0 at the optimum) and leaves the feasible set unchanged when dropped."""
    margin = REDUNDANT_MARGIN if margin is None else margin
    C = np.asarray(C, np.float64)
    d = np.asarray(d, np.float64)
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    with np.errstate(invalid="ignore"):
        sup = np.where(C > 0, C * hi, np.where(C < 0, C * lo, 0.0)).sum(axis=1)
    bmax = np.maximum(np.abs(lo), np.abs(hi))
    scale = np.where(C != 0, np.abs(C) * bmax, 0.0).sum(axis=1) + np.abs(d)
    return sup < d - margin * scale


def row_scaling(C):
    """s_r = 1 / max(|C_r|_2, 1e-8): unit rows, except rows that barely depend on U."""
    nr = np.sqrt((np.asarray(C, np.float64) ** 2).sum(axis=1))
    return 1.0 / np.maximum(nr, ROW_NORM_FLOOR)


def admm(H, g, lo, hi, C=None, d=None, rho=0.1, tol=1e-6, max_iter=4000, U0=None, y0=None,
         scale_rows=False, adapt_every=0, max_updates=5, detect_infeasible=True, return_info=False,
         stall_every=0, drop_redundant=True):
    """ADMM on l <= A~U <= h (fixed rho, alpha = 1, sigma = 0, unscaled residuals).

        P     = H + rho A~'A~                      (factored once)
        z^0   = Pi(A~ U^0),  y^0 = 0 unless given
        U     = P^{-1} (A~'(rho z - y) - g)
        a     = A~ U
        z     = Pi_[l,h](a + y / rho)
        y     = y + rho (a - z)
        r_p   = |a - z|_inf,   r_d = |H U + g + A~'y|_inf;  stop when both <= tol.

    scale_rows: run the recurrence on the half-space rows divided by their
    2-norms (C_r / |C_r|, d_r / |C_r|), which leaves the feasible set and U*
    unchanged; z and y are returned for the original rows (y_r = s_r y'_r).

    adapt_every > 0: after every adapt_every-th iteration (at most max_updates
    times) compare the residuals relative to their scales,
        ratio = (r_p / max(|a|, |z|)) / (r_d / max(|H U|, |A~'y|, |g|)),
    and re-factor P with rho sqrt(ratio) (clamped to [1e-6, 1e6]) when that
    changes rho by more than a factor 5.

    detect_infeasible: after every INFEAS_EVERY-th iteration that has not
    converged, stop when the dual step y - y_prev (on the rows the recurrence
    runs on) passes ``primal_infeasible``.

    stall_every > 0 with a warm start (U0 or y0 given): the stall rule.  After
    the first iteration, and again after each rho change, r = max(r_p, r_d) is
    recorded; every stall_every iterations at which rho does not change, r is
    compared with the record and becomes the new record.  When r is not below
    STALL_FACTOR times the record (a stall), or an iterate is NaN, the warm
    start is dropped and the recurrence restarts cold (U = 0, y = 0, rho = the
    given rho, P re-factored, a fresh max_iter and max_updates) at the same
    iteration count.  Before a restart rho may change once.

    drop_redundant: half-space rows that no U in the input box can violate
    (``redundant_rows``) take no part in the recurrence; their multipliers are
    0 and their z is C_r U.  The optimum is the same.

    Returns U, z, y, iterations (number of U updates), r_p, r_d, converged;
    return_info adds a dict {infeasible, dy, restarted} (dy for the original
    rows; restarted: the cold restart ran).
    """
    H = np.asarray(H, np.float64)
    g = np.asarray(g, np.float64)
    n = H.shape[0]
    keep = None
    if drop_redundant and C is not None and np.asarray(C).shape[0] > 0:
        keep = np.nonzero(~redundant_rows(C, d, lo, hi))[0]
        C_all, m_all = np.asarray(C, np.float64), np.asarray(C).shape[0]
        C = C_all[keep]
        d = np.asarray(d, np.float64)[keep]
        if y0 is not None:
            y0 = np.concatenate([np.asarray(y0, np.float64)[:n], np.asarray(y0, np.float64)[n:][keep]])
    s = None
    if scale_rows and C is not None and np.asarray(C).shape[0] > 0:
        s = row_scaling(C)
        C = np.asarray(C, np.float64) * s[:, None]
        d = np.asarray(d, np.float64) * s
        if y0 is not None:
            y0 = np.concatenate([y0[:n], y0[n:] / s])
    At, l, h = stack_rows(np.asarray(lo, np.float64), np.asarray(hi, np.float64), C, d)
    rho0 = rho
    P = H + rho * At.T @ At
    L = np.linalg.cholesky(P)
    U = np.zeros(n) if U0 is None else np.asarray(U0, np.float64).copy()
    y = np.zeros(At.shape[0]) if y0 is None else np.asarray(y0, np.float64).copy()
    z = np.clip(At @ U, l, h)
    r_p = r_d = np.inf
    it = 0
    ok = infeasible = restarted = False
    dy = np.zeros_like(y)
    updates = 0
    stall_on = stall_every > 0 and (U0 is not None or y0 is not None)
    stall_ref = None
    it0 = 0                                   # iteration count where the current start began
    while True:
        it += 1
        rhs = At.T @ (rho * z - y) - g
        U = np.linalg.solve(L.T, np.linalg.solve(L, rhs))
        a = At @ U
        z = np.clip(a + y / rho, l, h)
        y_prev = y
        y = y + rho * (a - z)
        r_p = np.abs(a - z).max()
        r_d = np.abs(H @ U + g + At.T @ y).max()
        if r_p <= tol and r_d <= tol:
            ok = True
            break
        bad = not (np.isfinite(r_p) and np.isfinite(r_d))
        if not bad and detect_infeasible and it % INFEAS_EVERY == 0:
            dy = y - y_prev
            if primal_infeasible(At, l, h, dy):
                infeasible = True
                break
        if bad and stall_on:
            stalled = True
        else:
            if bad or it - it0 >= max_iter:
                break
            stalled = False
            may_adapt = updates < max_updates and not (stall_on and updates >= 1)
            if adapt_every and it % adapt_every == 0 and may_adapt:
                ps = max(np.abs(a).max(), np.abs(z).max(), 1e-30)
                ds = max(np.abs(H @ U).max(), np.abs(At.T @ y).max(), np.abs(g).max(), 1e-30)
                ratio = (r_p / ps) / max(r_d / ds, 1e-30)
                rn = min(max(rho * np.sqrt(ratio), 1e-6), 1e6)
                if rn > 5 * rho or rn < 0.2 * rho:
                    rho = rn
                    updates += 1
                    L = np.linalg.cholesky(H + rho * At.T @ At)
                    stall_ref = None                  # the residuals' scale changed: new record
                    continue
            if stall_on:
                r = max(r_p, r_d)
                if stall_ref is None:
                    stall_ref = r
                elif (it - it0) % stall_every == 0:
                    stalled = not (r <= STALL_FACTOR * stall_ref)
                    stall_ref = r
        if stalled:
            # drop the warm start: cold from here, with the initial rho
            stall_on, restarted, it0, updates, rho = False, True, it, 0, rho0
            L = np.linalg.cholesky(H + rho * At.T @ At)
            U = np.zeros(n)
            y = np.zeros(At.shape[0])
            z = np.clip(At @ U, l, h)
            continue
    if s is not None:
        y = np.concatenate([y[:n], y[n:] * s])
        z = np.concatenate([z[:n], z[n:] / s])
        dy = np.concatenate([dy[:n], dy[n:] * s])
    if keep is not None:
        # dropped rows: multiplier 0, z = C_r U
        yf, df_ = np.zeros(n + m_all), np.zeros(n + m_all)
        zf = np.concatenate([z[:n], C_all @ U])
        yf[:n], df_[:n] = y[:n], dy[:n]
        yf[n + keep], zf[n + keep], df_[n + keep] = y[n:], z[n:], dy[n:]
        y, z, dy = yf, zf, df_
    if return_info:
        return U, z, y, it, r_p, r_d, ok, dict(infeasible=infeasible, dy=dy, restarted=restarted)
    return U, z, y, it, r_p, r_d, ok


def polish(H, g, lo, hi, C, d, U, z, y):
    """Re-solve on the active set guessed from (z, y): lower if z-l < -y, upper if h-z < y.

    Returns (U, y, accepted) where accepted means the re-solve is primal feasible,
    has correctly signed multipliers and a KKT certificate no worse than the input.
    """
    At, l, h = stack_rows(np.asarray(lo, np.float64), np.asarray(hi, np.float64), C, d)
    upper = [r for r in range(At.shape[0]) if np.isfinite(h[r]) and h[r] - z[r] < y[r]]
    lower = [r for r in range(At.shape[0]) if np.isfinite(l[r]) and z[r] - l[r] < -y[r]]
    res = equality_solve(H, g, At, l, h, upper, lower)
    if res is None:
        return U, y, False
    c0 = kkt_certificate(H, g, At, l, h, U, y)
    c1 = kkt_certificate(H, g, At, l, h, *res)
    if max(c1.values()) <= max(c0.values()):
        return res[0], res[1], True
    return U, y, False


def brute_force(H, g, lo, hi, C=None, d=None, tol=1e-9):
    """Try every active set (box rows: free/lower/upper; half-spaces: free/active)."""
    At, l, h = stack_rows(np.asarray(lo, np.float64), np.asarray(hi, np.float64), C, d)
    m = At.shape[0]
    choices = [((0, 1, 2) if np.isfinite(l[r]) else (0, 1)) for r in range(m)]
    best = None
    for pick in itertools.product(*choices):
        upper = [r for r in range(m) if pick[r] == 1]
        lower = [r for r in range(m) if pick[r] == 2]
        res = equality_solve(H, g, At, l, h, upper, lower)
        if res is None:
            continue
        cert = kkt_certificate(H, g, At, l, h, *res)
        if max(cert.values()) <= tol:
            if best is not None and np.abs(best[0] - res[0]).max() > 1e-8:
                raise AssertionError("two distinct KKT points of a strictly convex QP")
            best = res
    return best


def uncondensed(A, B, c, x0, Qdiag, Rdiag, x_ref, u_ref, lo, hi, Cx, dx, tol=1e-9):
    """Solve the QP in w = (x_0..x_N, u_0..u_{N-1}) with the dynamics as equalities.

    Eq. ocp_cost_norm / ocp_dynamics / ocp_initial_state with the tracking cost of
    Eq. linear_gnn_mpc_ocp_explicit (times 1/2).  Inequalities (input box and
    position half-spaces of stages 1..N) are handled by brute force over their
    active sets, each case a dense KKT solve.  Returns U.
    """
    N, nx, nu = B.shape
    M = nx // 6
    nX = (N + 1) * nx
    nw = nX + N * nu
    P = np.zeros((nw, nw))
    q = np.zeros(nw)
    Qd = np.asarray(Qdiag, np.float64).reshape(-1)
    P[:nX, :nX] = np.diag(Qd)
    q[:nX] = -Qd * np.asarray(x_ref, np.float64).reshape(-1)
    Rd = np.asarray(Rdiag, np.float64).reshape(-1)
    P[nX:, nX:] = np.diag(Rd)
    q[nX:] = -Rd * np.asarray(u_ref, np.float64).reshape(-1)
    Eq = np.zeros(((N + 1) * nx, nw))
    be = np.zeros((N + 1) * nx)
    Eq[:nx, :nx] = np.eye(nx)
    be[:nx] = x0
    for k in range(N):
        r = (k + 1) * nx
        Eq[r:r + nx, (k + 1) * nx:(k + 2) * nx] = np.eye(nx)
        Eq[r:r + nx, k * nx:(k + 1) * nx] = -A[k]
        Eq[r:r + nx, nX + k * nu:nX + (k + 1) * nu] = -B[k]
        be[r:r + nx] = c[k]
    rows, lows, highs = [], [], []
    for k in range(N):
        for a in range(nu):
            e = np.zeros(nw); e[nX + k * nu + a] = 1.0
            rows.append(e); lows.append(lo[k, a]); highs.append(hi[k, a])
    n_c = 0 if Cx is None else Cx.shape[2]
    for k in range(1, N + 1):
        for i in range(M):
            for s in range(n_c):
                e = np.zeros(nw)
                e[k * nx + 6 * i:k * nx + 6 * i + 3] = Cx[k - 1, i, s]
                rows.append(e); lows.append(-np.inf); highs.append(dx[k - 1, i, s])
    G = np.array(rows)
    lw, hw = np.array(lows), np.array(highs)
    m = G.shape[0]
    choices = [((0, 1, 2) if np.isfinite(lw[r]) else (0, 1)) for r in range(m)]
    for pick in itertools.product(*choices):
        act = [r for r in range(m) if pick[r] != 0]
        bnd = np.array([hw[r] if pick[r] == 1 else lw[r] for r in act])
        Ga = np.vstack([Eq] + ([G[act]] if act else []))
        ba = np.concatenate([be, bnd]) if act else be
        K = np.block([[P, Ga.T], [Ga, np.zeros((Ga.shape[0], Ga.shape[0]))]])
        try:
            sol = np.linalg.solve(K, np.concatenate([-q, ba]))
        except np.linalg.LinAlgError:
            continue
        w = sol[:nw]
        lam = sol[nw + Eq.shape[0]:]
        a = G @ w
        if np.any(a > hw + tol) or np.any(a < lw - tol):
            continue
        sgn = np.array([1.0 if pick[r] == 1 else -1.0 for r in act])
        if act and np.any(sgn * lam < -tol):
            continue
        return w[nX:].reshape(N, nu)
    return None
