"""Plain FP64 oracle of the Scaling Algorithm for OTLM (Algorithm 1) and its objective.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and bench.py's CPU legs,
never by the product path.  Slow and direct on purpose: every step is the paper's formula with
numpy/scipy primitives (matmul, exp/log, logsumexp, Lambert W) and no blocking or fusion.

Notation (paper, Sec. 3): X [N, M] non-negative dictionary, w [M] weights, y [N] target,
C [N, N] cost, K = exp(-C/eps) (Sec. 2.2), u1 target-side scaling (starts at 1), u2 source-side
scaling.  The plan is Q_ij = u2_i K_ij u1_j, so Q 1 = u2 * (K u1) and Q^T 1 = u1 * (K^T u2).

Readings of passages the paper leaves garbled or open:
  A1  objective: eps KL(Q||K) + lam L(Q^T 1 | y) + alpha R(w) with Q 1 = X w (the <C,Q> term
      printed beside eps KL(Q||K) would count the cost twice; Sec. 2.3 / Eq. OTLM).
  A2  Q_ij = u2_i K_ij u1_j (u2 scales the source rows; Sec. 2.3 updates, Algorithm 1).
  A3  Table 2, no penalty: the sum over i is restored inside the exponent.
  A4  Table 2, l1: the shift is alpha/(eps x_j), as derived in App. A (equal to alpha/eps when
      columns have unit mass).
  A5  Table 2, squared l2: w_j = W0(c_j e^{nu_j}) / c_j, c_j = alpha/(eps x_j), from App. A
      (ln w_j + c_j w_j = nu_j); R(w) = (alpha/2)||w||^2.
  A7  Table 1, Poisson: with L(s | y) = sum (s - y log s) (App. B's definition), stationarity of
      lam L(v | y) + eps KL(v || b) is eps log(v / b) + lam - lam y / v = 0 (App. B prints the
      sign of the lam term flipped; its next line follows the correct one), so u = lam y / (eps v)
      solves u e^u = (lam y / (eps b)) e^{lam / eps} and v = (lam y / eps) / W0(...): Table 1's
      "W0^{-1}" is read as the reciprocal 1 / W0.  For y = 0 the prox is b e^{-lam / eps}.
  A8  "not converged" (Algorithm 1): source-marginal violation
      e = ||u2 * (K u1) - X w||_1 / ||X w||_1, measured with the u1 of the next iteration; the
      weight change ||w_new - w_old||_1 / ||w_new||_1 and the duality gap of the current state
      are reported beside it and may be required as well (every enabled criterion must hold).
  A6  Table 2, elastic net alpha l1 + (beta/2) l2^2: Table 2 prints the prefactor alpha/beta and a
      y_j inside the sum; App. A's stationarity condition ln w_j + gamma_j w_j = nu_j with
      gamma_j = beta/(eps x_j) and nu_j shifted by -alpha/(eps x_j) is followed instead:
      w_j = W0(gamma_j e^{nu_j - alpha/(eps x_j)}) / gamma_j.
  A11 zeros: rows with (X w)_i = 0 contribute nothing to the MM sum (0 log 0 = 0), y_j = 0
      gives u1_j = 0 under the KL datafit.
  A18 more than one MM step per outer iteration (Sec. 4.2 allows running the MM iteration for
      prox_{alpha P}(K u1 | X) longer than one step): every inner step uses the same a = K u1 and
      its own previous w; the source step u2 = X w / a follows the last inner step.
"""
from __future__ import annotations

import numpy as np
from scipy.sparse import issparse
from scipy.special import lambertw, logsumexp, wrightomega

DATAFITS = ("balanced", "kl", "tv", "l2", "poisson")
PENALTIES = ("none", "l1", "l2sq", "elastic")


# ---------------------------------------------------------------------------------------------
# Building blocks (Sec. 2.2, Table 1, Table 2)
# ---------------------------------------------------------------------------------------------

def gibbs_kernel(C, eps):
    """K = exp(-C / eps), the Gibbs kernel of the entropic OT problem (Sec. 2.2)."""
    return np.exp(-np.asarray(C, dtype=np.float64) / eps)


def generalized_kl(P, R):
    """Generalised KL divergence, Eq. (generalized_kl): sum P log(P/R) - P + R, 0 log 0 = 0."""
    P = np.asarray(P, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        plogp = np.where(P > 0, P * np.log(P / R), 0.0)
    return float(np.sum(plogp - P + R))


def lambert_w0(z):
    """Principal branch W0 of the Lambert W function (library primitive: scipy)."""
    return np.real(lambertw(np.asarray(z, dtype=np.float64), 0))


def wright_omega(z):
    """Wright omega: omega(z) = W0(e^z) for real z (library primitive: scipy)."""
    return np.real(wrightomega(np.asarray(z, dtype=np.float64)))


def datafit_loss(datafit, t, y):
    """L(t | y) without the weight lam (Sec. 1 notation; Table 1 rows)."""
    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if datafit == "balanced":
        return 0.0 if np.allclose(t, y, rtol=1e-12, atol=0) else np.inf
    if datafit == "kl":
        return generalized_kl(t, y)
    if datafit == "tv":
        return float(np.sum(np.abs(t - y)))
    if datafit == "l2":
        return 0.5 * float(np.sum((t - y) ** 2))
    if datafit == "poisson":
        # negative Poisson log-likelihood without its constant (reading A7); y log t = 0 where y = 0
        with np.errstate(divide="ignore", invalid="ignore"):
            ylogt = np.where(y > 0, y * np.log(t), 0.0)
        return float(np.sum(t - ylogt))
    raise ValueError(datafit)


def penalty_value(penalty, w):
    """R(w): none -> 0, l1 -> sum w, l2sq -> (1/2)||w||^2 (Table 2 rows; w >= 0)."""
    w = np.asarray(w, dtype=np.float64)
    if penalty == "none":
        return 0.0
    if penalty == "l1":
        return float(np.sum(np.abs(w)))
    if penalty == "l2sq":
        return 0.5 * float(np.sum(w * w))
    raise ValueError(penalty)


def penalty_term(penalty, w, alpha, beta=0.0):
    """The weighted penalty of the objective: alpha R(w) for none / l1 / l2sq, and
    alpha ||w||_1 + (beta/2) ||w||^2 for the elastic net (Table 2, last row)."""
    if penalty == "elastic":
        return alpha * penalty_value("l1", w) + beta * penalty_value("l2sq", w)
    return alpha * penalty_value(penalty, w)


def prox_datafit(datafit, s, y, eps, lam):
    """prox^KL_{lam L}(s | y), Table 1, linear form."""
    s = np.asarray(s, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if datafit == "balanced":
        return y.copy()
    if datafit == "kl":
        return s ** (eps / (eps + lam)) * y ** (lam / (eps + lam))
    if datafit == "tv":
        return np.minimum(s * np.exp(lam / eps), np.maximum(s * np.exp(-lam / eps), y))
    if datafit == "l2":
        return (eps / lam) * lambert_w0((lam / eps) * s * np.exp((lam / eps) * y))
    if datafit == "poisson":
        c = lam * y / eps
        with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
            v = c / lambert_w0(c / s * np.exp(lam / eps))
        return np.where(y > 0, v, s * np.exp(-lam / eps))
    raise ValueError(datafit)


def _Z(X, w_prev):
    """Z_ij = X_ij w'_j / sum_k X_ik w'_k (Table 2 caption); 0 where X_ij w'_j = 0."""
    num = X * w_prev[None, :]
    den = num.sum(axis=1, keepdims=True)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(num > 0, num / den, 0.0)


def mm_step(penalty, a, w_prev, X, eps, alpha, beta=0.0):
    """One MM step wMMstep^KL_P(a, Z | X), Table 2 with the App. A readings A3-A6.

    `a` takes the place of y in Table 2 (Algorithm 1 calls it with K u1).  With
    L_j = sum_i X_ij log(Z_ij a_i / X_ij) (terms with X_ij = 0 dropped, 0 log 0 = 0) and the
    column mass x_j = sum_i X_ij:
        none : w_j = exp(L_j / x_j)
        l1   : w_j = exp(L_j / x_j - alpha / (eps x_j))
        l2sq : w_j = W0(c_j exp(L_j / x_j)) / c_j,   c_j = alpha / (eps x_j)
        elastic: w_j = W0(g_j exp(L_j / x_j - alpha / (eps x_j))) / g_j,   g_j = beta / (eps x_j)
    """
    X = np.asarray(X, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    w_prev = np.asarray(w_prev, dtype=np.float64)
    Z = _Z(X, w_prev)
    x = X.sum(axis=0)
    with np.errstate(divide="ignore", invalid="ignore"):
        terms = np.where(X > 0, X * np.log(Z * a[:, None] / X), 0.0)
    nu = terms.sum(axis=0) / x
    if penalty == "none":
        return np.exp(nu)
    if penalty == "l1":
        return np.exp(nu - alpha / (eps * x))
    if penalty == "l2sq":
        c = alpha / (eps * x)
        return lambert_w0(c * np.exp(nu)) / c
    if penalty == "elastic":
        gam = beta / (eps * x)
        return lambert_w0(gam * np.exp(nu - alpha / (eps * x))) / gam
    raise ValueError(penalty)


def mm_step_log(penalty, log_a, w_prev, X, eps, alpha, beta=0.0):
    """The same MM step written with log a instead of a (for kernels that underflow).

    Since Z_ij a_i / X_ij = w'_j a_i / s_i with s = X w' (wherever X_ij > 0), Table 2's
    exponent becomes nu_j = log w'_j + (1/x_j) sum_{i: s_i > 0} X_ij (log a_i - log s_i).
    The squared-l2 update is evaluated as omega(log c_j + nu_j) / c_j, which equals
    W0(c_j e^{nu_j}) / c_j but never overflows.  X may be a dense array or a scipy.sparse matrix
    (the products X w and X^T r are the same either way).
    """
    X = X if issparse(X) else np.asarray(X, dtype=np.float64)
    w_prev = np.asarray(w_prev, dtype=np.float64)
    s = X @ w_prev
    x = np.asarray(X.sum(axis=0), dtype=np.float64).ravel()
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(s > 0, log_a - np.log(np.where(s > 0, s, 1.0)), 0.0)
        nu = np.log(w_prev) + (X.T @ r) / x
    if penalty == "none":
        return np.exp(nu)
    if penalty == "l1":
        return np.exp(nu - alpha / (eps * x))
    if penalty == "l2sq":
        c = alpha / (eps * x)
        out = wright_omega(np.log(c) + nu) / c
        return np.where(np.isneginf(nu), 0.0, out)
    if penalty == "elastic":
        gam = beta / (eps * x)
        out = wright_omega(np.log(gam) + nu - alpha / (eps * x)) / gam
        return np.where(np.isneginf(nu), 0.0, out)
    raise ValueError(penalty)


def majorizer_G(w, w_prev, a, X, eps, alpha, penalty, beta=0.0):
    """G(w, w') of Eq. (obj_nnsx_majorized), with a in place of y.

    G = eps sum_ij Z_ij ( (X_ij w_j / Z_ij) log(X_ij w_j / (Z_ij a_i)) - X_ij w_j / Z_ij + a_i )
        + alpha R(w)   (the elastic net's alpha l1 + (beta/2) l2^2 for "elastic"),
    summed over the pairs with Z_ij > 0.
    """
    X = np.asarray(X, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    Z = _Z(X, np.asarray(w_prev, dtype=np.float64))
    total = 0.0
    for i in range(X.shape[0]):
        for j in range(X.shape[1]):
            if Z[i, j] <= 0:
                continue
            q = X[i, j] * w[j] / Z[i, j]
            term = (q * np.log(q / a[i]) if q > 0 else 0.0) - q + a[i]
            total += Z[i, j] * term
    return eps * total + penalty_term(penalty, w, alpha, beta)


def prox_objective_V(w, a, X, eps, alpha, penalty, beta=0.0):
    """V(w) = alpha R(w) + eps KL(X w || a), the objective of Eq. (ProxP) (Sec. 4.1)."""
    return penalty_term(penalty, w, alpha, beta) + eps * generalized_kl(np.asarray(X) @ np.asarray(w), a)


# ---------------------------------------------------------------------------------------------
# Algorithm 1, linear and log domain
# ---------------------------------------------------------------------------------------------

def marginal_violation(s, u2, a):
    """e = || u2 * a - s ||_1 / || s ||_1 with a = K u1 (reading A8)."""
    return float(np.sum(np.abs(u2 * a - s)) / np.sum(s))


def solve(C, X, y, eps, lam, alpha, datafit, penalty, w0, n_iter, tol=0.0, beta=0.0, mm_steps=1):
    """Algorithm 1 (Scaling Algorithm for OTLM) in the linear domain, FP64.

    Per iteration, in the paper's order: a = K u1; Z from the previous w; w <- wMMstep(a, Z|X)
    (`mm_steps` times with the same a, reading A18; one step in Algorithm 1);
    u2 = X w / a; b = K^T u2; v2 = prox_L(b | y); u1 = v2 / b.  `beta` is the elastic net's
    squared-l2 weight (ignored by the other penalties).
    Before every iteration after the first, the source-marginal violation of the current plan
    (reading A8) is measured with the new a = K u1; when tol > 0 and it is <= tol the loop
    stops and the state of the last completed iteration is returned (tol <= 0: run n_iter).

    Returns dict(w, u1, u2, Q, iters, err, err_hist, t=Q^T 1, s=Q 1).
    """
    C = np.asarray(C, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    K = gibbs_kernel(C, eps)
    u1 = np.ones(C.shape[1])
    u2 = None
    w = np.asarray(w0, dtype=np.float64).copy()
    s = None
    err = np.nan
    hist = []
    it = 0
    for it in range(n_iter + 1):
        a = K @ u1
        if it > 0:
            err = marginal_violation(s, u2, a)
            hist.append(err)
            if tol > 0 and err <= tol:
                break
        if it == n_iter:
            break
        for _ in range(mm_steps):
            w = mm_step(penalty, a, w, X, eps, alpha, beta)
        s = X @ w
        u2 = s / a
        b = K.T @ u2
        v2 = prox_datafit(datafit, b, y, eps, lam)
        with np.errstate(divide="ignore", invalid="ignore"):
            u1 = np.where(b > 0, v2 / b, 0.0)
    Q = u2[:, None] * K * u1[None, :]
    return dict(w=w, u1=u1, u2=u2, Q=Q, iters=it, err=err, err_hist=np.array(hist),
                t=Q.sum(axis=0), s=Q.sum(axis=1))


def _log_datafit_potential(datafit, log_b, y, eps, lam):
    """g = eps log(v2 / b) for v2 = prox_L(b | y), Table 1 rewritten with log b.

    balanced: g = eps (log y - log b)
    kl      : g = (eps lam / (eps + lam)) (log y - log b)
    tv      : g = clip(eps (log y - log b), -lam, lam)
    l2      : log v2 = log(eps/lam) + log omega(log(lam/eps) + log b + (lam/eps) y)
              (W0(e^z) = omega(z)), g = eps (log v2 - log b)
    poisson : log v2 = log(lam y/eps) - log omega(log(lam y/eps) - log b + lam/eps) for y > 0,
              g = -lam for y = 0 (reading A7)
    """
    with np.errstate(divide="ignore"):
        log_y = np.log(y)
    if datafit == "balanced":
        return eps * (log_y - log_b)
    if datafit == "kl":
        return (eps * lam / (eps + lam)) * (log_y - log_b)
    if datafit == "tv":
        return np.clip(eps * (log_y - log_b), -lam, lam)
    if datafit == "l2":
        z = np.log(lam / eps) + log_b + (lam / eps) * y
        log_v = np.log(eps / lam) + np.log(wright_omega(z))
        return eps * (log_v - log_b)
    if datafit == "poisson":
        with np.errstate(divide="ignore", invalid="ignore"):
            lc = np.log(lam * y / eps)
            g = eps * (lc - np.log(wright_omega(lc - log_b + lam / eps)) - log_b)
        return np.where(y > 0, g, -lam)
    raise ValueError(datafit)


def solve_log(C, X, y, eps, lam, alpha, datafit, penalty, w0, n_iter, tol=0.0, g0=None, beta=0.0, mm_steps=1,
              dw_tol=0.0, check_every=0, gap_tol=0.0):
    """Algorithm 1 with the scalings carried as potentials g = eps log u1, f = eps log u2.

    log (K u1)_i = LSE_j((g_j - C_ij)/eps), log (K^T u2)_j = LSE_i((f_i - C_ij)/eps); the MM step
    is `mm_step_log`; f = eps (log X w - log K u1) (-inf where X w = 0); g from
    `_log_datafit_potential`.  Same stopping rule, `beta`, `mm_steps` and outputs as `solve`, plus
    f, g, log_a and dw_hist (||w_new - w_old||_1 / ||w_new||_1 of every weight update).

    Further stopping criteria (reading A8 reports the weight change and the duality gap beside the
    violation; here they may also be required): with dw_tol > 0 a stop also needs the last update's
    weight change <= dw_tol; with gap_tol > 0 it needs, at an iteration that is a multiple of
    check_every, primal - dual <= gap_tol |primal| for the state (w, g) it would return
    (`objective_and_dual`).  Every enabled criterion must hold at the same iteration; gap_hist
    lists (iteration, primal, dual) of the checks.
    """
    C = np.asarray(C, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    g = np.zeros(C.shape[1]) if g0 is None else np.asarray(g0, dtype=np.float64).copy()
    f = None
    w = np.asarray(w0, dtype=np.float64).copy()
    s = None
    err = np.nan
    hist, dw_hist, gap_hist = [], [], []
    any_rule = tol > 0 or dw_tol > 0 or gap_tol > 0
    it = 0
    log_a = None
    for it in range(n_iter + 1):
        log_a = logsumexp((g[None, :] - C) / eps, axis=1)
        if it > 0:
            # u2 * K u1 = s * exp(log a_new - log a_old)
            err = float(np.sum(np.abs(s * np.expm1(log_a - log_a_old))) / np.sum(s))
            hist.append(err)
            gap_ok = True
            if gap_tol > 0:
                gap_ok = False
                if check_every > 0 and it % check_every == 0:
                    P, Dv, _ = objective_and_dual(w, g, C, X, y, eps, lam, alpha, datafit, penalty, beta)
                    gap_hist.append((it, P, Dv))
                    gap_ok = P - Dv <= gap_tol * abs(P)
            if (any_rule and (tol <= 0 or err <= tol) and (dw_tol <= 0 or dw_hist[-1] <= dw_tol) and gap_ok):
                break
        if it == n_iter:
            break
        w_prev = w
        for _ in range(mm_steps):
            w = mm_step_log(penalty, log_a, w, X, eps, alpha, beta)
        dw_hist.append(float(np.sum(np.abs(w - w_prev)) / np.sum(np.abs(w))))
        s = X @ w
        with np.errstate(divide="ignore"):
            f = eps * (np.log(s) - log_a)
        log_a_old = log_a
        log_b = logsumexp((f[:, None] - C) / eps, axis=0)
        g = _log_datafit_potential(datafit, log_b, y, eps, lam)
    # plan of the returned state: u2 from the last source step, u1 from the last target step
    with np.errstate(invalid="ignore"):
        logQ = (f[:, None] + g[None, :] - C) / eps
    Q = np.exp(logQ)
    return dict(w=w, f=f, g=g, Q=Q, iters=it, err=err, err_hist=np.array(hist), dw_hist=np.array(dw_hist),
                gap_hist=gap_hist, t=Q.sum(axis=0), s=Q.sum(axis=1), log_a=log_a)


def solve_converged(C, X, y, eps, lam, alpha, datafit, penalty, w0, rtol_w=1e-14, max_iter=10 ** 6, g0=None,
                    beta=0.0, mm_steps=1):
    """The long-run solution: Algorithm 1 (log domain) continued from (w0, g0) one iteration at a
    time until ||w_new - w||_1 / ||w_new||_1 < rtol_w or max_iter iterations.  The marginal
    violation of reading A8 reaches small tolerances long before w settles, so this is the
    reference for the solution quality of a solve stopped at tol.

    Returns dict(w, g, t, iters, dw) with dw the last relative change of w.
    """
    w = np.asarray(w0, dtype=np.float64).copy()
    g = None if g0 is None else np.asarray(g0, dtype=np.float64).copy()
    dw = np.inf
    r = None
    it = 0
    while it < max_iter:
        r = solve_log(C, X, y, eps, lam, alpha, datafit, penalty, w, 1, g0=g, beta=beta, mm_steps=mm_steps)
        it += 1
        dw = float(np.sum(np.abs(r["w"] - w)) / np.sum(np.abs(r["w"])))
        w, g = r["w"], r["g"]
        if dw < rtol_w:
            break
    return dict(w=w, g=g, t=r["t"], iters=it, dw=dw)


def band_to_dense(Cd, h):
    """Dense C [n, n] from the diagonal (DIA) storage Cd [2h+1, n] of a banded cost:
    C_{i, i+d-h} = Cd[d, i]; every pair outside the band, or stored as +inf, is forbidden
    (C = +inf, K = 0)."""
    Cd = np.asarray(Cd, dtype=np.float64)
    n = Cd.shape[1]
    C = np.full((n, n), np.inf)
    for d in range(2 * h + 1):
        for i in range(n):
            j = i + d - h
            if 0 <= j < n:
                C[i, j] = Cd[d, i]
    return C


def _band_lse_rows(v, Cd, h, eps):
    """log sum_j exp((v_j - C_ij) / eps) over the band of row i: j = i + d - h."""
    n = v.shape[0]
    terms = np.full((n, 2 * h + 1), -np.inf)
    for d in range(2 * h + 1):
        lo, hi = max(0, h - d), min(n, n + h - d)  # rows whose j = i + d - h lies in [0, n)
        i = np.arange(lo, hi)
        with np.errstate(invalid="ignore"):
            terms[i, d] = (v[i + d - h] - Cd[d, i]) / eps
    return logsumexp(terms, axis=1)


def _band_lse_cols(v, Cd, h, eps):
    """log sum_i exp((v_i - C_ij) / eps) over the band of column j: i = j + e - h, whose cost
    C_{i, j} sits in diagonal 2h - e of row i."""
    n = v.shape[0]
    terms = np.full((n, 2 * h + 1), -np.inf)
    for e in range(2 * h + 1):
        lo, hi = max(0, h - e), min(n, n + h - e)
        j = np.arange(lo, hi)
        i = j + e - h
        with np.errstate(invalid="ignore"):
            terms[j, e] = (v[i] - Cd[2 * h - e, i]) / eps
    return logsumexp(terms, axis=1)


def solve_log_banded(Cd, h, X, y, eps, lam, alpha, datafit, penalty, w0, n_iter, tol=0.0, g0=None, beta=0.0,
                     mm_steps=1):
    """`solve_log` for a banded cost given in diagonal storage (C = +inf off the band: K_ij = 0
    there, so the sums of Algorithm 1 run over the band only) and a dictionary X that may be a
    scipy.sparse matrix.  Same iteration, stopping rule, arguments and outputs as `solve_log`,
    except Q, which is not formed."""
    Cd = np.asarray(Cd, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    g = np.zeros(y.shape[0]) if g0 is None else np.asarray(g0, dtype=np.float64).copy()
    f = None
    w = np.asarray(w0, dtype=np.float64).copy()
    s = None
    err = np.nan
    hist = []
    it = 0
    log_a = None
    log_b = None
    for it in range(n_iter + 1):
        log_a = _band_lse_rows(g, Cd, h, eps)
        if it > 0:
            err = float(np.sum(np.abs(s * np.expm1(log_a - log_a_old))) / np.sum(s))
            hist.append(err)
            if tol > 0 and err <= tol:
                break
        if it == n_iter:
            break
        for _ in range(mm_steps):
            w = mm_step_log(penalty, log_a, w, X, eps, alpha, beta)
        s = X @ w
        with np.errstate(divide="ignore"):
            f = eps * (np.log(s) - log_a)
        log_a_old = log_a
        log_b = _band_lse_cols(f, Cd, h, eps)
        g = _log_datafit_potential(datafit, log_b, y, eps, lam)
    # t = Q^T 1 = u1 * K^T u2 of the returned state
    t = np.exp(g / eps + log_b) if log_b is not None else None
    return dict(w=w, f=f, g=g, iters=it, err=err, err_hist=np.array(hist), t=t, s=s, log_a=log_a)


# ---------------------------------------------------------------------------------------------
# Objective (reading A1) and a Fenchel dual lower bound
# ---------------------------------------------------------------------------------------------

def primal_objective(Q, w, C, y, eps, lam, alpha, datafit, penalty, beta=0.0):
    """eps KL(Q || K) + lam L(Q^T 1 | y) + alpha R(w) (Eq. OTLM, reading A1).

    The caller guarantees Q 1 = X w (the constraint of the second form of Eq. OTLM).
    """
    K = gibbs_kernel(C, eps)
    t = np.asarray(Q).sum(axis=0)
    lt = datafit_loss(datafit, t, y)
    return (eps * generalized_kl(Q, K) + (lam * lt if datafit != "balanced" else lt)
            + penalty_term(penalty, w, alpha, beta))


def _F2_conj_neg(datafit, g, y, lam):
    """F2*(-g) for F2 = lam L(. | y) on t >= 0 (convex conjugate, per datafit)."""
    y = np.asarray(y, dtype=np.float64)
    if datafit == "balanced":
        # <-g, y> over the bins with y > 0; a bin with y = 0 contributes 0 whatever g is
        with np.errstate(invalid="ignore"):
            return -float(np.sum(np.where(y > 0, g * y, 0.0)))
    if datafit == "kl":
        # lam sum y (e^{-g/lam} - 1); a bin with y = 0 contributes 0 whatever g is
        with np.errstate(over="ignore", invalid="ignore"):
            v = np.where(y > 0, y * np.expm1(-g / lam), 0.0)
        return lam * float(np.sum(v))
    if datafit == "tv":
        if np.any(g < -lam * (1 + 1e-12)):
            return np.inf
        return -float(np.sum(y * np.minimum(g, lam)))
    if datafit == "l2":
        inside = y - g / lam >= 0
        return float(np.sum(np.where(inside, -g * y + g * g / (2 * lam), -lam * y * y / 2)))
    if datafit == "poisson":
        # sup_t (-g t - lam t + lam y log t): finite only for g > -lam (y > 0) or g >= -lam (y = 0);
        # at t = lam y / (lam + g) it is lam y (log(lam y / (lam + g)) - 1)
        if np.any((y > 0) & (g <= -lam)) or np.any((y == 0) & (g < -lam * (1 + 1e-12))):
            return np.inf
        with np.errstate(divide="ignore", invalid="ignore"):
            v = np.where(y > 0, lam * y * (np.log(lam * y / (lam + g)) - 1.0), 0.0)
        return float(np.sum(v))
    raise ValueError(datafit)


def _F1_conj_neg(penalty, f, X, alpha, beta=0.0):
    """F1*(-f) = (alpha R + indicator(w >= 0))^*(-X^T f), F1(s) = alpha P_R(s | X) (Eq. P).

    Per column, sup_{w >= 0} (v w - h(w)) with v = -(X^T f)_j: 0 or +inf for h = alpha w (v <= alpha)
    and h = 0 (v <= 0); v+^2 / (2 alpha) for h = alpha w^2 / 2; (v - alpha)+^2 / (2 beta) for the
    elastic net h = alpha w + beta w^2 / 2.

    Rows of X that are entirely zero do not enter X^T f (0 * (-inf) taken as 0).
    """
    X = np.asarray(X, dtype=np.float64)
    with np.errstate(invalid="ignore"):
        prod = np.where(X > 0, X * f[:, None], 0.0)
    v = -prod.sum(axis=0)  # v = -X^T f
    # the feasibility tests allow a rounding slack of 1e-12 relative to the column mass
    slack = 1e-12 * (np.abs(prod).sum(axis=0) + alpha)
    if penalty == "none":
        return 0.0 if np.all(v <= slack) else np.inf
    if penalty == "l1":
        return 0.0 if np.all(v <= alpha + slack) else np.inf
    if penalty == "l2sq":
        return float(np.sum(np.maximum(v, 0.0) ** 2) / (2 * alpha))
    if penalty == "elastic":
        return float(np.sum(np.maximum(v - alpha, 0.0) ** 2) / (2 * beta))
    raise ValueError(penalty)


def dual_objective(f, g, C, X, y, eps, lam, alpha, datafit, penalty, beta=0.0):
    """D(f, g) = -F1*(-f) - F2*(-g) - eps sum_ij K_ij (e^{(f_i + g_j)/eps} - 1).

    For the l1 / unpenalised cases a constant shift f <- f + c 1 (c >= 0, the smallest that makes
    X^T f >= -alpha, resp. >= 0) restores dual feasibility; D stays a valid lower bound.
    """
    C = np.asarray(C, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    # A row whose source mass underflowed to 0 carries f = -inf; if the dictionary is non-zero
    # there, -inf would make X^T f infinite.  Any finite f is admissible in the dual, so such
    # rows take the smallest finite f instead (rows where X is entirely zero keep -inf).
    bad = np.isneginf(f) & (X.sum(axis=1) > 0)
    if np.any(bad):
        f = np.where(bad, np.min(f[np.isfinite(f)]), f)
    if datafit == "poisson":
        # any g > -lam is dual-feasible at a bin with y > 0; a prox step at a bin with tiny y leaves
        # g within rounding of -lam (g + lam = lam y / v), so such g are moved to -lam (1 - 2^-50),
        # which keeps D a lower bound and changes the entropic term by ~lam 2^-50 / eps
        gmin = -lam * (1.0 - 2.0 ** -50)
        g = np.where((np.asarray(y) > 0) & (g < gmin), gmin, g)
    if penalty in ("l1", "none"):
        bound = alpha if penalty == "l1" else 0.0
        with np.errstate(invalid="ignore"):
            xtf = np.where(X > 0, X * f[:, None], 0.0).sum(axis=0)
        x = X.sum(axis=0)
        c = float(np.max(np.maximum(0.0, (-bound - xtf) / x)))
        f = f + c
    K = gibbs_kernel(C, eps)
    with np.errstate(invalid="ignore", over="ignore"):
        E = np.exp((f[:, None] + g[None, :]) / eps)
    ent = eps * float(np.sum(K * E) - np.sum(K))
    return -_F1_conj_neg(penalty, f, X, alpha, beta) - _F2_conj_neg(datafit, g, y, lam) - ent


def objective_and_dual(w, g, C, X, y, eps, lam, alpha, datafit, penalty, beta=0.0):
    """Primal value, dual value and their plan, evaluated from a solver state (w, g).

    From (w, g): a = K u1 (u1 = e^{g/eps}), s = X w, f = eps log(s / a); the plan
    Q = diag(e^{f/eps}) K diag(e^{g/eps}) has Q 1 = X w exactly, so (Q, w) is feasible and gives
    the primal value.  The dual is evaluated at (f, g') with g' the datafit step from
    b = K^T u2, i.e. the g the next iteration would use.
    """
    C = np.asarray(C, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    log_a = logsumexp((g[None, :] - C) / eps, axis=1)
    s = X @ w
    with np.errstate(divide="ignore"):
        f = eps * (np.log(s) - log_a)
    Q = np.exp((f[:, None] + g[None, :] - C) / eps)
    P = primal_objective(Q, w, C, y, eps, lam, alpha, datafit, penalty, beta)
    log_b = logsumexp((f[:, None] - C) / eps, axis=0)
    g_next = _log_datafit_potential(datafit, log_b, y, eps, lam)
    Dv = dual_objective(f, g_next, C, X, y, eps, lam, alpha, datafit, penalty, beta)
    return P, Dv, Q
