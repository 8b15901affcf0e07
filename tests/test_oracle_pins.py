"""Pins of the FP64 oracle against facts the paper and the mathematics fix (CPU only).

Each test checks one oracle function against something other than itself: a closed form, a
textbook algorithm written out here, a 1-D numerical minimisation, a brute-force convex solve, or
an invariant.  Chosen so that a dropped term, a wrong sign, a swapped index or a transposed
operand in the oracle fails at least one of them (see also test_oracle_mutations.py).
"""
import numpy as np
import pytest
from scipy.optimize import brentq, minimize, minimize_scalar

import oracle
import spectra

EPS = 2e-2
BETA = 0.04  # the elastic net's squared-l2 weight; ignored by the other penalties


def _tiny(n=5, k=2, seed=0, symmetric=False):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.05, 1.0, size=(n, k))
    X /= X.sum(axis=0, keepdims=True)
    y = rng.uniform(0.1, 0.6, size=n)
    if symmetric:
        x = np.linspace(0, 1, n)
        C = (x[:, None] - x[None, :]) ** 2
    else:
        C = rng.uniform(0.0, 0.08, size=(n, n))
        np.fill_diagonal(C, 0.0)
    return X, y, C


# --- Lambert W / Wright omega (library primitives; pinned by their defining identities) -------

def test_lambert_w0_defining_identity():
    z = np.concatenate([-np.exp(-1) + np.logspace(-12, -1, 12), np.linspace(-0.3, 0.0, 7),
                        np.logspace(-12, 250, 60)])
    W = oracle.lambert_w0(z)
    assert np.all(W >= -1.0)
    small = z < 10
    np.testing.assert_allclose(W[small] * np.exp(W[small]), z[small], rtol=2e-14, atol=1e-300)
    # for large z, exp(W) amplifies W's rounding by W: compare in the log form W + log W = log z
    np.testing.assert_allclose(W[~small] + np.log(W[~small]), np.log(z[~small]), rtol=1e-15)


def test_wright_omega_identity_and_relation_to_w0():
    z = np.linspace(-700, 700, 1401)
    om = oracle.wright_omega(z)
    np.testing.assert_allclose(om + np.log(om), z, rtol=1e-14, atol=1e-12)
    zs = np.linspace(-20, 20, 41)
    np.testing.assert_allclose(oracle.wright_omega(zs), oracle.lambert_w0(np.exp(zs)), rtol=1e-14)


# --- Generalised KL, Eq. (generalized_kl) ------------------------------------------------------

def test_generalized_kl_closed_forms():
    assert oracle.generalized_kl([2.0], [1.0]) == pytest.approx(2 * np.log(2) - 2 + 1, rel=1e-15)
    assert oracle.generalized_kl([0.0], [3.0]) == pytest.approx(3.0, rel=1e-15)  # 0 log 0 = 0
    p = np.array([0.3, 1.7, 0.0, 2.2])
    assert oracle.generalized_kl(p, p) == pytest.approx(0.0, abs=1e-15)
    rng = np.random.default_rng(1)
    for _ in range(20):
        a, b = rng.uniform(0.01, 3, 6), rng.uniform(0.01, 3, 6)
        assert oracle.generalized_kl(a, b) > 0


# --- Table 1: datafit proximal operators -------------------------------------------------------

def _prox_by_minimisation(datafit, b, y, eps, lam):
    """argmin_v lam L(v | y) + eps KL(v || b) over v > 0, solved numerically in log v."""
    def obj(lv):
        v = np.exp(lv)
        if datafit == "kl":
            L = v * np.log(v / y) - v + y
        elif datafit == "tv":
            L = abs(v - y)
        elif datafit == "poisson":
            L = v - y * np.log(v)
        else:
            L = 0.5 * (v - y) ** 2
        return lam * L + eps * (v * np.log(v / b) - v + b)
    lo, hi = np.log(min(b, y)) - 30 * eps / lam - 5, np.log(max(b, y)) + 5
    res = minimize_scalar(obj, bounds=(lo, hi), method="bounded", options=dict(xatol=1e-13, maxiter=2000))
    return np.exp(res.x)


@pytest.mark.parametrize("datafit", ["kl", "tv", "l2", "poisson"])
@pytest.mark.parametrize("eps,lam", [(0.05, 1.0), (0.5, 0.3), (1.0, 2.0)])
def test_prox_matches_1d_minimisation(datafit, eps, lam):
    rng = np.random.default_rng(7)
    for _ in range(12):
        b, y = rng.uniform(0.05, 2.0), rng.uniform(0.05, 2.0)
        got = float(oracle.prox_datafit(datafit, np.array([b]), np.array([y]), eps, lam)[0])
        ref = _prox_by_minimisation(datafit, b, y, eps, lam)
        assert got == pytest.approx(ref, rel=2e-6), (datafit, b, y)


def test_poisson_prox_at_zero_target_bins():
    """y = 0 leaves lam v + eps KL(v || b), minimised at v = b e^{-lam/eps}; the prox must reach
    that limit continuously as y -> 0."""
    b = np.array([0.3, 1.7])
    for eps, lam in ((0.05, 1.0), (0.5, 0.3)):
        v0 = oracle.prox_datafit("poisson", b, np.zeros(2), eps, lam)
        np.testing.assert_allclose(v0, b * np.exp(-lam / eps), rtol=1e-14)
        # v = v0 (1 + lam y / (eps v0) + ...): y = 1e-9 v0 moves it by ~1e-9 lam / eps
        v_small = oracle.prox_datafit("poisson", b, 1e-9 * v0, eps, lam)
        np.testing.assert_allclose(v_small, v0, rtol=1e-6)


def test_prox_balanced_is_target():
    y = np.array([0.2, 0.0, 1.5])
    np.testing.assert_array_equal(oracle.prox_datafit("balanced", np.array([3.0, 1.0, 2.0]), y, 0.1, 1.0), y)


@pytest.mark.parametrize("datafit", ["balanced", "kl", "tv", "l2", "poisson"])
def test_log_potential_equals_linear_prox(datafit):
    """The log-domain potential update equals eps log(prox(b)/b); the second setting makes
    the TV clamp bind (|eps log(y/b)| > lam for part of the bins)."""
    from oracle.otlm import _log_datafit_potential
    rng = np.random.default_rng(3)
    b, y = rng.uniform(0.01, 2.0, 50), rng.uniform(0.01, 2.0, 50)
    for eps, lam in ((0.05, 1.0), (0.8, 0.5)):
        g = _log_datafit_potential(datafit, np.log(b), y, eps, lam)
        ref = eps * np.log(oracle.prox_datafit(datafit, b, y, eps, lam) / b)
        np.testing.assert_allclose(g, ref, rtol=1e-11, atol=1e-13)


# --- Table 2 / App. A: the MM step --------------------------------------------------------------

@pytest.mark.parametrize("penalty", ["none", "l1", "l2sq", "elastic"])
def test_mm_step_minimises_majorizer(penalty):
    """G(w, w') is separable in w_j: coordinate-wise 1-D minimisation must give the MM step."""
    X, _, _ = _tiny(n=6, k=3, seed=2)
    X[0, 1] = 0.0  # an exact zero in the dictionary (0 log 0 = 0)
    rng = np.random.default_rng(5)
    a = rng.uniform(0.1, 1.0, 6)
    w_prev = rng.uniform(0.2, 2.0, 3)
    alpha = 0.05
    w = oracle.mm_step(penalty, a, w_prev, X, EPS, alpha, BETA)
    for j in range(3):
        def obj(lv, j=j):
            ww = w.copy()
            ww[j] = np.exp(lv)
            return oracle.majorizer_G(ww, w_prev, a, X, EPS, alpha, penalty, BETA)
        res = minimize_scalar(obj, bounds=(np.log(w[j]) - 3, np.log(w[j]) + 3), method="bounded",
                              options=dict(xatol=1e-12))
        assert np.exp(res.x) == pytest.approx(w[j], rel=1e-6)


@pytest.mark.parametrize("penalty", ["none", "l1", "l2sq", "elastic"])
def test_majorizer_majorises_and_touches(penalty):
    X, _, _ = _tiny(n=6, k=3, seed=4)
    rng = np.random.default_rng(6)
    a = rng.uniform(0.1, 1.0, 6)
    w_prev = rng.uniform(0.2, 2.0, 3)
    V = lambda w: oracle.prox_objective_V(w, a, X, EPS, 0.05, penalty, BETA)  # noqa: E731
    G = lambda w: oracle.majorizer_G(w, w_prev, a, X, EPS, 0.05, penalty, BETA)  # noqa: E731
    assert G(w_prev) == pytest.approx(V(w_prev), rel=1e-13)
    for _ in range(30):
        w = rng.uniform(0.0, 3.0, 3)
        assert G(w) >= V(w) - 1e-13


@pytest.mark.parametrize("penalty", ["none", "l1", "l2sq", "elastic"])
def test_repeated_mm_steps_decrease_V_to_the_proxP_minimum(penalty):
    """MM on Eq. (ProxP) with a fixed: V non-increasing, and the limit minimises V over w >= 0."""
    X, _, _ = _tiny(n=7, k=3, seed=8)
    rng = np.random.default_rng(9)
    a = rng.uniform(0.2, 1.0, 7)
    alpha = 0.01
    w = np.ones(3)
    vals = [oracle.prox_objective_V(w, a, X, EPS, alpha, penalty, BETA)]
    for _ in range(4000):
        w = oracle.mm_step(penalty, a, w, X, EPS, alpha, BETA)
        vals.append(oracle.prox_objective_V(w, a, X, EPS, alpha, penalty, BETA))
    assert np.all(np.diff(vals) <= 1e-13 * np.abs(vals[:-1]) + 1e-16)
    res = minimize(lambda lw: oracle.prox_objective_V(np.exp(lw), a, X, EPS, alpha, penalty, BETA),
                   np.log(w) + 0.3, method="Nelder-Mead", options=dict(xatol=1e-12, fatol=1e-15, maxiter=20000))
    assert vals[-1] <= res.fun + 1e-12
    np.testing.assert_allclose(w, np.exp(res.x), rtol=1e-4)


@pytest.mark.parametrize("penalty", ["none", "l1", "l2sq", "elastic"])
def test_mm_step_log_equals_linear(penalty):
    X, _, _ = _tiny(n=8, k=4, seed=10)
    X[2, :2] = 0.0
    rng = np.random.default_rng(11)
    a = rng.uniform(0.1, 1.0, 8)
    w_prev = rng.uniform(0.2, 2.0, 4)
    np.testing.assert_allclose(oracle.mm_step_log(penalty, np.log(a), w_prev, X, EPS, 0.03, BETA),
                               oracle.mm_step(penalty, a, w_prev, X, EPS, 0.03, BETA), rtol=1e-13)


def test_elastic_step_solves_its_stationarity_condition():
    """App. A: with w~_j the unpenalised MM step, the elastic-net step is the root of
    eps x_j ln(w_j / w~_j) + alpha + beta w_j = 0 (found here by bisection on ln w_j); alpha = 0
    gives the squared-l2 step with weight beta, and beta -> 0 the l1 step."""
    X, _, _ = _tiny(n=6, k=3, seed=14)
    X[:, 2] *= 2.5  # a column of mass 2.5: a prefactor that forgets x_j lands elsewhere
    rng = np.random.default_rng(15)
    a = rng.uniform(0.1, 1.0, 6)
    w_prev = rng.uniform(0.2, 2.0, 3)
    alpha, beta = 0.05, 0.3
    x = X.sum(axis=0)
    w = oracle.mm_step("elastic", a, w_prev, X, EPS, alpha, beta)
    wt = oracle.mm_step("none", a, w_prev, X, EPS, 0.0)
    for j in range(3):
        def h(lv, j=j):
            return EPS * x[j] * (lv - np.log(wt[j])) + alpha + beta * np.exp(lv)
        lo = np.log(wt[j]) - (alpha + beta * wt[j]) / (EPS * x[j]) - 1.0
        root = brentq(h, lo, np.log(wt[j]), xtol=1e-15, rtol=1e-15)
        assert w[j] == pytest.approx(np.exp(root), rel=1e-11)
    np.testing.assert_allclose(oracle.mm_step("elastic", a, w_prev, X, EPS, 0.0, beta),
                               oracle.mm_step("l2sq", a, w_prev, X, EPS, beta), rtol=1e-13)
    np.testing.assert_allclose(oracle.mm_step("elastic", a, w_prev, X, EPS, alpha, 1e-12),
                               oracle.mm_step("l1", a, w_prev, X, EPS, alpha), rtol=1e-8)


@pytest.mark.parametrize("penalty", ["l1", "elastic"])
def test_many_inner_mm_steps_give_the_weight_prox(penalty):
    """Reading A18 with many inner steps: the weights after the first outer iteration minimise
    V(w) = eps KL(X w | a) + penalty over w >= 0 for a = K 1 (u1 starts at 1); V and a are written
    out here and minimised by a generic bounded optimiser."""
    X, y, C = _tiny(n=6, k=3, seed=16)
    eps, alpha = 0.05, 0.02
    r = oracle.solve(C, X, y, eps, 1.0, alpha, "kl", penalty, np.ones(3), 1, beta=BETA, mm_steps=20000)
    a = np.exp(-C / eps) @ np.ones(6)

    def V(w):
        s = X @ w
        pen = alpha * w.sum() + (0.5 * BETA * (w * w).sum() if penalty == "elastic" else 0.0)
        return eps * np.sum(s * np.log(s / a) - s + a) + pen
    res = minimize(V, r["w"] * 1.3, method="L-BFGS-B", bounds=[(1e-12, None)] * 3,
                   options=dict(ftol=1e-16, gtol=1e-13, maxiter=20000))
    assert V(r["w"]) <= res.fun + 1e-13
    np.testing.assert_allclose(r["w"], res.x, rtol=1e-5)


# --- Algorithm 1 --------------------------------------------------------------------------------

def test_balanced_single_column_reduces_to_sinkhorn():
    """Balanced datafit, one dictionary column, no penalty: classic Sinkhorn between
    w*a and y; at the fixed point w = sum(y)/sum(a) and both marginals are met."""
    n = 12
    x = np.linspace(0, 1, n)
    rng = np.random.default_rng(12)
    col = rng.uniform(0.2, 1.0, n)
    col /= col.sum() * 0.8  # column mass 1.25
    y = rng.uniform(0.1, 1.0, n)
    C = np.abs(x[:, None] - x[None, :]) * 0.7 + rng.uniform(0, 0.05, (n, n))  # not symmetric
    eps = 0.1
    r = oracle.solve(C, col[:, None], y, eps, 1.0, 0.0, "balanced", "none", np.array([1.0]), 3000)
    w_expected = y.sum() / col.sum()
    assert r["w"][0] == pytest.approx(w_expected, rel=1e-12)
    # textbook Sinkhorn, written out independently: Q = diag(p) K diag(q)
    K = np.exp(-C / eps)
    mu, nu = col * w_expected, y
    q = np.ones(n)
    for _ in range(5000):
        p = mu / (K @ q)
        q = nu / (K.T @ p)
    Q_ref = p[:, None] * K * q[None, :]
    np.testing.assert_allclose(r["Q"], Q_ref, rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(r["t"], y, rtol=1e-12)
    np.testing.assert_allclose(r["s"], mu, rtol=1e-9)


def _brute_force_primal(X, y, C, eps, lam, alpha, datafit, penalty, beta=0.0):
    """Minimise eps KL(Q||K) + lam L(Q^T 1|y) + alpha R(w) s.t. Q 1 = X w, Q >= 0, w >= 0,
    with Q_ij = (X w)_i softmax_j(theta_i), w = exp(eta); gradients by torch autograd (FP64)."""
    import torch
    n, k = X.shape
    Xt, yt, Kt = (torch.tensor(v, dtype=torch.float64) for v in (X, y, np.exp(-C / eps)))

    def obj(z):
        th = z[: n * n].reshape(n, n)
        w = torch.exp(z[n * n:])
        Q = (Xt @ w)[:, None] * torch.softmax(th, dim=1)
        kl = torch.sum(Q * torch.log(Q / Kt) - Q + Kt)
        t = Q.sum(0)
        if datafit == "kl":
            L = torch.sum(t * torch.log(t / yt) - t + yt)
        elif datafit == "poisson":
            L = torch.sum(t - yt * torch.log(t))
        else:
            L = 0.5 * torch.sum((t - yt) ** 2)
        if penalty == "elastic":
            pen = alpha * torch.sum(w) + 0.5 * beta * torch.sum(w * w)
        else:
            pen = alpha * (torch.sum(w) if penalty == "l1" else 0.5 * torch.sum(w * w))
        return eps * kl + lam * L + pen

    def fg(zn):
        z = torch.tensor(zn, dtype=torch.float64, requires_grad=True)
        v = obj(z)
        v.backward()
        return v.item(), z.grad.numpy().copy()

    z0 = np.concatenate([-C.ravel() / eps, np.zeros(k)])
    res = minimize(fg, z0, jac=True, method="L-BFGS-B", options=dict(maxiter=50000, ftol=1e-16, gtol=1e-13))
    return np.exp(res.x[n * n:]), res.fun


@pytest.mark.parametrize("datafit,penalty,mm_steps", [("kl", "l2sq", 1), ("l2", "l1", 1), ("kl", "l1", 1),
                                                      ("l2", "l2sq", 1), ("kl", "elastic", 1), ("l2", "elastic", 3),
                                                      ("kl", "l1", 4), ("poisson", "l1", 1), ("poisson", "l2sq", 2)])
def test_brute_force_tiny_instance(datafit, penalty, mm_steps):
    """Same convex problem solved by a generic optimiser; C is not symmetric, so a transposed
    K or a swapped marginal in Algorithm 1 lands on a different w.  Several inner MM steps per
    outer iteration (reading A18) change the path, not the optimum."""
    X, y, C = _tiny(n=5, k=2, seed=13)
    eps, lam, alpha = 0.05, 1.0, 0.02
    r = oracle.solve(C, X, y, eps, lam, alpha, datafit, penalty, np.ones(2), 20000, tol=1e-15,
                     beta=BETA, mm_steps=mm_steps)
    w_bf, P_bf = _brute_force_primal(X, y, C, eps, lam, alpha, datafit, penalty, BETA)
    P = oracle.primal_objective(r["Q"], r["w"], C, y, eps, lam, alpha, datafit, penalty, BETA)
    assert P == pytest.approx(P_bf, rel=1e-9, abs=1e-12)
    np.testing.assert_allclose(r["w"], w_bf, rtol=2e-5)


@pytest.mark.parametrize("datafit", oracle.DATAFITS)
@pytest.mark.parametrize("penalty", oracle.PENALTIES)
def test_linear_and_log_domain_agree(datafit, penalty):
    d = spectra.batch(99, 1, 48, 5, 3, dtype=np.float64)
    C = spectra.squared_cost(d["x"])
    y = d["y"][0]
    w0 = spectra.initial_weights(y, d["D"])
    a = oracle.solve(C, d["D"], y, 0.03, 1.0, 0.01, datafit, penalty, w0, 60, beta=BETA, mm_steps=2)
    b = oracle.solve_log(C, d["D"], y, 0.03, 1.0, 0.01, datafit, penalty, w0, 60, beta=BETA, mm_steps=2)
    np.testing.assert_allclose(b["w"], a["w"], rtol=1e-11, atol=1e-300)
    np.testing.assert_allclose(b["t"], a["t"], rtol=1e-10, atol=1e-300)
    assert b["iters"] == a["iters"] == 60


@pytest.mark.parametrize("datafit,penalty", [("kl", "l2sq"), ("kl", "l1"), ("tv", "l1"), ("l2", "l2sq"), ("l2", "none"),
                                             ("kl", "elastic"), ("poisson", "l2sq")])
def test_invariants_along_the_trajectory(datafit, penalty):
    """w >= 0, Q >= 0, Q 1 = X w after the source step; primal objective non-increasing (observed,
    not proved in the paper: slack 1e-12 relative); weak duality P >= D at every iterate;
    gap -> 0 at convergence."""
    d = spectra.batch(98, 1, 40, 5, 3, dtype=np.float64)
    C = spectra.squared_cost(d["x"])
    y, X = d["y"][0], d["D"]
    eps, lam, alpha = 0.03, 1.0, 0.01
    w, g = spectra.initial_weights(y, X), np.zeros(40)
    prev = np.inf
    for _ in range(150):
        r = oracle.solve_log(C, X, y, eps, lam, alpha, datafit, penalty, w, 1, g0=g, beta=BETA)
        w, g = r["w"], r["g"]
        assert np.all(w >= 0) and np.all(r["Q"] >= 0)
        P, Dv, Q = oracle.objective_and_dual(w, g, C, X, y, eps, lam, alpha, datafit, penalty, BETA)
        np.testing.assert_allclose(Q.sum(axis=1), X @ w, rtol=1e-12)
        assert P <= prev + 1e-12 * abs(prev) if np.isfinite(prev) else True
        assert P - Dv >= -1e-12 * abs(P)
        prev = P
    r = oracle.solve_log(C, X, y, eps, lam, alpha, datafit, penalty, w, 20000, tol=1e-15, g0=g, beta=BETA)
    P, Dv, _ = oracle.objective_and_dual(r["w"], r["g"], C, X, y, eps, lam, alpha, datafit, penalty, BETA)
    assert P - Dv <= 1e-9 * abs(P)


def test_balanced_target_marginal_met():
    d = spectra.batch(97, 1, 30, 4, 2, dtype=np.float64)
    C = spectra.squared_cost(d["x"])
    y = d["y"][0]
    r = oracle.solve(C, d["D"], y, 0.05, 1.0, 0.0, "balanced", "none", spectra.initial_weights(y, d["D"]), 10)
    np.testing.assert_allclose(r["t"], y, rtol=1e-12)


# --- banded cost in diagonal storage, sparse dictionary (the scalability test's form) ----------

def _banded_case(n=60, h=5, k=6, seed=21):
    """A non-symmetric truncated cost (a drift term for i > j, holes inside the band) written as a
    dense matrix, and its diagonal storage Cd[d, i] = C[i, i + d - h] built here from it."""
    rng = np.random.default_rng(seed)
    C = np.full((n, n), np.inf)
    for i in range(n):
        for j in range(max(0, i - h), min(n, i + h + 1)):
            C[i, j] = 0.01 * abs(i - j) + 0.004 * max(i - j, 0)
    holes = rng.choice(n, size=6, replace=False)
    for i in holes:
        j = min(n - 1, i + 2)
        if j != i:
            C[i, j] = np.inf
    Cd = np.full((2 * h + 1, n), np.inf)
    for d in range(2 * h + 1):
        for i in range(n):
            if 0 <= i + d - h < n:
                Cd[d, i] = C[i, i + d - h]
    col_ptr, row_idx, val = spectra.scaling_dictionary(n, k)
    X = spectra.csc_to_dense(n, col_ptr, row_idx, val)
    y = spectra.scaling_target(n, k, rng)
    return C, Cd, X, y


def test_band_to_dense_inverts_the_diagonal_storage():
    C, Cd, _, _ = _banded_case()
    np.testing.assert_array_equal(oracle.band_to_dense(Cd, 5), C)


@pytest.mark.parametrize("datafit,penalty,mm_steps", [("l2", "l2sq", 1), ("tv", "l1", 1), ("kl", "elastic", 1),
                                                      ("poisson", "l1", 1), ("kl", "l2sq", 3)])
def test_banded_solve_equals_the_dense_solve(datafit, penalty, mm_steps):
    """Forbidden pairs have K = 0, so summing Algorithm 1's applies over the band must reproduce
    the dense solve on the same cost; the cost is not symmetric, so reading the target apply's band
    from the wrong diagonal changes the result."""
    from scipy.sparse import csc_matrix
    C, Cd, X, y = _banded_case()
    eps, lam, alpha = 5e-3, 1.0, 1e-3
    w0 = np.full(X.shape[1], y.sum() / X.sum())
    a = oracle.solve_log(C, X, y, eps, lam, alpha, datafit, penalty, w0, 40, beta=BETA, mm_steps=mm_steps)
    b = oracle.solve_log_banded(Cd, 5, csc_matrix(X), y, eps, lam, alpha, datafit, penalty, w0, 40, beta=BETA,
                                mm_steps=mm_steps)
    np.testing.assert_allclose(b["w"], a["w"], rtol=1e-11)
    np.testing.assert_allclose(b["t"], a["t"], rtol=1e-10, atol=1e-300)
    np.testing.assert_allclose(b["err_hist"], a["err_hist"], rtol=1e-8)


@pytest.mark.parametrize("datafit,penalty", [("kl", "l1"), ("l2", "l2sq")])
def test_converged_solution_is_the_optimum(datafit, penalty):
    """The long-run solution (||dw||/||w|| < 1e-14) closes the duality gap and equals the brute-force
    optimum of the tiny instance."""
    X, y, C = _tiny(n=5, k=2, seed=13)
    eps, lam, alpha = 0.05, 1.0, 0.02
    r = oracle.solve_converged(C, X, y, eps, lam, alpha, datafit, penalty, np.ones(2), max_iter=200000)
    assert r["dw"] < 1e-14
    P, Dv, _ = oracle.objective_and_dual(r["w"], r["g"], C, X, y, eps, lam, alpha, datafit, penalty)
    assert P - Dv <= 1e-10 * abs(P)
    w_bf, _ = _brute_force_primal(X, y, C, eps, lam, alpha, datafit, penalty)
    np.testing.assert_allclose(r["w"], w_bf, rtol=2e-5)


@pytest.mark.parametrize("datafit,penalty", [("kl", "l1"), ("tv", "l2sq"), ("poisson", "l1")])
def test_violation_is_the_source_marginal_error_of_the_explicit_plan(datafit, penalty):
    """Reading A8: after an iteration the solver measures e = ||Q 1 - X w||_1 / ||X w||_1 for the plan
    Q = diag(u2) K diag(u1) with the u1 of the next iteration; formed here as a matrix from the
    returned scalings."""
    X, y, C = _tiny(n=7, k=3, seed=23)
    eps, lam, alpha = 0.05, 1.0, 0.02
    for T in (1, 2, 5):
        r = oracle.solve(C, X, y, eps, lam, alpha, datafit, penalty, np.ones(3), T)
        Q = r["u2"][:, None] * np.exp(-C / eps) * r["u1"][None, :]
        s = X @ r["w"]
        assert r["err"] == pytest.approx(np.abs(Q.sum(axis=1) - s).sum() / s.sum(), rel=1e-12)
        assert len(r["err_hist"]) == T


def test_weight_change_history_and_its_stopping_rule():
    """dw_hist[j] is ||w_{j+1} - w_j||_1 / ||w_{j+1}||_1 of the weights after j and j + 1 iterations
    (each taken from its own shorter run), and with dw_tol alone the solve stops at the first
    iteration whose previous update changed w by at most dw_tol (reading A8's weight change)."""
    d = spectra.batch(71, 1, 60, 5, 2)
    x, D, y = (d[key].astype(np.float64) for key in ("x", "D", "y"))
    y = y[0]
    C = spectra.squared_cost(x)
    w0 = spectra.initial_weights(y, D)
    args = (C, D, y, 1e-2, 1.0, 1e-2, "kl", "l1")
    full = oracle.solve_log(*args, w0, 30)
    ws = [oracle.solve_log(*args, w0, j)["w"] for j in range(1, 8)]
    for j in range(6):
        want = np.abs(ws[j + 1] - ws[j]).sum() / np.abs(ws[j + 1]).sum()
        assert full["dw_hist"][j + 1] == pytest.approx(want, rel=1e-12)
    dw_tol = float(np.sort(full["dw_hist"])[len(full["dw_hist"]) // 2])  # reached part-way
    first = int(np.argmax(full["dw_hist"] <= dw_tol))
    r = oracle.solve_log(*args, w0, 30, dw_tol=dw_tol)
    assert r["iters"] == first + 1
    np.testing.assert_array_equal(r["w"], oracle.solve_log(*args, w0, first + 1)["w"])


@pytest.mark.parametrize("datafit,penalty", [("kl", "l2sq"), ("l2", "l2sq"), ("tv", "l1")])
def test_gap_stopping_rule_stops_at_the_first_check_under_tolerance(datafit, penalty):
    """With gap_tol (checked every 3 iterations) and tol, the solve returns at the first check where
    the violation and the relative gap of the returned state are both under their tolerances; the
    gap recorded there is the returned state's own (objective_and_dual on it), and it is >= 0."""
    d = spectra.batch(72, 1, 50, 4, 2)
    x, D, y = (d[key].astype(np.float64) for key in ("x", "D", "y"))
    y = y[0]
    C = spectra.squared_cost(x)
    w0 = spectra.initial_weights(y, D)
    eps, lam, alpha = 2e-2, 1.0, 1e-2
    args = (C, D, y, eps, lam, alpha, datafit, penalty)
    ref = oracle.solve_log(*args, w0, 400)
    gaps = {}
    for it in range(3, 400, 3):
        st = oracle.solve_log(*args, w0, it)  # the state a stop at iteration `it` returns
        P, Dv, _ = oracle.objective_and_dual(st["w"], st["g"], *args)
        gaps[it] = (P, Dv)
        assert P - Dv >= -1e-10 * abs(P)
        if (P - Dv) <= 1e-5 * abs(P) and ref["err_hist"][it - 1] <= 1e-6:
            break
    r = oracle.solve_log(*args, w0, 400, tol=1e-6, check_every=3, gap_tol=1e-5)
    assert r["iters"] == it
    assert r["gap_hist"][-1][0] == it
    assert r["gap_hist"][-1][1] == pytest.approx(gaps[it][0], rel=1e-12)
    assert r["gap_hist"][-1][2] == pytest.approx(gaps[it][1], rel=1e-12)
    P, Dv, _ = oracle.objective_and_dual(r["w"], r["g"], *args)
    assert P == pytest.approx(gaps[it][0], rel=1e-12) and P - Dv <= 1e-5 * abs(P)
