"""Plant plausible mistakes in the oracle (CPU, monkeypatched) and check that a pin catches each.

This guards the pins themselves: if a pin passes on a broken oracle it pins nothing.
"""
import numpy as np
import pytest

import oracle.otlm as ot
from tests import test_oracle_pins as pins


def _fails(fn, *args):
    try:
        fn(*args)
    except AssertionError:
        return True
    return False


def test_transposed_kernel_is_caught(monkeypatch):
    good = ot.gibbs_kernel
    monkeypatch.setattr(ot, "gibbs_kernel", lambda C, eps: good(C, eps).T)
    assert _fails(pins.test_brute_force_tiny_instance, "kl", "l2sq", 1)


def test_wrong_l1_sign_is_caught(monkeypatch):
    good = ot.mm_step

    def bad(penalty, a, w_prev, X, eps, alpha, beta=0.0):
        return good(penalty, a, w_prev, X, eps, -alpha if penalty == "l1" else alpha, beta)
    monkeypatch.setattr(ot, "mm_step", bad)
    monkeypatch.setattr(pins.oracle, "mm_step", bad)
    assert _fails(pins.test_mm_step_minimises_majorizer, "l1")


def test_swapped_kl_prox_exponents_are_caught(monkeypatch):
    good = ot.prox_datafit

    def bad(datafit, s, y, eps, lam):
        if datafit == "kl":
            return np.asarray(s) ** (lam / (eps + lam)) * np.asarray(y) ** (eps / (eps + lam))
        return good(datafit, s, y, eps, lam)
    monkeypatch.setattr(pins.oracle, "prox_datafit", bad)
    assert _fails(pins.test_prox_matches_1d_minimisation, "kl", 0.05, 1.0)


def test_dropped_column_mass_in_mm_is_caught(monkeypatch):
    """nu_j without the 1/x_j factor: a dropped term that unit-mass columns would hide."""
    def bad(penalty, a, w_prev, X, eps, alpha, beta=0.0):
        X = np.asarray(X, dtype=float)
        Z = ot._Z(X, np.asarray(w_prev, dtype=float))
        with np.errstate(divide="ignore", invalid="ignore"):
            terms = np.where(X > 0, X * np.log(Z * np.asarray(a)[:, None] / X), 0.0)
        nu = terms.sum(axis=0)  # missing / x_j
        c = alpha / eps
        if penalty == "l2sq":
            return ot.lambert_w0(c * np.exp(nu)) / c
        return np.exp(nu - (alpha / eps if penalty == "l1" else 0.0))
    monkeypatch.setattr(pins.oracle, "mm_step", bad)
    assert _fails(pins.test_mm_step_minimises_majorizer, "l2sq")


def test_wrong_tv_clamp_is_caught(monkeypatch):
    good = ot._log_datafit_potential

    def bad(datafit, log_b, y, eps, lam):
        if datafit == "tv":
            return np.clip(eps * (np.log(y) - log_b), -lam / 2, lam / 2)
        return good(datafit, log_b, y, eps, lam)
    monkeypatch.setattr(ot, "_log_datafit_potential", bad)
    assert _fails(pins.test_log_potential_equals_linear_prox, "tv")


@pytest.mark.parametrize("which", ["f_sign", "entropy_sign"])
def test_broken_dual_is_caught(monkeypatch, which):
    good = ot.dual_objective

    def bad(f, g, C, X, y, eps, lam, alpha, datafit, penalty, beta=0.0):
        if which == "f_sign":
            return good(-np.asarray(f), g, C, X, y, eps, lam, alpha, datafit, penalty, beta)
        return good(f, g, C, X, y, eps, lam, alpha, datafit, penalty, beta) + 0.1
    monkeypatch.setattr(ot, "dual_objective", bad)
    assert _fails(pins.test_invariants_along_the_trajectory, "kl", "l2sq")


def test_table2_elastic_prefactor_is_caught(monkeypatch):
    """Table 2 as printed (prefactor alpha/beta, no column mass in gamma): App. A's stationarity
    condition must reject it."""
    good = ot.mm_step

    def bad(penalty, a, w_prev, X, eps, alpha, beta=0.0):
        if penalty != "elastic":
            return good(penalty, a, w_prev, X, eps, alpha, beta)
        X = np.asarray(X, dtype=float)
        x = X.sum(axis=0)
        nu = np.log(good("none", a, w_prev, X, eps, 0.0))
        return (alpha / beta) * ot.lambert_w0((beta / alpha) / x * np.exp(nu - alpha / (eps * x)))
    monkeypatch.setattr(pins.oracle, "mm_step", bad)
    assert _fails(pins.test_elastic_step_solves_its_stationarity_condition)


def test_elastic_without_the_l1_shift_is_caught(monkeypatch):
    good = ot.mm_step

    def bad(penalty, a, w_prev, X, eps, alpha, beta=0.0):
        if penalty == "elastic":
            return good("l2sq", a, w_prev, X, eps, beta)
        return good(penalty, a, w_prev, X, eps, alpha, beta)
    monkeypatch.setattr(pins.oracle, "mm_step", bad)
    assert _fails(pins.test_mm_step_minimises_majorizer, "elastic")


def test_inner_steps_with_a_stale_source_ratio_are_caught(monkeypatch):
    """Inner MM steps that keep the first step's Z (the previous w) instead of their own: the
    limit is no longer the weight prox."""
    good = ot.mm_step
    state = {}

    def bad(penalty, a, w_prev, X, eps, alpha, beta=0.0):
        key = id(a)
        if state.get("key") != key:
            state["key"], state["w0"] = key, np.asarray(w_prev, dtype=float).copy()
        return good(penalty, a, state["w0"], X, eps, alpha, beta)
    monkeypatch.setattr(ot, "mm_step", bad)
    assert _fails(pins.test_many_inner_mm_steps_give_the_weight_prox, "elastic")


def test_wrong_elastic_conjugate_is_caught(monkeypatch):
    good = ot._F1_conj_neg

    def bad(penalty, f, X, alpha, beta=0.0):
        if penalty == "elastic":
            return good("l2sq", f, X, beta)
        return good(penalty, f, X, alpha, beta)
    monkeypatch.setattr(ot, "_F1_conj_neg", bad)
    assert _fails(pins.test_invariants_along_the_trajectory, "kl", "elastic")


def test_transposed_target_band_is_caught(monkeypatch):
    """The target apply reading column j's costs from diagonal e instead of 2h - e (the source
    apply's band transposed wrongly)."""
    def bad(v, Cd, h, eps):
        n = v.shape[0]
        terms = np.full((n, 2 * h + 1), -np.inf)
        for e in range(2 * h + 1):
            lo, hi = max(0, h - e), min(n, n + h - e)
            j = np.arange(lo, hi)
            with np.errstate(invalid="ignore"):
                terms[j, e] = (v[j + e - h] - Cd[e, j + e - h]) / eps
        return ot.logsumexp(terms, axis=1)
    monkeypatch.setattr(ot, "_band_lse_cols", bad)
    assert _fails(pins.test_banded_solve_equals_the_dense_solve, "l2", "l2sq", 1)


def test_poisson_prox_with_the_printed_stationarity_sign_is_caught(monkeypatch):
    """App. B's stationarity line as printed (eps log(q/k) - lam y/q - lam = 0) leads to
    u e^u = (lam y / (eps s)) e^{-lam/eps}: the 1-D minimisation must reject it."""
    good = ot.prox_datafit

    def bad(datafit, s, y, eps, lam):
        if datafit == "poisson":
            c = lam * np.asarray(y) / eps
            return c / ot.lambert_w0(c / np.asarray(s) * np.exp(-lam / eps))
        return good(datafit, s, y, eps, lam)
    monkeypatch.setattr(pins.oracle, "prox_datafit", bad)
    assert _fails(pins.test_prox_matches_1d_minimisation, "poisson", 0.05, 1.0)
