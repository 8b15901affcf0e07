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
    assert _fails(pins.test_brute_force_tiny_instance, "kl", "l2sq")


def test_wrong_l1_sign_is_caught(monkeypatch):
    good = ot.mm_step

    def bad(penalty, a, w_prev, X, eps, alpha):
        return good(penalty, a, w_prev, X, eps, -alpha if penalty == "l1" else alpha)
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
    def bad(penalty, a, w_prev, X, eps, alpha):
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

    def bad(f, g, C, X, y, eps, lam, alpha, datafit, penalty):
        if which == "f_sign":
            return good(-np.asarray(f), g, C, X, y, eps, lam, alpha, datafit, penalty)
        return good(f, g, C, X, y, eps, lam, alpha, datafit, penalty) + 0.1
    monkeypatch.setattr(ot, "dual_objective", bad)
    assert _fails(pins.test_invariants_along_the_trajectory, "kl", "l2sq")
