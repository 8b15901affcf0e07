"""CPU checks of the C ABI: the library loads, exports every function include/otlm.h declares,
and rejects invalid arguments before touching the GPU."""
import ctypes
import os
import re

import pytest

from paper_2504_04609_gb300 import otlm as api

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _ensure_built():
    if not os.path.exists(api.LIB_PATH):
        from paper_2504_04609_gb300 import build
        build.build()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "otlm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(otlm_[a-z_]+)\s*\(", text)))


def test_header_declares_the_binding_exports():
    assert _declared_functions() == sorted(api.EXPORTS)


def test_library_exports_every_declared_symbol():
    _ensure_built()
    L = ctypes.CDLL(api.LIB_PATH)
    for name in _declared_functions():
        assert hasattr(L, name), name


def test_strerror_names_every_code():
    _ensure_built()
    for code in (api.OTLM_OK, api.OTLM_EINVAL, api.OTLM_ECUDA, api.OTLM_ENOMEM, api.OTLM_EUNSUPPORTED, api.OTLM_ESCRATCH):
        assert api.lib().otlm_strerror(code).decode() not in ("", "unknown otlm status")
    assert api.lib().otlm_strerror(12345).decode() == "unknown otlm status"


@pytest.mark.parametrize("field,value", [("n_max", 1), ("k_max", 0), ("k_max", 257), ("batch_max", 0),
                                         ("max_iter", 0), ("poll_every", 0), ("precision", 7),
                                         ("datafit", 9), ("penalty", -1), ("penalty", 4), ("mm_steps", -1),
                                         ("mm_steps", 65), ("check_every", -1), ("gap_tol", -1e-3),
                                         ("gap_tol", float("nan")), ("dw_tol", float("inf")), ("dw_tol", -1.0),
                                         ("gap_tol", 1e-4),  # a gap tolerance with no checks
                                         ("ragged_cta", 64), ("ragged_cta", 384),
                                         ("bf16_single_until", 1e-2),  # the schedule on an FP32 handle
                                         ("bf16_single_until", -1.0), ("cost", 2), ("cost", -1)])
def test_create_rejects_bad_config_without_gpu(field, value):
    _ensure_built()
    cfg = api.otlm_config(64, 8, 4, 0, 1, 2, 10, 0.0, 4)
    setattr(cfg, field, value)
    h = ctypes.c_void_p(123)
    rc = api.lib().otlm_create(ctypes.byref(h), ctypes.byref(cfg), None)
    assert rc == api.OTLM_EINVAL
    assert h.value is None


def test_null_handle_is_rejected():
    _ensure_built()
    rc = api.lib().otlm_solve(None, 1, 8, 2, 1, 1, 1, 0.1, 1.0, 0.1, 1, None, None, None, None, None)
    assert rc == api.OTLM_EINVAL
    # the dense-cost entry point (every precision takes a cost matrix of the handle's element type)
    rc = api.lib().otlm_solve_cost(None, 1, 8, 2, 1, 1, 1, 0.1, 1.0, 0.1, 1, None, None, None, None, None)
    assert rc == api.OTLM_EINVAL
    assert api.lib().otlm_launch_count(None) == -1


@pytest.mark.parametrize("beta", [0.0, -1.0, float("inf"), float("nan")])
def test_elastic_net_needs_a_finite_positive_beta(beta):
    _ensure_built()
    cfg = api.otlm_config(64, 8, 4, 0, 1, api.PENALTY["elastic"], 10, 0.0, 4, beta, 1)
    h = ctypes.c_void_p(123)
    assert api.lib().otlm_create(ctypes.byref(h), ctypes.byref(cfg), None) == api.OTLM_EINVAL
    assert h.value is None


def test_banded_entry_point_rejects_a_null_handle():
    _ensure_built()
    rc = api.lib().otlm_solve_banded(None, 1, 64, 3, 1, 4, 8, 1, 1, 1, 1, 1e-2, 1.0, 1e-3, 1, None, None, None, None,
                                     None)
    assert rc == api.OTLM_EINVAL


@pytest.mark.parametrize("eps,lam,alpha,tol", [(float("inf"), 1.0, 1e-3, 0.0), (1e-2, float("inf"), 1e-3, 0.0),
                                               (1e-2, 1.0, float("inf"), 0.0), (float("nan"), 1.0, 1e-3, 0.0),
                                               (1e-2, 1.0, 1e-3, float("inf")), (1e-2, 1.0, -1e-3, 0.0)])
def test_noalloc_rejects_non_finite_scalars_without_gpu(eps, lam, alpha, tol):
    """otlm_solve_noalloc refuses the scalars otlm_solve refuses, before any CUDA call (the
    pointers are dummies that are never dereferenced)."""
    _ensure_built()
    dummy = ctypes.c_void_p(1)
    rc = api.lib().otlm_solve_noalloc(4, 64, 8, dummy, dummy, dummy, eps, lam, alpha, 1, 2, 10, tol, dummy,
                                      None, None, None, None, None, None)
    assert rc == api.OTLM_EINVAL


@pytest.mark.parametrize("bad", [-1, 6])
def test_create_rejects_a_bad_rows_per_thread_entry(bad):
    _ensure_built()
    cfg = api.otlm_config(64, 8, 4, 0, 1, 2, 10, 0.0, 4)
    cfg.ragged_rows_log2[7] = bad
    h = ctypes.c_void_p(123)
    assert api.lib().otlm_create(ctypes.byref(h), ctypes.byref(cfg), None) == api.OTLM_EINVAL
    assert h.value is None


def test_precision_schedule_needs_a_tensor_core_handle_and_a_value_below_one():
    _ensure_built()
    for prec, v, rc in ((2, 1e-2, api.OTLM_OK), (2, 1.0, api.OTLM_EINVAL), (2, float("nan"), api.OTLM_EINVAL)):
        cfg = api.otlm_config(64, 8, 4, prec, 1, 2, 10, 0.0, 4)
        cfg.bf16_single_until = v
        h = ctypes.c_void_p()
        got = api.lib().otlm_create(ctypes.byref(h), ctypes.byref(cfg), None)
        if rc == api.OTLM_OK:
            # creation needs device memory: without a GPU it fails after validation, not with EINVAL
            assert got != api.OTLM_EINVAL
            if got == api.OTLM_OK:
                api.lib().otlm_destroy(h)
        else:
            assert got == rc


def test_absolute_distance_cost_passes_validation():
    """cost = 1 (|x_i - x_j|) is a valid grid cost on every precision: without a GPU creation fails
    only after validation."""
    _ensure_built()
    for prec in (0, 1, 2):
        cfg = api.otlm_config(64, 8, 4, prec, 1, 2, 10, 0.0, 4)
        cfg.cost = api.COST["abs"]
        h = ctypes.c_void_p()
        got = api.lib().otlm_create(ctypes.byref(h), ctypes.byref(cfg), None)
        assert got != api.OTLM_EINVAL
        if got == api.OTLM_OK:
            api.lib().otlm_destroy(h)


def test_wait_expiry_check_rejects_a_null_code_pointer():
    _ensure_built()
    assert api.lib().otlm_check_wait_expiry(0, None) == api.OTLM_EINVAL
