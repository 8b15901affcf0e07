"""ctypes binding of the C ABI in include/otlm.h (argument marshalling only).

Every step of the solver runs in libotlm.so; this module only converts torch tensors / numpy
arrays to pointers.  There is no CPU fallback: if the library is missing or cannot be loaded,
`lib()` raises.  Device buffers are torch CUDA tensors (torch provides memory and streams).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libotlm.so")

OTLM_OK, OTLM_EINVAL, OTLM_ECUDA, OTLM_ENOMEM, OTLM_EUNSUPPORTED, OTLM_ESCRATCH, OTLM_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
CONVERGED, MAX_ITER, NONFINITE, INVALID = 0, 1, 2, 3
DATAFIT = {"balanced": 0, "kl": 1, "tv": 2, "l2": 3, "poisson": 4}
PENALTY = {"none": 0, "l1": 1, "l2sq": 2, "elastic": 3}
PRECISION = {"fp32": 0, "fp64": 1, "bf16tc": 2}

EXPORTS = ("otlm_create", "otlm_destroy", "otlm_solve", "otlm_solve_cost", "otlm_solve_host", "otlm_objective",
           "otlm_launch_count", "otlm_set_timing", "otlm_get_timing", "otlm_solve_noalloc", "otlm_solve_ragged", "otlm_solve_banded",
           "otlm_tune_ragged", "otlm_ws_create", "otlm_ws_destroy", "otlm_ws_num_params", "otlm_ws_set_normalization",
           "otlm_ws_get_params", "otlm_ws_set_params", "otlm_ws_gradients", "otlm_ws_train_step", "otlm_ws_predict",
           "otlm_ws_make_targets", "otlm_ws_fit_normalization", "otlm_initial_weights", "otlm_solve_stats",
           "otlm_check_wait_expiry", "otlm_strerror")
TIMING_KINDS = ("apply", "mm_source", "compact", "other")
COST = {"sq": 0, "abs": 1}  # grid cost (x_i - x_j)^2 or |x_i - x_j| (otlm_cost_kind)


class otlm_config(ctypes.Structure):
    _fields_ = [("n_max", ctypes.c_int), ("k_max", ctypes.c_int), ("batch_max", ctypes.c_int),
                ("precision", ctypes.c_int), ("datafit", ctypes.c_int), ("penalty", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("tol", ctypes.c_double), ("poll_every", ctypes.c_int),
                ("beta", ctypes.c_double), ("mm_steps", ctypes.c_int), ("check_every", ctypes.c_int),
                ("gap_tol", ctypes.c_double), ("dw_tol", ctypes.c_double), ("ragged_cta", ctypes.c_int),
                ("ragged_rows_log2", ctypes.c_int * 16), ("bf16_single_until", ctypes.c_double),
                ("cost", ctypes.c_int)]


_LIB = None


def lib() -> ctypes.CDLL:
    """Load libotlm.so (built by paper_2504_04609_gb300.build); raises if it is not there."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2504_04609_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.otlm_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(otlm_config), vp]
        L.otlm_create.restype = i
        L.otlm_destroy.argtypes = [vp]
        L.otlm_destroy.restype = None
        solve_args = [vp, i, i, i, vp, vp, vp, d, d, d, vp, vp, vp, vp, vp, vp]
        L.otlm_solve.argtypes = solve_args
        L.otlm_solve.restype = i
        L.otlm_solve_host.argtypes = solve_args
        L.otlm_solve_host.restype = i
        L.otlm_check_wait_expiry.argtypes = [i, ctypes.POINTER(ctypes.c_int)]
        L.otlm_check_wait_expiry.restype = i
        L.otlm_solve_cost.argtypes = solve_args
        L.otlm_solve_cost.restype = i
        L.otlm_objective.argtypes = [vp, i, i, i, vp, vp, vp, d, d, d, vp, vp, vp, vp]
        L.otlm_objective.restype = i
        L.otlm_launch_count.argtypes = [vp]
        L.otlm_launch_count.restype = ctypes.c_longlong
        L.otlm_set_timing.argtypes = [vp, i]
        L.otlm_set_timing.restype = i
        L.otlm_get_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
        L.otlm_get_timing.restype = i
        L.otlm_solve_noalloc.argtypes = [i, i, i, vp, vp, vp, d, d, d, i, i, i, d, vp, vp, vp, vp, vp, vp, vp]
        L.otlm_solve_noalloc.restype = i
        L.otlm_solve_ragged.argtypes = [vp, i, vp, vp, vp, vp, vp, vp, vp, vp, vp, d, d, vp, vp, vp, vp, vp, vp]
        L.otlm_solve_ragged.restype = i
        L.otlm_solve_banded.argtypes = [vp, i, i, i, vp, i, i, vp, vp, vp, vp, d, d, d, vp, vp, vp, vp, vp, vp]
        L.otlm_solve_banded.restype = i
        L.otlm_tune_ragged.argtypes = [vp, i, vp, vp, vp, vp, vp, vp, vp, vp, vp, d, d, vp, i, i,
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.otlm_tune_ragged.restype = i
        L.otlm_ws_create.argtypes = [ctypes.POINTER(vp), i, i, i, i, ctypes.c_ulonglong, vp]
        L.otlm_ws_create.restype = i
        L.otlm_ws_destroy.argtypes = [vp]
        L.otlm_ws_destroy.restype = None
        L.otlm_ws_num_params.argtypes = [vp]
        L.otlm_ws_num_params.restype = ctypes.c_longlong
        for nm in ("otlm_ws_set_normalization",):
            getattr(L, nm).argtypes = [vp, vp, vp]
            getattr(L, nm).restype = i
        for nm in ("otlm_ws_get_params", "otlm_ws_set_params"):
            getattr(L, nm).argtypes = [vp, vp]
            getattr(L, nm).restype = i
        L.otlm_ws_gradients.argtypes = [vp, i, vp, vp, vp, vp]
        L.otlm_ws_gradients.restype = i
        L.otlm_ws_train_step.argtypes = [vp, i, vp, vp, d, d, vp]
        L.otlm_ws_train_step.restype = i
        L.otlm_ws_predict.argtypes = [vp, i, vp, d, vp, vp, vp]
        L.otlm_ws_predict.restype = i
        L.otlm_ws_make_targets.argtypes = [vp, i, vp, vp, d, d, vp]
        L.otlm_ws_make_targets.restype = i
        L.otlm_ws_fit_normalization.argtypes = [vp, i, vp, vp, vp]
        L.otlm_ws_fit_normalization.restype = i
        L.otlm_initial_weights.argtypes = [vp, i, i, i, vp, vp, vp]
        L.otlm_initial_weights.restype = i
        L.otlm_solve_stats.argtypes = [vp, i, vp, vp, vp]
        L.otlm_solve_stats.restype = i
        L.otlm_strerror.argtypes = [i]
        L.otlm_strerror.restype = ctypes.c_char_p
        _LIB = L
    return _LIB


class OTLMError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != OTLM_OK:
        raise OTLMError(f"{what}: {lib().otlm_strerror(rc).decode()} ({rc})")


def _ptr(t):
    """Device/host pointer of a torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    assert t.is_contiguous()
    return t.data_ptr()


@dataclass
class SolveResult:
    w: object
    g: object
    t: object
    iters: object
    err: object
    status: object


class Handle:
    """Owns one otlm handle (workspace sized for n_max x k_max x batch_max).

    beta: squared-l2 weight of the "elastic" penalty (alpha sum w + (beta/2) ||w||^2);
    mm_steps: MM steps of the weight update per iteration (1 in Algorithm 1);
    check_every, gap_tol, dw_tol: the FP64 objective / gap checks and the further stopping
    criteria of otlm_config; cost: "sq" (squared distance, default) or "abs" (absolute distance)
    for the grid solves."""

    def __init__(self, n_max, k_max, batch_max, precision="fp32", datafit="kl", penalty="l2sq",
                 max_iter=1000, tol=0.0, poll_every=8, stream=None, beta=0.0, mm_steps=1, check_every=0,
                 gap_tol=0.0, dw_tol=0.0, ragged_cta=0, ragged_rows_log2=None, bf16_single_until=0.0, cost="sq"):
        rows = (ctypes.c_int * 16)(*(list(ragged_rows_log2) if ragged_rows_log2 is not None else [0] * 16))
        self.cfg = otlm_config(n_max, k_max, batch_max, PRECISION[precision], DATAFIT[datafit], PENALTY[penalty],
                               max_iter, float(tol), poll_every, float(beta), mm_steps, check_every, float(gap_tol),
                               float(dw_tol), ragged_cta, rows, float(bf16_single_until),
                               COST[cost] if isinstance(cost, str) else int(cost))
        self.precision = precision
        self._h = ctypes.c_void_p()
        _check(lib().otlm_create(ctypes.byref(self._h), ctypes.byref(self.cfg), stream), "otlm_create")

    def close(self):
        if self._h:
            lib().otlm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def launches(self) -> int:
        return lib().otlm_launch_count(self._h)

    def set_timing(self, enable: bool):
        _check(lib().otlm_set_timing(self._h, int(bool(enable))), "otlm_set_timing")

    def get_timing(self):
        """{kind: (device ms, launches)} accumulated since the last call (resets the sums)."""
        ms = (ctypes.c_double * 4)()
        cnt = (ctypes.c_longlong * 4)()
        _check(lib().otlm_get_timing(self._h, ms, cnt), "otlm_get_timing")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(TIMING_KINDS)}

    def solve(self, x, D, y, eps, lam, alpha, w, g=None, t_out=None, iters=None, err=None, status=None):
        """otlm_solve on torch CUDA tensors; w (and g) are updated in place."""
        B, n = y.shape
        k = D.shape[1]
        rc = lib().otlm_solve(self._h, B, n, k, _ptr(x), _ptr(D), _ptr(y), eps, lam, alpha, _ptr(w), _ptr(g),
                              _ptr(t_out), _ptr(iters), _ptr(err), _ptr(status))
        _check(rc, "otlm_solve")
        return SolveResult(w, g, t_out, iters, err, status)

    def solve_cost(self, C, D, y, eps, lam, alpha, w, g=None, t_out=None, iters=None, err=None, status=None):
        """otlm_solve_cost: a dense cost C [n][n] (torch CUDA tensor; row = source bin, column = target
        bin, need not be symmetric, +inf forbids a pair; the handle's element type) instead of a grid."""
        B, n = y.shape
        k = D.shape[1]
        rc = lib().otlm_solve_cost(self._h, B, n, k, _ptr(C), _ptr(D), _ptr(y), eps, lam, alpha, _ptr(w), _ptr(g),
                                   _ptr(t_out), _ptr(iters), _ptr(err), _ptr(status))
        _check(rc, "otlm_solve_cost")
        return SolveResult(w, g, t_out, iters, err, status)

    def solve_host(self, x, D, y, eps, lam, alpha, w, g=None, t_out=None, iters=None, err=None, status=None):
        """otlm_solve_host on host (numpy or pinned torch CPU) buffers."""
        B, n = y.shape
        k = D.shape[1]
        rc = lib().otlm_solve_host(self._h, B, n, k, _ptr(x), _ptr(D), _ptr(y), eps, lam, alpha, _ptr(w), _ptr(g),
                                   _ptr(t_out), _ptr(iters), _ptr(err), _ptr(status))
        _check(rc, "otlm_solve_host")
        return SolveResult(w, g, t_out, iters, err, status)

    def solve_banded(self, Cd, hw, col_ptr, row_idx, val, y, eps, lam, alpha, w, g=None, t_out=None, iters=None,
                     err=None, status=None):
        """otlm_solve_banded: Cd [2hw+1, n] float32, col_ptr / row_idx int32 and val float32 (CSC
        dictionary), y [B, n], w [B, k] (in/out); all CUDA tensors."""
        B, n = y.shape
        k = col_ptr.shape[0] - 1
        rc = lib().otlm_solve_banded(self._h, B, n, hw, _ptr(Cd), k, val.shape[0], _ptr(col_ptr), _ptr(row_idx),
                                     _ptr(val), _ptr(y), eps, lam, alpha, _ptr(w), _ptr(g), _ptr(t_out), _ptr(iters),
                                     _ptr(err), _ptr(status))
        _check(rc, "otlm_solve_banded")

    def solve_ragged(self, rb, lam, alpha, w, g=None, t_out=None, iters=None, err=None, status=None):
        """otlm_solve_ragged on a RaggedBatch of device tensors (see ragged_batch)."""
        rc = lib().otlm_solve_ragged(self._h, rb.batch, _ptr(rb.n), _ptr(rb.k), _ptr(rb.eps), _ptr(rb.off_n),
                                     _ptr(rb.off_D), _ptr(rb.off_k), _ptr(rb.x), _ptr(rb.D), _ptr(rb.y), lam, alpha,
                                     _ptr(w), _ptr(g), _ptr(t_out), _ptr(iters), _ptr(err), _ptr(status))
        _check(rc, "otlm_solve_ragged")

    def tune_ragged(self, rb, lam, alpha, w, sample_every=40, iters=6, with_rows=False):
        """otlm_tune_ragged: returns the CTA size the tuner kept on this handle, and with
        with_rows=True also the rows-per-thread table (log2 by size bucket, otlm_config's form)."""
        out = ctypes.c_int(0)
        rows = (ctypes.c_int * 16)()
        rc = lib().otlm_tune_ragged(self._h, rb.batch, _ptr(rb.n), _ptr(rb.k), _ptr(rb.eps), _ptr(rb.off_n),
                                    _ptr(rb.off_D), _ptr(rb.off_k), _ptr(rb.x), _ptr(rb.D), _ptr(rb.y), lam, alpha,
                                    _ptr(w), sample_every, iters, ctypes.byref(out), rows)
        _check(rc, "otlm_tune_ragged")
        return (out.value, list(rows)) if with_rows else out.value

    def solve_stats(self, batch, dw_out=None, primal_out=None, dual_out=None):
        """otlm_solve_stats: per-problem weight change, FP64 primal and dual of the last solve."""
        _check(lib().otlm_solve_stats(self._h, batch, _ptr(dw_out), _ptr(primal_out), _ptr(dual_out)),
               "otlm_solve_stats")

    def initial_weights(self, D, y, w_out):
        """otlm_initial_weights: the cold-start weights sum(y) / (k x_j) into w_out [B, k]."""
        B, n = y.shape
        k = D.shape[1]
        _check(lib().otlm_initial_weights(self._h, B, n, k, _ptr(D), _ptr(y), _ptr(w_out)), "otlm_initial_weights")

    def objective(self, x, D, y, eps, lam, alpha, w, g, primal, dual):
        B, n = y.shape
        k = D.shape[1]
        rc = lib().otlm_objective(self._h, B, n, k, _ptr(x), _ptr(D), _ptr(y), eps, lam, alpha, _ptr(w), _ptr(g),
                                  _ptr(primal), _ptr(dual))
        _check(rc, "otlm_objective")


def solve_noalloc(x, D, y, eps, lam, alpha, datafit, penalty, max_iter, tol, w, g=None, t_out=None, iters=None,
                  err=None, status=None, stream=None):
    """otlm_solve_noalloc on float32 torch CUDA tensors: the solve with no device allocation by the
    library (workspace in its static 16 MiB device array).  Returns the C status code."""
    B, n = y.shape
    k = D.shape[1]
    return lib().otlm_solve_noalloc(B, n, k, _ptr(x), _ptr(D), _ptr(y), eps, lam, alpha, DATAFIT[datafit],
                                    PENALTY[penalty], max_iter, tol, _ptr(w), _ptr(g), _ptr(t_out), _ptr(iters),
                                    _ptr(err), _ptr(status), stream)


def solve(x, D, y, eps, lam, alpha, datafit, penalty, w0, g0=None, max_iter=1000, tol=0.0,
          precision="fp32", poll_every=8, beta=0.0, mm_steps=1, bf16_single_until=0.0, cost="sq"):
    """One-shot convenience: allocate a handle sized for this problem and solve on the GPU.

    Inputs are torch CUDA tensors of the handle's dtype.  Returns SolveResult of CUDA tensors.
    """
    import torch
    B, n = y.shape
    k = D.shape[1]
    h = Handle(n, k, B, precision, datafit, penalty, max_iter, tol, poll_every,
               stream=torch.cuda.current_stream().cuda_stream, beta=beta, mm_steps=mm_steps,
               bf16_single_until=bf16_single_until, cost=cost)
    dt = torch.float64 if precision == "fp64" else torch.float32
    w = w0.clone()
    g = torch.zeros_like(y) if g0 is None else g0.clone()
    t = torch.empty_like(y)
    iters = torch.empty(B, dtype=torch.int32, device=y.device)
    err = torch.empty(B, dtype=dt, device=y.device)
    status = torch.empty(B, dtype=torch.int32, device=y.device)
    h.solve(x, D, y, eps, lam, alpha, w, g, t, iters, err, status)
    torch.cuda.current_stream().synchronize()
    h.close()
    return SolveResult(w, g, t, iters, err, status)


@dataclass
class RaggedBatch:
    batch: int
    n: object
    k: object
    eps: object
    off_n: object
    off_D: object
    off_k: object
    x: object
    D: object
    y: object


def ragged_batch(problems, device="cuda"):
    """Concatenate a list of dicts(x, D, y, eps, n, k) (float32 arrays) into device tensors."""
    import torch
    n = np.array([p["n"] for p in problems], np.int32)
    k = np.array([p["k"] for p in problems], np.int32)
    off_n = np.concatenate([[0], np.cumsum(n.astype(np.int64))[:-1]]).astype(np.int64)
    off_D = np.concatenate([[0], np.cumsum((n.astype(np.int64) * k))[:-1]]).astype(np.int64)
    off_k = np.concatenate([[0], np.cumsum(k.astype(np.int64))[:-1]]).astype(np.int64)
    cat = lambda key: np.concatenate([np.asarray(p[key], np.float32).ravel() for p in problems])  # noqa: E731
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)  # noqa: E731
    return RaggedBatch(len(problems), t(n), t(k), t(np.array([p["eps"] for p in problems], np.float32)),
                       t(off_n), t(off_D), t(off_k), t(cat("x")), t(cat("D")), t(cat("y")))


class WarmStart:
    """The learned warm start network (otlm_ws_*): device tensors in, device tensors out."""

    def __init__(self, n, k, width=512, batch_max=512, seed=2504_04609, stream=None):
        self.n, self.k, self.width, self.batch_max = n, k, width, batch_max
        self._w = ctypes.c_void_p()
        _check(lib().otlm_ws_create(ctypes.byref(self._w), n, k, width, batch_max, seed, stream), "otlm_ws_create")

    @property
    def num_params(self) -> int:
        return lib().otlm_ws_num_params(self._w)

    def close(self):
        if self._w:
            lib().otlm_ws_destroy(self._w)
            self._w = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_normalization(self, mean, std):
        _check(lib().otlm_ws_set_normalization(self._w, _ptr(mean), _ptr(std)), "otlm_ws_set_normalization")

    def get_params(self, out):
        _check(lib().otlm_ws_get_params(self._w, _ptr(out)), "otlm_ws_get_params")

    def set_params(self, params):
        _check(lib().otlm_ws_set_params(self._w, _ptr(params)), "otlm_ws_set_params")

    def gradients(self, y, target, grad_out=None, loss_out=None):
        _check(lib().otlm_ws_gradients(self._w, y.shape[0], _ptr(y), _ptr(target), _ptr(grad_out), _ptr(loss_out)),
               "otlm_ws_gradients")

    def train_step(self, y, target, lr, weight_decay=0.0, loss_out=None):
        _check(lib().otlm_ws_train_step(self._w, y.shape[0], _ptr(y), _ptr(target), lr, weight_decay,
                                        _ptr(loss_out)), "otlm_ws_train_step")

    def make_targets(self, g, w, eps, g_floor, targets):
        _check(lib().otlm_ws_make_targets(self._w, g.shape[0], _ptr(g), _ptr(w), eps, g_floor, _ptr(targets)),
               "otlm_ws_make_targets")

    def fit_normalization(self, targets, mean_out=None, std_out=None):
        _check(lib().otlm_ws_fit_normalization(self._w, targets.shape[0], _ptr(targets), _ptr(mean_out),
                                               _ptr(std_out)), "otlm_ws_fit_normalization")

    def predict(self, y, eps, cold_w, g0, w0):
        _check(lib().otlm_ws_predict(self._w, y.shape[0], _ptr(y), eps, _ptr(cold_w), _ptr(g0), _ptr(w0)),
               "otlm_ws_predict")


def check_wait_expiry(two_sm: bool) -> tuple:
    """otlm_check_wait_expiry: (return code, recorded error code) of the bounded-wait self-check."""
    code = ctypes.c_int(0)
    rc = lib().otlm_check_wait_expiry(int(bool(two_sm)), ctypes.byref(code))
    return rc, code.value
