"""The allocation-free solve (otlm_solve_noalloc) against the regular entry point (otlm_solve).

otlm_solve_noalloc serves callers that cannot allocate device memory themselves, such as code
inside a host framework whose allocator owns the GPU's memory budget, or latency-critical loops
where cudaMalloc/cudaFree would synchronise the device: its workspace is a static 16 MiB device
array inside the library.  This file is collected last so that a run stopping at the first failure
has run every other test before it.  It must pass alone in a fresh process and after the others.
"""
import ctypes

import numpy as np
import pytest

import spectra

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2504_04609_gb300 import otlm as api  # noqa: E402

TOL32 = 1e-5


def rel_l1(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300))


def _buffers(d):
    dev = "cuda"
    B = d["y"].shape[0]
    x, D, y = (torch.tensor(d[k], device=dev) for k in ("x", "D", "y"))
    w = torch.tensor(spectra.initial_weights(d["y"], d["D"]), dtype=torch.float32, device=dev)
    out = dict(w=w, g=torch.zeros_like(y), t=torch.empty_like(y),
               iters=torch.empty(B, dtype=torch.int32, device=dev), err=torch.empty(B, device=dev),
               status=torch.empty(B, dtype=torch.int32, device=dev))
    return x, D, y, out


def _regular(d, eps, lam, alpha, datafit, penalty, iters, tol):
    x, D, y, o = _buffers(d)
    h = api.Handle(y.shape[1], D.shape[1], y.shape[0], "fp32", datafit, penalty, iters, tol, poll_every=8,
                   stream=torch.cuda.current_stream().cuda_stream)
    h.solve(x, D, y, eps, lam, alpha, o["w"], o["g"], o["t"], o["iters"], o["err"], o["status"])
    torch.cuda.synchronize()
    h.close()
    return {k: v.cpu().numpy() for k, v in o.items()}


def _noalloc(d, eps, lam, alpha, datafit, penalty, iters, tol):
    x, D, y, o = _buffers(d)
    rc = api.solve_noalloc(x, D, y, eps, lam, alpha, datafit, penalty, iters, tol, o["w"], o["g"], o["t"],
                           o["iters"], o["err"], o["status"], torch.cuda.current_stream().cuda_stream)
    assert rc == api.OTLM_OK, api.lib().otlm_strerror(rc)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in o.items()}


def test_noalloc_matches_regular_entry_point_on_two_calls_in_a_row():
    """Two different problems back to back through the same static scratch: each result must
    match otlm_solve (the second call must not see leftovers of the first)."""
    first = (spectra.batch(21, 9, 300, 12, 3), 5e-3, 1.0, 1e-2, "kl", "l1", 60, 1e-5)
    second = (spectra.batch(22, 5, 200, 10, 3), 1e-2, 1.0, 1e-3, "l2", "l2sq", 40, 0.0)
    for d, eps, lam, alpha, datafit, penalty, iters, tol in (first, second):
        ref = _regular(d, eps, lam, alpha, datafit, penalty, iters, tol)
        got = _noalloc(d, eps, lam, alpha, datafit, penalty, iters, tol)
        np.testing.assert_array_equal(got["iters"], ref["iters"])
        np.testing.assert_array_equal(got["status"], ref["status"])
        for p in range(d["y"].shape[0]):
            assert rel_l1(got["w"][p], ref["w"][p]) <= TOL32
            assert rel_l1(got["t"][p], ref["t"][p]) <= TOL32
            assert rel_l1(got["g"][p][np.isfinite(ref["g"][p])], ref["g"][p][np.isfinite(ref["g"][p])]) <= TOL32


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    B, n, k = 1024, 4096, 128  # about 84 MB of workspace, more than 16 MiB
    dummy = ctypes.c_void_p(1)
    rc = api.lib().otlm_solve_noalloc(B, n, k, dummy, dummy, dummy, 1e-2, 1.0, 1e-3, 1, 2, 10, 0.0, dummy,
                                      None, None, None, None, None, None)
    assert rc == api.OTLM_ESCRATCH
    assert "static scratch" in api.lib().otlm_strerror(rc).decode()
