"""Seeded synthetic spectra: the one input source shared by the FP64 oracle and the CUDA path.

This module draws problem instances and nothing else; it holds none of the solver's arithmetic.
Shapes and value distributions stand in for the paper's workloads (App. D, scaling test:
Gaussian basis functions on a 1-D grid, a sum of shifted peaks plus non-negative noise as the
target).  The paper's own spectra (muonic X-ray, Sec. 6.1 / App. E; infrared filters,
Sec. 6.2 / App. F) are not available; these draws stand in for them.

Recipe (every instance):
  * grid        x_i = i / (n - 1), i = 0..n-1, on [0, 1]
  * cost        C_ij = (x_i - x_j)^2        (squared distance on the grid)
  * dictionary  k Gaussian peaks, centres U[0.1, 0.9], widths exp(N(ln 0.02, 0.3)),
                each column normalised to unit mass (sum over bins = 1)
  * weights     w_true has `nnz` non-zeros at random atoms, values Gamma(shape 2, scale 1)
  * target      y = sum_j w_true_j * peak_j shifted by delta ~ N(0, 0.01) (std) in position
                and renormalised to unit mass, then y <- max(0, y * (1 + 0.01 xi)), xi ~ N(0, 1)

Seeds: numpy SeedSequence(2504_04609, spawn_key=(workload_id, ...)), one child stream for the
shared dictionary and one per target, so that a sub-batch of a workload reproduces exactly the
same problems as the full batch.

Every array is produced in float64 and then rounded to the precision the solver is given
(`dtype`; float32 subnormals flushed to zero), so both sides see bit-identical input values.
"""
from __future__ import annotations

import numpy as np

ROOT_SEED = 2504_04609


def _rng(*key: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(ROOT_SEED, spawn_key=tuple(int(v) for v in key)))


def grid(n: int) -> np.ndarray:
    """x_i = i/(n-1) on [0, 1]."""
    if n < 2:
        raise ValueError("grid needs n >= 2")
    return np.arange(n, dtype=np.float64) / (n - 1)


def squared_cost(x: np.ndarray) -> np.ndarray:
    """Dense C_ij = (x_i - x_j)^2 for tests that want the cost as a matrix."""
    return (x[:, None] - x[None, :]) ** 2


def abs_cost(x: np.ndarray) -> np.ndarray:
    """Dense C_ij = |x_i - x_j| (the absolute-distance grid cost; pass rho x for rho |x_i - x_j|)."""
    return np.abs(x[:, None] - x[None, :])


def _unit_peaks(x: np.ndarray, mu: np.ndarray, sigma: np.ndarray) -> np.ndarray:
    g = np.exp(-0.5 * ((x[:, None] - mu[None, :]) / sigma[None, :]) ** 2)
    return g / g.sum(axis=0, keepdims=True)


def peak_parameters(rng: np.random.Generator, k: int):
    mu = rng.uniform(0.1, 0.9, size=k)
    sigma = np.exp(rng.normal(np.log(0.02), 0.3, size=k))
    return mu, sigma


def dictionary(x: np.ndarray, k: int, rng: np.random.Generator):
    """D [n, k] of unit-mass Gaussian peaks plus their (centre, width) parameters."""
    mu, sigma = peak_parameters(rng, k)
    return _unit_peaks(x, mu, sigma), mu, sigma


def target(x: np.ndarray, mu: np.ndarray, sigma: np.ndarray, nnz: int, rng: np.random.Generator):
    """One target spectrum y [n] and its generating weights w_true [k]."""
    k = mu.shape[0]
    nnz = min(nnz, k)
    idx = rng.choice(k, size=nnz, replace=False)
    w_true = np.zeros(k)
    w_true[idx] = rng.gamma(2.0, 1.0, size=nnz)
    shift = rng.normal(0.0, 0.01, size=nnz)
    peaks = _unit_peaks(x, mu[idx] + shift, sigma[idx])
    y = peaks @ w_true[idx]
    y = np.maximum(0.0, y * (1.0 + 0.01 * rng.normal(size=x.shape[0])))
    return y, w_true


def to_dtype(a: np.ndarray, dtype) -> np.ndarray:
    """Round to `dtype`; in float32, values below the smallest normal number become 0, matching
    the flush-to-zero arithmetic of the FP32 kernels so both sides see the same input."""
    out = np.asarray(a).astype(dtype)
    if np.dtype(dtype) == np.float32:
        out[np.abs(out) < np.finfo(np.float32).tiny] = 0.0
    return out


def batch(workload: int, B: int, n: int, k: int, nnz: int, dtype=np.float32, first: int = 0):
    """A batch of B targets sharing one grid and one dictionary.

    Returns dict(x [n], D [n,k], y [B,n], w_true [B,k]) with x, D, y rounded to `dtype`
    (w_true stays float64; it is only a generator record).  Problem p of the batch is drawn
    from child stream (workload, 1, first + p), so problems are reproducible one by one.
    """
    x = grid(n)
    D, mu, sigma = dictionary(x, k, _rng(workload, 0))
    Y = np.empty((B, n))
    W = np.empty((B, k))
    for p in range(B):
        Y[p], W[p] = target(x, mu, sigma, nnz, _rng(workload, 1, first + p))
    return dict(x=to_dtype(x, dtype), D=to_dtype(D, dtype), y=to_dtype(Y, dtype), w_true=W)


def ragged(workload: int, count: int, n_range=(256, 4096), k_range=(8, 128), eps_range=(2e-3, 5e-2),
           nnz: int = 5, dtype=np.float32, first: int = 0):
    """Uneven batch: each problem draws its own n ~ U{n_range}, k ~ U{k_range},
    eps ~ logU[eps_range], its own grid and dictionary and one target.

    Returns a list of dicts(x, D, y, eps, n, k).
    """
    out = []
    for p in range(count):
        rng = _rng(workload, 2, first + p)
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        eps = float(np.exp(rng.uniform(np.log(eps_range[0]), np.log(eps_range[1]))))
        x = grid(n)
        D, mu, sigma = dictionary(x, k, rng)
        y, _ = target(x, mu, sigma, nnz, rng)
        out.append(dict(x=to_dtype(x, dtype), D=to_dtype(D, dtype), y=to_dtype(y, dtype), eps=eps, n=n, k=k))
    return out


def ragged_sizes(workload: int, count: int, n_range=(256, 4096), k_range=(8, 128), eps_range=(2e-3, 5e-2),
                 first: int = 0):
    """The (n, k, eps) of each problem of `ragged(workload, count, ..., first=first)` without the
    arrays: the first three draws of each problem's stream (int64, int64, float64 arrays), so that a
    packed layout can be planned before the problems are generated."""
    n = np.empty(count, np.int64)
    k = np.empty(count, np.int64)
    eps = np.empty(count, np.float64)
    for p in range(count):
        rng = _rng(workload, 2, first + p)
        n[p] = int(rng.integers(n_range[0], n_range[1] + 1))
        k[p] = int(rng.integers(k_range[0], k_range[1] + 1))
        eps[p] = float(np.exp(rng.uniform(np.log(eps_range[0]), np.log(eps_range[1]))))
    return n, k, eps


def scaling_dictionary(n: int, k: int, sigma_b: float = 2.0, trunc: float = 5.0):
    """Sparse dictionary of the paper's scalability test (App. "Performance Scalability Tests"):
    k Gaussians of height 1 on the sample grid x_i = i, means m n / k (m = 0..k-1), width sigma_b,
    truncated at +-trunc sigma_b.  Returns CSC arrays (col_ptr [k+1] int32, row_idx [nnz] int32,
    val [nnz] float64), rows ascending within each column."""
    half = int(np.floor(trunc * sigma_b))
    col_ptr = [0]
    rows, vals = [], []
    for m in range(k):
        mu = m * n / k
        lo, hi = max(0, int(np.ceil(mu - trunc * sigma_b))), min(n - 1, int(np.floor(mu + trunc * sigma_b)))
        i = np.arange(lo, hi + 1)
        rows.append(i)
        vals.append(np.exp(-0.5 * ((i - mu) / sigma_b) ** 2))
        col_ptr.append(col_ptr[-1] + i.size)
    assert half >= 0
    return (np.asarray(col_ptr, dtype=np.int32), np.concatenate(rows).astype(np.int32),
            np.concatenate(vals))


def truncated_cost_band(n: int, rho: float = 0.01, delta: float = 10.0):
    """Cost of the scalability test, C_ij = rho |x_i - x_j| when |x_i - x_j| < delta, +inf
    otherwise, on x_i = i, in diagonal storage: Cd[d, i] = C(i, i + d - h) with half-width
    h = ceil(delta) - 1, +inf where i + d - h falls outside [0, n).  Returns (Cd [2h+1, n], h)."""
    h = int(np.ceil(delta)) - 1
    Cd = np.full((2 * h + 1, n), np.inf)
    i = np.arange(n)
    for d in range(2 * h + 1):
        j = i + d - h
        ok = (j >= 0) & (j < n) & (np.abs(d - h) < delta)
        Cd[d, ok] = rho * np.abs(d - h)
    return Cd, h


def _skew_normal(x, mu, sigma, gamma):
    from scipy.special import ndtr
    z = (x - mu) / sigma
    return 2.0 / sigma * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi) * ndtr(gamma * z)


def scaling_target(n: int, k: int, rng: np.random.Generator) -> np.ndarray:
    """Target of the scalability test: y_i = sum_m a_m f(x_i; mu_m, sigma_m, gamma_m) + |n_i| with
    k skew-normal components, mu ~ U[0, n], sigma ~ |N(2, 0.2)|, a ~ |N(1, 0.2)| + 0.01,
    gamma ~ N(0, 2), noise n_i ~ N(0, 0.002).  Each component is evaluated within +-12 sigma_m of
    its mean (beyond that the density is below 1e-31 of its peak)."""
    mu = rng.uniform(0.0, n, size=k)
    sigma = np.abs(rng.normal(2.0, 0.2, size=k))
    amp = np.abs(rng.normal(1.0, 0.2, size=k)) + 0.01
    gamma = rng.normal(0.0, 2.0, size=k)
    noise = np.abs(rng.normal(0.0, 0.002, size=n))
    y = noise.copy()
    for m in range(k):
        lo, hi = max(0, int(mu[m] - 12 * sigma[m])), min(n, int(mu[m] + 12 * sigma[m]) + 2)
        x = np.arange(lo, hi, dtype=np.float64)
        y[lo:hi] += amp[m] * _skew_normal(x, mu[m], sigma[m], gamma[m])
    return y


def scaling_batch(workload: int, B: int, n: int, k: int = None, dtype=np.float32, first: int = 0):
    """B targets of the scalability test sharing its cost band and dictionary (k = n / 10 by
    default).  Returns dict(Cd [2h+1, n], h, col_ptr, row_idx, val, y [B, n], x_col [k]) with Cd,
    val and y rounded to `dtype`; x_col are the column masses of the rounded dictionary (float64).
    Target p comes from child stream (workload, 3, first + p)."""
    k = n // 10 if k is None else k
    Cd, h = truncated_cost_band(n)
    col_ptr, row_idx, val = scaling_dictionary(n, k)
    Y = np.stack([scaling_target(n, k, _rng(workload, 3, first + p)) for p in range(B)])
    val = to_dtype(val, dtype)
    x_col = np.add.reduceat(val.astype(np.float64), col_ptr[:-1])
    return dict(Cd=to_dtype(Cd, dtype), h=h, col_ptr=col_ptr, row_idx=row_idx, val=val,
                y=to_dtype(Y, dtype), x_col=x_col, n=n, k=k)


def csc_to_dense(n: int, col_ptr, row_idx, val) -> np.ndarray:
    """Dense [n, k] copy of a CSC dictionary (for small cases)."""
    k = len(col_ptr) - 1
    D = np.zeros((n, k))
    for m in range(k):
        for q in range(col_ptr[m], col_ptr[m + 1]):
            D[row_idx[q], m] = val[q]
    return D


def initial_weights(y: np.ndarray, D: np.ndarray) -> np.ndarray:
    """Cold-start weights w0_j = sum(y) / (k * x_j), x_j the column mass of D.

    The paper leaves the initial w to the caller (Algorithm 1 takes it as input); every w0_j
    must be > 0 because zero weights stay zero under multiplicative updates.  Shapes:
    y [..., n], D [n, k] -> w0 [..., k] in float64.
    """
    y = np.asarray(y, dtype=np.float64)
    D = np.asarray(D, dtype=np.float64)
    k = D.shape[1]
    col = D.sum(axis=0)
    return (y.sum(axis=-1)[..., None] / (k * col)) * np.ones(y.shape[:-1] + (k,))


# Workload catalogue: the configurations the solver is measured on, by what they are.
WORKLOADS = {
    "single_fp64_n200": dict(id=1, B=1, n=200, k=10, nnz=3, eps=1e-2, datafit="kl", lam=1.0,
                             penalty="l2sq", alpha=1e-3, iters=500, dtype=np.float64),
    "batch1024_n1024_kl_l1": dict(id=2, B=1024, n=1024, k=64, nnz=5, eps=5e-3, datafit="kl", lam=1.0,
                                  penalty="l1", alpha=1e-2, iters=2000, tol=1e-5, dtype=np.float32),
    "batch4096_n4096_l2_l2sq": dict(id=3, B=4096, n=4096, k=128, nnz=5, eps=1e-2, datafit="l2", lam=1.0,
                                    penalty="l2sq", alpha=1e-3, iters=2000, tol=1e-5, dtype=np.float32),
    # the n=4096 workload at a quarter of the batch: the profiling case (a few hundred MB on the device)
    "batch1024_n4096_l2_l2sq": dict(id=3, B=1024, n=4096, k=128, nnz=5, eps=1e-2, datafit="l2", lam=1.0,
                                    penalty="l2sq", alpha=1e-3, iters=2000, tol=1e-5, dtype=np.float32),
    "ragged10000_tv_l1": dict(id=4, count=10000, datafit="tv", lam=1.0, penalty="l1", alpha=1e-2,
                              iters=2000, tol=1e-5, dtype=np.float32),
    "warmstart_n2048_kl_l2sq": dict(id=5, n=2048, k=64, nnz=5, eps=5e-3, datafit="kl", lam=1.0,
                                    penalty="l2sq", alpha=1e-3, iters=2000, tol=1e-5, dtype=np.float32),
    # one target on a fine grid: the stored kernel (1 GiB as BF16 hi/lo) is streamed from HBM twice
    # per iteration; the same datafit and penalty as the n=4096 batch
    "hbm_single_n16384_l2_l2sq": dict(id=6, B=1, n=16384, k=128, nnz=5, eps=1e-2, datafit="l2", lam=1.0,
                                      penalty="l2sq", alpha=1e-3, iters=2000, tol=1e-5, dtype=np.float32),
    # the paper's scalability test at its largest size: truncated cost rho |x_i - x_j| (< 10 samples),
    # k = n / 10 truncated Gaussians, OT ridge (L2 datafit, squared-l2 penalty), 32 targets
    "banded32_n100000_ridge": dict(id=7, B=32, n=100000, eps=1e-3, datafit="l2", lam=1.0, penalty="l2sq",
                                   alpha=1e-3, iters=2000, tol=1e-5, dtype=np.float32),
}
