"""GPU parity of the banded-cost, sparse-dictionary solve (otlm_solve_banded) against the FP64
oracle's banded solve (itself pinned to the dense solve on CPU), on the inputs of the paper's
scalability test (App. "Performance Scalability Tests": x_i = i, cost rho |x_i - x_j| below 10
samples, k = n / 10 truncated Gaussians, lam = 1, alpha = eps = 1e-3) and on a non-symmetric
truncated cost with holes.

Bar: relative L1 1e-5 in w and t = Q^T 1, as for the other FP32 paths, at every eps including the
scalability test's 1e-3, where the log2 potentials reach lam / (eps ln2) = 1443: the kernels carry
them as split pairs (an integer-valued part and a fraction) so that FP32 rounding acts on numbers of
the size of the result, and take the datafit step and the MM sum through FP64."""
import numpy as np
import pytest

import oracle
import spectra

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2504_04609_gb300 import otlm as api  # noqa: E402
from scipy.sparse import csc_matrix  # noqa: E402

TOL32 = 1e-5


def rel_l1(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300))


def _w0(y, x_col):
    k = x_col.shape[0]
    return (np.asarray(y, dtype=np.float64).sum(axis=-1)[..., None] / (k * x_col)) * np.ones(
        np.shape(y)[:-1] + (k,))


def _gpu(d, datafit, penalty, eps, lam, alpha, iters, tol=0.0, beta=0.0, poll_every=8):
    dev = "cuda"
    Cd = torch.tensor(np.asarray(d["Cd"], dtype=np.float32), device=dev)
    col_ptr = torch.tensor(d["col_ptr"], dtype=torch.int32, device=dev)
    row_idx = torch.tensor(d["row_idx"], dtype=torch.int32, device=dev)
    val = torch.tensor(np.asarray(d["val"], dtype=np.float32), device=dev)
    y = torch.tensor(np.asarray(d["y"], dtype=np.float32), device=dev)
    B, n = y.shape
    w = torch.tensor(_w0(d["y"], d["x_col"]).astype(np.float32), device=dev)
    g = torch.zeros_like(y)
    t = torch.empty_like(y)
    it = torch.empty(B, dtype=torch.int32, device=dev)
    err = torch.empty(B, device=dev)
    st = torch.empty(B, dtype=torch.int32, device=dev)
    h = api.Handle(64, 8, B, "fp32", datafit, penalty, iters, tol, poll_every,
                   stream=torch.cuda.current_stream().cuda_stream, beta=beta)
    h.solve_banded(Cd, d["h"], col_ptr, row_idx, val, y, eps, lam, alpha, w, g, t, it, err, st)
    torch.cuda.synchronize()
    h.close()
    return dict(w=w.cpu().numpy(), g=g.cpu().numpy(), t=t.cpu().numpy(), iters=it.cpu().numpy(),
                err=err.cpu().numpy(), status=st.cpu().numpy())


def _oracle(d, p, datafit, penalty, eps, lam, alpha, iters, tol=0.0, beta=0.0):
    n, k = d["n"], d["k"]
    X = csc_matrix((np.asarray(d["val"], dtype=np.float64), d["row_idx"], d["col_ptr"]), shape=(n, k))
    y = np.asarray(d["y"][p], dtype=np.float64)
    return oracle.solve_log_banded(np.asarray(d["Cd"], dtype=np.float64), d["h"], X, y, eps, lam, alpha, datafit,
                                   penalty, _w0(y, d["x_col"]), iters, tol=tol, beta=beta)


@pytest.mark.parametrize("datafit,penalty", [
    ("l2", "l2sq"),       # OT ridge of the scalability test (potentials near 1e3 log2 units)
    ("tv", "l1"),         # OT-TV of the scalability test (TV clamp at 1443 log2 units)
    ("kl", "elastic"),
    ("poisson", "l1"),    # Poisson at eps = 1e-3: potentials up to lam / (eps ln2) as for TV
])
def test_scalability_inputs_trajectory_parity(datafit, penalty):
    """5 targets (a group of 4 per CTA and a short group of 1), n = 2300 (nine 256-bin tiles, the
    last ragged), k = 230, hw = 9, eps = alpha = 1e-3, 40 iterations."""
    d = spectra.scaling_batch(61, 5, 2300)
    r = _gpu(d, datafit, penalty, 1e-3, 1.0, 1e-3, 40, beta=2e-3)
    assert np.all(r["iters"] == 40) and np.all(r["status"] == api.MAX_ITER)
    for p in range(5):
        o = _oracle(d, p, datafit, penalty, 1e-3, 1.0, 1e-3, 40, beta=2e-3)
        ew, et = rel_l1(r["w"][p], o["w"]), rel_l1(r["t"][p], o["t"])
        assert ew <= TOL32 and et <= TOL32, (p, ew, et)


@pytest.mark.parametrize("datafit,penalty", [("l2", "l2sq"), ("tv", "l1"), ("kl", "l1")])
def test_nonsymmetric_truncated_cost_with_holes(datafit, penalty):
    """The oracle pins' non-symmetric banded cost (drift for i > j, forbidden pairs inside the
    band), n = 60, hw = 5: the target apply must read column j's costs from the right diagonals."""
    from tests.test_oracle_pins import _banded_case
    C, Cd, X, y = _banded_case()
    cp, ri, vv = spectra.scaling_dictionary(60, 6)
    d = dict(Cd=spectra.to_dtype(Cd, np.float32), h=5, col_ptr=cp, row_idx=ri, val=vv,
             y=np.stack([y, y[::-1].copy()]), n=60, k=6,
             x_col=np.add.reduceat(np.asarray(vv, dtype=np.float32).astype(np.float64), cp[:-1]))
    d["y"] = spectra.to_dtype(d["y"], np.float32)
    d["val"] = spectra.to_dtype(vv, np.float32)
    r = _gpu(d, datafit, penalty, 5e-3, 1.0, 1e-3, 30)
    for p in range(2):
        o = _oracle(d, p, datafit, penalty, 5e-3, 1.0, 1e-3, 30)
        ew, et = rel_l1(r["w"][p], o["w"]), rel_l1(r["t"][p], o["t"])
        assert ew <= TOL32 and et <= TOL32, (p, ew, et)


def test_full_size_n100000_to_tolerance():
    """The measured configuration: 32 targets at n = 100000, k = 10000, OT ridge, solved to the
    1e-5 tolerance as the benchmark solves them (about 700 iterations).  Target 0 is compared with
    the oracle's banded solve run for the GPU's own iteration count, and its stop with the oracle's
    stop under the same rule (equal, or one apart where the oracle's violation at the deciding
    iteration lies within 1 % of tol)."""
    d = spectra.scaling_batch(7, 32, 100000)
    r = _gpu(d, "l2", "l2sq", 1e-3, 1.0, 1e-3, 2000, tol=1e-5, poll_every=16)
    assert np.all(r["status"] == api.CONVERGED)
    gi = int(r["iters"][0])
    o = _oracle(d, 0, "l2", "l2sq", 1e-3, 1.0, 1e-3, gi + 1, tol=1e-5)
    if gi != o["iters"]:
        near = np.abs(o["err_hist"] / 1e-5 - 1) < 1e-2
        assert abs(gi - o["iters"]) == 1 and near.any(), (gi, o["iters"])
        o = _oracle(d, 0, "l2", "l2sq", 1e-3, 1.0, 1e-3, gi)
    ew, et = rel_l1(r["w"][0], o["w"]), rel_l1(r["t"][0], o["t"])
    assert ew <= TOL32 and et <= TOL32, (gi, ew, et)


def test_stopping_rule_matches_oracle():
    """tol = 1e-5 at eps = 3e-3 (about 120 iterations): each problem stops at the oracle's
    iteration, up to one where the oracle's violation sits within 1 % of tol at the deciding check,
    and its state matches the oracle run for the GPU's own iteration count."""
    d = spectra.scaling_batch(62, 3, 1500)
    r = _gpu(d, "kl", "l2sq", 3e-3, 1.0, 1e-3, 3000, tol=1e-5)
    for p in range(3):
        o = _oracle(d, p, "kl", "l2sq", 3e-3, 1.0, 1e-3, 3000, tol=1e-5)
        gi = int(r["iters"][p])
        assert r["status"][p] == api.CONVERGED
        if gi != o["iters"]:
            near = np.abs(o["err_hist"] / 1e-5 - 1) < 1e-2
            assert abs(gi - o["iters"]) == 1 and near.any(), (p, gi, o["iters"])
        assert float(r["err"][p]) <= 1e-5
        o2 = _oracle(d, p, "kl", "l2sq", 3e-3, 1.0, 1e-3, gi)
        assert rel_l1(r["w"][p], o2["w"]) <= TOL32 and rel_l1(r["t"][p], o2["t"]) <= TOL32


def test_invalid_inputs_are_refused():
    d = spectra.scaling_batch(63, 1, 300)
    dev = "cuda"
    Cd = torch.tensor(d["Cd"], device=dev)
    cp = torch.tensor(d["col_ptr"], dtype=torch.int32, device=dev)
    ri = torch.tensor(d["row_idx"], dtype=torch.int32, device=dev)
    val = torch.tensor(d["val"], device=dev)
    y = torch.tensor(d["y"], device=dev)
    w = torch.ones(1, d["k"], device=dev)
    h = api.Handle(64, 8, 1, "fp32", "kl", "l1", 5, 0.0)
    bad_ri = ri.clone()
    bad_ri[3] = 300  # row index outside [0, n)
    with pytest.raises(api.OTLMError):
        h.solve_banded(Cd, d["h"], cp, bad_ri, val, y, 1e-2, 1.0, 1e-3, w)
    zero = val.clone()
    zero[int(d["col_ptr"][2]):int(d["col_ptr"][3])] = 0.0  # a column of mass 0
    with pytest.raises(api.OTLMError):
        h.solve_banded(Cd, d["h"], cp, ri, zero, y, 1e-2, 1.0, 1e-3, w)
    nan_cost = Cd.clone()
    nan_cost[4, 10] = float("nan")
    with pytest.raises(api.OTLMError):
        h.solve_banded(nan_cost, d["h"], cp, ri, val, y, 1e-2, 1.0, 1e-3, w)
    with pytest.raises(api.OTLMError):  # half-width beyond 64
        h.solve_banded(torch.full((131, 300), float("inf"), device=dev), 65, cp, ri, val, y, 1e-2, 1.0, 1e-3, w)
    # a valid call on the same handle still works after the refusals
    h.solve_banded(Cd, d["h"], cp, ri, val, y, 1e-2, 1.0, 1e-3, w)
    torch.cuda.synchronize()
    h.close()
    assert torch.isfinite(w).all()
    h64 = api.Handle(64, 8, 1, "fp64", "kl", "l1", 5, 0.0)
    with pytest.raises(api.OTLMError):
        h64.solve_banded(Cd, d["h"], cp, ri, val, y, 1e-2, 1.0, 1e-3, w)
    h64.close()


@pytest.mark.parametrize("delta,B", [(41.0, 5), (41.0, 9), (4.0, 9), (15.0, 9), (10.0, 1)])
def test_band_buckets_and_problem_groups(delta, B):
    """Every band-width bucket (half-width 3: 9 diagonals in registers; 9: 19; 14: 33; 40: read
    from global memory) with one problem per CTA (B < 4) and four (B = 5, 9: a last group of one
    problem), n = 700 (a ragged third tile), eps = 5e-2 so that the far diagonals carry weight."""
    n, k = 700, 70
    Cd, h = spectra.truncated_cost_band(n, rho=0.01, delta=delta)
    cp, ri, vv = spectra.scaling_dictionary(n, k)
    Y = np.stack([spectra.scaling_target(n, k, np.random.default_rng(640 + p)) for p in range(B)])
    vv32 = spectra.to_dtype(vv, np.float32)
    d = dict(Cd=spectra.to_dtype(Cd, np.float32), h=h, col_ptr=cp, row_idx=ri, val=vv32,
             y=spectra.to_dtype(Y, np.float32), n=n, k=k, x_col=np.add.reduceat(vv32.astype(np.float64), cp[:-1]))
    r = _gpu(d, "kl", "l1", 5e-2, 1.0, 1e-3, 25)
    for p in range(B):
        o = _oracle(d, p, "kl", "l1", 5e-2, 1.0, 1e-3, 25)
        ew, et = rel_l1(r["w"][p], o["w"]), rel_l1(r["t"][p], o["t"])
        assert ew <= TOL32 and et <= TOL32, (p, h, ew, et)
