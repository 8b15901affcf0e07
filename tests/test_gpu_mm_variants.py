"""GPU parity of the weight-update variants against the FP64 oracle: the elastic-net penalty
alpha ||w||_1 + (beta/2) ||w||^2 (Table 2, last row, with App. A's stationarity condition) and
several MM steps per outer iteration, all with the same a = K u1 (Sec. 4.2).  Every solver path
is covered: FP32 and FP64 (SIMT MM kernel), tensor cores (TF32 dictionary GEMMs around the update
kernel), the uneven-batch persistent kernel, and the FP64 objective.  Bars as in the other parity
tests: relative L1 1e-5 for FP32 arithmetic, 1e-9 for FP64."""
import numpy as np
import pytest

import oracle
import spectra

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2504_04609_gb300 import otlm as api  # noqa: E402

TOL32 = 1e-5
TOL64 = 1e-9

CASES = [  # (datafit, penalty, eps, lam, alpha, beta, mm_steps)
    ("kl", "elastic", 1e-2, 1.0, 5e-3, 1e-2, 1),
    ("l2", "elastic", 1e-2, 1.0, 1e-3, 5e-3, 3),
    ("kl", "l1", 5e-3, 1.0, 1e-2, 0.0, 4),
    ("tv", "l2sq", 2e-2, 1.0, 1e-3, 0.0, 2),
]


def rel_l1(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300))


def _gpu(d, case, iters, precision):
    datafit, penalty, eps, lam, alpha, beta, mm = case
    dt = torch.float64 if precision == "fp64" else torch.float32
    x, D, y = (torch.tensor(d[k], dtype=dt, device="cuda") for k in ("x", "D", "y"))
    w = torch.tensor(spectra.initial_weights(d["y"], d["D"]), dtype=dt, device="cuda")
    r = api.solve(x, D, y, eps, lam, alpha, datafit, penalty, w, max_iter=iters, precision=precision,
                  poll_every=4, beta=beta, mm_steps=mm)
    return {k: getattr(r, k).cpu().numpy() for k in ("w", "g", "t", "iters", "status")}


def _oracle(x, D, y, case, iters, eps=None):
    datafit, penalty, eps_c, lam, alpha, beta, mm = case
    D = np.asarray(D, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return oracle.solve_log(spectra.squared_cost(np.asarray(x, dtype=np.float64)), D, y,
                            eps_c if eps is None else eps, lam, alpha, datafit, penalty,
                            spectra.initial_weights(y, D), iters, beta=beta, mm_steps=mm)


@pytest.mark.parametrize("precision", ["fp32", "bf16tc"])
@pytest.mark.parametrize("case", CASES)
def test_fp32_and_tensorcore_trajectory_parity(case, precision):
    """9 problems (a split-reduction batch on the tensor-core path), n = 300 (ragged row tiles),
    k = 12, 30 iterations."""
    d = spectra.batch(51, 9, 300, 12, 3)
    r = _gpu(d, case, 30, precision)
    assert np.all(r["iters"] == 30) and np.all(r["status"] == api.MAX_ITER)
    for p in range(9):
        o = _oracle(d["x"], d["D"], d["y"][p], case, 30)
        assert rel_l1(r["w"][p], o["w"]) <= TOL32, (p, rel_l1(r["w"][p], o["w"]))
        assert rel_l1(r["t"][p], o["t"]) <= TOL32, (p, rel_l1(r["t"][p], o["t"]))


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[2]])
def test_fp64_trajectory_parity(case):
    d = spectra.batch(52, 3, 257, 33, 4, dtype=np.float64)
    r = _gpu(d, case, 40, "fp64")
    for p in range(3):
        o = _oracle(d["x"], d["D"], d["y"][p], case, 40)
        assert rel_l1(r["w"][p], o["w"]) <= TOL64
        assert rel_l1(r["t"][p], o["t"]) <= TOL64


def test_tensorcore_inner_steps_over_two_column_tiles():
    """130 problems: two 128-wide column tiles of every GEMM, no split reduction."""
    case = ("l2", "elastic", 1e-2, 1.0, 1e-3, 5e-3, 2)
    d = spectra.batch(53, 130, 256, 16, 3)
    r = _gpu(d, case, 15, "bf16tc")
    for p in range(0, 130, 7):
        o = _oracle(d["x"], d["D"], d["y"][p], case, 15)
        assert rel_l1(r["w"][p], o["w"]) <= TOL32, (p, rel_l1(r["w"][p], o["w"]))
        assert rel_l1(r["t"][p], o["t"]) <= TOL32, (p, rel_l1(r["t"][p], o["t"]))


def test_ragged_elastic_with_inner_steps():
    """Eight uneven problems (own n, k, eps) through the persistent kernel, elastic net, 3 MM steps."""
    case = ("kl", "elastic", None, 1.0, 5e-3, 1e-2, 3)
    probs = spectra.ragged(54, 8, n_range=(256, 700), k_range=(8, 60))
    rb = api.ragged_batch(probs)
    w = torch.tensor(np.concatenate([spectra.initial_weights(p["y"], p["D"]) for p in probs]).astype(np.float32),
                     device="cuda")
    g = torch.zeros_like(rb.y)
    t = torch.empty_like(rb.y)
    B = len(probs)
    it = torch.empty(B, dtype=torch.int32, device="cuda")
    err = torch.empty(B, device="cuda")
    st = torch.empty(B, dtype=torch.int32, device="cuda")
    h = api.Handle(max(p["n"] for p in probs), max(p["k"] for p in probs), B, "fp32", "kl", "elastic", 20, 0.0,
                   stream=torch.cuda.current_stream().cuda_stream, beta=1e-2, mm_steps=3)
    h.solve_ragged(rb, 1.0, 5e-3, w, g, t, it, err, st)
    torch.cuda.synchronize()
    h.close()
    on, okk = rb.off_n.cpu().numpy(), rb.off_k.cpu().numpy()
    wn, tn = w.cpu().numpy(), t.cpu().numpy()
    assert np.all(it.cpu().numpy() == 20)
    for i, p in enumerate(probs):
        o = _oracle(p["x"], p["D"], p["y"], case, 20, eps=p["eps"])
        wi, ti = wn[okk[i]:okk[i] + p["k"]], tn[on[i]:on[i] + p["n"]]
        assert rel_l1(wi, o["w"]) <= TOL32, (i, rel_l1(wi, o["w"]))
        assert rel_l1(ti, o["t"]) <= TOL32, (i, rel_l1(ti, o["t"]))


def test_elastic_objective_and_gap_match_oracle():
    """Primal alpha ||w||_1 + (beta/2) ||w||^2 term and the conjugate (v - alpha)+^2 / (2 beta)."""
    case = CASES[0]
    datafit, penalty, eps, lam, alpha, beta, _ = case
    d = spectra.batch(55, 3, 200, 10, 3)
    r = _gpu(d, case, 30, "fp32")
    h = api.Handle(200, 10, 3, "fp32", datafit, penalty, 30, 0.0, 4, beta=beta)
    P = torch.empty(3, dtype=torch.float64, device="cuda")
    Dv = torch.empty(3, dtype=torch.float64, device="cuda")
    h.objective(torch.tensor(d["x"], device="cuda"), torch.tensor(d["D"], device="cuda"),
                torch.tensor(d["y"], device="cuda"), eps, lam, alpha, torch.tensor(r["w"], device="cuda"),
                torch.tensor(r["g"], device="cuda"), P, Dv)
    torch.cuda.synchronize()
    h.close()
    C = spectra.squared_cost(d["x"].astype(np.float64))
    for p in range(3):
        Po, Do, _ = oracle.objective_and_dual(r["w"][p].astype(np.float64), r["g"][p].astype(np.float64), C,
                                              d["D"].astype(np.float64), d["y"][p].astype(np.float64), eps, lam,
                                              alpha, datafit, penalty, beta)
        assert P[p].item() == pytest.approx(Po, rel=2e-6)
        assert Dv[p].item() == pytest.approx(Do, rel=2e-6)
        assert P[p].item() - Dv[p].item() >= -1e-6 * abs(Po)


def test_config_validation_and_one_step_default():
    """ELASTIC needs a finite beta > 0; mm_steps is 0..64 and 0 means one step."""
    for kw in (dict(beta=0.0), dict(beta=float("inf"))):
        with pytest.raises(api.OTLMError):
            api.Handle(64, 4, 2, "fp32", "kl", "elastic", 5, 0.0, **kw)
    for mm in (-1, 65):
        with pytest.raises(api.OTLMError):
            api.Handle(64, 4, 2, "fp32", "kl", "l1", 5, 0.0, mm_steps=mm)
    d = spectra.batch(56, 2, 64, 4, 2)
    a = _gpu(d, ("kl", "l1", 2e-2, 1.0, 1e-2, 0.0, 0), 10, "fp32")
    b = _gpu(d, ("kl", "l1", 2e-2, 1.0, 1e-2, 0.0, 1), 10, "fp32")
    np.testing.assert_array_equal(a["w"], b["w"])
    np.testing.assert_array_equal(a["t"], b["t"])
