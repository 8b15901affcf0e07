"""The stopping test inside the solve (Algorithm 1's "while not converged", reading A8) against the
FP64 oracle: the FP64 objective and duality gap of the returned state (check_every), the weight
change ||w_new - w_old||_1 / ||w_new||_1, and the two further stopping criteria (dw_tol, gap_tol),
on the FP32, FP64 and tensor-core paths, read through otlm_solve_stats.

Bars: the primal and dual of the returned state against oracle.objective_and_dual on that state
(FP64 sums of an FP32 evaluation, as otlm_objective's test: relative 2e-6; FP64 path 1e-9; the
tensor-core path evaluates its applies as BF16 hi/lo GEMMs, ~16 bits per sum: 2e-5).  The weight
change against the oracle's dw_hist at the same iteration: both weight vectors carry the 1e-5
trajectory bar, so the difference of two of them carries 2e-5 (absolute, relative to ||w||_1).
Stopping iterations: equal, or, where they differ, the oracle's deciding quantity lies within the
GPU's error of that quantity of its tolerance at every iteration (check) in between; the state is
then compared at the GPU's own iteration."""
import numpy as np
import pytest

import oracle
import spectra

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2504_04609_gb300 import otlm as api  # noqa: E402

TOL = {"fp32": 1e-5, "bf16tc": 1e-5, "fp64": 1e-9}
OBJ_TOL = {"fp32": 2e-6, "bf16tc": 2e-5, "fp64": 1e-9}
DW_TOL = {"fp32": 2e-5, "bf16tc": 2e-5, "fp64": 1e-9}


def rel_l1(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300))


def _gpu(d, prec, datafit, penalty, eps, lam, alpha, iters, tol=0.0, check_every=0, gap_tol=0.0, dw_tol=0.0):
    dt = torch.float64 if prec == "fp64" else torch.float32
    x, D, y = (torch.tensor(d[key], dtype=dt, device="cuda") for key in ("x", "D", "y"))
    B, n = y.shape
    k = D.shape[1]
    w = torch.tensor(spectra.initial_weights(d["y"], d["D"]), dtype=dt, device="cuda")
    g = torch.zeros_like(y)
    t = torch.empty_like(y)
    it = torch.empty(B, dtype=torch.int32, device="cuda")
    err = torch.empty(B, dtype=dt, device="cuda")
    st = torch.empty(B, dtype=torch.int32, device="cuda")
    dw = torch.empty(B, dtype=dt, device="cuda")
    h = api.Handle(n, k, B, prec, datafit, penalty, iters, tol, poll_every=4,
                   stream=torch.cuda.current_stream().cuda_stream, check_every=check_every, gap_tol=gap_tol,
                   dw_tol=dw_tol)
    h.solve(x, D, y, eps, lam, alpha, w, g, t, it, err, st)
    out = dict(dw=dw)
    if check_every > 0:
        out["P"] = torch.empty(B, dtype=torch.float64, device="cuda")
        out["D"] = torch.empty(B, dtype=torch.float64, device="cuda")
    h.solve_stats(B, dw, out.get("P"), out.get("D"))
    torch.cuda.synchronize()
    h.close()
    res = dict(w=w, g=g, t=t, iters=it, err=err, status=st, **out)
    return {key: v.cpu().numpy() for key, v in res.items()}


def _oracle(d, p, datafit, penalty, eps, lam, alpha, iters, **kw):
    x, D = d["x"].astype(np.float64), d["D"].astype(np.float64)
    y = d["y"][p].astype(np.float64)
    return oracle.solve_log(spectra.squared_cost(x), D, y, eps, lam, alpha, datafit, penalty,
                            spectra.initial_weights(y, D), iters, **kw)


CASES = [("kl", "l1", 5e-3, 1.0, 1e-2), ("l2", "l2sq", 1e-2, 1.0, 1e-3), ("tv", "l1", 2e-2, 1.0, 1e-2),
         ("poisson", "l2sq", 1e-2, 1.0, 1e-3), ("kl", "elastic", 1e-2, 1.0, 1e-3)]


@pytest.mark.parametrize("prec", ["fp32", "fp64", "bf16tc"])
@pytest.mark.parametrize("datafit,penalty,eps,lam,alpha", CASES[:4])
def test_returned_state_objective_and_weight_change(prec, datafit, penalty, eps, lam, alpha):
    """B = 5, n = 300 (two row tiles, ragged), k = 12, 23 iterations with checks every 10 (two
    checks and the final evaluation): the FP64 primal and dual that the solve reports for its
    returned state equal the oracle's objective_and_dual of that state, the gap is >= 0, and the
    last weight change equals the oracle's on the same trajectory."""
    d = spectra.batch(81, 5, 300, 12, 3)
    T = 23
    r = _gpu(d, prec, datafit, penalty, eps, lam, alpha, T, check_every=10)
    assert np.all(r["iters"] == T)
    x, D = d["x"].astype(np.float64), d["D"].astype(np.float64)
    C = spectra.squared_cost(x)
    for p in range(5):
        Po, Do, _ = oracle.objective_and_dual(r["w"][p].astype(np.float64), r["g"][p].astype(np.float64), C, D,
                                              d["y"][p].astype(np.float64), eps, lam, alpha, datafit, penalty)
        assert r["P"][p] == pytest.approx(Po, rel=OBJ_TOL[prec]), (p, r["P"][p], Po)
        assert r["D"][p] == pytest.approx(Do, rel=OBJ_TOL[prec]), (p, r["D"][p], Do)
        assert r["P"][p] - r["D"][p] >= -OBJ_TOL[prec] * abs(Po)
        o = _oracle(d, p, datafit, penalty, eps, lam, alpha, T)
        assert abs(float(r["dw"][p]) - o["dw_hist"][-1]) <= DW_TOL[prec], (p, r["dw"][p], o["dw_hist"][-1])
        assert rel_l1(r["w"][p], o["w"]) <= TOL[prec] and rel_l1(r["t"][p], o["t"]) <= TOL[prec]


def test_elastic_objective_through_otlm_objective_and_poisson_is_accepted():
    """otlm_objective now covers the Poisson datafit (its dual at g' = lam y / v' - lam) and the
    elastic net, against the oracle at the FP32 bar."""
    for datafit, penalty, eps, lam, alpha in (CASES[3], CASES[4], ("poisson", "l1", 2e-2, 1.0, 1e-2)):
        d = spectra.batch(82, 3, 160, 6, 2)
        d["y"][:, :20] = 0.0  # zero target bins: g = -lam there under the Poisson datafit
        dt = torch.float32
        x, D, y = (torch.tensor(d[key], dtype=dt, device="cuda") for key in ("x", "D", "y"))
        w = torch.tensor(spectra.initial_weights(d["y"], d["D"]), dtype=dt, device="cuda")
        r = api.solve(x, D, y, eps, lam, alpha, datafit, penalty, w, max_iter=25, beta=2e-3)
        h = api.Handle(160, 6, 3, "fp32", datafit, penalty, 25, 0.0, 4, beta=2e-3)
        P = torch.empty(3, dtype=torch.float64, device="cuda")
        Dv = torch.empty(3, dtype=torch.float64, device="cuda")
        h.objective(x, D, y, eps, lam, alpha, r.w, r.g, P, Dv)
        torch.cuda.synchronize()
        h.close()
        C = spectra.squared_cost(d["x"].astype(np.float64))
        for p in range(3):
            Po, Do, _ = oracle.objective_and_dual(r.w[p].cpu().numpy().astype(np.float64),
                                                  r.g[p].cpu().numpy().astype(np.float64), C,
                                                  d["D"].astype(np.float64), d["y"][p].astype(np.float64), eps,
                                                  lam, alpha, datafit, penalty, beta=2e-3)
            assert P[p].item() == pytest.approx(Po, rel=2e-6), (datafit, p)
            assert Dv[p].item() == pytest.approx(Do, rel=2e-6), (datafit, p)
            assert P[p].item() - Dv[p].item() >= -2e-6 * abs(Po)


@pytest.mark.parametrize("prec", ["fp32", "bf16tc"])
def test_weight_change_stopping_rule_matches_oracle(prec):
    """tol = 1e-5 and dw_tol = 3e-4 under KL + l1 at eps = 5e-3 (the weights settle long after the
    marginals: the rule takes 2-4x the iterations of the violation alone): each problem stops where
    the oracle with the same rule stops, or where the two differ the oracle's weight change at
    every iteration in between lies within the GPU's weight-change error (DW_TOL) of dw_tol; the
    state matches the oracle's at the GPU's own iteration count."""
    d = spectra.batch(83, 4, 256, 16, 5)
    dw_tol = 3e-4
    r = _gpu(d, prec, "kl", "l1", 5e-3, 1.0, 1e-2, 3000, tol=1e-5, dw_tol=dw_tol)
    assert np.all(r["status"] == api.CONVERGED)
    for p in range(4):
        o = _oracle(d, p, "kl", "l1", 5e-3, 1.0, 1e-2, 3000, tol=1e-5, dw_tol=dw_tol)
        gi, oi = int(r["iters"][p]), int(o["iters"])
        assert float(r["dw"][p]) <= dw_tol and float(r["err"][p]) <= 1e-5
        if gi != oi:
            full = _oracle(d, p, "kl", "l1", 5e-3, 1.0, 1e-2, max(gi, oi))
            between = full["dw_hist"][min(gi, oi) - 1:max(gi, oi) - 1]
            assert np.all(np.abs(between - dw_tol) <= DW_TOL[prec]), (p, gi, oi, between)
        assert oi > 1.5 * _oracle(d, p, "kl", "l1", 5e-3, 1.0, 1e-2, 3000, tol=1e-5)["iters"]
        o2 = _oracle(d, p, "kl", "l1", 5e-3, 1.0, 1e-2, gi)
        assert rel_l1(r["w"][p], o2["w"]) <= TOL[prec] and rel_l1(r["t"][p], o2["t"]) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "fp64", "bf16tc"])
def test_gap_stopping_rule_matches_oracle(prec):
    """The FP64 gap alone (tol = 0) decides, checked every 4 iterations, under TV + l1 at
    eps = 2e-2: gap_tol = 1e-5 relative (1e-4 on the tensor-core path, whose objective carries
    ~2e-5 relative error).  Each problem stops at the oracle's check, or where the two differ the
    oracle's relative gap at the checks in between lies within twice the objective bar of gap_tol;
    the reported gap of the returned state is under gap_tol; the state matches the oracle's at the
    GPU's iteration."""
    d = spectra.batch(84, 4, 200, 10, 3)
    args = ("tv", "l1", 2e-2, 1.0, 1e-2)
    gap_tol = 1e-4 if prec == "bf16tc" else 1e-5
    r = _gpu(d, prec, *args, 400, check_every=4, gap_tol=gap_tol)
    assert np.all(r["status"] == api.CONVERGED)
    for p in range(4):
        o = _oracle(d, p, *args, 400, check_every=4, gap_tol=gap_tol)
        gi, oi = int(r["iters"][p]), int(o["iters"])
        assert gi % 4 == 0 and r["P"][p] - r["D"][p] <= gap_tol * abs(r["P"][p])
        if gi != oi:
            full = _oracle(d, p, *args, max(gi, oi), check_every=4, gap_tol=1e-300)
            rel = {it: (P - Dv) / abs(P) for it, P, Dv in full["gap_hist"]}
            between = [rel[it] for it in range(min(gi, oi), max(gi, oi), 4)]
            assert all(abs(v - gap_tol) <= 2 * OBJ_TOL[prec] for v in between), (p, gi, oi, between)
        o2 = _oracle(d, p, *args, gi)
        assert rel_l1(r["w"][p], o2["w"]) <= TOL[prec] and rel_l1(r["t"][p], o2["t"]) <= TOL[prec]
