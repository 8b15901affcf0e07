"""Learned warm start on the GPU: the network's gradients against the FP64 reference, training
gains over the cold start, and the fallback to the cold start."""
import numpy as np
import pytest

import spectra
from oracle import mlp as ref

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2504_04609_gb300 import otlm as api  # noqa: E402
from paper_2504_04609_gb300 import warmstart as ws  # noqa: E402


def test_gradients_match_fp64_reference():
    n, k, H, B = 96, 10, 48, 24
    net = api.WarmStart(n, k, H, B, seed=7)
    rng = np.random.default_rng(1)
    y = rng.uniform(0.0, 1.0, (B, n)).astype(np.float32)
    y[:, :5] = 0.0
    t = rng.normal(-20, 5, (B, n + k)).astype(np.float32)
    t[:, 3] = -np.inf
    mean = rng.normal(-20, 1, n + k).astype(np.float32)
    std = rng.uniform(2, 6, n + k).astype(np.float32)
    dev = lambda a: torch.tensor(a, device="cuda")  # noqa: E731
    net.set_normalization(dev(mean), dev(std))
    P = net.num_params
    params = torch.empty(P, device="cuda")
    grads = torch.empty(P, device="cuda")
    loss = torch.empty(1, device="cuda")
    net.get_params(params)
    net.gradients(dev(y), dev(t), grads, loss)
    torch.cuda.synchronize()
    dims = ref.layer_dims(n, k, H)
    lo, go = ref.loss_and_grad(params.cpu().numpy().astype(np.float64), dims, y, t, mean.astype(np.float64),
                               std.astype(np.float64), round_weights=True)
    assert loss.item() == pytest.approx(lo, rel=1e-4)
    # element by element: |gpu - ref| <= 1e-5 M, where M is the entry's sum of absolute term
    # values through the chain rule (oracle.mlp.grad_magnitudes).  FP32 evaluation errs by about
    # sqrt(K) u M for a reduction of length K (K <= n + 1 = 97 here, u = 2^-24: ~6e-7 M) and by
    # at most K u M ~ 6e-6 M; 1e-5 M sits above both.
    mag = ref.grad_magnitudes(params.cpu().numpy().astype(np.float64), dims, y, t, mean.astype(np.float64),
                              std.astype(np.float64), round_weights=True)
    g = grads.cpu().numpy().astype(np.float64)
    assert g.shape == go.shape == mag.shape
    bad = np.abs(g - go) > 1e-5 * mag + 1e-30
    assert not bad.any(), (int(bad.sum()), float(np.max(np.abs(g - go) / (mag + 1e-30))))
    net.close()


@pytest.mark.parametrize("n,k,H,B", [(300, 12, 64, 200), (96, 10, 48, 24)])
def test_tensor_core_forward_matches_fp64_reference(n, k, H, B):
    """otlm_ws_predict runs the forward pass on the tensor cores (BF16 weights times activations
    carried as BF16 hi/lo pairs).  Its decoded outputs must match the FP64 forward pass with the
    same BF16 weights to 1e-3 (relative to 1 + |value|).  The first shape takes the bulk-copy
    epilogue (output widths multiples of 4) and spans two 128-row blocks of the batch; the second
    takes the per-element epilogue (n + k = 106)."""
    net = api.WarmStart(n, k, H, B, seed=11)
    rng = np.random.default_rng(4)
    y = rng.uniform(0.0, 1.0, (B, n)).astype(np.float32)
    y[:, :7] = 0.0
    mean = rng.normal(0, 1, n + k).astype(np.float32)
    std = rng.uniform(0.5, 2.0, n + k).astype(np.float32)
    dev = lambda a: torch.tensor(a, device="cuda")  # noqa: E731
    net.set_normalization(dev(mean), dev(std))
    eps = 5e-3
    cw = torch.full((B, k), 0.25, device="cuda")
    g0 = torch.empty(B, n, device="cuda")
    w0 = torch.empty(B, k, device="cuda")
    net.predict(dev(y), eps, cw, g0, w0)
    params = torch.empty(net.num_params, device="cuda")
    net.get_params(params)
    torch.cuda.synchronize()
    z, _, _ = ref.forward(params.cpu().numpy().astype(np.float64), ref.layer_dims(n, k, H), y, round_weights=True)
    v_ref = z * std.astype(np.float64) + mean.astype(np.float64)
    v_gpu = np.concatenate([g0.cpu().numpy().astype(np.float64) / eps, np.log(w0.cpu().numpy().astype(np.float64))],
                           axis=1)
    assert np.all(np.isfinite(v_gpu))
    np.testing.assert_array_less(np.abs(v_gpu - v_ref), 1e-3 * (1.0 + np.abs(v_ref)))
    net.close()


def _dataset(first, count, n, k):
    d = spectra.batch(5, count, n, k, 5, first=first)
    return (torch.tensor(d["x"], device="cuda"), torch.tensor(d["D"], device="cuda"),
            torch.tensor(d["y"], device="cuda"))


def test_trained_network_cuts_iterations_and_keeps_the_solution():
    """n = 256, k = 16, KL datafit + squared l2, eps = 5e-3: 4000 training problems labelled by the
    solver, 400 held out.  The warm start must converge every problem to the same tolerance in
    fewer iterations on average."""
    cfg = dict(spectra.WORKLOADS["warmstart_n2048_kl_l2sq"])
    n, k = 256, 16
    x, D, ytr = _dataset(0, 4000, n, k)
    _, _, yte = _dataset(1_000_000, 400, n, k)
    net = api.WarmStart(n, k, 256, 256, seed=3)
    t = ws.make_labels(net, x, D, ytr, cfg)
    ws.normalization(net, t)
    losses = ws.train(net, ytr, t, epochs=40, batch=128, lr=2e-3, weight_decay=1e-5, log_every=200)
    assert losses[-1] < 0.5 * losses[0]
    res = ws.evaluate(net, x, D, yte, cfg)
    assert np.all(res["cold_status"] == api.CONVERGED) and np.all(res["warm_status"] == api.CONVERGED)
    assert res["warm_iters"].mean() < 0.9 * res["cold_iters"].mean(), (res["warm_iters"].mean(),
                                                                       res["cold_iters"].mean())
    # the warm-started solves follow the oracle started from the same predicted state
    _warm_start_oracle_parity(net, x, D, yte[:6], cfg)
    net.close()


def _warm_start_oracle_parity(net, x, D, y, cfg, iters=25):
    """Trajectory parity from the network's prediction: the GPU solve (FP32 and tensor-core paths)
    and the FP64 oracle both start from the predicted (g0, w0) as float32 values and run `iters`
    iterations; w and t must agree to 1e-5 relative L1 per problem (the FP32 bar)."""
    import oracle
    g0, w0 = ws.predict(net, y, D, cfg["eps"])
    xs, Ds, ys = x.cpu().numpy().astype(np.float64), D.cpu().numpy().astype(np.float64), y.cpu().numpy()
    g0n, w0n = g0.cpu().numpy().astype(np.float64), w0.cpu().numpy().astype(np.float64)
    C = spectra.squared_cost(xs)
    refs = [oracle.solve_log(C, Ds, ys[p].astype(np.float64), cfg["eps"], cfg["lam"], cfg["alpha"], cfg["datafit"],
                             cfg["penalty"], w0n[p], iters, g0=g0n[p]) for p in range(y.shape[0])]
    for prec in ("fp32", "bf16tc"):
        r = api.solve(x, D, y, cfg["eps"], cfg["lam"], cfg["alpha"], cfg["datafit"], cfg["penalty"], w0, g0,
                      max_iter=iters, precision=prec)
        w, t = r.w.cpu().numpy(), r.t.cpu().numpy()
        for p, o in enumerate(refs):
            ew = float(np.abs(w[p] - o["w"]).sum() / np.abs(o["w"]).sum())
            et = float(np.abs(t[p] - o["t"]).sum() / np.abs(o["t"]).sum())
            assert ew <= 1e-5 and et <= 1e-5, (prec, p, ew, et)


def test_initial_weights_entry_point_matches_its_definition():
    """otlm_initial_weights: w0_j = sum(y) / (k x_j) (reading A10) for FP32 and FP64 handles,
    against the same formula in FP64 on the host (FP32 rounding of the result only)."""
    d = spectra.batch(5, 37, 300, 12, 5, first=4_000_000)
    ref = spectra.initial_weights(d["y"].astype(np.float64), d["D"].astype(np.float64))
    for prec, dt, tol in (("fp32", torch.float32, 2e-7), ("fp64", torch.float64, 1e-15)):
        D = torch.tensor(d["D"], dtype=dt, device="cuda")
        y = torch.tensor(d["y"], dtype=dt, device="cuda")
        h = api.Handle(300, 12, 37, prec, stream=torch.cuda.current_stream().cuda_stream)
        w = torch.empty(37, 12, dtype=dt, device="cuda")
        h.initial_weights(D, y, w)
        torch.cuda.synchronize()
        h.close()
        np.testing.assert_allclose(w.cpu().numpy().astype(np.float64), ref, rtol=tol, atol=0)


def test_training_targets_and_normalization_entry_points():
    """otlm_ws_make_targets ([g / eps clipped at the floor, log w], -inf where g is not finite or
    w <= 0) and otlm_ws_fit_normalization (mean and std over the finite entries, std floored at
    1e-3) against the same definitions in FP64 numpy; the fitted statistics are the network's."""
    n, k, B = 40, 6, 3000
    net = api.WarmStart(n, k, 16, 16, seed=2)
    rng = np.random.default_rng(12)
    g = rng.normal(-0.5, 0.6, (B, n)).astype(np.float32)
    g[:, 0] = -np.inf
    g[::7, 3] = -np.inf
    g[:, 5] = 0.25  # a constant output: std floored
    w = rng.gamma(2.0, 1.0, (B, k)).astype(np.float32)
    w[::5, 2] = 0.0
    eps, floor = 5e-3, -200.0
    tg = torch.empty(B, n + k, device="cuda")
    net.make_targets(torch.tensor(g, device="cuda"), torch.tensor(w, device="cuda"), eps, floor, tg)
    mean = torch.empty(n + k, device="cuda")
    std = torch.empty(n + k, device="cuda")
    net.fit_normalization(tg, mean, std)
    torch.cuda.synchronize()
    g64 = g.astype(np.float64)
    with np.errstate(divide="ignore"):
        want = np.concatenate([np.where(np.isfinite(g64), np.maximum(g64 * np.float64(np.float32(1.0 / eps)), floor),
                                        -np.inf),
                               np.where(w > 0, np.log(w.astype(np.float64)), -np.inf)], axis=1)
    got = tg.cpu().numpy().astype(np.float64)
    fin = np.isfinite(want)
    assert np.array_equal(fin, np.isfinite(got))
    np.testing.assert_allclose(got[fin], want[fin], rtol=1e-6, atol=1e-6)
    cnt = np.maximum(fin.sum(axis=0), 1)  # an output with no finite target gets mean 0, std 1e-3
    mu = np.where(fin, got, 0).sum(axis=0) / cnt
    sd = np.maximum(np.sqrt((np.where(fin, got - mu, 0) ** 2).sum(axis=0) / cnt), 1e-3)
    np.testing.assert_allclose(mean.cpu().numpy(), mu, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(std.cpu().numpy(), sd, rtol=1e-5, atol=1e-6)
    assert std.cpu().numpy()[5] == pytest.approx(1e-3) and std.cpu().numpy()[0] == pytest.approx(1e-3)
    net.close()


def test_prediction_then_tensor_core_solve():
    """The network's forward pass and the tensor-core solver launch the same GEMM kernel from two
    translation units; each must set up its own copy.  Predict, then solve warm and cold on the
    tensor-core path in the same process."""
    cfg = dict(spectra.WORKLOADS["warmstart_n2048_kl_l2sq"])
    n, k = 256, 16
    x, D, y = _dataset(3_000_000, 64, n, k)
    net = api.WarmStart(n, k, 64, 64, seed=9)
    g0, w0 = ws.predict(net, y, D, cfg["eps"])
    for wi, gi in ((w0, g0), (ws.cold_weights(y, D), None)):
        r = ws.solve(x, D, y, cfg, wi, gi, precision="bf16tc")
        assert torch.all(r[5] == api.CONVERGED)
    net.close()


def test_non_finite_network_falls_back_to_the_cold_start():
    cfg = dict(spectra.WORKLOADS["warmstart_n2048_kl_l2sq"])
    n, k = 128, 8
    x, D, y = _dataset(2_000_000, 20, n, k)
    net = api.WarmStart(n, k, 32, 32, seed=5)
    nanp = torch.full((net.num_params,), float("nan"), device="cuda")
    net.set_params(nanp)
    g0, w0 = ws.predict(net, y, D, cfg["eps"])
    assert torch.all(g0 == 0)
    torch.testing.assert_close(w0, ws.cold_weights(y, D), rtol=0, atol=0)
    a = ws.solve(x, D, y, cfg, ws.cold_weights(y, D))
    b = ws.solve(x, D, y, cfg, w0, g0)
    assert torch.equal(a[0], b[0]) and torch.equal(a[3], b[3])
    net.close()
