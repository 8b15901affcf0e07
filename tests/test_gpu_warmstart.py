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
    g = grads.cpu().numpy().astype(np.float64)
    off = 0
    for l in range(4):
        for size in (dims[l] * dims[l + 1], dims[l + 1]):
            a, b = g[off:off + size], go[off:off + size]
            assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b) + 1e-12, (l, size)
            off += size
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
    t = ws.make_labels(x, D, ytr, cfg)
    mean, std = ws.normalization(t)
    net = api.WarmStart(n, k, 256, 256, seed=3)
    net.set_normalization(mean, std)
    losses = ws.train(net, ytr, t, epochs=40, batch=128, lr=2e-3, weight_decay=1e-5, log_every=200)
    assert losses[-1] < 0.5 * losses[0]
    res = ws.evaluate(net, x, D, yte, cfg)
    assert np.all(res["cold_status"] == api.CONVERGED) and np.all(res["warm_status"] == api.CONVERGED)
    assert res["warm_iters"].mean() < 0.9 * res["cold_iters"].mean(), (res["warm_iters"].mean(),
                                                                       res["cold_iters"].mean())
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
