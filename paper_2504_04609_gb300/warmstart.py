"""Learned warm start: label generation with the solver, training, and cold-vs-warm evaluation.

Orchestration only: every numerical step runs in libotlm.so (the solver through otlm_solve, the
network through otlm_ws_*).  Labels are the solver's own results: each training target is solved
from the cold start (u1 = 1, w0_j = sum(y) / (k x_j)) to the stopping tolerance, and the network
learns (g / eps, log w) of that solution.  At inference the prediction replaces the cold start; the
same solver then runs to the same tolerance, so the plain iteration decides convergence: a poor
prediction can only cost iterations, never accuracy (non-finite predictions fall back to the cold
start inside otlm_ws_predict).
"""
from __future__ import annotations

import time

import numpy as np

from . import otlm as api

# float32 tensors on the device; the caller owns torch
G_FLOOR = -200.0  # g / eps labels below this are clipped (bins with y = 0 carry -inf; masked)


def cold_weights(y, D, chunk=4096, stream=None):
    """The cold-start weights w0_j = sum(y) / (k x_j) on the device (otlm_initial_weights)."""
    import torch
    B, n = y.shape
    k = D.shape[1]
    w0 = torch.empty(B, k, dtype=y.dtype, device=y.device)
    h = api.Handle(n, k, min(B, chunk), "fp64" if y.dtype == torch.float64 else "fp32", stream=stream)
    for s in range(0, B, chunk):
        h.initial_weights(D, y[s:s + chunk], w0[s:s + chunk])
    h.close()
    return w0


def solve(x, D, y, cfg, w0, g0=None, tol=None, stream=None, precision="fp32"):
    """Solve a batch with the library from (w0, g0); returns (w, g, t, iters, err, status, seconds)."""
    import torch
    B, n = y.shape
    k = D.shape[1]
    h = api.Handle(n, k, B, precision, cfg["datafit"], cfg["penalty"], cfg["iters"], cfg["tol"] if tol is None else tol,
                   poll_every=4, stream=stream)
    w = w0.clone()
    g = torch.zeros_like(y) if g0 is None else g0.clone()
    t = torch.empty_like(y)
    it = torch.empty(B, dtype=torch.int32, device=y.device)
    err = torch.empty(B, dtype=torch.float32, device=y.device)
    st = torch.empty(B, dtype=torch.int32, device=y.device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h.solve(x, D, y, cfg["eps"], cfg["lam"], cfg["alpha"], w, g, t, it, err, st)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    h.close()
    return w, g, t, it, err, st, secs


def make_labels(net, x, D, y, cfg, chunk=4096):
    """Targets [B][n + k] = [g / eps, log w] of the cold-start solutions (solved in chunks; the
    transform runs in otlm_ws_make_targets)."""
    import torch
    B, n = y.shape
    k = D.shape[1]
    out = torch.empty(B, n + k, dtype=torch.float32, device=y.device)
    for s in range(0, B, chunk):
        yb = y[s:s + chunk]
        w, g, _, _, _, st, _ = solve(x, D, yb, cfg, cold_weights(yb, D))
        net.make_targets(g, w, cfg["eps"], G_FLOOR, out[s:s + chunk])
    return out


def normalization(net, targets):
    """Per-output mean and std over the finite entries (std floored at 1e-3), fitted on the device
    (otlm_ws_fit_normalization) and set on the network; returns (mean, std) device tensors."""
    import torch
    cols = targets.shape[1]
    mean = torch.empty(cols, dtype=torch.float32, device=targets.device)
    std = torch.empty_like(mean)
    net.fit_normalization(targets, mean, std)
    return mean, std


def train(net, y, targets, epochs, batch, lr, weight_decay=0.0, seed=0, log_every=0):
    """Mini-batch AdamW over (y, targets); returns the per-step losses (host floats)."""
    import torch
    rng = np.random.default_rng(seed)
    N = y.shape[0]
    loss_dev = torch.zeros(1, device=y.device)
    losses = []
    step = 0
    steps_per_epoch = N // batch
    total = epochs * steps_per_epoch
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(N)).to(y.device)
        for s in range(steps_per_epoch):
            idx = perm[s * batch:(s + 1) * batch]
            yb = y.index_select(0, idx).contiguous()
            tb = targets.index_select(0, idx).contiguous()
            # cosine decay of the learning rate
            lr_t = lr * 0.5 * (1 + np.cos(np.pi * step / max(total, 1)))
            net.train_step(yb, tb, lr_t, weight_decay, loss_dev)
            step += 1
            if log_every and step % log_every == 0:
                losses.append(float(loss_dev.item()))
    torch.cuda.synchronize()
    losses.append(float(loss_dev.item()))
    return losses


def predict(net, y, D, eps, chunk=None, cold_w=None):
    """The network's initial state (g0, w0) for y; rows whose prediction is not finite take the
    cold start (cold_w, computed here when not given)."""
    import torch
    B, n = y.shape
    k = D.shape[1]
    g0 = torch.empty_like(y)
    w0 = torch.empty(B, k, device=y.device)
    cw = cold_weights(y, D) if cold_w is None else cold_w
    chunk = chunk or net.batch_max
    for s in range(0, B, chunk):
        net.predict(y[s:s + chunk], eps, cw[s:s + chunk], g0[s:s + chunk], w0[s:s + chunk])
    return g0, w0


def evaluate(net, x, D, y, cfg, precision="fp32"):
    """Cold start vs learned warm start on the same targets, same solver and tolerance."""
    import torch
    cw = cold_weights(y, D)
    wc, gc, tc, itc, _, stc, sc = solve(x, D, y, cfg, cw, precision=precision)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g0, w0 = predict(net, y, D, cfg["eps"], cold_w=cw)
    torch.cuda.synchronize()
    t_pred = time.perf_counter() - t0
    ww, gw, tw, itw, _, stw, sw = solve(x, D, y, cfg, w0, g0, precision=precision)
    rel = lambda a, b: ((a - b).abs().sum(dim=1) / b.abs().sum(dim=1).clamp(min=1e-30))  # noqa: E731
    return dict(cold_iters=itc.cpu().numpy(), warm_iters=itw.cpu().numpy(), cold_status=stc.cpu().numpy(),
                warm_status=stw.cpu().numpy(), cold_s=sc, warm_s=sw + t_pred, predict_s=t_pred,
                w_rel_diff=rel(ww, wc).cpu().numpy(), t_rel_diff=rel(tw, tc).cpu().numpy())
