"""FP64 CPU reference of the learned warm-start network (an extension of the solver; the paper has
no learned component).  TEST INFRASTRUCTURE ONLY, like the rest of oracle/.

Network: features x0 = [n y / sum(y), log sum(y)]; h_l = GELU(h_{l-1} W_l^T + b_l) for l = 1..3
(GELU(z) = z Phi(z), erf form); z = h_3 W_4^T + b_4.  Loss: mean over finite targets of
(z - (t - mean)/std)^2.  Parameters: one flat vector, per layer W [out][in] then b [out].
The forward pass may round the weights to BF16 (as the GPU's forward pass does); gradients are the
exact chain rule of that forward pass (weights held fixed at their rounded values).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def layer_dims(n, k, width):
    return [n + 1, width, width, width, n + k]


def unpack(params, dims):
    out, off = [], 0
    for l in range(len(dims) - 1):
        din, dout = dims[l], dims[l + 1]
        W = params[off:off + din * dout].reshape(dout, din)
        off += din * dout
        b = params[off:off + dout]
        off += dout
        out.append((W, b))
    assert off == params.size
    return out


def bf16(a):
    import torch
    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def features(y):
    y = np.asarray(y, np.float64)
    s = y.sum(axis=1, keepdims=True)
    n = y.shape[1]
    return np.concatenate([n * y / s, np.log(s)], axis=1)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward(params, dims, y, round_weights=True):
    layers = unpack(np.asarray(params, np.float64), dims)
    h = features(y)
    hs, pres = [h], []
    for l, (W, b) in enumerate(layers):
        Wf = bf16(W) if round_weights else W
        z = h @ Wf.T + b
        if l < len(layers) - 1:
            pres.append(z)
            h = gelu(z)
        else:
            h = z
        hs.append(h)
    return h, hs, pres


def loss_and_grad(params, dims, y, target, mean, std, round_weights=True):
    """Loss and d loss / d params (flat), by the chain rule."""
    params = np.asarray(params, np.float64)
    layers = unpack(params, dims)
    z, hs, pres = forward(params, dims, y, round_weights)
    t = np.asarray(target, np.float64)
    mask = np.isfinite(t)
    tn = np.where(mask, (np.where(mask, t, 0.0) - mean) / std, 0.0)
    r = np.where(mask, z - tn, 0.0)
    cnt = mask.sum()
    loss = float((r * r).sum() / cnt)
    d = 2.0 * r / cnt
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        W, b = layers[l]
        Wf = bf16(W) if round_weights else W
        dW = d.T @ hs[l]
        db = d.sum(axis=0)
        grads.append((dW, db))
        if l > 0:
            d = (d @ Wf) * gelu_grad(pres[l - 1])
    grads.reverse()
    flat = np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])
    return loss, flat


def grad_magnitudes(params, dims, y, target, mean, std, round_weights=True):
    """Per gradient entry, the sum of the absolute values of the terms the chain rule adds up:
    the same backward pass as `loss_and_grad` with every factor replaced by its absolute value
    (|d| @ |W|, |gelu'|, |d|^T @ |h|).  Floating-point evaluation of an entry errs by at most a
    multiple of this scale times the unit roundoff, so it is the natural per-entry tolerance scale
    for comparing a lower-precision gradient with this reference."""
    params = np.asarray(params, np.float64)
    layers = unpack(params, dims)
    z, hs, pres = forward(params, dims, y, round_weights)
    t = np.asarray(target, np.float64)
    mask = np.isfinite(t)
    tn = np.where(mask, (np.where(mask, t, 0.0) - mean) / std, 0.0)
    d = np.abs(np.where(mask, 2.0 * (z - tn), 0.0)) / mask.sum()
    mags = []
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        Wf = bf16(W) if round_weights else W
        mags.append(((d.T @ np.abs(hs[l])), d.sum(axis=0)))
        if l > 0:
            d = (d @ np.abs(Wf)) * np.abs(gelu_grad(pres[l - 1]))
    mags.reverse()
    return np.concatenate([np.concatenate([m.ravel(), mb]) for m, mb in mags])
