"""Pins of the FP64 warm-start network reference: the hand-written backward pass against central
finite differences of the loss (weights not rounded, so the loss is smooth), and GELU against its
definition z Phi(z)."""
import numpy as np
from scipy.stats import norm

from oracle import mlp


def test_gelu_is_z_times_normal_cdf_and_its_derivative():
    z = np.linspace(-6, 6, 101)
    np.testing.assert_allclose(mlp.gelu(z), z * norm.cdf(z), rtol=1e-12, atol=1e-15)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), rtol=1e-7, atol=1e-9)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    n, k, H, B = 6, 2, 5, 4
    dims = mlp.layer_dims(n, k, H)
    P = sum(dims[l] * dims[l + 1] + dims[l + 1] for l in range(4))
    params = rng.normal(0, 0.4, P)
    y = rng.uniform(0.01, 1.0, (B, n))
    t = rng.normal(0, 1, (B, n + k))
    t[0, 1] = -np.inf  # a masked target
    mean = rng.normal(0, 0.1, n + k)
    std = rng.uniform(0.5, 2.0, n + k)
    loss, g = mlp.loss_and_grad(params, dims, y, t, mean, std, round_weights=False)
    fd = np.empty(P)
    h = 1e-6
    for i in range(P):
        e = np.zeros(P)
        e[i] = h
        fd[i] = (mlp.loss_and_grad(params + e, dims, y, t, mean, std, False)[0]
                 - mlp.loss_and_grad(params - e, dims, y, t, mean, std, False)[0]) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)
    assert loss > 0
