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


def test_gradient_magnitudes_bound_the_gradient():
    """grad_magnitudes sums |terms| of the same chain rule, so it bounds |gradient| entry by entry
    (triangle inequality) and equals it when every factor is non-negative (here: positive weights,
    positive residuals, no GELU layers in play: a one-layer check through the output layer)."""
    rng = np.random.default_rng(3)
    n, k, H, B = 6, 2, 5, 4
    dims = mlp.layer_dims(n, k, H)
    P = sum(dims[l] * dims[l + 1] + dims[l + 1] for l in range(4))
    params = rng.normal(0, 0.4, P)
    y = rng.uniform(0.01, 1.0, (B, n))
    t = rng.normal(0, 1, (B, n + k))
    t[1, 2] = -np.inf
    mean, std = np.zeros(n + k), np.ones(n + k)
    _, g = mlp.loss_and_grad(params, dims, y, t, mean, std, round_weights=False)
    M = mlp.grad_magnitudes(params, dims, y, t, mean, std, round_weights=False)
    assert np.all(np.abs(g) <= M * (1 + 1e-12) + 1e-300)
    # output-layer bias gradient: sum_b 2 r_bj / cnt; with every residual of a column of one sign
    # the magnitude equals |gradient|
    z, _, _ = mlp.forward(params, dims, y, round_weights=False)
    t2 = z - 1.0  # residual z - t = +1 everywhere
    _, g2 = mlp.loss_and_grad(params, dims, y, t2, mean, std, round_weights=False)
    M2 = mlp.grad_magnitudes(params, dims, y, t2, mean, std, round_weights=False)
    nb = dims[4]
    np.testing.assert_allclose(g2[-nb:], M2[-nb:], rtol=1e-12)
