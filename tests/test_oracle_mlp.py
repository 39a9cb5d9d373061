"""Pins of the FP64 surrogate MLP reference: GELU against its closed-form
values and derivative, the analytic gradient against central finite
differences of the loss, and a linear network against ordinary least squares
geometry (gradient zero at the least-squares solution)."""
import numpy as np
from scipy.stats import norm

from oracle import mlp


def test_gelu_closed_form_and_derivative():
    x = np.linspace(-6, 6, 121)
    assert np.allclose(mlp.gelu(x), x * norm.cdf(x), rtol=1e-14, atol=1e-15)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.allclose(mlp.gelu_prime(x), fd, atol=1e-8)
    assert mlp.gelu(0.0) == 0.0 and abs(mlp.gelu_prime(0.0) - 0.5) < 1e-15


def test_gradient_matches_central_differences():
    dims = [2, 7, 5, 3]
    Ws, bs = mlp.init_params(dims, seed=3)
    r = np.random.default_rng(4)
    for l in range(len(bs)):
        bs[l] = 0.1 * r.standard_normal(bs[l].shape)
    X = r.standard_normal((11, 2))
    T = r.standard_normal((11, 3))
    L0, gW, gb = mlp.loss_and_grad(Ws, bs, X, T)
    theta = mlp.flatten(Ws, bs)
    g = mlp.flatten(gW, gb)
    h = 1e-6
    for i in r.choice(theta.size, 40, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss(*mlp.unflatten(tp, dims), X, T) - mlp.loss(*mlp.unflatten(tm, dims), X, T)) / (2 * h)
        assert abs(fd - g[i]) < 1e-7 * (1 + abs(fd)), (i, fd, g[i])


def test_linear_network_gradient_vanishes_at_least_squares():
    """One linear layer: the MSE gradient is zero at the least-squares fit."""
    r = np.random.default_rng(5)
    X = r.standard_normal((50, 3))
    T = r.standard_normal((50, 2))
    A = np.hstack([X, np.ones((50, 1))])
    sol, *_ = np.linalg.lstsq(A, T, rcond=None)
    W, b = sol[:3].T, sol[3]
    L, gW, gb = mlp.loss_and_grad([W], [b], X, T)
    assert np.max(np.abs(gW[0])) < 1e-13 and np.max(np.abs(gb[0])) < 1e-13
