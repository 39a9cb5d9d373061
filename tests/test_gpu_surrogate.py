"""Surrogate MLP on BF16 tensor cores against the FP64 reference (oracle/mlp.py).

Two bars per quantity.  (1) Against the reference evaluated with the operands
of every GEMM rounded to BF16 the way the kernels round them (round to nearest
even), the only remaining difference is FP32 accumulation order, so the match
is tight.  (2) Against the plain FP64 reference the difference is the BF16
operand rounding itself: unit roundoff u = 2^-9 on each of the two operands of
every product, about sqrt(2) u ~ 3e-3 relative per layer, growing over the
four layers to below 1e-2 in the Frobenius norm."""
import numpy as np
import pytest

import paper_2006_15122_gb300 as cl
from oracle import mlp

pytestmark = pytest.mark.gpu

DIMS = [2, 256, 256, 256, 34]


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def forward_bf16(Ws, bs, X):
    """The reference forward pass with BF16 GEMM operands (FP32 epilogue values)."""
    H = [bf16(X)]
    Z = []
    for l in range(len(Ws)):
        z = f32(H[-1] @ bf16(Ws[l]).T + bs[l])
        Z.append(z)
        if l < len(Ws) - 1:
            H.append(bf16(mlp.gelu(z)))
    return Z[-1], (H, Z)


def grad_bf16(Ws, bs, X, T):
    Y, (H, Z) = forward_bf16(Ws, bs, X)
    n, m = Y.shape
    dZ = f32(2.0 * (Y - T) / (n * m))
    gW, gb = [None] * len(Ws), [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        gW[l] = bf16(dZ).T @ H[l]
        gb[l] = dZ.sum(axis=0)
        if l > 0:
            dH = f32(bf16(dZ) @ bf16(Ws[l]))
            dZ = f32(dH * mlp.gelu_prime(Z[l - 1]))
    return gW, gb


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def data(n, seed):
    r = np.random.default_rng(seed)
    X = np.stack([r.uniform(1.0, 4.0, n), r.uniform(0.0, 2.0, n)], axis=1)
    T = r.standard_normal((n, DIMS[-1]))
    return X, T


def make_net(seed=7):
    net = cl.Surrogate(DIMS[0], DIMS[-1], DIMS[1], len(DIMS) - 2, seed=seed)
    Ws, bs = mlp.init_params(DIMS, seed=seed)
    r = np.random.default_rng(seed + 1)
    bs = [0.1 * r.standard_normal(b.shape) for b in bs]
    theta = f32(mlp.flatten(Ws, bs))
    net.set_params(theta)
    return net, mlp.unflatten(theta, DIMS)


def test_param_layout_roundtrip():
    net = cl.Surrogate(2, 34, 256, 3, seed=1)
    assert net.param_count() == sum(DIMS[i + 1] * DIMS[i] + DIMS[i + 1] for i in range(4))
    theta0 = net.get_params()
    Ws, bs = mlp.unflatten(theta0, DIMS)
    # Philox N(0, 1/fan_in) weights: sample moments of each layer, zero biases
    for l, W in enumerate(Ws):
        assert abs(W.mean()) < 4.0 / np.sqrt(W.size * DIMS[l])
        assert abs(W.var() * DIMS[l] - 1.0) < 4.0 * np.sqrt(2.0 / W.size)
        assert not np.any(bs[l])
    t = f32(np.random.default_rng(2).standard_normal(theta0.size))
    net.set_params(t)
    assert np.array_equal(net.get_params(), t)
    net.close()


@pytest.mark.parametrize("n", [1, 37, 64, 300, 1000])
def test_forward_matches_reference(n):
    net, (Ws, bs) = make_net()
    X, _ = data(n, n)
    Y = net.predict(X).astype(np.float64)
    Ye, _ = forward_bf16(Ws, bs, X)
    assert rel_fro(Y, Ye) < 2e-4, rel_fro(Y, Ye)
    Y64, _ = mlp.forward(Ws, bs, X)
    assert rel_fro(Y, Y64) < 1e-2, rel_fro(Y, Y64)
    net.close()


@pytest.mark.parametrize("n", [64, 200])
def test_gradient_matches_reference(n):
    net, (Ws, bs) = make_net(seed=11)
    X, T = data(n, 100 + n)
    loss, g = net.loss_grad(X, T)
    L64, gW64, gb64 = mlp.loss_and_grad(Ws, bs, X, T)
    assert abs(loss - L64) < 1e-2 * L64
    gWe, gbe = grad_bf16(Ws, bs, X, T)
    ge, g64 = mlp.flatten(gWe, gbe), mlp.flatten(gW64, gb64)
    assert rel_fro(g, ge) < 2e-3, rel_fro(g, ge)
    assert float(g @ g64 / (np.linalg.norm(g) * np.linalg.norm(g64))) > 0.999
    # per layer as well: no block may hide behind the others
    Wg, bg = mlp.unflatten(g, DIMS)
    for l in range(4):
        assert rel_fro(Wg[l], gWe[l]) < 5e-3, (l, rel_fro(Wg[l], gWe[l]))
        assert rel_fro(bg[l], gbe[l]) < 5e-3, (l, rel_fro(bg[l], gbe[l]))
    net.close()


def test_first_adam_step_is_sign_of_gradient():
    """With zero moments the first Adam update of every parameter is
    -lr g/(|g| + eps): -lr sign(g) wherever |g| >> eps."""
    net, (Ws, bs) = make_net(seed=5)
    X, T = data(128, 9)
    theta0 = net.get_params()
    gWe, gbe = grad_bf16(Ws, bs, X, T)
    ge = mlp.flatten(gWe, gbe)
    lr = 1e-3
    net.train(X, T, epochs=1, batch=128, lr=lr, eps=1e-12, standardize=False)
    step = net.get_params() - theta0
    big = np.abs(ge) > 1e-2 * np.sqrt(np.mean(ge ** 2))
    assert big.mean() > 0.5
    assert np.mean(np.sign(step[big]) == -np.sign(ge[big])) > 0.995
    assert np.allclose(np.abs(step[big]), lr, rtol=1e-3, atol=2e-7)
    net.close()


def test_training_fits_a_smooth_map_and_predict_undoes_standardization():
    r = np.random.default_rng(3)
    n = 4096
    X = np.stack([r.uniform(1.0, 4.0, n), r.uniform(0.0, 200.0, n)], axis=1)
    A = r.standard_normal((2, 34))
    c = r.uniform(10.0, 100.0, 34)
    Y = c * np.tanh(np.array([[1.0, 0.01]]) * X @ A) + 5.0 * c
    net = cl.Surrogate(2, 34, 256, 3, seed=4)
    hist = net.train(X[:3584], Y[:3584], epochs=100, batch=256, lr=2e-3)
    assert np.all(np.isfinite(hist)) and hist[-1] < 1e-2 * hist[0], hist[[0, -1]]
    P = net.predict(X[3584:]).astype(np.float64)
    err = np.sqrt(np.mean((P - Y[3584:]) ** 2, axis=0)) / Y[:3584].std(axis=0)
    assert np.max(err) < 0.1, err
    # predict == destandardize(reference forward of the standardized inputs)
    mu, sd = X[:3584].mean(0), X[:3584].std(0)
    muy, sdy = Y[:3584].mean(0), Y[:3584].std(0)
    Ws, bs = mlp.unflatten(net.get_params(), DIMS)
    Ye, _ = forward_bf16(Ws, bs, (X[3584:] - mu) / sd)
    assert rel_fro((P - muy) / sdy, Ye) < 1e-3, rel_fro((P - muy) / sdy, Ye)
    net.close()


def test_one_epoch_launch_equals_one_minibatch_per_call():
    """The fused epoch walks its minibatches in order inside one launch: its
    result equals, bit for bit, that of one call per minibatch (same rows, same
    Adam step count, constant step size), a ragged last minibatch included; and
    training is deterministic."""
    X, T = data(300, 21)
    nets = [make_net(seed=8)[0] for _ in range(3)]
    kw = dict(batch=128, lr=1e-3, standardize=False)
    nets[0].train(X, T, epochs=1, **kw)
    nets[1].train(X, T, epochs=1, **kw)
    for lo, hi in ((0, 128), (128, 256), (256, 300)):
        nets[2].train(X[lo:hi], T[lo:hi], epochs=1, **kw)
    p = [net.get_params() for net in nets]
    assert np.array_equal(p[0], p[1])
    assert np.array_equal(p[0], p[2]), np.max(np.abs(p[0] - p[2]))
    for net in nets:
        net.close()
