"""FP64 reference of the surrogate multilayer perceptron (numpy).

TEST INFRASTRUCTURE ONLY (part of the oracle).  The surrogate is a workload
pattern around the paper's method, not a part of the paper: an MLP maps
(log10 q, t) to the lattice observables.  This module is its plain definition:

    H_0 = X,  Z_l = H_l W_l^T + b_l,  H_{l+1} = GELU(Z_l)  (hidden layers),
    Y = Z_L (last layer linear),  loss = mean over samples and outputs of (Y - T)^2,
    GELU(x) = x/2 (1 + erf(x/sqrt(2))),
    GELU'(x) = (1 + erf(x/sqrt(2)))/2 + x exp(-x^2/2)/sqrt(2 pi),

with the gradient of the loss by the chain rule (reverse mode), written out
layer by layer.  Pinned by tests/test_oracle_mlp.py against central finite
differences of the loss and against closed forms.
"""
import numpy as np
from scipy.special import erf


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_prime(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def init_params(dims, seed):
    """Weights N(0, 1/fan_in), zero biases; dims = [n_in, width, ..., n_out]."""
    r = np.random.default_rng(seed)
    Ws, bs = [], []
    for i in range(len(dims) - 1):
        Ws.append(r.standard_normal((dims[i + 1], dims[i])) / np.sqrt(dims[i]))
        bs.append(np.zeros(dims[i + 1]))
    return Ws, bs


def forward(Ws, bs, X):
    """Returns (Y, cache) for X of shape (B, n_in)."""
    H = [np.asarray(X, dtype=np.float64)]
    Z = []
    L = len(Ws)
    for l in range(L):
        z = H[-1] @ Ws[l].T + bs[l]
        Z.append(z)
        if l < L - 1:
            H.append(gelu(z))
    return Z[-1], (H, Z)


def loss(Ws, bs, X, T):
    Y, _ = forward(Ws, bs, X)
    return float(np.mean((Y - T) ** 2))


def loss_and_grad(Ws, bs, X, T):
    """Mean squared error and its gradient with respect to every W_l, b_l."""
    Y, (H, Z) = forward(Ws, bs, X)
    B, n_out = Y.shape
    Lval = float(np.mean((Y - T) ** 2))
    dZ = 2.0 * (Y - T) / (B * n_out)
    gW, gb = [None] * len(Ws), [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        gW[l] = dZ.T @ H[l]
        gb[l] = dZ.sum(axis=0)
        if l > 0:
            dH = dZ @ Ws[l]
            dZ = dH * gelu_prime(Z[l - 1])
    return Lval, gW, gb


def flatten(Ws, bs):
    """Parameter vector in the library's order: W_0, b_0, W_1, b_1, ..."""
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in zip(Ws, bs)])


def unflatten(theta, dims):
    Ws, bs, o = [], [], 0
    for i in range(len(dims) - 1):
        n = dims[i + 1] * dims[i]
        Ws.append(theta[o:o + n].reshape(dims[i + 1], dims[i]))
        o += n
        bs.append(theta[o:o + dims[i + 1]].copy())
        o += dims[i + 1]
    return Ws, bs
