"""FP64 multilayer perceptron -- TEST INFRASTRUCTURE ONLY.

Plain numpy statement of the surrogate network the CUDA library trains:
fully connected layers, exact-erf GELU on hidden layers, linear output, loss
mean((Yhat - Y)^2), gradients by backpropagation.  Parameter vector layout:
for each layer W[n_out][n_in] then b[n_out] (the library's layout).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def unpack(params, dims):
    out, off = [], 0
    for l in range(len(dims) - 1):
        ni, no = dims[l], dims[l + 1]
        W = params[off:off + ni * no].reshape(no, ni)
        off += ni * no
        b = params[off:off + no]
        off += no
        out.append((W, b))
    return out


def forward(params, dims, X):
    """Returns (Yhat, list of pre-activations Z, list of activations A)."""
    layers = unpack(np.asarray(params, dtype=np.float64), dims)
    A = [np.asarray(X, dtype=np.float64)]
    Z = []
    for l, (W, b) in enumerate(layers):
        z = A[-1] @ W.T + b
        Z.append(z)
        A.append(gelu(z) if l < len(layers) - 1 else z)
    return A[-1], Z, A


def loss(params, dims, X, Y):
    Yhat, _, _ = forward(params, dims, X)
    return float(np.mean((Yhat - Y) ** 2))


def gradients(params, dims, X, Y):
    """Gradient of mean((Yhat - Y)^2) by backpropagation (FP64)."""
    layers = unpack(np.asarray(params, dtype=np.float64), dims)
    Yhat, Z, A = forward(params, dims, X)
    B, nout = Yhat.shape
    dz = 2.0 * (Yhat - Y) / (B * nout)
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        dW = dz.T @ A[l]
        db = dz.sum(axis=0)
        grads.append((dW, db))
        if l > 0:
            dz = (dz @ W) * gelu_grad(Z[l - 1])
    grads.reverse()
    return np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])


def init_params(dims, seed):
    """Seeded Xavier-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for l in range(len(dims) - 1):
        ni, no = dims[l], dims[l + 1]
        lim = np.sqrt(6.0 / (ni + no))
        parts.append(rng.uniform(-lim, lim, size=no * ni))
        parts.append(np.zeros(no))
    return np.concatenate(parts)
