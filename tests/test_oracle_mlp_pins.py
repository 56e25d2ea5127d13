"""Pins of the FP64 MLP oracle: backpropagation against central finite
differences, GELU against its closed-form values."""
import numpy as np

from oracle import mlp_oracle as mo


def test_gelu_values():
    assert mo.gelu(np.array([0.0]))[0] == 0.0
    # GELU(x) - GELU(-x) = x and GELU'(0) = 1/2
    x = np.linspace(-3, 3, 13)
    assert np.allclose(mo.gelu(x) - mo.gelu(-x), x, atol=1e-15)
    assert abs(mo.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15
    h = 1e-6
    assert np.allclose((mo.gelu(x + h) - mo.gelu(x - h)) / (2 * h), mo.gelu_grad(x), atol=1e-9)


def test_backprop_matches_finite_differences():
    dims = [7, 9, 6, 5]
    rng = np.random.default_rng(0)
    p = mo.init_params(dims, 1) + 0.1 * rng.standard_normal(sum(
        dims[l] * dims[l + 1] + dims[l + 1] for l in range(len(dims) - 1)))
    X = rng.standard_normal((11, dims[0]))
    Y = rng.standard_normal((11, dims[-1]))
    g = mo.gradients(p, dims, X, Y)
    h = 1e-6
    fd = np.zeros_like(p)
    for k in range(len(p)):
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd[k] = (mo.loss(pp, dims, X, Y) - mo.loss(pm, dims, X, Y)) / (2 * h)
    assert np.max(np.abs(g - fd)) <= 1e-6 * np.max(np.abs(fd))
