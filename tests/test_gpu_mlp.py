"""GPU MLP (BF16 tensor-core GEMMs with FP32 accumulation) against the FP64
numpy oracle: forward values, backpropagated gradients (BF16 bound 2e-2
relative to the largest gradient entry of each layer), and training."""
import numpy as np
import pytest

from oracle import mlp_oracle as mo

pytestmark = pytest.mark.gpu
DIMS = [96, 128, 128, 128, 40]


def test_forward_and_gradients_match_oracle():
    from paper_1710_02375_gb300.lbm import Mlp
    rng = np.random.default_rng(0)
    p = mo.init_params(DIMS, 3)
    X = rng.standard_normal((77, DIMS[0]))
    Y = rng.standard_normal((77, DIMS[-1]))
    m = Mlp(DIMS, max_batch=128)
    m.set_params(p)
    yg = m.forward(X)
    yo, _, _ = mo.forward(p, DIMS, X)
    assert np.max(np.abs(yg - yo)) <= 2e-2 * np.max(np.abs(yo))
    g, loss = m.gradients(X, Y)
    go = mo.gradients(p, DIMS, X, Y)
    assert abs(loss - mo.loss(p, DIMS, X, Y)) <= 2e-2 * mo.loss(p, DIMS, X, Y)
    off = 0
    for l in range(len(DIMS) - 1):
        n = DIMS[l] * DIMS[l + 1] + DIMS[l + 1]
        gl, ol = g[off:off + n], go[off:off + n]
        assert np.max(np.abs(gl - ol)) <= 2e-2 * np.max(np.abs(ol)), l
        off += n


def test_training_fits_a_smooth_map():
    from paper_1710_02375_gb300.lbm import Mlp
    rng = np.random.default_rng(1)
    A = rng.standard_normal((DIMS[0], DIMS[-1])) / np.sqrt(DIMS[0])
    X = rng.standard_normal((4096, DIMS[0])).astype(np.float32)
    Y = (np.tanh(X @ A) + 0.1 * (X @ A) ** 2).astype(np.float32)
    m = Mlp(DIMS, max_batch=256, lr=2e-3)
    m.set_params(mo.init_params(DIMS, 5))
    first = None
    for it in range(1500):
        idx = rng.integers(0, len(X), 256)
        l = m.train_step(X[idx], Y[idx], want_loss=(it % 100 == 0))
        if l is not None and first is None:
            first = l
    pred = m.forward(X[:256])
    final = float(np.mean((pred - Y[:256]) ** 2))
    assert final < 0.05 * first, (first, final)


@pytest.mark.parametrize("dims", [[465, 128, 128, 128, 93], [1200, 256, 256, 256, 240], [7, 33, 5]])
def test_single_launch_inference_equals_layer_by_layer(dims):
    """Batches of 1..16 rows go through the one-launch inference kernel, larger
    ones layer by layer; the rows of a small batch come out bit for bit as
    they do inside a large batch, and both agree with the FP64 oracle within
    the BF16 bound."""
    from paper_1710_02375_gb300.lbm import Mlp
    rng = np.random.default_rng(1)
    p = mo.init_params(dims, 5)
    X = rng.standard_normal((40, dims[0]))
    m = Mlp(dims, max_batch=64)
    m.set_params(p)
    big = m.forward(X)
    for B in (1, 3, 16):
        small = m.forward(X[:B])
        assert np.array_equal(small, big[:B]), B
    yo, _, _ = mo.forward(p, dims, X)
    assert np.max(np.abs(big - yo)) <= 2e-2 * np.max(np.abs(yo))
