"""Structural-step surrogate on the coupled plate (3-D): the network is
trained on the GPU (the library's BF16 forward / backward / Adam kernels) on
pairs from coupled oracle runs of the small plate case at three Reynolds
numbers and initial deflections, then guesses the shell's step in a coupled
GPU run at a Reynolds number outside the training set.  The shell's residual
accepts a guess or Newton continues from it; the test measures the Newton
solves and the time per step against plain Newton and against the
constant-velocity predictor alone (a zero network), and checks the plate's
motion against the run without the surrogate."""
import json
import multiprocessing as mp
import time

import numpy as np
import pytest

from tests import plate_case

pytestmark = pytest.mark.gpu
TRAIN = ((60.0, 3e-2), (100.0, 1e-2), (200.0, 2e-2))
RE_TEST, PERTURB_TEST = 140.0, 2e-2
STEPS = 600


@pytest.fixture(scope="module")
def pairs():
    with mp.get_context("spawn").Pool(len(TRAIN)) as pool:
        out = pool.map(plate_case.oracle_pairs, [(re, p, STEPS) for re, p in TRAIN])
    X = np.concatenate([o[0] for o in out])
    Y = np.concatenate([o[1] for o in out])
    return X, Y


def run(steps, mlp=None, stats=None, chunk=50):
    import torch
    from paper_1710_02375_gb300 import lbm as abi
    from paper_1710_02375_gb300 import surrogate
    L, S = plate_case.gpu_run(RE_TEST, PERTURB_TEST)
    if mlp is not None:
        surrogate.attach(L, mlp, stats, accept_tol=1e-3)
    tips = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps // chunk):
        L.step(chunk)
        u, _, _, _ = S.state()
        tips.append(u[-1].copy())
    dt = time.perf_counter() - t0
    L.check()
    counts = abi.fsi_get_structure_stats(L.ctx)
    return np.array(tips), counts, 1e3 * dt / steps


def test_plate_surrogate_gain_over_newton(pairs):
    from paper_1710_02375_gb300 import surrogate
    from paper_1710_02375_gb300.lbm import Mlp
    from oracle import mlp_oracle as mo
    X, Y = pairs
    nf = Y.shape[1]
    assert nf == 6 * (9 * 5 - 5) and X.shape[1] == surrogate.shell_input_width(nf)
    stats = surrogate.normalisation(X, Y)
    dims = [X.shape[1], 256, 256, 256, nf]
    net = Mlp(dims, max_batch=256)
    net.set_params(mo.init_params(dims, 0))
    hist = surrogate.train(net, X, Y, stats, steps=8000, lr=1e-3, log_every=500)
    assert hist[-1][1] < 0.05 * hist[0][1], hist
    zero = Mlp(dims, max_batch=1)
    zero.set_params(np.zeros(zero.nparam, np.float32))
    zstats = [stats[0], stats[1], np.zeros_like(stats[2]), stats[3]]

    tip_n, c_n, ms_n = run(STEPS)
    tip_z, c_z, ms_z = run(STEPS, zero, zstats)
    tip_s, c_s, ms_s = run(STEPS, net, stats)
    amp = np.max(np.abs(tip_n[:, 2]))
    dev = np.max(np.abs(tip_s[:, 2] - tip_n[:, 2])) / amp
    dev_z = np.max(np.abs(tip_z[:, 2] - tip_n[:, 2])) / amp
    summary = dict(steps=STEPS, pairs=int(X.shape[0]), newton=dict(counts=c_n, ms_per_step=ms_n),
                   velocity_predictor=dict(counts=c_z, ms_per_step=ms_z, tip_dev=dev_z),
                   network=dict(counts=c_s, ms_per_step=ms_s, tip_dev=dev),
                   train_loss=[hist[0][1], hist[-1][1]], tip_amplitude=amp)
    print("PLATE_SURROGATE", json.dumps(summary))
    assert c_n[3] == STEPS and c_n[0] == 0 and c_n[1] == 0
    assert c_s[0] + c_s[1] == STEPS and c_z[0] + c_z[1] == STEPS
    # the trained network saves Newton solves against both baselines
    assert c_s[2] <= 0.8 * c_n[2], summary
    assert c_s[2] < c_z[2], summary
    # the plate's motion stays close to the Newton run's
    assert dev <= 5e-2, summary
