"""Structural-step surrogate on the C1 flag: the network is trained on the
GPU (the library's BF16 forward / backward / Adam kernels) on pairs from
coupled oracle runs at Re = 100, 150 and 300, then guesses the structural
step of a coupled GPU run at Re = 200 (not in the training set).  The FEM
residual accepts a guess or Newton continues from it; the test measures what
the trained network gains over plain Newton (Newton solves per step, time per
step) and over the constant-velocity predictor alone (a zero network), and
checks the flag's motion against the run without the surrogate."""
import json
import multiprocessing as mp
import time

import numpy as np
import pytest

from tests import c1_flag_case as c1

pytestmark = pytest.mark.gpu
RE_TRAIN = (100.0, 150.0, 300.0)
RE_TEST = 200.0
STEPS = 2500


@pytest.fixture(scope="module")
def pairs():
    with mp.get_context("spawn").Pool(len(RE_TRAIN)) as pool:
        out = pool.map(c1.oracle_pairs, [(re, k + 1, STEPS) for k, re in enumerate(RE_TRAIN)])
    X = np.concatenate([o[0] for o in out])
    Y = np.concatenate([o[1] for o in out])
    return X, Y


def run(steps, mlp=None, stats=None, chunk=50, make=None):
    import torch
    from paper_1710_02375_gb300 import lbm as abi
    from paper_1710_02375_gb300 import surrogate
    L, gb = make() if make else c1.gpu_run(RE_TEST)
    if mlp is not None:
        surrogate.attach(L, mlp, stats, accept_tol=1e-3)
    tips = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps // chunk):
        L.step(chunk)
        u, _, _ = gb.state()
        tips.append(u[-3:].copy())
    dt = time.perf_counter() - t0
    L.check()
    counts = abi.fsi_get_structure_stats(L.ctx)
    return np.array(tips), counts, 1e3 * dt / steps


def test_surrogate_gain_over_newton(pairs):
    from paper_1710_02375_gb300 import surrogate
    from paper_1710_02375_gb300.lbm import Mlp
    from oracle import mlp_oracle as mo
    X, Y = pairs
    nn = 21
    assert X.shape[1] == surrogate.input_width(nn) and Y.shape[1] == 3 * nn - 3
    stats = surrogate.normalisation(X, Y)
    dims = [X.shape[1], 128, 128, 128, Y.shape[1]]
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
    amp = np.max(np.abs(tip_n[:, :2]))
    dev = np.max(np.abs(tip_s[:, :2] - tip_n[:, :2])) / amp
    dev_z = np.max(np.abs(tip_z[:, :2] - tip_n[:, :2])) / amp
    summary = dict(steps=STEPS, newton=dict(counts=c_n, ms_per_step=ms_n),
                   velocity_predictor=dict(counts=c_z, ms_per_step=ms_z, tip_dev=dev_z),
                   network=dict(counts=c_s, ms_per_step=ms_s, tip_dev=dev),
                   train_loss=[hist[0][1], hist[-1][1]], tip_amplitude=amp)
    print("SURROGATE", json.dumps(summary))
    # every structural step ran; plain Newton never sees a guess
    assert c_n[3] == STEPS and c_n[0] == 0 and c_n[1] == 0
    assert c_s[0] + c_s[1] == STEPS and c_z[0] + c_z[1] == STEPS
    # the trained network saves Newton solves against both baselines
    assert c_s[2] <= 0.8 * c_n[2], summary
    assert c_s[2] < c_z[2], summary
    assert c_s[0] > 0, summary
    # accepted guesses leave the flag's motion close to the Newton run's
    assert dev <= 5e-2, summary


@pytest.mark.slow
def test_surrogate_c5_scale():
    """The surrogate workload's size: 800 x 160 channel, D = 39, a 32-node
    flag (465 network inputs, 93 outputs).  Training pairs: 1500 steps of
    coupled oracle runs at Re = 100, 150, 250 and 300 (6000 pairs, the
    start-up through the 1000-step inflow ramp); deployment: a coupled GPU run
    at Re = 200 over the same 1500 steps.  Checks the gain in Newton solves
    and the flag motion against the Newton-only run, and reports time per
    step."""
    from paper_1710_02375_gb300 import surrogate, synth
    from paper_1710_02375_gb300.cases import flag_coupled
    from paper_1710_02375_gb300.lbm import Mlp
    from oracle import mlp_oracle as mo
    steps, res = 1500, (100.0, 150.0, 250.0, 300.0)
    with mp.get_context("spawn").Pool(len(res)) as pool:
        out = pool.map(c1.c5_pairs, [(re, k + 1, steps) for k, re in enumerate(res)])
    X = np.concatenate([o[0] for o in out])
    Y = np.concatenate([o[1] for o in out])
    nn = 32
    assert X.shape[1] == surrogate.input_width(nn) and Y.shape[1] == 3 * nn - 3
    stats = surrogate.normalisation(X, Y)
    dims = [X.shape[1], 128, 128, 128, Y.shape[1]]
    net = Mlp(dims, max_batch=256)
    net.set_params(mo.init_params(dims, 0))
    hist = surrogate.train(net, X, Y, stats, steps=8000, lr=1e-3, log_every=500)
    make = lambda: flag_coupled(synth.c5_case(RE_TEST))  # noqa: E731
    tip_n, c_n, ms_n = run(steps, make=make)
    tip_s, c_s, ms_s = run(steps, net, stats, make=make)
    amp = np.max(np.abs(tip_n[:, :2]))
    dev = np.max(np.abs(tip_s[:, :2] - tip_n[:, :2])) / amp
    summary = dict(steps=steps, pairs=int(X.shape[0]), newton=dict(counts=c_n, ms_per_step=ms_n),
                   network=dict(counts=c_s, ms_per_step=ms_s, tip_dev=dev),
                   train_loss=[hist[0][1], hist[-1][1]], tip_amplitude=amp)
    print("SURROGATE_C5", json.dumps(summary))
    assert c_n[3] == steps and c_s[0] + c_s[1] == steps
    assert c_s[2] <= 0.85 * c_n[2], summary
    assert dev <= 5e-2, summary
