"""Training of the structural-step surrogate network and its attachment to
a coupled lattice (argument marshalling and batching only: every forward,
backward and Adam step runs in the library's MLP kernels, and the coupled
step builds the network input, runs the network and checks its guess on the
GPU)."""
from __future__ import annotations

import math

import numpy as np

from . import lbm as abi


def input_width(nn):
    """Network inputs for an nn-node beam: three out-of-balance load vectors,
    u and v, each on the 3 nn - 3 free DOFs."""
    return 15 * nn - 15


def shell_input_width(nfree):
    """Network inputs for a shell with nfree free DOFs: three out-of-balance
    load vectors, the state and the velocities, each on the free DOFs."""
    return 5 * nfree


def normalisation(X, Y, floor=1e-30):
    """Per-feature mean and standard deviation (FP32) of inputs and targets;
    constant features get a unit scale."""
    xm, xs = X.mean(axis=0), X.std(axis=0)
    ym, ys = Y.mean(axis=0), Y.std(axis=0)
    xs = np.where(xs > floor, xs, 1.0)
    ys = np.where(ys > floor, ys, 1.0)
    return [np.ascontiguousarray(a, dtype=np.float32) for a in (xm, xs, ym, ys)]


def train(mlp, X, Y, stats, steps=8000, batch=256, lr=1e-3, seed=0, log_every=0):
    """Adam with a cosine learning-rate decay on normalised (X, Y) held on
    the device; returns [(step, batch loss)] every log_every steps."""
    import torch
    xm, xs, ym, ys = stats
    dev = torch.device("cuda")
    Xn = torch.from_numpy(((X - xm) / xs).astype(np.float32)).to(dev)
    Yn = torch.from_numpy(((Y - ym) / ys).astype(np.float32)).to(dev)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    hist = []
    for it in range(steps):
        mlp.set_learning_rate(lr * 0.5 * (1.0 + math.cos(math.pi * it / steps)) + 1e-7)
        idx = torch.randint(0, Xn.shape[0], (batch,), device=dev, generator=g)
        xb, yb = Xn[idx].contiguous(), Yn[idx].contiguous()
        torch.cuda.current_stream().synchronize()  # batch ready before the library stream reads it
        want = bool(log_every) and it % log_every == 0
        loss = mlp.train_step(xb, yb, want_loss=want)
        if want:
            hist.append((it, loss))
        if it % 64 == 63:
            mlp.stream.synchronize()  # bounds the batches held alive by the caching allocator
    mlp.stream.synchronize()
    return hist


def attach(lattice, mlp, stats, accept_tol=1e-3):
    """Use the network as the Newton initial guess of the coupled beam or
    shell."""
    xm, xs, ym, ys = stats
    abi.fsi_set_surrogate(lattice.ctx, mlp.ctx, xm, xs, ym, ys, accept_tol)


def detach(lattice):
    abi.fsi_set_surrogate(lattice.ctx, None, None, None, None, None, 1.0)
