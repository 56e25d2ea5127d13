"""Training pairs for the structural-step surrogate -- TEST INFRASTRUCTURE ONLY.

The pairs come from coupled runs of the oracle (fsi_oracle.CSSFlag: FP64
KBC fluid, Grad boundaries, momentum-exchange forces, co-rotational beam with
the theta-scheme and Newton, section "Fluid-structure coupling"); each
structural step of such a run gives one pair:
  input  = [F(t) - f(u), F(t-1) - f(u), F(t-2) - f(u), u, v]
           each block on the 3 nn - 3 free DOFs (nodes 1..nn-1, (ux, uy,
           theta) per node): F the nodal loads of the step (the sums of each
           node's two surface-vertex forces, zero moment; zero before the
           run starts), f the internal force at the state u before the step,
           u and v that state                       (15 nn - 15 values)
  target = u(t+1) - u(t) - dt v(t) on the free DOFs (3 nn - 3 values): the
           step's displacement beyond the constant-velocity predictor.
The out-of-balance form F - f(u) keeps the map from input to target close
to linear and well conditioned: the increment follows from the balance of
inertia against F - f, whose parts F and f nearly cancel in a slowly moving
flag.
"""
from __future__ import annotations

import numpy as np

from . import oracle as orc
from .fsi_oracle import nodal_loads


def features(beam: "orc.Beam", Fh, t, u, v):
    """Network input of step t; Fh[T, nn, 2] nodal loads (Fx, Fy) per step."""
    nn = beam.nn
    f, _ = beam.internal(u, want_K=False)
    parts = []
    for k in range(3):
        F = np.zeros((nn, 3))
        if t - k >= 0:
            F[:, :2] = Fh[t - k]
        parts.append(F.ravel()[3:] - f[3:])
    return np.concatenate(parts + [u[3:], v[3:]])


def pairs_from_run(css, steps: int, dt: float = 1.0):
    """Advance the coupled oracle run `css` (a CSSFlag) by `steps` steps and
    return (X[steps, 15 nn - 15], Y[steps, 3 nn - 3]) of its structural
    steps, plus the tip displacement history [steps, 3]."""
    beam = css.beam
    nn = beam.nn
    nr = css.x_rigid.shape[0]
    Fh = np.zeros((steps, nn, 2))
    X, Y, tip = [], [], []
    for t in range(steps):
        u0, v0 = css.u.copy(), css.v.copy()
        css.step()
        F = nodal_loads(beam.X, u0, None, css.vforce[nr:])
        Fh[t] = F.reshape(nn, 3)[:, :2]
        X.append(features(beam, Fh, t, u0, v0))
        Y.append(css.u[3:] - u0[3:] - dt * v0[3:])
        tip.append(css.u[-3:].copy())
    return np.array(X), np.array(Y), np.array(tip)
