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


def _rotvec(R):
    """Rotation vectors of rotation matrices R[..., 3, 3] (angles below pi)."""
    c = np.clip(0.5 * (np.trace(R, axis1=-2, axis2=-1) - 1.0), -1.0, 1.0)
    t = np.arccos(c)
    w = np.stack([R[..., 2, 1] - R[..., 1, 2], R[..., 0, 2] - R[..., 2, 0], R[..., 1, 0] - R[..., 0, 1]], -1)
    s = np.sin(t)
    g = np.where(t < 1e-6, 0.5 + t * t / 12.0, 0.5 * t / np.where(s == 0, 1.0, s))
    return g[..., None] * w


def shell_features(shell: "orc.Shell", Fh, t, u, R, v):
    """Network input of plate step t: the out-of-balance loads F(t-k) - f(u, R)
    for k = 0, 1, 2 (F: nodal loads [T, nn, 6], zero before the run starts;
    f: internal force at the state before the step), then the state
    (translations and rotation vectors) and the velocities (translational and
    angular); every block on the free DOFs (6 per node not held)."""
    free = shell.fixed == 0
    f = shell.internal(u, R).ravel()
    parts = []
    for k in range(3):
        F = Fh[t - k].ravel() if t - k >= 0 else np.zeros(6 * shell.nn)
        parts.append((F - f)[free])
    q = np.concatenate([u, _rotvec(R)], axis=1).ravel()
    parts += [q[free], v.ravel()[free]]
    return np.concatenate(parts)


def pairs_from_plate_run(css, steps: int, dt: float = 1.0, **shell_kw):
    """Advance the coupled oracle plate run `css` (a CSSPlate) by `steps`
    steps; returns (X[steps, 5 nf], Y[steps, nf]) with nf the free DOFs and
    the target the step's increment (translations; rotation vector of
    R1 R0^T) beyond dt times the velocity at the step's start."""
    shell = css.shell
    nn = shell.nn
    free = shell.fixed == 0
    Fh = np.zeros((steps, nn, 6))
    X, Y = [], []
    for t in range(steps):
        u0, R0, v0 = css.u.copy(), css.R.copy(), css.v.copy()
        css.step(**shell_kw)
        Fh[t, :, :3] = css.vforce[:nn] + css.vforce[nn:]
        X.append(shell_features(shell, Fh, t, u0, R0, v0))
        dphi = _rotvec(np.einsum("nij,nkj->nik", css.R, R0))
        inc = np.concatenate([css.u - u0, dphi], axis=1).ravel() - dt * v0.ravel()
        Y.append(inc[free])
    return np.array(X), np.array(Y)
