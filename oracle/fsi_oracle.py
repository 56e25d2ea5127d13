"""Conventional serial staggered (CSS) coupling of the KBC fluid and the beam
-- TEST INFRASTRUCTURE ONLY (section "Fluid-structure coupling": fluid step
with boundary conditions, traction on the solid, structural step, transfer of
velocity and displacement, geometry update).

Readings shared with the CUDA library:
  * the flag is a closed polygon around the beam centre line: bottom edge
    vertex j = x_j + (h/2)(sin th_j, -cos th_j), top edge (stored in reverse
    node order) x_j + (h/2)(-sin th_j, cos th_j); vertex velocities follow by
    differentiation, v_j -+ (h/2) dth_j (cos th_j, sin th_j) for top / bottom
    (x_j = X_j + u_j and th_j the nodal rotation);
  * nodal loads on beam node j: the sum of the momentum-exchange forces of its
    two surface vertices; the moments of these forces about the centre line
    are not transferred (the flag-tip rotation is a stiff mode, omega dt ~ 1.5
    at h = 2, that the one-step lag of the staggered scheme drives unstable
    when they are);
  * one structural step per fluid step (dt = 1), theta-scheme loads F^n (the
    previous step's) and F^{n+1} (this step's).
"""
from __future__ import annotations

import numpy as np

from . import oracle as orc


def flag_vertices(X, u, v, h):
    """Surface vertices x[2nn,2] and velocities [2nn,2] of the flag polygon."""
    nn = X.shape[0]
    U = u.reshape(nn, 3)
    V = v.reshape(nn, 3)
    xc = X + U[:, :2]
    th, om = U[:, 2], V[:, 2]
    nrm = np.stack([-np.sin(th), np.cos(th)], axis=1)          # unit normal (top side)
    dn = np.stack([-np.cos(th), -np.sin(th)], axis=1) * om[:, None]
    bot = xc - 0.5 * h * nrm
    top = xc + 0.5 * h * nrm
    vbot = V[:, :2] - 0.5 * h * dn
    vtop = V[:, :2] + 0.5 * h * dn
    x = np.concatenate([bot, top[::-1]])
    vel = np.concatenate([vbot, vtop[::-1]])
    return x, vel


def nodal_loads(X, u, xs, fs):
    """Beam nodal loads [3nn] from the forces fs[2nn,3] on the flag vertices
    (forces only, no moments)."""
    nn = X.shape[0]
    F = np.zeros((nn, 3))
    for j in range(nn):
        for vtx in (j, 2 * nn - 1 - j):
            F[j, 0] += fs[vtx, 0]
            F[j, 1] += fs[vtx, 1]
    return F.reshape(-1)


class CSSFlag:
    """Rigid bodies plus one flag body (the last body) whose surface vertices
    are the last 2 nn vertices of the surface mesh."""

    def __init__(self, lat, shape, beta, bc, face_u, inlet, ramp, x_rigid, e_all, body,
                 beam: "orc.Beam", h, rho0=None, u0=None):
        self.lat, self.shape, self.beta, self.bc = lat, shape, beta, bc
        self.face_u, self.inlet, self.ramp = face_u, inlet, ramp
        self.x_rigid = np.asarray(x_rigid, dtype=np.float64)
        self.e, self.body = e_all, body
        self.beam, self.h = beam, h
        n = 3 * beam.nn
        self.u = np.zeros(n)
        self.v = np.zeros(n)
        self.F0 = np.zeros(n)
        self.t = 0
        nz, ny, nx = shape
        dim = 2
        rho0 = np.ones(shape) if rho0 is None else rho0
        u0 = np.zeros((dim,) + shape) if u0 is None else u0
        self.f = orc.init_equilibrium(lat, rho0, u0)
        self.surf = self._surface()
        self.solid = orc.solid_mask(shape, self.surf)
        self.iterations = []

    def _surface(self):
        xf, vf = flag_vertices(self.beam.X, self.u, self.v, self.h)
        x = np.concatenate([self.x_rigid, xf])
        vel = np.concatenate([np.zeros_like(self.x_rigid), vf])
        return orc.Surface(x, vel, self.e, self.body)

    def step(self):
        s = 1.0
        if self.ramp and self.t < self.ramp:
            s = 0.5 * (1 - np.cos(np.pi * self.t / self.ramp))
        # 1. fluid step with the current geometry and wall velocities
        self.f, vf, bf, _ = orc.step_bc(self.lat, self.beta, self.f, bc=self.bc, face_u=self.face_u,
                                        inlet=self.inlet, inlet_scale=s, surf=self.surf,
                                        solid=self.solid)
        self.vforce, self.bforce = vf, bf
        # 2. traction on the structure, structural step
        nr = self.x_rigid.shape[0]
        F1 = nodal_loads(self.beam.X, self.u, self.surf.x[nr:], vf[nr:])
        self.u, self.v, it = self.beam.step(self.u, self.v, self.F0, F1)
        self.iterations.append(it)
        self.F0 = F1
        # 3. transfer displacement and velocity, update the geometry
        self.surf = self._surface()
        new_solid = orc.solid_mask(self.shape, self.surf)
        orc.fresh_init(self.lat, self.f, self.solid, new_solid, self.surf, periodic=(0, 0, 1))
        self.solid = new_solid
        self.t += 1


def plate_vertices(X, u, R, h):
    """Plate surface vertices [2 nn, 3]: node position plus / minus h/2 times
    the rotated reference normal (third column of the node rotation)."""
    d = R[:, :, 2]
    x = X + u
    return np.concatenate([x + 0.5 * h * d, x - 0.5 * h * d])


def plate_velocities(v, R, h):
    d = 0.5 * h * R[:, :, 2]
    w = np.cross(v[:, 3:], d)
    return np.concatenate([v[:, :3] + w, v[:, :3] - w])


class CSSPlate:
    """Conventional serial staggered loop of the 3-D plate: D3Q27 fluid step
    with Grad boundaries, nodal loads (each shell node: the forces of its
    vertices above and below, no moments), one shell step, new surface,
    solid mask and fresh nodes.  The plate is the only body; its surface
    mesh e (triangles over vertices [top nodes, bottom nodes]) is fixed."""

    def __init__(self, shape, beta, bc, face_u, shell: "orc.Shell", e, h, u0=None, R0=None,
                 rho0=None, vel0=None, periodic=(0, 1, 0)):
        self.shape, self.beta, self.bc, self.face_u = shape, beta, bc, face_u
        self.shell, self.e, self.h, self.periodic = shell, np.asarray(e, np.int32), h, periodic
        u, R, v = shell.rest()
        self.u = u if u0 is None else np.array(u0, dtype=np.float64)
        self.R = R if R0 is None else np.array(R0, dtype=np.float64)
        self.v = v
        self.F0 = np.zeros((shell.nn, 6))
        nz, ny, nx = shape
        rho0 = np.ones(shape) if rho0 is None else rho0
        vel0 = np.zeros((3,) + shape) if vel0 is None else vel0
        self.f = orc.init_equilibrium(27, rho0, vel0)
        self.surf = self._surface()
        self.solid = orc.solid_mask(shape, self.surf)
        self.iterations = []

    def _surface(self):
        x = plate_vertices(self.shell.X, self.u, self.R, self.h)
        vel = plate_velocities(self.v, self.R, self.h)
        return orc.Surface(x, vel, self.e, np.zeros(len(self.e), np.int32))

    def step(self, **shell_kw):
        self.f, vf, bf, _ = orc.step_bc(27, self.beta, self.f, bc=self.bc, face_u=self.face_u,
                                        surf=self.surf, solid=self.solid)
        self.vforce, self.bforce = vf, bf
        nn = self.shell.nn
        F1 = np.zeros((nn, 6))
        F1[:, :3] = vf[:nn] + vf[nn:]
        self.u, self.R, self.v, it = self.shell.step(self.u, self.R, self.v, self.F0, F1, **shell_kw)
        self.iterations.append(it)
        self.F0 = F1
        self.surf = self._surface()
        new_solid = orc.solid_mask(self.shape, self.surf)
        orc.fresh_init(27, self.f, self.solid, new_solid, self.surf, periodic=self.periodic)
        self.solid = new_solid


class CSSFlagSpan:
    """Quasi-two-dimensional form of CSSFlag (section "Turek Benchmark": a few
    lattice points spanwise, periodic for the fluid, plane strain for the
    solid): D3Q27 fluid on shape (nz, ny, nx) periodic along z; the rigid
    outlines and the flag polygon extruded along z over [z0, z1] (z0 < 0,
    z1 > nz, so the end caps lie outside the periodic box).  Vertex k of the
    2-D outline (rigid vertices, then the flag's 2 nn) sits at z0 as vertex k
    and at z1 as vertex n + k; the triangles e3 and their bodies are given.
    Nodal loads per unit span: the forces of a node's four vertices (two
    edges, two ends) summed and divided by nz; moments are not transferred,
    as in the 2-D loop."""

    def __init__(self, shape, beta, bc, inlet, ramp, x_rigid, e3, body3, beam: "orc.Beam", h,
                 z0, z1):
        self.shape, self.beta, self.bc, self.inlet, self.ramp = shape, beta, bc, inlet, ramp
        self.x_rigid = np.asarray(x_rigid, dtype=np.float64)
        self.e3, self.body3 = np.asarray(e3, np.int32), np.asarray(body3, np.int32)
        self.beam, self.h, self.z0, self.z1 = beam, h, z0, z1
        n = 3 * beam.nn
        self.u = np.zeros(n)
        self.v = np.zeros(n)
        self.F0 = np.zeros(n)
        self.t = 0
        self.f = orc.init_equilibrium(27, np.ones(shape), np.zeros((3,) + tuple(shape)))
        self.surf = self._surface()
        self.solid = orc.solid_mask(shape, self.surf)

    def _surface(self):
        xf, vf = flag_vertices(self.beam.X, self.u, self.v, self.h)
        x2 = np.concatenate([self.x_rigid, xf])
        v2 = np.concatenate([np.zeros_like(self.x_rigid), vf])
        n = len(x2)
        x3 = np.zeros((2 * n, 3))
        v3 = np.zeros((2 * n, 3))
        x3[:n, :2], x3[n:, :2] = x2, x2
        x3[:n, 2], x3[n:, 2] = self.z0, self.z1
        v3[:n, :2], v3[n:, :2] = v2, v2
        return orc.Surface(x3, v3, self.e3, self.body3)

    def step(self):
        s = 1.0
        if self.ramp and self.t < self.ramp:
            s = 0.5 * (1 - np.cos(np.pi * self.t / self.ramp))
        self.f, vf, bf, _ = orc.step_bc(27, self.beta, self.f, bc=self.bc, inlet=self.inlet,
                                        inlet_scale=s, surf=self.surf, solid=self.solid)
        self.vforce, self.bforce = vf, bf
        nn, nr = self.beam.nn, self.x_rigid.shape[0]
        n = nr + 2 * nn
        F1 = np.zeros((nn, 3))
        for j in range(nn):
            for vtx in (nr + j, nr + 2 * nn - 1 - j, n + nr + j, n + nr + 2 * nn - 1 - j):
                F1[j, 0] += vf[vtx, 0]
                F1[j, 1] += vf[vtx, 1]
        F1 = F1.reshape(-1) / self.shape[0]
        self.u, self.v, it = self.beam.step(self.u, self.v, self.F0, F1)
        self.F0 = F1
        self.surf = self._surface()
        new_solid = orc.solid_mask(self.shape, self.surf)
        orc.fresh_init(27, self.f, self.solid, new_solid, self.surf, periodic=(0, 0, 1))
        self.solid = new_solid
        self.t += 1
