"""ctypes binding of the FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

The oracle (``kbc_oracle.c`` and friends in this folder) is a plain, slow,
double-precision statement of the entropic lattice Boltzmann (KBC) method of
Dorschner, Chikatamarla & Karlin (arXiv 1710.02375).  Only the tests, the
smoke check and the CPU-baseline leg of ``bench.py`` may import this module;
the CUDA library never does, and this module never touches the CUDA library.

Each wrapper names the equation of the paper it follows; the C source states
the readings of points the paper leaves open.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["kbc_oracle.c", "kbc_oracle_bc.c", "fem_oracle.c", "shell_oracle.c"]
_LIB_PATH = os.path.join(_HERE, "libkbc_oracle.so")
_lib = None

D = ctypes.POINTER(ctypes.c_double)
I32 = ctypes.POINTER(ctypes.c_int32)
U8 = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle's C sources into a shared library with gcc."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIB_PATH):
        lib_mtime = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= lib_mtime for s in srcs):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
           "-o", tmp] + srcs + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


def _declare(L):
    c_int, c_double = ctypes.c_int, ctypes.c_double
    L.or_lattice_tables.argtypes = [c_int, I32, D]
    L.or_equilibrium.argtypes = [c_int, c_double, D, D]
    L.or_collide.argtypes = [c_int, c_double, c_int, D, D, D, D, D, D]
    L.or_init_equilibrium.argtypes = [c_int, c_int, c_int, c_int, D, D, D]
    L.or_macros.argtypes = [c_int, c_int, c_int, c_int, D, D, D]
    L.or_step_periodic.argtypes = [c_int, c_int, c_int, c_int, c_double, c_int, D, D, D]
    L.or_run_periodic.argtypes = [c_int, c_int, c_int, c_int, c_double, c_int, c_int, D, D]
    L.or_solid_mask.argtypes = [c_int, c_int, c_int, c_int, c_int, c_int, c_int, D, I32, I32, U8]
    L.or_step_bc.argtypes = [c_int, c_int, c_int, c_int, c_double, c_int, I32, D,
                             ctypes.POINTER(D), c_double, U8, c_int, c_int, c_int, D, D, I32, I32,
                             D, D, D, D, D]
    L.or_beam_step.argtypes = [c_int, D, c_double, c_double, c_double, I32, c_double, c_double,
                               c_double, c_double, c_double, c_int, D, D, D, D]
    L.or_beam_static.argtypes = [c_int, D, c_double, c_double, I32, D, c_double, c_double, c_double,
                                 c_int, D]
    L.or_beam_internal.argtypes = [c_int, D, c_double, c_double, D, D, D]
    L.or_shell_internal.argtypes = [c_int, c_int, D, c_double, c_double, c_double, c_double, I32, D, D, D]
    L.or_shell_mass.argtypes = [c_int, c_int, D, c_double, c_double, c_double, c_double, D, D]
    L.or_shell_step.argtypes = [c_int, c_int, D, c_double, c_double, c_double, c_double, I32, c_double,
                                c_double, c_double, c_double, c_double, c_int, D, D, D, D, D]
    L.or_shell_static.argtypes = [c_int, c_int, D, c_double, c_double, c_double, I32, D, c_double,
                                  c_double, c_double, c_int, D, D]
    L.or_beam_mass.argtypes = [c_int, D, c_double, D]
    L.or_fresh_init.argtypes = [c_int, c_int, c_int, c_int, I32, U8, U8, c_int, D, D, D]
    L.or_links.argtypes = [c_int, c_int, c_int, c_int, I32, U8, c_int, c_int, c_int, D, D, I32, I32,
                           c_int, I32, I32, D, I32, D]
    L.or_eos.argtypes = [c_int, c_int, D, D]
    L.or_step_multiphase.argtypes = [c_int, c_int, c_int, c_int, c_double, c_int, c_double, c_int, D,
                                     D, D, D]
    L.or_step_multiphase_wall.argtypes = [c_int, c_int, c_int, c_int, c_double, c_int, c_double, c_int,
                                          D, c_double, c_int, D, D, D, D]
    L.or_refine_step.argtypes = [c_int, c_int, c_double, c_double, c_int, c_int, c_int, c_int,
                                 c_int, D, D, D, D]


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(D)


def _check(rc):
    if rc < 0:
        raise RuntimeError(f"oracle call failed with status {rc}")
    return rc


def lattice(lat: int):
    """Velocities c[Q,3] and weights W[Q] (tensor product of D1Q3)."""
    Q = lat
    c = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q, dtype=np.float64)
    _check(lib().or_lattice_tables(lat, c.ctypes.data_as(I32), _p(w)))
    return c, w


def equilibrium(lat: int, rho: float, u) -> np.ndarray:
    """Minimiser of H(f) = sum f ln(f/W) at given rho, u (Eqs. feq_min, conservationLaws)."""
    uu = np.zeros(3)
    uu[: len(u)] = u
    feq = np.zeros(lat)
    _check(lib().or_equilibrium(lat, float(rho), _p(uu), _p(feq)))
    return feq


def collide(lat: int, beta: float, f: np.ndarray, mode: int = 0):
    """One KBC collision (Eqs. f_equations, f_mirr, gamma_min_approx) at one node.

    mode 0 is KBC, mode 1 fixes gamma = 2 (LBGK with omega = 2 beta).
    Returns (f_post, gamma, ds, dh, feq)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    fo = np.zeros(lat)
    g = np.zeros(1)
    ds = np.zeros(lat)
    dh = np.zeros(lat)
    feq = np.zeros(lat)
    _check(lib().or_collide(lat, float(beta), int(mode), _p(f), _p(fo), _p(g), _p(ds), _p(dh), _p(feq)))
    return fo, float(g[0]), ds, dh, feq


def init_equilibrium(lat: int, rho: np.ndarray, u: np.ndarray) -> np.ndarray:
    """State f[Q, nz, ny, nx] = feq(rho, u) per node; rho[nz,ny,nx], u[dim,nz,ny,nx]."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    nz, ny, nx = rho.shape
    u3 = np.zeros((3,) + rho.shape)
    u3[: u.shape[0]] = u
    f = np.zeros((lat,) + rho.shape)
    _check(lib().or_init_equilibrium(lat, nx, ny, nz, _p(rho), _p(u3), _p(f)))
    return f


def macros(lat: int, f: np.ndarray):
    """Density rho[nz,ny,nx] and velocity u[3,nz,ny,nx] of a state."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    _, nz, ny, nx = f.shape
    rho = np.zeros((nz, ny, nx))
    u = np.zeros((3, nz, ny, nx))
    _check(lib().or_macros(lat, nx, ny, nz, _p(f), _p(rho), _p(u)))
    return rho, u


def step_periodic(lat: int, beta: float, f: np.ndarray, mode: int = 0, want_gamma: bool = False):
    """One fully periodic pull-stream + collide step (Eq. f_equations)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    _, nz, ny, nx = f.shape
    fo = np.zeros_like(f)
    g = np.zeros((nz, ny, nx)) if want_gamma else None
    _check(lib().or_step_periodic(lat, nx, ny, nz, float(beta), int(mode), _p(f), _p(fo),
                                  _p(g) if want_gamma else None))
    return (fo, g) if want_gamma else fo


def run_periodic(lat: int, beta: float, f: np.ndarray, nsteps: int, mode: int = 0) -> np.ndarray:
    """nsteps periodic steps starting from the post-collision state f."""
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    work = np.zeros_like(f)
    _, nz, ny, nx = f.shape
    _check(lib().or_run_periodic(lat, nx, ny, nz, float(beta), int(mode), int(nsteps), _p(f), _p(work)))
    return f


# ---------------------------------------------------------------- boundaries
class Surface:
    """Closed surface mesh in lattice units: vertices x[nv,dim], vertex
    velocities v[nv,dim], elements e[ne,dim] (segments / triangles) and a body
    id per element."""

    def __init__(self, x, v, e, body, nbodies=None):
        self.x = np.ascontiguousarray(x, dtype=np.float64)
        self.v = np.ascontiguousarray(v, dtype=np.float64)
        self.e = np.ascontiguousarray(e, dtype=np.int32)
        self.body = np.ascontiguousarray(body, dtype=np.int32)
        self.dim = self.x.shape[1]
        self.nb = int(nbodies if nbodies is not None else (self.body.max() + 1 if len(self.body) else 0))

    @staticmethod
    def empty(dim):
        return Surface(np.zeros((0, dim)), np.zeros((0, dim)), np.zeros((0, dim), np.int32),
                       np.zeros(0, np.int32), 0)


def solid_mask(shape, surf: "Surface") -> np.ndarray:
    """Interior nodes inside any closed body (crossing-number test)."""
    nz, ny, nx = shape
    m = np.zeros(shape, dtype=np.uint8)
    if surf.e.shape[0]:
        _check(lib().or_solid_mask(surf.dim, nx, ny, nz, surf.x.shape[0], surf.e.shape[0], surf.nb,
                                   _p(surf.x), surf.e.ctypes.data_as(I32), surf.body.ctypes.data_as(I32),
                                   m.ctypes.data_as(U8)))
    return m


def step_bc(lat, beta, f, bc, face_u=None, inlet=None, inlet_scale=1.0, surf=None, solid=None,
            mode=0, want_sigma=False):
    """One step with Grad boundaries (walls, open faces, immersed surfaces).

    bc: 6 face kinds; face_u[6,3]; inlet: dict face -> profile [3, face nodes];
    returns (f_new, vertex_force[nv,3], body_force[nb,3], n_links), plus
    sigma[nz, ny, nx, 7] when want_sigma (fluid stress xx, yy, zz, xy, xz, yz
    of the pre-collision state at immersed boundary nodes, last entry 1 there
    and 0 elsewhere)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    Q, nz, ny, nx = f.shape
    dim = 2 if lat == 9 else 3
    surf = surf if surf is not None else Surface.empty(dim)
    if solid is None:
        solid = solid_mask((nz, ny, nx), surf)
    solid = np.ascontiguousarray(solid, dtype=np.uint8)
    bcv = np.ascontiguousarray(bc, dtype=np.int32)
    fu = np.zeros((6, 3)) if face_u is None else np.ascontiguousarray(face_u, dtype=np.float64)
    keep = []
    arr = (D * 6)()
    for fc in range(6):
        if inlet is not None and fc in inlet:
            prof = np.ascontiguousarray(inlet[fc], dtype=np.float64)
            keep.append(prof)
            arr[fc] = _p(prof)
        else:
            arr[fc] = None
    fo = np.zeros_like(f)
    nv, ne, nb = surf.x.shape[0], surf.e.shape[0], max(surf.nb, 1)
    vf = np.zeros((max(nv, 1), 3))
    bf = np.zeros((nb, 3))
    x = surf.x if nv else np.zeros((1, dim))
    v = surf.v if nv else np.zeros((1, dim))
    e = surf.e if ne else np.zeros((1, dim), np.int32)
    b = surf.body if ne else np.zeros(1, np.int32)
    sig = np.zeros((nz, ny, nx, 7)) if want_sigma else None
    n = lib().or_step_bc(lat, nx, ny, nz, float(beta), int(mode), bcv.ctypes.data_as(I32), _p(fu), arr,
                         float(inlet_scale), solid.ctypes.data_as(U8), nv, ne, surf.nb, _p(x), _p(v),
                         e.ctypes.data_as(I32), b.ctypes.data_as(I32), _p(f), _p(fo), _p(vf), _p(bf),
                         _p(sig) if sig is not None else None)
    _check(n)
    if want_sigma:
        return fo, vf[:nv], bf[: surf.nb], n, sig
    return fo, vf[:nv], bf[: surf.nb], n


def traction(surf: "Surface", sigma):
    """Surface traction forces from the boundary-node stresses of step_bc
    (section "Fluid-structure coupling", the stress path): each element takes
    the stress of the boundary node nearest to its centroid (squared distance
    summed over the axes in order; ties: the lower node index (z, y, x)),
    t = sigma n with n the outward unit normal of its body (orientation from
    the body's signed area / volume), times the element length (2-D) or area
    (3-D); the force is shared equally by the element's vertices.
    Returns (vertex_force[nv,3], body_force[nb,3], element_force[ne,3])."""
    dim = surf.x.shape[1]
    nz, ny, nx, _ = sigma.shape
    zz, yy, xx = np.nonzero(sigma[..., 6] == 1.0)          # C order = increasing index
    pos = np.stack([xx + 0.5, yy + 0.5, zz + 0.5], axis=1)
    orient = np.zeros(surf.nb)
    for k, el in enumerate(surf.e):
        P = surf.x[el]
        if dim == 2:
            orient[surf.body[k]] += 0.5 * (P[0, 0] * P[1, 1] - P[1, 0] * P[0, 1])
        else:
            orient[surf.body[k]] += np.dot(P[0], np.cross(P[1], P[2])) / 6.0
    vf = np.zeros((surf.x.shape[0], 3))
    bf = np.zeros((surf.nb, 3))
    ef = np.zeros((surf.e.shape[0], 3))
    if len(pos) == 0:
        return vf, bf, ef
    for k, el in enumerate(surf.e):
        P = surf.x[el]
        sg = 1.0 if orient[surf.body[k]] >= 0.0 else -1.0
        nA = np.zeros(3)
        if dim == 2:
            xc = np.array([0.5 * (P[0, 0] + P[1, 0]), 0.5 * (P[0, 1] + P[1, 1]), 0.0])
            nA[0] = sg * (P[1, 1] - P[0, 1])
            nA[1] = -sg * (P[1, 0] - P[0, 0])
        else:
            xc = (P[0] + P[1] + P[2]) / 3.0
            nA = 0.5 * sg * np.cross(P[1] - P[0], P[2] - P[0])
        d2 = np.zeros(len(pos))
        for q in range(dim):
            d2 = d2 + (pos[:, q] - xc[q]) ** 2
        best = int(np.argmin(d2))                           # first minimum = lowest index
        s6 = sigma[zz[best], yy[best], xx[best], :6]
        S = np.array([[s6[0], s6[3], s6[4]], [s6[3], s6[1], s6[5]], [s6[4], s6[5], s6[2]]])
        F = S @ nA
        ef[k, :dim] = F[:dim]
        bf[surf.body[k], :dim] += F[:dim]
        for m in range(dim):
            vf[el[m], :dim] += F[:dim] / dim
    return vf, bf, ef


def links(lat, shape, surf: "Surface", periodic=(1, 1, 1), solid=None):
    """Immersed cut links of a static configuration: dict of arrays node, dir,
    q, elem, uw (q = -1 and elem = -1 where no crossing was found)."""
    nz, ny, nx = shape
    if solid is None:
        solid = solid_mask(shape, surf)
    solid = np.ascontiguousarray(solid, dtype=np.uint8)
    per = np.ascontiguousarray(periodic, dtype=np.int32)
    args = lambda cap, a: (lat, nx, ny, nz, per.ctypes.data_as(I32), solid.ctypes.data_as(U8),
                           surf.x.shape[0], surf.e.shape[0], surf.nb, _p(surf.x), _p(surf.v),
                           surf.e.ctypes.data_as(I32), surf.body.ctypes.data_as(I32), cap,
                           a["node"].ctypes.data_as(I32), a["dir"].ctypes.data_as(I32), _p(a["q"]),
                           a["elem"].ctypes.data_as(I32), _p(a["uw"]))

    def alloc(cap):
        return {"node": np.zeros(cap, np.int32), "dir": np.zeros(cap, np.int32), "q": np.zeros(cap),
                "elem": np.zeros(cap, np.int32), "uw": np.zeros((cap, 3))}
    a = alloc(1)
    n = _check(lib().or_links(*args(0, a)))
    a = alloc(max(n, 1))
    _check(lib().or_links(*args(n, a)))
    return {k: v[:n] for k, v in a.items()}


def fresh_init(lat, f, old_solid, new_solid, surf: "Surface", periodic=(0, 0, 1)):
    """Initialise nodes uncovered by a moving surface (in place); returns their count."""
    Q, nz, ny, nx = f.shape
    assert f.dtype == np.float64 and f.flags["C_CONTIGUOUS"]
    per = np.ascontiguousarray(periodic, dtype=np.int32)
    a = np.ascontiguousarray(old_solid, dtype=np.uint8)
    b = np.ascontiguousarray(new_solid, dtype=np.uint8)
    return _check(lib().or_fresh_init(lat, nx, ny, nz, per.ctypes.data_as(I32), a.ctypes.data_as(U8),
                                      b.ctypes.data_as(U8), surf.x.shape[0], _p(surf.x), _p(surf.v),
                                      _p(f)))


# ---------------------------------------------------------------- multiphase
def eos(rho, kind=0):
    """Pressure of Eq. (eos) (kind 0) or of the ideal gas rho c_s^2 (kind 1)."""
    r = np.ascontiguousarray(np.atleast_1d(rho), dtype=np.float64)
    p = np.zeros_like(r)
    _check(lib().or_eos(int(kind), r.size, _p(r), _p(p)))
    return p


def step_multiphase(lat, beta, f, kappa, eos_kind=0, g_ext=None, mode=0, want_force=False):
    """One periodic multiphase KBC step (mean-field Korteweg force, exact
    difference forcing, shifted entropic product for gamma); returns f_new
    (and the force field F[3, nz, ny, nx] when want_force)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    _, nz, ny, nx = f.shape
    fo = np.zeros_like(f)
    g = None if g_ext is None else np.ascontiguousarray(g_ext, dtype=np.float64)
    F = np.zeros((3, nz, ny, nx)) if want_force else None
    _check(lib().or_step_multiphase(lat, nx, ny, nz, float(beta), int(mode), float(kappa), int(eos_kind),
                                    _p(g) if g is not None else None, _p(f), _p(fo),
                                    _p(F) if F is not None else None))
    return (fo, F) if want_force else fo


def step_multiphase_wall(lat, beta, f, kappa, kappa_w, wall_axis, F_prev=None, eos_kind=0,
                         g_ext=None, mode=0):
    """One multiphase step between two planar walls normal to wall_axis (x =
    0, y = 1, z = 2; half a cell outside the faces, at rest; the other axes
    periodic) with the wetting force of strength kappa_w; F_prev: the force
    of the step that produced f (None: zero).  Returns (f_new, F)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    _, nz, ny, nx = f.shape
    fo = np.zeros_like(f)
    F = np.zeros((3, nz, ny, nx))
    g = None if g_ext is None else np.ascontiguousarray(g_ext, dtype=np.float64)
    fp = None if F_prev is None else np.ascontiguousarray(F_prev, dtype=np.float64)
    _check(lib().or_step_multiphase_wall(lat, nx, ny, nz, float(beta), int(mode), float(kappa),
                                         int(eos_kind), _p(g) if g is not None else None,
                                         float(kappa_w), int(wall_axis), _p(f),
                                         _p(fp) if fp is not None else None, _p(fo), _p(F)))
    return fo, F


# ---------------------------------------------------------------- refinement
def refine_step(beta_c, fc, ff, i0, j0, mode=0):
    """One coarse step of the two-level refinement (D2Q9): the periodic coarse
    state fc[9, 1, nyc, nxc] and the fine patch ff[9, 1, nfy, nfx] (spacing
    1/2, covering the coarse cells [i0, i0 + nfx/2) x [j0, j0 + nfy/2), two
    fine steps at nu_fine = 2 nu_coarse).  Returns (fc_new, ff_new)."""
    fc = np.ascontiguousarray(fc, dtype=np.float64)
    ff = np.ascontiguousarray(ff, dtype=np.float64)
    _, _, nyc, nxc = fc.shape
    _, _, nfy, nfx = ff.shape
    nu_c = (1.0 / (2.0 * beta_c) - 0.5) / 3.0
    beta_f = 1.0 / (6.0 * 2.0 * nu_c + 1.0)
    fco, ffo = np.zeros_like(fc), np.zeros_like(ff)
    _check(lib().or_refine_step(nxc, nyc, float(beta_c), beta_f, int(mode), int(i0), int(j0), nfx, nfy,
                                _p(fc), _p(ff), _p(fco), _p(ffo)))
    return fco, ffo


def macros_forced(lat, f, F):
    """Density and fluid velocity of a post-collision state f of a forced step
    with force F: the momentum before the step's forcing was j - F, the fluid
    velocity of the step (j - F/2) / rho."""
    rho, u = macros(lat, f)
    return rho, u - 0.5 * F / rho


# ---------------------------------------------------------------- structure
class Beam:
    """2-D co-rotational Euler-Bernoulli beam (FP64 oracle): reference nodes
    X[nn,2], axial stiffness EA, bending stiffness EI, mass per length rhoA,
    fixed[3 nn] Dirichlet mask (DOFs ux, uy, theta per node)."""

    def __init__(self, X, EA, EI, rhoA, fixed):
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        self.nn = self.X.shape[0]
        self.EA, self.EI, self.rhoA = float(EA), float(EI), float(rhoA)
        self.fixed = np.ascontiguousarray(fixed, dtype=np.int32)

    def internal(self, u, want_K=True):
        n = 3 * self.nn
        f = np.zeros(n)
        K = np.zeros((n, n)) if want_K else None
        u = np.ascontiguousarray(u, dtype=np.float64)
        lib().or_beam_internal(self.nn, _p(self.X), self.EA, self.EI, _p(u), _p(f),
                               _p(K) if want_K else None)
        return f, K

    def mass(self):
        n = 3 * self.nn
        M = np.zeros((n, n))
        lib().or_beam_mass(self.nn, _p(self.X), self.rhoA, _p(M))
        return M

    def step(self, u, v, F0, F1, dt=1.0, theta=0.5, lam=0.7, rtol=1e-10, atol=1e-13, max_it=200):
        """One theta-scheme step (Eq. timeInt) with Newton + line search lambda;
        returns (u1, v1, iterations)."""
        u = np.array(u, dtype=np.float64)
        v = np.array(v, dtype=np.float64)
        F0 = np.ascontiguousarray(F0, dtype=np.float64)
        F1 = np.ascontiguousarray(F1, dtype=np.float64)
        it = lib().or_beam_step(self.nn, _p(self.X), self.EA, self.EI, self.rhoA,
                                self.fixed.ctypes.data_as(I32), dt, theta, lam, rtol, atol, max_it,
                                _p(F0), _p(F1), _p(u), _p(v))
        return u, v, it

    def static(self, F, lam=1.0, rtol=1e-12, atol=1e-13, max_it=200, u0=None):
        u = np.zeros(3 * self.nn) if u0 is None else np.array(u0, dtype=np.float64)
        F = np.ascontiguousarray(F, dtype=np.float64)
        it = lib().or_beam_static(self.nn, _p(self.X), self.EA, self.EI, self.fixed.ctypes.data_as(I32),
                                  _p(F), lam, rtol, atol, max_it, _p(u))
        return u, it


class Shell:
    """3-D co-rotational flat shell of 4-node quadrilaterals on an nx x ny node
    grid (FP64 oracle): reference nodes X[nx*ny, 3] (node i*ny + j), Young's
    modulus E, Poisson ratio nu, thickness h, density rho, fixed[6 nn] mask
    (ux, uy, uz, three rotations per node).  State: u[nn,3] translations,
    R[nn,3,3] nodal rotation matrices, v[nn,6] translational and angular
    velocities."""

    def __init__(self, X, nx, ny, E, nu, h, rho, fixed):
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        self.nx, self.ny = int(nx), int(ny)
        self.nn = self.nx * self.ny
        assert self.X.shape == (self.nn, 3)
        self.E, self.nu, self.h, self.rho = float(E), float(nu), float(h), float(rho)
        self.fixed = np.ascontiguousarray(fixed, dtype=np.int32)

    def rest(self):
        u = np.zeros((self.nn, 3))
        R = np.tile(np.eye(3), (self.nn, 1, 1))
        v = np.zeros((self.nn, 6))
        return u, R, v

    def internal(self, u, R):
        f = np.zeros((self.nn, 6))
        u = np.ascontiguousarray(u, dtype=np.float64)
        R = np.ascontiguousarray(R, dtype=np.float64)
        _check(lib().or_shell_internal(self.nx, self.ny, _p(self.X), self.E, self.nu, self.h, self.rho,
                                       self.fixed.ctypes.data_as(I32), _p(u), _p(R), _p(f)))
        return f

    def mass(self):
        m = np.zeros(self.nn)
        J = np.zeros(self.nn)
        _check(lib().or_shell_mass(self.nx, self.ny, _p(self.X), self.E, self.nu, self.h, self.rho,
                                   _p(m), _p(J)))
        return m, J

    def step(self, u, R, v, F0, F1, dt=1.0, theta=0.5, lam=0.7, rtol=1e-10, atol=1e-13, max_it=200):
        """One theta-scheme step; returns (u1, R1, v1, iterations)."""
        u = np.array(u, dtype=np.float64)
        R = np.array(R, dtype=np.float64)
        v = np.array(v, dtype=np.float64)
        F0 = np.ascontiguousarray(F0, dtype=np.float64)
        F1 = np.ascontiguousarray(F1, dtype=np.float64)
        it = lib().or_shell_step(self.nx, self.ny, _p(self.X), self.E, self.nu, self.h, self.rho,
                                 self.fixed.ctypes.data_as(I32), dt, theta, lam, rtol, atol, max_it,
                                 _p(F0), _p(F1), _p(u), _p(R), _p(v))
        return u, R, v, it

    def static(self, F, lam=1.0, rtol=1e-12, atol=1e-14, max_it=200, u=None, R=None):
        u0, R0, _ = self.rest()
        u = u0 if u is None else np.array(u, dtype=np.float64)
        R = R0 if R is None else np.array(R, dtype=np.float64)
        F = np.ascontiguousarray(F, dtype=np.float64)
        it = lib().or_shell_static(self.nx, self.ny, _p(self.X), self.E, self.nu, self.h,
                                   self.fixed.ctypes.data_as(I32), _p(F), lam, rtol, atol, max_it,
                                   _p(u), _p(R))
        return u, R, it
