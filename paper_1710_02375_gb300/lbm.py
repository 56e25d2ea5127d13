"""Python binding of the C ABI in include/kbc_lbm.h (argument marshalling only).

Every function here has the name of the C entry point it calls and passes
plain pointers and sizes; all lattice Boltzmann work runs in the CUDA library
libkbcfsi.so.  PyTorch provides device memory (the context workspace) and the
CUDA stream.  There is no CPU fallback: if the library is missing or does not
load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkbcfsi.so")
_lib = None

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_ECAPACITY, LBM_ESTATE = (
    0, -1, -2, -3, -4, -5, -6, -7)
STATUS_NAMES = {0: "LBM_OK", -1: "LBM_EINVAL", -2: "LBM_ENOMEM", -3: "LBM_ECUDA", -4: "LBM_EUNSTABLE",
                -5: "LBM_ETIMEOUT", -6: "LBM_ECAPACITY", -7: "LBM_ESTATE"}
LBM_D2Q9, LBM_D3Q27 = 9, 27
LBM_STORE_F32, LBM_STORE_F16, LBM_STORE_BF16, LBM_STORE_F64, LBM_STORE_F16N = 0, 1, 2, 3, 4
LBM_COLLIDE_KBC, LBM_COLLIDE_BGK = 0, 1
LBM_BC_PERIODIC, LBM_BC_WALL, LBM_BC_INLET, LBM_BC_OUTLET, LBM_BC_FREESTREAM = 0, 1, 2, 3, 4


class lbm_config(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("beta", ctypes.c_double),
        ("storage", ctypes.c_int),
        ("collision", ctypes.c_int),
        ("bc", ctypes.c_int * 6),
        ("face_velocity", (ctypes.c_double * 3) * 6),
        ("max_links", ctypes.c_int),
        ("max_vertices", ctypes.c_int),
        ("max_elements", ctypes.c_int),
        ("inlet_ramp_steps", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("multiphase", ctypes.c_int),
    ]


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load():
    """Load libkbcfsi.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    L.lbm_workspace_size.argtypes = [ctypes.POINTER(lbm_config), ctypes.POINTER(sz)]
    L.lbm_create.argtypes = [ctypes.POINTER(lbm_config), vp, sz, ctypes.POINTER(vp)]
    L.lbm_init_equilibrium.argtypes = [vp, vp, vp]
    L.lbm_set_populations.argtypes = [vp, vp]
    L.lbm_get_populations.argtypes = [vp, vp]
    L.lbm_step.argtypes = [vp, i32]
    L.lbm_get_macros.argtypes = [vp, vp, vp]
    L.lbm_get_macros_f32.argtypes = [vp, vp, vp]
    L.lbm_check.argtypes = [vp]
    L.lbm_set_inlet_profile.argtypes = [vp, i32, vp]
    L.lbm_set_geometry.argtypes = [vp, i32, vp, i32, vp, i32, vp, vp, ctypes.c_double]
    L.lbm_update_surface.argtypes = [vp, vp, vp]
    L.lbm_get_interface_force.argtypes = [vp, vp, vp]
    L.lbm_get_traction_force.argtypes = [vp, vp, vp]
    L.lbm_get_traction_force.restype = ctypes.c_int
    L.lbm_set_traction_output.argtypes = [vp, ctypes.c_int]
    L.lbm_set_traction_output.restype = ctypes.c_int
    L.lbm_get_boundary_info.argtypes = [vp, vp]
    for name in ("lbm_set_inlet_profile", "lbm_set_geometry", "lbm_update_surface",
                 "lbm_get_interface_force", "lbm_get_boundary_info"):
        getattr(L, name).restype = ctypes.c_int
    L.fsi_set_surrogate.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.c_double]
    L.fsi_set_surrogate.restype = ctypes.c_int
    L.fsi_get_structure_stats.argtypes = [vp, ctypes.POINTER(i32), i32]
    L.fsi_get_structure_stats.restype = ctypes.c_int
    L.lbm_step_graph.argtypes = [vp, i32, i32]
    L.lbm_step_graph.restype = ctypes.c_int
    L.lbm_probe_interface_force_static.argtypes = [vp, vp, vp]
    L.lbm_probe_interface_force_static.restype = ctypes.c_int
    L.lbm_set_sweep_variant.argtypes = [vp, i32]
    L.lbm_set_sweep_variant.restype = ctypes.c_int
    L.lbm_stream.argtypes = [vp]
    L.lbm_stream.restype = vp
    L.lbm_last_error.argtypes = [vp]
    L.lbm_last_error.restype = ctypes.c_char_p
    L.lbm_destroy.argtypes = [vp]
    L.lbm_destroy.restype = None
    for name in ("lbm_workspace_size", "lbm_create", "lbm_init_equilibrium", "lbm_set_populations",
                 "lbm_get_populations", "lbm_step", "lbm_get_macros", "lbm_get_macros_f32",
                 "lbm_check"):
        getattr(L, name).restype = ctypes.c_int
    _extend(L)
    _lib = L
    return L


def _extend(L):
    """Declarations of the entry points added by later subsystems (if exported)."""
    from . import _abi_ext
    _abi_ext.declare(L)


def _ptr(a):
    """Raw pointer of a numpy array or torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _chk(ctx, st):
    if st != LBM_OK:
        msg = load().lbm_last_error(ctx).decode(errors="replace") if True else ""
        raise LbmError(st, msg)


def make_config(lattice, nx, ny, nz, beta, storage=LBM_STORE_F32, collision=LBM_COLLIDE_KBC,
                bc=(0, 0, 0, 0, 0, 0), face_velocity=None, max_links=0, max_vertices=0,
                max_elements=0, stream=None, inlet_ramp_steps=0, multiphase=False) -> lbm_config:
    c = lbm_config()
    c.lattice, c.nx, c.ny, c.nz = lattice, nx, ny, nz
    c.beta, c.storage, c.collision = beta, storage, collision
    for k in range(6):
        c.bc[k] = bc[k]
        if face_velocity is not None:
            for a in range(3):
                c.face_velocity[k][a] = face_velocity[k][a]
    c.max_links, c.max_vertices, c.max_elements = max_links, max_vertices, max_elements
    c.inlet_ramp_steps = inlet_ramp_steps
    c.stream = stream
    c.multiphase = int(bool(multiphase))
    return c


def lbm_workspace_size(cfg: lbm_config) -> int:
    n = ctypes.c_size_t()
    st = load().lbm_workspace_size(ctypes.byref(cfg), ctypes.byref(n))
    if st != LBM_OK:
        raise LbmError(st, load().lbm_last_error(None).decode())
    return n.value


def lbm_create(cfg: lbm_config, workspace_ptr: int | None, workspace_bytes: int):
    out = ctypes.c_void_p()
    st = load().lbm_create(ctypes.byref(cfg), workspace_ptr, workspace_bytes, ctypes.byref(out))
    if st != LBM_OK:
        raise LbmError(st, load().lbm_last_error(None).decode())
    return out.value


def lbm_init_equilibrium(ctx, rho, u):
    _chk(ctx, load().lbm_init_equilibrium(ctx, _ptr(rho), _ptr(u)))


def lbm_set_populations(ctx, f):
    _chk(ctx, load().lbm_set_populations(ctx, _ptr(f)))


def lbm_get_populations(ctx, f):
    _chk(ctx, load().lbm_get_populations(ctx, _ptr(f)))


def lbm_step(ctx, n: int):
    _chk(ctx, load().lbm_step(ctx, int(n)))


def lbm_step_graph(ctx, n: int, repeats: int):
    _chk(ctx, load().lbm_step_graph(ctx, int(n), int(repeats)))


def lbm_get_macros(ctx, rho, u):
    _chk(ctx, load().lbm_get_macros(ctx, _ptr(rho), _ptr(u)))


def lbm_get_macros_f32(ctx, rho, u):
    """FP32 density and velocity (float32 arrays, host or device)."""
    _chk(ctx, load().lbm_get_macros_f32(ctx, _ptr(rho), _ptr(u)))


LBM_SWEEP_AUTO, LBM_SWEEP_DIRECT, LBM_SWEEP_ROWS, LBM_SWEEP_ASYNC, LBM_SWEEP_PAIR = 0, 1, 2, 3, 4


def lbm_set_sweep_variant(ctx, variant: int):
    _chk(ctx, load().lbm_set_sweep_variant(ctx, int(variant)))


LBM_EOS_PAPER, LBM_EOS_IDEAL = 0, 1


def lbm_set_multiphase(ctx, kappa, eos=LBM_EOS_PAPER, g=(0.0, 0.0, 0.0), kappa_w=0.0):
    """Switch to the multiphase step (kappa None: back to single phase)."""
    if kappa is None:
        _chk(ctx, load().lbm_set_multiphase(ctx, None))
        return
    from ._abi_ext import lbm_multiphase_params
    p = lbm_multiphase_params()
    p.kappa, p.eos, p.kappa_w = float(kappa), int(eos), float(kappa_w)
    for a in range(3):
        p.g[a] = float(g[a]) if a < len(g) else 0.0
    _chk(ctx, load().lbm_set_multiphase(ctx, ctypes.byref(p)))


def lbm_get_force_field(ctx, F):
    _chk(ctx, load().lbm_get_force_field(ctx, _ptr(F)))


def lbm_refine_workspace_size(coarse, fine) -> int:
    n = ctypes.c_size_t()
    _chk(coarse, load().lbm_refine_workspace_size(coarse, fine, ctypes.byref(n)))
    return n.value


def lbm_refine_couple(coarse, fine, i0, j0, workspace_ptr, workspace_bytes):
    """Couple a fine patch to a coarse lattice (fine None: uncouple)."""
    _chk(coarse, load().lbm_refine_couple(coarse, fine, int(i0), int(j0), workspace_ptr,
                                          int(workspace_bytes)))


def lbm_set_inlet_profile(ctx, face, u):
    _chk(ctx, load().lbm_set_inlet_profile(ctx, int(face), _ptr(u)))


def lbm_set_geometry(ctx, nbodies, verts, nv, elems, ne, elem_body, vert_vel, band_margin):
    _chk(ctx, load().lbm_set_geometry(ctx, int(nbodies), _ptr(verts), int(nv), _ptr(elems), int(ne),
                                      _ptr(elem_body), _ptr(vert_vel), float(band_margin)))


def lbm_update_surface(ctx, verts, vert_vel):
    _chk(ctx, load().lbm_update_surface(ctx, _ptr(verts), _ptr(vert_vel)))


def lbm_get_interface_force(ctx, vert_force, body_force):
    _chk(ctx, load().lbm_get_interface_force(ctx, _ptr(vert_force), _ptr(body_force)))


def lbm_set_traction_output(ctx, enable):
    _chk(ctx, load().lbm_set_traction_output(ctx, int(bool(enable))))


def lbm_get_traction_force(ctx, vert_force, body_force):
    _chk(ctx, load().lbm_get_traction_force(ctx, _ptr(vert_force), _ptr(body_force)))


def lbm_get_boundary_info(ctx, info):
    _chk(ctx, load().lbm_get_boundary_info(ctx, _ptr(info)))


def lbm_probe_interface_force_static(ctx, vert_force, body_force):
    _chk(ctx, load().lbm_probe_interface_force_static(ctx, _ptr(vert_force), _ptr(body_force)))


def fsi_couple_shell(ctx, shell_ctx, first_vertex):
    _chk(ctx, load().fsi_couple_shell(ctx, shell_ctx, int(first_vertex)))


def fsi_set_surrogate(ctx, mlp_ctx, in_mean, in_std, out_mean, out_std, accept_tol):
    """Attach (mlp_ctx not None) or remove the structural-step surrogate."""
    if mlp_ctx is None:
        _chk(ctx, load().fsi_set_surrogate(ctx, None, None, None, None, None, 1.0))
        return
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (in_mean, in_std, out_mean, out_std)]
    _chk(ctx, load().fsi_set_surrogate(ctx, mlp_ctx, *[_ptr(a) for a in arrs], float(accept_tol)))


def fsi_get_structure_stats(ctx, reset=False):
    """(accepted, rejected, newton_solves, steps) of the coupled beam or shell."""
    st = (ctypes.c_int * 4)()
    _chk(ctx, load().fsi_get_structure_stats(ctx, st, int(bool(reset))))
    return tuple(st)


def lbm_check(ctx):
    _chk(ctx, load().lbm_check(ctx))


def lbm_stream(ctx) -> int:
    return load().lbm_stream(ctx)


def lbm_last_error(ctx) -> str:
    return load().lbm_last_error(ctx).decode(errors="replace")


def lbm_destroy(ctx):
    if ctx:
        load().lbm_destroy(ctx)


class Lattice:
    """Owner of one context: torch allocates the workspace, the library does the work.

    Arrays passed in or out may be numpy arrays (host) or torch tensors on the
    context's device; layouts follow include/kbc_lbm.h."""

    def __init__(self, lattice, nx, ny, nz, beta, storage=LBM_STORE_F32, collision=LBM_COLLIDE_KBC,
                 bc=(0, 0, 0, 0, 0, 0), face_velocity=None, max_links=0, max_vertices=0,
                 max_elements=0, stream=None, device="cuda", inlet_ramp_steps=0, multiphase=False):
        import torch

        self.torch = torch
        self.Q = lattice
        self.dim = 2 if lattice == 9 else 3
        self.shape = (nz, ny, nx)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        self.cfg = make_config(lattice, nx, ny, nz, beta, storage, collision, bc, face_velocity,
                               max_links, max_vertices, max_elements,
                               stream=self.stream.cuda_stream, inlet_ramp_steps=inlet_ramp_steps,
                               multiphase=multiphase)
        nbytes = lbm_workspace_size(self.cfg)
        # 256-byte alignment: torch's caching allocator returns 512-byte aligned blocks
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.ctx = lbm_create(self.cfg, self.workspace.data_ptr(), nbytes)

    @property
    def n(self):
        nz, ny, nx = self.shape
        return nx * ny * nz

    def _after_producers(self, *arrays):
        """Order the lattice stream after torch's current stream when an input
        is a CUDA tensor (the work that wrote it may still be queued there)."""
        if any(isinstance(a, self.torch.Tensor) and a.is_cuda for a in arrays):
            self.stream.wait_stream(self.torch.cuda.current_stream(self.device))

    def init_equilibrium(self, rho, u):
        self._after_producers(rho, u)
        lbm_init_equilibrium(self.ctx, rho, u)

    def set_populations(self, f):
        self._after_producers(f)
        lbm_set_populations(self.ctx, f)

    def get_populations(self, out=None):
        if out is None:
            out = np.zeros((self.Q,) + self.shape)
        lbm_get_populations(self.ctx, out)
        return out

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def step_graph(self, n, repeats):
        lbm_step_graph(self.ctx, n, repeats)

    def macros(self):
        rho = np.zeros(self.shape)
        u = np.zeros((self.dim,) + self.shape)
        lbm_get_macros(self.ctx, rho, u)
        return rho, u

    def set_multiphase(self, kappa, eos=LBM_EOS_PAPER, g=(0.0, 0.0, 0.0), kappa_w=0.0):
        lbm_set_multiphase(self.ctx, kappa, eos, g, kappa_w)

    def force_field(self):
        """Force F[3, nz, ny, nx] of the last multiphase step."""
        F = np.zeros((3,) + self.shape)
        lbm_get_force_field(self.ctx, F)
        return F

    def set_sweep_variant(self, variant):
        lbm_set_sweep_variant(self.ctx, variant)

    def couple_fine(self, fine, i0, j0):
        """Make `fine` (a Lattice on the same stream) the refined patch over the
        coarse cells from (i0, j0); this lattice's step then steps both."""
        nbytes = lbm_refine_workspace_size(self.ctx, fine.ctx)
        ws = self.torch.empty(nbytes, dtype=self.torch.uint8, device=self.device)
        lbm_refine_couple(self.ctx, fine.ctx, i0, j0, ws.data_ptr(), nbytes)
        self._refine_ws, self._refine_fine = ws, fine

    def check(self):
        lbm_check(self.ctx)

    def set_inlet_profile(self, face, u):
        lbm_set_inlet_profile(self.ctx, face, np.ascontiguousarray(u, dtype=np.float64))

    def set_geometry(self, verts, elems, elem_body, nbodies=None, vel=None, band_margin=0.0):
        verts = np.ascontiguousarray(verts, dtype=np.float64)
        elems = np.ascontiguousarray(elems, dtype=np.int32)
        elem_body = np.ascontiguousarray(elem_body, dtype=np.int32)
        vel = None if vel is None else np.ascontiguousarray(vel, dtype=np.float64)
        nb = int(nbodies if nbodies is not None else elem_body.max() + 1)
        self._nv, self._nb = verts.shape[0], nb
        lbm_set_geometry(self.ctx, nb, verts, verts.shape[0], elems, elems.shape[0], elem_body, vel,
                         band_margin)

    def update_surface(self, verts, vel=None):
        lbm_update_surface(self.ctx, np.ascontiguousarray(verts, dtype=np.float64),
                           None if vel is None else np.ascontiguousarray(vel, dtype=np.float64))

    def interface_force(self):
        vf = np.zeros((self._nv, 3))
        bf = np.zeros((self._nb, 3))
        lbm_get_interface_force(self.ctx, vf, bf)
        return vf, bf

    def set_traction_output(self, enable=True):
        lbm_set_traction_output(self.ctx, enable)

    def traction_force(self):
        """Stress-path surface forces of the last step: (vertex[nv,3], body[nb,3])."""
        vf = np.zeros((self._nv, 3))
        bf = np.zeros((self._nb, 3))
        lbm_get_traction_force(self.ctx, vf, bf)
        return vf, bf

    def boundary_info(self):
        info = np.zeros(4, dtype=np.int32)
        lbm_get_boundary_info(self.ctx, info)
        return info

    def close(self):
        if getattr(self, "ctx", None):
            lbm_destroy(self.ctx)
            self.ctx = None
            self._refine_ws = self._refine_fine = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def refined_pair(nx, ny, beta, fine_nx, fine_ny, i0, j0, storage=LBM_STORE_F32,
                 collision=LBM_COLLIDE_KBC, device="cuda"):
    """A periodic D2Q9 coarse lattice nx x ny and a fine patch fine_nx x fine_ny
    at half the spacing over the coarse cells from (i0, j0), on one stream,
    coupled (beta_f from nu_f = 2 nu_c).  Returns (coarse, fine)."""
    coarse = Lattice(9, nx, ny, 1, beta, storage=storage, collision=collision, device=device)
    fine = Lattice(9, fine_nx, fine_ny, 1, 1.0 / (2.0 / beta - 1.0), storage=storage,
                   collision=collision, bc=(LBM_BC_FREESTREAM,) * 4 + (0, 0),
                   stream=coarse.stream, device=device)
    coarse.couple_fine(fine, i0, j0)
    return coarse, fine


# ---------------------------------------------------------------- structure
def _fem_chk(f, st):
    if st != LBM_OK:
        raise LbmError(st, load().fem_last_error(f).decode(errors="replace"))


def fem_beam_create(cfg, workspace_ptr, nbytes):
    out = ctypes.c_void_p()
    st = load().fem_beam_create(ctypes.byref(cfg), workspace_ptr, nbytes, ctypes.byref(out))
    if st != LBM_OK:
        raise LbmError(st, load().fem_last_error(None).decode())
    return out.value


def fem_beam_step(f, F1):
    _fem_chk(f, load().fem_beam_step(f, _ptr(F1)))


def fem_beam_get_state(f, u, v, iterations):
    _fem_chk(f, load().fem_beam_get_state(f, _ptr(u), _ptr(v), _ptr(iterations)))


def fem_beam_set_state(f, u, v, F0):
    _fem_chk(f, load().fem_beam_set_state(f, _ptr(u), _ptr(v), _ptr(F0)))


def fem_destroy(f):
    if f:
        load().fem_destroy(f)


def fsi_couple(ctx, f, first_vertex):
    _chk(ctx, load().fsi_couple(ctx, f, int(first_vertex)))


def fsi_couple_span(ctx, f, first_vertex_z0, first_vertex_z1, z0, z1):
    """Quasi-2-D coupling of a beam to a D3Q27 lattice periodic in z (the
    flag polygon extruded over [z0, z1])."""
    _chk(ctx, load().fsi_couple_span(ctx, f, int(first_vertex_z0), int(first_vertex_z1),
                                     float(z0), float(z1)))


class Beam:
    """Owner of one GPU beam context (FP64 co-rotational beam, theta-scheme,
    Newton with relaxation lambda); torch allocates the workspace."""

    def __init__(self, X, EA, EI, rhoA, fixed, thickness=0.0, theta=0.5, lam=0.7, rtol=1e-10,
                 atol=1e-13, max_it=200, dt=1.0, stream=None, device="cuda", solve_fp64=False):
        import torch
        from ._abi_ext import fem_beam_config
        load()
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        self.fixed = np.ascontiguousarray(fixed, dtype=np.int32)
        self.nn = self.X.shape[0]
        self.stream = stream if stream is not None else torch.cuda.Stream(device=torch.device(device))
        c = fem_beam_config()
        c.nn = self.nn
        c.X = self.X.ctypes.data
        c.EA, c.EI, c.rhoA, c.thickness = EA, EI, rhoA, thickness
        c.fixed = self.fixed.ctypes.data
        c.theta, c.lambda_, c.rtol, c.atol, c.max_it, c.dt = theta, lam, rtol, atol, max_it, dt
        c.stream = self.stream.cuda_stream
        c.solve_fp64 = int(bool(solve_fp64))
        n = ctypes.c_size_t()
        st = load().fem_beam_workspace_size(ctypes.byref(c), ctypes.byref(n))
        if st != LBM_OK:
            raise LbmError(st, "fem_beam_workspace_size")
        self.workspace = torch.empty(n.value, dtype=torch.uint8, device=torch.device(device))
        self.ctx = fem_beam_create(c, self.workspace.data_ptr(), n.value)

    def step(self, F1):
        fem_beam_step(self.ctx, np.ascontiguousarray(F1, dtype=np.float64))

    def state(self):
        u = np.zeros(3 * self.nn)
        v = np.zeros(3 * self.nn)
        it = np.zeros(1, dtype=np.int32)
        fem_beam_get_state(self.ctx, u, v, it)
        return u, v, int(it[0])

    def set_state(self, u, v, F0):
        fem_beam_set_state(self.ctx, *(np.ascontiguousarray(a, dtype=np.float64) for a in (u, v, F0)))

    def close(self):
        if getattr(self, "ctx", None):
            fem_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- batches
def _batch_chk(b, st):
    if st != LBM_OK:
        raise LbmError(st, load().lbm_batch_last_error(b).decode(errors="replace"))


class Shell:
    """GPU co-rotational flat shell (fem_shell_*): nx x ny node grid with
    reference positions X[nn, 3], Dirichlet mask fixed[6 nn]; torch
    allocates the workspace."""

    def __init__(self, X, nx, ny, E, nu, h, rho, fixed, theta=0.5, lam=0.7, rtol=1e-10, atol=1e-13,
                 max_it=200, dt=1.0, max_cg=0, cg_rtol=0.0, stream=None, device="cuda"):
        import torch
        from ._abi_ext import fem_shell_config
        L = load()
        self.nx, self.ny = int(nx), int(ny)
        self.nn = self.nx * self.ny
        self.stream = stream if stream is not None else torch.cuda.Stream(device=torch.device(device))
        self._X = np.ascontiguousarray(X, dtype=np.float64)
        self._fixed = np.ascontiguousarray(fixed, dtype=np.int32)
        c = fem_shell_config()
        c.nx, c.ny = self.nx, self.ny
        c.X = self._X.ctypes.data
        c.E, c.nu, c.h, c.rho = E, nu, h, rho
        c.fixed = self._fixed.ctypes.data
        c.theta, c.lambda_, c.rtol, c.atol, c.max_it, c.dt = theta, lam, rtol, atol, max_it, dt
        c.max_cg, c.cg_rtol = max_cg, cg_rtol
        c.stream = self.stream.cuda_stream
        n = ctypes.c_size_t()
        if L.fem_shell_workspace_size(ctypes.byref(c), ctypes.byref(n)) != LBM_OK:
            raise LbmError(LBM_EINVAL, "fem_shell_workspace_size")
        self.workspace = torch.empty(n.value, dtype=torch.uint8, device=torch.device(device))
        out = ctypes.c_void_p()
        st = L.fem_shell_create(ctypes.byref(c), self.workspace.data_ptr(), n.value, ctypes.byref(out))
        if st != LBM_OK:
            raise LbmError(st, L.fem_shell_last_error(None).decode())
        self.ctx = out.value

    def _chk(self, st):
        if st != LBM_OK:
            raise LbmError(st, load().fem_shell_last_error(self.ctx).decode(errors="replace"))

    def step(self, F1):
        F1 = np.ascontiguousarray(F1, dtype=np.float64).reshape(-1)
        self._chk(load().fem_shell_step(self.ctx, _ptr(F1)))
        self._F1 = F1  # the copy is asynchronous

    def set_state(self, u=None, R=None, v=None, F0=None):
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (u, R, v, F0)]
        self._chk(load().fem_shell_set_state(self.ctx, *[_ptr(a) for a in arrs]))

    def state(self):
        u = np.zeros((self.nn, 3))
        R = np.zeros((self.nn, 3, 3))
        v = np.zeros((self.nn, 6))
        it = np.zeros(2, dtype=np.int32)
        self._chk(load().fem_shell_get_state(self.ctx, _ptr(u), _ptr(R), _ptr(v), _ptr(it)))
        return u, R, v, (int(it[0]), int(it[1]))

    def close(self):
        if getattr(self, "ctx", None):
            load().fem_shell_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SvkSolid:
    """GPU St Venant-Kirchhoff continuum with Q2 elements (fem_svk_*): nodes
    X[nn, dim], elements conn[ne, 3^dim] (local node i + 3 j (+ 9 k)),
    Dirichlet mask fixed[nn * dim]; torch allocates the workspace."""

    def __init__(self, X, conn, E, nu, rho, fixed, theta=0.5, lam=0.7, rtol=1e-10, atol=1e-13,
                 max_it=500, dt=1.0, max_cg=0, cg_rtol=0.0, solve_fp64=False, stream=None,
                 device="cuda"):
        import torch
        from ._abi_ext import fem_svk_config
        L = load()
        self._X = np.ascontiguousarray(X, dtype=np.float64)
        self.nn, self.dim = self._X.shape
        self._conn = np.ascontiguousarray(conn, dtype=np.int32)
        self._fixed = np.ascontiguousarray(fixed, dtype=np.int32).reshape(-1)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=torch.device(device))
        c = fem_svk_config()
        c.dim, c.nn, c.ne = self.dim, self.nn, self._conn.shape[0]
        c.X, c.conn, c.fixed = self._X.ctypes.data, self._conn.ctypes.data, self._fixed.ctypes.data
        c.E, c.nu, c.rho = E, nu, rho
        c.theta, c.lambda_, c.rtol, c.atol, c.max_it, c.dt = theta, lam, rtol, atol, max_it, dt
        c.max_cg, c.cg_rtol = max_cg, cg_rtol
        c.stream = self.stream.cuda_stream
        c.solve_fp64 = int(bool(solve_fp64))
        n = ctypes.c_size_t()
        if L.fem_svk_workspace_size(ctypes.byref(c), ctypes.byref(n)) != LBM_OK:
            raise LbmError(LBM_EINVAL, "fem_svk_workspace_size")
        self.workspace = torch.empty(n.value, dtype=torch.uint8, device=torch.device(device))
        out = ctypes.c_void_p()
        st = L.fem_svk_create(ctypes.byref(c), self.workspace.data_ptr(), n.value, ctypes.byref(out))
        if st != LBM_OK:
            raise LbmError(st, L.fem_svk_last_error(None).decode())
        self.ctx = out.value

    def _chk(self, st):
        if st != LBM_OK:
            raise LbmError(st, load().fem_svk_last_error(self.ctx).decode(errors="replace"))

    def step(self, F1):
        F1 = np.ascontiguousarray(F1, dtype=np.float64).reshape(-1)
        self._chk(load().fem_svk_step(self.ctx, _ptr(F1)))
        self._F1 = F1  # the copy is asynchronous

    def body_load(self, b):
        F = np.zeros(self.nn * self.dim)
        self._chk(load().fem_svk_body_load(self.ctx, _ptr(np.ascontiguousarray(b, dtype=np.float64)),
                                           _ptr(F)))
        return F

    def set_state(self, u=None, v=None, F0=None):
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
                for a in (u, v, F0)]
        self._chk(load().fem_svk_set_state(self.ctx, *[_ptr(a) for a in arrs]))

    def state(self):
        u = np.zeros(self.nn * self.dim)
        v = np.zeros(self.nn * self.dim)
        it = np.zeros(2, dtype=np.int32)
        self._chk(load().fem_svk_get_state(self.ctx, _ptr(u), _ptr(v), _ptr(it)))
        return u, v, (int(it[0]), int(it[1]))

    def close(self):
        if getattr(self, "ctx", None):
            load().fem_svk_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many Lattice objects advanced with one launch per phase (lbm_batch_*).

    The member lattices must share lattice type, storage and stream; torch
    allocates the batch workspace."""

    def __init__(self, lattices):
        import torch
        self.lattices = list(lattices)
        n = len(self.lattices)
        self._arr = (ctypes.c_void_p * n)(*[L.ctx for L in self.lattices])
        nb = ctypes.c_size_t()
        _batch_chk(None, load().lbm_batch_workspace_size(self._arr, n, ctypes.byref(nb)))
        self.workspace = torch.empty(nb.value, dtype=torch.uint8, device=self.lattices[0].device)
        out = ctypes.c_void_p()
        st = load().lbm_batch_create(self._arr, n, self.workspace.data_ptr(), nb.value, ctypes.byref(out))
        if st != LBM_OK:
            raise LbmError(st, load().lbm_batch_last_error(None).decode())
        self.b = out.value
        self.stream = self.lattices[0].stream

    def step(self, n=1):
        _batch_chk(self.b, load().lbm_batch_step(self.b, int(n)))

    def step_graph(self, n, repeats):
        _batch_chk(self.b, load().lbm_batch_step_graph(self.b, int(n), int(repeats)))

    def set_tuning(self, rows_per_tile, ctas_per_sm):
        _batch_chk(self.b, load().lbm_batch_set_tuning(self.b, int(rows_per_tile), int(ctas_per_sm)))

    def size_bucket(self):
        """Autotuner cache key: lattice, storage, member count and the total
        node count rounded to a power of two."""
        nodes = sum(int(np.prod(L.shape)) for L in self.lattices)
        L0 = self.lattices[0]
        return f"Q{L0.Q}-s{int(L0.cfg.storage)}-m{len(self.lattices)}-n2^{int(round(np.log2(max(nodes, 1))))}"

    def autotune(self, steps=4, cache=None):
        """Pick the sweep's tile height and resident CTAs per SM by timing
        (lbm_batch_autotune; the timed steps advance the batch).  With a JSON
        cache path, a size bucket tuned before is applied without timing and a
        new result is added to the file.  Returns (rows, ctas, us_per_step or
        None when taken from the cache)."""
        import json
        import os
        key = self.size_bucket()
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as fh:
                table = json.load(fh)
            if key in table:
                rows, ctas = table[key]["rows_per_tile"], table[key]["ctas_per_sm"]
                self.set_tuning(rows, ctas)
                return rows, ctas, None
        r, c, us = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        _batch_chk(self.b, load().lbm_batch_autotune(self.b, int(steps), ctypes.byref(r), ctypes.byref(c),
                                                      ctypes.byref(us)))
        if cache:
            table[key] = {"rows_per_tile": r.value, "ctas_per_sm": c.value, "us_per_step": us.value}
            tmp = cache + ".tmp"
            with open(tmp, "w") as fh:
                json.dump(table, fh, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return r.value, c.value, us.value

    def close(self):
        if getattr(self, "b", None):
            load().lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- MLP surrogate
class Mlp:
    """GPU MLP (BF16 tensor-core GEMMs, FP32 accumulation, Adam); torch
    allocates the workspace."""

    def __init__(self, dims, max_batch=256, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None,
                 device="cuda"):
        import torch
        from ._abi_ext import mlp_config
        L = load()
        self.dims = list(dims)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=torch.device(device))
        c = mlp_config()
        c.n_layers = len(dims) - 1
        for k, d in enumerate(dims):
            c.dims[k] = d
        c.max_batch, c.lr, c.beta1, c.beta2, c.eps = max_batch, lr, beta1, beta2, eps
        c.stream = self.stream.cuda_stream
        n = ctypes.c_size_t()
        st = L.mlp_workspace_size(ctypes.byref(c), ctypes.byref(n))
        if st != LBM_OK:
            raise LbmError(st, "mlp_workspace_size")
        self.workspace = torch.empty(n.value, dtype=torch.uint8, device=torch.device(device))
        out = ctypes.c_void_p()
        st = L.mlp_create(ctypes.byref(c), self.workspace.data_ptr(), n.value, ctypes.byref(out))
        if st != LBM_OK:
            raise LbmError(st, L.mlp_last_error(None).decode())
        self.ctx = out.value
        self.nparam = L.mlp_param_count(self.ctx)

    def _chk(self, st):
        if st != LBM_OK:
            raise LbmError(st, load().mlp_last_error(self.ctx).decode(errors="replace"))

    def set_params(self, p):
        p32 = np.ascontiguousarray(p, dtype=np.float32)  # held until the copy returns
        self._chk(load().mlp_set_params(self.ctx, _ptr(p32)))

    def params(self):
        p = np.zeros(self.nparam, dtype=np.float32)
        self._chk(load().mlp_get_params(self.ctx, _ptr(p)))
        return p

    def forward(self, X):
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.zeros((X.shape[0], self.dims[-1]), dtype=np.float32)
        self._chk(load().mlp_forward(self.ctx, _ptr(X), X.shape[0], _ptr(Y)))
        return Y

    def gradients(self, X, Y):
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.ascontiguousarray(Y, dtype=np.float32)
        g = np.zeros(self.nparam, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        self._chk(load().mlp_gradients(self.ctx, _ptr(X), _ptr(Y), X.shape[0], _ptr(g), _ptr(loss)))
        return g, float(loss[0])

    def set_learning_rate(self, lr):
        self._chk(load().mlp_set_learning_rate(self.ctx, float(lr)))

    def train_step(self, X, Y, want_loss=False):
        """X, Y: numpy arrays or device tensors (FP32, row-major)."""
        if isinstance(X, np.ndarray):
            X = np.ascontiguousarray(X, dtype=np.float32)
        if isinstance(Y, np.ndarray):
            Y = np.ascontiguousarray(Y, dtype=np.float32)
        for a in (X, Y):
            if not isinstance(a, np.ndarray) and (str(a.dtype) != "torch.float32" or not a.is_contiguous()):
                raise ValueError("device inputs must be contiguous float32 tensors")
        loss = np.zeros(1, dtype=np.float32) if want_loss else None
        self._chk(load().mlp_train_step(self.ctx, _ptr(X), _ptr(Y), X.shape[0], _ptr(loss)))
        return float(loss[0]) if want_loss else None

    def close(self):
        if getattr(self, "ctx", None):
            load().mlp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
