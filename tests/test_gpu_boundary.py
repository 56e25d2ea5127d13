"""GPU-vs-oracle parity of the boundary treatment through the C ABI: Grad
walls, inlet/outlet, immersed rigid and moving bodies (cut links, fresh
nodes) and the FP64 momentum-exchange force.

Tolerances: velocity max |u_gpu - u_or| / max |u_or| <= 1e-5 on laminar cases;
per-body force |F_gpu - F_or| / |F_or| <= 1e-4 and per-vertex force error
<= 1e-4 of the largest vertex force."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1710_02375_gb300 import synth

pytestmark = pytest.mark.gpu
WALL, INLET, OUTLET, FREE = 1, 2, 3, 4


def lattice(lat, shape, beta, **kw):
    from paper_1710_02375_gb300.lbm import Lattice
    nz, ny, nx = shape
    return Lattice(lat, nx, ny, nz, beta, **kw)


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def test_couette_face_walls():
    nx, ny, U, beta, steps = 6, 12, 0.02, 0.8, 400
    bc = (0, 0, WALL, WALL, 0, 0)
    fu = np.zeros((6, 3))
    fu[3, 0] = U
    L = lattice(9, (1, ny, nx), beta, bc=bc, face_velocity=fu)
    rho0, u0 = np.ones((1, ny, nx)), np.zeros((2, 1, ny, nx))
    L.init_equilibrium(rho0, u0)
    L.step(steps)
    L.check()
    _, ug = L.macros()
    f = orc.init_equilibrium(9, rho0, u0)
    for _ in range(steps):
        f, _, _, _ = orc.step_bc(9, beta, f, bc=bc, face_u=fu)
    _, uo = orc.macros(9, f)
    assert rel(ug, uo[:2]) <= 1e-5
    assert L.boundary_info()[0] == 2 * nx


def slabs(nx, ny, y_lo, y_hi, U):
    xa, ea = synth.rect_polygon(-3.0, 0.0, nx + 2.0, y_lo)
    xb, eb = synth.rect_polygon(-3.0, y_hi, nx + 2.0, float(ny))
    x = np.concatenate([xa, xb])
    e = np.concatenate([ea, eb + len(xa)])
    v = np.zeros_like(x)
    v[len(xa):, 0] = U
    body = np.array([0] * len(ea) + [1] * len(eb), dtype=np.int32)
    return x, v, e, body


def test_couette_immersed_walls_force():
    nx, ny, U, beta, steps = 5, 16, 0.01, 0.7, 400
    x, v, e, body = slabs(nx, ny, 2.3, 13.6, U)
    L = lattice(9, (1, ny, nx), beta, max_links=400, max_vertices=16, max_elements=16)
    L.set_geometry(x, e, body, vel=v)
    rho0, u0 = np.ones((1, ny, nx)), np.zeros((2, 1, ny, nx))
    L.init_equilibrium(rho0, u0)
    L.step(steps)
    L.check()
    _, ug = L.macros()
    vf_g, bf_g = L.interface_force()
    surf = orc.Surface(x, v, e, body)
    f = orc.init_equilibrium(9, rho0, u0)
    solid = orc.solid_mask((1, ny, nx), surf)
    for _ in range(steps):
        f, vf_o, bf_o, _ = orc.step_bc(9, beta, f, bc=(0,) * 6, surf=surf, solid=solid)
    _, uo = orc.macros(9, f)
    uo[:, solid.astype(bool)] = 0
    assert rel(ug, uo[:2]) <= 1e-5
    for b in range(2):
        assert np.linalg.norm(bf_g[b] - bf_o[b]) <= 1e-4 * np.linalg.norm(bf_o[b])
    assert np.max(np.abs(vf_g - vf_o)) <= 1e-4 * np.max(np.abs(vf_o))


def c1_setup(with_flag=False):
    nx, ny = 220, 41
    u_max, Re, D = 0.05, 100.0, 10.0
    nu = (2.0 / 3.0) * u_max * D / Re
    beta = 1.0 / (6 * nu + 1)
    prof = synth.parabolic_profile(ny, u_max, noise=1e-4, seed=0)
    x, e, body, _ = synth.cylinder_flag_2d(with_flag=with_flag)
    return nx, ny, beta, prof, x, e, body


def run_c1(with_flag, steps, ramp=1000):
    """Oracle run of the C1 channel; returns (u, solid, vertex forces, body forces)."""
    nx, ny, beta, prof, x, e, body = c1_setup(with_flag)
    bc = (INLET, OUTLET, WALL, WALL, 0, 0)
    surf = orc.Surface(x, np.zeros_like(x), e, body)
    solid = orc.solid_mask((1, ny, nx), surf)
    f = orc.init_equilibrium(9, np.ones((1, ny, nx)), np.zeros((2, 1, ny, nx)))
    for t in range(steps):
        s = 0.5 * (1 - np.cos(np.pi * t / ramp)) if t < ramp else 1.0
        f, vf_o, bf_o, _ = orc.step_bc(9, beta, f, bc=bc, inlet={0: prof}, inlet_scale=s, surf=surf,
                                       solid=solid)
    _, uo = orc.macros(9, f)
    uo[:, solid.astype(bool)] = 0
    return uo[:2], solid, vf_o, bf_o


def gpu_c1(with_flag, steps, ramp=1000):
    nx, ny, beta, prof, x, e, body = c1_setup(with_flag)
    bc = (INLET, OUTLET, WALL, WALL, 0, 0)
    L = lattice(9, (1, ny, nx), beta, bc=bc, max_links=4000, max_vertices=200, max_elements=200,
                inlet_ramp_steps=ramp)
    L.set_inlet_profile(0, prof)
    L.set_geometry(x, e, body)
    L.init_equilibrium(np.ones((1, ny, nx)), np.zeros((2, 1, ny, nx)))
    L.step(steps)
    L.check()
    _, ug = L.macros()
    vf, bf = L.interface_force()
    return ug, vf, bf, body


@pytest.mark.parametrize("with_flag", [False, True])
def test_channel_cylinder_c1_geometry_700_steps(with_flag):
    """The C1 channel (220 x 41, parabolic inflow u_max = 0.05 with 1e-4 static
    noise, Re = 100 on D = 10, 1000-step inflow ramp) around the rigid cylinder
    (and flag): 700 steps at the FP32 bounds."""
    ug, vf_g, bf_g, body = gpu_c1(with_flag, 700)
    uo, solid, vf_o, bf_o = run_c1(with_flag, 700)
    assert rel(ug, uo) <= 1e-5
    for b in range(body.max() + 1):
        assert np.linalg.norm(bf_g[b] - bf_o[b]) <= 1e-4 * np.linalg.norm(bf_o[b])
    assert np.max(np.abs(vf_g - vf_o)) <= 1e-4 * np.max(np.abs(vf_o))


@pytest.mark.parametrize("with_flag", [False, True])
def test_channel_cylinder_c1_1000_steps(with_flag):
    """The C1 channel over the whole 1000-step inflow ramp at the plain FP32
    bounds.  (With gamma unbounded, gamma reached 6.7 at the outlet nodes next
    to the walls near step 830 and grew round-off differences 1e5-fold; held
    in [0, 2/beta] the oracle's own 1e-8 perturbation stays at 5e-10.)"""
    ug, vf_g, bf_g, body = gpu_c1(with_flag, 1000)
    uo, solid, vf_o, bf_o = run_c1(with_flag, 1000)
    assert rel(ug, uo) <= 1e-5, rel(ug, uo)
    for b in range(body.max() + 1):
        assert np.linalg.norm(bf_g[b] - bf_o[b]) <= 1e-4 * np.linalg.norm(bf_o[b])
    assert np.max(np.abs(vf_g - vf_o)) <= 1e-4 * np.max(np.abs(vf_o))


def test_sphere_channel_d3q27():
    """Steady flow past a sphere (D = 8.4, Re = 29) in a D3Q27 channel with an
    inlet, an outlet, face walls and free-stream faces, 1000 steps."""
    nx, ny, nz = 36, 20, 18
    beta, steps = 0.95, 1000
    bc = (INLET, OUTLET, WALL, WALL, FREE, FREE)
    fu = np.zeros((6, 3))
    fu[0, 0] = 0.03
    fu[4, 0] = fu[5, 0] = 0.03
    x, e = synth.icosphere((12.3, 9.6, 8.7), 4.2, level=2)
    body = np.zeros(len(e), np.int32)
    L = lattice(27, (nz, ny, nx), beta, bc=bc, face_velocity=fu, max_links=20000,
                max_vertices=len(x), max_elements=len(e), inlet_ramp_steps=50)
    L.set_geometry(x, e, body)
    rho0, u0 = np.ones((nz, ny, nx)), np.zeros((3, nz, ny, nx))
    L.init_equilibrium(rho0, u0)
    L.step(steps)
    L.check()
    _, ug = L.macros()
    vf_g, bf_g = L.interface_force()
    surf = orc.Surface(x, np.zeros_like(x), e, body)
    solid = orc.solid_mask((nz, ny, nx), surf)
    f = orc.init_equilibrium(27, rho0, u0)
    for t in range(steps):
        s = 0.5 * (1 - np.cos(np.pi * t / 50)) if t < 50 else 1.0
        f, vf_o, bf_o, _ = orc.step_bc(27, beta, f, bc=bc, face_u=fu, inlet_scale=s, surf=surf,
                                       solid=solid)
    _, uo = orc.macros(27, f)
    uo[:, solid.astype(bool)] = 0
    assert rel(ug, uo) <= 1e-5
    assert np.linalg.norm(bf_g[0] - bf_o[0]) <= 1e-4 * np.linalg.norm(bf_o[0])
    assert np.max(np.abs(vf_g - vf_o)) <= 1e-4 * np.max(np.abs(vf_o))


def test_moving_cylinder_fresh_nodes():
    """A cylinder translating through a periodic box: the surface moves every
    step, uncovered nodes are initialised from their neighbours."""
    nx, ny = 48, 32
    beta, steps, U = 0.9, 150, 0.03
    x0, e = synth.circle_polygon(14.3, 15.7, 5.2, 48)
    body = np.zeros(len(e), np.int32)
    vel = np.zeros_like(x0)
    vel[:, 0] = U
    L = lattice(9, (1, ny, nx), beta, max_links=2000, max_vertices=len(x0), max_elements=len(e))
    L.set_geometry(x0, e, body, vel=vel, band_margin=U * steps + 1)
    rho0, u0 = np.ones((1, ny, nx)), np.zeros((2, 1, ny, nx))
    L.init_equilibrium(rho0, u0)
    f = orc.init_equilibrium(9, rho0, u0)
    surf = orc.Surface(x0, vel, e, body)
    solid = orc.solid_mask((1, ny, nx), surf)
    nfresh = 0
    for t in range(steps):
        L.step(1)
        f, vf_o, bf_o, _ = orc.step_bc(9, beta, f, bc=(0,) * 6, surf=surf, solid=solid)
        xt = x0 + vel * (t + 1)
        L.update_surface(xt, vel)
        surf = orc.Surface(xt, vel, e, body)
        new_solid = orc.solid_mask((1, ny, nx), surf)
        nfresh += orc.fresh_init(9, f, solid, new_solid, surf, periodic=(1, 1, 1))
        solid = new_solid
    L.check()
    assert nfresh > 0
    _, ug = L.macros()
    _, uo = orc.macros(9, f)
    uo[:, solid.astype(bool)] = 0
    assert rel(ug, uo[:2]) <= 1e-5


def test_graph_replay_matches_direct_stepping():
    """lbm_step_graph (CUDA graph of n steps) gives the populations lbm_step gives."""
    nx, ny, beta, prof, x, e, body = c1_setup(True)
    bc = (INLET, OUTLET, WALL, WALL, 0, 0)
    out = []
    for use_graph in (False, True):
        L = lattice(9, (1, ny, nx), beta, bc=bc, max_links=4000, max_vertices=200,
                    max_elements=200, inlet_ramp_steps=50)
        L.set_inlet_profile(0, prof)
        L.set_geometry(x, e, body)
        L.init_equilibrium(np.ones((1, ny, nx)), np.zeros((2, 1, ny, nx)))
        if use_graph:
            L.step_graph(10, 12)
        else:
            L.step(120)
        L.check()
        out.append(L.get_populations())
        assert L.boundary_info()[3] == 120  # ramp clock advanced once per step
        L.close()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("storage,tol", [(0, 3e-5), (3, 1e-7)])
def test_stress_traction_matches_oracle(storage, tol):
    """Stress-path traction (lbm_set_traction_output): immersed Couette walls
    (the exact wall shear rho nu U / H) and the C1 cylinder with a rigid flag
    after 300 steps, against the oracle's boundary-node stresses and element
    quadrature; per vertex <= tol of the largest vertex force, per body <= tol
    of the body force (C1) or of the vertex scale (Couette).  Measured with
    FP32 storage: Couette 5.5e-6, C1 body 1.4e-6, C1 vertex 1.6e-7; with FP64
    storage (D2Q9; limited by the FP32 link data of the library): 2.3e-8,
    1.1e-9, 1.2e-10."""
    # Couette
    nx, ny, U, beta, steps = 5, 16, 0.01, 0.7, 400
    x, v, e, body = slabs(nx, ny, 2.3, 13.6, U)
    L = lattice(9, (1, ny, nx), beta, storage=storage, max_links=400, max_vertices=16,
                max_elements=16)
    L.set_geometry(x, e, body, vel=v)
    L.set_traction_output(True)
    rho0, u0 = np.ones((1, ny, nx)), np.zeros((2, 1, ny, nx))
    L.init_equilibrium(rho0, u0)
    L.step(steps)
    L.check()
    tv_g, tb_g = L.traction_force()
    surf = orc.Surface(x, v, e, body)
    f = orc.init_equilibrium(9, rho0, u0)
    solid = orc.solid_mask((1, ny, nx), surf)
    for _ in range(steps):
        f, _, _, _, sig = orc.step_bc(9, beta, f, bc=(0,) * 6, surf=surf, solid=solid,
                                      want_sigma=True)
    tv_o, tb_o, _ = orc.traction(surf, sig)
    # the slabs' totals cancel (their far faces lie outside the periodic box
    # and see the same stress), so they are compared on the vertex-force scale
    scale = np.max(np.abs(tv_o))
    e_couette = max(np.max(np.abs(tb_g - tb_o)), np.max(np.abs(tv_g - tv_o))) / scale
    assert scale > 0 and e_couette <= tol, (tb_g, tb_o)
    # C1 geometry, rigid flag
    nx, ny, beta, prof, x, e, body = c1_setup(True)
    if storage == 3:  # the library keeps inlet profiles in FP32: both sides take that array
        prof = prof.astype(np.float32).astype(np.float64)
    bc = (INLET, OUTLET, WALL, WALL, 0, 0)
    steps = 300
    L = lattice(9, (1, ny, nx), beta, storage=storage, bc=bc, max_links=4000, max_vertices=200,
                max_elements=200, inlet_ramp_steps=1000)
    L.set_inlet_profile(0, prof)
    L.set_geometry(x, e, body)
    L.set_traction_output(True)
    L.init_equilibrium(np.ones((1, ny, nx)), np.zeros((2, 1, ny, nx)))
    L.step(steps)
    L.check()
    tv_g, tb_g = L.traction_force()
    _, mb_g = L.interface_force()
    surf = orc.Surface(x, np.zeros_like(x), e, body)
    solid = orc.solid_mask((1, ny, nx), surf)
    f = orc.init_equilibrium(9, np.ones((1, ny, nx)), np.zeros((2, 1, ny, nx)))
    for t in range(steps):
        s = 0.5 * (1 - np.cos(np.pi * t / 1000))
        f, _, _, _, sig = orc.step_bc(9, beta, f, bc=bc, inlet={0: prof}, inlet_scale=s, surf=surf,
                                      solid=solid, want_sigma=True)
    tv_o, tb_o, _ = orc.traction(surf, sig)
    e_body = max(np.linalg.norm(tb_g[b] - tb_o[b]) / np.linalg.norm(tb_o[b]) for b in range(2))
    e_vert = np.max(np.abs(tv_g - tv_o)) / np.max(np.abs(tv_o))
    print(f"traction storage {storage}: Couette {e_couette:.2e}, C1 body {e_body:.2e}, "
          f"C1 vertex {e_vert:.2e}")
    assert e_body <= tol and e_vert <= tol, (e_body, e_vert)
    print("TRACTION vs momentum exchange (C1, 300 steps):", tb_g[:, :2].tolist(), mb_g[:, :2].tolist())

