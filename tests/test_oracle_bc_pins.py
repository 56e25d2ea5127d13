"""Pins of the oracle's boundary treatment (section "Fluid boundary
conditions": Grad's approximation, Eq. grad, with target values) and of its
cut-link geometry, against closed forms and analytic intersections."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1710_02375_gb300 import synth

WALL, INLET, OUTLET = 1, 2, 3


def run_bc(lat, f, beta, steps, **kw):
    for _ in range(steps):
        f, vf, bf, _ = orc.step_bc(lat, beta, f, **kw)
    return f, vf, bf


def test_couette_face_walls_linear_profile():
    """Top face wall moving with U, bottom at rest, walls half a cell outside
    the faces: the steady profile is u_x = U (y + 1/2) / H."""
    nx, ny, U, beta = 4, 12, 0.02, 0.5
    bc = (0, 0, WALL, WALL, 0, 0)
    fu = np.zeros((6, 3))
    fu[3, 0] = U
    f = orc.init_equilibrium(9, np.ones((1, ny, nx)), np.zeros((2, 1, ny, nx)))
    f, _, _ = run_bc(9, f, beta, 3000, bc=bc, face_u=fu)
    _, u = orc.macros(9, f)
    y = np.arange(ny)
    exact = U * (y + 0.5) / ny
    assert np.max(np.abs(u[0, 0, :, 1] - exact)) < 1e-6 * U
    assert np.max(np.abs(u[1])) < 1e-9


def slab_surface(nx, y_lo, y_hi, ny, U):
    """Two x-invariant slabs: y in [0, y_lo] at rest and y in [y_hi, ny] moving
    with U along x (periodic box; node y sits at y + 1/2)."""
    xa, ea = synth.rect_polygon(-3.0, 0.0, nx + 2.0, y_lo)
    xb, eb = synth.rect_polygon(-3.0, y_hi, nx + 2.0, float(ny))
    x = np.concatenate([xa, xb])
    e = np.concatenate([ea, eb + len(xa)])
    v = np.zeros_like(x)
    v[len(xa):, 0] = U
    body = np.array([0] * len(ea) + [1] * len(eb), dtype=np.int32)
    return orc.Surface(x, v, e, body)


@pytest.mark.parametrize("y_lo,y_hi", [(2.25, 13.75), (2.5, 13.5), (2.75, 13.3)])
def test_couette_immersed_walls_off_lattice(y_lo, y_hi):
    """Immersed walls at off-lattice positions: linear steady profile and the
    wall shear force rho nu U / H per unit length (momentum exchange)."""
    nx, ny, U = 3, 16, 0.01
    nu = 1.0 / 6.0
    beta = 1.0 / (6 * nu + 1)
    surf = slab_surface(nx, y_lo, y_hi, ny, U)
    f = orc.init_equilibrium(9, np.ones((1, ny, nx)), np.zeros((2, 1, ny, nx)))
    f, vf, bf = run_bc(9, f, beta, 3000, bc=(0,) * 6, surf=surf)
    rho, u = orc.macros(9, f)
    H = y_hi - y_lo
    solid = orc.solid_mask((1, ny, nx), surf)[0, :, 1].astype(bool)
    y = np.arange(ny) + 0.5  # cell-centred node positions
    exact = U * (y - y_lo) / H
    err = np.max(np.abs(u[0, 0, :, 1] - exact)[~solid])
    assert err < 1e-3 * U, err
    tau = nu * U / H
    # per unit length along x: fluid drags the moving top wall back, the bottom forward
    assert abs(bf[1, 0] / nx + tau) < 2e-2 * tau, (bf, tau)
    assert abs(bf[0, 0] / nx - tau) < 2e-2 * tau, (bf, tau)


def poiseuille_error(H, nu=1.0 / 6.0, U=0.02):
    beta = 1.0 / (6 * nu + 1)
    nx, ny = 2 * H, H
    y = np.arange(ny)
    prof = np.zeros((3, ny))
    prof[0] = 4 * U * (y + 0.5) * (H - y - 0.5) / H ** 2
    bc = (INLET, OUTLET, WALL, WALL, 0, 0)
    f = orc.init_equilibrium(9, np.ones((1, ny, nx)), np.zeros((2, 1, ny, nx)))
    for t in range(int(4 * H * H / nu) + 400):
        ramp = 0.5 * (1 - np.cos(np.pi * min(t, 200) / 200))
        f, _, _, _ = orc.step_bc(9, beta, f, bc=bc, inlet={0: prof}, inlet_scale=ramp)
    _, u = orc.macros(9, f)
    return (np.max(np.abs(u[0, 0, :, nx // 2] - prof[0])) / U,
            np.max(np.abs(u[1, 0, :, nx // 2])) / U)


def test_poiseuille_inlet_outlet_parabola():
    """Parabolic inflow between face walls relaxes to the same parabola; the
    mid-channel error falls at (at least) second order with the height."""
    e8, v8 = poiseuille_error(8)
    e16, v16 = poiseuille_error(16)
    assert e16 < 1e-2
    assert e8 / e16 > 3.5
    assert v16 < 1e-3


def test_circle_links_match_analytic_intersection():
    """q of every cut link against the exact line/circle crossing (within the
    polygon's sagitta), solid mask against the exact disk away from the rim."""
    cx, cy, R, n = 10.3, 9.7, 4.6, 512
    x, e = synth.circle_polygon(cx, cy, R, n)
    surf = orc.Surface(x, np.zeros_like(x), e, np.zeros(len(e), np.int32))
    shape = (1, 20, 21)
    solid = orc.solid_mask(shape, surf)[0]
    Y, X = np.mgrid[0:20, 0:21] + 0.5
    d = np.hypot(X - cx, Y - cy)
    sag = R * (1 - np.cos(np.pi / n))
    far = np.abs(d - R) > 2 * sag
    assert np.array_equal(solid[far], (d < R)[far])
    L = orc.links(9, shape, surf)
    c, _ = orc.lattice(9)
    assert len(L["q"]) > 0 and np.all(L["elem"] >= 0)
    for k in range(len(L["q"])):
        node, i = L["node"][k], L["dir"][k]
        p = np.array([node % 21, node // 21], dtype=float) + 0.5
        dvec = -c[i, :2].astype(float)
        # |p + s d - c|^2 = R^2, smallest root in (0, 1]
        a = dvec @ dvec
        b = 2 * dvec @ (p - [cx, cy])
        cc = (p - [cx, cy]) @ (p - [cx, cy]) - R * R
        s = (-b - np.sqrt(b * b - 4 * a * cc)) / (2 * a)
        assert abs(L["q"][k] - s) < 4 * sag, (k, L["q"][k], s)


def test_sphere_links_and_mask_3d():
    cen, R = (6.4, 6.1, 5.8), 3.7
    x, e = synth.icosphere(cen, R, level=3)
    surf = orc.Surface(x, np.zeros_like(x), e, np.zeros(len(e), np.int32))
    shape = (12, 13, 13)
    solid = orc.solid_mask(shape, surf)
    Z, Y, X = np.mgrid[0:12, 0:13, 0:13] + 0.5
    d = np.sqrt((X - cen[0]) ** 2 + (Y - cen[1]) ** 2 + (Z - cen[2]) ** 2)
    tol = 0.08  # mesh deviation from the sphere at level 3
    far = np.abs(d - R) > tol
    assert np.array_equal(solid[far].astype(bool), (d < R)[far])
    L = orc.links(27, shape, surf)
    c, _ = orc.lattice(27)
    assert np.all(L["elem"] >= 0)
    for k in range(0, len(L["q"]), 7):
        node, i = L["node"][k], L["dir"][k]
        p = np.array([node % 13, (node // 13) % 13, node // 169], dtype=float) + 0.5
        dvec = -c[i].astype(float)
        a = dvec @ dvec
        b = 2 * dvec @ (p - cen)
        cc = (p - cen) @ (p - cen) - R * R
        disc = b * b - 4 * a * cc
        s = (-b - np.sqrt(max(disc, 0))) / (2 * a)
        assert abs(L["q"][k] - s) * np.sqrt(a) < 2 * tol


@pytest.mark.parametrize("y_lo,y_hi", [(2.25, 13.75), (2.75, 13.3)])
def test_stress_traction_couette_wall_shear(y_lo, y_hi):
    """The stress path (sigma_f = -p I - (1 - beta) Pi^(1) at the boundary
    nodes, t = sigma n on the wall elements): steady Couette gives the wall
    shear stress rho nu U / H exactly on both walls (the fluid drags the
    resting wall forward and the moving wall back) and no normal traction."""
    nx, ny, U = 3, 16, 0.01
    nu = 1.0 / 6.0
    beta = 1.0 / (6 * nu + 1)
    surf = slab_surface(nx, y_lo, y_hi, ny, U)
    f = orc.init_equilibrium(9, np.ones((1, ny, nx)), np.zeros((2, 1, ny, nx)))
    for _ in range(3000):
        f, _, _, _, sig = orc.step_bc(9, beta, f, bc=(0,) * 6, surf=surf, want_sigma=True)
    _, _, ef = orc.traction(surf, sig)
    tau = nu * U / (y_hi - y_lo)
    seen = 0
    for k, el in enumerate(surf.e):
        P = surf.x[el]
        if abs(P[0, 1] - P[1, 1]) > 0 or not (0 < P[0, 1] < ny):
            continue
        L = abs(P[1, 0] - P[0, 0])
        want = tau if P[0, 1] == y_lo else -tau
        assert abs(ef[k, 0] / L - want) <= 1e-9 * tau, (ef[k], want)
        assert abs(ef[k, 1] / L) <= 1e-9 * tau
        seen += 1
    assert seen == 2


def test_stress_traction_uniform_pressure():
    """A resting body in a uniform fluid at rho0 = 1.01: every element carries
    exactly -(rho0 - 1) c_s^2 times its outward area vector, so the closed
    body's total vanishes while each element feels the gauge pressure."""
    ny = nx = 16
    rho0 = 1.01
    xs, es = synth.circle_polygon(8.0, 8.0, 3.3, 24)
    surf = orc.Surface(xs, np.zeros_like(xs), es, np.zeros(len(es), np.int32))
    f = orc.init_equilibrium(9, np.full((1, ny, nx), rho0), np.zeros((2, 1, ny, nx)))
    for _ in range(3):
        f, _, _, _, sig = orc.step_bc(9, 0.9, f, bc=(0,) * 6, surf=surf, want_sigma=True)
    vf, bf, ef = orc.traction(surf, sig)
    area = 0.5 * sum(xs[a, 0] * xs[b, 1] - xs[b, 0] * xs[a, 1] for a, b in es)
    sg = 1.0 if area > 0 else -1.0
    p = (rho0 - 1.0) / 3.0
    for k, (a, b) in enumerate(es):
        nA = sg * np.array([xs[b, 1] - xs[a, 1], -(xs[b, 0] - xs[a, 0])])
        np.testing.assert_allclose(ef[k, :2], -p * nA, rtol=0, atol=1e-12)
    assert np.max(np.abs(bf)) <= 1e-12
