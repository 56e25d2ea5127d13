"""Pins of the oracle's co-rotational flat shell (the plate structure that
replaces the paper's Q2 continuum elements, section "Structural modeling";
theta-scheme of Eq. timeInt with Newton and lambda = 0.7) against closed forms,
rigid-body invariance, the elastica and the cantilever eigenvalue."""
import numpy as np
import pytest

from oracle import oracle as orc
from test_oracle_fem_pins import elastica_tip


def strip(nx=17, ny=9, L=40.0, b=20.0, E=1000.0, nu=0.0, h=2.0, rho=1.0):
    xs = np.linspace(0.0, L, nx)
    ys = np.linspace(-b / 2, b / 2, ny)
    X = np.array([[x, y, 0.0] for x in xs for y in ys])
    fixed = np.zeros(6 * nx * ny, np.int32)
    fixed[: 6 * ny] = 1  # clamped edge x = 0
    return orc.Shell(X, nx, ny, E, nu, h, rho, fixed)


def edge_load(S, comp, P):
    """Total load P on the free edge (x = L) along comp, consistent for the
    bilinear edge (half weights at the corners)."""
    F = np.zeros((S.nn, 6))
    w = np.ones(S.ny)
    w[0] = w[-1] = 0.5
    F[-S.ny:, comp] = P * w / w.sum()
    return F


def rot(axis_angle):
    a = np.asarray(axis_angle, dtype=float)
    t = np.linalg.norm(a)
    k = a / t
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(t) * K + (1 - np.cos(t)) * K @ K


def test_rigid_motion_has_no_internal_force():
    """A large rigid rotation plus translation of the whole plate leaves every
    element's local deformation zero (frames, log map and projector)."""
    S = strip(nu=0.3)
    Q = rot([0.9, -1.4, 0.6])
    u = S.X @ Q.T - S.X + np.array([3.0, -2.0, 5.0])
    R = np.tile(Q, (S.nn, 1, 1))
    f = S.internal(u, R)
    assert np.max(np.abs(f)) <= 1e-12 * S.E * S.h * 40.0


def test_membrane_tension_is_exact():
    """Uniform tension (nu = 0): the bilinear membrane reproduces the constant
    strain state, tip extension P L / (E h b)."""
    S = strip()
    P = 0.5
    u, R, it = S.static(edge_load(S, 0, P).ravel(), atol=1e-10)
    assert it >= 0
    exact = P * 40.0 / (S.E * S.h * 20.0)
    np.testing.assert_allclose(u[-S.ny:, 0], exact, rtol=1e-9)
    assert np.max(np.abs(u[:, 2])) < 1e-12


def test_plate_strip_end_load_linear_limit():
    """Small transverse end load (nu = 0): tip deflection against
    P L^3 / (3 D b) + P L / (kappa G h b), D = E h^3 / 12, kappa = 5/6; the
    error shrinks with the mesh."""
    errs = []
    for nx, ny in ((9, 5), (17, 9)):
        S = strip(nx=nx, ny=ny)
        P = 1e-4
        u, R, it = S.static(edge_load(S, 2, P).ravel(), atol=1e-9)
        assert it >= 0, it
        D, G = S.E * S.h ** 3 / 12, S.E / 2
        exact = P * 40.0 ** 3 / (3 * D * 20.0) + P * 40.0 / (5 / 6 * G * S.h * 20.0)
        errs.append(abs(u[-S.ny:, 2].mean() - exact) / exact)
    assert errs[1] < 2e-3, errs
    assert errs[1] < errs[0], errs


def test_plate_strip_large_deflection_matches_elastica():
    """Dead end load P = 2 EI / L^2 (nu = 0, EI = D b): the tip of the strip
    against the inextensible elastica (load applied in five increments)."""
    S = strip(E=1e4)
    EI = S.E * S.h ** 3 / 12 * 20.0
    P = 2.0 * EI / 40.0 ** 2
    u, R = None, None
    for k in range(1, 6):
        u, R, it = S.static(edge_load(S, 2, P * k / 5).ravel(), lam=1.0, max_it=300, atol=1e-8,
                            u=u, R=R)
        assert it >= 0, it
    xe, ye, _ = elastica_tip(P, EI, 40.0)
    assert abs(u[-S.ny:, 2].mean() - ye) < 1e-2 * ye
    assert abs(40.0 + u[-S.ny:, 0].mean() - xe) < 1e-2 * 40.0


def test_free_vibration_frequency_and_energy():
    """Released from a small static tip deflection (nu = 0), theta = 1/2:
    the period matches the first cantilever mode 2 pi / ((1.8751)^2
    sqrt(EI / (rho h b L^4))) within 1 %, and the energy is conserved."""
    S = strip(E=1e3, rho=1.0)
    F = edge_load(S, 2, 2e-4)
    u, R, it = S.static(F.ravel(), atol=1e-9)
    v = np.zeros((S.nn, 6))
    EI = S.E * S.h ** 3 / 12 * 20.0
    w1 = 1.8751040687119611 ** 2 * np.sqrt(EI / (S.rho * S.h * 20.0 * 40.0 ** 4))
    T = 2 * np.pi / w1
    dt = T / 200
    zero = np.zeros(6 * S.nn)
    tip = []
    for _ in range(500):
        u, R, v, it = S.step(u, R, v, zero, zero, dt=dt, atol=1e-10)
        assert it >= 0
        tip.append(u[-S.ny:, 2].mean())
    tip = np.array(tip)
    t = dt * np.arange(1, len(tip) + 1)
    k = np.nonzero(tip[:-1] * tip[1:] < 0)[0]
    tc = t[k] - dt * tip[k] / (tip[k + 1] - tip[k])
    period = 2 * np.mean(np.diff(tc))
    assert abs(period - T) < 1e-2 * T, (period, T)
    assert abs(tip.max() - tip.min() - 2 * abs(tip[0])) < 2e-2 * abs(tip[0])
