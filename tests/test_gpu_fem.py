"""GPU beam (FP64 co-rotational, theta-scheme, Newton with lambda = 0.7) and
the coupled conventional serial staggered loop against the oracle."""
import numpy as np
import pytest

from oracle import oracle as orc
from oracle import fsi_oracle
from paper_1710_02375_gb300 import synth

pytestmark = pytest.mark.gpu


def test_beam_prescribed_loads_matches_oracle():
    X, EA, EI, rhoA, fixed = synth.c1_flag_beam()
    from paper_1710_02375_gb300.lbm import Beam
    gb = Beam(X, EA, EI, rhoA, fixed, thickness=2.0)
    ob = orc.Beam(X, EA, EI, rhoA, fixed)
    n = 3 * len(X)
    u, v, F0 = np.zeros(n), np.zeros(n), np.zeros(n)
    s = (X[:, 0] - X[0, 0]) / (X[-1, 0] - X[0, 0])
    worst = 0.0
    for t in range(300):
        F1 = np.zeros(n)
        F1[1::3] = 2e-3 * np.sin(0.02 * t) * s
        F1[0::3] = 5e-4 * s
        gb.step(F1)
        u, v, it = ob.step(u, v, F0, F1)
        F0 = F1
        ug, vg, itg = gb.state()
        assert itg >= 0 and it >= 0
        worst = max(worst, np.max(np.abs(ug - u)) / max(np.max(np.abs(u)), 1e-30))
    assert worst < 1e-8
    assert np.max(np.abs(u[1::3])) > 0.5  # large deflection regime reached


def test_coupled_flag_c1_matches_oracle():
    """C1 (Turek-type cylinder + elastic flag, Re = 100, rho_s/rho_f = 10,
    Ae = 1.4e3): 400 coupled steps of fluid + Grad + force + beam + geometry."""
    from paper_1710_02375_gb300.lbm import Beam, Lattice
    nx, ny = 220, 41
    u_max, Re, D = 0.05, 100.0, 10.0
    nu = (2.0 / 3.0) * u_max * D / Re
    beta = 1.0 / (6 * nu + 1)
    prof = synth.parabolic_profile(ny, u_max, noise=1e-4, seed=0)
    x, e, body, _ = synth.cylinder_flag_2d()
    X, EA, EI, rhoA, fixed = synth.c1_flag_beam()
    h = 2.0
    ncyl = int(np.sum(body == 0))
    bc = (2, 3, 1, 1, 0, 0)
    ramp, steps = 1000, 600
    L = Lattice(9, nx, ny, 1, beta, bc=bc, max_links=4000, max_vertices=len(x),
                max_elements=len(e), inlet_ramp_steps=ramp)
    L.set_inlet_profile(0, prof)
    L.set_geometry(x, e, body, band_margin=8.0)
    L.init_equilibrium(np.ones((1, ny, nx)), np.zeros((2, 1, ny, nx)))
    gb = Beam(X, EA, EI, rhoA, fixed, thickness=h, stream=L.stream)
    from paper_1710_02375_gb300 import lbm as abi
    abi.fsi_couple(L.ctx, gb.ctx, ncyl)
    L.step(steps)
    L.check()
    _, ug = L.macros()
    vf_g, bf_g = L.interface_force()
    u_beam_g, _, it_g = gb.state()

    ob = orc.Beam(X, EA, EI, rhoA, fixed)
    css = fsi_oracle.CSSFlag(9, (1, ny, nx), beta, bc, None, {0: prof}, ramp, x[:ncyl], e, body, ob, h)
    for _ in range(steps):
        css.step()
    _, uo = orc.macros(9, css.f)
    uo[:, css.solid.astype(bool)] = 0
    err_u = np.max(np.abs(ug - uo[:2])) / np.max(np.abs(uo))
    assert err_u <= 1e-5, err_u
    tip_o = css.u[-2]
    assert abs(u_beam_g[-2] - tip_o) <= 1e-4 * max(abs(tip_o), 1e-6), (u_beam_g[-2], tip_o)
    for b in range(2):
        assert np.linalg.norm(bf_g[b] - css.bforce[b]) <= 1e-4 * np.linalg.norm(css.bforce[b])
