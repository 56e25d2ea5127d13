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


def test_beam_solve_precision_modes():
    """The Newton matrix and its solve in FP64 (solve_fp64: the exact Newton
    step of the oracle) and in FP32 (the default inexact step), the same
    prescribed large-deflection loads: FP64 agrees with the oracle to
    round-off, FP32 to the Newton stopping test; time per step of each."""
    import time
    import torch
    from paper_1710_02375_gb300.lbm import Beam
    X, EA, EI, rhoA, fixed = synth.c1_flag_beam()
    n = 3 * len(X)
    s = (X[:, 0] - X[0, 0]) / (X[-1, 0] - X[0, 0])
    loads = []
    for t in range(300):
        F1 = np.zeros(n)
        F1[1::3] = 2e-3 * np.sin(0.02 * t) * s
        F1[0::3] = 5e-4 * s
        loads.append(F1)
    ob = orc.Beam(X, EA, EI, rhoA, fixed)
    u, v, F0 = np.zeros(n), np.zeros(n), np.zeros(n)
    ref = []
    for F1 in loads:
        u, v, _ = ob.step(u, v, F0, F1)
        F0 = F1
        ref.append(u.copy())
    out = {}
    for fp64 in (True, False):
        gb = Beam(X, EA, EI, rhoA, fixed, thickness=2.0, solve_fp64=fp64)
        worst, t_total = 0.0, 0.0
        for k, F1 in enumerate(loads):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            gb.step(F1)
            ug, _, itg = gb.state()
            t_total += time.perf_counter() - t0
            assert itg >= 0
            worst = max(worst, np.max(np.abs(ug - ref[k])) / max(np.max(np.abs(ref[k])), 1e-30))
        out["fp64" if fp64 else "fp32"] = (worst, 1e3 * t_total / len(loads))
    print("BEAM SOLVE MODES (max relative error vs oracle, ms per step incl. readback):", out)
    assert out["fp64"][0] < 1e-12, out
    assert out["fp32"][0] < 1e-8, out


def test_beam_csm3_matches_oracle():
    """CSM3 (flag under gravity, large deflection, dt = 5 ms, 1200 steps) on
    the GPU beam against the oracle beam, which the paper's CSM3 table pins."""
    from paper_1710_02375_gb300.lbm import Beam
    E, nu_s, rho_s, grav, Lb, h, ne, dt = 1.4e6, 0.4, 1e3, 2.0, 0.35, 0.02, 20, 0.005
    Ep = E / (1 - nu_s ** 2)
    X = np.stack([np.linspace(0, Lb, ne + 1), np.zeros(ne + 1)], 1)
    fixed = np.zeros(3 * (ne + 1), np.int32)
    fixed[:3] = 1
    args = (X, Ep * h, Ep * h ** 3 / 12, rho_s * h, fixed)
    gb = Beam(*args, thickness=h, dt=dt, atol=1e-14)
    ob = orc.Beam(*args)
    F = np.zeros(3 * (ne + 1))
    F[1::3] = -rho_s * grav * h * Lb / ne
    F[1] *= 0.5
    F[-2] *= 0.5
    u, v = np.zeros(3 * (ne + 1)), np.zeros(3 * (ne + 1))
    gb.step(F)  # the first step's previous load F0 is zero on the GPU beam
    u, v, _ = ob.step(u, v, np.zeros_like(F), F, dt=dt, atol=1e-14)
    worst = 0.0
    for _ in range(1199):
        gb.step(F)
        u, v, it = ob.step(u, v, F, F, dt=dt, atol=1e-14)
        ug, _, itg = gb.state()
        assert it >= 0 and itg >= 0
        worst = max(worst, np.max(np.abs(ug - u)) / np.max(np.abs(u)))
    assert worst < 1e-8, worst
    assert np.min(u[1::3]) < -0.1  # past the first downswing


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


def test_coupled_flag_graph_replay_matches_direct_stepping():
    """The C1 coupled step (Grad fill, sweep, beam Newton step, flag surface,
    new geometry) captured as a CUDA graph of 10 steps and replayed 30 times
    matches 300 direct steps (up to the order of the FP64 atomic sums in the
    force gather)."""
    from paper_1710_02375_gb300.cases import c1_coupled
    La, ba, _ = c1_coupled(100.0)
    La.step(300)
    La.check()
    Lb, bb, _ = c1_coupled(100.0)
    Lb.step_graph(10, 30)
    Lb.check()
    ua, _, _ = ba.state()
    ub, _, _ = bb.state()
    fa, fb = La.get_populations(), Lb.get_populations()
    assert Lb.boundary_info()[3] == 300  # inflow-ramp clock advanced once per step
    assert np.max(np.abs(fa - fb)) <= 1e-6 * np.max(np.abs(fa))
    assert np.max(np.abs(ua - ub)) <= 1e-9 * max(np.max(np.abs(ua)), 1e-30)


@pytest.mark.parametrize("fac", [3.4, 3.8])
def test_beam_large_rotation_steps_match_oracle(fac):
    """A tip moment fac x 1.5 pi EI / L held on the C1 flag beam for 100
    steps: the element chords turn by up to 0.28 rad in one step (the atan2
    branch of the chord rotation, beyond the arctangent series) and, at fac
    3.8, through +-pi (chord angles up to 4.5 rad: the wrap of atan2).  The
    GPU beam against the oracle at every step."""
    from paper_1710_02375_gb300.lbm import Beam
    X, EA, EI, rhoA, fixed = synth.c1_flag_beam()
    L = X[-1, 0] - X[0, 0]
    gb = Beam(X, EA, EI, rhoA, fixed, thickness=2.0)
    ob = orc.Beam(X, EA, EI, rhoA, fixed)
    n = 3 * len(X)
    u, v, F0 = np.zeros(n), np.zeros(n), np.zeros(n)
    F1 = np.zeros(n)
    F1[-1] = fac * 1.5 * np.pi * EI / L
    worst, chord = 0.0, 0.0
    for _ in range(100):
        gb.step(F1)
        u, v, it = ob.step(u, v, F0, F1)
        F0 = F1
        ug, _, itg = gb.state()
        assert it >= 0 and itg >= 0
        worst = max(worst, np.max(np.abs(ug - u)) / np.max(np.abs(u)))
        x, y = X[:, 0] + u[0::3], X[:, 1] + u[1::3]
        chord = max(chord, np.abs(np.unwrap(np.arctan2(np.diff(y), np.diff(x)))).max())
    print(f"large rotations (fac {fac}): max chord angle {chord:.2f} rad, GPU vs oracle {worst:.2e}")
    assert chord > (3.0 if fac < 3.6 else np.pi)
    assert worst < 1e-12, worst  # measured 8.6e-15 / 8.5e-15
