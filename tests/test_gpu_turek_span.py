"""Quasi-two-dimensional Turek set-up (section "Turek Benchmark": a few
lattice points spanwise, periodic for the fluid, plane strain for the solid)
on the C1 geometry: D3Q27 channel 220 x 41 with nz spanwise nodes, periodic
along z; the cylinder and the flag extruded along z past both periodic
faces; the flag an elastic beam coupled through fsi_couple_span (nodal loads
per unit span).  GPU against the FP64 oracle's quasi-2-D CSS loop, at the
FP32 bounds of the boundary tests."""
import numpy as np
import pytest

from oracle import fsi_oracle
from oracle import oracle as orc
from paper_1710_02375_gb300 import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def case(nz=2, z0=-2.0, z1=None):
    nx, ny = 220, 41
    z1 = nz + 2.0 if z1 is None else z1
    u_max, Re, D = 0.05, 100.0, 10.0
    nu = (2.0 / 3.0) * u_max * D / Re
    beta = 1.0 / (6 * nu + 1)
    prof2 = synth.parabolic_profile(ny, u_max, noise=1e-4, seed=0)
    prof = np.zeros((3, nz * ny))
    for z in range(nz):
        prof[:, z * ny:(z + 1) * ny] = prof2      # face index z * ny + y
    x2, e2, body2, _ = synth.cylinder_flag_2d()
    x3, e3, b3 = synth.extrude_polygons(x2, e2, body2, z0, z1)
    X, EA, EI, rhoA, fixed = synth.c1_flag_beam()
    return dict(nx=nx, ny=ny, nz=nz, beta=beta, prof=prof, x2=x2, x3=x3, e3=e3, b3=b3,
                ncyl=int(np.sum(body2 == 0)), beam=(X, EA, EI, rhoA, fixed), h=2.0, z0=z0, z1=z1)


def test_span_coupling_rejects_bad_set_ups():
    from paper_1710_02375_gb300 import lbm as abi
    from paper_1710_02375_gb300.lbm import Beam, Lattice
    c = case()
    L = Lattice(27, c["nx"], c["ny"], c["nz"], c["beta"], bc=(2, 3, 1, 1, 0, 0), max_links=20000,
                max_vertices=len(c["x3"]), max_elements=len(c["e3"]))
    L.set_geometry(c["x3"], c["e3"], c["b3"], band_margin=8.0)
    gb = Beam(*c["beam"], thickness=c["h"], stream=L.stream)
    n2 = len(c["x2"])
    with pytest.raises(abi.LbmError):   # the span must cover the periodic box
        abi.fsi_couple_span(L.ctx, gb.ctx, c["ncyl"], n2 + c["ncyl"], 0.5, c["z1"])
    with pytest.raises(abi.LbmError):   # overlapping vertex ranges
        abi.fsi_couple_span(L.ctx, gb.ctx, c["ncyl"], c["ncyl"] + 1, c["z0"], c["z1"])
    with pytest.raises(abi.LbmError):   # the 2-D coupling is D2Q9 only
        abi.fsi_couple(L.ctx, gb.ctx, c["ncyl"])


def test_quasi_2d_flag_matches_oracle():
    """600 coupled steps from rest into the inflow ramp (1000 steps).
    Measured: velocity 5.5e-7, tip 3.5e-5, body force 5.2e-6, spanwise spread
    0 (the z layers compute identical bits)."""
    from paper_1710_02375_gb300 import lbm as abi
    from paper_1710_02375_gb300.lbm import Beam, Lattice
    c = case()
    steps, ramp, bc = 600, 1000, (2, 3, 1, 1, 0, 0)
    nx, ny, nz = c["nx"], c["ny"], c["nz"]
    n2 = len(c["x2"])
    L = Lattice(27, nx, ny, nz, c["beta"], bc=bc, max_links=20000, max_vertices=len(c["x3"]),
                max_elements=len(c["e3"]), inlet_ramp_steps=ramp)
    L.set_inlet_profile(0, c["prof"])
    L.set_geometry(c["x3"], c["e3"], c["b3"], band_margin=8.0)
    L.init_equilibrium(np.ones((nz, ny, nx)), np.zeros((3, nz, ny, nx)))
    gb = Beam(*c["beam"], thickness=c["h"], stream=L.stream)
    abi.fsi_couple_span(L.ctx, gb.ctx, c["ncyl"], n2 + c["ncyl"], c["z0"], c["z1"])
    L.step(steps)
    L.check()
    _, ug = L.macros()
    _, bf_g = L.interface_force()
    u_beam_g, _, it_g = gb.state()
    assert it_g >= 0

    css = fsi_oracle.CSSFlagSpan((nz, ny, nx), c["beta"], bc, {0: c["prof"]}, ramp,
                                 c["x2"][:c["ncyl"]], c["e3"], c["b3"], orc.Beam(*c["beam"]), c["h"],
                                 c["z0"], c["z1"])
    for _ in range(steps):
        css.step()
    _, uo = orc.macros(27, css.f)
    uo[:, css.solid.astype(bool)] = 0
    eu = rel(ug, uo)
    tip_o = css.u[-2]
    et = abs(u_beam_g[-2] - tip_o) / max(abs(tip_o), 1e-12)
    ef = max(np.linalg.norm(bf_g[b] - css.bforce[b]) / np.linalg.norm(css.bforce[b]) for b in range(2))
    # the flow stays uniform along the span
    spread = np.max(np.abs(ug[:, 1:] - ug[:, :1])) / np.max(np.abs(ug))
    print(f"QUASI-2D {steps} steps: velocity {eu:.2e} tip {et:.2e} (tip {tip_o:.3e}) "
          f"body force {ef:.2e} spanwise spread {spread:.2e}")
    assert eu <= 1e-5 and et <= 1e-4 and ef <= 1e-4, (eu, et, ef)
    assert spread <= 1e-6
