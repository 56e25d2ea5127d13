"""Lattices of the synthetic workloads (set-up through the public binding)."""
from __future__ import annotations

import numpy as np


def c4_lattice(inst, coupled, stream, storage=0):
    """One member of the batched flag ensemble (synth.c4_instances): D2Q9
    channel with parabolic inflow, cylinder and flag; with coupled=True the
    flag is an elastic beam (fsi_couple), else a rigid body.  Returns
    (Lattice, Beam or None)."""
    from . import lbm
    from .lbm import Beam, Lattice
    L = Lattice(9, inst["nx"], inst["ny"], 1, inst["beta"], storage=storage, bc=(2, 3, 1, 1, 0, 0),
                max_links=8000, max_vertices=len(inst["x"]), max_elements=len(inst["e"]),
                inlet_ramp_steps=300, stream=stream)
    L.set_inlet_profile(0, inst["inlet"])
    L.set_geometry(inst["x"], inst["e"], inst["body"], band_margin=0.5 * inst["D"])
    L.init_equilibrium(np.ones((1, inst["ny"], inst["nx"])), np.zeros((2, 1, inst["ny"], inst["nx"])))
    beam = None
    if coupled:
        X, EA, EI, rhoA, fixed = inst["beam"]
        beam = Beam(X, EA, EI, rhoA, fixed, thickness=inst["h"], stream=stream)
        lbm.fsi_couple(L.ctx, beam.ctx, inst["ncyl"])
    return L, beam


C1 = dict(nx=220, ny=41, D=10.0, u_max=0.05, h=2.0, ramp=1000, bc=(2, 3, 1, 1, 0, 0))


def c1_coupled(Re, seed=0, stream=None):
    """The C1 flag case (channel 220 x 41, cylinder D = 10 with an elastic flag
    of length 3.5 D and thickness 0.2 D, rho_s / rho_f = 10, Ae = 1.4e3,
    parabolic inflow u_max = 0.05 with a 1000-step ramp) at Reynolds number
    Re on the mean inflow speed and D, CSS-coupled.  Returns (Lattice, Beam,
    first flag vertex)."""
    from . import lbm, synth
    from .lbm import Beam, Lattice
    c = C1
    nu = (2.0 / 3.0) * c["u_max"] * c["D"] / Re
    beta = 1.0 / (6 * nu + 1)
    prof = synth.parabolic_profile(c["ny"], c["u_max"], noise=1e-4, seed=seed)
    x, e, body, _ = synth.cylinder_flag_2d()
    X, EA, EI, rhoA, fixed = synth.c1_flag_beam()
    ncyl = int(np.sum(body == 0))
    L = Lattice(9, c["nx"], c["ny"], 1, beta, bc=c["bc"], max_links=4000, max_vertices=len(x),
                max_elements=len(e), inlet_ramp_steps=c["ramp"], stream=stream)
    L.set_inlet_profile(0, prof)
    L.set_geometry(x, e, body, band_margin=8.0)
    L.init_equilibrium(np.ones((1, c["ny"], c["nx"])), np.zeros((2, 1, c["ny"], c["nx"])))
    beam = Beam(X, EA, EI, rhoA, fixed, thickness=c["h"], stream=L.stream)
    lbm.fsi_couple(L.ctx, beam.ctx, ncyl)
    return L, beam, ncyl


def flag_coupled(inst, stream=None, ramp=1000):
    """A synth.flag_channel case (e.g. synth.c5_case) CSS-coupled: walls top
    and bottom, parabolic inlet on -x with the inflow ramp, outlet on +x.
    Returns (Lattice, Beam)."""
    from . import lbm
    from .lbm import Beam, Lattice
    nx, ny = inst["nx"], inst["ny"]
    L = Lattice(9, nx, ny, 1, inst["beta"], bc=(2, 3, 1, 1, 0, 0), max_links=16000,
                max_vertices=len(inst["x"]), max_elements=len(inst["e"]), inlet_ramp_steps=ramp,
                stream=stream)
    L.set_inlet_profile(0, inst["inlet"])
    L.set_geometry(inst["x"], inst["e"], inst["body"], band_margin=0.5 * inst["D"])
    L.init_equilibrium(np.ones((1, ny, nx)), np.zeros((2, 1, ny, nx)))
    X, EA, EI, rhoA, fixed = inst["beam"]
    beam = Beam(X, EA, EI, rhoA, fixed, thickness=inst["h"], stream=L.stream)
    lbm.fsi_couple(L.ctx, beam.ctx, inst["ncyl"])
    return L, beam


def plate_coupled(c, storage=0, stream=None, band=None, atol=1e-13):
    """A synth.plate_case lattice with its CSS-coupled shell (fsi_couple_shell),
    started from uniform flow at the inflow speed with the plate's initial
    deflection.  Returns (Lattice, Shell)."""
    from . import lbm, synth
    from .lbm import Lattice, Shell
    sh = c["shell"]
    nn = sh["nx"] * sh["ny"]
    L = Lattice(27, c["nx"], c["ny"], c["nz"], c["beta"], storage=storage, bc=c["bc"],
                face_velocity=c["face_u"], max_links=200000, max_vertices=2 * nn,
                max_elements=len(c["e"]), stream=stream)
    x = synth.plate_vertices(sh["X"], c["u0"], c["R0"], sh["h"])
    L.set_geometry(x, c["e"], np.zeros(len(c["e"]), np.int32),
                   band_margin=0.5 * c["L"] if band is None else band)
    vel = np.zeros((3, c["nz"], c["ny"], c["nx"]))
    vel[0] = c["u_in"]
    L.init_equilibrium(np.ones((c["nz"], c["ny"], c["nx"])), vel)
    S = Shell(sh["X"], sh["nx"], sh["ny"], sh["E"], sh["nu"], sh["h"], sh["rho"], sh["fixed"],
              atol=atol, stream=L.stream)
    S.set_state(u=c["u0"], R=c["R0"])
    lbm.fsi_couple_shell(L.ctx, S.ctx, 0)
    return L, S


def turek_span_coupled(nz=2, Re=100.0, stream=None, seed=0):
    """The quasi-2-D Turek set-up on the C1 geometry (section "Turek
    Benchmark"): D3Q27 channel 220 x 41 x nz periodic along z, parabolic
    inflow with the 1000-step ramp, cylinder and flag extruded along z over
    [-2, nz + 2], the flag an elastic beam coupled per unit span
    (fsi_couple_span).  Returns (Lattice, Beam)."""
    from . import lbm, synth
    from .lbm import Beam, Lattice
    c = C1
    nx, ny = c["nx"], c["ny"]
    nu = (2.0 / 3.0) * c["u_max"] * c["D"] / Re
    beta = 1.0 / (6 * nu + 1)
    prof2 = synth.parabolic_profile(ny, c["u_max"], noise=1e-4, seed=seed)
    prof = np.tile(prof2, (1, nz))           # face index z * ny + y
    x2, e2, body2, _ = synth.cylinder_flag_2d()
    z0, z1 = -2.0, nz + 2.0
    x3, e3, b3 = synth.extrude_polygons(x2, e2, body2, z0, z1)
    ncyl = int(np.sum(body2 == 0))
    L = Lattice(27, nx, ny, nz, beta, bc=c["bc"], max_links=20000, max_vertices=len(x3),
                max_elements=len(e3), inlet_ramp_steps=c["ramp"], stream=stream)
    L.set_inlet_profile(0, prof)
    L.set_geometry(x3, e3, b3, band_margin=8.0)
    L.init_equilibrium(np.ones((nz, ny, nx)), np.zeros((3, nz, ny, nx)))
    X, EA, EI, rhoA, fixed = synth.c1_flag_beam()
    beam = Beam(X, EA, EI, rhoA, fixed, thickness=c["h"], stream=L.stream)
    lbm.fsi_couple_span(L.ctx, beam.ctx, ncyl, len(x2) + ncyl, z0, z1)
    return L, beam
