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
