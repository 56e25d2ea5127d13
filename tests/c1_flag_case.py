"""The C1 flag case (Turek-type channel, cylinder D = 10, elastic flag,
rho_s / rho_f = 10, Ae = 1.4e3, 1000-step inflow ramp) at a chosen Reynolds
number, for the oracle and for the CUDA library; and the worker that turns an
oracle run into surrogate training pairs (importable by spawned processes)."""
from __future__ import annotations

import numpy as np

from paper_1710_02375_gb300 import synth

NX, NY, D, U_MAX, H, RAMP = 220, 41, 10.0, 0.05, 2.0, 1000
BC = (2, 3, 1, 1, 0, 0)


def case(Re, seed=0):
    nu = (2.0 / 3.0) * U_MAX * D / Re
    beta = 1.0 / (6 * nu + 1)
    prof = synth.parabolic_profile(NY, U_MAX, noise=1e-4, seed=seed)
    x, e, body, _ = synth.cylinder_flag_2d()
    beam = synth.c1_flag_beam()
    return dict(beta=beta, prof=prof, x=x, e=e, body=body, ncyl=int(np.sum(body == 0)), beam=beam)


def oracle_run(Re, seed=0):
    from oracle import fsi_oracle
    from oracle import oracle as orc
    c = case(Re, seed)
    X, EA, EI, rhoA, fixed = c["beam"]
    ob = orc.Beam(X, EA, EI, rhoA, fixed)
    return fsi_oracle.CSSFlag(9, (1, NY, NX), c["beta"], BC, None, {0: c["prof"]}, RAMP,
                              c["x"][:c["ncyl"]], c["e"], c["body"], ob, H)


def oracle_pairs(args):
    """(X, Y) surrogate pairs of `steps` steps of the oracle run at (Re, seed)."""
    from oracle import surrogate_data
    Re, seed, steps = args
    X, Y, _ = surrogate_data.pairs_from_run(oracle_run(Re, seed), steps)
    return X, Y


def oracle_run_inst(inst, ramp=RAMP):
    """Coupled oracle run of a synth.flag_channel case (walls top and bottom,
    inlet -x, outlet +x)."""
    from oracle import fsi_oracle
    from oracle import oracle as orc
    X, EA, EI, rhoA, fixed = inst["beam"]
    ob = orc.Beam(X, EA, EI, rhoA, fixed)
    nc = inst["ncyl"]
    return fsi_oracle.CSSFlag(9, (1, inst["ny"], inst["nx"]), inst["beta"], BC, None, {0: inst["inlet"]},
                              ramp, inst["x"][:nc], inst["e"], inst["body"], ob, inst["h"])


def c5_pairs(args):
    """(X, Y) surrogate pairs of `steps` steps of the oracle C5 flag run at (Re, seed)."""
    from oracle import surrogate_data
    Re, seed, steps = args
    X, Y, _ = surrogate_data.pairs_from_run(oracle_run_inst(synth.c5_case(Re, seed)), steps)
    return X, Y


def gpu_run(Re, seed=0):
    """(Lattice, Beam) of the CUDA library, coupled, at step 0."""
    from paper_1710_02375_gb300.cases import c1_coupled
    L, gb, _ = c1_coupled(Re, seed)
    return L, gb
