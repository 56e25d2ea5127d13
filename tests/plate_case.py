"""The plate-in-crossflow case at small size (48 x 24 x 24 D3Q27 channel,
plate 16 x 8 x 2 as 8 x 4 shell elements, clamped leading edge) at a chosen
Reynolds number and initial tip deflection, for the oracle and for the CUDA
library; and the worker that turns an oracle run into surrogate training
pairs (importable by spawned processes)."""
from __future__ import annotations

import numpy as np

from paper_1710_02375_gb300 import synth


def case(Re=100.0, perturb=2e-2):
    return synth.plate_case(nxl=48, nyl=24, nzl=24, L=16.0, b=8.0, h=2.0, x0=12.0, u_in=0.04,
                            Re=Re, ex=8, ey=4, perturb=perturb)


def oracle_run(Re=100.0, perturb=2e-2):
    from oracle import fsi_oracle
    from oracle import oracle as orc
    c = case(Re, perturb)
    sh = c["shell"]
    shell = orc.Shell(sh["X"], sh["nx"], sh["ny"], sh["E"], sh["nu"], sh["h"], sh["rho"], sh["fixed"])
    vel = np.zeros((3, c["nz"], c["ny"], c["nx"]))
    vel[0] = c["u_in"]
    return fsi_oracle.CSSPlate((c["nz"], c["ny"], c["nx"]), c["beta"], c["bc"], c["face_u"], shell,
                               c["e"], sh["h"], u0=c["u0"], R0=c["R0"], vel0=vel)


def oracle_pairs(args):
    """(X, Y) surrogate pairs of `steps` steps of the oracle plate run at
    (Re, perturb)."""
    from oracle import surrogate_data
    Re, perturb, steps = args
    return surrogate_data.pairs_from_plate_run(oracle_run(Re, perturb), steps, atol=1e-13)


def gpu_run(Re=100.0, perturb=2e-2, storage=0, stream=None):
    """The same case coupled on the GPU (fsi_couple_shell); (Lattice, Shell)."""
    from paper_1710_02375_gb300.cases import plate_coupled
    return plate_coupled(case(Re, perturb), storage=storage, stream=stream, band=4.0)
