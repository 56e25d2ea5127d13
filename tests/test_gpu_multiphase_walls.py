"""Multiphase model between planar walls on the GPU (Grad fill of the wall
nodes, mirrored fields, wetting force F_s; multiphase.cu k_mp_wall_band /
k_mp_wall_fill and the wall terms of the passes) against the oracle's
step_multiphase_wall, through the C ABI."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1710_02375_gb300 import synth

pytestmark = pytest.mark.gpu
F32, F64 = 0, 3


def walled(lat, shape, wa, beta, kappa, kappa_w, storage=F32, collision=0, eos=0,
           g=(0.0, 0.0, 0.0)):
    from paper_1710_02375_gb300.lbm import Lattice
    nz, ny, nx = shape
    bc = [0] * 6
    bc[2 * wa] = bc[2 * wa + 1] = 1
    L = Lattice(lat, nx, ny, nz, beta, storage=storage, collision=collision, bc=tuple(bc),
                multiphase=True)
    L.set_multiphase(kappa, eos, g, kappa_w=kappa_w)
    return L


def werr(lat, a, b):
    w = synth.lattice_weights(lat).reshape((lat, 1, 1, 1))
    return np.max(np.abs(a - b) / w)


def two_phase_state(lat, shape, seed):
    rng = np.random.default_rng(seed)
    R = 0.3 * min(s for s in shape if s > 1)
    rho = synth.droplet_density(shape, R, rho_l=7.5, rho_v=0.08, noise=1e-3, seed=seed)
    dim = 2 if lat == 9 else 3
    u = 0.02 * rng.uniform(-1, 1, size=(dim,) + shape)
    f = orc.init_equilibrium(lat, rho, u)
    return f * (1 + 0.01 * rng.uniform(-1, 1, size=f.shape))


@pytest.mark.parametrize("lat,shape,wa", [(9, (1, 37, 53), 1), (9, (1, 37, 53), 0),
                                          (27, (13, 11, 17), 2), (27, (13, 11, 17), 1),
                                          (27, (13, 11, 17), 0), (27, (41, 12, 20), 2),
                                          (27, (41, 12, 20), 1)])
def test_three_steps_match_oracle_fp32(lat, shape, wa):
    """Three steps from a random two-phase state (the second and third fill
    the wall nodes with the force of the step before), kappa_w = -0.1, on
    ragged sizes and every wall axis.  Measured 1.9e-6 .. 3.1e-6 W,
    force 5e-7 .. 1e-6."""
    beta, kappa, kw = 0.8, 0.02, -0.1
    f0 = two_phase_state(lat, shape, seed=5)
    L = walled(lat, shape, wa, beta, kappa, kw)
    L.set_populations(f0)
    L.step(3)
    L.check()
    got = L.get_populations()
    Fg = L.force_field()
    f, F = f0, None
    for _ in range(3):
        f, F = orc.step_multiphase_wall(lat, beta, f, kappa, kw, wa, F_prev=F)
    ep = werr(lat, got, f)
    ef = np.max(np.abs(Fg - F)) / np.max(np.abs(F))
    print(f"D{'2Q9' if lat == 9 else '3Q27'} walls on axis {wa}, 3 steps: populations {ep:.2e} W, "
          f"force {ef:.2e}")
    assert ep <= 2e-5 and ef <= 2e-5, (ep, ef)


@pytest.mark.parametrize("collision", [0, 1])
def test_three_steps_match_oracle_fp64(collision):
    lat, shape, wa, beta, kappa, kw = 9, (1, 29, 31), 1, 0.8, 0.02, 0.07
    f0 = two_phase_state(lat, shape, seed=6)
    L = walled(lat, shape, wa, beta, kappa, kw, storage=F64, collision=collision)
    L.set_populations(f0)
    L.step(3)
    got = L.get_populations()
    f, F = f0, None
    for _ in range(3):
        f, F = orc.step_multiphase_wall(lat, beta, f, kappa, kw, wa, F_prev=F, mode=collision)
    ep = werr(lat, got, f)
    print(f"FP64 walls, 3 steps: {ep:.2e} W")  # measured 1.5e-14 / 1.7e-14
    assert ep <= 1e-12, ep


def test_droplet_on_wall_400_steps_fp64():
    """A D2Q9 droplet settling on the lower wall (kappa_w = -0.05), FP64 on
    both sides: density and fluid velocity."""
    lat, nx, ny, beta, kappa, kw = 9, 48, 24, 0.5, 0.025, -0.05
    rho = synth.droplet_density((1, ny, nx), 8.0, center=(nx / 2, 0.0, 0.5), rho_l=7.5, rho_v=0.08)
    f = orc.init_equilibrium(lat, rho, np.zeros((2, 1, ny, nx)))
    L = walled(lat, (1, ny, nx), 1, beta, kappa, kw, storage=F64)
    L.set_populations(f)
    L.step(400)
    L.check()
    rg, ug = L.macros()
    F = None
    for _ in range(400):
        f, F = orc.step_multiphase_wall(lat, beta, f, kappa, kw, 1, F_prev=F)
    ro, uo = orc.macros_forced(lat, f, F)
    er = np.max(np.abs(rg - ro)) / np.max(ro)
    eu = np.max(np.abs(ug - uo[:2])) / np.max(np.abs(uo))
    # measured: density 5.5e-14, velocity 4.2e-13
    print(f"FP64 droplet on a wall, 400 steps: density {er:.2e}, velocity {eu:.2e}")
    assert er <= 1e-11 and eu <= 1e-9, (er, eu)


def test_droplet_on_wall_d3q27_fp32():
    """A D3Q27 droplet on the lower wall (wall axis y, kappa_w = +0.05),
    150 steps, FP32 against the FP64 oracle."""
    lat, shape, beta, kappa, kw = 27, (20, 16, 24), 0.6, 0.025, 0.05
    nz, ny, nx = shape
    rho = synth.droplet_density(shape, 6.0, center=(nx / 2, 0.0, nz / 2), rho_l=7.5, rho_v=0.08)
    f = orc.init_equilibrium(lat, rho, np.zeros((3,) + shape))
    L = walled(lat, shape, 1, beta, kappa, kw)
    L.set_populations(f)
    L.step(150)
    L.check()
    rg, ug = L.macros()
    F = None
    for _ in range(150):
        f, F = orc.step_multiphase_wall(lat, beta, f, kappa, kw, 1, F_prev=F)
    ro, uo = orc.macros_forced(lat, f, F)
    er = np.max(np.abs(rg - ro)) / np.max(ro)
    eu = np.max(np.abs(ug - uo)) / np.max(np.abs(uo))
    # measured: density 2.2e-6, velocity 1.8e-5
    print(f"D3Q27 droplet on a wall, 150 steps FP32: density {er:.2e}, velocity {eu:.2e}")
    assert er <= 1e-5 and eu <= 1e-4, (er, eu)


def test_wall_set_ups_rejected():
    from paper_1710_02375_gb300 import lbm as abi
    from paper_1710_02375_gb300.lbm import Lattice
    for bc, fu in (((1, 1, 1, 1, 0, 0), None),           # walls on two axes
                   ((2, 3, 0, 0, 0, 0), None),           # inlet / outlet
                   ((0, 0, 1, 1, 0, 0), [[0, 0, 0], [0, 0, 0], [0.01, 0, 0], [0, 0, 0],
                                         [0, 0, 0], [0, 0, 0]])):  # a moving wall
        L = Lattice(9, 16, 12, 1, 0.8, bc=bc, face_velocity=fu, multiphase=True)
        with pytest.raises(abi.LbmError) as e:
            L.set_multiphase(0.02, kappa_w=-0.1)
        assert e.value.status == abi.LBM_EINVAL
    L = Lattice(9, 16, 12, 1, 0.8, bc=(0, 0, 1, 1, 0, 0), multiphase=True)
    with pytest.raises(abi.LbmError):
        L.set_multiphase(0.02, kappa_w=float("inf"))
    L.set_multiphase(0.02, kappa_w=-0.1)
    L.step(2)
    L.check()
