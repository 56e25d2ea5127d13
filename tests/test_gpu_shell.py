"""GPU co-rotational flat shell (FP64, cooperative launch, conjugate-gradient
tangent solves) against the oracle shell under prescribed loads: the plate
of the crossflow case (40 x 20 x 2 cells, 16 x 8 elements, clamped leading
edge, rho_s / rho_f = 20, bending number 1e-4) driven into large deflection."""
import numpy as np
import pytest

from oracle import oracle as orc

pytestmark = pytest.mark.gpu


def plate(nx=17, ny=9, L=40.0, b=20.0):
    xs = np.linspace(0.0, L, nx)
    ys = np.linspace(-b / 2, b / 2, ny)
    X = np.array([[x, y, 0.0] for x in xs for y in ys])
    fixed = np.zeros(6 * nx * ny, np.int32)
    fixed[: 6 * ny] = 1
    return X, fixed


def test_shell_prescribed_loads_matches_oracle():
    from paper_1710_02375_gb300.lbm import Shell
    nx, ny = 17, 9
    X, fixed = plate(nx, ny)
    E, nu, h, rho = 0.0129, 0.4, 2.0, 20.0
    args = (X, nx, ny, E, nu, h, rho, fixed)
    gs = Shell(*args, atol=1e-12)
    os_ = orc.Shell(*args)
    u, R, v = os_.rest()
    F0 = np.zeros((nx * ny, 6))
    s = X[:, 0] / 40.0
    worst, its = 0.0, []
    for t in range(120):
        F1 = np.zeros((nx * ny, 6))
        F1[:, 2] = 0.08 * s * (1.0 + 0.5 * np.sin(0.05 * t))   # pressure-like, growing with x
        F1[:, 0] = 0.01 * s
        F1[:, 1] = 0.01 * np.sin(0.1 * t) * (X[:, 1] / 10.0)
        gs.step(F1)
        u, R, v, it = os_.step(u, R, v, F0, F1, atol=1e-12)
        F0 = F1
        ug, Rg, vg, (itg, ncg) = gs.state()
        assert it >= 0 and itg >= 0, (it, itg)
        its.append((it, itg, ncg))
        worst = max(worst, np.max(np.abs(ug - u)) / max(np.max(np.abs(u)), 1e-30),
                    np.max(np.abs(Rg - R)))
    print("SHELL iterations (oracle, gpu, cg) first/last:", its[0], its[-1], "worst", worst)
    assert worst < 1e-7, worst
    assert np.max(np.abs(u[:, 2])) > 2.0  # tip deflection of several lattice units
