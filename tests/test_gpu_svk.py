"""The St Venant-Kirchhoff Q2 continuum on the GPU (csrc/fem_svk.cu: one
cooperative launch per theta step, Newton with the Gateaux tangent, Jacobi
CG on element products in FP32 or FP64) against the oracle (oracle/svk_oracle.py), through
the C ABI (fem_svk_*)."""
import numpy as np
import pytest

from oracle import svk_oracle as so
from paper_1710_02375_gb300 import synth

pytestmark = pytest.mark.gpu


def _solid(X, conn, fixed, **kw):
    from paper_1710_02375_gb300.lbm import SvkSolid
    return SvkSolid(X, conn, fixed=fixed.astype(np.int32), **kw)


def _distorted(n, L):
    dim = len(n)

    def dist(Y):
        s = np.prod([np.sin(np.pi * Y[:, d] / L[d]) for d in range(dim)], axis=0)
        return Y + 0.15 * s[:, None] * np.array([1.0, -0.7, 0.5][:dim]) * min(L)

    return synth.q2_box_mesh(n, L, distort=dist)


@pytest.mark.parametrize("dim", [2, 3])
def test_body_load_matches_oracle(dim):
    X, conn = _distorted([3, 2] if dim == 2 else [2, 2, 2], [3.0, 1.0] if dim == 2 else [2.0, 1.0, 1.5])
    fixed = np.zeros(X.size, bool)
    b = np.array([0.3, -2.0, 0.7])[:dim]
    G = _solid(X, conn, fixed, E=1e3, nu=0.3, rho=2.5, dt=0.01)
    O = so.SVK(X, conn, 1e3, 0.3, 2.5, fixed)
    got, ref = G.body_load(b), O.body_load(b)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    G.close()


@pytest.mark.parametrize("solve_fp64", [False, True])
def test_csm3_steps_match_oracle(solve_fp64):
    """CSM3 (20 x 2 plane-strain Q2 elements, gravity from rest, dt = 10 ms,
    theta = 1/2, lambda = 0.7), 40 steps: displacement and velocity.  Newton
    to |G| <= 1e-10 |G_0| (the round-off floor of this thin flag is near
    1e-11)."""
    E, nu, rho, g, L, h, dt = 1.4e6, 0.4, 1e3, 2.0, 0.35, 0.02, 0.01
    X, conn = synth.q2_box_mesh([20, 2], [L, h], origin=[0.0, -h / 2])
    fixed = np.repeat(X[:, 0] < 1e-12, 2)
    kw = dict(rtol=1e-10, atol=1e-16)
    G = _solid(X, conn, fixed, E=E, nu=nu, rho=rho, dt=dt, solve_fp64=solve_fp64, **kw)
    O = so.SVK(X, conn, E, nu, rho, fixed, **kw)
    F = O.body_load([0.0, -g])
    Fg = G.body_load([0.0, -g])
    G.set_state(F0=Fg)  # gravity acts from t = 0 (the oracle's F0 = F)
    u, v = np.zeros(X.size), np.zeros(X.size)
    worst_u = worst_v = 0.0
    for k in range(40):
        G.step(Fg)
        u, v, it = O.step(u, v, F, F, dt)
        ug, vg, (itg, cg) = G.state()
        assert itg >= 0 and it >= 0
        worst_u = max(worst_u, np.abs(ug - u).max() / np.abs(u).max())
        worst_v = max(worst_v, np.abs(vg - v).max() / np.abs(v).max())
    print(f"CSM3 40 steps: displacement {worst_u:.2e}, velocity {worst_v:.2e} (relative to the max); "
          f"last step Newton {itg} (oracle {it}), CG {cg}")
    assert worst_u <= 1e-8 and worst_v <= 1e-7, (worst_u, worst_v)
    G.close()


@pytest.mark.parametrize("solve_fp64", [False, True])
def test_3d_hex_cantilever_large_deflection_matches_oracle(solve_fp64):
    """Distorted 27-node hexahedra (4 x 2 x 2), clamped face, a tip load large
    enough for a finite rotation of the end, theta = 0.6, 12 steps."""
    E, nu, rho, dt = 2e3, 0.3, 1.0, 0.05
    X, conn = _distorted([4, 2, 2], [4.0, 1.0, 1.0])
    fixed = np.repeat(X[:, 0] < 1e-12, 3)
    kw = dict(theta=0.6, rtol=1e-12, atol=1e-16)
    G = _solid(X, conn, fixed, E=E, nu=nu, rho=rho, dt=dt, solve_fp64=solve_fp64, **kw)
    O = so.SVK(X, conn, E, nu, rho, fixed, **kw)
    F = O.body_load([0.0, -0.5, 0.2])
    tip = np.abs(X[:, 0] - 4.0) < 1e-12
    F.reshape(-1, 3)[tip, 1] -= 4.0 / tip.sum()
    u, v = np.zeros(X.size), np.zeros(X.size)
    F0 = np.zeros(X.size)
    for k in range(12):
        G.step(F)
        u, v, it = O.step(u, v, F0, F, dt)
        F0 = F
    ug, vg, (itg, cg) = G.state()
    eu = np.abs(ug - u).max() / np.abs(u).max()
    ev = np.abs(vg - v).max() / np.abs(v).max()
    print(f"3-D hexahedra, 12 steps: tip deflection {-u.reshape(-1, 3)[tip, 1].mean():.3f}; "
          f"displacement {eu:.2e}, velocity {ev:.2e}; Newton {itg} (oracle {it}), CG {cg}")
    assert u.reshape(-1, 3)[tip, 1].mean() < -0.5  # a large deflection of the 4-long bar
    assert eu <= 1e-9 and ev <= 1e-8, (eu, ev)
    G.close()


def test_set_state_and_rejections():
    from paper_1710_02375_gb300 import lbm as abi
    X, conn = synth.q2_box_mesh([2, 1], [2.0, 1.0])
    fixed = np.repeat(X[:, 0] < 1e-12, 2)
    with pytest.raises(abi.LbmError):
        _solid(X, conn[:, [2, 1, 0, 5, 4, 3, 8, 7, 6]].copy(), fixed, E=1.0, nu=0.3,
               rho=1.0)                                                     # mirrored: inverted
    bad = conn.copy()
    bad[0, 0] = len(X)
    with pytest.raises(abi.LbmError):
        _solid(X, bad, fixed, E=1.0, nu=0.3, rho=1.0)                       # node out of range
    with pytest.raises(abi.LbmError):
        _solid(X, conn, fixed, E=1.0, nu=0.5, rho=1.0)                      # nu = 1/2
    G = _solid(X, conn, fixed, E=1e3, nu=0.3, rho=1.0, dt=0.1)
    rng = np.random.default_rng(0)
    u = 0.01 * rng.standard_normal(X.size) * ~fixed
    v = 0.1 * rng.standard_normal(X.size) * ~fixed
    G.set_state(u, v, np.zeros(X.size))
    ug, vg, _ = G.state()
    assert np.array_equal(ug, u) and np.array_equal(vg, v)
    O = so.SVK(X, conn, 1e3, 0.3, 1.0, fixed)
    G.step(np.zeros(X.size))
    uo, vo, _ = O.step(u, v, np.zeros(X.size), np.zeros(X.size), 0.1)
    ug, vg, _ = G.state()
    assert np.abs(ug - uo).max() <= 1e-9 * np.abs(uo).max()
    G.close()
