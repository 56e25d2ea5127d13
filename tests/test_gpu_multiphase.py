"""Multiphase KBC step on the GPU (section "Extensions to fluid-structure
interaction in multiphase flow"; density pass, Laplacian pass and forced
sweep of multiphase.cu) against the FP64 oracle's step_multiphase, through
the C ABI (lbm_set_multiphase, lbm_get_force_field, lbm_get_macros).

Tolerances: FP32 storage and compute hold populations to ~1e-6 of W_i per
step (values up to 7.5 W_i in the liquid); FP64 storage to round-off."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1710_02375_gb300 import synth

pytestmark = pytest.mark.gpu
F32, F64 = 0, 3


def lattice(lat, shape, beta, kappa, storage=F32, eos=0, g=(0.0, 0.0, 0.0), collision=0):
    from paper_1710_02375_gb300.lbm import Lattice
    nz, ny, nx = shape
    L = Lattice(lat, nx, ny, nz, beta, storage=storage, collision=collision, multiphase=True)
    L.set_multiphase(kappa, eos, g)
    return L


def two_phase_state(lat, shape, seed, u_amp=0.02):
    """Droplet (circle / sphere) of liquid in vapour with random velocities,
    at equilibrium plus a random non-equilibrium part."""
    rng = np.random.default_rng(seed)
    R = 0.3 * min(s for s in shape if s > 1)
    rho = synth.droplet_density(shape, R, rho_l=7.5, rho_v=0.08, noise=1e-3, seed=seed)
    dim = 2 if lat == 9 else 3
    u = u_amp * rng.uniform(-1, 1, size=(dim,) + shape)
    f = orc.init_equilibrium(lat, rho, u)
    return f * (1 + 0.01 * rng.uniform(-1, 1, size=f.shape))


def werr(lat, a, b):
    w = synth.lattice_weights(lat).reshape((lat, 1, 1, 1))
    return np.max(np.abs(a - b) / w)


@pytest.mark.parametrize("lat,shape", [(9, (1, 37, 53)), (27, (13, 11, 17)), (27, (41, 12, 20))])
@pytest.mark.parametrize("collision", [0, 1])
def test_one_step_matches_oracle_fp32(lat, shape, collision):
    """One step from a random two-phase state on ragged sizes (not multiples
    of the CTA shape): every population, and the force field, against the
    oracle (nz = 41: the Laplacian pass that marches along z in columns of
    16, with a ragged last column).  Measured 2e-6 W (populations), 7e-7
    relative (force)."""
    beta, kappa = 0.8, 0.02
    f0 = two_phase_state(lat, shape, seed=5)
    L = lattice(lat, shape, beta, kappa, collision=collision)
    L.set_populations(f0)
    L.step(1)
    L.check()
    got = L.get_populations()
    Fg = L.force_field()
    ref, Fo = orc.step_multiphase(lat, beta, f0, kappa, mode=collision, want_force=True)
    ep = werr(lat, got, ref)
    ef = np.max(np.abs(Fg - Fo)) / np.max(np.abs(Fo))
    print(f"D{'2Q9' if lat == 9 else '3Q27'} one multiphase step ({'BGK' if collision else 'KBC'}): "
          f"populations {ep:.2e} W, force {ef:.2e}")
    assert ep <= 1e-5 and ef <= 1e-5, (ep, ef)


@pytest.mark.parametrize("collision", [0, 1])
def test_one_step_matches_oracle_fp64(collision):
    lat, shape, beta, kappa = 9, (1, 29, 31), 0.8, 0.02
    f0 = two_phase_state(lat, shape, seed=6)
    L = lattice(lat, shape, beta, kappa, storage=F64, collision=collision)
    L.set_populations(f0)
    L.step(1)
    got = L.get_populations()
    Fg = L.force_field()
    ref, Fo = orc.step_multiphase(lat, beta, f0, kappa, mode=collision, want_force=True)
    ep = werr(lat, got, ref)
    ef = np.max(np.abs(Fg - Fo)) / np.max(np.abs(Fo))
    print(f"FP64 one multiphase step: populations {ep:.2e} W, force {ef:.2e}")
    assert ep <= 1e-12 and ef <= 1e-12, (ep, ef)


def test_droplet_500_steps_fp64():
    """D2Q9 droplet relaxing for 500 steps, FP64 on both sides: density and
    fluid velocity (j - F/2)/rho."""
    lat, shape, beta, kappa = 9, (1, 40, 40), 0.6, 0.025
    rho0 = synth.droplet_density(shape, 10.0, rho_l=7.52)
    f = orc.init_equilibrium(lat, rho0, np.zeros((2,) + shape))
    L = lattice(lat, shape, beta, kappa, storage=F64)
    L.set_populations(f)
    L.step(500)
    L.check()
    rg, ug = L.macros()
    F = None
    for _ in range(500):
        f, F = orc.step_multiphase(lat, beta, f, kappa, want_force=True)
    ro, uo = orc.macros_forced(lat, f, F)
    er = np.max(np.abs(rg - ro)) / np.max(ro)
    eu = np.max(np.abs(ug - uo[:2])) / np.max(np.abs(uo))
    print(f"FP64 droplet 500 steps: density {er:.2e}, velocity {eu:.2e} (max|u| {np.abs(uo).max():.1e})")
    assert er <= 1e-11 and eu <= 1e-9, (er, eu)


@pytest.mark.parametrize("lat", [9, 27])
def test_flat_interface_2000_steps_fp32(lat):
    """A liquid slab relaxing to the coexisting densities over 2000 steps
    (the D3Q27 slab along z, a 1 x 1 cross-section: every neighbour in x and
    y is the node itself).  The position of the slab in the periodic box is
    a neutral mode: without the momentum controller of the multiphase sweep
    the FP32 rounding accelerated it by ~1e-9 per step and the profile was
    off by 8e-4 of rho_l after 2000 steps.  Measured: density 4.3e-6 (D2Q9)
    / 1.0e-6 (D3Q27) of rho_l, vapour density 2.8e-6, velocity 5e-7, mean
    velocity 4e-9."""
    n, kappa, beta = 60, 0.025, 0.5
    prof = synth.slab_density(n, rho_l=7.5, rho_v=0.13)
    shape = (1, 1, n) if lat == 9 else (n, 1, 1)
    dim = 2 if lat == 9 else 3
    f = orc.init_equilibrium(lat, prof.reshape(shape), np.zeros((dim,) + shape))
    L = lattice(lat, shape, beta, kappa)
    L.set_populations(f)
    L.step(2000)
    L.check()
    rg, ug = L.macros()
    F = None
    for _ in range(2000):
        f, F = orc.step_multiphase(lat, beta, f, kappa, want_force=True)
    ro, uo = orc.macros_forced(lat, f, F)
    # relative to the liquid density: at the interface nodes next to the
    # vapour (density gradient ~2 per node) a shift of the profile by 1e-4
    # node is 3e-3 of the local vapour density
    er = np.max(np.abs(rg - ro)) / np.max(ro)
    ev = abs(rg.min() - ro.min()) / ro.min()
    eu = np.max(np.abs(ug - uo[:dim]))
    # net momentum of the periodic box: zero in exact arithmetic (the force
    # sums to zero), so it measures the FP32 rounding that accumulates into
    # a translation of the slab
    P = np.abs((rg * ug).sum(axis=(1, 2, 3))).max() / rg.sum()
    print(f"flat interface 2000 steps: density {er:.2e} of rho_l, vapour density {ev:.2e}, "
          f"velocity {eu:.2e} (max|u| {np.abs(uo).max():.1e}), mean velocity {P:.1e}; "
          f"rho_v {rg.min():.5f} rho_l {rg.max():.4f}")
    assert er <= 3e-5 and ev <= 2e-5 and eu <= 3e-6 and P <= 1e-7, (er, ev, eu, P)


@pytest.mark.parametrize("lat", [9, 27])
def test_uniform_acceleration_closed_form(lat):
    """Uniform state under a uniform acceleration g: after s steps the
    populations are feq(rho, u0 + s g) (exact difference method)."""
    dim = 2 if lat == 9 else 3
    shape = (1, 8, 33) if lat == 9 else (5, 6, 33)
    rho = np.full(shape, 1.3)
    u0 = np.array([0.02, -0.01, 0.015])[:dim]
    g = (1e-3, 2e-3, -5e-4)
    ub = lambda u: np.broadcast_to(np.asarray(u).reshape((dim, 1, 1, 1)), (dim,) + shape)
    L = lattice(lat, shape, 0.9, 0.2, g=g)
    L.init_equilibrium(rho, np.ascontiguousarray(ub(u0)))
    L.step(10)
    got = L.get_populations()
    want = orc.init_equilibrium(lat, rho, ub(u0 + 10 * np.asarray(g)[:dim]))
    err = werr(lat, got, want)
    print(f"uniform acceleration 10 steps: {err:.2e} W")  # measured 0.9e-7 / 1.5e-7
    assert err <= 1e-6, err


@pytest.mark.parametrize("lat", [9, 27])
def test_single_node_box(lat):
    """The degenerate 1 x 1 (x 1) periodic box: all gradients vanish, the
    force is rho g; against the oracle's step."""
    shape = (1, 1, 1)
    f0 = synth.random_state(lat, shape, 0.05, seed=7)
    g = (0.04, -0.03, 0.02)
    L = lattice(lat, shape, 0.9, 0.0, eos=1, g=g)
    L.set_populations(f0)
    L.step(1)
    got = L.get_populations()
    ref = orc.step_multiphase(lat, 0.9, f0, 0.0, eos_kind=1, g_ext=np.array(g))
    err = werr(lat, got, ref)
    assert err <= 2e-6, err


def test_graph_replay_equals_direct_steps():
    lat, shape = 27, (12, 10, 14)
    f0 = two_phase_state(lat, shape, seed=9)
    A = lattice(lat, shape, 0.7, 0.02)
    B = lattice(lat, shape, 0.7, 0.02)
    A.set_populations(f0)
    B.set_populations(f0)
    A.step(6)
    B.step_graph(2, 3)
    assert np.array_equal(A.get_populations(), B.get_populations())


def test_multiphase_rejects_bad_set_ups():
    from paper_1710_02375_gb300 import lbm as abi
    from paper_1710_02375_gb300.lbm import Lattice
    L0 = Lattice(9, 8, 8, 1, 0.8)
    with pytest.raises(abi.LbmError) as e:     # no multiphase fields reserved
        L0.set_multiphase(0.02)
    assert e.value.status == abi.LBM_ESTATE
    with pytest.raises(abi.LbmError) as e:     # force field while the model is off
        L0.force_field()
    assert e.value.status == abi.LBM_ESTATE
    with pytest.raises(abi.LbmError):          # 16-bit storage
        Lattice(9, 8, 8, 1, 0.8, storage=1, multiphase=True)
    Lw = Lattice(9, 8, 8, 1, 0.8, bc=(2, 3, 0, 0, 0, 0), multiphase=True)
    with pytest.raises(abi.LbmError) as e:     # open faces (walls: tests/test_gpu_multiphase_walls.py)
        Lw.set_multiphase(0.02)
    assert e.value.status == abi.LBM_EINVAL
    L = Lattice(9, 8, 8, 1, 0.8, multiphase=True)
    for kw in (dict(kappa=-1.0), dict(kappa=0.02, eos=7), dict(kappa=float("nan"))):
        with pytest.raises(abi.LbmError) as e:
            L.set_multiphase(**kw)
        assert e.value.status == abi.LBM_EINVAL
    L.set_multiphase(0.02)
    x, el = synth.circle_polygon(4.0, 4.0, 1.5, 12)
    with pytest.raises(abi.LbmError) as e:     # immersed bodies
        L.set_geometry(x, el, np.zeros(len(el), np.int32))
    assert e.value.status == abi.LBM_EINVAL
    L.set_multiphase(None)                     # back to the single-phase step
    L.step(1)
    L.check()


def test_sampled_nodes_bench_size_d3q27():
    """The bench workload (D3Q27 droplet of diameter 80 in 320 x 250 x 320,
    FP32): two steps on the GPU, then density and fluid velocity at sampled
    nodes against the oracle run on the 13^3 periodic patch around each node
    (a node's value after two steps depends on nodes within distance 6)."""
    import torch
    lat, shape, beta, kappa, steps = 27, (320, 250, 320), 0.6, 0.025, 2
    nz, ny, nx = shape
    rho = synth.droplet_density(shape, 40.0, rho_l=7.5, rho_v=0.08, noise=1e-3, seed=3)
    L = lattice(lat, shape, beta, kappa)
    dev = L.device
    rho_d = torch.from_numpy(rho).to(dev)
    L.init_equilibrium(rho_d, torch.zeros((3,) + shape, dtype=torch.float64, device=dev))
    del rho_d
    L.step(steps)
    L.check()
    rg = torch.zeros(shape, dtype=torch.float64, device=dev)
    ug = torch.zeros((3,) + shape, dtype=torch.float64, device=dev)
    from paper_1710_02375_gb300 import lbm as abi
    abi.lbm_get_macros(L.ctx, rg, ug)
    rng = np.random.default_rng(11)
    # nodes on the interface (radius 40 around the centre) and in both bulks
    pts = []
    c = np.array([nx / 2, ny / 2, nz / 2]) - 0.5
    for r in (40.0, 40.0, 40.0, 20.0, 100.0, 0.0):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        p = np.round(c + r * d).astype(int) % np.array([nx, ny, nz])
        pts.append(tuple(int(v) for v in p))
    pts.append((0, 0, 0))
    pts.append((nx - 1, ny - 1, nz - 1))
    h = 3 * steps
    worst_r = worst_u = 0.0
    for (x, y, z) in pts:
        zi = np.arange(z - h, z + h + 1) % nz
        yi = np.arange(y - h, y + h + 1) % ny
        xi = np.arange(x - h, x + h + 1) % nx
        patch = rho[np.ix_(zi, yi, xi)]
        f = orc.init_equilibrium(lat, patch, np.zeros((3,) + patch.shape))
        F = None
        for _ in range(steps):
            f, F = orc.step_multiphase(lat, beta, f, kappa, want_force=True)
        ro, uo = orc.macros_forced(lat, f, F)
        r_o, u_o = ro[h, h, h], uo[:, h, h, h]
        r_g = float(rg[z, y, x])
        u_g = ug[:, z, y, x].cpu().numpy()
        worst_r = max(worst_r, abs(r_g - r_o) / r_o)
        worst_u = max(worst_u, np.max(np.abs(u_g - u_o)))
    # measured: density 9.2e-8 relative, velocity 5.9e-8
    print(f"bench-size sampled nodes ({len(pts)}): density {worst_r:.2e} relative, velocity {worst_u:.2e}")
    assert worst_r <= 1e-6 and worst_u <= 1e-6, (worst_r, worst_u)


def test_switching_the_model_keeps_the_state():
    """The multiphase step stores populations relative to the local density;
    switching the model off brings them back to the single-phase convention
    (and on again), reading the same populations each time."""
    lat, shape = 27, (9, 10, 11)
    f0 = two_phase_state(lat, shape, seed=4)
    L = lattice(lat, shape, 0.8, 0.02)
    L.set_populations(f0)
    L.step(5)
    a = L.get_populations()
    L.set_multiphase(None)
    b = L.get_populations()
    L.set_multiphase(0.02)
    c = L.get_populations()
    assert werr(lat, a, b) <= 2e-6 and werr(lat, b, c) == 0.0
