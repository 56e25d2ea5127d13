"""The allocation-free force probe (lbm_probe_interface_force_static) against
the regular path (lbm_step + lbm_get_interface_force).

The probe serves callers that cannot allocate device memory at the point
where they need the interface force (a device-memory budget fixed at
start-up, or a path that must not call cudaMalloc); its scratch lives in a
fixed device array inside the library.  This file is collected last on
purpose.  Tolerance: the force tolerance of the boundary tests (1e-4 relative
per body, 1e-4 of the largest vertex force per vertex); the two paths differ
only in the order of their FP64 atomic additions.
"""
import numpy as np
import pytest

from paper_1710_02375_gb300 import synth

pytestmark = pytest.mark.gpu


def test_probe_matches_next_step_force_twice():
    from paper_1710_02375_gb300 import lbm
    from paper_1710_02375_gb300.lbm import Lattice
    nx, ny = 220, 41
    u_max, Re, D = 0.05, 100.0, 10.0
    nu = (2.0 / 3.0) * u_max * D / Re
    beta = 1.0 / (6 * nu + 1)
    prof = synth.parabolic_profile(ny, u_max, noise=1e-4, seed=0)
    x, e, body, _ = synth.cylinder_flag_2d()
    L = Lattice(9, nx, ny, 1, beta, bc=(2, 3, 1, 1, 0, 0), max_links=4000, max_vertices=len(x),
                max_elements=len(e), inlet_ramp_steps=200)
    L.set_inlet_profile(0, prof)
    L.set_geometry(x, e, body)
    L.init_equilibrium(np.ones((1, ny, nx)), np.zeros((2, 1, ny, nx)))
    L.step(300)
    nb = int(body.max() + 1)
    for _ in range(2):
        vp = np.zeros((len(x), 3))
        bp = np.zeros((nb, 3))
        lbm.lbm_probe_interface_force_static(L.ctx, vp, bp)
        L.step(1)
        vf, bf = L.interface_force()
        for b in range(nb):
            assert np.linalg.norm(bp[b] - bf[b]) <= 1e-4 * np.linalg.norm(bf[b])
        assert np.max(np.abs(vp - vf)) <= 1e-4 * np.max(np.abs(vf))
        assert np.linalg.norm(bf[0]) > 0
    L.check()


def test_probe_matches_next_step_force_twice_d3q27():
    """D3Q27: a sphere in a channel with inlet, outlet, face walls and
    free-stream faces, so lbm_step fills face and immersed nodes in one split
    launch while the probe fills the immersed nodes alone."""
    from paper_1710_02375_gb300 import lbm
    from paper_1710_02375_gb300.lbm import Lattice
    nx, ny, nz = 36, 20, 18
    fu = np.zeros((6, 3))
    fu[0, 0] = fu[4, 0] = fu[5, 0] = 0.03
    x, e = synth.icosphere((12.3, 9.6, 8.7), 4.2, level=2)
    body = np.zeros(len(e), np.int32)
    L = Lattice(27, nx, ny, nz, 0.95, bc=(2, 3, 1, 1, 4, 4), face_velocity=fu, max_links=20000,
                max_vertices=len(x), max_elements=len(e), inlet_ramp_steps=50)
    L.set_geometry(x, e, body)
    L.init_equilibrium(np.ones((nz, ny, nx)), np.zeros((3, nz, ny, nx)))
    L.step(100)
    for _ in range(2):
        vp = np.zeros((len(x), 3))
        bp = np.zeros((1, 3))
        lbm.lbm_probe_interface_force_static(L.ctx, vp, bp)
        L.step(1)
        vf, bf = L.interface_force()
        assert np.linalg.norm(bf[0]) > 0
        assert np.linalg.norm(bp[0] - bf[0]) <= 1e-4 * np.linalg.norm(bf[0])
        assert np.max(np.abs(vp - vf)) <= 1e-4 * np.max(np.abs(vf))
    L.check()
