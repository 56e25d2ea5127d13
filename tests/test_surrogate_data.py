"""Surrogate training pairs from a coupled oracle run (CPU): the input blocks
are the out-of-balance nodal loads and the state, and each target is the
oracle's structural step -- the theta-scheme residual (section "Structural
modeling") at u + dt v + target vanishes to the Newton tolerance."""
import numpy as np

from oracle import surrogate_data as sd
from oracle.fsi_oracle import nodal_loads
from tests import c1_flag_case as c1
from tests import plate_case


def test_pairs_are_oracle_structural_steps():
    steps = 40
    css = c1.oracle_run(150.0, seed=3)
    ref = c1.oracle_run(150.0, seed=3)
    X, Y, tip = sd.pairs_from_run(css, steps)
    beam = ref.beam
    nn, nr = beam.nn, ref.x_rigid.shape[0]
    nf = 3 * nn - 3
    assert X.shape == (steps, 15 * nn - 15) and Y.shape == (steps, nf)
    M = beam.mass()
    free = beam.fixed == 0
    loads = []
    for t in range(steps):
        u0, v0, F0 = ref.u.copy(), ref.v.copy(), ref.F0.copy()
        ref.step()
        F1 = nodal_loads(beam.X, u0, None, ref.vforce[nr:])
        loads.append(F1)
        f0, _ = beam.internal(u0, want_K=False)
        for k in range(3):
            Fk = loads[t - k] if t - k >= 0 else np.zeros(3 * nn)
            np.testing.assert_allclose(X[t, k * nf:(k + 1) * nf], Fk[3:] - f0[3:], rtol=0, atol=1e-15)
        np.testing.assert_array_equal(X[t, 3 * nf:4 * nf], u0[3:])
        np.testing.assert_array_equal(X[t, 4 * nf:], v0[3:])
        # theta = 1/2 residual of the step at the target
        u1 = u0.copy()
        u1[3:] += v0[3:] + Y[t]
        f1, _ = beam.internal(u1, want_K=False)
        v1 = 2.0 * (u1 - u0) - v0
        R = M @ (v1 - v0) - 0.5 * (F1 - f1) - 0.5 * (F0 - f0)
        R0 = M @ (-2.0 * v0) - 0.5 * (F1 - f0) - 0.5 * (F0 - f0)
        assert np.linalg.norm(R[free]) <= 1e-9 * max(np.linalg.norm(R0[free]), 1e-30) + 1e-12
        np.testing.assert_array_equal(tip[t], ref.u[-3:])


def test_plate_pairs_are_oracle_shell_steps():
    """Plate pairs: the blocks are the loads against the internal force, the
    state and the velocities on the free DOFs; the rotation-vector block and
    the rotational target agree with scipy's rotation vectors, the target
    rebuilds the oracle's step exactly, and the theta-scheme residual at the
    rebuilt state vanishes to the Newton tolerance."""
    from scipy.spatial.transform import Rotation
    steps = 6
    css, ref = plate_case.oracle_run(), plate_case.oracle_run()
    X, Y = sd.pairs_from_plate_run(css, steps)
    shell = ref.shell
    nn = shell.nn
    free = shell.fixed == 0
    nf = int(free.sum())
    assert nf == 6 * (nn - shell.ny)
    assert X.shape == (steps, 5 * nf) and Y.shape == (steps, nf)
    m, J = shell.mass()
    mass = np.stack([m, m, m, J, J, J], axis=1).ravel()
    loads = []
    for t in range(steps):
        u0, R0, v0, F0 = ref.u.copy(), ref.R.copy(), ref.v.copy(), ref.F0.copy()
        ref.step()
        F1 = np.zeros((nn, 6))
        F1[:, :3] = ref.vforce[:nn] + ref.vforce[nn:]
        loads.append(F1)
        f0 = shell.internal(u0, R0)
        for k in range(3):
            Fk = loads[t - k] if t - k >= 0 else np.zeros((nn, 6))
            np.testing.assert_allclose(X[t, k * nf:(k + 1) * nf], (Fk - f0).ravel()[free], rtol=0,
                                       atol=1e-15)
        phi = Rotation.from_matrix(R0).as_rotvec()
        q = np.concatenate([u0, phi], axis=1).ravel()[free]
        np.testing.assert_allclose(X[t, 3 * nf:4 * nf], q, rtol=0, atol=1e-13)
        np.testing.assert_array_equal(X[t, 4 * nf:], v0.ravel()[free])
        # the target rebuilds the step: translations and exp(phi) R0
        inc = np.zeros(6 * nn)
        inc[free] = Y[t] + v0.ravel()[free]
        inc = inc.reshape(nn, 6)
        np.testing.assert_allclose(u0 + inc[:, :3], ref.u, rtol=0, atol=1e-13)
        R1 = Rotation.from_rotvec(inc[:, 3:]).as_matrix() @ R0
        np.testing.assert_allclose(R1, ref.R, rtol=0, atol=1e-12)
        # theta = 1/2 residual at the rebuilt state (lumped mass, dt = 1)
        f1 = shell.internal(ref.u, ref.R)
        v1 = 2.0 * inc.ravel() - v0.ravel()
        Rv = mass * (v1 - v0.ravel()) - 0.5 * (F1 - f1).ravel() - 0.5 * (F0 - f0).ravel()
        Rs = mass * (-2.0 * v0.ravel()) - 0.5 * (F1 - f0).ravel() - 0.5 * (F0 - f0).ravel()
        assert np.linalg.norm(Rv[free]) <= 1e-9 * np.linalg.norm(Rs[free]) + 1e-12, t
