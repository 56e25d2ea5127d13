"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each check uses an independent route: a Newton solve of the constrained
entropy minimisation (Eqs. feq_min, conservationLaws), a moment-matrix
inversion for the k/s/h split (Eq. popSplit), a parabola fitted to the
quadratic entropy norm for gamma (Eq. gamma_min_approx), a numpy brute-force
step built from those pieces, conservation laws, lattice symmetry and the
closed-form Taylor-Green decay that Eq. (visc) implies.
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1710_02375_gb300 import synth


# ---------------------------------------------------------------- helpers
def newton_equilibrium(c, w, rho, u, dim):
    """Constrained minimiser of H = sum f ln(f/W): f_i = W_i exp(a + lam.c_i),
    with (a, lam) from Newton's method on the mass/momentum constraints."""
    cc = c[:, :dim].astype(float)
    x = np.zeros(1 + dim)
    target = np.concatenate([[rho], rho * np.asarray(u[:dim])])
    A = np.concatenate([np.ones((len(w), 1)), cc], axis=1)
    for _ in range(100):
        f = w * np.exp(A @ x)
        r = A.T @ f - target
        if np.max(np.abs(r)) < 1e-17:
            break
        J = A.T @ (f[:, None] * A)
        x -= np.linalg.solve(J, r)
    return w * np.exp(A @ x)


def moment_matrix(c, dim):
    """Rows: natural moments M_pqr (p,q,r in 0..2) re-based so the second-order
    diagonal block is (trace, N_xz, N_yz) [3-D] or (trace, N) [2-D].
    Returns (M, names) with names tagging 'k', 's' or 'h'."""
    rows, tags = [], []
    rng = range(3)
    combos = [p for p in itertools.product(rng, repeat=dim)]
    cf = c[:, :dim].astype(float)
    by = {}
    for pqr in combos:
        by[pqr] = np.prod([cf[:, a] ** pqr[a] for a in range(dim)], axis=0)
    if dim == 2:
        diag = [(2, 0), (0, 2)]
        for pqr in combos:
            if pqr in diag:
                continue
            rows.append(by[pqr])
            order = sum(pqr)
            tags.append("k" if order <= 1 else ("s" if pqr == (1, 1) else "h"))
        rows += [by[(2, 0)] + by[(0, 2)], by[(2, 0)] - by[(0, 2)]]
        tags += ["h", "s"]
    else:
        diag = [(2, 0, 0), (0, 2, 0), (0, 0, 2)]
        for pqr in combos:
            if pqr in diag:
                continue
            rows.append(by[pqr])
            order = sum(pqr)
            is_shear = order == 2 and max(pqr) == 1
            tags.append("k" if order <= 1 else ("s" if is_shear else "h"))
        rows += [by[(2, 0, 0)] + by[(0, 2, 0)] + by[(0, 0, 2)],
                 by[(2, 0, 0)] - by[(0, 0, 2)], by[(0, 2, 0)] - by[(0, 0, 2)]]
        tags += ["h", "s", "s"]
    return np.array(rows), np.array(tags)


def part(M, tags, f, which):
    """Population carrying only the natural moments tagged `which` of f."""
    m = M @ f
    m = np.where(tags == which, m, 0.0)
    return np.linalg.solve(M, m)


def parabola_argmin(qfun):
    """Vertex of the parabola through q(0), q(1), q(2) (exact for a quadratic)."""
    q0, q1, q2 = qfun(0.0), qfun(1.0), qfun(2.0)
    a = (q0 - 2 * q1 + q2) / 2.0
    b = (q1 - q0) - a
    return -b / (2 * a)


def bounded_argmin(qfun, lo, hi):
    """Minimiser of a convex quadratic over [lo, hi]: its vertex if inside,
    else the end point with the smaller value (compared, not assumed)."""
    g = parabola_argmin(qfun)
    if lo <= g <= hi:
        return g
    return lo if qfun(lo) <= qfun(hi) else hi


LATS = [(9, 2), (27, 3)]


# ---------------------------------------------------------------- lattice
@pytest.mark.parametrize("lat,dim", LATS)
def test_lattice_isotropy(lat, dim):
    c, w = orc.lattice(lat)
    cs2 = 1.0 / 3.0
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(w @ c, 0, atol=1e-16)
    M2 = np.einsum("i,ia,ib->ab", w, c, c)[:dim, :dim]
    assert np.allclose(M2, cs2 * np.eye(dim), atol=1e-15)
    M4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)[:dim, :dim, :dim, :dim]
    d = np.eye(dim)
    iso = cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(M4, iso, atol=1e-15)
    # opposite direction is Q-1-i
    assert np.array_equal(c[::-1], -c)


# ---------------------------------------------------------------- equilibrium
@pytest.mark.parametrize("lat,dim", LATS)
def test_equilibrium_is_entropy_minimiser(lat, dim):
    c, w = orc.lattice(lat)
    rng = np.random.default_rng(1)
    for _ in range(50):
        rho = rng.uniform(0.5, 2.0)
        u = np.zeros(3)
        u[:dim] = rng.uniform(-0.3, 0.3, size=dim)
        feq = orc.equilibrium(lat, rho, u)
        ref = newton_equilibrium(c, w, rho, u, dim)
        assert np.max(np.abs(feq - ref)) <= 1e-13 * rho
        # conservation laws, Eq. (conservationLaws)
        assert abs(feq.sum() - rho) < 1e-14
        assert np.allclose(feq @ c[:, :dim], rho * u[:dim], atol=1e-14)


# ---------------------------------------------------------------- split / gamma
@pytest.mark.parametrize("lat,dim", LATS)
def test_shear_part_matches_moment_inversion(lat, dim):
    c, w = orc.lattice(lat)
    M, tags = moment_matrix(c, dim)
    for seed in range(10):
        f = synth.random_state(lat, (1,), 0.05, seed)[:, 0]
        _, _, ds, dh, feq = orc.collide(lat, 0.9, f)
        df = f - feq
        ds_ref = part(M, tags, df, "s")
        dh_ref = part(M, tags, df, "h")
        assert np.max(np.abs(ds - ds_ref)) < 1e-14
        assert np.max(np.abs(dh - dh_ref)) < 1e-14
        # the kinematic part of df vanishes (conserved moments)
        assert np.max(np.abs(part(M, tags, df, "k"))) < 1e-14


@pytest.mark.parametrize("lat,dim", LATS)
def test_gamma_is_argmin_of_quadratic_entropy(lat, dim):
    c, w = orc.lattice(lat)
    M, tags = moment_matrix(c, dim)
    beta = 0.97
    for seed in range(10):
        f = synth.random_state(lat, (1,), 0.02, 100 + seed)[:, 0]
        fpost, gamma, _, _, _ = orc.collide(lat, beta, f)
        rho = f.sum()
        u = (f @ c) / rho
        feq = newton_equilibrium(c, w, rho, u, dim)
        df = f - feq
        ds, dh = part(M, tags, df, "s"), part(M, tags, df, "h")

        def qnorm(g):
            fp = f - beta * (2 * ds + g * dh)
            return np.sum((fp - feq) ** 2 / feq)

        g_ref = parabola_argmin(qnorm)
        assert abs(gamma - g_ref) < 1e-9 * max(1.0, abs(g_ref))


@pytest.mark.parametrize("lat,dim", LATS)
@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_gamma_outside_the_non_growing_range_is_the_bounded_argmin(lat, dim, sign):
    """A state built with a large shear part and a small higher-order part
    correlated (sign -1) or anti-correlated (sign +1) with it in the
    1/feq-weighted product puts the vertex of the quadratic entropy norm
    outside [0, 2/beta], where (1 - beta gamma) dh would grow; gamma is then
    the norm's minimiser over that range, found here by a scan of the range."""
    c, w = orc.lattice(lat)
    M, tags = moment_matrix(c, dim)
    beta = 0.97
    f0 = synth.random_state(lat, (1,), 0.02, 321)[:, 0]
    rho = f0.sum()
    feq = newton_equilibrium(c, w, rho, (f0 @ c) / rho, dim)
    ds0, dh0 = part(M, tags, f0 - feq, "s"), part(M, tags, f0 - feq, "h")
    ip, hh = np.sum(ds0 * dh0 / feq), np.sum(dh0 * dh0 / feq)
    # f = feq + ds0 + b dh0: the vertex is 1/beta - (2 - 1/beta) ip / (b hh);
    # b is chosen to put it one unit beyond the range
    target = 2.0 / beta + 1.0 if sign > 0 else -1.0
    b = (2.0 - 1.0 / beta) * ip / (hh * (1.0 / beta - target))
    f = feq + ds0 + b * dh0
    assert np.all(f > 0)
    fpost, gamma, ds, dh, _ = orc.collide(lat, beta, f)

    def qnorm(g):
        fp = f - beta * (2 * ds + g * dh)
        return np.sum((fp - feq) ** 2 / feq)

    vertex = parabola_argmin(qnorm)
    assert vertex > 2.0 / beta if sign > 0 else vertex < 0.0, vertex
    grid = np.linspace(0.0, 2.0 / beta, 20001)
    g_scan = grid[np.argmin([qnorm(g) for g in grid])]
    assert gamma == (2.0 / beta if sign > 0 else 0.0)
    assert abs(gamma - g_scan) < 2e-4
    np.testing.assert_allclose(fpost, f - beta * (2 * ds + gamma * dh), rtol=0, atol=1e-15)


@pytest.mark.parametrize("lat,dim", LATS)
def test_gamma_approximates_entropy_argmin_near_equilibrium(lat, dim):
    """Eq. (gamma_min_approx) is the small-deviation estimate of the gamma that
    minimises H(f') itself; the two approach each other as f -> feq."""
    from scipy.optimize import minimize_scalar

    c, w = orc.lattice(lat)
    beta = 0.95
    errs = []
    for amp in (1e-2, 1e-3):
        f = synth.random_state(lat, (1,), amp, 7)[:, 0]
        _, gamma, ds, dh, _ = orc.collide(lat, beta, f)

        def H(g):
            fp = f - beta * (2 * ds + g * dh)
            return np.sum(fp * np.log(fp / w))

        res = minimize_scalar(H, bracket=(gamma - 0.5, gamma + 0.5), tol=1e-12)
        errs.append(abs(res.x - gamma))
    assert errs[0] / errs[1] > 5.0  # first-order approach as the deviation shrinks
    assert errs[1] < 2e-4


@pytest.mark.parametrize("lat,dim", LATS)
def test_gamma_two_is_lbgk(lat, dim):
    """gamma = 2 turns Eq. (f_mirr) into plain LBGK with omega = 2 beta."""
    c, w = orc.lattice(lat)
    beta = 0.8
    for seed in range(5):
        f = synth.random_state(lat, (1,), 0.05, 200 + seed)[:, 0]
        fpost, gamma, _, _, _ = orc.collide(lat, beta, f, mode=1)
        assert gamma == 2.0
        rho = f.sum()
        feq = newton_equilibrium(c, w, rho, (f @ c) / rho, dim)
        ref = f + 2 * beta * (feq - f)
        assert np.max(np.abs(fpost - ref)) < 1e-14


# ---------------------------------------------------------------- whole step
def brute_force_step(lat, dim, beta, f):
    """Numpy step: np.roll pull-stream, Newton equilibrium, k/s/h parts from the
    moment matrix, gamma from the parabola of the entropy norm, then Eqs.
    (f_mirr) and (f_equations) on the parts."""
    c, w = orc.lattice(lat)
    M, tags = moment_matrix(c, dim)
    fs = np.empty_like(f)
    for i in range(lat):
        fs[i] = np.roll(f[i], shift=(int(c[i, 2]), int(c[i, 1]), int(c[i, 0])), axis=(0, 1, 2))
    out = np.empty_like(f)
    Q, nz, ny, nx = f.shape
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        fi = fs[:, z, y, x]
        rho = fi.sum()
        feq = newton_equilibrium(c, w, rho, (fi @ c) / rho, dim)
        k, s, h = part(M, tags, fi, "k"), part(M, tags, fi, "s"), part(M, tags, fi, "h")
        seq, heq = part(M, tags, feq, "s"), part(M, tags, feq, "h")

        def mirr(g):
            return k + (2 * seq - s) + ((1 - g) * h + g * heq)

        def qnorm(g):
            fp = (1 - beta) * fi + beta * mirr(g)
            return np.sum((fp - feq) ** 2 / feq)

        g = bounded_argmin(qnorm, 0.0, 2.0 / beta)
        out[:, z, y, x] = (1 - beta) * fi + beta * mirr(g)
    return out


@pytest.mark.parametrize("lat,dim,shape", [(9, 2, (1, 5, 4)), (27, 3, (3, 4, 5))])
def test_step_matches_brute_force(lat, dim, shape):
    f = synth.random_state(lat, shape, 0.03, 11)
    beta = 0.93
    got = orc.step_periodic(lat, beta, f)
    ref = brute_force_step(lat, dim, beta, f)
    assert np.max(np.abs(got - ref)) < 2e-13


@pytest.mark.parametrize("lat,shape", [(9, (1, 12, 10)), (27, (5, 6, 7))])
def test_conservation_over_many_steps(lat, shape):
    f = synth.random_state(lat, shape, 0.05, 5)
    c, _ = orc.lattice(lat)
    m0 = f.sum()
    j0 = f.reshape(lat, -1).sum(axis=1) @ c
    g = orc.run_periodic(lat, 0.99, f, 100)
    assert abs(g.sum() - m0) / m0 < 1e-13
    j1 = g.reshape(lat, -1).sum(axis=1) @ c
    assert np.max(np.abs(j1 - j0)) < 1e-12 * m0


def test_rotation_symmetry_d3q27():
    """A 90-degree rotation about z commutes with the step."""
    lat = 27
    c, _ = orc.lattice(lat)
    N = 6
    f = synth.random_state(lat, (4, N, N), 0.04, 3)
    # rotation (x, y) -> (-y, x): direction i -> j with c_j = R c_i
    R = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]])
    perm = [int(np.where((c == R @ c[i]).all(axis=1))[0][0]) for i in range(lat)]

    def rot(g):
        out = np.empty_like(g)
        for i in range(lat):
            # new(x', y') = old(x, y) with x' = -y, y' = x  (mod N)
            src = g[i]
            dst = np.empty_like(src)
            for y in range(N):
                for x in range(N):
                    dst[:, x % N, (-y) % N] = src[:, y, x]
            out[perm[i]] = dst
        return out

    a = orc.step_periodic(lat, 0.97, rot(f))
    b = rot(orc.step_periodic(lat, 0.97, f))
    assert np.max(np.abs(a - b)) < 1e-14


# ---------------------------------------------------------------- viscosity
@pytest.mark.parametrize("lat", [9, 27])
def test_taylor_green_decay_gives_eq_visc(lat):
    """2-D Taylor-Green vortex: kinetic energy decays as exp(-4 nu k^2 t) with
    nu = c_s^2 (1/(2 beta) - 1/2), Eq. (visc); the error falls at second order."""
    nu = 0.02
    beta = 1.0 / (6 * nu + 1.0)
    errs = []
    for N in (16, 32):
        rho, u = synth.tgv_fields(N, N, 1, 1e-3, three_d=False)
        f = orc.init_equilibrium(lat, rho, u[: (2 if lat == 9 else 3)])
        k = 2 * np.pi / N
        t1 = int(round(0.1 / (4 * nu * k * k)))
        t2 = int(round(0.6 / (4 * nu * k * k)))
        f1 = orc.run_periodic(lat, beta, f, t1)
        f2 = orc.run_periodic(lat, beta, f1, t2 - t1)

        def ek(g):
            r, uu = orc.macros(lat, g)
            return np.sum(r * (uu ** 2).sum(axis=0))

        nu_fit = -np.log(ek(f2) / ek(f1)) / (4 * k * k * (t2 - t1))
        errs.append(abs(nu_fit - nu) / nu)
    assert errs[1] < 2e-3
    assert errs[0] / errs[1] > 3.0  # second order
