"""Pins of the oracle's two-level grid refinement (D2Q9; the multi-domain
refinement of the validation cases, whose algorithm the paper cites without
printing it; reading in oracle/kbc_oracle.c, or_refine_step):

- a uniform flow stays uniform to the O(u^3) truncation of Grad's
  approximation (the error grows 8-fold when u doubles);
- a Taylor-Green vortex with the fine patch over the middle of the box
  decays at the rate of the single coarse grid (no extra dissipation at the
  interface), its error against the analytic solution stays within that of
  the coarse grid and falls at second order between 32^2 and 64^2;
- mass is conserved to the interface truncation (the transfers are not
  conservative by construction)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1710_02375_gb300 import synth


def tgv_case(n, U0):
    rc, uc = synth.tgv_fields(n, n, 1, U0, three_d=False)
    rf, uf = synth.tgv_fields(2 * n, 2 * n, 1, U0, three_d=False)
    i0 = j0 = n // 4
    fc = orc.init_equilibrium(9, rc, uc[:2])
    ffull = orc.init_equilibrium(9, rf, uf[:2])
    sl = (slice(None), slice(None), slice(2 * j0, 2 * j0 + n), slice(2 * i0, 2 * i0 + n))
    return fc, ffull[sl].copy(), ffull, uc[:2], uf[:2][sl], i0, j0


def run(n, steps, nu_c=0.01, U0=0.03):
    beta_c = 1 / (6 * nu_c + 1)
    fc, ff, _, uc, ufp, i0, j0 = tgv_case(n, U0)
    fco = fc.copy()
    m0 = fc.sum()
    for _ in range(steps):
        fc, ff = orc.refine_step(beta_c, fc, ff, i0, j0)
        fco = orc.step_periodic(9, beta_c, fco)
    dec = np.exp(-2 * nu_c * (2 * np.pi / n) ** 2 * steps)
    mask = np.ones((n, n), bool)
    mask[j0:j0 + n // 2, i0:i0 + n // 2] = False
    _, ur = orc.macros(9, fc)
    _, uo = orc.macros(9, fco)
    _, ufr = orc.macros(9, ff)
    err_ref = max(np.abs(ur[:2] - uc * dec)[:, 0][:, mask].max(), np.abs(ufr[:2] - ufp * dec).max())
    err_coarse = np.abs(uo[:2] - uc * dec).max()
    k = 2 * np.pi / n
    amp = lambda u: np.sum(u[:2, 0][:, mask] * uc[:, 0][:, mask]) / np.sum(uc[:, 0][:, mask] ** 2)
    rate_ref = -np.log(amp(ur)) / steps / (2 * nu_c * k * k)
    rate_coarse = -np.log(amp(uo)) / steps / (2 * nu_c * k * k)
    mass = (fc[:, 0][:, mask].sum() + ff.sum() / 4) / m0 - 1
    return err_ref / (U0 * dec), err_coarse / (U0 * dec), rate_ref, rate_coarse, mass


def test_uniform_flow_to_grad_truncation():
    n = 16
    errs = []
    for U in (0.02, 0.04):
        u0 = np.array([U, 0.5 * U])
        fc = orc.init_equilibrium(9, np.ones((1, n, n)), np.broadcast_to(u0.reshape(2, 1, 1, 1),
                                                                          (2, 1, n, n)).copy())
        ff = orc.init_equilibrium(9, np.ones((1, n, n)), np.broadcast_to(u0.reshape(2, 1, 1, 1),
                                                                          (2, 1, n, n)).copy())
        a, b = fc.copy(), ff.copy()
        for _ in range(4):
            a, b = orc.refine_step(1 / (6 * 0.02 + 1), a, b, n // 4, n // 4)
        errs.append(max(np.abs(a - fc).max(), np.abs(b - ff).max()))
    print("uniform flow:", errs, "ratio", errs[1] / errs[0])
    assert errs[0] < 1e-5 and 6.0 < errs[1] / errs[0] < 10.0


def test_taylor_green_across_the_interface():
    """32^2 (200 steps) and 64^2 (800 steps, the same physical time), patch
    over the middle half of the box, nu = 0.01."""
    e32 = run(32, 200)
    e64 = run(64, 800)
    for name, e in (("32", e32), ("64", e64)):
        print(f"TGV {name}: refined {e[0]:.2e} coarse-only {e[1]:.2e} decay rate / analytic "
              f"{e[2]:.4f} (coarse-only {e[3]:.4f}) mass {e[4]:.1e}")
    for e in (e32, e64):
        assert e[0] <= 1.2 * e[1]                 # within the coarse grid's own error
        assert abs(e[2] - e[3]) <= 0.01           # no extra dissipation at the interface
        assert abs(e[4]) <= 1e-5
    assert e32[0] / e64[0] >= 3.5                 # second order
