"""Reduced-precision storage (populations kept as h = f/W - 1 in 16 bits,
arithmetic in FP32) against the FP64 oracle.

The target for 16-bit storage is a relative velocity error <= 1e-3 after
1000 laminar steps.  F16N (sign, 3 exponent bits, 12 stored significand
bits: the exponent range of IEEE half narrowed to the [2^-6, 2) that h
occupies) meets it.  IEEE half (10 stored significand bits) and bfloat16 (7)
do not on these small Taylor-Green boxes: their rounding of the O(u)
deviations leaves a broadband velocity noise; the asserted bounds for them
are their measured levels with margin, stated as such."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1710_02375_gb300 import synth

pytestmark = pytest.mark.gpu
F16, BF16, F16N = 1, 2, 4


def make(lat, shape, beta, **kw):
    from paper_1710_02375_gb300.lbm import Lattice
    nz, ny, nx = shape
    return Lattice(lat, nx, ny, nz, beta, **kw)


@pytest.mark.parametrize("storage,bits,floor", [(F16, 11, 2.0 ** -25), (BF16, 8, 0.0),
                                                (F16N, 13, 2.0 ** -19)])
def test_encoding_roundtrip(storage, bits, floor):
    """Stored value h = f/W - 1 rounds to nearest: |f_back - f| <= W max(|h|
    2^-bits, floor), floor the half step of the evenly spaced small codes."""
    lat, shape = 27, (3, 4, 5)
    f0 = synth.random_state(lat, shape, 0.05, 9)
    w = synth.lattice_weights(lat).reshape((lat, 1, 1, 1))
    # include deviations below the narrow format's smallest normal, 2^-6
    f0[:, 0] = w[:, 0] * (1 + 0.01 * np.sign(f0[:, 0] - w[:, 0]) * np.abs(f0[:, 0] / w[:, 0] - 1))
    L = make(lat, shape, 0.9, storage=storage)
    L.set_populations(f0)
    got = L.get_populations()
    h = f0 / w - 1
    assert np.all(np.abs(got - f0) <= w * np.maximum(np.abs(h) * 2.0 ** -bits, floor) * 1.001 + 1e-300)


@pytest.mark.parametrize("lat,shape,nu", [(27, (16, 20, 24), 0.002), (9, (1, 48, 64), 0.005)])
@pytest.mark.parametrize("storage", [F16N, F16, BF16])
def test_taylor_green_1000_steps_reduced_storage(lat, shape, nu, storage):
    nz, ny, nx = shape
    rho, u = synth.tgv_fields(nx, ny, nz, 0.05, three_d=(lat == 27))
    dim = 2 if lat == 9 else 3
    beta = 1.0 / (6.0 * nu + 1.0)
    L = make(lat, shape, beta, storage=storage)
    L.init_equilibrium(rho, np.ascontiguousarray(u[:dim]))
    L.step(1000)
    L.check()
    _, ug = L.macros()
    f = orc.run_periodic(lat, beta, orc.init_equilibrium(lat, rho, u[:dim]), 1000)
    _, uo = orc.macros(lat, f)
    err = np.max(np.abs(ug - uo[:dim])) / np.max(np.abs(uo))
    print(f"storage {storage} lattice {lat}: relative velocity error {err:.3e}")
    # F16N: the 1e-3 target.  IEEE half / bfloat16: measured levels (a CPU
    # emulation of the rounding gives 1.9e-3 for half on the D3Q27 box)
    bound = {F16N: 1e-3, F16: 5e-3, BF16: 3e-2}[storage]
    assert err <= bound, err
