"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the lattice Boltzmann method itself: it only
draws fields (density, velocity, random population vectors, surface meshes)
that both the CUDA path and the CPU oracle take as inputs.  Each side turns
them into populations with its own code.

Workloads (sizes follow the paper's set-ups in lattice units):
  * Taylor-Green vortex (periodic box): node-centred x = 2 pi (i + 1/2) / N,
      u =  u0 sin x cos y cos z,  v = -u0 cos x sin y cos z,  w = 0,
      rho = 1 + 3 (u0^2/16) (cos 2x + cos 2y)(cos 2z + 2)   (p = rho / 3).
  * Random near-equilibrium population vectors f_i = W_i (1 + a xi_i),
    xi ~ U(-1, 1), for brute-force comparisons on small lattices.
"""
from __future__ import annotations

import numpy as np


def lattice_weights(q: int) -> np.ndarray:
    """Tensor-product D1Q3 weights in the library's direction order
    (x fastest, then y, then z; component -1, 0, +1)."""
    w1 = np.array([1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0])
    if q == 9:
        return np.einsum("y,x->yx", w1, w1).reshape(9)
    if q == 27:
        return np.einsum("z,y,x->zyx", w1, w1, w1).reshape(27)
    raise ValueError(q)


def tgv_fields(nx: int, ny: int, nz: int, u0: float, three_d: bool = True):
    """Taylor-Green vortex density rho[nz,ny,nx] and velocity u[3,nz,ny,nx].

    three_d=False gives the 2-D vortex (uniform in z, rho from the 2-D pressure)."""
    x = 2.0 * np.pi * (np.arange(nx) + 0.5) / nx
    y = 2.0 * np.pi * (np.arange(ny) + 0.5) / ny
    z = 2.0 * np.pi * (np.arange(nz) + 0.5) / nz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    u = np.zeros((3, nz, ny, nx))
    if three_d:
        u[0] = u0 * np.sin(X) * np.cos(Y) * np.cos(Z)
        u[1] = -u0 * np.cos(X) * np.sin(Y) * np.cos(Z)
        rho = 1.0 + 3.0 * (u0 * u0 / 16.0) * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
    else:
        u[0] = u0 * np.sin(X) * np.cos(Y)
        u[1] = -u0 * np.cos(X) * np.sin(Y)
        rho = 1.0 + 3.0 * (u0 * u0 / 4.0) * (np.cos(2 * X) + np.cos(2 * Y))
    return rho, u


def random_state(q: int, shape, amp: float, seed: int) -> np.ndarray:
    """Random population field f[q, *shape] = W_i (1 + amp xi), xi ~ U(-1,1)."""
    rng = np.random.default_rng(seed)
    w = lattice_weights(q).reshape((q,) + (1,) * len(shape))
    xi = rng.uniform(-1.0, 1.0, size=(q,) + tuple(shape))
    return w * (1.0 + amp * xi)


def random_macros(shape, u_amp: float, rho_amp: float, seed: int, dim: int = 3):
    """Smooth-free random density and velocity fields (for equilibrium initial states)."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + rho_amp * rng.uniform(-1, 1, size=shape)
    u = np.zeros((3,) + tuple(shape))
    u[:dim] = u_amp * rng.uniform(-1, 1, size=(dim,) + tuple(shape))
    return rho, u
