"""Seeded synthetic inputs for the FMM-preconditioned Poisson workloads.

This module is the only code shared by the CPU oracle legs and the GPU path.  It holds
input recipes only (grid coordinates, source terms, seeds), none of the method's
arithmetic.  All fields are FP64, natural order ``[j][i]`` (x fastest), interior nodes
of an ``n x n`` grid on ``[x0, x0+side]^2`` with ``h = side / (n + 1)``.

Recipes:
* ``manufactured_sin``: f = 2 pi^2 sin(pi x) sin(pi y), exact u = sin(pi x) sin(pi y)
  on the unit square (the small 64x64 configuration).
* ``gaussian_mixture``: f = sum_k a_k exp(-|x - c_k|^2 / (2 s_k^2)), 16 terms,
  centres U[0.1, 0.9]^2, widths U[0.01, 0.05], amplitudes N(0, 1), all relative to the
  domain; numpy PCG64 ``default_rng(seed)``, drawn in the order centres, widths,
  amplitudes.  Right-hand side r of a multi-RHS batch uses seed ``base + r``.
* ``batched_sides``: grid sides of the 64 uneven problems,
  ``default_rng(0).choice([128, 256, 512, 1024, 2048], 64)``.
* ``random_field``: i.i.d. N(0,1) node values (parity tests).
* ``diffusion_coefficient``: a = 1 + mu sin(m pi x) sin(k pi y) at the (n+2)^2 nodes of the
  full grid, boundary ring included (the variable-coefficient problems).
"""
from __future__ import annotations

import numpy as np


def grid_coords(n: int, x0: float = 0.0, y0: float = 0.0, side: float = 1.0):
    h = side / (n + 1)
    x = x0 + (np.arange(n) + 1) * h
    y = y0 + (np.arange(n) + 1) * h
    X, Y = np.meshgrid(x, y)
    return X.ravel(), Y.ravel(), h


def manufactured_sin(n: int):
    X, Y, _ = grid_coords(n)
    u = np.sin(np.pi * X) * np.sin(np.pi * Y)
    return 2.0 * np.pi ** 2 * u, u


def gaussian_mixture(n: int, seed: int, k: int = 16, x0: float = 0.0, y0: float = 0.0,
                     side: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.1, 0.9, size=(k, 2))
    s = rng.uniform(0.01, 0.05, size=k)
    a = rng.standard_normal(k)
    X, Y, _ = grid_coords(n, x0, y0, side)
    u = (X - x0) / side
    v = (Y - y0) / side
    f = np.zeros(n * n)
    for q in range(k):
        f += a[q] * np.exp(-((u - c[q, 0]) ** 2 + (v - c[q, 1]) ** 2) / (2.0 * s[q] ** 2))
    return f


def gaussian_mixture_batch(n: int, nrhs: int, base_seed: int = 0) -> np.ndarray:
    return np.stack([gaussian_mixture(n, base_seed + r) for r in range(nrhs)])


def random_field(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(n * n)


def batched_sides(seed: int = 0, count: int = 64) -> np.ndarray:
    return np.random.default_rng(seed).choice([128, 256, 512, 1024, 2048], count)


def boundary_values(n: int, fn, x0: float = 0.0, y0: float = 0.0, side: float = 1.0):
    """Dirichlet data at the 4n stencil neighbours outside the interior block, ordered
    bottom (x increasing), right (y increasing), top (x decreasing), left (y decreasing)."""
    h = side / (n + 1)
    t = (np.arange(n) + 1) * h
    x1, y1 = x0 + side, y0 + side
    bottom = fn(x0 + t, np.full(n, y0))
    right = fn(np.full(n, x1), y0 + t)
    top = fn(x0 + t[::-1], np.full(n, y1))
    left = fn(np.full(n, x0), y0 + t[::-1])
    return np.concatenate([bottom, right, top, left])


def diffusion_coefficient(n: int, mu: float, m: int, k: int, x0: float = 0.0, y0: float = 0.0,
                          side: float = 1.0) -> np.ndarray:
    """a = 1 + mu sin(m pi x) sin(k pi y) at the (n+2)^2 full-grid nodes, row-major, so that
    interior node (i, j) sits at (j+1)(n+2) + (i+1)."""
    h = side / (n + 1)
    t = np.arange(n + 2) * h
    X, Y = np.meshgrid(x0 + t, y0 + t)
    return (1.0 + mu * np.sin(m * np.pi * X) * np.sin(k * np.pi * Y)).ravel()
