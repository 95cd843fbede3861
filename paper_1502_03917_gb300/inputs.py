"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module draws random numbers only; it holds none of the method's
arithmetic.  Every field is a vector of nodal values on the uniform grid of the
unit square with n = 2^L cells per side, node (i h, j h) at index j*(n+1)+i.
The recipes follow the workloads the paper's method is exercised on: random
desired states, smooth targets with noise, piecewise-constant targets, random
initial guesses (section 3 starts from a random initial guess).
"""
from __future__ import annotations

import numpy as np


def grid(L: int):
    """Nodal coordinates (x, y) as flat float64 arrays of length (2^L+1)^2."""
    n = 1 << L
    t = np.arange(n + 1, dtype=np.float64) / n
    X, Y = np.meshgrid(t, t, indexing="xy")  # Y varies with the row j
    return X.ravel(), Y.ravel()


def yd_uniform(L: int, seed: int) -> np.ndarray:
    """y_D nodal values i.i.d. U(-1, 1)."""
    n = (1 << L) + 1
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n * n)


def yd_sine_noise(L: int, seed: int) -> np.ndarray:
    """y_D = sin(2 pi x) sin(2 pi y) + 0.1 N(0, 1) at the nodes."""
    X, Y = grid(L)
    noise = np.random.default_rng(seed).standard_normal(X.size)
    return np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y) + 0.1 * noise


def yd_piecewise(L: int, seed: int) -> np.ndarray:
    """y_D = +1 on [0.25, 0.75]^2, -1 elsewhere, plus U(-0.05, 0.05) noise."""
    X, Y = grid(L)
    inside = (X >= 0.25) & (X <= 0.75) & (Y >= 0.25) & (Y <= 0.75)
    noise = np.random.default_rng(seed).uniform(-0.05, 0.05, X.size)
    return np.where(inside, 1.0, -1.0) + noise


def x_uniform(L: int, seed: int) -> np.ndarray:
    """A random iterate (y, lambda), both fields i.i.d. U(-1, 1)."""
    n = (1 << L) + 1
    return np.random.default_rng(seed).uniform(-1.0, 1.0, 2 * n * n)


def f32_exact(v: np.ndarray) -> np.ndarray:
    """Round to the nearest float32 and back, so that an input is exactly
    representable in single precision."""
    return np.asarray(v, dtype=np.float32).astype(np.float64)


def u_target(L: int, seed: int) -> np.ndarray:
    """Target control for the differentiation workload: i.i.d. N(0, 1)."""
    n = (1 << L) + 1
    return np.random.default_rng(seed).standard_normal(n * n)


def batch_instances(count: int, seed: int, lmin: int = 6, lmax: int = 10):
    """Independent problem instances: levels uniform in [lmin, lmax], alpha
    log-uniform in [1e-8, 1], y_D i.i.d. U(-1, 1).  One generator draws the
    levels, then the alphas, then the fields, in that order."""
    rng = np.random.default_rng(seed)
    levels = rng.integers(lmin, lmax + 1, size=count)
    alphas = 10.0 ** rng.uniform(-8.0, 0.0, size=count)
    yds = [rng.uniform(-1.0, 1.0, ((1 << int(L)) + 1) ** 2) for L in levels]
    return [int(L) for L in levels], [float(a) for a in alphas], yds


# ---------------------------------------------------------------- Stokes --
# Stokes control unknowns of level L (n = 2^L cells per side):
# x = (v_1, v_2, p, lambda_1, lambda_2, mu); velocities on the (2n-1)^2
# interior nodes of the half-step grid, pressures on the (n+1)^2 vertices.


def stokes_sizes(L: int) -> tuple[int, int, int]:
    """(unknowns per velocity component, pressure vertices, all unknowns)."""
    n = 1 << L
    nv, npn = (2 * n - 1) ** 2, (n + 1) ** 2
    return nv, npn, 4 * nv + 2 * npn


def stokes_x_uniform(L: int, seed: int) -> np.ndarray:
    """A random Stokes iterate, every unknown i.i.d. U(-1, 1)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, stokes_sizes(L)[2])


def stokes_vd_vortex(L: int, seed: int) -> np.ndarray:
    """Desired velocity at all (2n+1)^2 nodes of the half-step grid (component
    major): the divergence-free vortex v_D = curl of sin(pi x)^2 sin(pi y)^2,
    plus 0.1 N(0, 1) noise per component."""
    n = 1 << L
    t = np.arange(2 * n + 1, dtype=np.float64) / (2 * n)
    X, Y = (a.ravel() for a in np.meshgrid(t, t, indexing="xy"))
    sx, sy = np.sin(np.pi * X), np.sin(np.pi * Y)
    u = 2 * np.pi * sx * sx * sy * np.cos(np.pi * Y)
    v = -2 * np.pi * sy * sy * sx * np.cos(np.pi * X)
    noise = 0.1 * np.random.default_rng(seed).standard_normal(2 * X.size)
    return np.concatenate([u, v]) + noise
