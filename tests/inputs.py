"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

This module holds no arithmetic of the method: it draws smooth random fields and
arbitrary population vectors.  Admissibility (rho > 0, E above the kinetic
energy) is ensured with bounds only: |m| <= m_max, rho >= rho_min and
E >= m_max^2 / rho_min, which exceeds |m|^2 / (2 rho) everywhere.
"""

from __future__ import annotations

import numpy as np


def smooth_field(rng: np.random.Generator, nx: int, ny: int, modes: int = 4) -> np.ndarray:
    """Periodic smooth field in [-1, 1] built from a few random Fourier modes."""
    x = np.arange(nx) / nx
    y = np.arange(ny) / ny
    X, Y = np.meshgrid(x, y)
    f = np.zeros((ny, nx))
    for _ in range(modes):
        kx, ky = rng.integers(0, 3, size=2)
        ph = rng.uniform(0, 2 * np.pi)
        f += rng.uniform(-1, 1) * np.sin(2 * np.pi * (kx * X + ky * Y) + ph)
    m = np.abs(f).max()
    return f / m if m > 0 else f


def random_state(seed: int, nx: int, ny: int, rough: float = 0.0, m_max: float = 1.0,
                 rho_min: float = 0.5, rho_max: float = 2.0, e_extra: float = 1.0):
    """Admissible conserved field u[4, ny, nx] plus arbitrary populations
    pops[16, ny, nx] (u/4 plus noise; the step map accepts any finite vector).
    ``rough`` adds cell-to-cell noise to exercise the limiter."""
    rng = np.random.default_rng(seed)
    rho = rho_min + (rho_max - rho_min) * 0.5 * (1 + smooth_field(rng, nx, ny))
    m1 = m_max * smooth_field(rng, nx, ny)
    m2 = m_max * smooth_field(rng, nx, ny)
    if rough > 0:
        rho = np.clip(rho * (1 + rough * rng.uniform(-1, 1, rho.shape)), rho_min, None)
        m1 = np.clip(m1 + rough * m_max * rng.uniform(-1, 1, m1.shape), -m_max, m_max)
        m2 = np.clip(m2 + rough * m_max * rng.uniform(-1, 1, m2.shape), -m_max, m_max)
    E = m_max * m_max / rho_min + e_extra * (1.5 + 0.5 * smooth_field(rng, nx, ny))
    if rough > 0:
        E = E + rough * e_extra * rng.uniform(0, 1, E.shape)
    u = np.stack([rho, m1, m2, E])
    pops = np.zeros((16, ny, nx))
    for k in range(4):
        for c in range(4):
            pops[4 * k + c] = 0.25 * u[c] * (1 + 0.2 * rng.uniform(-1, 1, (ny, nx)))
    return u, pops


def random_samples(seed: int, M: int, ny: int, nx: int, dist: str = "lognormal") -> np.ndarray:
    """M positive samples per cell, shape [M, ny, nx], with per-cell location
    and spread varying over the grid (density-like values)."""
    rng = np.random.default_rng(seed)
    loc = 1.0 + 4.0 * rng.uniform(0, 1, (ny, nx))
    spread = 0.05 + 0.5 * rng.uniform(0, 1, (ny, nx))
    if dist == "lognormal":
        z = rng.standard_normal((M, ny, nx))
        return loc * np.exp(spread * z)
    if dist == "ties":
        return np.round(loc * (1 + spread * rng.standard_normal((M, ny, nx))), 1)
    raise ValueError(dist)
