"""Seeded input generators (no lattice-Boltzmann arithmetic here).

Every generator takes an explicit integer seed and returns numpy arrays with
the node layout used by both sides: arrays shaped (..., nz, ny, nx), x fastest.
"""
from __future__ import annotations

import numpy as np

Q = 27


def normal_field(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """i.i.d. N(0, scale^2) numbers in float64 with the given shape."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(shape)


def population_perturbation(nx: int, ny: int, nz: int, seed: int,
                            scale: float = 1.0) -> np.ndarray:
    """(27, nz, ny, nx) array of i.i.d. N(0, scale^2) perturbations.

    A test forms an initial state f_i = w_i * (rho0 + ...) from it with the
    weights of whichever side it feeds."""
    return normal_field((Q, nz, ny, nx), seed, scale)


def sine_profile(n: int, amplitude: float, mode: int = 1) -> np.ndarray:
    """amplitude * sin(2 pi mode y / n) for y = 0..n-1 (shear-wave profile)."""
    y = np.arange(n, dtype=np.float64)
    return amplitude * np.sin(2.0 * np.pi * mode * y / n)


def uniform_taus(count: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """count relaxation times drawn uniformly from [lo, hi)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=count)
