"""Seeded random vectors and coefficients.

Seeds follow one fixed convention so that every consumer draws identical data:
jitter 0, u 1, w/g 2, k 3, cell/vertex shuffle 4.
"""
from __future__ import annotations

import numpy as np

SEEDS = {"jitter": 0, "u": 1, "w": 2, "k": 3, "shuffle": 4}


def uniform_vector(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """n float64 values drawn from U[lo, hi] with numpy's PCG64 seeded by `seed`."""
    return np.random.default_rng(seed).uniform(lo, hi, size=n)


def lognormal_coefficients(shape, seed: int, sigma: float = 0.5) -> np.ndarray:
    """k = exp(N(0, sigma)) with sigma the standard deviation of the underlying normal."""
    return np.exp(np.random.default_rng(seed).normal(0.0, sigma, size=shape))
