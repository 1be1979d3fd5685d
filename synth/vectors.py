"""Seeded dense vectors and right-hand-side blocks."""
from __future__ import annotations

import numpy as np


def uniform_vector(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """FP64 vector with entries U[lo, hi)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=n)


def uniform_block(n: int, k: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Row-major n x k FP64 block with entries U[lo, hi) (k right-hand sides)."""
    return np.ascontiguousarray(np.random.default_rng(seed).uniform(lo, hi, size=(n, k)))


def permutation(n: int, seed: int) -> np.ndarray:
    """Random labelling of n vertices (``labels[old] = new``)."""
    return np.random.default_rng(seed).permutation(n)
