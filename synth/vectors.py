"""Seeded vectors: every random vector is drawn once on the host in FP64 (numpy PCG64)."""
import numpy as np


def gaussian_vector(m: int, seed: int) -> np.ndarray:
    """N(0,1) entries from numpy's default_rng(seed) (PCG64), float64, length m."""
    return np.random.default_rng(seed).standard_normal(m)
