"""Seeded vectors: every random vector is drawn once on the host in FP64 (numpy PCG64)."""
import numpy as np


def gaussian_vector(m: int, seed: int) -> np.ndarray:
    """N(0,1) entries from numpy's default_rng(seed) (PCG64), float64, length m."""
    return np.random.default_rng(seed).standard_normal(m)


def graded_factors(m: int, n: int, seed: int):
    """Orthonormal U (m x n) and V (n x n): the Q factors of N(0,1) matrices drawn with
    seeds ``seed`` (column by column) and ``seed + 1``."""
    B = gaussian_vector(m * n, seed).reshape(n, m).T
    U, _ = np.linalg.qr(B)
    V, _ = np.linalg.qr(gaussian_vector(n * n, seed + 1).reshape(n, n))
    return U, V


def graded_matrix(m: int, n: int, kappa: float, seed: int, factors=None) -> np.ndarray:
    """Seeded m x n matrix (m >= n) with 2-norm condition number ``kappa``: U diag(sigma) V^T
    with (U, V) = graded_factors(m, n, seed) (or the given ``factors``) and sigma
    log-spaced from 1 down to 1/kappa.  Returned as a C-ordered (m, n) float64 array.
    (For kappa near 1/eps the rounded product's condition number is only approximately
    kappa.)"""
    U, V = graded_factors(m, n, seed) if factors is None else factors
    sigma = np.logspace(0.0, -np.log10(kappa), n)
    return (U * sigma) @ V.T
