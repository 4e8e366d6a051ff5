"""Stability metrics of Section 6.1 (test infrastructure only).

loo: loss of orthogonality ||I - Q^T Q||_F.
rre: relative representation error ||A Q_{:,0:n} - Q H||_F / ||A||_F (Arnoldi relation).
Both are plain definitions; tests/test_oracle_metrics.py pins them with closed-form values:
two unit columns at a known angle, orthogonal columns off unit norm, an exact Arnoldi pair
of a scaled cyclic shift (rre = 0) and planted perturbations of one entry of H or of the
last basis column with known rre = |delta| / ||A||_F.
"""
import numpy as np


def loo(Q):
    k = Q.shape[1]
    return float(np.linalg.norm(np.eye(k) - Q.T @ Q))


def rre(A, Q, H):
    n = H.shape[1]
    AQ = np.column_stack([A @ Q[:, j] for j in range(n)])
    normA = np.sqrt((A.multiply(A)).sum()) if hasattr(A, "multiply") else np.linalg.norm(A)
    return float(np.linalg.norm(AQ - Q[:, :n + 1] @ H) / normA)
