"""Stability metrics of Section 5.1 (test infrastructure only).

loo: loss of orthogonality ||I - Q^T Q||_F.
rre: relative representation error ||A Q_{:,0:n} - Q H||_F / ||A||_F (Arnoldi relation).
Both are plain definitions; they are pinned by exact orthonormal / exact Arnoldi inputs in
tests/test_oracle_arnoldi.py.
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
