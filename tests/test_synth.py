"""Pins of the synthetic input generators (CPU only)."""
import os

import numpy as np
import pytest

from synth import (config1_operator, convdiff_csr, gaussian_vector, manteuffel_csr,
                   varcoef_fields_2d)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "manteuffel_k50.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        out[k] = float(v)
    return out


def test_manteuffel_matches_printed_table():
    """Table "stab_manteuffel" (Section 6.1): ||A||_2, cond(A) and non-normality, k = 50."""
    g = _golden()
    A = manteuffel_csr(50).to_scipy().toarray()
    s = np.linalg.svd(A, compute_uv=False)
    nn = np.linalg.norm(A.T @ A - A @ A.T) / np.linalg.norm(A) ** 2
    assert abs(s[0] - g["norm2_A"]) <= 0.005 * g["norm2_A"]
    assert abs(s[0] / s[-1] - g["cond_A"]) <= 0.005 * g["cond_A"]
    assert abs(nn - g["nonnormality_F"]) <= 0.005 * g["nonnormality_F"]


def test_manteuffel_closed_form_spectrum():
    """Eigenvalues 2[2 - sqrt(1-(beta/2)^2)(cos(l pi/L) + cos(j pi/L))], L = k+1 (Section 6.1)."""
    k, beta = 9, 0.5
    A = manteuffel_csr(k, beta).to_scipy().toarray()
    L = k + 1
    exact = np.sort([2 * (2 - np.sqrt(1 - (beta / 2) ** 2) * (np.cos(l * np.pi / L) + np.cos(j * np.pi / L)))
                     for l in range(1, k + 1) for j in range(1, k + 1)])
    ev = np.linalg.eigvals(A)
    assert np.abs(ev.imag).max() < 1e-8
    assert np.abs(np.sort(ev.real) - exact).max() < 1e-8


def test_config_sizes():
    A = config1_operator()
    assert A.m == 10_000 and A.nnz == 49_600
    B = convdiff_csr(10, 3, [1.0, 0.5, 0.25])
    assert B.nnz == 7 * 1000 - 6 * 100
    # strictly increasing columns in every row
    for r in range(B.m):
        cols = B.col_idx[B.row_ptr[r]:B.row_ptr[r + 1]]
        assert np.all(np.diff(cols) > 0)


def test_constant_coefficient_stencil_values():
    """Interior row of the 2D operator: diagonal 4 + h(|bx|+|by|), upwind neighbours."""
    N = 5
    h = 1.0 / (N + 1)
    A = convdiff_csr(N, 2, [3.0, -2.0]).to_scipy().toarray()
    r = 2 + N * 2
    assert A[r, r] == pytest.approx(4 + h * 5.0)
    assert A[r, r - 1] == pytest.approx(-1 - 3.0 * h)      # bx > 0: upwind is x-1
    assert A[r, r + 1] == pytest.approx(-1.0)
    assert A[r, r + N] == pytest.approx(-1 - 2.0 * h)      # by < 0: upwind is y+1
    assert A[r, r - N] == pytest.approx(-1.0)
    # M-matrix: zero row sums in the interior, positive on the boundary
    rs = A.sum(axis=1)
    assert rs.min() > -1e-12


def test_harmonic_face_kappa():
    k = np.array([[1.0, 3.0], [2.0, 5.0]])
    A = convdiff_csr(2, 2, [0.0, 0.0], kappa=k).to_scipy().toarray()
    # face between (0,0) and (0,1) in x: harmonic mean of 1 and 3
    assert A[0, 1] == pytest.approx(-2 * 1 * 3 / 4)


def test_vectors_and_fields_are_seeded():
    assert np.array_equal(gaussian_vector(10, 3), gaussian_vector(10, 3))
    k1, w1 = varcoef_fields_2d(32, 5)
    k2, w2 = varcoef_fields_2d(32, 5)
    assert np.array_equal(k1, k2) and np.array_equal(w1, w2)
    assert np.abs(np.log(k1)).std() == pytest.approx(1.0, rel=0.05) or np.log(k1).std() > 0.5
    assert np.sqrt(w1[0] ** 2 + w1[1] ** 2).max() == pytest.approx(100.0)
