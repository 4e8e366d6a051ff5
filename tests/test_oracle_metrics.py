"""Pins of the stability metrics of Section 6.1 (CPU only).

loo(Q) = ||I - Q^T Q||_F and rre(A, Q, H) = ||A Q_{:,0:n} - Q H||_F / ||A||_F are checked
on inputs whose values are known in closed form, so that a wrong normaliser (2-norm
instead of Frobenius, no division), a sliced H or Q (dropping the subdiagonal row or the
last basis column) or a transposed product changes the result.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.metrics import loo, rre


def test_loo_two_unit_columns_at_a_known_angle():
    """Two unit columns at angle theta: Q^T Q = [[1, c], [c, 1]] with c = cos theta, so
    ||I - Q^T Q||_F = sqrt(2) |c|."""
    for theta in (np.pi / 2, np.pi / 3, 0.25, 1e-3):
        Q = np.zeros((5, 2))
        Q[0, 0] = 1.0
        Q[0, 1] = np.cos(theta)
        Q[3, 1] = np.sin(theta)
        assert abs(loo(Q) - np.sqrt(2.0) * abs(np.cos(theta))) <= 1e-15


def test_loo_columns_off_unit_norm():
    """Orthogonal columns of norms a and b: ||I - Q^T Q||_F = sqrt((1 - a^2)^2 + (1 - b^2)^2)."""
    a, b = 0.75, 1.25
    Q = np.zeros((4, 2))
    Q[1, 0] = a
    Q[2, 1] = b
    assert abs(loo(Q) - np.hypot(1 - a * a, 1 - b * b)) <= 1e-15
    assert loo(np.eye(7)[:, :3]) == 0.0


def _shift_pair(m, n, c):
    """A = c P with P the cyclic shift e_i -> e_{i+1}: the Krylov basis from e_0 is
    Q = [e_0, ..., e_n] and H = c times the (n+1) x n subdiagonal identity, exactly."""
    P = sp.csr_matrix((np.ones(m), (np.roll(np.arange(m), -1), np.arange(m))), shape=(m, m))
    A = c * P
    Q = np.eye(m)[:, :n + 1]
    H = np.zeros((n + 1, n))
    H[np.arange(1, n + 1), np.arange(n)] = c
    return A, Q, H


@pytest.mark.parametrize("dense", [False, True])
def test_rre_exact_arnoldi_pair_is_zero(dense):
    A, Q, H = _shift_pair(12, 5, 3.0)
    assert rre(A.toarray() if dense else A, Q, H) == 0.0


@pytest.mark.parametrize("dense", [False, True])
@pytest.mark.parametrize("where", [(0, 0), (2, 3), (5, 4)])
def test_rre_planted_entry_in_H(dense, where):
    """A perturbation delta of one H entry leaves a residual with one entry -delta:
    rre = |delta| / ||A||_F = |delta| / (c sqrt(m)).  (5, 4) is the subdiagonal entry of the
    last column, which a sliced H would drop; ||A||_2 = c would give a sqrt(m) larger value."""
    m, n, c, delta = 12, 5, 3.0, 2.0 ** -10      # c + delta exact
    A, Q, H = _shift_pair(m, n, c)
    H[where] += delta
    got = rre(A.toarray() if dense else A, Q, H)
    assert abs(got - delta / (c * np.sqrt(m))) <= 1e-15 * got


def test_rre_planted_entry_in_last_basis_column():
    """Q[:, n] += delta e_p (p > n) changes Q H by delta c e_p e_{n-1}^T only:
    rre = delta c / (c sqrt(m)) = delta / sqrt(m).  A version that multiplies H by Q[:, :n]
    (or drops row n of H) would miss it."""
    m, n, c, delta = 12, 5, 2.0, 2.0 ** -13
    A, Q, H = _shift_pair(m, n, c)
    Q[9, n] += delta
    got = rre(A, Q, H)
    assert abs(got - delta / np.sqrt(m)) <= 1e-15 * got


def test_rre_is_scale_invariant_and_not_symmetric_in_A():
    """rre(s A, Q, s H) = rre(A, Q, H); with A^T in place of A the exact pair is no longer an
    Arnoldi pair (P^T shifts the other way), which a transposed product would not notice."""
    A, Q, H = _shift_pair(10, 4, 1.5)
    H[1, 2] += 2e-3
    r1 = rre(A, Q, H)
    assert abs(rre(7.0 * A, Q, 7.0 * H) - r1) <= 1e-15 * r1
    assert rre(A.T.tocsr(), Q, H) > 0.1
