"""Pins of the ICWY-MGS oracle (Section 5: the inverse compact WY projector
I - Q (I + L)^{-1} Q^T, one reduction per iteration).  In exact arithmetic the projector
is the product of MGS's rank-1 projections, so ICWY-MGS is MGS (agreement on
well-conditioned inputs, against MGS level 1 and Householder QR); in floating point it
keeps MGS's class of Table 3, loss of orthogonality O(eps) kappa (the row of the level-2
MGS variants), with an O(eps) representation error.  Planted mistakes in the triangular
correction (T = I, i.e. no L; L transposed) leave that class."""
import numpy as np
import pytest

from oracle import arnoldi as orc
from oracle.metrics import loo, rre
from synth import convdiff_csr, gaussian_vector, graded_matrix

EPS = 2.0 ** -52


def test_icwy_qr_equals_mgs_and_householder_when_well_conditioned():
    B = graded_matrix(600, 20, 10.0, 41)
    Q, R = orc.icwy_qr(B)
    Qm, Rm = orc.mgs_qr(B)
    assert np.abs(Q - Qm).max() <= 1e-13 and np.abs(R - Rm).max() <= 1e-13
    Qh, Rh = np.linalg.qr(B)
    sg = np.sign(np.diag(Rh))
    assert np.abs(Q - Qh * sg).max() <= 1e-12
    assert np.abs(R - sg[:, None] * Rh).max() <= 1e-12
    assert np.allclose(np.tril(R, -1), 0.0)


@pytest.fixture(scope="module")
def classes():
    out = {}
    for e in (2, 4, 6, 8, 10):
        B = graded_matrix(2000, 30, 10.0 ** e, 500 + e)
        Q, R = orc.icwy_qr(B)
        out[e] = (loo(Q), np.linalg.norm(B - Q @ R) / np.linalg.norm(B))
    return out


def test_icwy_qr_loses_orthogonality_like_kappa(classes):
    for e in (4, 6, 8, 10):
        lo = classes[e][0]
        assert 1e-3 * EPS * 10.0 ** e <= lo <= 1e2 * EPS * 10.0 ** e, (e, lo)
    r = classes[10][0] / classes[4][0]
    assert 1e4 <= r <= 1e8
    for e, (_, res) in classes.items():
        assert res <= 10 * EPS, (e, res)


@pytest.mark.parametrize("mistake", ["no_L", "L_transposed"])
def test_planted_mistakes_leave_the_class(monkeypatch, mistake):
    """With T = I the projection is CGS (O(eps) kappa^2); a transposed L is no projector."""
    if mistake == "no_L":
        monkeypatch.setattr(orc, "_forward_solve_unit_lower", lambda L, r: np.array(r))
    else:
        def transposed(L, r):
            y = np.array(r, dtype=np.float64, copy=True)
            for i in range(y.shape[0]):
                y[i] -= L.T[i, :i] @ y[:i]
            return y
        monkeypatch.setattr(orc, "_forward_solve_unit_lower", transposed)
    B = graded_matrix(2000, 30, 1e6, 506)
    Q, _ = orc.icwy_qr(B)
    assert loo(Q) > 1e2 * EPS * 1e6          # above the MGS class bound at kappa = 1e6


def test_icwy_arnoldi_relation_start_and_agreement_with_mgs():
    A = convdiff_csr(10, 3, [1.0, 0.5, 0.25]).to_scipy()
    r0 = gaussian_vector(A.shape[0], 1002)
    n = 12
    Q, H = orc.icwy_arnoldi(A, r0, n)
    assert np.abs(Q[:, 0] - r0 / np.linalg.norm(r0)).max() <= 1e-16
    assert rre(A, Q, H) <= 1e-15                       # exact by construction
    Qm, Hm = orc.mgs_arnoldi(A, r0, n)
    assert np.linalg.norm(H - Hm) / np.linalg.norm(Hm) <= 1e-12
    assert np.abs(Q - Qm).max() <= 1e-12
    assert np.allclose(np.tril(H, -2), 0.0)            # Hessenberg
