"""Loss of orthogonality (LOO) classes of the QR variants over graded condition numbers
(Table 3, Section 5): CGS loses orthogonality as O(eps) kappa^2, MGS level 1 as
O(eps) kappa, CGS2 and DCGS2 (QR) keep it at O(eps); the representation error
||A - Q R|| / ||A|| stays at O(eps) for every variant.  A variant with a dropped second
pass, a lost Stephen's-trick correction or a wrong Pythagorean norm falls out of its class
here."""
import numpy as np
import pytest

from oracle import arnoldi as orc
from oracle.metrics import loo
from synth import graded_matrix

M, N = 2000, 30
EPS = 2.0 ** -52


@pytest.fixture(scope="module")
def table():
    out = {}
    for e in (2, 4, 6, 8, 10, 12, 14):
        B = graded_matrix(M, N, 10.0 ** e, 500 + e)
        row = {}
        for name, f in (("cgs", orc.cgs_qr), ("mgs", orc.mgs_qr), ("cgs2", orc.cgs2_qr),
                        ("dcgs2", orc.dcgs2_qr)):
            Q, R = f(B)
            row[name] = (loo(Q), np.linalg.norm(B - Q @ R) / np.linalg.norm(B))
        out[e] = row
    return out


def test_graded_matrix_has_the_requested_condition_number():
    for e in (2, 6, 10):
        s = np.linalg.svd(graded_matrix(500, 20, 10.0 ** e, 7), compute_uv=False)
        assert abs(np.log10(s[0] / s[-1]) - e) < 1e-6


def test_cgs2_and_dcgs2_keep_orthogonality_at_eps(table):
    for e, row in table.items():
        for name in ("cgs2", "dcgs2"):
            assert row[name][0] <= 100 * EPS, (e, name, row[name])


def test_mgs_loses_orthogonality_like_kappa(table):
    for e in (4, 6, 8, 10):
        lo = table[e]["mgs"][0]
        assert 1e-3 * EPS * 10.0 ** e <= lo <= 1e2 * EPS * 10.0 ** e, (e, lo)
    # one decade of LOO per decade of kappa (two decades per step of the table)
    r = table[10]["mgs"][0] / table[4]["mgs"][0]
    assert 1e4 <= r <= 1e8


def test_cgs_loses_orthogonality_like_kappa_squared(table):
    for e in (2, 4, 6):
        lo = table[e]["cgs"][0]
        assert 1e-3 * EPS * 10.0 ** (2 * e) <= lo <= 1e2 * EPS * 10.0 ** (2 * e), (e, lo)
    assert table[14]["cgs"][0] > 1.0                 # orthogonality lost entirely


def test_representation_error_at_eps_for_every_variant(table):
    for e, row in table.items():
        for name, (_, res) in row.items():
            assert res <= 10 * EPS, (e, name, res)
