"""Pins of the oracle's Krylov-Schur eigensolver (CPU only)."""
import numpy as np

from oracle.krylov_schur import krylov_schur, wanted_set
from synth import config3_operator, gaussian_vector, manteuffel_csr


def test_ks_matches_dense_eigenvalues_on_small_copy():
    """Config-3 family on a 40 x 40 grid: the 10 largest-real-part eigenvalues."""
    A = config3_operator(40).to_scipy()
    res = krylov_schur(A, gaussian_vector(A.shape[0], 7), nev=10, ncv=40, nkeep=20, tol=1e-10)
    assert res["nconv"] == 10
    ev = np.linalg.eigvals(A.toarray())
    ev = ev[np.argsort(-ev.real)][:10]
    got = np.sort_complex(res["eigs"])
    assert np.abs(got - np.sort_complex(ev)).max() / np.abs(ev).max() < 1e-9
    assert np.all(res["resid"] <= 1e-10 * np.abs(res["eigs"]))


def test_ks_manteuffel_closed_form():
    """Largest distinct Manteuffel eigenvalues from the closed form (Section 6.1)."""
    k, beta = 20, 0.5
    A = manteuffel_csr(k, beta).to_scipy()
    res = krylov_schur(A, gaussian_vector(A.shape[0], 8), nev=4, ncv=30, nkeep=15, tol=1e-10)
    L = k + 1
    exact = sorted({round(2 * (2 - np.sqrt(1 - (beta / 2) ** 2) *
                                (np.cos(l * np.pi / L) + np.cos(j * np.pi / L))), 12)
                    for l in range(1, k + 1) for j in range(1, k + 1)}, reverse=True)[:4]
    got = np.sort(res["eigs"].real)[::-1]
    assert np.abs(got - np.array(exact)).max() < 1e-7      # the paper's absolute tolerance


def test_wanted_set_keeps_conjugate_pairs():
    ev = np.array([5.0, 3 + 1j, 3 - 1j, 1.0])
    assert sorted(wanted_set(ev, 2)) == [0, 1, 2]
    assert sorted(wanted_set(ev, 3)) == [0, 1, 2]
