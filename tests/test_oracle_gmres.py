"""Pins of the oracle's GMRES, FGMRES and iterative refinement (CPU only)."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from oracle.gmres import gmres, ir, round_bf16
from synth import config1_operator, convdiff_csr, gaussian_vector


def test_gmres_matches_direct_solve():
    A = config1_operator().to_scipy()
    b = gaussian_vector(A.shape[0], 1001)
    x, info = gmres(A, b, restart=30, rtol=1e-10)
    assert info["rel_resid_true"] <= 1e-10
    xs = sla.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-7


def test_residual_estimate_is_true_residual_within_a_cycle():
    """|g_k| (Givens) equals ||b - A x_k|| in exact arithmetic; check at k = 12."""
    A = convdiff_csr(20, 2, [5.0, 5.0]).to_scipy()
    b = gaussian_vector(A.shape[0], 3)
    x, info = gmres(A, b, restart=12, rtol=1e-30, maxit=12)
    est = info["history"][-1]
    true = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert abs(est - true) < 1e-10 * max(true, 1e-3)


def test_one_cycle_equals_minimum_residual_over_krylov_space():
    """After one full cycle x minimises ||b - A x|| over K_n(A, b): compare with a
    dense least-squares solve on an explicitly orthonormalised Krylov basis (LAPACK)."""
    A = convdiff_csr(8, 2, [2.0, 1.0]).to_scipy()
    b = gaussian_vector(A.shape[0], 4)
    n = 6
    x, info = gmres(A, b, restart=n, rtol=1e-30, maxit=n)
    Kry = np.empty((A.shape[0], n))
    Kry[:, 0] = b
    for j in range(1, n):
        Kry[:, j] = A @ Kry[:, j - 1]
    Qk, _ = np.linalg.qr(Kry)
    y, *_ = np.linalg.lstsq(A @ Qk, b, rcond=None)
    assert np.linalg.norm(x - Qk @ y) < 1e-9 * np.linalg.norm(x)


def test_fgmres_with_identity_equals_gmres():
    A = convdiff_csr(15, 2, [4.0, 1.0]).to_scipy()
    b = gaussian_vector(A.shape[0], 5)
    x1, i1 = gmres(A, b, restart=20, rtol=1e-10)
    x2, i2 = gmres(A, b, restart=20, rtol=1e-10, precond=lambda w: w.copy())
    assert i1["iters"] == i2["iters"]
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x1) < 1e-10


def test_fgmres_with_exact_inverse_converges_in_one_step():
    A = convdiff_csr(10, 2, [4.0, 1.0]).to_scipy().tocsc()
    b = gaussian_vector(A.shape[0], 6)
    lu = sla.splu(A)
    x, info = gmres(A.tocsr(), b, restart=10, rtol=1e-10, precond=lu.solve)
    assert info["rel_resid_true"] <= 1e-10
    assert info["iters"] <= 3


def test_iterative_refinement_reaches_fp64_accuracy():
    """An FP32 inner solve cannot reach 1e-10 alone; FP64 refinement does."""
    A = convdiff_csr(30, 2, [10.0, 10.0]).to_scipy()
    b = gaussian_vector(A.shape[0], 7)
    for basis in ("f32", "bf16"):
        x, info = ir(A, b, restart=50, basis=basis)
        assert info["rel_resid_true"] <= 1e-10, basis
        assert info["outer"] >= 2


def test_round_bf16():
    x = np.array([1.0, 1.00390625, 1.0078125, 1.01171875, -3.0e-5], dtype=np.float32)
    r = round_bf16(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                 # halfway between 1 and 1+2^-7: ties to even
    assert r[2] == np.float32(1.0078125)
    assert r[3] == np.float32(1.015625)  # halfway, ties to even (odd mantissa rounds up)
    assert abs(r[4] + 3.0e-5) < 3.0e-5 * 2 ** -8
