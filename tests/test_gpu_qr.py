"""GPU parity of the DCGS2 QR (Algorithm 2) against the FP64 oracle.

Bar: R to 1e-12 relative (Frobenius), Q to 1e-10 absolute, A = Q R and Q^T Q = I at O(eps),
in both FP64 modes (every product in FP64, and the float-float offload)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import arnoldi as orc  # noqa: E402
from oracle.metrics import loo  # noqa: E402
from synth import gaussian_vector, graded_factors, graded_matrix  # noqa: E402


@pytest.fixture(scope="module")
def kc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2104_01253_gb300 as kc
    return kc


@pytest.fixture(scope="module")
def ctx(kc):
    return kc.Context(0)


def _matrix(m, n, seed, graded=False):
    """Seeded m x n matrix; `graded` scales its singular values over 6 decades."""
    B = gaussian_vector(m * n, seed).reshape(n, m).T.copy()
    if graded:
        U, _ = np.linalg.qr(B)
        V, _ = np.linalg.qr(gaussian_vector(n * n, seed + 1).reshape(n, n))
        B = (U * np.logspace(0, -6, n)) @ V.T
    return B


def _run(kc, ctx, B, mode):
    m, n = B.shape
    ld = m + (m & 1)                                   # even leading dimension
    At = torch.zeros((n, ld), dtype=torch.float64, device="cuda")
    At[:, :m] = torch.as_tensor(B.T)
    Qt = torch.zeros_like(At)
    Rt = torch.full((n, n), 7.0, dtype=torch.float64, device="cuda")   # lower part must be zeroed
    ctx.set_fp64_mode(mode)
    try:
        kc.dcgs2_qr(ctx, At, Qt, Rt)
    finally:
        ctx.set_fp64_mode(1)
    torch.cuda.synchronize()
    return Qt[:, :m].cpu().numpy().T, Rt.cpu().numpy().T


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("m,n,graded", [(1000, 1, False), (1000, 2, False), (5001, 17, False),
                                        (20000, 40, True), (40000, 64, False)])
def test_dcgs2_qr_matches_oracle(kc, ctx, m, n, graded, mode):
    B = _matrix(m, n, 300 + n, graded)
    Qg, Rg = _run(kc, ctx, B, mode)
    Qo, Ro = orc.dcgs2_qr(B)
    assert np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro) <= 1e-12
    assert np.abs(Qg - Qo).max() <= 1e-10
    assert np.allclose(np.tril(Rg, -1), 0.0)
    assert np.linalg.norm(B - Qg @ Rg) / np.linalg.norm(B) <= 1e-14
    assert loo(Qg) <= 1e-13
    assert ctx.read_status() == 0


def test_dcgs2_qr_rejects_bad_arguments(kc, ctx):
    At = torch.zeros((4, 100), dtype=torch.float64, device="cuda")
    Qt = torch.zeros_like(At)
    Rt = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(kc.KrylovError):                 # R leading dimension below n
        kc.dcgs2_qr(ctx, At, Qt, torch.zeros((4, 3), dtype=torch.float64, device="cuda"))
    with pytest.raises(kc.KrylovError):                 # odd leading dimension of A
        kc.dcgs2_qr(ctx, torch.zeros((4, 101), dtype=torch.float64, device="cuda"), Qt, Rt)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_dcgs2_qr_orthogonality_over_condition_numbers(kc, ctx, mode):
    """Table 3: DCGS2 (QR) keeps the loss of orthogonality at O(eps) whatever kappa(A), and
    the representation error at O(eps).  Graded matrices with kappa from 1e2 to 1e14 (one
    pair of orthonormal factors, seed 900); R against the oracle at every kappa, Q where it
    is well determined (kappa <= 1e5)."""
    eps = 2.0 ** -52
    m, n = 20000, 40
    factors = graded_factors(m, n, 900)
    for e in (2, 5, 8, 11, 14):
        B = graded_matrix(m, n, 10.0 ** e, 900, factors=factors)
        Qg, Rg = _run(kc, ctx, B, mode)
        assert loo(Qg) <= 100 * eps, (e, loo(Qg))
        assert np.linalg.norm(B - Qg @ Rg) / np.linalg.norm(B) <= 10 * eps
        assert ctx.read_status() == 0
        Qo, Ro = orc.dcgs2_qr(B)
        assert np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro) <= 1e-12
        if e <= 5:
            assert np.abs(Qg - Qo).max() <= 1e-9
