"""The basis Gram matrix (kc_basis_gram) and the loss-of-orthogonality diagnostic of
gmres_solve (kc_gmres_opts.diag_loo), against numpy on the same stored basis values."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import config2_operator, gaussian_vector  # noqa: E402


@pytest.fixture(scope="module")
def kc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2104_01253_gb300 as kc
    return kc


@pytest.fixture(scope="module")
def ctx(kc):
    return kc.Context(0)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("m,ncols", [(100003, 51), (4099, 128), (31, 1)])
def test_gram_matches_numpy(kc, ctx, dtype, m, ncols):
    """G = Q^T Q of the stored values, summed in FP64 (the products of FP32 and BF16
    values are exact in FP64): to 1e-13 of max |G| in every entry."""
    ld = m + 5
    g = torch.Generator(device="cuda").manual_seed(11)
    Qd = (torch.randn((ncols, ld), dtype=torch.float64, device="cuda", generator=g)
          / np.sqrt(m)).to(dtype)
    G = kc.basis_gram(ctx, Qd, m, ncols).cpu().numpy()
    Qh = Qd[:, :m].to(torch.float64).cpu().numpy()
    Go = Qh @ Qh.T
    assert np.abs(G - Go).max() <= 1e-13 * np.abs(Go).max()
    assert np.array_equal(G, G.T)


def test_gmres_diag_loo(kc, ctx):
    """The diagnostic leaves the solve unchanged and reports the worst loss of
    orthogonality over the cycles' bases: O(eps) for the FP64 solve, O(u) of FP32 / BF16 for
    the reduced-precision inner solves of iterative refinement."""
    Ah = config2_operator(30)
    A = kc.DeviceCSR(Ah)
    A32 = kc.DeviceCSR(Ah, dtype=torch.float32)
    b = torch.as_tensor(gaussian_vector(Ah.m, 1004), device="cuda")
    for prec, lo, hi in ((0, 0.0, 1e-13), (1, 1e-9, 1e-3), (2, 1e-6, 1e-1)):
        x1 = torch.zeros_like(b)
        x2 = torch.zeros_like(b)
        i1 = kc.gmres_solve(ctx, A, b, x1, restart=50, rtol=1e-10, precision=prec, A32=A32)
        i2 = kc.gmres_solve(ctx, A, b, x2, restart=50, rtol=1e-10, precision=prec, A32=A32,
                            diag_loo=True)
        assert i1["status"] == 0 and i2["status"] == 0
        assert i2["rel_resid_true"] <= 1e-10
        if prec > 0:                 # same path: the diagnostic changes nothing
            assert i1["iters"] == i2["iters"]
            assert torch.equal(x1, x2)
        print("precision %d: max LOO %.3e" % (prec, i2["max_loo"]))
        assert lo <= i2["max_loo"] <= hi, (prec, i2["max_loo"])
