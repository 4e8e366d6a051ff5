"""GPU parity of gmres_solve (FP64 DCGS2-GMRES and FP32 / BF16 inner solves in FP64
iterative refinement) against the oracle.

Solutions are compared after the same number of iterations (one full GMRES(30) cycle) to
1e-10 relative; converged solves must reach a true FP64 relative residual of 1e-10.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.gmres import gmres as orc_gmres, ir as orc_ir  # noqa: E402
from synth import config1_operator, convdiff_csr, gaussian_vector  # noqa: E402


@pytest.fixture(scope="module")
def kc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2104_01253_gb300 as kc
    return kc


@pytest.fixture(scope="module")
def ctx(kc):
    return kc.Context(0)


def test_one_cycle_solution_matches_oracle(kc, ctx):
    Ah = config1_operator()
    b = gaussian_vector(Ah.m, 1001)
    A = kc.DeviceCSR(Ah)
    bd = torch.as_tensor(b, device="cuda")
    x = torch.zeros_like(bd)
    info = kc.gmres_solve(ctx, A, bd, x, restart=30, rtol=1e-10, maxit=30)
    xo, io = orc_gmres(Ah.to_scipy(), b, restart=30, rtol=1e-10, maxit=30)
    xg = x.cpu().numpy()
    assert info["iters"] == io["iters"] == 30
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-10
    assert abs(info["rel_resid_true"] - io["rel_resid_true"]) <= 1e-8 * io["rel_resid_true"]


def test_config1_converges_to_1e10(kc, ctx):
    Ah = config1_operator()
    b = gaussian_vector(Ah.m, 1001)
    A = kc.DeviceCSR(Ah)
    bd = torch.as_tensor(b, device="cuda")
    x = torch.zeros_like(bd)
    info = kc.gmres_solve(ctx, A, bd, x, restart=30, rtol=1e-10)
    assert info["status"] == 0
    xg = x.cpu().numpy()
    true = np.linalg.norm(b - Ah.to_scipy() @ xg) / np.linalg.norm(b)
    assert true <= 1e-10
    assert abs(true - info["rel_resid_true"]) <= 1e-3 * true
    _, io = orc_gmres(Ah.to_scipy(), b, restart=30, rtol=1e-10)
    assert abs(info["iters"] - io["iters"]) <= 2


def test_early_convergence_inside_a_cycle(kc, ctx):
    """A well-conditioned operator converges before the basis fills: the device stop flag
    skips the remaining kernels of the cycle."""
    Ah = convdiff_csr(20, 2, [1.0, 1.0])
    b = gaussian_vector(Ah.m, 5)
    A = kc.DeviceCSR(Ah)
    bd = torch.as_tensor(b, device="cuda")
    x = torch.zeros_like(bd)
    info = kc.gmres_solve(ctx, A, bd, x, restart=120, rtol=1e-10)
    _, io = orc_gmres(Ah.to_scipy(), b, restart=120, rtol=1e-10)
    assert info["status"] == 0 and info["rel_resid_true"] <= 1e-10
    assert info["restarts"] == 1 and info["iters"] < 120
    assert abs(info["iters"] - io["iters"]) <= 1


@pytest.mark.parametrize("precision,basis", [(1, "f32"), (2, "bf16")])
def test_iterative_refinement_reaches_fp64_accuracy(kc, ctx, precision, basis):
    Ah = convdiff_csr(30, 3, [50.0, 25.0, 12.5])
    b = gaussian_vector(Ah.m, 1004)
    A = kc.DeviceCSR(Ah)
    A32 = kc.DeviceCSR(Ah, dtype=torch.float32)
    bd = torch.as_tensor(b, device="cuda")
    x = torch.zeros_like(bd)
    info = kc.gmres_solve(ctx, A, bd, x, restart=50, rtol=1e-10, precision=precision, A32=A32,
                          inner_rtol=1e-4, inner_max_cycles=3)
    xg = x.cpu().numpy()
    true = np.linalg.norm(b - Ah.to_scipy() @ xg) / np.linalg.norm(b)
    assert info["status"] == 0
    assert true <= 1e-10
    xo, io = orc_ir(Ah.to_scipy(), b, restart=50, inner_rtol=1e-4, inner_max_restarts=2,
                    basis=basis)
    assert io["rel_resid_true"] <= 1e-10
    # same number of refinement steps as the oracle, give or take one
    assert abs(info["outer"] - io["outer"]) <= 1
    xs = xo
    assert np.linalg.norm(xg - xs) / np.linalg.norm(xs) <= 1e-8
