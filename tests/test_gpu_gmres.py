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


PATHS = [1, 2, 3]  # Context.GMRES_MULTI_KERNEL, GMRES_CLUSTER, GMRES_GRID


@pytest.fixture
def path(ctx, request):
    ctx.set_gmres_path(request.param)
    yield request.param
    ctx.set_gmres_path(0)


@pytest.mark.parametrize("path", PATHS, indirect=True)
def test_one_cycle_solution_matches_oracle(kc, ctx, path):
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


@pytest.mark.parametrize("path", PATHS, indirect=True)
def test_config1_converges_to_1e10(kc, ctx, path):
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


def test_tensor_core_reduction_mode_in_gmres(kc, ctx):
    """FP64 mode 2 (the reduction as exact digit products on the tensor cores) inside the
    multi-kernel GMRES path, whose reduction epilogue also runs the Givens update: one
    cycle matches the oracle to 1e-10 and the full solve converges like the oracle."""
    Ah = config1_operator()
    b = gaussian_vector(Ah.m, 1001)
    A = kc.DeviceCSR(Ah)
    bd = torch.as_tensor(b, device="cuda")
    ctx.set_gmres_path(1)
    ctx.set_fp64_mode(2)
    try:
        x = torch.zeros_like(bd)
        info = kc.gmres_solve(ctx, A, bd, x, restart=30, rtol=1e-10, maxit=30)
        xo, io = orc_gmres(Ah.to_scipy(), b, restart=30, rtol=1e-10, maxit=30)
        assert info["iters"] == io["iters"] == 30
        assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= 1e-10
        x.zero_()
        info = kc.gmres_solve(ctx, A, bd, x, restart=30, rtol=1e-10)
        assert info["status"] == 0
        true = np.linalg.norm(b - Ah.to_scipy() @ x.cpu().numpy()) / np.linalg.norm(b)
        assert true <= 1e-10
        _, io = orc_gmres(Ah.to_scipy(), b, restart=30, rtol=1e-10)
        assert abs(info["iters"] - io["iters"]) <= 2
    finally:
        ctx.set_fp64_mode(1)
        ctx.set_gmres_path(0)


@pytest.mark.parametrize("path", PATHS, indirect=True)
def test_early_convergence_inside_a_cycle(kc, ctx, path):
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


@pytest.mark.parametrize("make", [lambda: convdiff_csr(31, 2, [7.0, 7.0]),       # m = 961
                                  lambda: convdiff_csr(10, 3, [3.0, 1.0, 0.5]),   # m = 1000
                                  lambda: convdiff_csr(50, 3, [50.0, 25.0, 12.5])])  # m = 125000
def test_cluster_path_matches_multi_kernel_path(kc, ctx, make):
    """The one-launch solves (one cluster, one CTA per SM; ragged row blocks, the basis in
    shared or global memory) take the same iterations as the multi-kernel path, and all
    reach a true residual of 1e-10."""
    Ah = make()
    b = gaussian_vector(Ah.m, 77)
    A = kc.DeviceCSR(Ah)
    bd = torch.as_tensor(b, device="cuda")
    out = {}
    try:
        for p in (1, 2, 3):
            ctx.set_gmres_path(p)
            x = torch.zeros_like(bd)
            info = kc.gmres_solve(ctx, A, bd, x, restart=30, rtol=1e-10)
            xg = x.cpu().numpy()
            true = np.linalg.norm(b - Ah.to_scipy() @ xg) / np.linalg.norm(b)
            assert info["status"] == 0 and true <= 1e-10
            assert abs(true - info["rel_resid_true"]) <= 1e-3 * true
            out[p] = (info, xg)
    finally:
        ctx.set_gmres_path(0)
    for p in (2, 3):
        assert abs(out[1][0]["iters"] - out[p][0]["iters"]) <= 1
        assert out[1][0]["restarts"] == out[p][0]["restarts"]
        x1, xp = out[1][1], out[p][1]
        assert np.linalg.norm(x1 - xp) / np.linalg.norm(x1) <= 1e-6


def test_cluster_path_on_stencil_operator(kc, ctx):
    import synth
    st = synth.config1_stencil()
    Ah = config1_operator()
    b = gaussian_vector(st.m, 1001)
    bd = torch.as_tensor(b, device="cuda")
    x = torch.zeros_like(bd)
    ctx.set_gmres_path(2)
    try:
        info = kc.gmres_solve(ctx, kc.DeviceStencil7(st), bd, x, restart=30, rtol=1e-10)
    finally:
        ctx.set_gmres_path(0)
    _, io = orc_gmres(Ah.to_scipy(), b, restart=30, rtol=1e-10)
    xg = x.cpu().numpy()
    assert info["status"] == 0
    assert np.linalg.norm(b - Ah.to_scipy() @ xg) / np.linalg.norm(b) <= 1e-10
    assert abs(info["iters"] - io["iters"]) <= 2


@pytest.mark.parametrize("path", PATHS, indirect=True)
def test_iteration_cap_and_zero_rhs(kc, ctx, path):
    """maxit below one cycle: the cycle runs, the solve stops unconverged with the same
    count on both paths; b = 0 returns x = 0 at once."""
    Ah = config1_operator()
    A = kc.DeviceCSR(Ah)
    bd = torch.as_tensor(gaussian_vector(Ah.m, 1001), device="cuda")
    x = torch.zeros_like(bd)
    info = kc.gmres_solve(ctx, A, bd, x, restart=30, rtol=1e-10, maxit=10)
    assert info["status"] == 5 and info["iters"] == 30 and info["restarts"] == 1
    z = torch.zeros_like(bd)
    x = torch.ones_like(bd)
    info = kc.gmres_solve(ctx, A, z, x, restart=30, rtol=1e-10)
    assert info["status"] == 0 and info["iters"] == 0
    assert torch.count_nonzero(x).item() == 0


def test_grid_barrier_wait_is_bounded(kc, ctx):
    """Failure detection without a GPU fault: the test hook makes the grid form's first
    barrier wait for an arrival that never comes; every CTA gives up after about a second,
    the solve reports KC_ERR_TIMEOUT (7), and the next solve on the context succeeds."""
    Ah = config1_operator()
    A = kc.DeviceCSR(Ah)
    bd = torch.as_tensor(gaussian_vector(Ah.m, 1001), device="cuda")
    x = torch.zeros_like(bd)
    ctx.set_gmres_path(3)
    try:
        assert ctx.lib.kc_set_barrier_test(ctx.handle, 1) == 0
        with pytest.raises(kc.KrylovError) as e:
            kc.gmres_solve(ctx, A, bd, x, restart=30, rtol=1e-10)
        assert e.value.status == 7
        x.zero_()
        info = kc.gmres_solve(ctx, A, bd, x, restart=30, rtol=1e-10)
        assert info["status"] == 0 and info["rel_resid_true"] <= 1e-10
    finally:
        ctx.set_gmres_path(0)
