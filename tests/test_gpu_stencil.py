"""GPU parity of the matrix-free 7-point stencil operator against the oracle.

The stencil kernel sums a row's terms in CSR column order, so on the coefficients of the
equivalent CSR matrix its product is bitwise that of the CSR SpMV, and every Krylov result
built on it equals the CSR run bit for bit.  Against the oracle: the product to a few ulps
of sum |c| |x|, DCGS2-Arnoldi H to 1e-12 relative, converged solves to a true FP64
residual of 1e-10, Manteuffel eigenvalues to the closed form.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import arnoldi as orc  # noqa: E402
from oracle.gmres import ir as orc_ir  # noqa: E402
from oracle.metrics import loo, rre  # noqa: E402
from oracle.stencil import stencil7_matrix, stencil7_matvec  # noqa: E402
import synth  # noqa: E402
from synth import gaussian_vector  # noqa: E402


@pytest.fixture(scope="module")
def kc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2104_01253_gb300 as kc
    return kc


@pytest.fixture(scope="module")
def ctx(kc):
    return kc.Context(0)


GRIDS = [(1, 1, 1), (7, 1, 1), (1, 5, 3), (37, 23, 11), (100, 100, 1), (252, 252, 5)]


@pytest.mark.parametrize("grid", GRIDS)
def test_stencil_product_matches_oracle(kc, ctx, grid):
    rng = np.random.default_rng(int(np.prod(grid)))
    c = tuple(rng.standard_normal(7))
    m = int(np.prod(grid))
    A = kc.DeviceStencil7(synth.Stencil7(grid, c))
    x = gaussian_vector(m, 11)
    xd = torch.as_tensor(x, device="cuda")
    y = torch.zeros_like(xd)
    kc.kc_spmv(ctx, A, xd, y)
    ref = stencil7_matvec(grid, c, x)
    scale = stencil7_matvec(grid, np.abs(c), np.abs(x))      # sum |c| |x| per row
    assert np.all(np.abs(y.cpu().numpy() - ref) <= 8 * 2.0 ** -53 * scale)


@pytest.mark.parametrize("grid", [(37, 23, 11), (100, 100, 1)])
def test_stencil_product_fp32(kc, ctx, grid):
    rng = np.random.default_rng(3)
    c = tuple(rng.standard_normal(7))
    m = int(np.prod(grid))
    A32 = kc.DeviceStencil7(synth.Stencil7(grid, c), dtype=torch.float32)
    x = gaussian_vector(m, 12).astype(np.float32)
    xd = torch.as_tensor(x, device="cuda")
    y = torch.zeros_like(xd)
    kc.kc_spmv(ctx, A32, xd, y)
    c32 = np.asarray(c, dtype=np.float32).astype(np.float64)
    ref = stencil7_matvec(grid, c32, x.astype(np.float64))
    scale = stencil7_matvec(grid, np.abs(c32), np.abs(x.astype(np.float64)))
    assert np.all(np.abs(y.cpu().numpy() - ref) <= 8 * 2.0 ** -24 * scale)


@pytest.mark.parametrize("N,dim", [(24, 3), (61, 2)])
def test_stencil_product_bitwise_equals_csr(kc, ctx, N, dim):
    wind = [50.0, 25.0, 12.5][:dim]
    As = kc.DeviceStencil7(synth.convdiff_stencil7(N, dim, wind))
    Ac = kc.DeviceCSR(synth.convdiff_csr(N, dim, wind))
    x = torch.as_tensor(gaussian_vector(As.m, 13), device="cuda")
    ys = torch.zeros_like(x)
    yc = torch.zeros_like(x)
    kc.kc_spmv(ctx, As, x, ys)
    kc.kc_spmv(ctx, Ac, x, yc)
    assert torch.equal(ys, yc)


def _arnoldi(kc, ctx, A, m, r0, n):
    st = kc.ArnoldiState(m, n + 1, kc.KC_F64)
    kc.dcgs2_arnoldi_init(ctx, A, st, torch.as_tensor(r0, device="cuda"))
    for _ in range(n):
        kc.dcgs2_arnoldi_step(ctx, A, st)
    kc.dcgs2_arnoldi_finish(ctx, A, st)
    torch.cuda.synchronize()
    return st.Q(n + 1).cpu().numpy(), st.H(n + 1, n).cpu().numpy()


STENCILS = [
    ("config2_family_N24", lambda: synth.config2_stencil(24)),            # m = 13,824
    ("manteuffel_k23", lambda: synth.manteuffel_stencil7(23)),            # m = 529
    ("ragged_37x23x11", lambda: synth.Stencil7((37, 23, 11),
                                               (6.5, -1.2, -0.8, -1.1, -0.9, -1.3, -0.7))),
]


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("name,make", STENCILS)
def test_dcgs2_on_stencil_matches_oracle(kc, ctx, name, make, mode):
    st = make()
    n = 50
    r0 = gaussian_vector(st.m, 1002)
    ctx.set_fp64_mode(mode)
    try:
        Qg, Hg = _arnoldi(kc, ctx, kc.DeviceStencil7(st), st.m, r0, n)
    finally:
        ctx.set_fp64_mode(1)
    Ao = stencil7_matrix(st.grid, st.c)
    Qo, Ho = orc.dcgs2_arnoldi(Ao, r0, n)
    assert np.linalg.norm(Hg - Ho) / np.linalg.norm(Ho) <= 1e-12
    assert np.abs(Qg - Qo).max() <= 1e-10
    assert loo(Qg) <= 1e-13
    assert rre(Ao, Qg, Hg) <= 1e-14
    assert ctx.read_status() == 0


def test_dcgs2_on_stencil_bitwise_equals_csr(kc, ctx):
    st = synth.config2_stencil(24)
    r0 = gaussian_vector(st.m, 1002)
    Qs, Hs = _arnoldi(kc, ctx, kc.DeviceStencil7(st), st.m, r0, 30)
    Qc, Hc = _arnoldi(kc, ctx, kc.DeviceCSR(synth.config2_operator(24)), st.m, r0, 30)
    assert np.array_equal(Hs, Hc) and np.array_equal(Qs, Qc)


def test_gmres_config1_on_stencil(kc, ctx):
    st = synth.config1_stencil()
    Ah = synth.config1_operator()
    b = gaussian_vector(st.m, 1001)
    bd = torch.as_tensor(b, device="cuda")
    xs = torch.zeros_like(bd)
    xc = torch.zeros_like(bd)
    inf_s = kc.gmres_solve(ctx, kc.DeviceStencil7(st), bd, xs, restart=30, rtol=1e-10)
    inf_c = kc.gmres_solve(ctx, kc.DeviceCSR(Ah), bd, xc, restart=30, rtol=1e-10)
    assert inf_s["status"] == 0 and inf_s["iters"] == inf_c["iters"]
    assert torch.equal(xs, xc)
    x = xs.cpu().numpy()
    assert np.linalg.norm(b - Ah.to_scipy() @ x) / np.linalg.norm(b) <= 1e-10


def test_iterative_refinement_with_fp32_stencil(kc, ctx):
    wind = [50.0, 25.0, 12.5]
    st = synth.convdiff_stencil7(30, 3, wind)
    Ah = synth.convdiff_csr(30, 3, wind)
    b = gaussian_vector(st.m, 1004)
    bd = torch.as_tensor(b, device="cuda")
    x = torch.zeros_like(bd)
    info = kc.gmres_solve(ctx, kc.DeviceStencil7(st), bd, x, restart=50, rtol=1e-10,
                          precision=1, A32=kc.DeviceStencil7(st, dtype=torch.float32),
                          inner_rtol=1e-4, inner_max_cycles=3)
    xg = x.cpu().numpy()
    assert info["status"] == 0
    assert np.linalg.norm(b - Ah.to_scipy() @ xg) / np.linalg.norm(b) <= 1e-10
    _, io = orc_ir(Ah.to_scipy(), b, restart=50, inner_rtol=1e-4, inner_max_restarts=2,
                   basis="f32")
    assert abs(info["outer"] - io["outer"]) <= 1


def test_krylov_schur_manteuffel_stencil_closed_form(kc, ctx):
    k, beta = 20, 0.5
    st = synth.manteuffel_stencil7(k, beta)
    v0 = gaussian_vector(st.m, 8)
    res = kc.krylov_schur_eigs(ctx, kc.DeviceStencil7(st), torch.as_tensor(v0, device="cuda"),
                               nev=4, ncv=30, nkeep=15, tol=1e-10)
    assert res["nconv"] == 4
    L = k + 1
    exact = sorted({round(2 * (2 - np.sqrt(1 - (beta / 2) ** 2) *
                                (np.cos(l * np.pi / L) + np.cos(j * np.pi / L))), 12)
                    for l in range(1, k + 1) for j in range(1, k + 1)}, reverse=True)[:4]
    got = np.sort(res["eigs"].real)[::-1]
    assert np.abs(got - np.array(exact)).max() < 1e-7


def test_stencil_rejected_where_entries_are_read(kc, ctx):
    st = synth.Stencil7((8, 8, 1), (4.0, -1.0, -1.0, -1.0, -1.0, 0.0, 0.0))
    A = kc.DeviceStencil7(st)
    b = torch.ones(64, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(kc.KrylovError) as e:
        kc.fgmres_solve(ctx, A, None, 8, 8, b, x, restart=10)
    assert e.value.status == 1
    lib = ctx.lib
    s = kc.ArnoldiState(64, 4, kc.KC_F64)
    assert lib.dcgs2_arnoldi_step_noalloc(C.byref(A.c), C.byref(s.c), None) == 1


def test_stencil_grid_must_match_m(kc, ctx):
    A = kc.DeviceStencil7(synth.Stencil7((4, 4, 4), (6.0, -1, -1, -1, -1, -1, -1)))
    A.c.m = 63
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(kc.KrylovError) as e:
        kc.kc_spmv(ctx, A, x, y)
    assert e.value.status == 1
