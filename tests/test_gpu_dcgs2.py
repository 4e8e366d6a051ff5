"""GPU parity of the DCGS2 / CGS2 / MGS Arnoldi kernels against the FP64 oracle.

Tolerances (FP64): H relative Frobenius <= 1e-12 (the stated bar), basis entries
<= 1e-10 absolute, loss of orthogonality and representation error at O(eps).
"""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import arnoldi as orc  # noqa: E402
from oracle.metrics import loo, rre  # noqa: E402
from synth import CSR, convdiff_csr, gaussian_vector, manteuffel_csr  # noqa: E402

H_TOL = 1e-12


@pytest.fixture(scope="module")
def kc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2104_01253_gb300 as kc
    return kc


@pytest.fixture(scope="module")
def ctx(kc):
    return kc.Context(0)


def _csr_from_scipy(A):
    A = A.tocsr()
    A.sort_indices()
    return CSR(A.shape[0], A.indptr.astype(np.int32), A.indices.astype(np.int32),
               A.data.astype(np.float64))


CASES = [
    ("convdiff3d_N10", lambda: convdiff_csr(10, 3, [1.0, 0.5, 0.25])),        # m = 1000
    ("convdiff2d_N31_odd", lambda: convdiff_csr(31, 2, [7.0, 7.0])),          # m = 961 (odd)
    ("manteuffel_k23", lambda: manteuffel_csr(23)),                          # m = 529
    ("convdiff3d_N37", lambda: convdiff_csr(37, 3, [50.0, 25.0, 12.5])),      # m = 50653
]


def _run_dcgs2(kc, ctx, Ah, r0, n, q_dtype=None):
    q_dtype = kc.KC_F64 if q_dtype is None else q_dtype
    A = kc.DeviceCSR(Ah)
    st = kc.ArnoldiState(Ah.m, n + 1, q_dtype)
    r0d = torch.as_tensor(r0, device="cuda")
    kc.dcgs2_arnoldi_init(ctx, A, st, r0d)
    for _ in range(n):
        kc.dcgs2_arnoldi_step(ctx, A, st)
    kc.dcgs2_arnoldi_finish(ctx, A, st)
    torch.cuda.synchronize()
    return st


@pytest.mark.parametrize("name,make", CASES)
def test_spmv_matches_scipy(kc, ctx, name, make):
    Ah = make()
    A = kc.DeviceCSR(Ah)
    x = gaussian_vector(Ah.m, 5)
    xd = torch.as_tensor(x, device="cuda")
    y = torch.zeros_like(xd)
    kc.kc_spmv(ctx, A, xd, y)
    ref = Ah.to_scipy() @ x
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("staged", [0, 2, 3, 4, 8])
@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("n", [1, 2, 17, 50])
def test_dcgs2_matches_oracle(kc, ctx, name, make, n, mode, staged):
    """The FP64 modes: all-FP64 products (0), FP64 with float-float offload (1) and the
    reduction as exact digit products on the tensor cores (2, which takes precedence over
    the staged reduction); the register-streaming kernels with the bounded FP32 products
    of Q C (staged 0) and without them (4), the tensor-copy staged reduction (2) and that
    with the bulk-copy staged update (3); flag 8 fuses v = A w into the reduction's pass
    for the first steps (k <= 4) in mode 1."""
    Ah = make()
    r0 = gaussian_vector(Ah.m, 1002)
    ctx.set_fp64_mode(mode)
    ctx.set_staged(staged)
    try:
        st = _run_dcgs2(kc, ctx, Ah, r0, n)
    finally:
        ctx.set_fp64_mode(1)
        ctx.set_staged(0)
    Qg = st.Q(n + 1).cpu().numpy()
    Hg = st.H(n + 1, n).cpu().numpy()
    Qo, Ho = orc.dcgs2_arnoldi(Ah.to_scipy(), r0, n)
    assert np.linalg.norm(Hg - Ho) / np.linalg.norm(Ho) <= H_TOL
    assert np.abs(Qg - Qo).max() <= 1e-10
    assert loo(Qg) <= 1e-13
    assert rre(Ah.to_scipy(), Qg, Hg) <= 1e-14
    assert ctx.read_status() == 0


def test_fused_first_steps_agree_with_separate_passes(kc, ctx):
    """With flag 8 the first steps in FP64 mode 1 form v = A w inside the reduction's pass
    (one launch); by default the SpMV and the reduction run apart.  The row arithmetic of v
    is shared, so step 0's v (from the same w = r0) is bitwise equal; later steps and H
    agree to rounding (the sums run in another order), and both runs match the oracle."""
    Ah = convdiff_csr(37, 3, [50.0, 25.0, 12.5])                         # m = 50653
    r0 = gaussian_vector(Ah.m, 1002)
    A = kc.DeviceCSR(Ah)
    n = 8
    runs = []
    for flags in (0, 8):
        ctx.set_staged(flags)
        try:
            st = kc.ArnoldiState(Ah.m, n + 1, kc.KC_F64)
            kc.dcgs2_arnoldi_init(ctx, A, st, torch.as_tensor(r0, device="cuda"))
            kc.dcgs2_arnoldi_step(ctx, A, st)
            v0 = st.v.clone()
            for _ in range(n - 1):
                kc.dcgs2_arnoldi_step(ctx, A, st)
            kc.dcgs2_arnoldi_finish(ctx, A, st)
            torch.cuda.synchronize()
        finally:
            ctx.set_staged(0)
        runs.append((v0, st.Q(n + 1).cpu().numpy(), st.H(n + 1, n).cpu().numpy()))
    assert torch.equal(runs[0][0], runs[1][0])
    Qo, Ho = orc.dcgs2_arnoldi(Ah.to_scipy(), r0, n)
    for _, Qg, Hg in runs:
        assert np.linalg.norm(Hg - Ho) / np.linalg.norm(Ho) <= H_TOL
        assert np.abs(Qg - Qo).max() <= 1e-10
    assert np.linalg.norm(runs[0][2] - runs[1][2]) / np.linalg.norm(Ho) <= 1e-14
    assert ctx.read_status() == 0


@pytest.mark.parametrize("case", ["tiny_entries", "huge_operator"])
def test_offload_falls_back_to_fp64_outside_the_float_range(kc, ctx, case):
    """Operands outside [2^-80, 2^98) take the FP64 path of the offload kernels: a start
    vector with entries of 1e-30 (basis entries far below 2^-80) and an operator scaled by
    1e35 (v = A w above 2^98).  The result must still match the oracle to 1e-12."""
    Ah = convdiff_csr(12, 3, [1.0, 0.5, 0.25])                           # m = 1728
    r0 = gaussian_vector(Ah.m, 1005)
    if case == "tiny_entries":
        r0[::3] *= 1e-30
    else:
        Ah = CSR(Ah.m, Ah.row_ptr, Ah.col_idx, Ah.val * 1e35)
    n = 20
    ctx.set_fp64_mode(1)
    st = _run_dcgs2(kc, ctx, Ah, r0, n)
    Hg = st.H(n + 1, n).cpu().numpy()
    Qg = st.Q(n + 1).cpu().numpy()
    Qo, Ho = orc.dcgs2_arnoldi(Ah.to_scipy(), r0, n)
    assert np.linalg.norm(Hg - Ho) / np.linalg.norm(Ho) <= H_TOL
    assert loo(Qg) <= 1e-13
    assert ctx.read_status() == 0


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_dcgs2_stepwise_state_matches_oracle(kc, ctx, mode):
    """After every step: pending w, the lagged H columns and alpha agree with the oracle.
    (The offload mode's S error shows in w at about 1e-13 relative; H is unaffected.)"""
    ctx.set_fp64_mode(mode)
    Ah = convdiff_csr(9, 3, [3.0, 1.0, 0.5])
    r0 = gaussian_vector(Ah.m, 7)
    A = kc.DeviceCSR(Ah)
    st = kc.ArnoldiState(Ah.m, 12, kc.KC_F64)
    kc.dcgs2_arnoldi_init(ctx, A, st, torch.as_tensor(r0, device="cuda"))
    ref = orc.DCGS2Arnoldi(Ah.to_scipy(), r0, 12)
    for k in range(10):
        kc.dcgs2_arnoldi_step(ctx, A, st)
        alpha_o = ref.step()
        alpha_g, beta_g, s_g = ctx.last_scalars()
        assert abs(alpha_g - alpha_o) <= 1e-13 * alpha_o
        w = st.w[:Ah.m].cpu().numpy()
        assert np.abs(w - ref.w).max() <= 1e-11 * np.abs(ref.w).max()
        if k >= 1:
            Hg = st.H(k + 1, k).cpu().numpy()
            assert np.abs(Hg - ref.H[:k + 1, :k]).max() <= 1e-12 * np.abs(ref.H[:k + 1, :k]).max()
    ctx.set_fp64_mode(1)


@pytest.mark.parametrize("m", [255, 256, 257, 3001])
def test_tensor_core_reduction_scalars_match_exact_sums(kc, ctx, m):
    """Mode 2 on a single step: alpha, beta and s from the tensor-core reduction against
    the oracle's step, on sizes around one 256-row chunk (empty tail, exact fit, one row
    over) and a start vector with a 10^12 dynamic range."""
    rng = np.random.default_rng(m)
    r0 = rng.standard_normal(m)
    r0[::3] *= 1e-12
    Ah = CSR(m, np.arange(m + 1, dtype=np.int32), np.arange(m, dtype=np.int32),
             np.linspace(1.0, 3.0, m))
    A = kc.DeviceCSR(Ah)
    ref = orc.DCGS2Arnoldi(Ah.to_scipy(), r0, 4)
    st = kc.ArnoldiState(m, 4, kc.KC_F64)
    ctx.set_fp64_mode(2)
    try:
        kc.dcgs2_arnoldi_init(ctx, A, st, torch.as_tensor(r0, device="cuda"))
        for _ in range(3):
            kc.dcgs2_arnoldi_step(ctx, A, st)
            alpha_o = ref.step()
            alpha_g, _, _ = ctx.last_scalars()
            assert abs(alpha_g - alpha_o) <= 1e-13 * alpha_o
    finally:
        ctx.set_fp64_mode(1)
    assert ctx.read_status() == 0


def test_tensor_core_reduction_flags_a_basis_entry_out_of_range(kc, ctx):
    """The fixed-point form holds basis entries below 2 in magnitude: a stored column
    entry of 3 (a column far from unit norm) makes the step report KC_ERR_NONFINITE."""
    Ah = convdiff_csr(8, 3, [1.0, 1.0, 1.0])
    r0 = gaussian_vector(Ah.m, 3)
    A = kc.DeviceCSR(Ah)
    st = kc.ArnoldiState(Ah.m, 6, kc.KC_F64)
    ctx.set_fp64_mode(2)
    try:
        kc.dcgs2_arnoldi_init(ctx, A, st, torch.as_tensor(r0, device="cuda"))
        kc.dcgs2_arnoldi_step(ctx, A, st)
        kc.dcgs2_arnoldi_step(ctx, A, st)
        torch.cuda.synchronize()
        assert ctx.read_status() == 0
        st.Qbuf[0, 5] = 3.0
        kc.dcgs2_arnoldi_step(ctx, A, st)
        torch.cuda.synchronize()
        assert ctx.read_status() == kc._lib.KC_ERR_NONFINITE
    finally:
        ctx.set_fp64_mode(1)


def test_first_step_normalises_r0(kc, ctx):
    Ah = convdiff_csr(8, 3, [1.0, 1.0, 1.0])
    r0 = gaussian_vector(Ah.m, 3)
    A = kc.DeviceCSR(Ah)
    st = kc.ArnoldiState(Ah.m, 4, kc.KC_F64)
    kc.dcgs2_arnoldi_init(ctx, A, st, torch.as_tensor(r0, device="cuda"))
    kc.dcgs2_arnoldi_step(ctx, A, st)
    q0 = st.Q(1).cpu().numpy()[:, 0]
    assert np.abs(q0 - r0 / np.linalg.norm(r0)).max() <= 1e-15
    alpha, beta, _ = ctx.last_scalars()
    assert abs(alpha - np.linalg.norm(r0)) <= 1e-13 * alpha


def test_identity_reports_breakdown(kc, ctx):
    Ah = _csr_from_scipy(sp.eye(300, format="csr"))
    A = kc.DeviceCSR(Ah)
    st = kc.ArnoldiState(300, 5, kc.KC_F64)
    kc.dcgs2_arnoldi_init(ctx, A, st, torch.as_tensor(gaussian_vector(300, 9), device="cuda"))
    kc.dcgs2_arnoldi_step(ctx, A, st)
    assert ctx.read_status() == 0
    kc.dcgs2_arnoldi_step(ctx, A, st)
    status = ctx.read_status()
    assert status in (4, 8)        # KC_ERR_BREAKDOWN or KC_ERR_PYTHAGORAS_NEG


@pytest.mark.parametrize("variant", ["cgs2", "mgs"])
def test_baselines_match_oracle(kc, ctx, variant):
    Ah = convdiff_csr(12, 3, [2.0, 1.0, 0.5])
    r0 = gaussian_vector(Ah.m, 11)
    n = 25
    A = kc.DeviceCSR(Ah)
    st = kc.ArnoldiState(Ah.m, n + 1, kc.KC_F64)
    kc.cgs2_arnoldi_init(ctx, A, st, torch.as_tensor(r0, device="cuda"))
    step = kc.cgs2_arnoldi_step if variant == "cgs2" else kc.mgs_arnoldi_step
    for _ in range(n):
        step(ctx, A, st)
    torch.cuda.synchronize()
    Qg = st.Qbuf[:n + 1, :Ah.m].T.cpu().numpy()
    Hg = st.Hbuf[:n, :n + 1].T.cpu().numpy()
    f = orc.cgs2_arnoldi if variant == "cgs2" else orc.mgs_arnoldi
    Qo, Ho = f(Ah.to_scipy(), r0, n)
    assert np.linalg.norm(Hg - Ho) / np.linalg.norm(Ho) <= H_TOL
    assert np.abs(Qg - Qo).max() <= 1e-10
    assert rre(Ah.to_scipy(), Qg, Hg) <= 1e-14
    # the three variants agree with each other on this well-conditioned problem
    Qd, Hd = orc.dcgs2_arnoldi(Ah.to_scipy(), r0, n)
    assert np.linalg.norm(Hg - Hd) / np.linalg.norm(Hd) <= 1e-11


def test_invalid_arguments_are_rejected(kc, ctx):
    Ah = convdiff_csr(6, 3, [1.0, 1.0, 1.0])
    A = kc.DeviceCSR(Ah)
    st = kc.ArnoldiState(Ah.m, 3, kc.KC_F64)
    kc.dcgs2_arnoldi_init(ctx, A, st, torch.as_tensor(gaussian_vector(Ah.m, 1), device="cuda"))
    kc.dcgs2_arnoldi_step(ctx, A, st)
    kc.dcgs2_arnoldi_step(ctx, A, st)              # k = 2: the finish still has column 2
    with pytest.raises(kc.KrylovError):            # basis full: k + 2 > ncap
        kc.dcgs2_arnoldi_step(ctx, A, st)
    bad = kc.ArnoldiState(Ah.m, 3, kc.KC_F64)
    bad.c.ldq = Ah.m - 1
    with pytest.raises(kc.KrylovError):
        kc.dcgs2_arnoldi_init(ctx, A, bad, st.w)
    st32 = kc.ArnoldiState(Ah.m, 3, kc.KC_F32)     # FP32 basis with FP64 matrix values
    with pytest.raises(kc.KrylovError):
        kc.dcgs2_arnoldi_init(ctx, A, st32, st32.w)
