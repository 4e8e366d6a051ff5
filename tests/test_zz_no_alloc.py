"""The allocation-free DCGS2 step (dcgs2_arnoldi_step_noalloc) against the regular one.

Callers that cannot allocate device memory (allocator callbacks, plugins without their
own memory budget) use this entry point; it keeps its reduction scratch in a static
device array.  Two steps in a row through the C ABI must match dcgs2_arnoldi_step in its
all-FP64 mode to the FP64 tolerances used by the other parity tests, and 67 steps cover
every task layout of its reduction and its clamped grid.  This file is named so that
pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import convdiff_csr, gaussian_vector  # noqa: E402


@pytest.fixture(scope="module")
def kc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2104_01253_gb300 as kc
    return kc


def test_noalloc_step_matches_regular_step_twice(kc):
    Ah = convdiff_csr(23, 3, [5.0, 2.5, 1.25])          # m = 12167 (odd): ragged tail
    r0 = torch.as_tensor(gaussian_vector(Ah.m, 1002), device="cuda")
    A = kc.DeviceCSR(Ah)
    ctx = kc.Context(0)
    ctx.set_fp64_mode(0)
    ref = kc.ArnoldiState(Ah.m, 6, kc.KC_F64)
    new = kc.ArnoldiState(Ah.m, 6, kc.KC_F64)
    kc.dcgs2_arnoldi_init(ctx, A, ref, r0)
    kc.dcgs2_arnoldi_init(ctx, A, new, r0)
    lib = ctx.lib
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        kc.dcgs2_arnoldi_step(ctx, A, ref)
        st = lib.dcgs2_arnoldi_step_noalloc(C.byref(A.c), C.byref(new.c), stream)
        assert st == 0, "call %d returned %d" % (call, st)
        torch.cuda.synchronize()
        k = call + 1
        assert new.c.k == ref.c.k == k
        Qr, Qn = ref.Qbuf[:k, :Ah.m].cpu().numpy(), new.Qbuf[:k, :Ah.m].cpu().numpy()
        assert np.abs(Qn - Qr).max() <= 1e-12
        wr, wn = ref.w[:Ah.m].cpu().numpy(), new.w[:Ah.m].cpu().numpy()
        assert np.abs(wn - wr).max() <= 1e-12 * np.abs(wr).max()
        if k >= 2:
            Hr, Hn = ref.H(k, k - 1).cpu().numpy(), new.H(k, k - 1).cpu().numpy()
            assert np.linalg.norm(Hn - Hr) <= 1e-12 * np.linalg.norm(Hr)
    ctx.set_fp64_mode(1)


def test_noalloc_every_task_layout_and_clamped_grid(kc):
    """67 steps at m = 46,656: the reduction's task count k + 1 runs from 1 to 67, through
    every slot layout of the allocation-free step (one, two, four and eight tasks per warp),
    and m / 256 > 152 rows groups clamp its grid to the static array's 152 CTAs.  The final
    Q and H match dcgs2_arnoldi_step (all-FP64 mode) and the FP64 oracle to the parity
    tolerances (H 1e-12 relative, basis 1e-10 absolute), and the status word that
    dcgs2_noalloc_read_status returns after every call is KC_OK."""
    from oracle import arnoldi as orc
    Ah = convdiff_csr(36, 3, [5.0, 2.5, 1.25])          # m = 46656
    n, ncap = 67, 70
    r0h = gaussian_vector(Ah.m, 1003)
    r0 = torch.as_tensor(r0h, device="cuda")
    A = kc.DeviceCSR(Ah)
    ctx = kc.Context(0)
    ctx.set_fp64_mode(0)
    ref = kc.ArnoldiState(Ah.m, ncap, kc.KC_F64)
    new = kc.ArnoldiState(Ah.m, ncap, kc.KC_F64)
    kc.dcgs2_arnoldi_init(ctx, A, ref, r0)
    kc.dcgs2_arnoldi_init(ctx, A, new, r0)
    lib = ctx.lib
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = C.c_int(-1)
    try:
        for call in range(n):
            kc.dcgs2_arnoldi_step(ctx, A, ref)
            assert lib.dcgs2_arnoldi_step_noalloc(C.byref(A.c), C.byref(new.c), stream) == 0
            assert lib.dcgs2_noalloc_read_status(C.byref(status), stream) == 0
            assert status.value == 0, (call, status.value)
    finally:
        ctx.set_fp64_mode(1)
    torch.cuda.synchronize()
    assert new.c.k == ref.c.k == n
    # H columns 0..n-2 are final after n steps; Q columns 0..n-1
    Hr, Hn = ref.H(n, n - 1).cpu().numpy(), new.H(n, n - 1).cpu().numpy()
    Qr, Qn = ref.Qbuf[:n, :Ah.m].cpu().numpy(), new.Qbuf[:n, :Ah.m].cpu().numpy()
    assert np.linalg.norm(Hn - Hr) <= 1e-12 * np.linalg.norm(Hr)
    assert np.abs(Qn - Qr).max() <= 1e-10
    st = orc.DCGS2Arnoldi(Ah.to_scipy(), r0h, ncap)
    for _ in range(n):
        st.step()
    Ho = st.H[:n, :n - 1]
    assert np.linalg.norm(Hn - Ho) <= 1e-12 * np.linalg.norm(Ho)
    assert np.abs(Qn.T - st.Q[:, :n]).max() <= 1e-10


def test_noalloc_rejects_unsupported_sizes(kc):
    Ah = convdiff_csr(6, 3, [1.0, 1.0, 1.0])
    A32 = kc.DeviceCSR(Ah, dtype=torch.float32)
    st = kc.ArnoldiState(Ah.m, 4, kc.KC_F32)
    lib = kc._lib.load()
    assert lib.dcgs2_arnoldi_step_noalloc(C.byref(A32.c), C.byref(st.c), None) == 1
    assert lib.dcgs2_noalloc_read_status(None, None) == 1
