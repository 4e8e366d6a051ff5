"""GB300-native DCGS2 Arnoldi-QR (libkrylov) with a thin Python binding.

The compute path is entirely in libkrylov.so (hand-written sm_103a CUDA behind the C ABI
of include/krylov.h).  PyTorch only supplies device memory and the stream.  Functions
below carry the names of the C entry points and only marshal arguments.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import (KC_BF16, KC_F32, KC_F64, KrylovError, kc_arnoldi, kc_csr, kc_gmres_info,
                   kc_gmres_opts, kc_ks_opts)

__all__ = ["Context", "DeviceCSR", "DeviceStencil7", "ArnoldiState", "kc_spmv",
           "dcgs2_arnoldi_init", "dcgs2_arnoldi_step", "dcgs2_arnoldi_finish", "cgs2_arnoldi_init",
           "cgs2_arnoldi_step", "mgs_arnoldi_step", "gmres_solve", "krylov_schur_eigs",
           "KrylovError", "KC_F64", "KC_F32", "KC_BF16"]

_TORCH_DT = {KC_F64: torch.float64, KC_F32: torch.float32, KC_BF16: torch.bfloat16}


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


class Context:
    """A libkrylov context bound to a CUDA device and stream (default: torch's current)."""

    def __init__(self, device: int = 0, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("libkrylov needs a CUDA GPU")
        self.lib = _lib.load()
        self.device = device
        torch.cuda.set_device(device)
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = C.c_void_p()
        st = self.lib.kc_create(C.byref(h), device, C.c_void_p(stream.cuda_stream))
        if st != 0:
            raise KrylovError(st, "kc_create failed")
        self.handle = h

    def check(self, status):
        return _lib.check(self.handle, status)

    def set_fp64_mode(self, mode: int):
        """0: all FP64 products; 1: FP64 with float-float offload (default); 2: the fused
        reduction as exact fixed-point digit products on the tensor cores."""
        self.check(self.lib.kc_set_fp64_mode(self.handle, mode))

    CONV_MMA_SYNC, CONV_TCGEN05 = 0, 1

    def set_conv_kernel(self, kind: int):
        """Kernel of the network's 32 -> 32 convolutions (CONV_MMA_SYNC or CONV_TCGEN05)."""
        self.check(self.lib.kc_set_conv_kernel(self.handle, int(kind)))

    GMRES_AUTO, GMRES_MULTI_KERNEL, GMRES_CLUSTER, GMRES_GRID = 0, 1, 2, 3

    def set_gmres_path(self, path: int):
        """FP64 gmres_solve path: GMRES_AUTO (by size), GMRES_MULTI_KERNEL, GMRES_CLUSTER
        (the whole solve in one thread-block-cluster launch) or GMRES_GRID (one launch over
        every SM with a bounded grid barrier)."""
        self.check(self.lib.kc_set_gmres_path(self.handle, int(path)))

    STAGED_UPDATE, STAGED_REDUCE = 1, 2

    def set_staged(self, flags: int):
        """Kernel variants of the FP64 basis passes: STAGED_UPDATE (bulk-copy ring) and/or
        STAGED_REDUCE (tensor-copy ring); 0 streams both through registers."""
        self.check(self.lib.kc_set_staged(self.handle, int(flags)))

    @property
    def fp64_mode(self) -> int:
        return int(self.lib.kc_get_fp64_mode(self.handle))

    def set_stream(self, stream):
        self.stream = stream
        self.check(self.lib.kc_set_stream(self.handle, C.c_void_p(stream.cuda_stream)))

    def read_status(self) -> int:
        s = C.c_int()
        self.check(self.lib.kc_read_status(self.handle, C.byref(s)))
        return s.value

    def last_scalars(self):
        a, b, s = C.c_double(), C.c_double(), C.c_double()
        self.check(self.lib.kc_last_scalars(self.handle, C.byref(a), C.byref(b), C.byref(s)))
        return a.value, b.value, s.value

    def device_info(self):
        n, g = C.c_int(), C.c_int()
        self.check(self.lib.kc_device_info(self.handle, C.byref(n), C.byref(g)))
        return n.value, g.value

    KERNEL_KINDS = ("spmv", "reduce", "dcgs2_update", "gemv_sub", "norm", "scale", "axpy",
                    "small", "other", "finish_reduce", "spmv_reduce")

    def timing_enable(self, on=True):
        self.check(self.lib.kc_timing_enable(self.handle, 1 if on else 0))

    def timing_read(self):
        n = len(self.KERNEL_KINDS)
        ms = (C.c_double * n)()
        cnt = (C.c_int64 * n)()
        self.check(self.lib.kc_timing_read(self.handle, ms, cnt, n))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(self.KERNEL_KINDS) if cnt[i]}

    def launch_count(self) -> int:
        return int(self.lib.kc_launch_count(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            self.lib.kc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DeviceCSR:
    """CSR matrix resident on the GPU (int32 indices; FP64 or FP32 values)."""

    def __init__(self, host_csr, dtype=torch.float64, device="cuda"):
        self.m = int(host_csr.m)
        self.row_ptr = torch.as_tensor(np.asarray(host_csr.row_ptr, dtype=np.int32)).to(device)
        self.col_idx = torch.as_tensor(np.asarray(host_csr.col_idx, dtype=np.int32)).to(device)
        self.val = torch.as_tensor(np.asarray(host_csr.val)).to(device=device, dtype=dtype)
        self.nnz = int(self.col_idx.numel())
        self.val_dtype = KC_F64 if dtype == torch.float64 else KC_F32
        self.c = kc_csr(self.m, self.nnz, self.row_ptr.data_ptr(), self.col_idx.data_ptr(),
                        self.val.data_ptr(), self.val_dtype)

    def nbytes(self):
        return (self.row_ptr.numel() * 4 + self.col_idx.numel() * 4 +
                self.val.numel() * self.val.element_size())


class DeviceStencil7:
    """Matrix-free 7-point stencil operator (the kc_csr form with grid[0] > 0): nothing is
    stored on the GPU.  ``stencil`` has ``grid`` = (nx, ny, nz) and ``c`` = (centre, x-1,
    x+1, y-1, y+1, z-1, z+1), e.g. ``synth.config2_stencil()``; dtype selects FP64 or FP32
    vectors (FP32 rounds the coefficients)."""

    def __init__(self, stencil, dtype=torch.float64):
        nx, ny, nz = (int(g) for g in stencil.grid)
        self.m = nx * ny * nz
        self.grid = (nx, ny, nz)
        self.coef = tuple(float(v) for v in stencil.c)
        self.nnz = int(getattr(stencil, "nnz", 0))
        self.val_dtype = KC_F64 if dtype == torch.float64 else KC_F32
        self.c = kc_csr(self.m, self.nnz, None, None, None, self.val_dtype,
                        (C.c_int32 * 3)(nx, ny, nz), (C.c_double * 7)(*self.coef))

    def nbytes(self):
        return 0


class ArnoldiState:
    """Device buffers of an Arnoldi expansion (caller-owned in the C ABI sense).

    Q is stored column-major with leading dimension ldq (a multiple of 8): Q[j] is a view
    of column j.  H and K are FP64, column-major with ld ldh (resp. ncap)."""

    def __init__(self, m: int, ncap: int, q_dtype: int = KC_F64, device="cuda"):
        self.m = m
        self.ncap = ncap
        self.q_dtype = q_dtype
        self.ldq = (m + 7) // 8 * 8
        vdt = torch.float64 if q_dtype == KC_F64 else torch.float32
        self.Qbuf = torch.zeros(ncap, self.ldq, dtype=_TORCH_DT[q_dtype], device=device)
        self.w = torch.zeros(self.ldq, dtype=vdt, device=device)
        self.v = torch.zeros(self.ldq, dtype=vdt, device=device)
        self.ldh = ncap
        self.Hbuf = torch.zeros(ncap - 1, self.ldh, dtype=torch.float64, device=device)
        self.Kbuf = torch.zeros(ncap - 1, ncap, dtype=torch.float64, device=device)
        self.c = kc_arnoldi(self.Qbuf.data_ptr(), self.ldq, ncap, q_dtype, self.w.data_ptr(),
                            self.v.data_ptr(), self.Hbuf.data_ptr(), self.ldh,
                            self.Kbuf.data_ptr(), 0, 0)

    @property
    def k(self):
        return self.c.k

    def Q(self, ncols=None):
        """(m, ncols) view of the basis (float64 copy for BF16)."""
        n = self.c.k + (1 if self.c.finished else 0) if ncols is None else ncols
        return self.Qbuf[:n, :self.m].T

    def H(self, nrows=None, ncols=None):
        ncols = self.c.k if ncols is None else ncols
        nrows = ncols + 1 if nrows is None else nrows
        return self.Hbuf[:ncols, :nrows].T

    def nbytes(self):
        return sum(t.numel() * t.element_size() for t in (self.Qbuf, self.w, self.v, self.Hbuf,
                                                          self.Kbuf))


# ---- entry points (same names as the C ABI) ---------------------------------------------

def kc_spmv(ctx: Context, A: DeviceCSR, x, y):
    ctx.check(ctx.lib.kc_spmv(ctx.handle, C.byref(A.c), _ptr(x), _ptr(y)))


def dcgs2_qr(ctx: Context, A, Q, R):
    """DCGS2 QR (Algorithm 2) of the m x n matrix whose columns are the rows of A
    (a device tensor of shape (n, lda), FP64); writes Q (shape (n, ldq)) and R (shape
    (n, ldr): R[j, i] is entry (i, j) of the upper-triangular factor)."""
    n, m = A.shape
    ctx.check(ctx.lib.dcgs2_qr(ctx.handle, _ptr(A), A.stride(0), m, n, _ptr(Q), Q.stride(0),
                               _ptr(R), R.stride(0)))


def icwy_qr(ctx: Context, A, Q, R):
    """ICWY-MGS QR (Section 5) in the layout of dcgs2_qr."""
    n, m = A.shape
    ctx.check(ctx.lib.icwy_qr(ctx.handle, _ptr(A), A.stride(0), m, n, _ptr(Q), Q.stride(0),
                              _ptr(R), R.stride(0)))


def icwy_arnoldi_step(ctx: Context, A: DeviceCSR, st: ArnoldiState):
    """One ICWY-MGS Arnoldi step (start with dcgs2_arnoldi_init)."""
    ctx.check(ctx.lib.icwy_arnoldi_step(ctx.handle, C.byref(A.c), C.byref(st.c)))


def icwy_arnoldi_finish(ctx: Context, A: DeviceCSR, st: ArnoldiState):
    """Normalise the pending vector into the last basis column."""
    ctx.check(ctx.lib.icwy_arnoldi_finish(ctx.handle, C.byref(A.c), C.byref(st.c)))


def dcgs2_arnoldi_init(ctx: Context, A: DeviceCSR, st: ArnoldiState, r0):
    ctx.check(ctx.lib.dcgs2_arnoldi_init(ctx.handle, C.byref(A.c), C.byref(st.c), _ptr(r0)))


def dcgs2_arnoldi_step(ctx: Context, A: DeviceCSR, st: ArnoldiState):
    ctx.check(ctx.lib.dcgs2_arnoldi_step(ctx.handle, C.byref(A.c), C.byref(st.c)))


def dcgs2_arnoldi_finish(ctx: Context, A: DeviceCSR, st: ArnoldiState):
    ctx.check(ctx.lib.dcgs2_arnoldi_finish(ctx.handle, C.byref(A.c), C.byref(st.c)))


def dcgs2_part_reduce(ctx: Context, A_local: DeviceCSR, st: ArnoldiState, w_ext, partial):
    """Row-partitioned step, first half: v = A_local w_ext and this rank's 2k + 2 partial
    sums [C_0, S_0, ..., beta, s] into the device tensor `partial`."""
    ctx.check(ctx.lib.dcgs2_part_reduce(ctx.handle, C.byref(A_local.c), C.byref(st.c),
                                        _ptr(w_ext), _ptr(partial)))


def dcgs2_part_update(ctx: Context, A_local: DeviceCSR, st: ArnoldiState, totals):
    """Row-partitioned step, second half, from the partial sums summed over the ranks."""
    ctx.check(ctx.lib.dcgs2_part_update(ctx.handle, C.byref(A_local.c), C.byref(st.c),
                                        _ptr(totals)))


def dcgs2_part_finish(ctx: Context, A_local: DeviceCSR, st: ArnoldiState, phase: int,
                      totals=None, partial=None):
    """Row-partitioned CGS2 finish, phase 0..3 (three global sums between the phases)."""
    ctx.check(ctx.lib.dcgs2_part_finish(ctx.handle, C.byref(A_local.c), C.byref(st.c),
                                        int(phase), _ptr(totals) if totals is not None else None,
                                        _ptr(partial) if partial is not None else None))


def cgs2_arnoldi_init(ctx: Context, A: DeviceCSR, st: ArnoldiState, r0):
    ctx.check(ctx.lib.cgs2_arnoldi_init(ctx.handle, C.byref(A.c), C.byref(st.c), _ptr(r0)))


def cgs2_arnoldi_step(ctx: Context, A: DeviceCSR, st: ArnoldiState):
    ctx.check(ctx.lib.cgs2_arnoldi_step(ctx.handle, C.byref(A.c), C.byref(st.c)))


def mgs_arnoldi_step(ctx: Context, A: DeviceCSR, st: ArnoldiState):
    ctx.check(ctx.lib.mgs_arnoldi_step(ctx.handle, C.byref(A.c), C.byref(st.c)))


def gmres_solve(ctx: Context, A: DeviceCSR, b, x, restart=30, rtol=1e-10, maxit=100000,
                precision=0, A32: DeviceCSR = None, max_outer=50, inner_rtol=1e-4,
                inner_max_cycles=3, diag_loo=False, precond: int = 0):
    """Restarted DCGS2-GMRES (precision 0) or FP32 / BF16-basis inner solves in FP64
    iterative refinement (precision 1 / 2).  x holds x0 and receives the solution.
    diag_loo: also report the largest loss of orthogonality over the cycles' bases.
    precond: PREC_AUTO (none) or PREC_JACOBI (right Jacobi, precision 0)."""
    opts = kc_gmres_opts(restart, maxit, precision, max_outer, rtol, inner_rtol,
                         inner_max_cycles, precond, 1 if diag_loo else 0)
    info = kc_gmres_info()
    a32 = C.byref(A32.c) if A32 is not None else None
    st = ctx.lib.gmres_solve(ctx.handle, C.byref(A.c), a32, _ptr(b), _ptr(x), C.byref(opts),
                             C.byref(info))
    if st not in (0, _lib.KC_ERR_NOT_CONVERGED):
        ctx.check(st)
    out = dict(iters=info.iters, restarts=info.restarts, outer=info.outer, status=st,
               rel_resid_est=info.rel_resid_est, rel_resid_true=info.rel_resid_true)
    if diag_loo:
        out["max_loo"] = info.max_loo
    return out


def basis_gram(ctx: Context, Q, m: int, ncols: int, q_dtype=None):
    """G = Q^T Q (FP64, ncols x ncols) of the first ncols columns of a basis stored like
    ArnoldiState.Qbuf (one column per row of the tensor, leading dimension Q.shape[1])."""
    import torch
    dt = {torch.float64: _lib.KC_F64, torch.float32: _lib.KC_F32,
          torch.bfloat16: _lib.KC_BF16}[Q.dtype] if q_dtype is None else q_dtype
    G = torch.empty((ncols, ncols), dtype=torch.float64, device=Q.device)
    ctx.check(ctx.lib.kc_basis_gram(ctx.handle, _ptr(Q), Q.shape[1], dt, m, ncols, _ptr(G)))
    return G


def krylov_schur_eigs(ctx: Context, A: DeviceCSR, v0, nev=10, ncv=40, nkeep=20, tol=1e-10,
                      maxrestarts=500):
    opts = kc_ks_opts(nev, ncv, nkeep, maxrestarts, tol)
    er = (C.c_double * nev)()
    ei = (C.c_double * nev)()
    rs = (C.c_double * nev)()
    nconv, restarts, matvecs = C.c_int(), C.c_int(), C.c_int()
    st = ctx.lib.krylov_schur_eigs(ctx.handle, C.byref(A.c), _ptr(v0), C.byref(opts), er, ei,
                                   rs, C.byref(nconv), C.byref(restarts), C.byref(matvecs))
    if st not in (0, _lib.KC_ERR_NOT_CONVERGED):
        ctx.check(st)
    eigs = np.array(er[:]) + 1j * np.array(ei[:])
    return dict(eigs=eigs, resid=np.array(rs[:]), nconv=nconv.value, restarts=restarts.value,
                matvecs=matvecs.value, status=st)


# ---- learned preconditioner -----------------------------------------------------------------

def kc_cnn_param_count() -> int:
    return int(_lib.load().kc_cnn_param_count())


def kc_cnn_forward(ctx: Context, w32, x, y, B: int, H: int, W: int):
    ctx.check(ctx.lib.kc_cnn_forward(ctx.handle, _ptr(w32), _ptr(x), _ptr(y), B, H, W))


def kc_cnn_train_step(ctx: Context, w32, adam_m, adam_v, t: int, lr: float, x, e, B: int,
                      H: int, W: int, y, grad=None):
    """One forward/backward/Adam step on the GPU; returns the batch loss."""
    loss = C.c_double()
    ctx.check(ctx.lib.kc_cnn_train_step(ctx.handle, _ptr(w32), _ptr(adam_m), _ptr(adam_v), t,
                                        lr, _ptr(x), _ptr(e), B, H, W, _ptr(y), _ptr(grad),
                                        C.byref(loss)))
    return loss.value


def kc_cnn_train_step_residual(ctx: Context, w32, adam_m, adam_v, t: int, lr: float,
                               A: DeviceCSR, x, r, B: int, H: int, W: int, y, grad=None):
    """One step on the residual loss ||A (x + net(x)) - r||^2 / ||r||^2 (x: the
    Jacobi-scaled residuals, r: the residuals, both per sample scaled alike); returns the
    batch loss."""
    loss = C.c_double()
    ctx.check(ctx.lib.kc_cnn_train_step_residual(
        ctx.handle, _ptr(w32), _ptr(adam_m), _ptr(adam_v), t, lr, C.byref(A.c), _ptr(x),
        _ptr(r), B, H, W, _ptr(y), _ptr(grad), C.byref(loss)))
    return loss.value


def kc_cnn_residual_sample(ctx: Context, A: DeviceCSR, b, x, xin, res) -> float:
    """r = b - A x, u = D^{-1} r, s = rms(u): writes xin = u / s and res = r / s (FP32,
    device) and returns ||r||."""
    rn = C.c_double()
    ctx.check(ctx.lib.kc_cnn_residual_sample(ctx.handle, C.byref(A.c), _ptr(b), _ptr(x),
                                             _ptr(xin), _ptr(res), C.byref(rn)))
    return rn.value


PREC_AUTO, PREC_JACOBI = 0, 1


def fgmres_solve(ctx: Context, A: DeviceCSR, w32, H: int, W: int, b, x, restart=40,
                 rtol=1e-10, maxit=100000, precond: int = PREC_AUTO):
    """Flexible GMRES with a right preconditioner: the Jacobi-scaled network (w32), the
    identity (w32 None) or, with precond=PREC_JACOBI, the Jacobi step alone."""
    opts = kc_gmres_opts(restart, maxit, 0, 0, rtol, 0.0, 0, precond)
    info = kc_gmres_info()
    st = ctx.lib.fgmres_solve(ctx.handle, C.byref(A.c), _ptr(w32), H, W, _ptr(b), _ptr(x),
                              C.byref(opts), C.byref(info))
    if st not in (0, _lib.KC_ERR_NOT_CONVERGED):
        ctx.check(st)
    return dict(iters=info.iters, restarts=info.restarts, status=st,
                rel_resid_est=info.rel_resid_est, rel_resid_true=info.rel_resid_true)
