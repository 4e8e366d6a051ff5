"""ctypes binding of libkrylov (include/krylov.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  The library must have
been built (``paper_2104_01253_gb300.build.build()``); loading fails loudly otherwise:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkrylov.so")

KC_OK, KC_ERR_INVALID_ARG, KC_ERR_CUDA, KC_ERR_OOM, KC_ERR_BREAKDOWN = 0, 1, 2, 3, 4
KC_ERR_NOT_CONVERGED, KC_ERR_NONFINITE, KC_ERR_TIMEOUT, KC_ERR_PYTHAGORAS_NEG = 5, 6, 7, 8
STATUS_NAMES = {0: "KC_OK", 1: "KC_ERR_INVALID_ARG", 2: "KC_ERR_CUDA", 3: "KC_ERR_OOM",
                4: "KC_ERR_BREAKDOWN", 5: "KC_ERR_NOT_CONVERGED", 6: "KC_ERR_NONFINITE",
                7: "KC_ERR_TIMEOUT", 8: "KC_ERR_PYTHAGORAS_NEG"}
KC_F64, KC_F32, KC_BF16 = 0, 1, 2


class kc_csr(C.Structure):
    _fields_ = [("m", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("val", C.c_void_p), ("val_dtype", C.c_int32),
                ("grid", C.c_int32 * 3), ("stencil", C.c_double * 7)]


class kc_arnoldi(C.Structure):
    _fields_ = [("Q", C.c_void_p), ("ldq", C.c_int64), ("ncap", C.c_int32),
                ("q_dtype", C.c_int32), ("w", C.c_void_p), ("v", C.c_void_p),
                ("H", C.c_void_p), ("ldh", C.c_int32), ("K", C.c_void_p), ("k", C.c_int32),
                ("finished", C.c_int32)]


class kc_gmres_opts(C.Structure):
    _fields_ = [("restart", C.c_int32), ("maxit", C.c_int32), ("precision", C.c_int32),
                ("max_outer", C.c_int32), ("rtol", C.c_double), ("inner_rtol", C.c_double),
                ("inner_max_cycles", C.c_int32), ("precond", C.c_int32),
                ("diag_loo", C.c_int32)]


class kc_gmres_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("restarts", C.c_int32), ("outer", C.c_int32),
                ("status", C.c_int32), ("rel_resid_est", C.c_double),
                ("rel_resid_true", C.c_double), ("max_loo", C.c_double)]


class kc_ks_opts(C.Structure):
    _fields_ = [("nev", C.c_int32), ("ncv", C.c_int32), ("nkeep", C.c_int32),
                ("maxrestarts", C.c_int32), ("tol", C.c_double)]


_P = C.c_void_p
_SIGS = {
    "kc_create": ([C.POINTER(C.c_void_p), C.c_int, _P], C.c_int),
    "kc_destroy": ([_P], C.c_int),
    "kc_set_stream": ([_P, _P], C.c_int),
    "kc_set_fp64_mode": ([_P, C.c_int], C.c_int),
    "kc_get_fp64_mode": ([_P], C.c_int),
    "kc_set_staged": ([_P, C.c_int], C.c_int),
    "kc_last_error": ([_P], C.c_char_p),
    "kc_device_info": ([_P, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "kc_launch_count": ([_P], C.c_int64),
    "kc_read_status": ([_P, C.POINTER(C.c_int)], C.c_int),
    "kc_timing_enable": ([_P, C.c_int], C.c_int),
    "kc_timing_read": ([_P, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int], C.c_int),
    "kc_last_scalars": ([_P, C.POINTER(C.c_double), C.POINTER(C.c_double),
                         C.POINTER(C.c_double)], C.c_int),
    "kc_spmv": ([_P, C.POINTER(kc_csr), _P, _P], C.c_int),
    "dcgs2_arnoldi_init": ([_P, C.POINTER(kc_csr), C.POINTER(kc_arnoldi), _P], C.c_int),
    "dcgs2_arnoldi_step": ([_P, C.POINTER(kc_csr), C.POINTER(kc_arnoldi)], C.c_int),
    "dcgs2_arnoldi_finish": ([_P, C.POINTER(kc_csr), C.POINTER(kc_arnoldi)], C.c_int),
    "dcgs2_arnoldi_step_noalloc": ([C.POINTER(kc_csr), C.POINTER(kc_arnoldi), _P], C.c_int),
    "dcgs2_noalloc_read_status": ([C.POINTER(C.c_int), _P], C.c_int),
    "dcgs2_part_reduce": ([_P, C.POINTER(kc_csr), C.POINTER(kc_arnoldi), _P, _P], C.c_int),
    "dcgs2_part_update": ([_P, C.POINTER(kc_csr), C.POINTER(kc_arnoldi), _P], C.c_int),
    "dcgs2_part_finish": ([_P, C.POINTER(kc_csr), C.POINTER(kc_arnoldi), C.c_int, _P, _P],
                          C.c_int),
    "kc_basis_gram": ([_P, _P, C.c_int64, C.c_int, C.c_int64, C.c_int, _P], C.c_int),
    "dcgs2_qr": ([_P, _P, C.c_int64, C.c_int64, C.c_int, _P, C.c_int64, _P, C.c_int], C.c_int),
    "icwy_qr": ([_P, _P, C.c_int64, C.c_int64, C.c_int, _P, C.c_int64, _P, C.c_int], C.c_int),
    "icwy_arnoldi_step": ([_P, C.POINTER(kc_csr), C.POINTER(kc_arnoldi)], C.c_int),
    "icwy_arnoldi_finish": ([_P, C.POINTER(kc_csr), C.POINTER(kc_arnoldi)], C.c_int),
    "cgs2_arnoldi_init": ([_P, C.POINTER(kc_csr), C.POINTER(kc_arnoldi), _P], C.c_int),
    "cgs2_arnoldi_step": ([_P, C.POINTER(kc_csr), C.POINTER(kc_arnoldi)], C.c_int),
    "mgs_arnoldi_step": ([_P, C.POINTER(kc_csr), C.POINTER(kc_arnoldi)], C.c_int),
    "gmres_solve": ([_P, C.POINTER(kc_csr), C.POINTER(kc_csr), _P, _P,
                     C.POINTER(kc_gmres_opts), C.POINTER(kc_gmres_info)], C.c_int),
    "kc_set_conv_kernel": ([_P, C.c_int], C.c_int),
    "kc_set_gmres_path": ([_P, C.c_int], C.c_int),
    "kc_set_barrier_test": ([_P, C.c_int], C.c_int),
    "kc_cnn_param_count": ([], C.c_int64),
    "kc_cnn_forward": ([_P, _P, _P, _P, C.c_int, C.c_int, C.c_int], C.c_int),
    "kc_cnn_train_step": ([_P, _P, _P, _P, C.c_int64, C.c_float, _P, _P, C.c_int, C.c_int,
                           C.c_int, _P, _P, C.POINTER(C.c_double)], C.c_int),
    "kc_cnn_train_step_residual": ([_P, _P, _P, _P, C.c_int64, C.c_float, C.POINTER(kc_csr), _P,
                                    _P, C.c_int, C.c_int, C.c_int, _P, _P,
                                    C.POINTER(C.c_double)], C.c_int),
    "kc_cnn_residual_sample": ([_P, C.POINTER(kc_csr), _P, _P, _P, _P, C.POINTER(C.c_double)],
                               C.c_int),
    "fgmres_solve": ([_P, C.POINTER(kc_csr), _P, C.c_int, C.c_int, _P, _P,
                      C.POINTER(kc_gmres_opts), C.POINTER(kc_gmres_info)], C.c_int),
    "krylov_schur_eigs": ([_P, C.POINTER(kc_csr), _P, C.POINTER(kc_ks_opts),
                           C.POINTER(C.c_double), C.POINTER(C.c_double),
                           C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_int),
                           C.POINTER(C.c_int)], C.c_int),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libkrylov.so and declare every entry point's signature."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libkrylov.so is not built (%s); run paper_2104_01253_gb300.build" % path)
    lib = C.CDLL(path)
    for name, (args, res) in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def exported_names():
    return list(_SIGS)


class KrylovError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def check(ctx_ptr, status):
    if status != KC_OK:
        msg = load().kc_last_error(ctx_ptr)
        raise KrylovError(status, msg.decode() if msg else "")
    return status
