"""ctypes declarations of libmpkrylov.so (include/mpkrylov.h)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmpkrylov.so")

MP_OK, MP_ERR_ARG, MP_ERR_PREC, MP_ERR_ALLOC, MP_ERR_CUDA = 0, 1, 2, 3, 4
MP_ERR_SPAN, MP_ERR_BREAKDOWN, MP_ERR_NOCONV, MP_ERR_TIMEOUT, MP_ERR_DIVZERO = 5, 6, 7, 8, 9
MP_ORDERED, MP_EXACT = 0, 1
MP_OP_MUL, MP_OP_ADD, MP_OP_SUB, MP_OP_DIV = 0, 1, 2, 3
MP_CSR_TRANSPOSE = 1
EXP_ZERO = -(1 << 61)
SPAN_CAP = 16384


class MpVec(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("prec_bits", ctypes.c_int32),
                ("ld", ctypes.c_int64), ("data", ctypes.c_void_p)]


class MpSolveOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("atol", ctypes.c_double),
                ("maxit", ctypes.c_int64), ("mode", ctypes.c_int32),
                ("poll_every", ctypes.c_int32), ("history", MpVec),
                ("transpose", ctypes.c_int32), ("time_limit_ms", ctypes.c_int32)]


class MpSolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("status", ctypes.c_int32),
                ("relres", ctypes.c_double), ("ms", ctypes.c_double)]


class MpRefineOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_outer", ctypes.c_int64),
                ("inner_rtol", ctypes.c_double), ("inner_maxit", ctypes.c_int64),
                ("equilibrate", ctypes.c_int32), ("poll_every", ctypes.c_int32)]


class MpRefineInfo(ctypes.Structure):
    _fields_ = [("outer", ctypes.c_int64), ("inner_iters", ctypes.c_int64),
                ("status", ctypes.c_int32), ("correction", ctypes.c_double),
                ("relres", ctypes.c_double), ("ms", ctypes.c_double)]


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)

SIGNATURES = {
    "mp_csr_create": (_i32, [_i64, _vp, _vp, _vp, _i32, _i32, _vp, ctypes.POINTER(_vp)]),
    "mp_csr_create_f64": (_i32, [_i64, _vp, _vp, _vp, _i32, _i32, _vp, ctypes.POINTER(_vp)]),
    "mp_csr_destroy": (_i32, [_vp]),
    "mp_csr_info": (_i32, [_vp, _i64p, _i64p, _i32p, _i64p, _i64p]),
    "mp_csr_set_config": (_i32, [_vp, _i32, _i32, _i32, _i32]),
    "mp_csr_get_config": (_i32, [_vp, _i32, _i32p, _i32p, _i32p]),
    "mp_csr_tune": (_i32, [_vp, _i32, _i32, _i32p, _i32p, _i32p, ctypes.POINTER(ctypes.c_double),
                           _vp]),
    "mp_spmv": (_i32, [_vp, MpVec, MpVec, _i32, _vp]),
    "mp_spmv_t": (_i32, [_vp, MpVec, MpVec, _i32, _vp]),
    "mp_residual": (_i32, [_vp, MpVec, MpVec, MpVec, _vp]),
    "mp_dot": (_i32, [MpVec, MpVec, MpVec, _vp]),
    "mp_dot_noalloc": (_i32, [MpVec, MpVec, MpVec, _vp]),
    "mp_axpy": (_i32, [MpVec, MpVec, MpVec, _vp]),
    "mp_ewise": (_i32, [_i32, MpVec, MpVec, MpVec, _vp]),
    "mp_vec_from_f64": (_i32, [_vp, MpVec, _vp]),
    "mp_vec_to_f64": (_i32, [MpVec, _vp, _vp]),
    "mp_bicg": (_i32, [_vp, MpVec, MpVec, ctypes.POINTER(MpSolveOpts),
                       ctypes.POINTER(MpSolveInfo), _vp]),
    "mp_gpbicg": (_i32, [_vp, MpVec, MpVec, ctypes.POINTER(MpSolveOpts),
                         ctypes.POINTER(MpSolveInfo), _vp]),
    "mp_cgs": (_i32, [_vp, MpVec, MpVec, ctypes.POINTER(MpSolveOpts),
                      ctypes.POINTER(MpSolveInfo), _vp]),
    "mp_bicgstab": (_i32, [_vp, MpVec, MpVec, ctypes.POINTER(MpSolveOpts),
                           ctypes.POINTER(MpSolveInfo), _vp]),
    "mp_csr_grad": (_i32, [_vp, MpVec, MpVec, MpVec, _vp]),
    "mp_ilu0_create": (_i32, [_vp, _vp, ctypes.POINTER(_vp)]),
    "mp_ilu0_destroy": (_i32, [_vp]),
    "mp_ilu0_info": (_i32, [_vp, _i64p, _i64p]),
    "mp_ilu0_factor": (_i32, [_vp, MpVec, _vp]),
    "mp_ilu0_apply": (_i32, [_vp, MpVec, MpVec, _vp]),
    "mp_bicgstab_ilu0": (_i32, [_vp, _vp, MpVec, MpVec, ctypes.POINTER(MpSolveOpts),
                                ctypes.POINTER(MpSolveInfo), _vp]),
    "mp_bicgstab_ilu0_right": (_i32, [_vp, _vp, MpVec, MpVec, ctypes.POINTER(MpSolveOpts),
                                      ctypes.POINTER(MpSolveInfo), _vp]),
    "mp_gemv": (_i32, [_i64, _i64, MpVec, MpVec, MpVec, _vp]),
    "mp_batch_create_f64": (_i32, [_i32, _vp, _vp, _vp, _vp, _i32, _vp, ctypes.POINTER(_vp)]),
    "mp_batch_destroy": (_i32, [_vp]),
    "mp_batch_info": (_i32, [_vp, _i32p, _i64p, _i64p]),
    "mp_batch_matrix": (_i32, [_vp, ctypes.POINTER(_vp)]),
    "mp_batch_gpbicg": (_i32, [_vp, MpVec, MpVec, ctypes.POINTER(MpSolveOpts),
                               ctypes.POINTER(MpSolveInfo), _vp]),
    "mp_refine": (_i32, [_vp, MpVec, MpVec, ctypes.POINTER(MpRefineOpts),
                         ctypes.POINTER(MpRefineInfo), _vp]),
    "mp_check": (_i32, [_vp]),
    "mp_status_string": (ctypes.c_char_p, [_i32]),
    "mp_last_error": (ctypes.c_char_p, []),
    "mp_launch_count": (_i64, [_i32]),
    "mp_debug_fail": (_i32, [ctypes.c_char_p, _i64]),
    "mp_debug_pool_used": (_i32, [_i64p]),
    "mp_imad_probe": (_i32, [ctypes.POINTER(ctypes.c_double), _vp]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads the native library; raises if it has not been built (there is
    no fallback implementation)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with paper_1411_2377_gb300.build.build() "
            "(nvcc, sm_103a); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib
