"""ctypes declarations of the liblqcd C ABI (include/lqcd.h)."""
import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_longlong, c_size_t, c_uint, c_void_p

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "liblqcd.so")

LQ_OK = 0
STATUS_NAMES = {0: "LQ_OK", -1: "LQ_ERR_ARG", -2: "LQ_ERR_GEOM", -3: "LQ_ERR_OOM", -4: "LQ_ERR_CUDA",
                -5: "LQ_ERR_TIMEOUT", -6: "LQ_ERR_NUMERIC", -7: "LQ_ERR_UNSUPPORTED"}
LQ_LINKS, LQ_COLOR_MATRIX, LQ_COLOR_VECTOR, LQ_COMPLEX, LQ_REAL, LQ_FERMION = range(6)
LQ_F32, LQ_F64 = 0, 1
(LQ_OP_LOAD, LQ_OP_ADJ, LQ_OP_MUL, LQ_OP_ADD, LQ_OP_SUB, LQ_OP_SCALE, LQ_OP_TRACE, LQ_OP_RETR,
 LQ_OP_STORE) = range(9)


class LqOp(ctypes.Structure):
    _fields_ = [("code", c_int), ("dst", c_int), ("a", c_int), ("b", c_int), ("dir", c_int), ("mu", c_int),
                ("sign", c_int), ("pad", c_int), ("re", c_double), ("im", c_double)]


class LqStoutOpts(ctypes.Structure):
    _fields_ = [("struct_size", c_int), ("reproject", c_int), ("use_graph", c_int), ("variant", c_int),
                ("block", c_int), ("sites_per_thread", c_int), ("work", c_void_p), ("work_bytes", c_size_t)]


class LqBackwardOpts(ctypes.Structure):
    _fields_ = [("struct_size", c_int), ("checkpoint_every", c_int)]


_P = c_void_p
# name: (restype, argtypes)
SIGNATURES = {
    "lq_last_error": (ctypes.c_char_p, []),
    "lq_abi_version": (c_int, []),
    "lq_geom_create": (c_int, [POINTER(c_int), POINTER(_P)]),
    "lq_geom_destroy": (c_int, [_P]),
    "lq_geom_info": (c_int, [_P, POINTER(c_int), POINTER(c_longlong)]),
    "lq_field_bytes": (c_int, [_P, c_int, c_int, POINTER(c_size_t)]),
    "lq_field_alloc": (c_int, [_P, c_int, c_int, _P, POINTER(_P)]),
    "lq_field_wrap": (c_int, [_P, c_int, c_int, _P, c_size_t, POINTER(_P)]),
    "lq_field_free": (c_int, [_P]),
    "lq_field_device_ptr": (c_int, [_P, POINTER(_P)]),
    "lq_field_upload": (c_int, [_P, _P, _P]),
    "lq_field_download": (c_int, [_P, _P, _P]),
    "lq_field_save": (c_int, [_P, ctypes.c_char_p, _P]),
    "lq_field_load": (c_int, [_P, ctypes.c_char_p, _P]),
    "lq_shift": (c_int, [_P, _P, c_int, c_int, _P]),
    "lq_expr_eval": (c_int, [_P, POINTER(LqOp), c_int, POINTER(_P), c_int, POINTER(c_double), _P]),
    "lq_expr_eval_jit": (c_int, [_P, POINTER(LqOp), c_int, POINTER(_P), c_int, POINTER(c_double), _P]),
    "lq_expr_jit_prepare": (c_int, [_P, POINTER(LqOp), c_int, POINTER(_P), c_int, c_int]),
    "lq_jit_cache_dir": (c_int, [ctypes.c_char_p]),
    "lq_jit_stats": (c_int, [POINTER(ctypes.c_longlong)]),
    "lq_reduce_sum": (c_int, [_P, POINTER(c_double), _P]),
    "lq_reduce_trace": (c_int, [_P, POINTER(c_double), _P]),
    "lq_plaquette": (c_int, [_P, POINTER(c_double), _P]),
    "lq_plaquette_sums": (c_int, [_P, c_longlong, c_longlong, POINTER(c_double), _P]),
    "lq_wilson_action": (c_int, [_P, c_double, POINTER(c_double), _P]),
    "lq_stout_smear": (c_int, [_P, c_double, c_int, c_uint, POINTER(LqStoutOpts), _P]),
    "lq_stout_backward": (c_int, [_P, c_double, c_int, c_uint, _P, c_double, _P, _P, POINTER(LqBackwardOpts), _P]),
    "lq_stout_backward_step": (c_int, [_P, _P, _P, _P, _P, _P, _P, c_int, c_double, c_double, c_uint, c_longlong,
                                       c_longlong, _P]),
    "lq_ape_backward": (c_int, [_P, c_double, c_int, c_uint, _P, c_double, _P, _P, POINTER(LqBackwardOpts), _P]),
    "lq_hyp_backward": (c_int, [_P, c_double, c_double, c_double, c_int, _P, c_double, _P, _P,
                                POINTER(LqBackwardOpts), _P]),
    "lq_stout_smear_batch": (c_int, [POINTER(_P), c_int, c_double, c_int, c_uint, POINTER(LqStoutOpts), _P]),
    "lq_stout_smear_noalloc": (c_int, [_P, c_double, c_int, c_uint, _P]),
    "lq_jacobi_smear": (c_int, [_P, _P, c_double, c_int, c_double, c_uint, _P]),
    "lq_jacobi_smear_ex": (c_int, [_P, _P, c_double, c_int, c_double, c_uint, _P, _P]),
    "lq_ape_smear": (c_int, [_P, c_double, c_int, c_uint, _P]),
    "lq_hyp_smear": (c_int, [_P, c_double, c_double, c_double, c_int, _P]),
    "lq_expiq": (c_int, [_P, _P, _P]),
    "lq_stout_ch_stats": (c_int, [_P, c_double, c_int, c_uint, _P, _P]),
    "lq_stout_step_range": (c_int, [_P, _P, c_double, c_uint, c_longlong, c_longlong, POINTER(LqStoutOpts), _P]),
    "lq_stout_smear_host": (c_int, [_P, _P, _P, c_int, c_double, c_int, c_uint, c_int, _P, _P, _P]),
    "lq_peak_probe": (c_int, [c_int, POINTER(c_double), _P]),
    "lq_tune": (c_int, [ctypes.c_char_p]),
    "lq_tune_lookup": (c_int, [c_int, POINTER(c_int), c_uint, POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
    "lq_free_all": (c_int, []),
}

_lib = None


def load():
    """Loads liblqcd.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1105_2279_gb300.build.build_library()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
