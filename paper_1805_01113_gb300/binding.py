"""ctypes binding of include/mls.h: the same entry points, structures and codes.

Argument marshalling only: every computation runs in libmls_gb300.so.  Loading
fails loudly when the library has not been built; there is no fallback.
"""

import ctypes as C
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libmls_gb300.so")

MLS_OK = 0
MLS_ERR_INVALID_ARG = 1
MLS_ERR_CAPACITY = 2
MLS_ERR_UNSUPPORTED = 3
MLS_ERR_CUDA = 4
MLS_ERR_OUT_OF_DOMAIN = 5

MLS_EXACT = 0
MLS_FAST = 1
MLS_SURROGATE = 2
MLS_MLP_PARAMS = 6363
MLS_TABLE_ROW = 28

MLS_F64 = 0
MLS_F32 = 1
MLS_BF16 = 2

MLS_NOALLOC_MAX_MARKERS = 262144
MLS_NOALLOC_MAX_BINS = 266240


class mls_grid(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("periodic", C.c_int32 * 3), ("faces", C.POINTER(C.c_double) * 3)]


class mls_options(C.Structure):
    _fields_ = [("real", C.c_int32), ("field", C.c_int32), ("eps", C.c_double), ("n_sub", C.c_int32),
                ("brick_log2", C.c_int32 * 3), ("cond_max", C.c_double), ("refine", C.c_int32),
                ("residual_max", C.c_double), ("basis", C.c_int32)]


class mls_transfer_arrays(C.Structure):
    _fields_ = [("M", C.c_int64), ("phi", C.c_void_p), ("c", C.c_void_p), ("home", C.c_void_p),
                ("perm", C.c_void_p), ("capacity", C.c_int64)]


class mls_status(C.Structure):
    _fields_ = [("dropped", C.c_int64), ("nonfinite", C.c_int64), ("refined_fp64", C.c_int64),
                ("surrogate_fallback", C.c_int64)]


class mls_train_options(C.Structure):
    _fields_ = [("n_samples", C.c_int64), ("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_double),
                ("lr_final", C.c_double), ("seed", C.c_uint64)]


class mls_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char_p), ("launches", C.c_int64), ("total_ms", C.c_double)]


# name -> (restype, argtypes); every entry point declared in include/mls.h.
SIGNATURES = {
    "mls_options_default": (C.c_int, [C.POINTER(mls_options)]),
    "mls_create": (C.c_int, [C.POINTER(mls_grid), C.POINTER(mls_options), C.POINTER(C.c_void_p)]),
    "mls_destroy": (C.c_int, [C.c_void_p]),
    "mls_transfer_create": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_void_p)]),
    "mls_transfer_destroy": (C.c_int, [C.c_void_p]),
    "mls_marker_prep": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                  C.c_void_p, C.c_void_p]),
    "mls_marker_prep_range": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int64,
                                        C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mls_marker_prep_locate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                         C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mls_build_transfer": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                     C.c_void_p]),
    "mls_interpolate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mls_build_interpolate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                        C.c_void_p, C.c_void_p, C.c_void_p]),
    "mls_build_direct_forcing": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                           C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_void_p]),
    "mls_spread": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mls_interpolate_gradient": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mls_direct_forcing": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p]),
    "mls_collisions": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p]),
    "mls_refine_markers": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_double, C.c_int32,
                                     C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p]),
    "mls_transfer_view": (C.c_int, [C.c_void_p, C.POINTER(mls_transfer_arrays)]),
    "mls_transfer_status": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(mls_status)]),
    "mls_fast_table": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_int64),
                                 C.POINTER(C.c_int32)]),
    "mls_build_transfer_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                             C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                             C.c_void_p]),
    "mls_train_options_default": (C.c_int, [C.POINTER(mls_train_options)]),
    "mls_surrogate_train": (C.c_int, [C.c_void_p, C.POINTER(mls_train_options), C.c_void_p, C.POINTER(C.c_double)]),
    "mls_surrogate_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32]),
    "mls_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "mls_load": (C.c_int, [C.c_void_p, C.c_char_p]),
    "mls_surrogate_samples": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_uint64, C.c_void_p, C.c_void_p,
                                        C.c_void_p]),
    "mls_surrogate_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]),
    "mls_surrogate_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                          C.c_void_p]),
    "mls_timing_enable": (C.c_int, [C.c_void_p, C.c_int32]),
    "mls_timing_read": (C.c_int, [C.c_void_p, C.POINTER(mls_kernel_time), C.c_int32, C.POINTER(C.c_int32)]),
    "mls_strerror": (C.c_char_p, [C.c_int32]),
    "mls_last_error": (C.c_char_p, []),
}

_lib = None


class MlsError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        lib = load()
        msg = lib.mls_last_error().decode(errors="replace")
        super().__init__(f"{where}: {lib.mls_strerror(code).decode()} ({msg})")


def load(path=LIB_PATH):
    """Load libmls_gb300.so and declare its entry points (cached)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run __graft_entry__.build() (nvcc) first; "
                           "there is no CPU fallback")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code, where):
    if code != MLS_OK:
        raise MlsError(code, where)
    return code
