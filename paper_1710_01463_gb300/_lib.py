"""ctypes binding of librsvd.so (argument marshalling only).

The library is loaded from this package directory.  There is no fallback: if
the shared library is missing or cannot be loaded, every call raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librsvd.so")

RSVD_OK = 0
RSVD_ERR_INVALID_SIZE = -1
RSVD_ERR_NULL_POINTER = -2
RSVD_ERR_PRECISION = -3
RSVD_ERR_WORKSPACE = -4
RSVD_ERR_LAUNCH = -5
RSVD_ERR_NONFINITE = -6
RSVD_ERR_SCRATCH_LIMIT = -7
RSVD_ERR_TIMEOUT = -8
RSVD_WARN_NOCONV = 1
RSVD_WARN_CG = 2

RSVD_PATH_EXACT = 1
RSVD_PATH_HOUSEHOLDER = 2

RSVD_F64 = 0
RSVD_F32 = 1
RSVD_TF32 = 2
RSVD_BF16 = 3
RSVD_FLAG_F64_SIMT = 1
RSVD_FLAG_FULL_SVD = 2
RSVD_FLAG_SERIAL = 4
RSVD_FLAG_TEST_NO_EXCHANGE = 1 << 30

EXPORTED = (
    "rsvd_gaussian",
    "rsvd_workspace_size",
    "rsvd_truncate",
    "rsvd_batched_workspace_size",
    "rsvd_truncate_batched",
    "tebd_workspace_size",
    "tebd_bond_update",
    "tebd_product_workspace_size",
    "tebd_product_update",
    "rsvd_factored_workspace_size",
    "rsvd_truncate_factored",
    "rsvd_tol_workspace_size",
    "rsvd_sectors_adaptive_workspace_size",
    "rsvd_truncate_sectors_adaptive",
    "rsvd_truncate_tol",
    "rsvd_status_string",
    "rsvd_profile_enable",
    "rsvd_profile_collect",
    "rsvd_profile_class_name",
    "rsvd_gemm_tc",
    "rsvd_gemm_f64_tc_workspace_size",
    "rsvd_gemm_f64_tc",
    "rsvd_backward_workspace_size",
    "rsvd_truncate_backward_batched",
    "rsvd_complex_workspace_size",
    "rsvd_truncate_complex",
    "rsvd_truncate_sectors_adaptive_device",
    "rsvd_autotune_enable",
    "rsvd_autotune_entries",
    "rsvd_autotune_clear",
    "rsvd_autotune_save",
    "rsvd_autotune_load",
    "rsvd_truncate_noalloc",
    "rsvd_noalloc_scratch_bytes",
)


class RsvdParams(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_int),
        ("p", ctypes.c_int),
        ("q", ctypes.c_int),
        ("prec", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("stream", ctypes.c_uint64),
        ("max_sweeps", ctypes.c_int),
        ("flags", ctypes.c_int),
    ]


class RsvdInfo(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("path", ctypes.c_int),
        ("chol_fallbacks", ctypes.c_int),
        ("jacobi_sweeps", ctypes.c_int),
        ("l", ctypes.c_int),
        ("rotations", ctypes.c_int),
        ("qr_columns", ctypes.c_int),
        ("qr_kflop", ctypes.c_int),
        ("jacobi_pairs", ctypes.c_int),
        ("cg_iterations", ctypes.c_int),
    ]


INFO_INTS = ctypes.sizeof(RsvdInfo) // 4

_lib = None


class RsvdError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = load().rsvd_status_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: status {code} ({msg})")


def status_string(code):
    """rsvd_status_string of a status code."""
    return load().rsvd_status_string(int(code)).decode()


def load():
    """Load librsvd.so (raises OSError if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise OSError(f"librsvd.so not built at {LIB_PATH}; run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    ip = ctypes.POINTER(ctypes.c_int)
    pp = ctypes.POINTER(ctypes.c_void_p)
    par = ctypes.POINTER(RsvdParams)
    lib.rsvd_gaussian.argtypes = [i, i, ctypes.c_uint64, ctypes.c_uint64, vp, i, vp]
    lib.rsvd_workspace_size.argtypes = [i, i, par, ctypes.POINTER(sz)]
    lib.rsvd_truncate.argtypes = [i, i, vp, i, par, vp, vp, i, vp, i, vp, sz, vp, vp]
    lib.rsvd_batched_workspace_size.argtypes = [i, ip, ip, ip, par, ctypes.POINTER(sz)]
    lib.rsvd_truncate_batched.argtypes = [i, ip, ip, pp, ip, ip, par, pp, pp, ip, pp, ip, i, vp, vp, sz, vp, vp]
    lib.tebd_workspace_size.argtypes = [i, i, ip, i, par, ctypes.POINTER(sz)]
    lib.tebd_bond_update.argtypes = [i, i, ip, i, ip, vp, sz, vp, sz, vp, par, vp, vp, sz, vp, vp]
    lib.rsvd_status_string.argtypes = [i]
    lib.rsvd_status_string.restype = ctypes.c_char_p
    lib.rsvd_profile_enable.argtypes = [i]
    lib.rsvd_profile_collect.argtypes = [ctypes.POINTER(ctypes.c_double), ip, i]
    lib.rsvd_gemm_tc.argtypes = [i, i, i, i, vp, i, vp, i, vp, i, vp, i, vp]
    lib.rsvd_gemm_f64_tc_workspace_size.argtypes = [i, i, i]
    lib.rsvd_gemm_f64_tc_workspace_size.restype = sz
    lib.rsvd_gemm_f64_tc.argtypes = [i, i, i, vp, i, vp, i, vp, i, vp, sz, vp, vp]
    lib.rsvd_backward_workspace_size.argtypes = [i, ip, ip, ip, i, ctypes.POINTER(sz)]
    lib.rsvd_truncate_backward_batched.argtypes = [i, ip, ip, ip, i, pp, ip, pp, pp, ip, pp, ip, pp, ip, pp, pp, ip,
                                                   pp, ip, i, ctypes.c_double, vp, sz, vp, vp]
    lib.rsvd_truncate_noalloc.argtypes = [i, i, vp, i, par, vp, vp, i, vp, i, vp, vp]
    lib.rsvd_autotune_enable.argtypes = [i]
    lib.rsvd_autotune_entries.argtypes = []
    lib.rsvd_autotune_clear.argtypes = []
    lib.rsvd_autotune_save.argtypes = [ctypes.c_char_p]
    lib.rsvd_autotune_load.argtypes = [ctypes.c_char_p]
    lib.rsvd_complex_workspace_size.argtypes = [i, i, par, ctypes.POINTER(sz)]
    lib.rsvd_truncate_complex.argtypes = [i, i, vp, i, par, vp, vp, i, vp, i, vp, sz, vp, vp]
    dbl = ctypes.c_double
    lib.tebd_product_workspace_size.argtypes = [i, i, ip, i, i, par, ctypes.POINTER(sz)]
    lib.tebd_product_update.argtypes = [i, i, ip, i, ip, vp, sz, vp, sz, i, vp, vp, par, vp, vp, sz, vp, vp]
    lib.rsvd_factored_workspace_size.argtypes = [i, i, i, par, ctypes.POINTER(sz)]
    lib.rsvd_truncate_factored.argtypes = [i, i, i, vp, i, vp, i, par, vp, vp, i, vp, i, vp, sz, vp, vp]
    lib.rsvd_tol_workspace_size.argtypes = [i, i, i, par, ctypes.POINTER(sz)]
    lib.rsvd_truncate_tol.argtypes = [i, i, vp, i, dbl, i, par, vp, vp, i, vp, i, ip, ctypes.POINTER(dbl), vp, sz, vp,
                                      vp]
    lib.rsvd_sectors_adaptive_workspace_size.argtypes = [i, ip, ip, i, par, ctypes.POINTER(sz)]
    lib.rsvd_truncate_sectors_adaptive.argtypes = [i, ip, ip, pp, ip, ip, par, i, pp, pp, ip, pp, ip, vp, ip, vp, sz,
                                                   vp, vp]
    lib.rsvd_truncate_sectors_adaptive_device.argtypes = [i, ip, ip, pp, ip, ip, par, i, pp, pp, ip, pp, ip, vp, vp,
                                                          vp, vp, sz, vp, vp]
    lib.rsvd_noalloc_scratch_bytes.argtypes = []
    lib.rsvd_noalloc_scratch_bytes.restype = ctypes.c_size_t
    lib.rsvd_profile_class_name.argtypes = [i]
    lib.rsvd_profile_class_name.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name not in ("rsvd_status_string", "rsvd_profile_class_name", "rsvd_noalloc_scratch_bytes"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def check(code, where):
    if code != RSVD_OK:
        raise RsvdError(code, where)


def int_array(vals):
    return (ctypes.c_int * len(vals))(*[int(v) for v in vals])


def ptr_array(vals):
    return (ctypes.c_void_p * len(vals))(*[ctypes.c_void_p(int(v)) for v in vals])
