"""ctypes binding of libsipg.so (include/sipg.h): argument marshalling only.

Every function here calls the C entry point of the same name; no arithmetic
of the method happens in Python.  Loading fails loudly when the library has
not been built (no CPU fallback exists).
"""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libsipg.so")

SIPG_OK = 0
SIPG_EINVAL = -1
SIPG_ENOMEM_WORKSPACE = -2
SIPG_ECUDA = -3
SIPG_ENOCONV = -4
SIPG_EBREAKDOWN = -5
SIPG_ETIMEOUT = -6
SIPG_EUNSUPPORTED = -7
SIPG_ESTATE = -8
STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM_WORKSPACE", -3: "ECUDA", -4: "ENOCONV",
                -5: "EBREAKDOWN", -6: "ETIMEOUT", -7: "EUNSUPPORTED", -8: "ESTATE"}

SIPG_FP64 = 0
SIPG_FP32 = 1
SIPG_TF32 = 2
SIPG_SMOOTHER_CONSISTENT = 0
SIPG_SMOOTHER_PAPER = 1
SIPG_SMOOTHER_FULL = 2
SIPG_SMOOTHER_CLAMPED = 3
SIPG_GMRES_MAX_RESTART = 64


class sipg_params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("degree", ctypes.c_int), ("log2_cells", ctypes.c_int),
                ("n_levels", ctypes.c_int), ("kappa", ctypes.c_double),
                ("penalty_factor", ctypes.c_double), ("vcycle_precision", ctypes.c_int),
                ("smoother", ctypes.c_int), ("nrhs", ctypes.c_int), ("use_graphs", ctypes.c_int)]


class sipg_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("status", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("nu", ctypes.c_double),
                ("history", ctypes.POINTER(ctypes.c_double)), ("history_capacity", ctypes.c_int),
                ("history_len", ctypes.c_int)]


_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_st = ctypes.c_int

# name -> (restype, argtypes); the list is the ABI checked by the tests
SIGNATURES = {
    "sipg_create": (_st, [ctypes.POINTER(sipg_params), ctypes.POINTER(_vp)]),
    "sipg_destroy": (None, [_vp]),
    "sipg_last_error": (ctypes.c_char_p, [_vp]),
    "sipg_version": (ctypes.c_char_p, []),
    "sipg_workspace_bytes": (ctypes.c_size_t, [_vp]),
    "sipg_bind_workspace": (_st, [_vp, _vp, ctypes.c_size_t, _vp]),
    "sipg_ndofs": (ctypes.c_size_t, [_vp, _i]),
    "sipg_launch_count": (ctypes.c_uint64, [_vp]),
    "sipg_rhs": (_st, [_vp, _vp, _vp, _vp]),
    "sipg_manufactured_source": (_st, [_vp, _vp, _vp]),
    "sipg_apply": (_st, [_vp, _i, _i, _vp, _vp, _vp]),
    "sipg_residual": (_st, [_vp, _i, _i, _vp, _vp, _vp, _vp]),
    "sipg_apply_penalty": (_st, [_vp, _vp, _vp, _vp]),
    "sipg_smooth_colour": (_st, [_vp, _i, _i, _i, _vp, _vp, _vp]),
    "sipg_smooth": (_st, [_vp, _i, _i, _i, _vp, _vp, _vp]),
    "sipg_restrict": (_st, [_vp, _i, _i, _vp, _vp, _vp]),
    "sipg_prolongate_add": (_st, [_vp, _i, _i, _vp, _vp, _vp]),
    "sipg_coarse_solve": (_st, [_vp, _i, _vp, _vp, _vp]),
    "sipg_vcycle": (_st, [_vp, _i, _vp, _vp, _vp]),
    "sipg_solve": (_st, [_vp, _vp, _vp, _d, _i, ctypes.POINTER(sipg_info), _vp]),
    "sipg_solve_zero": (_st, [_vp, _vp, _vp, _d, _i, ctypes.POINTER(sipg_info), _vp]),
    "sipg_adjoint_solve": (_st, [_vp, _vp, _vp, _d, _i, ctypes.POINTER(sipg_info), _vp]),
    "sipg_solve_host": (_st, [_vp, _vp, _vp, _d, _i, ctypes.POINTER(sipg_info), _vp]),
    "sipg_gmres_workspace_bytes": (ctypes.c_size_t, [_vp, _i]),
    "sipg_gmres_solve": (_st, [_vp, _vp, _vp, _d, _i, _i, _vp, ctypes.c_size_t,
                               ctypes.POINTER(sipg_info), _vp]),
    "sipg_gmres_solve_left": (_st, [_vp, _vp, _vp, _d, _i, _i, _vp, ctypes.c_size_t,
                                    ctypes.POINTER(sipg_info), _vp]),
    "sipg_dot": (_st, [_vp, _vp, _vp, _vp, _vp]),
    "sipg_dot_noalloc": (_st, [_vp, _vp, _vp, _vp, _vp]),
    "sipg_selftest_barrier": (_st, [_vp, _i, _vp]),
    "sipg_selftest_mma_tf32": (_st, [_vp, _vp, _vp, _vp, _vp]),
    "sipg_get_constants": (_st, [_vp, _i, _i, _i, _vp, _i, ctypes.POINTER(_i), _vp]),
    "sipg_tuning": (_st, [_vp, _i, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "sipg_batch_create": (_st, [ctypes.POINTER(sipg_params), _i, ctypes.POINTER(_vp)]),
    "sipg_batch_destroy": (None, [_vp]),
    "sipg_batch_last_error": (ctypes.c_char_p, [_vp]),
    "sipg_batch_count": (_i, [_vp]),
    "sipg_batch_member": (_vp, [_vp, _i]),
    "sipg_batch_workspace_bytes": (ctypes.c_size_t, [_vp]),
    "sipg_batch_bind_workspace": (_st, [_vp, _vp, ctypes.c_size_t, _vp]),
    "sipg_batch_solve": (_st, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _d, _i,
                               ctypes.POINTER(sipg_info), _vp]),
}

_lib = None


def load(path=LIB_PATH):
    """Load libsipg.so and declare every entry point; raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"libsipg.so not found at {path}: build it first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SipgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status
