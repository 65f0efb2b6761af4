"""ctypes declarations of the C ABI in include/lcp_gb300.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblcp_gb300.so")

LCP_OK = 0
LCP_ERR_INVALID_ARG = -1
LCP_ERR_OOM = -2
LCP_ERR_CUDA = -3
LCP_ERR_NOT_CONVERGED = -4
LCP_ERR_NUMERICAL = -5
LCP_ERR_TIMEOUT = -6
LCP_ERR_REJECTED = -8
LCP_FP64, LCP_MIXED, LCP_DF64 = 0, 1, 2
LCP_MONO_PQN, LCP_BI_PQN, LCP_BB_PGD = 0, 1, 2
LCP_HIGH, LCP_LOW_RPY, LCP_LOW_BIE = 0, 1, 2
LCP_WARM_SLIP, LCP_WARM_FORCES, LCP_WARM_NO_INIT = 1, 2, 4

STATUS_NAMES = {0: "LCP_OK", -1: "LCP_ERR_INVALID_ARG", -2: "LCP_ERR_OOM", -3: "LCP_ERR_CUDA",
                -4: "LCP_ERR_NOT_CONVERGED", -5: "LCP_ERR_NUMERICAL", -6: "LCP_ERR_TIMEOUT",
                -8: "LCP_ERR_REJECTED"}


class lcp_config(ctypes.Structure):
    _fields_ = [("n_theta", ctypes.c_int), ("n_phi", ctypes.c_int), ("radius", ctypes.c_double),
                ("contact_radius", ctypes.c_double), ("viscosity", ctypes.c_double),
                ("dt", ctypes.c_double), ("delta", ctypes.c_double), ("precision", ctypes.c_int),
                ("gmres_tol", ctypes.c_double), ("gmres_restart", ctypes.c_int),
                ("gmres_maxit", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("ir_maxit", ctypes.c_int), ("kmax", ctypes.c_int), ("kmax_inner", ctypes.c_int),
                ("memory", ctypes.c_int), ("ssn_maxit", ctypes.c_int), ("forcing", ctypes.c_double),
                ("precondition", ctypes.c_int), ("residual_precision", ctypes.c_int),
                ("autotune", ctypes.c_int), ("own_stream", ctypes.c_int), ("h0_scaling", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p), ("lowfi_n_theta", ctypes.c_int),
                ("lowfi_n_phi", ctypes.c_int), ("lowfi_tol", ctypes.c_double),
                ("init_forcing", ctypes.c_double), ("warm_start", ctypes.c_int),
                ("recycle", ctypes.c_int), ("self_quadrature", ctypes.c_int)]


class lcp_contact(ctypes.Structure):
    _fields_ = [("i", ctypes.c_int), ("j", ctypes.c_int), ("normal", ctypes.c_double * 3),
                ("gap", ctypes.c_double)]


class lcp_stats(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int), ("iterations", ctypes.c_int), ("hi_mvps", ctypes.c_int),
                ("lo_mvps", ctypes.c_int), ("inner_iterations", ctypes.c_int),
                ("gmres_iterations", ctypes.c_int), ("fp64_applies", ctypes.c_int),
                ("fp32_applies", ctypes.c_int), ("kkt_abs", ctypes.c_double),
                ("kkt_dot", ctypes.c_double), ("e_mvps", ctypes.c_double),
                ("hi_mvp_seconds", ctypes.c_double), ("lo_mvp_seconds", ctypes.c_double),
                ("seconds", ctypes.c_double), ("df64_applies", ctypes.c_int), ("resets", ctypes.c_int),
                ("ssn_iterations", ctypes.c_int), ("ssn_fallbacks", ctypes.c_int), ("h0_delta", ctypes.c_double),
                ("unc_gmres_iterations", ctypes.c_int), ("unc_warm_started", ctypes.c_int),
                ("lo_gmres_iterations", ctypes.c_int), ("recycled_solves", ctypes.c_int),
                ("warm_x0", ctypes.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.c_int

PROTOTYPES = {
    "lcp_default_config": (None, [ctypes.POINTER(lcp_config)]),
    "lcp_setup": (_I, [ctypes.POINTER(lcp_config), _I, _D, _D, _I, ctypes.POINTER(lcp_contact),
                       ctypes.POINTER(_P)]),
    "lcp_destroy": (None, [_P]),
    "lcp_update": (_I, [_P, _D, _D, _I, ctypes.POINTER(lcp_contact)]),
    "lcp_update_dev": (_I, [_P, _P, _P]),
    "lcp_step": (_I, [_P, ctypes.c_double, _D, _D]),
    "lcp_profile": (_I, [_P, _I]),
    "lcp_launch_count": (_I, [_P, ctypes.POINTER(ctypes.c_ulonglong)]),
    "lcp_self_correction": (_I, [ctypes.c_int, ctypes.c_int, ctypes.c_double, _P]),
    "lcp_solve_counters": (_I, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    "lcp_profile_read": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double)]),
    "lcp_last_error": (ctypes.c_char_p, [_P]),
    "lcp_sizes": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "lcp_get_contacts": (_I, [_P, ctypes.POINTER(lcp_contact)]),
    "lcp_get_b": (_I, [_P, _D]),
    "lcp_get_unc": (_I, [_P, _D]),
    "mobility_apply": (_I, [_P, _D, _D, _I, _I]),
    "mobility_apply_dev": (_I, [_P, _P, _P, _I, _I]),
    "lcp_apply_A": (_I, [_P, _D, _D, _I]),
    "lcp_solve": (_I, [_P, _I, ctypes.c_double, _D, _D, ctypes.POINTER(lcp_stats)]),
    "lcp_solve_dev": (_I, [_P, _I, ctypes.c_double, _P, _P, ctypes.POINTER(lcp_stats)]),
    "lcp_stokes_apply_dev": (_I, [_P, _P, _P, _I]),
    "lcp_stokes_rhs_dev": (_I, [_P, _P, _I, _P]),
    "lcp_rigid_velocity_dev": (_I, [_P, _P, _P]),
    "lcp_stokes_apply_noalloc": (_I, [_I, _I, _I, ctypes.c_double, _P, _P, _P, _I, _P]),
    "lcp_footprint": (_I, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "lcp_footprint_estimate": (_I, [ctypes.POINTER(lcp_config), _I, _I, ctypes.POINTER(ctypes.c_size_t)]),
    "lcp_kernel_variant": (ctypes.c_char_p, [_P]),
    "lcp_select_kernel_variant": (_I, [_P, ctypes.c_char_p]),
    "lcp_batch_solve": (_I, [ctypes.POINTER(_P), _I, _I, ctypes.c_double, ctypes.POINTER(_P),
                             ctypes.POINTER(lcp_stats), ctypes.POINTER(_I), _I]),
    "lcp_server_create": (_I, [_I, ctypes.c_size_t, ctypes.POINTER(_P)]),
    "lcp_server_destroy": (None, [_P]),
    "lcp_server_admit": (_I, [_P, _P]),
    "lcp_server_release": (_I, [_P, _P]),
    "lcp_server_submit": (_I, [_P, _P, _I, ctypes.c_double, ctypes.POINTER(ctypes.c_uint64)]),
    "lcp_server_poll": (_I, [_P, ctypes.c_uint64, _D, _I, ctypes.POINTER(lcp_stats), _I]),
    "lcp_server_stats": (_I, [_P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "lcp_server_open": (_I, [_P, ctypes.POINTER(lcp_config), _I, _D, _D, ctypes.POINTER(ctypes.c_uint64)]),
    "lcp_server_request": (_I, [_P, ctypes.c_uint64, _I, ctypes.c_double, ctypes.c_double,
                                ctypes.POINTER(ctypes.c_uint64)]),
    "lcp_server_close": (_I, [_P, ctypes.c_uint64]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the compiled library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with `python -m paper_2604_10089_gb300.build`")
        lib = ctypes.CDLL(path)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
