"""ctypes declarations of the C ABI in include/efgp.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libefgp.so")

EFGP_OK, EFGP_EINVAL, EFGP_ERANGE, EFGP_ENOMEM, EFGP_ENOTCONV, EFGP_ETIMEOUT, EFGP_ECUDA, EFGP_ESTATE, \
    EFGP_EUNSUPPORTED = range(9)
KERNEL_SE, KERNEL_MATERN = 0, 1
MIXED, FP64, MIXED_CG64 = 0, 1, 2
F32, F64 = 0, 1


class efgp_kernel(C.Structure):
    _fields_ = [("family", C.c_int), ("nu", C.c_double), ("lengthscale", C.c_double), ("variance", C.c_double)]


class efgp_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("coord_dtype", C.c_int), ("value_dtype", C.c_int), ("x_layout", C.c_int),
                ("host_io", C.c_int), ("cg_tol", C.c_double), ("max_iter", C.c_int64), ("nufft_tol", C.c_double),
                ("m_override", C.c_int), ("h_override", C.c_double), ("fft_len_override", C.c_int),
                ("upsampfac", C.c_double), ("es_width", C.c_int), ("iters_per_launch", C.c_int),
                ("autotune", C.c_int), ("profile", C.c_int), ("cg_mode", C.c_int),
                ("stream", C.c_void_p), ("setup_path", C.c_int),
                ("precond", C.c_int)]


class efgp_params(C.Structure):
    _fields_ = [("d", C.c_int), ("h", C.c_double), ("m", C.c_int), ("M", C.c_int64), ("L", C.c_int),
                ("nf1", C.c_int), ("w1", C.c_int), ("beta1", C.c_double), ("upsamp1", C.c_double),
                ("nf2", C.c_int), ("w2", C.c_int), ("beta2", C.c_double), ("upsamp2", C.c_double),
                ("poly_deg1", C.c_int), ("poly_deg2", C.c_int), ("es_err1", C.c_double), ("es_err2", C.c_double),
                ("tile", C.c_int), ("kernel_l2norm", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class efgp_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int64), ("rel_residual", C.c_double), ("true_rel_residual", C.c_double),
                ("converged", C.c_int), ("solve_ms", C.c_double)]


class efgp_phase_times(C.Structure):
    _fields_ = [("bin_count_ms", C.c_double), ("bin_scatter_ms", C.c_double), ("spread_ms", C.c_double),
                ("fine_fft_ms", C.c_double), ("what_ms", C.c_double), ("cg_ms", C.c_double),
                ("predict_fft_ms", C.c_double), ("interp_ms", C.c_double), ("n_setup", C.c_int64),
                ("n_solve", C.c_int64), ("n_predict", C.c_int64), ("launches", C.c_int64),
                ("cg_iters", C.c_int64), ("setups_fused", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class efgp_problem(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("N", C.c_int64), ("d", C.c_int), ("kern", efgp_kernel),
                ("sigma", C.c_double), ("eps", C.c_double)]


# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("efgp_default_options", C.c_int, [C.POINTER(efgp_options)]),
    ("efgp_status_string", C.c_char_p, [C.c_int]),
    ("efgp_last_error", C.c_char_p, []),
    ("efgp_version", C.c_char_p, []),
    ("efgp_plan", C.c_int, [C.c_int, C.c_int64, C.POINTER(efgp_kernel), C.c_double, C.c_double,
                            C.POINTER(efgp_options), C.POINTER(efgp_params)]),
    ("efgp_setup", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.POINTER(efgp_kernel), C.c_double,
                             C.c_double, C.POINTER(efgp_options), C.POINTER(C.c_void_p)]),
    ("efgp_solve", C.c_int, [C.c_void_p, C.POINTER(efgp_solve_info)]),
    ("efgp_predict", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    ("efgp_predict_noalloc", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    ("efgp_destroy", None, [C.c_void_p]),
    ("efgp_get_params", C.c_int, [C.c_void_p, C.POINTER(efgp_params)]),
    ("efgp_get_beta", C.c_int, [C.c_void_p, C.c_void_p]),
    ("efgp_get_phase_times", C.c_int, [C.c_void_p, C.POINTER(efgp_phase_times)]),
    ("efgp_get_system", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("efgp_set_beta", C.c_int, [C.c_void_p, C.c_void_p]),
    ("efgp_apply_system_device", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("efgp_apply_system", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("efgp_batch_setup", C.c_int, [C.POINTER(efgp_problem), C.c_int, C.POINTER(efgp_options),
                                   C.POINTER(C.c_void_p), C.POINTER(C.c_int)]),
    ("efgp_batch_solve", C.c_int, [C.c_void_p, C.POINTER(efgp_solve_info)]),
    ("efgp_batch_predict", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.c_void_p]),
    ("efgp_batch_get_params", C.c_int, [C.c_void_p, C.c_int, C.POINTER(efgp_params)]),
    ("efgp_batch_handle", C.c_void_p, [C.c_void_p, C.c_int]),
    ("efgp_batch_destroy", None, [C.c_void_p]),
]

_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libefgp.so is not built ({LIB_PATH}); run paper_2210_10210_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib
