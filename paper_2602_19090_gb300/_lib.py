"""ctypes loader and signatures of the frx C ABI (include/frx.h)."""
from __future__ import annotations

import ctypes as C
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libfrx.so")

c_i64 = C.c_int64
c_p = C.c_void_p


class Opts(C.Structure):
    _fields_ = [("slices_A", C.c_int), ("xi", C.c_double), ("beta_ceil", C.c_int),
                ("theory_alpha", C.c_int), ("beta_override", C.c_int), ("k_cap", C.c_int),
                ("max_iter", C.c_int), ("xi_stop", C.c_double), ("cluster_omega", C.c_double),
                ("x_planes", C.c_int), ("sparse_rule", C.c_int)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("beta", C.c_int), ("alpha", C.c_int),
                ("s_X", C.c_int), ("k_V", C.c_int), ("k_W", C.c_int), ("k_U", C.c_int),
                ("products", C.c_longlong), ("err_est", C.c_double), ("step", C.c_double),
                ("min_gap", C.c_double), ("max_lambda", C.c_double), ("omega", C.c_double),
                ("clustered_pairs", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Profile(C.Structure):
    _fields_ = [("kernel_launches", C.c_longlong), ("gemm_launches", C.c_longlong),
                ("gemm_ms", C.c_double), ("gemm_ops", C.c_double), ("gemm_bytes", C.c_double),
                ("simt_launches", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_SIGS = {
    "frx_default_opts": (None, [C.POINTER(Opts)]),
    "frx_status_string": (C.c_char_p, [C.c_int]),
    "frx_refine_workspace_bytes": (C.c_size_t, [c_i64, C.POINTER(Opts)]),
    "frx_refine": (C.c_int, [c_p, c_i64, c_p, c_i64, c_p, c_i64, C.c_double, C.POINTER(Opts),
                             c_p, C.c_size_t, C.POINTER(Info), c_p]),
    "frx_refine_step": (C.c_int, [c_p, c_i64, c_p, c_i64, c_p, c_i64, C.c_double, C.POINTER(Opts),
                                  C.c_double, c_p, C.c_size_t, C.POINTER(Info),
                                  c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_p]),
    "frx_refine_batched_workspace_bytes": (C.c_size_t, [C.POINTER(c_i64), C.c_int, C.POINTER(Opts)]),
    "frx_refine_batched": (C.c_int, [C.POINTER(c_p), C.POINTER(c_i64), C.POINTER(c_p), C.POINTER(c_i64),
                                     C.POINTER(c_p), C.POINTER(c_i64), C.c_int, C.c_double, C.POINTER(Opts),
                                     c_p, C.c_size_t, C.POINTER(Info), c_p]),
    "frx_ozaki_gemm_workspace_bytes": (C.c_size_t, [c_i64, c_i64, c_i64, C.c_int]),
    "frx_ozaki_gemm": (C.c_int, [c_p, c_i64, c_p, c_i64, c_p, c_i64, c_p, c_i64, c_i64, c_i64,
                                 C.c_int, C.c_int, c_p, C.c_size_t, c_p]),
    "frx_exponents_workspace_bytes": (C.c_size_t, [c_i64]),
    "frx_exponents": (C.c_int, [c_p, c_i64, c_i64, c_i64, C.c_int, c_p, c_p, C.c_size_t, c_p]),
    "frx_slice_planes": (C.c_int, [c_p, c_i64, c_i64, c_i64, C.c_int, c_p, C.c_int, c_p, c_i64,
                                   c_i64, c_p]),
    "frx_group_size": (C.c_int, [C.c_int, C.c_int, C.c_int, c_i64]),
    "frx_plane_products": (C.c_int, [c_p, c_i64, c_p, c_i64, c_i64, c_i64, c_i64, c_i64, C.c_int,
                                     C.c_int, C.c_int, c_p, c_p]),
    "frx_ozaki_gemm_static": (C.c_int, [c_p, c_i64, c_p, c_i64, c_p, c_i64, c_p, c_i64, c_i64,
                                        c_i64, C.c_int, C.c_int, c_p]),
    "frx_profile_enable": (None, [C.c_int]),
    "frx_profile_read": (C.c_int, [C.POINTER(Profile), C.c_int]),
    "frx_check_wait_timeout": (C.c_int, [c_p, C.c_size_t, c_p]),
    "frx_set_tile": (C.c_int, [C.c_int]),
    "frx_last_tile": (C.c_int, []),
    "frx_tune_stats": (C.c_int, [C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                 C.POINTER(C.c_longlong), C.c_int]),
}

_lib = None


def load(path: str | None = None) -> C.CDLL:
    """Load libfrx.so (raises if it has not been built: there is no fallback path)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"frx CUDA library missing at {p}; build it with "
                           "`python -m paper_2602_19090_gb300.build_lib`")
    lib = C.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def exported_names():
    return sorted(_SIGS)
