"""ctypes declarations for libiga_helmholtz.so (include/iga_helmholtz.h).

Loading fails loudly if the library has not been built: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

IGA_MAX_LINES = 8

STATUS = {
    0: "IGA_OK", 1: "IGA_NOT_CONVERGED", -1: "IGA_E_INVALID", -2: "IGA_E_CUDA", -3: "IGA_E_OOM",
    -4: "IGA_E_BREAKDOWN", -5: "IGA_E_NONFINITE", -6: "IGA_E_TIMEOUT", -7: "IGA_E_UNSUPPORTED",
}


class IgaParams(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("p", C.c_int),
        ("n_el", C.c_int),
        ("n_lines", C.c_int),
        ("lines", (C.c_double * 3) * IGA_MAX_LINES),
        ("k_values", C.c_double * (IGA_MAX_LINES + 1)),
        ("beta1", C.c_double),
        ("beta2", C.c_double),
        ("eps", C.c_double),
        ("nu_pre", C.c_int),
        ("nu_post", C.c_int),
        ("omega", C.c_double),
        ("n_vcycles", C.c_int),
        ("precision", C.c_int),
        ("flexible", C.c_int),
        ("skip_deflation", C.c_int),
        ("arnoldi", C.c_int),
        ("fused_vcycle", C.c_int),
        ("host_loop", C.c_int),
        ("stream", C.c_void_p),
        ("precond", C.c_int),
        ("deflation", C.c_int),
        ("robin", C.c_int),
    ]


_VP = C.c_void_p
_SIG = {
    "iga_default_params": (None, [C.POINTER(IgaParams)]),
    "iga_setup": (C.c_int, [C.POINTER(IgaParams), C.POINTER(C.c_void_p)]),
    "iga_destroy": (None, [_VP]),
    "iga_ndof": (C.c_size_t, [_VP]),
    "iga_coarse_ndof": (C.c_size_t, [_VP]),
    "iga_num_levels": (C.c_int, [_VP]),
    "iga_level_nx": (C.c_int, [_VP, C.c_int]),
    "iga_level_nel": (C.c_int, [_VP, C.c_int]),
    "iga_status_str": (C.c_char_p, [C.c_int]),
    "iga_launch_count": (C.c_ulonglong, []),
    "iga_tile_choice": (C.c_int, [_VP, C.c_int, C.c_int]),
    "iga_set_tile": (C.c_int, [_VP, C.c_int, C.c_int, C.c_int]),
    "iga_solve_batched": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                     C.POINTER(C.c_int), C.c_double, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                     _VP]),
    "iga_net_num_params": (C.c_int, []),
    "iga_net_create": (C.c_int, [C.c_ulonglong, C.POINTER(C.c_void_p)]),
    "iga_net_destroy": (None, [_VP]),
    "iga_net_last_error": (C.c_char_p, [_VP]),
    "iga_net_get_params": (C.c_int, [_VP, _VP, C.c_int]),
    "iga_net_set_params": (C.c_int, [_VP, _VP, C.c_int]),
    "iga_net_forward": (C.c_int, [_VP, _VP, _VP, C.c_int, C.c_int, C.c_int, _VP]),
    "iga_net_grad": (C.c_int, [_VP, _VP, _VP, C.c_int, C.c_int, C.c_int, _VP, _VP, _VP]),
    "iga_net_train_step": (C.c_int, [_VP, _VP, _VP, C.c_int, C.c_int, C.c_int, C.c_float, _VP, _VP]),
    "iga_attach_net": (C.c_int, [_VP, _VP, C.c_double]),
    "iga_precond_pair": (C.c_int, [_VP, _VP, _VP, _VP, C.c_int]),
    "iga_net_pack": (C.c_int, [_VP, _VP, _VP, C.c_int, C.c_int, C.c_int, C.c_int, _VP, _VP, C.c_double]),
    "iga_mgs_noalloc": (C.c_int, [_VP, C.c_size_t, C.c_size_t, C.c_int, _VP, _VP, _VP]),
    "iga_last_error": (C.c_char_p, [_VP]),
    "iga_get_knots": (C.c_int, [_VP, C.c_int, _VP, C.c_int]),
    "iga_get_band": (C.c_int, [_VP, C.c_int, C.c_int, _VP, C.c_size_t]),
    "iga_get_prolongation": (C.c_int, [_VP, C.c_int, _VP, C.c_size_t]),
    "iga_apply_A": (C.c_int, [_VP, _VP, _VP]),
    "iga_apply_Mshift": (C.c_int, [_VP, C.c_int, _VP, _VP]),
    "iga_jacobi": (C.c_int, [_VP, C.c_int, _VP, _VP, _VP, C.c_int]),
    "iga_apply_Mshift32": (C.c_int, [_VP, C.c_int, _VP, _VP]),
    "iga_jacobi32": (C.c_int, [_VP, C.c_int, _VP, _VP, _VP]),
    "iga_restrict": (C.c_int, [_VP, C.c_int, _VP, _VP]),
    "iga_prolong_add": (C.c_int, [_VP, C.c_int, _VP, _VP]),
    "iga_coarse_solve": (C.c_int, [_VP, _VP, _VP]),
    "iga_vcycle_cslp": (C.c_int, [_VP, _VP, _VP]),
    "iga_precond": (C.c_int, [_VP, _VP, _VP]),
    "iga_set_wait_limit": (C.c_int, [_VP, C.c_longlong, C.c_int]),
    "iga_zt": (C.c_int, [_VP, _VP, _VP]),
    "iga_z": (C.c_int, [_VP, _VP, _VP]),
    "iga_esolve": (C.c_int, [_VP, _VP, _VP]),
    "iga_deflate": (C.c_int, [_VP, _VP, _VP]),
    "iga_load_point_source": (C.c_int, [_VP, C.c_double, C.c_double, _VP]),
    "iga_load_dirichlet": (C.c_int, [_VP, C.c_double, C.c_double, _VP]),
    "iga_mgs": (C.c_int, [_VP, _VP, C.c_size_t, C.c_int, _VP, _VP]),
    "iga_solve": (C.c_int, [_VP, _VP, _VP, C.c_double, C.c_int, C.POINTER(C.c_int), _VP, C.POINTER(C.c_double)]),
    "iga_solve_host": (C.c_int, [_VP, _VP, _VP, C.c_double, C.c_int, C.POINTER(C.c_int), _VP,
                                 C.POINTER(C.c_double)]),
}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libiga_helmholtz.so")
_lib = None


def lib():
    """Load the shared library (once) and declare every entry point."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2010_10232_gb300.build.build() "
                               "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIG.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_names():
    return list(_SIG.keys())
