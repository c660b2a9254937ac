"""ctypes binding of libmsbicg: the C ABI of include/msbicg.h, same names.

Argument marshalling only.  Every computation runs in the CUDA kernels of the
library; there is no Python or CPU fallback.  Loading fails loudly when the
library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmsbicg.so")

MSB_OK, MSB_EINVAL, MSB_ENOMEM, MSB_ECUDA, MSB_EBREAKDOWN, MSB_EMAXITER, MSB_ENONFINITE, MSB_ETIMEOUT = range(8)
STATUS_NAMES = {0: "MSB_OK", 1: "MSB_EINVAL", 2: "MSB_ENOMEM", 3: "MSB_ECUDA", 4: "MSB_EBREAKDOWN",
                5: "MSB_EMAXITER", 6: "MSB_ENONFINITE", 7: "MSB_ETIMEOUT"}
MSB_FP64, MSB_FP32_MIXED = 0, 1


class msb_complex(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class msb_model(C.Structure):
    _fields_ = [("L", C.c_int), ("n_up", C.c_int), ("n_dn", C.c_int), ("periodic", C.c_int),
                ("t", C.c_double), ("U", C.c_double), ("Uc", C.c_double), ("core_site", C.c_int),
                ("o2_spin", C.c_int), ("o1_spin", C.c_int), ("lx", C.c_int), ("tp", C.c_double),
                ("flux", C.c_double)]


class msb_map_params(C.Structure):
    _fields_ = [("Gamma", C.c_double), ("eta", C.c_double), ("gs_tol", C.c_double), ("gs_maxit", C.c_int),
                ("solve_tol", C.c_double), ("maxit", C.c_int), ("cf_tol", C.c_double), ("cf_check", C.c_int),
                ("cf_maxdepth", C.c_int), ("seed_index", C.c_int), ("block", C.c_int), ("precision", C.c_int)]


class msb_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("n_converged", C.c_int), ("matvecs", C.c_int64),
                ("flushes", C.c_int64), ("seed_residual", C.c_double), ("max_shift_residual", C.c_double),
                ("E_G", C.c_double), ("gs_residual", C.c_double), ("cf_depth_max", C.c_int),
                ("cf_depth_min", C.c_int), ("seconds_ground_state", C.c_double), ("seconds_solve", C.c_double),
                ("seconds_second_step", C.c_double), ("seconds_total", C.c_double),
                ("device_bytes", C.c_int64), ("kernel_launches", C.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class msb_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_int64), ("ms", C.c_double), ("alg_bytes", C.c_double),
                ("alg_flops", C.c_double)]


_P = C.c_void_p
_I = C.c_int
_D = C.c_double
_I64 = C.c_int64
_PD = C.POINTER(C.c_double)
_PI = C.POINTER(C.c_int)

# name -> (restype, argtypes); the complete C ABI of include/msbicg.h
SIGNATURES = {
    "msb_last_error": (C.c_char_p, []),
    "msb_version": (C.c_char_p, []),
    "msb_map_params_default": (None, [C.POINTER(msb_map_params)]),
    "msb_basis_create": (_I, [_I, _I, _I, C.POINTER(_P)]),
    "msb_basis_dims": (_I, [_P, C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I64)]),
    "msb_basis_states": (_I, [_P, _I, C.POINTER(C.c_uint32)]),
    "msb_basis_destroy": (None, [_P]),
    "msb_op_create_hubbard": (_I, [C.POINTER(msb_model), _I, C.POINTER(_P)]),
    "msb_basis_row_layout": (_I, [_P, _I, C.POINTER(C.c_uint16), _PI, C.POINTER(C.c_uint16), _PD, _PD]),
    "msb_basis_row_order": (_I, [_P, _I, C.POINTER(C.c_uint16)]),
    "msb_op_create_csr": (_I, [_I64, C.POINTER(C.c_int64), C.POINTER(C.c_int32), _PD, C.POINTER(_P)]),
    "msb_op_create_direct_sum": (_I, [C.POINTER(_P), _PD, _I, C.POINTER(_P)]),
    "msb_op_dim": (_I, [_P, C.POINTER(_I64)]),
    "msb_op_destroy": (None, [_P]),
    "msb_op_apply": (_I, [_P, msb_complex, _P, _P, _I, _I, _P]),
    "msb_apply_cdag_up": (_I, [C.POINTER(msb_model), _I, _P, _P, _I, _I, _P]),
    "msb_apply_c_up": (_I, [C.POINTER(msb_model), _I, _P, _P, _I, _I, _P]),
    "msb_ground_state": (_I, [_P, _D, _I, _P, _PD, _P, _PD, _P]),
    "msb_ground_state_noalloc": (_I, [_P, _D, _I, _P, _PD, _P, _PD, _P]),
    "msb_multishift_bicg_solve": (_I, [_P, msb_complex, _P, C.POINTER(msb_complex), _I, _D, _I, _I, _I, _P,
                                       _PI, _PD, _PI, C.POINTER(msb_solve_info), _P]),
    "msb_multishift_bicg_dual_solve": (_I, [_P, msb_complex, _P, C.POINTER(msb_complex), _I, _D, _I, _I, _I, _P,
                                            _PI, _PD, _PI, C.POINTER(msb_solve_info), _P]),
    "msb_bicgstab_solve": (_I, [_P, msb_complex, _P, C.POINTER(msb_complex), _I, _D, _I, _I, _P, _PI, _PD, _PI,
                                _PI, C.POINTER(msb_solve_info), _P]),
    "msb_autotune": (_I, [C.POINTER(msb_model), _I, _I, _PI, _PI, _PD, _PD, _P]),
    "msb_autotune_forget": (None, []),
    "msb_multishift_bicg_reseeded": (_I, [_P, msb_complex, _P, C.POINTER(msb_complex), _I, _D, _I, _I, _I, _D, _I,
                                          _I, _P, _PI, _PI, _PD, _PI, _PI, C.POINTER(msb_solve_info), _P]),
    "msb_continued_fraction": (_I, [_P, _P, _I, _D, _PD, _I, _D, _D, _I, _I, _I, _PD, _PI, _P]),
    "msb_rixs_map": (_I, [C.POINTER(msb_model), C.POINTER(msb_map_params), _P, _D, _PD, _I, _PD, _I, _PD,
                          C.POINTER(msb_solve_info), _P]),
    "msb_rixs_map_ops": (_I, [_P, _P, C.POINTER(msb_map_params), _P, _D, _PD, _I, _PD, _I, _P,
                              C.POINTER(msb_solve_info), _P]),
    "msb_rixs_map_sites": (_I, [C.POINTER(msb_model), C.POINTER(msb_map_params), C.POINTER(C.c_int), _I, _PD, _I,
                                _PD, _I, _PD, C.POINTER(msb_solve_info), _P]),
    "msb_rixs_map_clusters": (_I, [C.POINTER(msb_model), _I, C.POINTER(msb_map_params), _PD, _I, _PD, _I, _PD,
                                   _PD, C.POINTER(msb_solve_info), _P]),
    "msb_rixs_map_q": (_I, [C.POINTER(msb_model), C.POINTER(msb_map_params), _PD, _I, _PD, _I, _PD, _I, _PD,
                            C.POINTER(msb_solve_info), _P]),
    "msb_profile_enable": (None, [_I]),
    "msb_profile_reset": (None, []),
    "msb_profile_read": (_I, [C.POINTER(msb_kernel_stat), _I]),
}


def profile_read() -> list:
    """Per kernel class: dict(name, launches, ms, alg_bytes, alg_flops)."""
    lib = load()
    n = lib.msb_profile_read(None, 0)
    arr = (msb_kernel_stat * max(n, 1))()
    n = lib.msb_profile_read(arr, n)
    return [dict(name=a.name.decode(), launches=a.launches, ms=a.ms, alg_bytes=a.alg_bytes, alg_flops=a.alg_flops)
            for a in arr[:n]]


class MsbError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libmsbicg.so (built by paper_2506_09551_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int, allow=()) -> int:
    if status != MSB_OK and status not in allow:
        raise MsbError(status, load().msb_last_error().decode())
    return status


def last_error() -> str:
    return load().msb_last_error().decode()


def __getattr__(name):
    """Module-level access to the raw C functions: native.msb_op_apply(...)."""
    if name in SIGNATURES:
        return getattr(load(), name)
    raise AttributeError(name)
