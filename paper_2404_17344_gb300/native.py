"""ctypes declarations of the C ABI in include/addker.h: the same names, plain pointers and sizes.

Loading fails loudly when the library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libaddker.so")

# status codes and selectors, as in include/addker.h
ADDKER_OK = 0
ADDKER_EINVAL = -1
ADDKER_EDOMAIN = -2
ADDKER_ENOMEM = -3
ADDKER_ECUDA = -4
ADDKER_ETIMEOUT = -5
ADDKER_ELIMIT = -6
ADDKER_ELL_SHARED = -1
ADDKER_SIGMA_F = -2
ADDKER_WIN_KB = 0
ADDKER_WIN_ES = 1
ADDKER_KERNEL_GAUSS = 0
ADDKER_KERNEL_MATERN12 = 1
ADDKER_REG_DEFAULT = -1
ADDKER_REG_SEPARABLE = 0
ADDKER_REG_RADIAL = 1


def ADDKER_ELL(s: int) -> int:
    return int(s)


class addker_opts(ctypes.Structure):
    _fields_ = [("sigma_os", ctypes.c_double), ("eps_B", ctypes.c_double), ("p", ctypes.c_int),
                ("window", ctypes.c_int), ("kernel", ctypes.c_int),
                ("compensated", ctypes.c_int), ("reg", ctypes.c_int), ("stream", ctypes.c_void_p)]


# name -> (restype, argtypes); every entry point of include/addker.h
_VP, _I, _I64, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
SIGNATURES = {
    "addker_opts_default": (_I, [ctypes.POINTER(addker_opts)]),
    "addker_setup": (_I, [ctypes.POINTER(_VP), _VP, _I64, _I, _VP, _VP, _I, _VP, _D, _VP, _I,
                          ctypes.POINTER(addker_opts)]),
    "addker_set_params": (_I, [_VP, _VP, _D]),
    "addker_set_stream": (_I, [_VP, _VP]),
    "addker_set_graphs": (_I, [_VP, _I]),
    "addker_set_precond": (_I, [_VP, _I]),
    "addker_set_schedule": (_I, [_VP, _I, _I, _I, _I]),
    "addker_autotune": (_I, [_VP, _VP, _I, _VP, _VP, _I]),
    "addker_gsi": (_I, [_VP, _VP, _I, _VP, _VP, _VP]),
    "addker_cg": (_I, [_VP, ctypes.c_double, _VP, _VP, _I, ctypes.c_double, _I, _VP, _VP]),
    "addker_gp_grad": (_I, [_VP, ctypes.c_double, _VP, _VP, _I, ctypes.c_double, _I, _VP, _VP, _VP, _VP]),
    "addker_matvec": (_I, [_VP, _VP, _VP, _I]),
    "addker_dmatvec": (_I, [_VP, _I, _VP, _VP, _I]),
    "addker_matvec_all": (_I, [_VP, _VP, _VP, _VP, _I]),
    "addker_matvec_all_host": (_I, [_VP, _VP, _VP, _VP, _I]),
    "addker_sync": (_I, [_VP]),
    "addker_free": (_I, [_VP]),
    "addker_strerror": (ctypes.c_char_p, [_I]),
    "addker_prescale": (_I, [_VP, _I64, _I, _VP, _VP, _I, _D, _VP, ctypes.POINTER(_D), _VP]),
    "addker_prescale_cube": (_I, [_VP, _I64, _I, _VP, _VP, _I, _D, _VP, ctypes.POINTER(_D), _VP]),
    "addker_info": (_I, [_VP, ctypes.POINTER(_I64), _I]),
    "addker_debug_stage": (_I, [_VP, _I, _I, _VP, _VP, _I64]),
    "addker_profile": (_I, [_VP, _I]),
    "addker_vjp": (_I, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "addker_fastsum_noalloc": (_I, [_VP, _I64, _I, _D, _D, _I, _I, _VP, _VP, _VP, _VP]),
    "addker_profile_read": (_I, [_VP, ctypes.POINTER(_D), ctypes.POINTER(_I64), _I]),
}

_lib = None


def lib():
    """Load libaddker.so (built by paper_2404_17344_gb300.build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing; run "
                               "`python -c 'import __graft_entry__ as g; g.build()'` first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class AddkerError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().addker_strerror(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")
        self.status = status


def check(status: int, where: str) -> None:
    if status != ADDKER_OK:
        raise AddkerError(status, where)
