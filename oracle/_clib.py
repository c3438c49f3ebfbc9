"""Build and load the oracle's C part (oracle.c) with gcc. Test infrastructure only."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liborc.so (portable flags: builds on x86 and Arm)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            P = ctypes.c_void_p
            L.orc_direct.argtypes = [i64, i32, P, i32, P, P, P, f64, P, i64, P, P, P]
            L.orc_direct.restype = None
            L.orc_spread.argtypes = [i64, i32, P, P, i32, i32, f64, i32, P]
            L.orc_spread.restype = None
            L.orc_gather.argtypes = [i64, i32, P, i32, i32, f64, i32, i32, P, P]
            L.orc_gather.restype = None
            L.orc_direct_grad_x.argtypes = [i64, i32, P, i32, P, P, P, f64, P, P, i64, P, P]
            L.orc_direct_grad_x.restype = None
            L.orc_gather_grad.argtypes = [i64, i32, P, i32, i32, f64, P, P, P]
            L.orc_gather_grad.restype = None
            L.orc_num_threads.argtypes = []
            L.orc_num_threads.restype = i32
            L.orc_set_threads.argtypes = [i32]
            L.orc_set_threads.restype = None
            _lib = L
    return _lib


def ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)
