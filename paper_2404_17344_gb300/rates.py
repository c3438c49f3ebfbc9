"""ctypes binding of include/addker_rates.h: the device-rate microbenchmark (measurement tooling, built into
_lib/libaddker_rates.so apart from the product library). Loading fails loudly when it has not been built."""
from __future__ import annotations

import ctypes
import os

from . import native

LIB_PATH = os.path.join(native.HERE, "_lib", "libaddker_rates.so")
_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"rate library not built: {LIB_PATH} is missing; run "
                               "`python -c 'import __graft_entry__ as g; g.build()'` first")
        L = ctypes.CDLL(LIB_PATH)
        L.addker_device_rates.restype = ctypes.c_int
        L.addker_device_rates.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int]
        _lib = L
    return _lib


def device_rates():
    """Device rates for roofline accounting (addker_device_rates): a dict with the SM count, the SM
    clock under FP32 load (MHz), FFMA and packed FFMA2 TFLOP/s, shared and global float atomic adds
    (10^9/s, distinct words; the global ones into an L2-resident 1 MiB grid) and global double atomic adds."""
    out = (ctypes.c_double * 8)()
    n = lib().addker_device_rates(out, 8)
    native.check(min(n, 0), "addker_device_rates")
    keys = ("sms", "sm_mhz_under_load", "ffma_tflops", "ffma2_tflops", "shared_atomic_gops",
            "global_atomic_gops", "ffma_launch_ms", "global_atomic64_gops")
    return {k: float(out[i]) for i, k in enumerate(keys)}
