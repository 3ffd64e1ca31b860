"""Build and load the oracle's plain-C integrators (gcc, FP64, no FMA contraction).

Test infrastructure: only tests, the smoke check and the benchmark's CPU
baseline load this library.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = ["l96.c"]
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile oracle/*.c into oracle/_liboracle.so if missing or stale."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    if not force and os.path.exists(_LIB):
        t_lib = os.path.getmtime(_LIB)
        if all(os.path.getmtime(s) <= t_lib for s in srcs):
            return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-fPIC",
           "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            i, d = ctypes.c_int, ctypes.c_double
            L.l96_rhs.argtypes = [i, d, dp, dp]
            L.l96_nl.argtypes = [i, i, d, d, dp, dp]
            L.l96_tl.argtypes = [i, i, d, d, dp, dp, dp]
            L.l96_ad.argtypes = [i, i, d, d, dp, dp, dp]
            for f in (L.l96_rhs, L.l96_nl, L.l96_tl, L.l96_ad):
                f.restype = None
            _lib = L
    return _lib


def ptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
