"""ctypes loader for oracle.c (TEST INFRASTRUCTURE; see the package docstring).

``build()`` compiles oracle.c with gcc into ``liboracle.so`` next to it; ``lib()`` loads it,
building on first use.  Flags: -O2 -ffp-contract=off (no fused multiply-add, so every
product is rounded before it is added, exactly as Python's float arithmetic does) and
-fopenmp for Listing 1's parallel loop (oracle_csr3_spmv_omp); where the compiler has no
OpenMP the file builds without it and that function runs on one thread.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_handle = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC]
        if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
            subprocess.run(base, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _handle
    with _lock:
        if _handle is None:
            h = ctypes.CDLL(build())
            h.oracle_csr_spmv.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p,
                                          ctypes.c_double, ctypes.c_double, _f64p]
            h.oracle_csr_spmv.restype = None
            h.oracle_csr_spmv_rows.argtypes = [_i32p, _i32p, _f64p, _f64p, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_void_p, _i64p,
                                               ctypes.c_int64, _f64p]
            h.oracle_csr_spmv_rows.restype = None
            h.oracle_csr3_spmv.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, _i32p, _f64p,
                                           _f64p, _f64p]
            h.oracle_csr3_spmv.restype = None
            h.oracle_csr3_spmv_omp.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, _i32p, _f64p,
                                               _f64p, _f64p, ctypes.c_int]
            h.oracle_csr3_spmv_omp.restype = ctypes.c_int
            h.oracle_csr_spmm.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, ctypes.c_int32,
                                          _f64p, ctypes.c_int64, ctypes.c_double,
                                          ctypes.c_double, _f64p, ctypes.c_int64]
            h.oracle_csr_spmm.restype = None
            h.oracle_rcm.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p]
            h.oracle_rcm.restype = ctypes.c_int
            _handle = h
        return _handle
