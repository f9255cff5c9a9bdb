"""Second CPU oracle (test infrastructure only): global typed graphlet counts
by non-induced pattern counts and their inversion (``tg_oracle2.c``).

It follows neither the paper's Alg. 1-3 nor the first oracle, and shares no
code with either or with the CUDA library, so agreement between the three is
evidence about each.  Only the tests load it.

Parity status: pinned against brute force on tiny graphs and against the
closed-form graph families (tests/test_oracle2.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tg_oracle2.c")
_LIB = os.path.join(_HERE, "libtgoracle2.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the second oracle with gcc (OpenMP, no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
            L.tgo2_count_global.restype = ctypes.c_int
            L.tgo2_count_global.argtypes = [i64, i64, vp, vp, vp, i32, i32, vp, i32]
            L.tgo2_global_len.restype = ctypes.c_int
            L.tgo2_global_len.argtypes = [i32, i32]
            L.tgo2_max_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def global_counts(n, src, dst, types, L, k=4, threads=0) -> np.ndarray:
    """Induced typed graphlet counts, in the library's global layout."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    types = np.ascontiguousarray(types, dtype=np.uint8)
    if src.shape != dst.shape or types.shape[0] != int(n):
        raise ValueError("oracle 2: inconsistent graph input")
    length = int(lib().tgo2_global_len(int(L), int(k)))
    if length < 0:
        raise ValueError("oracle 2: bad L or k")
    out = np.zeros(max(length, 1), np.uint64)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = lib().tgo2_count_global(int(n), src.shape[0], p(src), p(dst), p(types), int(L), int(k),
                                 p(out), int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle 2 failed ({rc})")
    return out[:length]


def global_counts_of(G, k=4, threads=0) -> np.ndarray:
    return global_counts(G.n, G.src, G.dst, G.types, G.L, k, threads)


def max_threads() -> int:
    return int(lib().tgo2_max_threads())
