"""CPU oracle for typed 3/4-node graphlet counts (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  It is a plain C implementation of the
paper's Alg. 1-3 with the closed forms of Sec. "Combinatorial Relationships"
(``tg_oracle.c``, loaded through ctypes) plus a brute-force enumeration of the
graphlet definitions (``brute.py``).  It shares no code with the CUDA library.

Parity status: every function here is pinned (brute force on tiny graphs,
closed-form graph families, invariants and the paper's printed Table 1
numbers; see tests/test_oracle_*.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tg_oracle.c")
_LIB = os.path.join(_HERE, "libtgoracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (OpenMP, no CUDA)."""
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
            L.tgo_build.restype = vp
            L.tgo_build.argtypes = [i64, i64, vp, vp, vp, i32]
            L.tgo_free.argtypes = [vp]
            L.tgo_num_edges.restype = i64
            L.tgo_num_edges.argtypes = [vp]
            L.tgo_edges.argtypes = [vp, vp, vp]
            L.tgo_slots.restype = i64
            L.tgo_slots.argtypes = [i32, i32, i32]
            L.tgo_global_len.restype = i64
            L.tgo_global_len.argtypes = [i32, i32]
            L.tgo_npairs.restype = i64
            L.tgo_npairs.argtypes = [i32]
            L.tgo_rank.restype = i64
            L.tgo_rank.argtypes = [vp, i32]
            L.tgo_pair_index.restype = i64
            L.tgo_pair_index.argtypes = [i32, i32, i32]
            L.tgo_count_per_edge.restype = ctypes.c_int
            L.tgo_count_per_edge.argtypes = [vp, i32, i32, vp, i64, vp, i32]
            L.tgo_count_global.restype = ctypes.c_int
            L.tgo_count_global.argtypes = [vp, i32, vp, i32]
            L.tgo_max_threads.restype = i32
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleGraph:
    """A simplified typed graph held by the C oracle."""

    def __init__(self, n, src, dst, types, L):
        self._lib = lib()
        self.n = int(n)
        self.L = int(L)
        self._src = np.ascontiguousarray(src, dtype=np.int32)
        self._dst = np.ascontiguousarray(dst, dtype=np.int32)
        self._types = np.ascontiguousarray(types, dtype=np.uint8)
        h = self._lib.tgo_build(self.n, self._src.shape[0], _ptr(self._src), _ptr(self._dst),
                                _ptr(self._types), self.L)
        if not h:
            raise ValueError("oracle: invalid graph input")
        self._h = ctypes.c_void_p(h)
        self.M = int(self._lib.tgo_num_edges(self._h))

    @classmethod
    def from_edges(cls, G):
        return cls(G.n, G.src, G.dst, G.types, G.L)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.tgo_free(h)
            self._h = None

    def edges(self):
        u = np.empty(self.M, np.int32)
        v = np.empty(self.M, np.int32)
        self._lib.tgo_edges(self._h, _ptr(u), _ptr(v))
        return u, v

    def per_edge(self, k=4, level="graphlet", edges=None, threads=0) -> np.ndarray:
        lvl = 1 if level == "orbit" else 0
        width = int(self._lib.tgo_slots(self.L, k, lvl))
        if edges is None:
            rows = np.zeros((self.M, width), np.uint64)
            rc = self._lib.tgo_count_per_edge(self._h, k, lvl, None, self.M, _ptr(rows), threads)
        else:
            idx = np.ascontiguousarray(edges, dtype=np.int64)
            rows = np.zeros((idx.shape[0], width), np.uint64)
            rc = self._lib.tgo_count_per_edge(self._h, k, lvl, _ptr(idx), idx.shape[0], _ptr(rows), threads)
        if rc != 0:
            raise RuntimeError(f"oracle per-edge count failed ({rc})")
        return rows

    def global_counts(self, k=4, threads=0) -> np.ndarray:
        out = np.zeros(int(self._lib.tgo_global_len(self.L, k)), np.uint64)
        rc = self._lib.tgo_count_global(self._h, k, _ptr(out), threads)
        if rc != 0:
            raise RuntimeError(f"oracle global count failed ({rc})")
        return out


def slots(L, k, level="graphlet"):
    return int(lib().tgo_slots(L, k, 1 if level == "orbit" else 0))


def global_len(L, k):
    return int(lib().tgo_global_len(L, k))


def rank(c):
    a = np.ascontiguousarray(sorted(c), dtype=np.int32)
    return int(lib().tgo_rank(_ptr(a), a.shape[0]))


def max_threads():
    return int(lib().tgo_max_threads())
