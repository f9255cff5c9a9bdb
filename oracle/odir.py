"""Directed typed 3-node graphlet oracle (test infrastructure only): the
paper's Alg. 1 over the out/in split of every typed neighbourhood
(Sec. "Directed Typed Graphlets"), in ``tg_oracle_dir.c``.

Shares no code with the CUDA library.  Parity status: pinned against the
dyad-census brute force of ``brute_dir.py``, closed forms and the undirected
3-node counts (tests/test_oracle_directed.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tg_oracle_dir.c")
_LIB = os.path.join(_HERE, "libtgoracledir.so")
_lock = threading.Lock()
_lib = None

NCLS = 13


_SRC4 = os.path.join(_HERE, "tg_oracle_dir4.c")
_LIB4 = os.path.join(_HERE, "libtgoracledir4.so")
_lib4 = None


def _compile(src, lib, force):
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, src])
        os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """Compile the directed oracles (3- and 4-node) with gcc (no CUDA)."""
    _compile(_SRC4, _LIB4, force)
    return _compile(_SRC, _LIB, force)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
            L.tgod_count.restype = ctypes.c_int
            L.tgod_count.argtypes = [i64, i64, vp, vp, vp, i32, vp, vp]
            L.tgod_edges.restype = i64
            L.tgod_edges.argtypes = [i64, i64, vp, vp]
            L.tgod_global_len.restype = i64
            L.tgod_global_len.argtypes = [i32]
            _lib = L
    return _lib


def _inputs(G):
    return (np.ascontiguousarray(G.src, dtype=np.int32), np.ascontiguousarray(G.dst, dtype=np.int32),
            np.ascontiguousarray(G.types, dtype=np.uint8))


def counts_of(G, rows: bool = True):
    """(per-edge rows M x 13 L or None, global counts 13 C(L+2, 3)) of the
    digraph with arcs src -> dst."""
    src, dst, types = _inputs(G)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    M = int(lib().tgod_edges(int(G.n), src.shape[0], p(src), p(dst)))
    out_rows = np.zeros((M, NCLS * G.L), np.uint64) if rows else None
    glob = np.zeros(int(lib().tgod_global_len(int(G.L))), np.uint64)
    rc = lib().tgod_count(int(G.n), src.shape[0], p(src), p(dst), p(types), int(G.L),
                          p(out_rows) if rows else None, p(glob))
    if rc != 0:
        raise RuntimeError(f"directed oracle failed ({rc})")
    return out_rows, glob


def lib4():
    global _lib4
    with _lock:
        if _lib4 is None:
            build()
            L = ctypes.CDLL(_LIB4)
            vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
            L.tgod4_count.restype = ctypes.c_int
            L.tgod4_count.argtypes = [i64, i64, vp, vp, vp, i32, vp, vp]
            L.tgod4_global_len.restype = i64
            L.tgod4_global_len.argtypes = [i32]
            L.tgod4_classes.restype = ctypes.c_int
            L.tgod4_classes.argtypes = [vp, vp]
            _lib4 = L
    return _lib4


NCLS4 = 199


def classes4():
    """(canonical codes, underlying edge counts) of the 199 connected 4-node
    digraph classes, in class order."""
    codes = np.zeros(NCLS4, np.int32)
    edges = np.zeros(NCLS4, np.int32)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    if lib4().tgod4_classes(p(codes), p(edges)) != NCLS4:
        raise RuntimeError("directed 4-node oracle: class table")
    return codes, edges


def counts4_of(G, rows: bool = True):
    """(per-edge rows M x 199 P or None, global counts 199 C(L+3, 4)) of the
    directed typed 4-node graphlets of the digraph with arcs src -> dst."""
    src, dst, types = _inputs(G)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    M = int(lib().tgod_edges(int(G.n), src.shape[0], p(src), p(dst)))
    P = G.L * (G.L + 1) // 2
    out_rows = np.zeros((M, NCLS4 * P), np.uint64) if rows else None
    glob = np.zeros(int(lib4().tgod4_global_len(int(G.L))), np.uint64)
    rc = lib4().tgod4_count(int(G.n), src.shape[0], p(src), p(dst), p(types), int(G.L),
                            p(out_rows) if rows else None, p(glob))
    if rc != 0:
        raise RuntimeError(f"directed 4-node oracle failed ({rc})")
    return out_rows, glob
