"""Python binding of the typed-graphlet C ABI (include/tg.h).

Argument marshalling only: every step of the counting path runs in the CUDA
library ``libtg.so`` built in-tree by ``build.build()``.  Importing this
module never computes anything on the host; if the library is missing the
first call raises instead of falling back to anything else.

Arrays: numpy arrays are host memory; torch CUDA tensors (or anything with a
``data_ptr()`` on the device) are device memory.  ``stream`` is a
``torch.cuda.Stream`` or a raw ``cudaStream_t`` integer (None: torch's current
stream when torch is loaded, else the legacy default stream).
"""
from __future__ import annotations

import ctypes
import os
import sys

import numpy as np

from . import build as _build

__all__ = [
    "TGError", "Graph", "lib", "tg_build_csr", "tg_free_graph", "tg_graph_info", "tg_edge_list",
    "tg_count_global", "tg_count_global_noalloc", "tg_count_directed_global",
    "tg_count_directed_per_edge", "tg_dir_slots", "tg_dir_global_len", "TRIAD_NAMES",
    "tg_count_directed4_global", "tg_count_directed4_per_edge", "tg_dir4_slots", "tg_dir4_global_len", "tg_count_per_edge", "tg_count_shard", "tg_count_per_edge_sparse", "tg_sparse_ids", "tg_sparse_id", "Batch", "tg_count_batch", "Server", "tg_count_range", "tg_global_finalize",
    "tg_work_model", "tg_slots", "tg_global_len", "tg_config_count", "tg_config_rank",
    "tg_config_unrank", "tg_paper_hash", "tg_slot_config", "tg_strerror", "tg_version",
    "tg_debug_fail_alloc", "tg_set_tune", "tg_get_tune", "tg_autotune", "tg_autotune_reset", "tg_launch_count", "tg_last_timing",
    "tg_last_cuda_error", "tg_set_memory_retention", "tg_trim_memory", "TG_GRAPHLET", "TG_ORBIT",
]

TG_OK = 0
TG_EINVAL = -1
TG_ENOMEM = -2
TG_ECUDA = -3
TG_EOVERFLOW = -4
TG_EINTERNAL = -5
TG_EBUSY = -6
TG_ENOMEM_ADMIT = -7
TG_ETIMEDOUT = -8
TG_ENOTFOUND = -9
TG_INPUT_DEVICE = 1
TG_DIRECTED = 2
TG_TRIAD_CLASSES = 13
TRIAD_NAMES = ("021D", "021U", "021C", "111D", "111U", "030T", "030C", "201", "120D", "120U",
               "120C", "210", "300")
TG_GRAPHLET = 0
TG_ORBIT = 1

_lib = None


class TGError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {tg_strerror(status)} ({status})" if what else tg_strerror(status))


class TGTune(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("cta_threads", ctypes.c_int32), ("unroll", ctypes.c_int32),
                ("hash_slots", ctypes.c_int32), ("bitmap_bits", ctypes.c_int64),
                ("grid_limit", ctypes.c_int32), ("edge_pass", ctypes.c_int32),
                ("edge_batch", ctypes.c_int32), ("c4_bin_fill", ctypes.c_int32)]


class TGTiming(ctypes.Structure):
    _fields_ = [("tau_ms", ctypes.c_double), ("aggregate_ms", ctypes.c_double),
                ("count_ms", ctypes.c_double), ("edges", ctypes.c_uint64),
                ("gamma_entries", ctypes.c_uint64), ("walked_entries", ctypes.c_uint64),
                ("probe_pairs", ctypes.c_uint64), ("t_members", ctypes.c_uint64),
                ("cycles_ms", ctypes.c_double), ("cliques_ms", ctypes.c_double),
                ("wedges", ctypes.c_uint64), ("clique_tests", ctypes.c_uint64),
                ("cliques", ctypes.c_uint64)]


TG_BATCH_GLOBAL = 0
TG_BATCH_PER_EDGE_GRAPHLET = 1
TG_BATCH_PER_EDGE_ORBIT = 2

TG_KERNEL_AUTO = 0
TG_KERNEL_WARP_SEARCH = 1
TG_KERNEL_CTA_BITMAP = 2
TG_KERNEL_REUSE = 3
TG_KERNEL_CYCLES = 4
TG_EDGE_PASS_AUTO = 0
TG_EDGE_PASS_FUSED = 1


class TGServeCfg(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("queue_cap", ctypes.c_int32),
                ("mem_budget_bytes", ctypes.c_int64), ("device", ctypes.c_int32),
                ("batch_max", ctypes.c_int32), ("batch_edges", ctypes.c_int64)]


class TGRequest(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("src", ctypes.c_void_p),
                ("dst", ctypes.c_void_p), ("type", ctypes.c_void_p), ("L", ctypes.c_int32),
                ("k", ctypes.c_int32)]


class TGResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("cuda_error", ctypes.c_int32), ("len", ctypes.c_int64),
                ("latency_ms", ctypes.c_double)]


class TGServeStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64), ("queued", ctypes.c_uint64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("graphs_per_s", ctypes.c_double), ("peak_in_flight", ctypes.c_int64),
                ("peak_bytes", ctypes.c_int64), ("batched_launches", ctypes.c_uint64),
                ("grouped_requests", ctypes.c_uint64)]


class _Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m_input", ctypes.c_int64), ("M", ctypes.c_int64),
                ("n_nonisolated", ctypes.c_int64), ("max_degree", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("L", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def lib():
    """The loaded libtg.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise ImportError(f"libtg.so not built ({_build.LIB}); run __graft_entry__.build()")
        L = ctypes.CDLL(_build.LIB)
        vp, i64, i32, u32, u64 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32,
                                  ctypes.c_uint64)
        sig = {
            "tg_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "tg_version": (ctypes.c_int, []),
            "tg_build_csr": (ctypes.c_int, [i64, i64, vp, vp, vp, i32, u32, vp, ctypes.POINTER(vp)]),
            "tg_free_graph": (ctypes.c_int, [vp]),
            "tg_graph_info": (ctypes.c_int, [vp, ctypes.POINTER(_Info)]),
            "tg_edge_list": (ctypes.c_int, [vp, vp, vp, vp]),
            "tg_slots": (i64, [i32, i32, i32]),
            "tg_global_len": (i64, [i32, i32]),
            "tg_config_count": (i64, [i32, i32]),
            "tg_config_rank": (i64, [vp, i32]),
            "tg_config_unrank": (ctypes.c_int, [i64, i32, vp]),
            "tg_paper_hash": (u64, [i32, vp, i32, i32]),
            "tg_slot_config": (ctypes.c_int, [i32, i32, i32, i32, i32, i64, vp, vp, vp]),
            "tg_count_global": (ctypes.c_int, [vp, i32, vp, vp]),
            "tg_dir_slots": (i64, [i32]),
            "tg_dir_global_len": (i64, [i32]),
            "tg_count_directed_global": (ctypes.c_int, [vp, vp, vp]),
            "tg_count_directed_per_edge": (ctypes.c_int, [vp, vp, vp]),
            "tg_dir4_slots": (i64, [i32]),
            "tg_dir4_global_len": (i64, [i32]),
            "tg_count_directed4_global": (ctypes.c_int, [vp, vp, vp]),
            "tg_count_directed4_per_edge": (ctypes.c_int, [vp, vp, vp]),
            "tg_count_per_edge": (ctypes.c_int, [vp, i32, i32, vp, vp]),
            "tg_count_range": (ctypes.c_int, [vp, i32, i64, i64, vp, vp]),
            "tg_count_shard": (ctypes.c_int, [vp, i32, i32, i32, vp, vp]),
            "tg_count_per_edge_sparse": (ctypes.c_int, [vp, i32, i32, vp, vp, vp, i64, vp, vp]),
            "tg_sparse_ids": (i64, [i32, i32, i32]),
            "tg_sparse_id": (ctypes.c_int, [i32, i32, i32, i64, vp, vp, vp]),
            "tg_global_finalize": (ctypes.c_int, [i32, i32, vp, vp]),
            "tg_work_model": (ctypes.c_int, [vp, vp, vp]),
            "tg_set_allocator": (ctypes.c_int, [vp, vp, vp]),
            "tg_set_memory_retention": (ctypes.c_int, [u64]),
            "tg_trim_memory": (ctypes.c_int, []),
            "tg_debug_fail_alloc": (ctypes.c_int, [i64]),
            "tg_set_tune": (ctypes.c_int, [vp]),
            "tg_launch_count": (u64, []),
            "tg_last_cuda_error": (i32, []),
            "tg_count_global_noalloc": (ctypes.c_int, [vp, i32, vp, vp]),
            "tg_batch_create": (ctypes.c_int, [i32, vp, i32, i32, vp, vp, vp, ctypes.POINTER(vp)]),
            "tg_batch_run": (ctypes.c_int, [vp, vp]),
            "tg_batch_tune": (ctypes.c_int, [vp, vp, ctypes.POINTER(i32)]),
            "tg_batch_destroy": (ctypes.c_int, [vp]),
            "tg_count_batch": (ctypes.c_int, [i32, vp, i32, i32, vp, vp, vp]),
            "tg_serve_create": (vp, [vp]),
            "tg_serve_submit": (ctypes.c_int, [vp, vp, ctypes.POINTER(u64)]),
            "tg_serve_wait": (ctypes.c_int, [vp, u64, i32, vp, i64, vp]),
            "tg_serve_stats": (ctypes.c_int, [vp, vp]),
            "tg_serve_destroy": (None, [vp]),
            "tg_last_timing": (ctypes.c_int, [vp]),
            "tg_get_tune": (ctypes.c_int, [vp]),
            "tg_autotune": (ctypes.c_int, [vp, i32, vp, vp]),
            "tg_autotune_reset": (ctypes.c_int, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


# ------------------------------------------------------------- marshalling --
def _is_device(x) -> bool:
    dev = getattr(x, "is_cuda", None)
    return bool(dev)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(x.ctypes.data)
    if hasattr(x, "data_ptr"):
        if hasattr(x, "is_contiguous") and not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    raise TypeError(f"unsupported buffer type {type(x)!r}")


def _stream(stream):
    if stream is None:
        torch = sys.modules.get("torch")
        if torch is not None and torch.cuda.is_available() and torch.cuda.is_initialized():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _check(rc: int, what: str):
    if rc != TG_OK:
        if rc == TG_ECUDA:  # name the CUDA error (recorded per host thread)
            what = f"{what} (cudaError_t {int(lib().tg_last_cuda_error())})"
        raise TGError(rc, what)


def tg_strerror(status: int) -> str:
    return lib().tg_strerror(status).decode()


def tg_version() -> int:
    return lib().tg_version()


# --------------------------------------------------------------- graphs -----
class Graph:
    """Owner of a ``tg_graph*``; freed with the object (or ``close()``)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle
        info = _Info()
        _check(lib().tg_graph_info(self._h, ctypes.byref(info)), "tg_graph_info")
        self.n, self.m_input, self.M = info.n, info.m_input, info.M
        self.n_nonisolated, self.max_degree = info.n_nonisolated, info.max_degree
        self.device_bytes, self.L = info.device_bytes, info.L

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("graph is closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().tg_free_graph(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        return dict(n=self.n, m_input=self.m_input, M=self.M, n_nonisolated=self.n_nonisolated,
                    max_degree=self.max_degree, device_bytes=self.device_bytes, L=self.L)


def tg_build_csr(n: int, src, dst, types, L: int, stream=None, directed: bool = False) -> Graph:
    """Build the resident typed CSR (host numpy or device tensors); ``directed``
    keeps the arcs src -> dst for the directed counts (TG_DIRECTED)."""
    dev = _is_device(src)
    if dev != _is_device(dst) or dev != _is_device(types):
        raise ValueError("src, dst and types must all be host arrays or all device tensors")
    if not dev:
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
        types = np.ascontiguousarray(types, dtype=np.uint8)
    m = int(src.shape[0])
    if int(dst.shape[0]) != m or int(types.shape[0]) != int(n):
        raise ValueError("length mismatch")
    h = ctypes.c_void_p()
    rc = lib().tg_build_csr(int(n), m, _ptr(src), _ptr(dst), _ptr(types), int(L),
                            (TG_INPUT_DEVICE if dev else 0) | (TG_DIRECTED if directed else 0),
                            _stream(stream), ctypes.byref(h))
    _check(rc, "tg_build_csr")
    return Graph(h)


def tg_free_graph(g: Graph) -> None:
    g.close()


def tg_graph_info(g: Graph) -> dict:
    return g.info()


def tg_edge_list(g: Graph, stream=None):
    u = np.empty(g.M, np.int32)
    v = np.empty(g.M, np.int32)
    _check(lib().tg_edge_list(g.handle, _ptr(u), _ptr(v), _stream(stream)), "tg_edge_list")
    return u, v


# --------------------------------------------------------------- layout -----
def tg_slots(L: int, k: int = 4, level: int = TG_GRAPHLET) -> int:
    return int(lib().tg_slots(L, k, level))


def tg_global_len(L: int, k: int = 4) -> int:
    return int(lib().tg_global_len(L, k))


def tg_config_count(L: int, k: int) -> int:
    return int(lib().tg_config_count(L, k))


def tg_config_rank(types) -> int:
    a = np.ascontiguousarray(types, dtype=np.int32)
    return int(lib().tg_config_rank(_ptr(a), a.shape[0]))


def tg_config_unrank(rank: int, k: int):
    a = np.zeros(k, np.int32)
    _check(lib().tg_config_unrank(int(rank), k, _ptr(a)), "tg_config_unrank")
    return tuple(int(x) for x in a)


def tg_paper_hash(g: int, types, L: int) -> int:
    a = np.ascontiguousarray(types, dtype=np.int32)
    return int(lib().tg_paper_hash(g, _ptr(a), a.shape[0], L))


def tg_slot_config(L: int, k: int, level: int, phi_i: int, phi_j: int, slot: int):
    motif = ctypes.c_int32()
    kk = ctypes.c_int32()
    t = np.zeros(4, np.int32)
    _check(lib().tg_slot_config(L, k, level, phi_i, phi_j, slot, ctypes.byref(motif), _ptr(t),
                                ctypes.byref(kk)), "tg_slot_config")
    return int(motif.value), tuple(int(x) for x in t[: kk.value])


# -------------------------------------------------------------- counting ----
def tg_count_global(g: Graph, k: int = 4, out=None, stream=None):
    """Global typed counts; ``out`` (host array or device tensor) or a new numpy array."""
    if out is None:
        out = np.zeros(tg_global_len(g.L, k), np.uint64)
    _check(lib().tg_count_global(g.handle, k, _ptr(out), _stream(stream)), "tg_count_global")
    return out


def tg_dir_slots(L: int) -> int:
    return int(lib().tg_dir_slots(L))


def tg_dir_global_len(L: int) -> int:
    return int(lib().tg_dir_global_len(L))


def tg_count_directed_global(g: Graph, out=None, stream=None):
    """Directed typed 3-node graphlet counts of a graph built with ``directed=True``:
    13 triad classes x C(L+2, 3) type multisets (``out`` host array or device tensor)."""
    if out is None:
        out = np.zeros(tg_dir_global_len(g.L), np.uint64)
    _check(lib().tg_count_directed_global(g.handle, _ptr(out), _stream(stream)),
           "tg_count_directed_global")
    return out


def tg_count_directed_per_edge(g: Graph, rows=None, stream=None):
    """Per-edge directed typed 3-node rows (M x 13 L, slot c L + t)."""
    if rows is None:
        rows = np.zeros((g.M, tg_dir_slots(g.L)), np.uint64)
    _check(lib().tg_count_directed_per_edge(g.handle, _ptr(rows), _stream(stream)),
           "tg_count_directed_per_edge")
    return rows


def tg_dir4_slots(L: int) -> int:
    return int(lib().tg_dir4_slots(L))


def tg_dir4_global_len(L: int) -> int:
    return int(lib().tg_dir4_global_len(L))


def tg_count_directed4_global(g: Graph, out=None, stream=None):
    """Directed typed 4-node graphlet counts of a graph built with ``directed=True``:
    199 classes x C(L+3, 4) type multisets."""
    if out is None:
        out = np.zeros(tg_dir4_global_len(g.L), np.uint64)
    _check(lib().tg_count_directed4_global(g.handle, _ptr(out), _stream(stream)),
           "tg_count_directed4_global")
    return out


def tg_count_directed4_per_edge(g: Graph, rows=None, stream=None):
    """Per-edge directed typed 4-node rows (M x 199 P)."""
    if rows is None:
        rows = np.zeros((g.M, tg_dir4_slots(g.L)), np.uint64)
    _check(lib().tg_count_directed4_per_edge(g.handle, _ptr(rows), _stream(stream)),
           "tg_count_directed4_per_edge")
    return rows


def tg_count_global_noalloc(g: Graph, k: int, out, stream=None):
    """Global counts into the caller's ``out``; the library allocates nothing
    (fixed scratch array, see include/tg.h)."""
    _check(lib().tg_count_global_noalloc(g.handle, k, _ptr(out), _stream(stream)),
           "tg_count_global_noalloc")
    return out


def _handles(graphs, outs):
    G = len(graphs)
    if len(outs) != G:
        raise ValueError("one output per graph")
    hs = (ctypes.c_void_p * max(G, 1))(*[g.handle.value for g in graphs])
    ps = (ctypes.c_void_p * max(G, 1))(*[_ptr(o).value for o in outs])
    return G, hs, ps


class Batch:
    """A batched-count plan over resident graphs (include/tg.h, tg_batch_*).

    ``outs`` are device tensors, one per graph (global histograms or per-edge
    rows, by ``mode``).  The graphs and outputs must outlive the plan."""

    PATHS = {"auto": TG_KERNEL_AUTO, "union": TG_KERNEL_CYCLES, "persistent": TG_KERNEL_WARP_SEARCH}

    def __init__(self, graphs, k, mode, outs, cta_threads=0, stream=None, path="auto"):
        """``path``: "auto" (union when it can be built; tune() picks), "union"
        (required) or "persistent" (the single persistent launch only)."""
        self._graphs, self._outs = list(graphs), list(outs)
        G, hs, ps = _handles(self._graphs, self._outs)
        self._keep = (hs, ps)
        kern = self.PATHS[path]
        tune = TGTune(kern, cta_threads, 0, 0, 0, 0, 0, 0, 0) if (cta_threads or kern) else None
        h = ctypes.c_void_p()
        _check(lib().tg_batch_create(G, hs, k, mode, ps, ctypes.byref(tune) if tune else None,
                                     _stream(stream), ctypes.byref(h)), "tg_batch_create")
        self._h = h

    def run(self, stream=None):
        _check(lib().tg_batch_run(self._h, _stream(stream)), "tg_batch_run")

    def tune(self, stream=None) -> int:
        best = ctypes.c_int32(0)
        _check(lib().tg_batch_tune(self._h, _stream(stream), ctypes.byref(best)), "tg_batch_tune")
        return int(best.value)

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().tg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tg_count_batch(graphs, k, mode, outs, cta_threads=0, stream=None):
    """One-shot batched count (autotuned unless ``cta_threads`` is given)."""
    G, hs, ps = _handles(list(graphs), list(outs))
    tune = TGTune(0, cta_threads, 0, 0, 0, 0, 0, 0, 0) if cta_threads else None
    _check(lib().tg_count_batch(G, hs, k, mode, ps, ctypes.byref(tune) if tune else None,
                                _stream(stream)), "tg_count_batch")
    return outs


class Server:
    """The serving loop (include/tg.h, tg_serve_*)."""

    def __init__(self, slots=4, mem_budget_bytes=8 << 30, queue_cap=4096, device=0, batch_max=32,
                 batch_edges=20000):
        self._cfg = TGServeCfg(slots, queue_cap, mem_budget_bytes, device, batch_max, batch_edges)
        h = lib().tg_serve_create(ctypes.byref(self._cfg))
        if not h:
            raise TGError(TG_ENOMEM, "tg_serve_create")
        self._h = ctypes.c_void_p(h)
        self._meta = {}

    def submit(self, n, src, dst, types, L, k=4) -> int:
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
        types = np.ascontiguousarray(types, dtype=np.uint8)
        req = TGRequest(int(n), int(src.shape[0]), _ptr(src), _ptr(dst), _ptr(types), int(L), int(k))
        t = ctypes.c_uint64(0)
        _check(lib().tg_serve_submit(self._h, ctypes.byref(req), ctypes.byref(t)), "tg_serve_submit")
        self._meta[t.value] = (L, k)
        return int(t.value)

    def wait(self, ticket, timeout_ms=60000):
        L, k = self._meta.get(ticket, (16, 4))
        out = np.zeros(max(1, tg_global_len(L, k)), np.uint64)
        info = TGResult()
        rc = lib().tg_serve_wait(self._h, ticket, int(timeout_ms), _ptr(out), out.shape[0],
                                 ctypes.byref(info))
        if rc == TG_ECUDA and info.cuda_error:
            raise TGError(rc, f"tg_serve_wait (cudaError_t {info.cuda_error})")
        _check(rc, "tg_serve_wait")
        self._meta.pop(ticket, None)
        return out[: info.len], info.latency_ms

    def stats(self) -> dict:
        st = TGServeStats()
        _check(lib().tg_serve_stats(self._h, ctypes.byref(st)), "tg_serve_stats")
        return {f: getattr(st, f) for f, _ in TGServeStats._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().tg_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tg_count_per_edge(g: Graph, k: int = 4, level: int = TG_GRAPHLET, rows=None, stream=None):
    if rows is None:
        rows = np.zeros((g.M, tg_slots(g.L, k, level)), np.uint64)
    _check(lib().tg_count_per_edge(g.handle, k, level, _ptr(rows), _stream(stream)),
           "tg_count_per_edge")
    return rows


def tg_count_range(g: Graph, k: int, e0: int, e1: int, sums=None, stream=None):
    if sums is None:
        sums = np.zeros(tg_global_len(g.L, k), np.uint64)
    _check(lib().tg_count_range(g.handle, k, int(e0), int(e1), _ptr(sums), _stream(stream)),
           "tg_count_range")
    return sums


def tg_count_per_edge_sparse(g: Graph, k: int = 4, level: int = TG_GRAPHLET, stream=None):
    """Sparse per-edge counts: (offsets [M+1], ids, counts) as numpy arrays."""
    offsets = np.zeros(g.M + 1, np.int64)
    nnz = ctypes.c_int64(0)
    _check(lib().tg_count_per_edge_sparse(g.handle, k, level, _ptr(offsets), None, None, 0,
                                          ctypes.byref(nnz), _stream(stream)), "tg_count_per_edge_sparse")
    ids = np.zeros(max(1, nnz.value), np.uint32)
    counts = np.zeros(max(1, nnz.value), np.uint64)
    _check(lib().tg_count_per_edge_sparse(g.handle, k, level, _ptr(offsets), _ptr(ids), _ptr(counts),
                                          ids.shape[0], ctypes.byref(nnz), _stream(stream)),
           "tg_count_per_edge_sparse")
    return offsets, ids[: nnz.value], counts[: nnz.value]


def tg_sparse_ids(L: int, k: int = 4, level: int = TG_GRAPHLET) -> int:
    return int(lib().tg_sparse_ids(L, k, level))


def tg_sparse_id(L: int, k: int, level: int, sid: int):
    """(graphlet or orbit number, sorted types) of a sparse id."""
    motif = ctypes.c_int32()
    kk = ctypes.c_int32()
    t = np.zeros(4, np.int32)
    _check(lib().tg_sparse_id(L, k, level, int(sid), ctypes.byref(motif), _ptr(t), ctypes.byref(kk)),
           "tg_sparse_id")
    return int(motif.value), tuple(int(x) for x in t[: kk.value])


def tg_count_shard(g: Graph, k: int, shard: int, nshards: int, sums=None, stream=None):
    """Undivided sums of one shard of a global count split over ``nshards``."""
    if sums is None:
        sums = np.zeros(tg_global_len(g.L, k), np.uint64)
    _check(lib().tg_count_shard(g.handle, k, int(shard), int(nshards), _ptr(sums), _stream(stream)),
           "tg_count_shard")
    return sums


def tg_global_finalize(L: int, k: int, sums) -> np.ndarray:
    s = np.ascontiguousarray(sums, dtype=np.uint64)
    out = np.zeros_like(s)
    _check(lib().tg_global_finalize(L, k, _ptr(s), _ptr(out)), "tg_global_finalize")
    return out


def tg_work_model(g: Graph, stream=None) -> int:
    v = np.zeros(1, np.uint64)
    _check(lib().tg_work_model(g.handle, _ptr(v), _stream(stream)), "tg_work_model")
    return int(v[0])


def tg_set_tune(kernel=0, cta_threads=0, unroll=0, hash_slots=0, bitmap_bits=0, grid_limit=0,
                edge_pass=0, edge_batch=0, c4_bin_fill=0, reset=False) -> None:
    """Set the counting kernels' launch configuration (``reset`` restores defaults)."""
    if reset:
        _check(lib().tg_set_tune(None), "tg_set_tune")
        return
    t = TGTune(kernel, cta_threads, unroll, hash_slots, bitmap_bits, grid_limit, edge_pass, edge_batch,
               c4_bin_fill)
    _check(lib().tg_set_tune(ctypes.byref(t)), "tg_set_tune")


def tg_autotune(g: Graph, k: int, stream=None) -> dict:
    """Search the launch configuration for ``g``'s class (tg_autotune); the winner
    becomes the process-wide tuning and is returned as a dict."""
    t = TGTune()
    _check(lib().tg_autotune(g.handle, int(k), ctypes.byref(t), _stream(stream)), "tg_autotune")
    return {f: getattr(t, f) for f, _ in TGTune._fields_}


def tg_autotune_reset() -> None:
    """Forget every cached autotune class."""
    _check(lib().tg_autotune_reset(), "tg_autotune_reset")


def tg_get_tune() -> dict:
    t = TGTune()
    _check(lib().tg_get_tune(ctypes.byref(t)), "tg_get_tune")
    return {f: getattr(t, f) for f, _ in TGTune._fields_}


def tg_launch_count() -> int:
    """Kernels launched by libtg.so so far in this process."""
    return int(lib().tg_launch_count())


def tg_set_memory_retention(nbytes: int) -> None:
    """Keep up to ``nbytes`` of freed device scratch mapped between calls (0 restores
    the default pool, which returns scratch to the device at each synchronisation)."""
    _check(lib().tg_set_memory_retention(int(nbytes)), "tg_set_memory_retention")


def tg_trim_memory() -> None:
    """Release the scratch the library's pools keep, keeping the retention setting."""
    _check(lib().tg_trim_memory(), "tg_trim_memory")


def tg_last_cuda_error() -> int:
    """cudaError_t of this thread's last failed CUDA call inside libtg.so (0 if none)."""
    return int(lib().tg_last_cuda_error())


def tg_last_timing() -> dict:
    """Per-phase device times (ms) and work counters of the last count call."""
    t = TGTiming()
    _check(lib().tg_last_timing(ctypes.byref(t)), "tg_last_timing")
    return {f: getattr(t, f) for f, _ in TGTiming._fields_}


def tg_debug_fail_alloc(n: int) -> None:
    _check(lib().tg_debug_fail_alloc(int(n)), "tg_debug_fail_alloc")
