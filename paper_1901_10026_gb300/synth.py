"""Seeded synthetic typed graphs: the inputs both the CUDA path and the oracle see.

This module holds none of the counting arithmetic.  It only draws random
undirected edge lists (with possible duplicates and self-loops, which the
graph builders on both sides remove) and node-type vectors.  Every draw goes
through numpy's Philox counter-based generator keyed by a SeedSequence, whose
output is defined bit for bit independently of the host CPU, so the same seed
gives the same graph on x86 and on Arm.

Graph families (node-typed, undirected; the paper's synthetic families are
Erdos-Renyi and Chung-Lu, Sec. 7 "Experiments", Table 3 synthetic rows):

* ``erdos_renyi(n, p)``: every unordered pair kept independently with
  probability p, sampled exactly by geometric skipping over the pair index.
* ``chung_lu_exact(n, m, gamma)``: weights w_v = (v+1)^(-1/(gamma-1)); both
  endpoints of each draw are i.i.d. proportional to w; draws continue until the
  prefix of draws holds exactly m distinct non-loop pairs.  The returned list is
  that whole prefix (duplicates and loops included).
* ``chung_lu_draws(n, draws, gamma)``: the same endpoint law, a fixed number of
  draws (the unique edge count is then whatever comes out).
* ``rmat(scale, edge_factor, a, b, c, d)``: recursive-matrix draws, no noise.

Type laws: ``uniform_types`` and ``zipf_types`` (P(t) proportional to
(t+1)^-s on t in [0, L)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "TypedEdgeList",
    "rng",
    "erdos_renyi",
    "chung_lu_exact",
    "chung_lu_draws",
    "rmat",
    "uniform_types",
    "zipf_types",
    "er_1000",
    "cl_1m",
    "rmat_23",
    "batch_spec",
    "batch_graph",
    "serve_stream",
    "tiny_random",
    "er_avg_degree",
    "er_exact",
    "cl_sweep",
    "type_permutations",
    "er_directed",
]


@dataclass
class TypedEdgeList:
    """An undirected node-typed graph as raw int32 endpoint arrays.

    ``src``/``dst`` may hold duplicates, both orientations of a pair and
    self-loops; consumers simplify the graph themselves.
    """

    n: int
    src: np.ndarray  # int32
    dst: np.ndarray  # int32
    types: np.ndarray  # uint8, length n
    L: int
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.src.shape[0])


def rng(*key: int) -> np.random.Generator:
    """Philox stream for an integer key tuple (platform independent)."""
    return np.random.Generator(np.random.Philox(np.random.SeedSequence(list(key))))


def _pair_index_to_uv(k: np.ndarray):
    """Linear index over pairs (u < v), ordered by v then u, to (u, v)."""
    k = k.astype(np.int64)
    v = np.floor((1.0 + np.sqrt(1.0 + 8.0 * k.astype(np.float64))) / 2.0).astype(np.int64)
    # exact correction of the float estimate
    for _ in range(2):
        too_big = v * (v - 1) // 2 > k
        v = np.where(too_big, v - 1, v)
        too_small = (v + 1) * v // 2 <= k
        v = np.where(too_small, v + 1, v)
    u = k - v * (v - 1) // 2
    return u, v


def erdos_renyi(n: int, p: float, g: np.random.Generator):
    """G(n, p) by geometric skipping: exact Bernoulli(p) on each of the C(n,2) pairs."""
    total = n * (n - 1) // 2
    if total == 0 or p <= 0.0:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    if p >= 1.0:
        k = np.arange(total, dtype=np.int64)
    else:
        chunks = []
        pos = -1
        expect = int(total * p * 1.1) + 64
        while True:
            gaps = g.geometric(p, size=expect).astype(np.int64)
            idx = pos + np.cumsum(gaps)
            keep = idx[idx < total]
            chunks.append(keep)
            if keep.shape[0] < idx.shape[0]:
                break
            pos = int(idx[-1])
        k = np.concatenate(chunks) if chunks else np.zeros(0, np.int64)
    u, v = _pair_index_to_uv(k)
    return u.astype(np.int32), v.astype(np.int32)


def _cl_sampler(n: int, gamma: float):
    w = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (gamma - 1.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    return cdf


def _cl_endpoints(cdf: np.ndarray, count: int, g: np.random.Generator) -> np.ndarray:
    x = g.random(count)
    out = np.searchsorted(cdf, x, side="right")
    np.minimum(out, cdf.shape[0] - 1, out=out)
    return out.astype(np.int32)


def chung_lu_draws(n: int, draws: int, gamma: float, g: np.random.Generator):
    """``draws`` i.i.d. endpoint pairs with P(v) proportional to (v+1)^(-1/(gamma-1))."""
    cdf = _cl_sampler(n, gamma)
    u = _cl_endpoints(cdf, draws, g)
    v = _cl_endpoints(cdf, draws, g)
    return u, v


def chung_lu_exact(n: int, m: int, gamma: float, g: np.random.Generator):
    """Chung-Lu draws until the draw prefix holds exactly ``m`` distinct non-loop pairs.

    Draws come in blocks of (u-block, v-block); the prefix length K is the
    smallest for which the first K draws contain m distinct unordered pairs
    with u != v.  Returns the first K draws.
    """
    cdf = _cl_sampler(n, gamma)
    us, vs = [], []
    total = 0
    block = max(1024, int(m * 1.25))
    while True:
        us.append(_cl_endpoints(cdf, block, g))
        vs.append(_cl_endpoints(cdf, block, g))
        total += block
        u = np.concatenate(us)
        v = np.concatenate(vs)
        lo = np.minimum(u, v).astype(np.int64)
        hi = np.maximum(u, v).astype(np.int64)
        key = lo * n + hi
        key = np.where(lo == hi, -1, key)
        uniq, first = np.unique(key, return_index=True)
        if uniq.shape[0] and uniq[0] == -1:
            first = first[1:]
        if first.shape[0] >= m:
            first.sort()
            K = int(first[m - 1]) + 1
            return u[:K].copy(), v[:K].copy()
        block = max(1024, int((m - first.shape[0]) * 2.0 * total / max(first.shape[0], 1)) + 1024)
        if total > 64 * m + (1 << 20):
            raise RuntimeError("chung_lu_exact: target edge count not reachable")


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, d: float,
         g: np.random.Generator, chunk: int = 1 << 24):
    """R-MAT draws: ``edge_factor * 2^scale`` pairs, one quadrant choice per bit level."""
    n = 1 << scale
    draws = edge_factor * n
    us = np.empty(draws, np.int32)
    vs = np.empty(draws, np.int32)
    ab = a + b
    abc = a + b + c
    for s in range(0, draws, chunk):
        e = min(draws, s + chunk)
        cnt = e - s
        u = np.zeros(cnt, np.int64)
        v = np.zeros(cnt, np.int64)
        for level in range(scale):
            x = g.random(cnt)
            bit = np.int64(1) << (scale - 1 - level)
            # quadrants: a = (0,0), b = (0,1), c = (1,0), d = (1,1)
            right = ((x >= a) & (x < ab)) | (x >= abc)
            down = x >= ab
            u += np.where(down, bit, 0)
            v += np.where(right, bit, 0)
        us[s:e] = u
        vs[s:e] = v
    return us, vs


def uniform_types(n: int, L: int, g: np.random.Generator) -> np.ndarray:
    return g.integers(0, L, size=n, dtype=np.int64).astype(np.uint8)


def zipf_types(n: int, L: int, s: float, g: np.random.Generator) -> np.ndarray:
    p = (np.arange(L, dtype=np.float64) + 1.0) ** (-s)
    cdf = np.cumsum(p)
    cdf /= cdf[-1]
    t = np.searchsorted(cdf, g.random(n), side="right")
    return np.minimum(t, L - 1).astype(np.uint8)


# --------------------------------------------------------------------------
# The five workloads (sizes as named in each docstring)
# --------------------------------------------------------------------------

def er_1000(seed: int = 1) -> TypedEdgeList:
    """Erdos-Renyi G(n=1000, p=0.01), L=3 uniform types."""
    g = rng(1, seed)
    u, v = erdos_renyi(1000, 0.01, g)
    t = uniform_types(1000, 3, g)
    return TypedEdgeList(1000, u, v, t, 3, "er-1000-p0.01-L3")


def cl_1m(seed: int = 2, n: int = 1_000_000, m: int = 8_000_000) -> TypedEdgeList:
    """Chung-Lu, n=1M, exactly 8M distinct edges (average degree 16), gamma=2.1,
    L=5 types drawn Zipf(s=1.2)."""
    g = rng(2, seed, n, m)
    u, v = chung_lu_exact(n, m, 2.1, g)
    t = zipf_types(n, 5, 1.2, g)
    return TypedEdgeList(n, u, v, t, 5, f"cl-n{n}-m{m}-g2.1-L5zipf1.2")


def rmat_23(seed: int = 3, scale: int = 23) -> TypedEdgeList:
    """R-MAT scale 23, edge factor 16, (0.57, 0.19, 0.19, 0.05), L=8 uniform types."""
    g = rng(3, seed, scale)
    u, v = rmat(scale, 16, 0.57, 0.19, 0.19, 0.05, g)
    t = uniform_types(1 << scale, 8, g)
    return TypedEdgeList(1 << scale, u, v, t, 8, f"rmat-s{scale}-ef16-L8")


@dataclass
class BatchItem:
    idx: int
    family: str  # "er" or "cl"
    n: int
    avg_degree: float
    gamma: float
    L: int


def batch_spec(count: int = 10_000, seed: int = 5):
    """Per-graph parameters of the batched workload.

    n = floor(exp(U(ln 20, ln 5000))); even index -> ER with average degree
    U[4, 32] (p = dbar/(n-1), capped at 1); odd index -> Chung-Lu with exponent
    U[2.0, 2.8] and the same average-degree law, capped at (n-1)/2; L uniform
    on {2..8}; uniform node types.
    """
    out = []
    for idx in range(count):
        g = rng(5, seed, idx)
        n = int(math.floor(math.exp(g.uniform(math.log(20.0), math.log(5000.0)))))
        dbar = float(g.uniform(4.0, 32.0))
        gamma = float(g.uniform(2.0, 2.8))
        L = int(g.integers(2, 9))
        fam = "er" if idx % 2 == 0 else "cl"
        if fam == "cl":
            dbar = min(dbar, (n - 1) / 2.0)
        out.append(BatchItem(idx, fam, n, dbar, gamma, L))
    return out


def batch_graph(item: BatchItem, seed: int = 5) -> TypedEdgeList:
    """The graph of one batch item (ER: exact G(n,p); CL: round(n*dbar/2) draws)."""
    g = rng(6, seed, item.idx)
    if item.family == "er":
        p = min(1.0, item.avg_degree / max(item.n - 1, 1))
        u, v = erdos_renyi(item.n, p, g)
    else:
        draws = int(round(item.n * item.avg_degree / 2.0))
        u, v = chung_lu_draws(item.n, draws, item.gamma, g)
    t = uniform_types(item.n, item.L, g)
    return TypedEdgeList(item.n, u, v, t, item.L, f"batch-{item.idx}-{item.family}")


def serve_stream(count: int = 2000, seed: int = 7, e_lo: float = 1e3, e_hi: float = 2e6,
                 L: int = 6, gamma: float = 2.1, rate: float = 1.0):
    """Request stream of the serving workload: (arrival_time, target_edges, key).

    Target edges are log-uniform in [e_lo, e_hi]; each request graph is a
    Chung-Lu graph with average degree 16 (n = edges/8), exponent ``gamma``,
    ``L`` uniform types; inter-arrival gaps are Exponential(1/rate).
    """
    g = rng(7, seed)
    gaps = g.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    edges = np.floor(np.exp(g.uniform(math.log(e_lo), math.log(e_hi), size=count))).astype(np.int64)
    return [(float(t[r]), int(edges[r]), (8, seed, r)) for r in range(count)]


def serve_graph(target_edges: int, key, L: int = 6, gamma: float = 2.1) -> TypedEdgeList:
    n = max(16, target_edges // 8)
    g = rng(*key)
    u, v = chung_lu_exact(n, min(target_edges, n * (n - 1) // 4), gamma, g)
    t = uniform_types(n, L, g)
    return TypedEdgeList(n, u, v, t, L, f"serve-{key[-1]}")


def er_avg_degree(n: int, dbar: float, L: int, seed: int = 1) -> TypedEdgeList:
    """Erdos-Renyi G(n, p = dbar / (n - 1)), L uniform types (the paper's
    scalability series: average degree 10, n from 100 to 10^6)."""
    g = rng(9, seed, n, int(round(dbar * 1000)), L)
    u, v = erdos_renyi(n, min(1.0, dbar / max(n - 1, 1)), g)
    return TypedEdgeList(n, u, v, uniform_types(n, L, g), L, f"er-n{n}-d{dbar:g}-L{L}")


def er_exact(n: int, m: int, L: int, seed: int = 1) -> TypedEdgeList:
    """G(n, m): m distinct pairs drawn uniformly (repeats redrawn), L uniform
    types (the number-of-types sweep's Erdos-Renyi graph)."""
    g = rng(10, seed, n, m, L)
    total = n * (n - 1) // 2
    if m > total:
        raise ValueError("er_exact: more edges than pairs")
    keys = np.zeros(0, np.int64)
    while keys.shape[0] < m:
        draw = g.integers(0, total, size=int((m - keys.shape[0]) * 1.1) + 16, dtype=np.int64)
        keys = np.unique(np.concatenate([keys, draw]))
    keys = g.permutation(keys)[:m]
    u, v = _pair_index_to_uv(keys)
    return TypedEdgeList(n, u.astype(np.int32), v.astype(np.int32), uniform_types(n, L, g), L,
                         f"er-n{n}-m{m}-L{L}")


def cl_sweep(n: int, m: int, L: int, gamma: float = 2.1, seed: int = 1) -> TypedEdgeList:
    """Chung-Lu with exactly m distinct edges, L uniform types (the
    number-of-types sweep's skewed graph)."""
    g = rng(11, seed, n, m, L)
    u, v = chung_lu_exact(n, m, gamma, g)
    return TypedEdgeList(n, u, v, uniform_types(n, L, g), L, f"cl-n{n}-m{m}-L{L}")


def type_permutations(types: np.ndarray, count: int, seed: int = 1):
    """`count` random permutations of a node-type vector (the null model of
    Sec. "Exploratory Analysis": same topology, same type counts)."""
    g = rng(12, seed, int(types.shape[0]), count)
    return [g.permutation(types).astype(np.uint8) for _ in range(count)]


def er_directed(n: int, m: int, recip: float, L: int, seed: int = 1) -> TypedEdgeList:
    """m arcs src -> dst with endpoints uniform (loops and repeats possible),
    and the reverse of each arc added with probability ``recip`` (pairs with
    arcs both ways); L uniform types.  Read with TG_DIRECTED."""
    g = rng(14, seed, n, m, int(round(recip * 1000)), L)
    src = g.integers(0, n, size=m, dtype=np.int64).astype(np.int32)
    dst = g.integers(0, n, size=m, dtype=np.int64).astype(np.int32)
    back = g.random(m) < recip
    return TypedEdgeList(n, np.concatenate([src, dst[back]]), np.concatenate([dst, src[back]]),
                         uniform_types(n, L, g), L, f"dir-er-n{n}-m{m}-r{recip:g}-L{L}")


def tiny_random(n: int, density: float, L: int, g: np.random.Generator) -> TypedEdgeList:
    """Small G(n, density) with uniform types and a few duplicate/reversed/loop draws."""
    u, v = erdos_renyi(n, density, g)
    t = uniform_types(n, L, g) if n > 0 else np.zeros(0, np.uint8)
    if u.shape[0] and n > 0:
        extra = min(3, u.shape[0])
        pick = g.integers(0, u.shape[0], size=extra)
        u = np.concatenate([u, v[pick], np.array([0], np.int32)])
        v = np.concatenate([v, u[pick], np.array([0], np.int32)])
    return TypedEdgeList(n, u.astype(np.int32), v.astype(np.int32), t, L, f"tiny-{n}")
