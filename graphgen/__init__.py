"""Seeded synthetic graphs shaped like the paper's workloads (Section 5 uses
undirected SNAP/KONECT graphs; those are not available, so Erdos-Renyi, R-MAT
and Chung-Lu graphs stand in for them).

This package produces inputs only and holds none of the Katz arithmetic: the
CPU oracle and the CUDA path both consume its CSR graphs.  The generators'
graphs are undirected, stored as a symmetric CSR (int64 ``rowptr``, int32
``col``) with sorted rows, no self-loops and no duplicate arcs; ``orient`` and
the ``directed_*`` helpers derive directed graphs (the same CSR, not
symmetric) and directed update batches from them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None

# Seeds: one per workload, derived from the paper's arXiv id.
SEED_BASE = 180703847


def build(force: bool = False) -> str:
    """Compile ``libgraphgen.so`` next to its source (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i64, u64, dbl = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            lib.gg_er.restype = P
            lib.gg_er.argtypes = [i64, i64, u64]
            lib.gg_rmat.restype = P
            lib.gg_rmat.argtypes = [ctypes.c_int, i64, dbl, dbl, dbl, u64]
            lib.gg_chung_lu.restype = P
            lib.gg_chung_lu.argtypes = [i64, i64, dbl, dbl, u64]
            lib.gg_band_union.restype = P
            lib.gg_band_union.argtypes = [i64, P, P, i64, i64, i64]
            lib.gg_from_pairs.restype = P
            lib.gg_from_pairs.argtypes = [i64, i64, P, P]
            lib.gg_n.restype = i64
            lib.gg_n.argtypes = [P]
            lib.gg_nnz.restype = i64
            lib.gg_nnz.argtypes = [P]
            lib.gg_copy.restype = None
            lib.gg_copy.argtypes = [P, P, P]
            lib.gg_free.restype = None
            lib.gg_free.argtypes = [P]
            lib.gg_max_threads.restype = ctypes.c_int
            lib.gg_update_batch.restype = i64
            lib.gg_update_batch.argtypes = [i64, P, P, i64, dbl, u64, P, P, P]
            lib.gg_stream_total.restype = i64
            lib.gg_stream_total.argtypes = [i64, i64, i64, u64]
            lib.gg_stream.restype = i64
            lib.gg_stream.argtypes = [i64, P, P, i64, i64, i64, i64, dbl, dbl, u64, i64, P, P, P, P, P]
            _lib = lib
    return _lib


class Graph:
    """Undirected graph as a symmetric CSR on the host."""

    def __init__(self, rowptr: np.ndarray, col: np.ndarray, name: str = ""):
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.name = name

    @property
    def n(self) -> int:
        return int(self.rowptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.rowptr)

    def deg_max(self) -> int:
        return int(self.degrees().max()) if self.n else 0

    def __repr__(self) -> str:
        return f"Graph({self.name!r}, n={self.n}, nnz={self.nnz})"


def _take(ptr, name: str) -> Graph:
    lib = _load()
    if not ptr:
        raise MemoryError(f"graph generator failed for {name}")
    try:
        n, nnz = lib.gg_n(ptr), lib.gg_nnz(ptr)
        rowptr = np.empty(n + 1, dtype=np.int64)
        col = np.empty(max(nnz, 1), dtype=np.int32)
        lib.gg_copy(ptr, rowptr.ctypes.data, col.ctypes.data)
    finally:
        lib.gg_free(ptr)
    return Graph(rowptr, col[:nnz], name)


def erdos_renyi(n: int, m: int, seed: int) -> Graph:
    """G(n, m): m distinct uniform undirected edges, no self-loops."""
    return _take(_load().gg_er(n, m, seed), f"er_n{n}_m{m}_s{seed}")


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = SEED_BASE) -> Graph:
    """R-MAT with 2^scale vertices and edge_factor*2^scale generated pairs,
    symmetrised and deduplicated (no noise, no vertex permutation)."""
    return _take(_load().gg_rmat(scale, edge_factor, a, b, c, seed), f"rmat{scale}_ef{edge_factor}_s{seed}")


def chung_lu(n: int, mean_degree: float = 16.0, exponent: float = 2.1, seed: int = SEED_BASE,
             pairs: int | None = None) -> Graph:
    """Chung-Lu graph with Pareto expected degrees (pdf exponent ``exponent``,
    scale chosen for the requested mean before capping at sqrt(sum w))."""
    tail = exponent - 1.0
    x_m = mean_degree * (tail - 1.0) / tail
    if pairs is None:
        pairs = int(n * mean_degree // 2)
    return _take(_load().gg_chung_lu(n, pairs, tail, x_m, seed), f"chunglu_n{n}_s{seed}")


def band_union(g: Graph, n_band: int, d: int, n_pad: int = 0) -> Graph:
    """g, then a band graph on n_band nodes (i ~ j iff 0 < |i - j| <= d), then
    n_pad isolated nodes, as one undirected graph (disjoint union)."""
    return _take(_load().gg_band_union(g.n, g.rowptr.ctypes.data, g.col.ctypes.data, n_band, d, n_pad),
                 f"{g.name}+band{n_band}x{d}+{n_pad}")


def padded_to(g: Graph, total: int, d: int = 128) -> Graph:
    """g padded by a band of half-width d and isolated nodes so that n + nnz
    of the result is exactly `total` (e.g. just below 2^31 - 1, the limit of
    32-bit row offsets).  A band node adds 2d + 1 to n + nnz, less d(d+1) in all
    for the band's two ends."""
    rest = total - (g.n + g.nnz)
    if rest < 0:
        raise ValueError("graph already larger than the target")
    n_band = (rest + d * (d + 1)) // (2 * d + 1)
    while n_band > 0 and n_band * (2 * d + 1) - d * (d + 1) > rest:
        n_band -= 1
    if n_band <= d:
        n_band = 0
    band = 2 * d * n_band - d * (d + 1) + n_band if n_band else 0
    out = band_union(g, n_band, d, rest - band)
    assert out.n + out.nnz == total
    return out


def from_edges(n: int, u, v, name: str = "pairs") -> Graph:
    """Symmetric CSR of the undirected pairs (u[i], v[i]) (self-loops dropped,
    repeats merged)."""
    u = np.ascontiguousarray(u, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.int32)
    assert u.shape == v.shape
    return _take(_load().gg_from_pairs(n, u.shape[0], u.ctypes.data, v.ctypes.data), name)


def complete(n: int) -> Graph:
    iu, ju = np.triu_indices(n, 1)
    return from_edges(n, iu, ju, f"K{n}")


def star(leaves: int) -> Graph:
    return from_edges(leaves + 1, np.zeros(leaves, np.int32), np.arange(1, leaves + 1), f"star{leaves}")


def path(n: int) -> Graph:
    return from_edges(n, np.arange(n - 1), np.arange(1, n), f"path{n}")


def cycle(n: int) -> Graph:
    return from_edges(n, np.arange(n), (np.arange(n) + 1) % n, f"cycle{n}")


def update_batch(g: Graph, m: int, seed: int, p_insert: float = 0.5):
    """Draw m undirected updates against g: inserts are uniform non-edges,
    deletes are uniform existing edges; no pair repeats within the batch.
    Returns (src, dst, is_insert) as int32/int32/uint8 arrays."""
    lib = _load()
    src = np.empty(max(m, 1), np.int32)
    dst = np.empty(max(m, 1), np.int32)
    ins = np.empty(max(m, 1), np.uint8)
    got = lib.gg_update_batch(g.n, g.rowptr.ctypes.data, g.col.ctypes.data, m, p_insert, seed,
                              src.ctypes.data, dst.ctypes.data, ins.ctypes.data)
    return src[:got], dst[:got], ins[:got]


class Stream:
    """A sequence of update batches with arrival times (seconds)."""

    def __init__(self, offsets, src, dst, is_insert, arrival):
        self.offsets, self.src, self.dst, self.is_insert, self.arrival = offsets, src, dst, is_insert, arrival

    def __len__(self) -> int:
        return len(self.arrival)

    def batch(self, j: int):
        a, b = self.offsets[j], self.offsets[j + 1]
        return self.src[a:b], self.dst[a:b], self.is_insert[a:b]

    def sizes(self) -> np.ndarray:
        return np.diff(self.offsets)


def stream(g: Graph, batches: int, seed: int, min_size: int = 1, max_size: int = 10000, p_insert: float = 0.5,
           rate: float = 200.0, deg_bound: int | None = None) -> Stream:
    """Update batches applied one after another to g: sizes log-uniform in
    [min_size, max_size]; inserts are uniform non-edges (degrees kept at or
    below deg_bound), deletes uniform existing edges, no pair twice within a
    batch; Poisson arrivals at `rate` batches per second."""
    lib = _load()
    total = lib.gg_stream_total(batches, min_size, max_size, seed)
    offsets = np.zeros(batches + 1, np.int64)
    src = np.empty(max(total, 1), np.int32)
    dst = np.empty(max(total, 1), np.int32)
    ins = np.empty(max(total, 1), np.uint8)
    arrival = np.empty(max(batches, 1), np.float64)
    D = int(deg_bound) if deg_bound is not None else g.deg_max() + 64
    got = lib.gg_stream(g.n, g.rowptr.ctypes.data, g.col.ctypes.data, D, batches, min_size, max_size, p_insert,
                        rate, seed, total, offsets.ctypes.data, src.ctypes.data, dst.ctypes.data, ins.ctypes.data,
                        arrival.ctypes.data)
    if got < 0:
        raise MemoryError("gg_stream: out of memory")
    return Stream(offsets, src[:got], dst[:got], ins[:got], arrival[:batches])


def apply_batch(g: Graph, src, dst, is_insert) -> Graph:
    """The graph after an update batch (host-side, for building test inputs)."""
    n = g.n
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.rowptr))
    keys = rows * n + g.col.astype(np.int64)
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    ins = np.asarray(is_insert).astype(bool)
    dele = np.concatenate([src[~ins] * n + dst[~ins], dst[~ins] * n + src[~ins]])
    keep = keys[~np.isin(keys, dele)]
    add = np.concatenate([src[ins] * n + dst[ins], dst[ins] * n + src[ins]])
    allk = np.concatenate([keep, add])
    u = (allk // n).astype(np.int32)
    v = (allk % n).astype(np.int32)
    sel = u < v
    return from_edges(n, u[sel], v[sel], g.name + "+batch")


def directed_from_arcs(n: int, u, v, name: str = "arcs") -> Graph:
    """CSR of the arcs u[i] -> v[i] (self-loops dropped, repeats merged)."""
    u = np.asarray(u, np.int64)
    v = np.asarray(v, np.int64)
    keep = u != v
    keys = np.unique(u[keep] * n + v[keep])
    rows = keys // n
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, rows + 1, 1)
    return Graph(np.cumsum(rowptr), (keys % n).astype(np.int32), name)


def orient(g: Graph, seed: int, p_keep: float = 0.5) -> Graph:
    """A directed graph from an undirected one: each arc of the symmetric CSR
    is kept independently with probability p_keep, so some edges stay
    reciprocal, some become one-way and some vanish."""
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.rowptr))
    keep = rng.random(g.nnz) < p_keep
    return directed_from_arcs(g.n, rows[keep], g.col[keep], g.name + f"_dir{seed}")


def reverse(g: Graph) -> Graph:
    """The reverse graph: arc v -> u for every arc u -> v of g."""
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.rowptr))
    return directed_from_arcs(g.n, g.col.astype(np.int64), rows, g.name + "_rev")


def directed_update_batch(g: Graph, m: int, seed: int, p_insert: float = 0.5, deg_bound: int | None = None):
    """Draw m directed updates against the directed graph g: inserts are
    uniform ordered non-arcs (out-degrees kept at or below deg_bound), deletes
    uniform existing arcs; no ordered pair repeats within the batch (a -> b
    and b -> a may both appear).  Returns (src, dst, is_insert)."""
    rng = np.random.default_rng(seed)
    n = g.n
    D = int(deg_bound) if deg_bound is not None else (g.deg_max() if g.n else 0) + 64
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.rowptr))
    present = rows * n + g.col.astype(np.int64)  # sorted: rows ascending, columns sorted
    n_ins = int(rng.binomial(m, p_insert)) if m > 0 else 0
    n_del = min(m - n_ins, len(present))
    dels = rng.choice(present, size=n_del, replace=False) if n_del > 0 else np.zeros(0, np.int64)
    outdeg = np.diff(g.rowptr).astype(np.int64)
    ins_keys, seen = [], set()
    tries = 0
    while len(ins_keys) < n_ins and tries < 50 * (n_ins + 1):
        tries += 1
        a, b = int(rng.integers(0, n)), int(rng.integers(0, n))
        key = a * n + b
        if a == b or key in seen:
            continue
        pos = np.searchsorted(present, key)
        if pos < len(present) and present[pos] == key:
            continue
        if outdeg[a] + 1 > D:
            continue
        seen.add(key)
        outdeg[a] += 1
        ins_keys.append(key)
    keys = np.concatenate([np.array(ins_keys, np.int64), dels])
    ins = np.concatenate([np.ones(len(ins_keys), np.uint8), np.zeros(len(dels), np.uint8)])
    order = rng.permutation(len(keys))
    keys, ins = keys[order], ins[order]
    return (keys // n).astype(np.int32), (keys % n).astype(np.int32), ins


def apply_directed_batch(g: Graph, src, dst, is_insert) -> Graph:
    """The directed graph after an update batch (host-side, for test inputs)."""
    n = g.n
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.rowptr))
    keys = rows * n + g.col.astype(np.int64)
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    ins = np.asarray(is_insert).astype(bool)
    keep = keys[~np.isin(keys, src[~ins] * n + dst[~ins])]
    allk = np.concatenate([keep, src[ins] * n + dst[ins]])
    return directed_from_arcs(n, allk // n, allk % n, g.name + "+batch")


def workload(name: str) -> Graph:
    """The named synthetic workloads (sizes as in the measurement plan)."""
    if name == "er16k":
        return erdos_renyi(16384, 131072, SEED_BASE + 0)
    if name.startswith("rmat"):
        scale = int(name[4:])
        return rmat(scale, 16, seed=SEED_BASE + scale)
    if name.startswith("chunglu"):  # chunglu27: the large workload; smaller scales for profiling
        scale = int(name[7:])
        return chung_lu(1 << scale, 16.0, 2.1, SEED_BASE + scale)
    raise KeyError(name)
