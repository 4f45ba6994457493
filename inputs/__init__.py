"""Seeded synthetic graph inputs shared by the CPU oracle, the tests and the bench.

This module generates inputs only: R-MAT and Erdos-Renyi edge streams, CSR/CSC
assembly (duplicates removed, rows sorted), the symmetric edge-weight draw and a
few hand-shaped graphs. It holds none of the vertex-centric method's arithmetic.

The heavy lifting is in ``graphgen.c`` (compiled on first use with gcc; OpenMP
when available). Random numbers are counter based (SplitMix64 output function),
so every array depends only on the seed and the sizes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB_PATH = os.path.join(_HERE, "libgraphgen.so")
_lib = None
_lock = threading.Lock()

U32 = ctypes.POINTER(ctypes.c_uint32)
U64 = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile graphgen.c into libgraphgen.so (OpenMP if the compiler has it)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O3", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.gg_rmat_edges.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_uint64, U32, U32]
            lib.gg_er_edges.argtypes = [ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint64, U32, U32]
            lib.gg_pack_keys.argtypes = [ctypes.c_int64, U32, U32, ctypes.c_int, U64]
            lib.gg_pack_keys.restype = ctypes.c_int64
            lib.gg_radix_sort64.argtypes = [U64, U64, ctypes.c_int64]
            lib.gg_unique_sorted.argtypes = [U64, ctypes.c_int64]
            lib.gg_unique_sorted.restype = ctypes.c_int64
            lib.gg_keys_to_csr.argtypes = [ctypes.c_uint32, U64, ctypes.c_int64, U32, U32]
            lib.gg_transpose.argtypes = [ctypes.c_uint32, U32, U32, U32, U32, U32, U32, U32]
            lib.gg_sym_weights.argtypes = [ctypes.c_uint32, U32, U32, ctypes.c_uint64, U32]
            lib.gg_uniform_vertices.argtypes = [ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint64, U32]
            lib.gg_loguniform.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_uint64, U32]
            lib.gg_random_keys.argtypes = [ctypes.c_int64, ctypes.c_uint64, U64]
            lib.gg_random_keys.restype = None
            lib.gg_mix64.argtypes = [ctypes.c_uint64]
            lib.gg_mix64.restype = ctypes.c_uint64
            lib.gg_num_threads.restype = ctypes.c_int
            _lib = lib
        return _lib


def _p32(a):
    return a.ctypes.data_as(U32) if a is not None else None


def _p64(a):
    return a.ctypes.data_as(U64)


@dataclass
class Graph:
    """A directed graph in CSR (out-edges) and CSC (in-edges), uint32 everywhere.

    ``w``/``wt`` are per-edge weights in CSR / CSC order (None when unweighted).
    For a symmetric graph the CSC arrays are the CSR arrays themselves.
    """
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    t_ptr: np.ndarray
    t_idx: np.ndarray
    w: np.ndarray | None = None
    wt: np.ndarray | None = None
    symmetric: bool = False
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.row_ptr[-1])

    def out_degree(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))

    def in_degree(self) -> np.ndarray:
        return np.diff(self.t_ptr.astype(np.int64))

    def edges(self):
        """(src, dst) arrays in CSR order."""
        src = np.repeat(np.arange(self.n, dtype=np.uint32), self.out_degree())
        return src, self.col


def rmat_edges(scale: int, m: int, a=0.57, b=0.19, c=0.19, seed=1):
    src = np.empty(m, np.uint32)
    dst = np.empty(m, np.uint32)
    _L().gg_rmat_edges(scale, m, a, b, c, seed, _p32(src), _p32(dst))
    return src, dst


def er_edges(n: int, m: int, seed=1):
    src = np.empty(m, np.uint32)
    dst = np.empty(m, np.uint32)
    _L().gg_er_edges(n, m, seed, _p32(src), _p32(dst))
    return src, dst


def from_edges(n: int, src, dst, symmetrize=False, weighted=False, wseed=1, name="") -> Graph:
    """Assemble a Graph from an edge list: (symmetrise), sort, remove duplicates."""
    src = np.ascontiguousarray(src, dtype=np.uint32)
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    m = src.shape[0]
    if m and (int(src.max()) >= n or int(dst.max()) >= n):
        raise ValueError("edge endpoint out of range")
    L = _L()
    nk = 2 * m if symmetrize else m
    keys = np.empty(max(nk, 1), np.uint64)
    L.gg_pack_keys(m, _p32(src), _p32(dst), int(bool(symmetrize)), _p64(keys))
    tmp = np.empty(max(nk, 1), np.uint64)
    L.gg_radix_sort64(_p64(keys), _p64(tmp), nk)
    del tmp
    e = L.gg_unique_sorted(_p64(keys), nk)
    if e >= 2**32:
        raise ValueError("more than 2^32-1 edges")
    row_ptr = np.empty(n + 1, np.uint32)
    col = np.empty(max(e, 1), np.uint32)
    L.gg_keys_to_csr(n, _p64(keys), e, _p32(row_ptr), _p32(col))
    del keys
    col = col[:e]
    w = None
    if weighted:
        w = np.empty(max(e, 1), np.uint32)
        L.gg_sym_weights(n, _p32(row_ptr), _p32(col), wseed, _p32(w))
        w = w[:e]
    if symmetrize:
        return Graph(n, row_ptr, col, row_ptr, col, w, w, True, name)
    t_ptr, t_idx, wt = transpose(n, row_ptr, col, w)
    return Graph(n, row_ptr, col, t_ptr, t_idx, w, wt, False, name)


def transpose(n, row_ptr, col, w=None):
    """Stable transposition: in-lists with sources in increasing order."""
    e = int(row_ptr[-1])
    t_ptr = np.empty(n + 1, np.uint32)
    t_idx = np.empty(max(e, 1), np.uint32)
    t_w = np.empty(max(e, 1), np.uint32) if w is not None else None
    cursor = np.empty(max(n, 1), np.uint32)
    col = np.ascontiguousarray(col, dtype=np.uint32)
    if e == 0:
        col = np.zeros(1, np.uint32)
    _L().gg_transpose(n, _p32(row_ptr), _p32(col), _p32(w) if w is not None and e else None,
                      _p32(t_ptr), _p32(t_idx), _p32(t_w) if t_w is not None else None, _p32(cursor))
    return t_ptr, t_idx[:e], (t_w[:e] if t_w is not None else None)


def random_permutation(n: int, seed: int) -> np.ndarray:
    """Seeded uniform random permutation of [0, n): the order that sorts the items'
    counter-based keys (gg_random_keys); the same on every machine."""
    keys = np.empty(max(n, 1), np.uint64)
    _L().gg_random_keys(n, seed, _p64(keys))
    return np.argsort(keys[:n], kind="stable").astype(np.uint32)


def rmat_graph(scale: int, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=1, symmetrize=False,
               weighted=False, wseed=None, permute_seed=None) -> Graph:
    """R-MAT graph: n = 2^scale, edge_factor * n drawn edges, duplicates removed.
    permute_seed: relabel vertex v as perm[v] (random_permutation(n, permute_seed))
    before assembly, so the high-degree vertices are not the low ids."""
    n = 1 << scale
    src, dst = rmat_edges(scale, edge_factor * n, a, b, c, seed)
    if permute_seed is not None:
        perm = random_permutation(n, permute_seed)
        src, dst = perm[src], perm[dst]
    g = from_edges(n, src, dst, symmetrize, weighted, seed if wseed is None else wseed,
                   name=f"rmat{scale}{'s' if symmetrize else ''}{'p' if permute_seed is not None else ''}")
    g.meta.update(kind="rmat", scale=scale, edge_factor=edge_factor, a=a, b=b, c=c, seed=seed,
                  permute_seed=permute_seed)
    return g


def rmat_sized(n: int, edge_factor=8, a=0.57, b=0.19, c=0.19, seed=1, symmetrize=True) -> Graph:
    """R-MAT graph on exactly n vertices: edge_factor * n draws at scale ceil(log2 n),
    keeping the draws whose endpoints are both below n."""
    scale = max(1, int(np.ceil(np.log2(max(n, 2)))))
    src, dst = rmat_edges(scale, edge_factor * n, a, b, c, seed)
    keep = (src < n) & (dst < n)
    g = from_edges(n, src[keep], dst[keep], symmetrize, name=f"rmat_n{n}")
    g.meta.update(kind="rmat_sized", n=n, edge_factor=edge_factor, seed=seed)
    return g


def hashmin_instances(k=1000, lo=1000, hi=100000, edge_factor=8, seed=1):
    """k R-MAT instances with log-uniform sizes in [lo, hi], symmetrised, seeds seed..seed+k-1."""
    sizes = loguniform_ints(k, lo, hi, seed=seed)
    return [rmat_sized(int(n), edge_factor, seed=seed + i) for i, n in enumerate(sizes)]


def er_graph(n: int, m: int, seed=1, symmetrize=False, weighted=False, wseed=None) -> Graph:
    src, dst = er_edges(n, m, seed)
    g = from_edges(n, src, dst, symmetrize, weighted, seed if wseed is None else wseed, name=f"er{n}")
    g.meta.update(kind="er", seed=seed)
    return g


def uniform_vertices(n: int, k: int, seed=1) -> np.ndarray:
    out = np.empty(max(k, 1), np.uint32)
    _L().gg_uniform_vertices(n, k, seed, _p32(out))
    return out[:k]


def loguniform_ints(k: int, lo: float, hi: float, seed=1) -> np.ndarray:
    out = np.empty(max(k, 1), np.uint32)
    _L().gg_loguniform(k, lo, hi, seed, _p32(out))
    return out[:k]


# ---------------------------------------------------------------- hand-shaped graphs
def directed_cycle(n: int) -> Graph:
    src = np.arange(n, dtype=np.uint32)
    return from_edges(n, src, (src + 1) % n, name=f"cycle{n}")


def complete_digraph(n: int) -> Graph:
    s, d = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    mask = s != d
    return from_edges(n, s[mask], d[mask], name=f"complete{n}")


def star(k: int, symmetric=True) -> Graph:
    """Centre 0 plus leaves 1..k."""
    leaves = np.arange(1, k + 1, dtype=np.uint32)
    centre = np.zeros(k, np.uint32)
    return from_edges(k + 1, centre, leaves, symmetrize=symmetric, name=f"star{k}")


def path(n: int, symmetric=True, weighted=False, wseed=1) -> Graph:
    s = np.arange(n - 1, dtype=np.uint32)
    return from_edges(n, s, s + 1, symmetrize=symmetric, weighted=weighted, wseed=wseed, name=f"path{n}")


def empty_graph(n: int) -> Graph:
    z = np.zeros(0, np.uint32)
    return from_edges(n, z, z, name=f"empty{n}")


def block_diagonal(graphs) -> tuple[Graph, np.ndarray]:
    """Disjoint union of graphs, vertex ranges concatenated in order.

    Returns the union and the vertex offsets (k+1 entries)."""
    offs = np.zeros(len(graphs) + 1, np.int64)
    for i, g in enumerate(graphs):
        offs[i + 1] = offs[i] + g.n
    n = int(offs[-1])
    m = sum(g.m for g in graphs)
    if m >= 2**32 or n >= 2**32:
        raise ValueError("union too large for uint32 indices")

    def cat(ptr_name, idx_name, w_name):
        ptr = np.empty(n + 1, np.uint32)
        idx = np.empty(m, np.uint32)
        w = np.empty(m, np.uint32) if all(getattr(g, w_name) is not None for g in graphs) else None
        e0 = 0
        for i, g in enumerate(graphs):
            p = getattr(g, ptr_name)
            ptr[offs[i]:offs[i + 1]] = p[:-1] + e0
            idx[e0:e0 + g.m] = getattr(g, idx_name) + np.uint32(offs[i])
            if w is not None:
                w[e0:e0 + g.m] = getattr(g, w_name)
            e0 += g.m
        ptr[n] = e0
        return ptr, idx, w

    row_ptr, col, w = cat("row_ptr", "col", "w")
    sym = all(g.symmetric for g in graphs)
    if sym:
        t_ptr, t_idx, wt = row_ptr, col, w
    else:
        t_ptr, t_idx, wt = cat("t_ptr", "t_idx", "wt")
    return Graph(n, row_ptr, col, t_ptr, t_idx, w, wt, sym, "block_diagonal"), offs


def num_threads() -> int:
    return int(_L().gg_num_threads())
