"""CPU oracle — TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct CPU implementations of what the GPU library
computes, used by the tests, the smoke check and the benchmark's CPU-baseline
leg, and by nothing else. The GPU product path never imports this package.

* ``pregel.c`` — a single-threaded synchronous Pregel engine (Section 4.2,
  Fig. 3; vertex selection of Section 4.3.1; combined one-slot mailboxes of
  Section 4.3.3) running PageRank (Fig. 8 with the Pregel constant of
  Fig. 12), Hashmin (Fig. 9) and weighted SSSP (Fig. 10 with per-edge
  weights). PageRank runs in FP64.
* ``pagerank_update`` — compute() of Fig. 8 for chosen vertices in one superstep,
  from the ranks of the superstep before (FP64 numpy): checks a single superstep
  of a run too large for the full oracle, one vertex at a time.
  ``pagerank_superstep`` is the same update for a range of vertices in C, used
  to check and to time one superstep of a billion-edge graph;
  ``hashmin_superstep`` is one Hashmin superstep (Fig. 9) in the same form.
* PageRank to convergence (``pagerank(..., tolerance=eps)``): the run ends after
  the first superstep whose L1 rank change is below eps.
* ``reliability`` — the most reliable path (an application the paper does not
  have, the GPU library's example of its vertex-program interface) in the same
  engine: FP32 products of edge probabilities, max combiner.
* ``mlp.py`` — FP64 forward/backward of the 8-32-32-3 mode-selector MLP.

The compiled part is built on first use with gcc (``build()``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pregel.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()
INF = 0xFFFFFFFF

U32 = ctypes.POINTER(ctypes.c_uint32)
U64 = ctypes.POINTER(ctypes.c_uint64)
F64 = ctypes.POINTER(ctypes.c_double)


class _Stats(ctypes.Structure):
    _fields_ = [("supersteps", ctypes.c_uint32), ("halted", ctypes.c_int32), ("cap", ctypes.c_uint32),
                ("active", U32), ("broadcasters", U32), ("messages", U64), ("delta", F64)]


def build(force: bool = False) -> str:
    """Compile pregel.c into liboracle.so (single-threaded, -O2)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"], check=True,
                   capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            st = ctypes.POINTER(_Stats)
            lib.oracle_pagerank.argtypes = [ctypes.c_uint32, U32, U32, ctypes.c_uint32, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_uint32, F64, st]
            lib.oracle_pagerank_superstep.argtypes = [ctypes.c_uint32, U32, U32, U32, F64, ctypes.c_double,
                                                      ctypes.c_uint32, ctypes.c_uint32, F64]
            lib.oracle_pagerank_superstep.restype = None
            U8 = ctypes.POINTER(ctypes.c_uint8)
            lib.oracle_hashmin_superstep.argtypes = [ctypes.c_uint32, U32, U32, U32, U8, ctypes.c_uint32,
                                                     ctypes.c_uint32, U32, U8]
            lib.oracle_hashmin_superstep.restype = None
            lib.oracle_hashmin.argtypes = [ctypes.c_uint32, U32, U32, ctypes.c_uint32, U32, st]
            lib.oracle_sssp.argtypes = [ctypes.c_uint32, U32, U32, U32, ctypes.c_uint32, ctypes.c_uint32, U32, st]
            lib.oracle_reliability.argtypes = [ctypes.c_uint32, U32, U32, U32, ctypes.c_uint32, ctypes.c_uint32,
                                               ctypes.POINTER(ctypes.c_float), st]
            for f in (lib.oracle_pagerank, lib.oracle_hashmin, lib.oracle_sssp, lib.oracle_reliability):
                f.restype = ctypes.c_int
            _lib = lib
        return _lib


def _u32(a):
    a = np.ascontiguousarray(a, dtype=np.uint32)
    if a.size == 0:
        a = np.zeros(1, np.uint32)
    return a


def _stats(cap):
    act = np.zeros(max(cap, 1), np.uint32)
    bc = np.zeros(max(cap, 1), np.uint32)
    msg = np.zeros(max(cap, 1), np.uint64)
    dl = np.zeros(max(cap, 1), np.float64)
    s = _Stats(0, 0, cap, act.ctypes.data_as(U32), bc.ctypes.data_as(U32), msg.ctypes.data_as(U64),
               dl.ctypes.data_as(F64))
    return s, (act, bc, msg, dl)


def _finish(r, s, arrs):
    if r < 0:
        raise MemoryError("oracle allocation failed")
    n = min(s.supersteps, s.cap)
    act, bc, msg, dl = arrs
    return dict(supersteps=int(s.supersteps), halted=bool(s.halted), active=act[:n].copy(),
                broadcasters=bc[:n].copy(), messages=msg[:n].copy(), delta=dl[:n].copy())


def pagerank(n, row_ptr, col, T=30, damping=0.85, max_supersteps=None, stats_cap=None, tolerance=0.0):
    """FP64 synchronous-Pregel PageRank (Fig. 8). Returns (rank[n] float64, stats).

    tolerance > 0: PageRank to convergence — the run also ends after the first
    superstep s >= 1 whose L1 change sum_v |r_s(v) - r_(s-1)(v)| (stats["delta"][s])
    is below tolerance; T still bounds the run."""
    if max_supersteps is None:
        max_supersteps = T + 1
    cap = max_supersteps if stats_cap is None else stats_cap
    out = np.zeros(max(n, 1), np.float64)
    s, arrs = _stats(cap)
    r = _L().oracle_pagerank(n, _u32(row_ptr).ctypes.data_as(U32), _u32(col).ctypes.data_as(U32), T,
                             float(damping), float(tolerance), max_supersteps, out.ctypes.data_as(F64),
                             ctypes.byref(s))
    return out[:n], _finish(r, s, arrs)


def pagerank_superstep(n, in_ptr, in_src, out_degree, prev_rank, damping=0.85, v_begin=0, v_end=None):
    """One superstep s >= 1 of PageRank (Fig. 8) for the vertices [v_begin, v_end),
    in C (pregel.c, oracle_pagerank_superstep): the same definition as
    pagerank_update, fast enough to check or time a billion-edge superstep.
    in_ptr/in_src: in-edge arrays (uint32); out_degree: uint32; prev_rank: float64.
    Returns rank[v_end - v_begin] float64."""
    v_end = n if v_end is None else v_end
    ip, isrc = _u32(in_ptr), _u32(in_src)
    od = _u32(out_degree)
    prev = np.ascontiguousarray(prev_rank, dtype=np.float64)
    out = np.empty(max(v_end - v_begin, 1), np.float64)
    _L().oracle_pagerank_superstep(n, ip.ctypes.data_as(U32), isrc.ctypes.data_as(U32), od.ctypes.data_as(U32),
                                   prev.ctypes.data_as(F64), float(damping), int(v_begin), int(v_end),
                                   out.ctypes.data_as(F64))
    return out[:v_end - v_begin]


def hashmin_superstep(n, in_ptr, in_src, prev_label, bcast, v_begin=0, v_end=None, with_recv=False):
    """One superstep s >= 1 of Hashmin (Fig. 9) for the vertices [v_begin, v_end),
    in C, from the receiving side: bcast[u] (uint8) marks the vertices that broadcast
    prev_label[u] in superstep s-1. Returns the new labels (and, with with_recv,
    which vertices received a message)."""
    v_end = n if v_end is None else v_end
    ip, isrc, pl = _u32(in_ptr), _u32(in_src), _u32(prev_label)
    bc = np.ascontiguousarray(bcast, dtype=np.uint8)
    out = np.empty(max(v_end - v_begin, 1), np.uint32)
    rc = np.empty(max(v_end - v_begin, 1), np.uint8)
    U8 = ctypes.POINTER(ctypes.c_uint8)
    _L().oracle_hashmin_superstep(n, ip.ctypes.data_as(U32), isrc.ctypes.data_as(U32), pl.ctypes.data_as(U32),
                                  bc.ctypes.data_as(U8), int(v_begin), int(v_end), out.ctypes.data_as(U32),
                                  rc.ctypes.data_as(U8))
    k = v_end - v_begin
    return (out[:k], rc[:k].astype(bool)) if with_recv else out[:k]


def hashmin(n, row_ptr, col, max_supersteps=1 << 30, stats_cap=4096):
    """Hashmin labels (Fig. 9). Returns (label[n] uint32, stats)."""
    out = np.zeros(max(n, 1), np.uint32)
    s, arrs = _stats(stats_cap)
    rp, c = _u32(row_ptr), _u32(col)
    r = _L().oracle_hashmin(n, rp.ctypes.data_as(U32), c.ctypes.data_as(U32), max_supersteps,
                            out.ctypes.data_as(U32), ctypes.byref(s))
    return out[:n], _finish(r, s, arrs)


def sssp(n, row_ptr, col, w=None, source=0, max_supersteps=1 << 30, stats_cap=4096):
    """SSSP distances (Fig. 10, message = value + w(u,v), INF = 0xFFFFFFFF). Returns (dist, stats)."""
    out = np.zeros(max(n, 1), np.uint32)
    s, arrs = _stats(stats_cap)
    rp, c = _u32(row_ptr), _u32(col)
    wp = _u32(w).ctypes.data_as(U32) if w is not None else None
    r = _L().oracle_sssp(n, rp.ctypes.data_as(U32), c.ctypes.data_as(U32), wp, source, max_supersteps,
                         out.ctypes.data_as(U32), ctypes.byref(s))
    return out[:n], _finish(r, s, arrs)


def reliability(n, row_ptr, col, w=None, source=0, max_supersteps=1 << 30, stats_cap=4096):
    """Most reliable path (not in the paper): FP32 value = the largest product of
    edge probabilities w/256 over the paths from source (1/256 per edge without
    weights), products taken along the path from the source; 0 where unreachable.
    Returns (value[n] float32, stats)."""
    out = np.zeros(max(n, 1), np.float32)
    s, arrs = _stats(stats_cap)
    rp, c = _u32(row_ptr), _u32(col)
    wp = _u32(w).ctypes.data_as(U32) if w is not None else None
    r = _L().oracle_reliability(n, rp.ctypes.data_as(U32), c.ctypes.data_as(U32), wp, source, max_supersteps,
                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(s))
    return out[:n], _finish(r, s, arrs)


def run_app(app: str, g, **kw):
    """Dispatch on an app name for a graph object with row_ptr/col/w/n."""
    if app == "pagerank":
        return pagerank(g.n, g.row_ptr, g.col, **kw)
    if app == "hashmin":
        return hashmin(g.n, g.row_ptr, g.col, **kw)
    if app == "sssp":
        return sssp(g.n, g.row_ptr, g.col, g.w, **kw)
    if app == "reliability":
        return reliability(g.n, g.row_ptr, g.col, g.w, **kw)
    raise ValueError(app)


def batch_sssp(g, sources, **kw):
    """Independent SSSP runs, one per source: dist[k, n] (source-major)."""
    return np.stack([sssp(g.n, g.row_ptr, g.col, g.w, int(s), **kw)[0] for s in sources]) if len(sources) \
        else np.zeros((0, g.n), np.uint32)


def batch_hashmin(graphs):
    """Hashmin on each graph separately: list of label arrays (local vertex IDs)."""
    return [hashmin(h.n, h.row_ptr, h.col)[0] for h in graphs]


def pagerank_update(vertices, n, in_ptr, in_src, out_degree, prev_rank, damping=0.85):
    """One superstep s >= 1 of PageRank (Fig. 8) for the given vertices: every
    in-neighbour u broadcast prev_rank[u] / out_degree[u] in superstep s - 1 (Fig.
    8 sends rank / number of out-neighbours), and the vertex takes (1 - d)/N (the
    constant of Fig. 12) plus d times the sum of what it received. in_ptr/in_src
    are the in-edge (transposed) arrays. FP64; returns rank[len(vertices)]."""
    prev = np.asarray(prev_rank, np.float64)
    deg = np.asarray(out_degree, np.float64)
    out = np.empty(len(vertices), np.float64)
    for i, v in enumerate(vertices):
        us = np.asarray(in_src[int(in_ptr[v]):int(in_ptr[v + 1])], np.int64)
        out[i] = (1.0 - damping) / n + damping * float(np.sum(prev[us] / deg[us]))
    return out
