"""Python binding of libipregel_gb300.so (the C ABI declared in include/ipregel.h).

Argument marshalling only: every superstep runs in the library's CUDA kernels.
Arrays may be numpy arrays (host memory) or CUDA torch tensors (device memory);
PyTorch supplies device memory and streams, nothing else. There is no CPU
fallback: if the compiled library is missing, importing a handle raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

IP_OK = 0
IP_E_INVAL = -1
IP_E_RANGE = -2
IP_E_NOMEM = -3
IP_E_CUDA = -4
IP_E_TIMEOUT = -5
IP_E_MAXSTEPS = -6
IP_E_DEVICE_ASSERT = -7
IP_E_STATE = -8

PAGERANK, HASHMIN, SSSP, RELIABILITY = 0, 1, 2, 3
APPS = {"pagerank": PAGERANK, "hashmin": HASHMIN, "sssp": SSSP, "reliability": RELIABILITY}
FLOAT_APPS = ("pagerank", "reliability")
PUSH_SPARSE, PUSH_DENSE, PULL = 0, 1, 2
MODES = {"push_sparse": PUSH_SPARSE, "push_dense": PUSH_DENSE, "pull": PULL}
PR_ENGINES = {"auto": 0, "gather": 1, "blocked": 2}
POLICY_AUTO, POLICY_THRESHOLD, POLICY_MLP, POLICY_FORCED, POLICY_SEQUENCE = 0, 1, 2, 3, 4
SELECTOR_BYTES = 16 * 4 + (32 * 8 + 32 * 32 + 3 * 32) * 2 + (32 + 32 + 3) * 4
N_FEATURES = 8
INF = 0xFFFFFFFF

_U32P = ctypes.POINTER(ctypes.c_uint32)


class IPError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class Options(ctypes.Structure):
    _fields_ = [("damping", ctypes.c_float), ("pr_iterations", ctypes.c_uint32), ("source", ctypes.c_uint32),
                ("policy", ctypes.c_int32), ("forced_mode", ctypes.c_int32),
                ("mode_sequence", ctypes.POINTER(ctypes.c_uint8)), ("mode_sequence_len", ctypes.c_uint32),
                ("t1", ctypes.c_uint32), ("t2", ctypes.c_uint32), ("thr_sparse", ctypes.c_float),
                ("thr_pull", ctypes.c_float), ("use_graph", ctypes.c_int32), ("collect_labels", ctypes.c_int32),
                ("profile_kernels", ctypes.c_int32), ("stream", ctypes.c_void_p), ("pr_engine", ctypes.c_int32),
                ("pr_tolerance", ctypes.c_float), ("pull_early_exit", ctypes.c_int32)]


class RunStatsC(ctypes.Structure):
    _fields_ = [("supersteps", ctypes.c_uint32), ("halted", ctypes.c_int32), ("capacity", ctypes.c_uint32),
                ("mode", ctypes.POINTER(ctypes.c_uint8)), ("active", _U32P), ("broadcasters", _U32P),
                ("messages", ctypes.POINTER(ctypes.c_uint64)), ("features", ctypes.POINTER(ctypes.c_float)),
                ("mode_ms", ctypes.POINTER(ctypes.c_float)), ("kernel_ms", ctypes.POINTER(ctypes.c_float)),
                ("elapsed_ms", ctypes.c_float), ("pr_delta", ctypes.POINTER(ctypes.c_float))]


class BatchStatsC(ctypes.Structure):
    _fields_ = [("supersteps", ctypes.c_uint32), ("halted", ctypes.c_int32), ("messages", ctypes.c_uint64),
                ("instance_supersteps", _U32P), ("elapsed_ms", ctypes.c_float),
                ("barrier_timeout_ns", ctypes.c_uint64), ("engine", ctypes.c_int32)]


class GraphInfo(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_uint32), ("n_edges", ctypes.c_uint64), ("max_out_degree", ctypes.c_uint32),
                ("max_in_degree", ctypes.c_uint32), ("csc_is_csr", ctypes.c_uint32), ("weighted", ctypes.c_uint32),
                ("num_sms", ctypes.c_uint32), ("device_bytes", ctypes.c_uint64), ("bytes_graph", ctypes.c_uint64),
                ("bytes_vertex_state", ctypes.c_uint64), ("bytes_degree_bins", ctypes.c_uint64),
                ("bytes_blocked_layout", ctypes.c_uint64), ("bytes_renumbering", ctypes.c_uint64),
                ("bytes_other", ctypes.c_uint64)]


_lib = None

# every symbol include/ipregel.h declares
EXPORTS = ("ip_options_default", "ip_release_cached_memory", "ip_graph_create", "ip_graph_destroy", "ip_graph_info", "ip_run", "ip_get_values",
           "ip_set_selector", "ip_strerror", "ip_hashmin_noalloc", "ip_mlp_workspace_bytes", "ip_mlp_forward",
           "ip_mlp_backward", "ip_mlp_adam", "ip_mlp_pack", "ip_run_batch_sssp", "ip_run_batch_hashmin", "ip_graph_relabel")
BATCH_MAX_SOURCES = 256
MLP_PARAMS = 32 * 8 + 32 + 32 * 32 + 32 + 3 * 32 + 3
NOALLOC_MAX_VERTICES = 1 << 20
RELABEL_AUTO_EDGES = 1 << 20  # graphs this large are renumbered by degree class unless asked otherwise
CREATE_DEVICE_PTRS, CREATE_RELABEL = 1, 2


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the shared library (building it first if asked and it is missing/stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"{_build.LIB} is missing: run __graft_entry__.build()")
    L = ctypes.CDLL(_build.LIB)
    vp = ctypes.c_void_p
    L.ip_options_default.argtypes = [ctypes.POINTER(Options)]
    L.ip_options_default.restype = None
    L.ip_graph_create.argtypes = [ctypes.POINTER(vp), ctypes.c_uint32, ctypes.c_uint64, vp, vp, vp, vp, vp, vp,
                                  ctypes.c_int, vp]
    L.ip_graph_destroy.argtypes = [vp]
    L.ip_graph_destroy.restype = None
    L.ip_graph_info.argtypes = [vp, ctypes.POINTER(GraphInfo)]
    L.ip_graph_relabel.argtypes = [vp, vp]
    L.ip_run.argtypes = [vp, ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(Options), ctypes.POINTER(RunStatsC)]
    L.ip_get_values.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_int, vp]
    L.ip_set_selector.argtypes = [vp, vp, ctypes.c_size_t]
    L.ip_hashmin_noalloc.argtypes = [ctypes.c_uint32, ctypes.c_uint64, vp, vp, vp, ctypes.c_uint32,
                                     ctypes.POINTER(ctypes.c_uint32), vp]
    L.ip_hashmin_noalloc.restype = ctypes.c_int
    L.ip_mlp_workspace_bytes.argtypes = []
    L.ip_mlp_workspace_bytes.restype = ctypes.c_size_t
    L.ip_mlp_forward.argtypes = [vp, vp, vp, ctypes.c_uint32, vp, vp]
    L.ip_mlp_backward.argtypes = [vp, vp, vp, vp, vp, ctypes.c_uint32, ctypes.c_float, vp, vp, vp, ctypes.c_size_t,
                                  vp]
    L.ip_mlp_adam.argtypes = [vp, vp, vp, vp, ctypes.c_uint32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                              ctypes.c_float, ctypes.c_uint32, vp]
    L.ip_mlp_pack.argtypes = [vp, vp, vp, vp]
    for name in ("ip_mlp_forward", "ip_mlp_backward", "ip_mlp_adam", "ip_mlp_pack"):
        getattr(L, name).restype = ctypes.c_int
    bs = ctypes.POINTER(BatchStatsC)
    L.ip_run_batch_sssp.argtypes = [vp, _U32P, ctypes.c_uint32, vp, ctypes.c_int, ctypes.c_uint32, bs, vp]
    L.ip_run_batch_hashmin.argtypes = [vp, _U32P, ctypes.c_uint32, vp, ctypes.c_int, ctypes.c_uint32, bs, vp]
    L.ip_run_batch_sssp.restype = ctypes.c_int
    L.ip_run_batch_hashmin.restype = ctypes.c_int
    L.ip_strerror.argtypes = [ctypes.c_int]
    L.ip_strerror.restype = ctypes.c_char_p
    L.ip_release_cached_memory.argtypes = []
    L.ip_release_cached_memory.restype = ctypes.c_int
    for name in ("ip_graph_create", "ip_graph_info", "ip_run", "ip_get_values", "ip_set_selector"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def strerror(code: int) -> str:
    try:
        return load().ip_strerror(code).decode()
    except Exception:  # library not loadable: still describe the code
        return {0: "ok"}.get(code, f"error {code}")


def _check(code, where):
    if code != IP_OK:
        raise IPError(code, where)


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a):
    """(pointer, is_device, keepalive) for a numpy array or torch tensor (uint32)."""
    if a is None:
        return None, None, None
    if _is_torch(a):
        import torch
        if a.dtype not in (torch.int32, torch.uint32) and str(a.dtype) != "torch.uint32":
            raise TypeError("uint32/int32 tensor expected")
        if not a.is_contiguous():
            raise ValueError("contiguous tensor expected")
        return a.data_ptr(), a.is_cuda, a
    arr = np.ascontiguousarray(a, dtype=np.uint32)
    return arr.ctypes.data, False, arr


_TUNED = None


def tuned_defaults() -> dict:
    """Per-app cutoffs written by the autotuner (tuned_defaults.json), or {}."""
    global _TUNED
    if _TUNED is None:
        import json
        p = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_defaults.json")
        _TUNED = json.load(open(p)) if os.path.exists(p) else {}
    return _TUNED


def release_cached_memory():
    """Frees the device buffers the library keeps cached from destroyed graphs."""
    _check(load().ip_release_cached_memory(), "ip_release_cached_memory")


def default_options(app=None, relabeled=True, **kw) -> Options:
    """Options with the library defaults, the autotuned cutoffs for `app` (tuned on
    graphs renumbered by degree class, or in the caller's order when relabeled is
    False: the best cutoffs differ), then kw."""
    o = Options()
    load().ip_options_default(ctypes.byref(o))
    t = tuned_defaults()
    bins = t.get("bins", {}) if relabeled else t.get("bins_caller_order", t.get("bins", {}))
    if app is not None and app in bins:
        o.t1, o.t2 = bins[app]["t1"], bins[app]["t2"]
    if "modes" in t:
        o.thr_sparse, o.thr_pull = t["modes"]["thr_sparse"], t["modes"]["thr_pull"]
    seq = kw.pop("mode_sequence", None)
    for k, v in kw.items():
        if k == "policy" and isinstance(v, str):
            v = {"auto": POLICY_AUTO, "threshold": POLICY_THRESHOLD, "mlp": POLICY_MLP, "forced": POLICY_FORCED,
                 "sequence": POLICY_SEQUENCE}[v]
        if k == "forced_mode" and isinstance(v, str):
            v = MODES[v]
        if k == "pr_engine" and isinstance(v, str):
            v = PR_ENGINES[v]
        if k == "stream" and v is not None and not isinstance(v, int):
            v = v.cuda_stream  # torch.cuda.Stream
        setattr(o, k, v)
    # a cutoff given alone keeps the tuned other one only where the pair stays ordered (t1 < t2)
    if "t2" in kw and "t1" not in kw and o.t2 and o.t1 >= o.t2:
        o.t1 = o.t2 - 1
    if "t1" in kw and "t2" not in kw and o.t1 and o.t2 and o.t2 <= o.t1:
        o.t2 = o.t1 + 1
    if seq is not None:
        buf = (ctypes.c_uint8 * len(seq))(*[MODES[m] if isinstance(m, str) else int(m) for m in seq])
        o.mode_sequence = ctypes.cast(buf, ctypes.POINTER(ctypes.c_uint8))
        o.mode_sequence_len = len(seq)
        o._seq_keepalive = buf
        if "policy" not in kw:
            o.policy = POLICY_SEQUENCE
    return o


@dataclass
class RunStats:
    code: int
    supersteps: int
    halted: bool
    elapsed_ms: float
    mode: np.ndarray
    active: np.ndarray
    broadcasters: np.ndarray
    messages: np.ndarray
    features: np.ndarray
    mode_ms: np.ndarray
    kernel_ms: np.ndarray
    pr_delta: np.ndarray


class Graph:
    """A graph resident on the current CUDA device (owns its device memory)."""

    def __init__(self, n, csr_offsets, csr_cols, csr_weights=None, csc_offsets=None, csc_rows=None,
                 csc_weights=None, symmetric=False, stream=None, selector="default", relabel="auto"):
        """selector: "default" loads the trained selector shipped with the package
        (if present), None loads nothing, bytes load that blob.
        relabel: True renumbers the vertices inside the handle by degree class
        (ip_graph_relabel; results keep the caller's numbering), False keeps the
        given numbering, "auto" renumbers graphs of at least RELABEL_AUTO_EDGES edges."""
        L = load()
        self._h = ctypes.c_void_p()
        arrays = [csr_offsets, csr_cols, csr_weights, csc_offsets, csc_rows, csc_weights]
        ptrs = [_ptr(a) for a in arrays]
        dev = {p[1] for p in ptrs if p[0] is not None}
        if len(dev) > 1:
            raise ValueError("mix of host and device arrays")
        device_ptrs = int(dev == {True})
        p = [x[0] for x in ptrs]
        if symmetric:  # declare the CSC to be the CSR itself
            p[3], p[4], p[5] = p[0], p[1], p[2]
        m = int(len(csr_cols)) if csr_cols is not None else 0
        self.n = int(n)
        self.m = m
        st = _stream_handle(stream)
        if relabel == "auto":
            relabel = m >= RELABEL_AUTO_EDGES
        flags = device_ptrs | (CREATE_RELABEL if relabel else 0)  # renumbered during creation
        _check(L.ip_graph_create(ctypes.byref(self._h), self.n, m, *p, flags, st), "ip_graph_create")
        self._keep = None  # the library copied everything
        self.relabeled = bool(relabel)
        if selector == "default":
            from .selector import load_default_blob
            selector = load_default_blob()
        if selector is not None:
            self.set_selector(selector)

    @classmethod
    def from_inputs(cls, g, stream=None, build_csc_on_device=False, selector="default", relabel="auto"):
        """From an inputs.Graph (host numpy arrays)."""
        kw = dict(stream=stream, selector=selector, relabel=relabel)
        if g.symmetric:
            return cls(g.n, g.row_ptr, g.col, g.w, symmetric=True, **kw)
        if build_csc_on_device:
            return cls(g.n, g.row_ptr, g.col, g.w, **kw)
        return cls(g.n, g.row_ptr, g.col, g.w, g.t_ptr, g.t_idx, g.wt, **kw)

    def relabel(self, stream=None):
        """Renumber the vertices inside the handle by degree class (ip_graph_relabel)."""
        _check(load().ip_graph_relabel(self._h, _stream_handle(stream)), "ip_graph_relabel")
        self.relabeled = True

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().ip_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def info(self) -> dict:
        i = GraphInfo()
        _check(load().ip_graph_info(self._h, ctypes.byref(i)), "ip_graph_info")
        return {k: getattr(i, k) for k, _ in GraphInfo._fields_}

    def run(self, app, max_supersteps=100000, stats_capacity=1024, raise_on_maxsteps=False, **opts) -> RunStats:
        name = app if isinstance(app, str) else {v: k for k, v in APPS.items()}[int(app)]
        app = APPS[name]
        o = default_options(name, relabeled=self.relabeled, **opts)
        cap = stats_capacity
        arr = dict(mode=np.zeros(cap, np.uint8), active=np.zeros(cap, np.uint32),
                   broadcasters=np.zeros(cap, np.uint32), messages=np.zeros(cap, np.uint64),
                   features=np.zeros(cap * N_FEATURES, np.float32), mode_ms=np.zeros(cap * 3, np.float32),
                   kernel_ms=np.zeros(cap * 4, np.float32), pr_delta=np.zeros(cap, np.float32))
        s = RunStatsC()
        s.capacity = cap
        s.mode = arr["mode"].ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        s.active = arr["active"].ctypes.data_as(_U32P)
        s.broadcasters = arr["broadcasters"].ctypes.data_as(_U32P)
        s.messages = arr["messages"].ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
        s.features = arr["features"].ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        s.mode_ms = arr["mode_ms"].ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        s.kernel_ms = arr["kernel_ms"].ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        s.pr_delta = arr["pr_delta"].ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        code = load().ip_run(self._h, app, int(max_supersteps), ctypes.byref(o), ctypes.byref(s))
        if code not in (IP_OK, IP_E_MAXSTEPS) or (raise_on_maxsteps and code == IP_E_MAXSTEPS):
            raise IPError(code, "ip_run")
        n = min(s.supersteps, cap)
        return RunStats(code, s.supersteps, bool(s.halted), s.elapsed_ms, arr["mode"][:n], arr["active"][:n],
                        arr["broadcasters"][:n], arr["messages"][:n], arr["features"].reshape(cap, N_FEATURES)[:n],
                        arr["mode_ms"].reshape(cap, 3)[:n], arr["kernel_ms"].reshape(cap, 4)[:n],
                        arr["pr_delta"][:n])

    def values(self, app=None, out=None, stream=None):
        """Values of the last run: float32 ranks or uint32 labels/distances.

        out: None (returns a new numpy array) or a preallocated numpy array / CUDA tensor."""
        L = load()
        st = _stream_handle(stream)
        if out is None:
            name = app if isinstance(app, str) or app is None else {v: k for k, v in APPS.items()}[int(app)]
            dt = np.float32 if name in FLOAT_APPS else np.uint32
            out = np.empty(self.n, dt)
        if _is_torch(out):
            _check(L.ip_get_values(self._h, out.data_ptr(), out.numel() * out.element_size(), int(out.is_cuda), st),
                   "ip_get_values")
        else:
            _check(L.ip_get_values(self._h, out.ctypes.data, out.nbytes, 0, st), "ip_get_values")
        return out

    def _batch(self, fn, arr, k, out, out_rows, max_supersteps, stream, barrier_timeout_ns, engine=0):
        L = load()
        arr = np.ascontiguousarray(arr, dtype=np.uint32)
        per = np.zeros(k, np.uint32)
        st = BatchStatsC()
        st.instance_supersteps = per.ctypes.data_as(_U32P)
        st.barrier_timeout_ns = int(barrier_timeout_ns)
        st.engine = int(engine)
        if out is None:
            out = np.empty((out_rows, self.n) if out_rows else self.n, np.uint32)
        if _is_torch(out):
            ptr, dev = out.data_ptr(), int(out.is_cuda)
        else:
            ptr, dev = out.ctypes.data, 0
        code = getattr(L, fn)(self._h, arr.ctypes.data_as(_U32P), k, ptr, dev, int(max_supersteps),
                              ctypes.byref(st), _stream_handle(stream))
        if code not in (IP_OK, IP_E_MAXSTEPS):
            raise IPError(code, fn)
        return out, dict(code=code, supersteps=st.supersteps, halted=bool(st.halted), messages=st.messages,
                         instance_supersteps=per, elapsed_ms=st.elapsed_ms)

    def run_batch_sssp(self, sources, out=None, max_supersteps=100000, stream=None, barrier_timeout_ns=0):
        """SSSP from every source in one persistent launch: (dist[k, n], stats)."""
        k = len(sources)
        return self._batch("ip_run_batch_sssp", sources, k, out, k, max_supersteps, stream, barrier_timeout_ns)

    def run_batch_hashmin(self, instance_offsets, out=None, max_supersteps=100000, stream=None,
                          barrier_timeout_ns=0, engine="graph"):
        """Hashmin of every block-diagonal instance in one launch: (local labels[n], stats).
        engine: "graph" (device-driven superstep graph) or "persistent" (cooperative kernel)."""
        k = len(instance_offsets) - 1
        return self._batch("ip_run_batch_hashmin", instance_offsets, k, out, 0, max_supersteps, stream,
                           barrier_timeout_ns, 0 if engine == "graph" else 1)

    def set_selector(self, blob: bytes):
        b = bytes(blob)
        _check(load().ip_set_selector(self._h, b, len(b)), "ip_set_selector")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def hashmin_noalloc(n, csr_offsets, csr_cols, labels, max_supersteps=100000, stream=None):
    """Hashmin through ip_hashmin_noalloc: no device allocation by the library.

    For callers that may not allocate device memory (e.g. inside another
    framework's memory pool): all arguments are CUDA tensors the caller owns.
    Returns (code, supersteps)."""
    for t in (csr_offsets, csr_cols, labels):
        if not (_is_torch(t) and t.is_cuda):
            raise TypeError("CUDA tensors expected")
    steps = ctypes.c_uint32(0)
    code = load().ip_hashmin_noalloc(int(n), int(csr_cols.numel()), csr_offsets.data_ptr(), csr_cols.data_ptr(),
                                     labels.data_ptr(), int(max_supersteps), ctypes.byref(steps),
                                     _stream_handle(stream))
    return code, steps.value
