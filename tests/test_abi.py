"""The C-ABI library builds, loads without a GPU, and exports every symbol that
include/ipregel.h declares; host-side argument checks need no device."""
import ctypes
import os
import re

import pytest

import paper_2010_08781_gb300 as ipg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(ip_\w+)\s*\(", text, flags=re.M))
    return names


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("ip_graph_create", "ip_run", "ip_get_values", "ip_graph_destroy", "ip_strerror", "ip_set_selector"):
        assert name in d


def test_library_exports_every_declared_symbol():
    lib = ipg.load()
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(ipg.EXPORTS) <= _declared()


def test_strerror_and_defaults_without_gpu():
    assert ipg.strerror(0) == "ok"
    assert "cap" in ipg.strerror(ipg.IP_E_MAXSTEPS)
    o = ipg.default_options()
    assert abs(o.damping - 0.85) < 1e-7 and o.pr_iterations == 30 and o.use_graph == 1


def test_create_rejects_bad_arguments_on_host():
    lib = ipg.load()
    h = ctypes.c_void_p()
    # n_vertices == 0 and NULL offsets are rejected before any CUDA call
    assert lib.ip_graph_create(ctypes.byref(h), 0, 0, None, None, None, None, None, None, 0, None) == ipg.IP_E_INVAL
    assert lib.ip_graph_create(ctypes.byref(h), 4, 0, None, None, None, None, None, None, 0, None) == ipg.IP_E_INVAL
    assert lib.ip_graph_create(ctypes.byref(h), 4, 1 << 32, None, None, None, None, None, None, 0,
                               None) in (ipg.IP_E_INVAL, ipg.IP_E_RANGE)
    assert lib.ip_run(None, 0, 10, None, None) == ipg.IP_E_INVAL
    assert lib.ip_get_values(None, None, 0, 0, None) == ipg.IP_E_INVAL


def test_single_cutoff_override_keeps_the_pair_ordered():
    """A caller who sets one degree-bin cutoff gets the tuned other one only while
    t1 < t2 still holds; both given are passed through as they are."""
    for app in ("hashmin", "sssp", "pagerank"):
        o = ipg.default_options(app, t2=4)
        assert o.t2 == 4 and o.t1 < 4
        o = ipg.default_options(app, t1=100000)
        assert o.t1 == 100000 and o.t2 > 100000
    o = ipg.default_options("hashmin", t1=10, t2=5)
    assert (o.t1, o.t2) == (10, 5)  # rejected by ip_run with IP_E_INVAL


def test_tuned_cutoffs_follow_the_vertex_order():
    """Graphs renumbered by degree class and graphs in the caller's order have their
    own tuned degree-bin cutoffs; the binding picks the set that matches."""
    t = ipg.tuned_defaults()
    if "bins_caller_order" not in t:
        pytest.skip("no tuned cutoffs shipped")
    for app in ("hashmin", "sssp", "pagerank"):
        a = ipg.default_options(app)
        b = ipg.default_options(app, relabeled=False)
        assert (a.t1, a.t2) == (t["bins"][app]["t1"], t["bins"][app]["t2"])
        assert (b.t1, b.t2) == (t["bins_caller_order"][app]["t1"], t["bins_caller_order"][app]["t2"])
        assert a.t1 < a.t2 and b.t1 < b.t2
