"""Pins for the CPU oracle: each test checks it against something other than itself.

- Hashmin (Fig. 9) against union-find written here and scipy's connected components.
- SSSP (Fig. 10, weighted) against scipy's Dijkstra; with unit weights, the
  per-superstep broadcaster counts against BFS layer sizes (this also pins the
  BSP visibility rule of Section 4.2: an asynchronous engine would finish in
  fewer supersteps).
- PageRank (Fig. 8 with the constant of Fig. 12) against closed forms
  (directed cycle, complete digraph, symmetric star), exact rational arithmetic,
  a dense FP64 matrix iteration, and the sum-to-one invariant.
- Hand-worked examples in tests/golden/.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import inputs
import oracle

INF = oracle.INF


def _csr_matrix(g, weights=None):
    data = np.ones(g.m) if weights is None else weights.astype(np.float64)
    return sp.csr_matrix((data, g.col.astype(np.int64), g.row_ptr.astype(np.int64)), shape=(g.n, g.n))


# ------------------------------------------------------------------ golden
def _parse_edges(s, directed=False):
    src, dst, w = [], [], []
    for tok in s.split():
        if ":" in tok:
            e, wt = tok.split(":")
        else:
            e, wt = tok, "1"
        a, b = (int(x) for x in e.split("-"))
        src.append(a), dst.append(b), w.append(int(wt))
        if not directed:
            src.append(b), dst.append(a), w.append(int(wt))
    return np.array(src, np.uint32), np.array(dst, np.uint32), np.array(w, np.uint32)


def _ints(s):
    return [INF if t == "INF" else int(t) for t in s.split()]


def test_golden_hashmin(golden):
    ex = golden["hashmin_two_components"]
    n = int(ex["n"])
    s, d, _ = _parse_edges(ex["edges"])
    g = inputs.from_edges(n, s, d)
    lab, st = oracle.hashmin(g.n, g.row_ptr, g.col)
    assert lab.tolist() == _ints(ex["labels"])
    assert st["supersteps"] == int(ex["supersteps"]) and st["halted"]
    assert st["active"].tolist() == _ints(ex["active"])
    assert st["broadcasters"].tolist() == _ints(ex["broadcasters"])
    assert st["messages"].tolist() == _ints(ex["messages"])


def test_golden_sssp(golden):
    ex = golden["sssp_weighted"]
    n = int(ex["n"])
    s, d, w = _parse_edges(ex["edges"])
    # weights keyed by (src, dst) in CSR order
    g = inputs.from_edges(n, s, d)
    wmap = {(int(a), int(b)): int(c) for a, b, c in zip(s, d, w)}
    src, dst = g.edges()
    wc = np.array([wmap[(int(a), int(b))] for a, b in zip(src, dst)], np.uint32)
    dist, st = oracle.sssp(g.n, g.row_ptr, g.col, wc, source=int(ex["source"]))
    assert dist.tolist() == _ints(ex["dist"])
    assert st["supersteps"] == int(ex["supersteps"])
    assert st["active"].tolist() == _ints(ex["active"])
    assert st["broadcasters"].tolist() == _ints(ex["broadcasters"])
    assert st["messages"].tolist() == _ints(ex["messages"])


def test_golden_pagerank(golden):
    ex = golden["pagerank_three"]
    n = int(ex["n"])
    s, d, _ = _parse_edges(ex["directed_edges"], directed=True)
    g = inputs.from_edges(n, s, d)
    r, st = oracle.pagerank(g.n, g.row_ptr, g.col, T=int(ex["T"]))
    want = [float(Fraction(t)) for t in ex["rank"].split()]
    np.testing.assert_allclose(r, want, rtol=1e-15)
    assert st["supersteps"] == int(ex["supersteps"])
    assert st["active"].tolist() == _ints(ex["active"])
    assert st["broadcasters"].tolist() == _ints(ex["broadcasters"])
    assert st["messages"].tolist() == _ints(ex["messages"])


# ------------------------------------------------------------------ Hashmin
class _UF:
    def __init__(self, n):
        self.p = list(range(n))

    def find(self, x):
        while self.p[x] != x:
            self.p[x] = self.p[self.p[x]]
            x = self.p[x]
        return x

    def union(self, a, b):
        ra, rb = self.find(a), self.find(b)
        if ra != rb:
            self.p[max(ra, rb)] = min(ra, rb)  # the root is the smaller id


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_hashmin_union_find_tiny(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 40))
    m = int(rng.integers(0, 3 * n))
    g = inputs.from_edges(n, rng.integers(0, n, m), rng.integers(0, n, m), symmetrize=True)
    lab, st = oracle.hashmin(g.n, g.row_ptr, g.col)
    uf = _UF(n)
    src, dst = g.edges()
    for a, b in zip(src, dst):
        uf.union(int(a), int(b))
    assert lab.tolist() == [uf.find(v) for v in range(n)]
    assert st["halted"]


@pytest.mark.parametrize("scale", [8, 12])
def test_hashmin_scipy_components(scale):
    g = inputs.rmat_graph(scale, symmetrize=True)
    lab, _ = oracle.hashmin(g.n, g.row_ptr, g.col)
    _, comp = csg.connected_components(_csr_matrix(g), directed=False)
    # min vertex id of each component
    mins = np.full(comp.max() + 1, np.iinfo(np.int64).max)
    np.minimum.at(mins, comp, np.arange(g.n))
    assert np.array_equal(lab, mins[comp].astype(np.uint32))


def test_hashmin_directed_reachability():
    """Directed graphs: label(v) = min id over vertices that can reach v."""
    rng = np.random.default_rng(7)
    n, m = 30, 45
    g = inputs.from_edges(n, rng.integers(0, n, m), rng.integers(0, n, m))
    lab, _ = oracle.hashmin(g.n, g.row_ptr, g.col)
    reach = csg.shortest_path(_csr_matrix(g), unweighted=True, directed=True)
    want = [min(u for u in range(n) if np.isfinite(reach[u, v])) for v in range(n)]
    assert lab.tolist() == want


def test_hashmin_path_closed_form():
    """Undirected path 0-1-...-(n-1): value(v) after s supersteps is max(v-s, 0), so
    superstep s>=1 has n-s broadcasters and the run ends after n+1 supersteps."""
    n = 9
    g = inputs.path(n)
    lab, st = oracle.hashmin(g.n, g.row_ptr, g.col)
    assert lab.tolist() == [0] * n
    assert st["supersteps"] == n + 1
    assert st["broadcasters"].tolist() == [n] + [n - s for s in range(1, n)] + [0]


def test_hashmin_no_edges():
    g = inputs.empty_graph(5)
    lab, st = oracle.hashmin(g.n, g.row_ptr, g.col)
    assert lab.tolist() == list(range(5))
    assert st["supersteps"] == 1 and st["messages"].tolist() == [0]


# --------------------------------------------------------------------- SSSP
@pytest.mark.parametrize("scale,sym", [(8, True), (11, True), (10, False)])
def test_sssp_dijkstra(scale, sym):
    g = inputs.rmat_graph(scale, symmetrize=sym, weighted=True)
    src = 0
    dist, st = oracle.sssp(g.n, g.row_ptr, g.col, g.w, source=src)
    ref = csg.dijkstra(_csr_matrix(g, g.w), directed=True, indices=src)
    want = np.where(np.isfinite(ref), ref, INF).astype(np.uint64)
    assert np.array_equal(dist.astype(np.uint64), want)
    assert st["halted"]


def test_sssp_er_other_source():
    g = inputs.er_graph(500, 1500, seed=3, weighted=True)
    for s in (0, 17, 499):
        dist, _ = oracle.sssp(g.n, g.row_ptr, g.col, g.w, source=s)
        ref = csg.dijkstra(_csr_matrix(g, g.w), directed=True, indices=s)
        assert np.array_equal(dist.astype(np.float64), np.where(np.isfinite(ref), ref, INF))


@pytest.mark.parametrize("scale", [9, 12])
def test_sssp_unit_weights_bfs_layers(scale):
    """Unit weights (Fig. 10 exactly): distances are BFS depths, superstep s has
    exactly |layer s| broadcasters, and the run takes eccentricity + 2 supersteps."""
    g = inputs.rmat_graph(scale, symmetrize=True)
    dist, st = oracle.sssp(g.n, g.row_ptr, g.col, None, source=0)
    depth = csg.shortest_path(_csr_matrix(g), unweighted=True, indices=0)
    want = np.where(np.isfinite(depth), depth, INF)
    assert np.array_equal(dist.astype(np.float64), want)
    ecc = int(depth[np.isfinite(depth)].max())
    layers = np.bincount(depth[np.isfinite(depth)].astype(np.int64), minlength=ecc + 1)
    assert st["supersteps"] == ecc + 2
    assert st["broadcasters"].tolist() == layers.tolist() + [0]


def test_sssp_saturates_at_inf():
    """A message that would pass INF saturates at INF (it still arrives)."""
    g = inputs.from_edges(3, np.array([0, 1]), np.array([1, 2]))
    w = np.array([0xFFFFFFF0, 0x20], np.uint32)
    dist, st = oracle.sssp(g.n, g.row_ptr, g.col, w, source=0)
    assert dist.tolist() == [0, 0xFFFFFFF0, INF]
    # v2 receives INF in superstep 2: it is active but does not improve
    assert st["active"].tolist() == [3, 1, 1]


def test_sssp_isolated_source():
    g = inputs.empty_graph(4)
    dist, st = oracle.sssp(g.n, g.row_ptr, g.col, None, source=2)
    assert dist.tolist() == [INF, INF, 0, INF]
    assert st["supersteps"] == 1


# ----------------------------------------------------------------- PageRank
@pytest.mark.parametrize("n,T", [(7, 30), (100, 5), (1, 3)])
def test_pagerank_cycle_uniform(n, T):
    """Directed cycle: every iterate is exactly 1/N since (1-d)/N + d/N = 1/N."""
    g = inputs.directed_cycle(n) if n > 1 else inputs.from_edges(1, [0], [0])
    r, st = oracle.pagerank(g.n, g.row_ptr, g.col, T=T)
    np.testing.assert_allclose(r, 1.0 / n, rtol=1e-14)
    assert st["supersteps"] == T + 1


def test_pagerank_complete_uniform():
    g = inputs.complete_digraph(12)
    r, _ = oracle.pagerank(g.n, g.row_ptr, g.col, T=30)
    np.testing.assert_allclose(r, 1.0 / 12, rtol=1e-14)


@pytest.mark.parametrize("k,T", [(5, 30), (40, 30), (3, 1), (8, 7)])
def test_pagerank_star_closed_form(k, T):
    """Symmetric star, centre plus k leaves, N = k+1. With errors from the fixed point
    e_c(t), e_l(t): e_c(t+1) = d*k*e_l(t) and e_l(t+1) = d*e_c(t)/k."""
    d, N = 0.85, k + 1
    rc = (1 + d * k) / (N * (1 + d))
    rl = (1 - d) / N + d * rc / k
    ec, el = 1.0 / N - rc, 1.0 / N - rl
    for _ in range(T):
        ec, el = d * k * el, d * ec / k
    g = inputs.star(k)
    r, _ = oracle.pagerank(g.n, g.row_ptr, g.col, T=T, damping=d)
    np.testing.assert_allclose(r[0], rc + ec, rtol=1e-13)
    np.testing.assert_allclose(r[1:], rl + el, rtol=1e-13)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_pagerank_dense_matrix_iteration(seed):
    """r <- (1-d)/N + d * A^T D^+ r with D^+ the inverse out-degree (0 if dangling)."""
    rng = np.random.default_rng(seed)
    n = 25
    m = 60
    s = rng.integers(0, n, m)
    t = rng.integers(0, n, m)
    keep = s != n - 1  # vertex n-1 is dangling
    s = np.concatenate([s[keep], [0]])  # plus a self-loop at 0
    t = np.concatenate([t[keep], [0]])
    g = inputs.from_edges(n, s, t)
    A = np.zeros((n, n))
    src, dst = g.edges()
    A[src, dst] = 1.0
    deg = A.sum(axis=1)
    Dp = np.where(deg > 0, 1.0 / np.where(deg > 0, deg, 1), 0.0)
    d, T = 0.85, 30
    r = np.full(n, 1.0 / n)
    for _ in range(T):
        r = (1 - d) / n + d * (A.T @ (Dp * r))
    got, _ = oracle.pagerank(g.n, g.row_ptr, g.col, T=T, damping=d)
    np.testing.assert_allclose(got, r, rtol=1e-12, atol=0)
    assert (deg == 0).any() and np.diag(A).any()


def test_pagerank_exact_fractions():
    """Brute force with exact rationals on a small graph with a dangling vertex."""
    edges = [(0, 1), (0, 2), (1, 2), (2, 0), (2, 3), (4, 2)]
    n, T, d = 5, 6, Fraction(85, 100)
    g = inputs.from_edges(n, [a for a, _ in edges], [b for _, b in edges])
    outd = [sum(1 for a, _ in edges if a == v) for v in range(n)]
    r = [Fraction(1, n)] * n
    for _ in range(T):
        nr = [(1 - d) / n] * n
        for a, b in edges:
            nr[b] += d * r[a] / outd[a]
        r = nr
    got, _ = oracle.pagerank(g.n, g.row_ptr, g.col, T=T)
    np.testing.assert_allclose(got, [float(x) for x in r], rtol=1e-14)


def test_pagerank_sum_to_one_without_dangling():
    g0 = inputs.rmat_graph(10, symmetrize=True)
    # connect every vertex to the next so none is dangling
    s, t = g0.edges()
    ring = np.arange(g0.n, dtype=np.uint32)
    g = inputs.from_edges(g0.n, np.concatenate([s, ring]), np.concatenate([t, (ring + 1) % g0.n]))
    assert (g.out_degree() > 0).all()
    r, st = oracle.pagerank(g.n, g.row_ptr, g.col, T=30)
    assert abs(r.sum() - 1.0) < 1e-12
    assert st["active"].tolist() == [g.n] * 31
    assert st["messages"].tolist() == [g.m] * 30 + [0]


def test_pagerank_dangling_mass_dropped():
    """Mass at dangling vertices leaves the system (Pregel semantics), so the sum drops."""
    g = inputs.from_edges(2, [0], [1])
    r, _ = oracle.pagerank(g.n, g.row_ptr, g.col, T=1)
    # s1: r0 = 0.15/2, r1 = 0.15/2 + 0.85 * 0.5
    np.testing.assert_allclose(r, [0.075, 0.075 + 0.425], rtol=1e-15)


def test_pagerank_cap_stops_early():
    g = inputs.directed_cycle(4)
    r, st = oracle.pagerank(g.n, g.row_ptr, g.col, T=30, max_supersteps=5)
    assert st["supersteps"] == 5 and not st["halted"]


def test_pagerank_update_exact_fractions():
    """The one-superstep update against exact rationals: from a non-uniform rank
    vector with a dangling in-neighbour, a self-loop and a vertex with no in-edges."""
    edges = [(0, 1), (0, 2), (1, 2), (2, 0), (2, 3), (4, 2), (3, 3)]
    n, d = 5, Fraction(85, 100)
    g = inputs.from_edges(n, [a for a, _ in edges], [b for _, b in edges])
    outd = [sum(1 for a, _ in edges if a == v) for v in range(n)]
    prev = [Fraction(k + 1, 17) for k in range(n)]
    want = [(1 - d) / n] * n
    for a, b in edges:
        want[b] += d * prev[a] / outd[a]
    got = oracle.pagerank_update(range(n), n, g.t_ptr, g.t_idx, g.out_degree(), [float(x) for x in prev])
    np.testing.assert_allclose(got, [float(x) for x in want], rtol=1e-15)


@pytest.mark.parametrize("name", ["rmat10", "er"])
def test_pagerank_update_iterated_is_the_engine(name):
    """T updates of every vertex from 1/N reproduce the synchronous engine's run."""
    g = inputs.rmat_graph(10, seed=4) if name == "rmat10" else inputs.er_graph(500, 1500, seed=5)
    r = np.full(g.n, 1.0 / g.n)
    for _ in range(12):
        r = oracle.pagerank_update(range(g.n), g.n, g.t_ptr, g.t_idx, g.out_degree(), r)
    want, _ = oracle.pagerank(g.n, g.row_ptr, g.col, T=12)
    np.testing.assert_allclose(r, want, rtol=1e-12)
    assert (g.out_degree() == 0).any()


@pytest.mark.parametrize("scale", [12, 14])
def test_pagerank_sparse_power_iteration(scale):
    """At R-MAT scale (self-loops, dangling vertices, hubs): T = 30 steps of
    r <- (1-d)/N + d * A^T (D^+ r) with scipy's sparse matrix product."""
    g = inputs.rmat_graph(scale, seed=7)
    A = _csr_matrix(g)
    deg = np.asarray(A.sum(axis=1)).ravel()
    inv = np.where(deg > 0, 1.0 / np.where(deg > 0, deg, 1.0), 0.0)
    d, n = 0.85, g.n
    r = np.full(n, 1.0 / n)
    AT = A.T.tocsr()
    for _ in range(30):
        r = (1 - d) / n + d * (AT @ (inv * r))
    got, st = oracle.pagerank(g.n, g.row_ptr, g.col, T=30, damping=d)
    np.testing.assert_allclose(got, r, rtol=1e-12, atol=0)
    assert (deg == 0).any() and A.diagonal().any()
    assert st["supersteps"] == 31 and st["messages"].tolist() == [g.m] * 30 + [0]


# ------------------------------------------------- PageRank, one superstep in C
def test_pagerank_superstep_exact_fractions():
    """The C one-superstep update (pull form) against exact rationals, any split of
    the vertex range giving the same values."""
    edges = [(0, 1), (0, 2), (1, 2), (2, 0), (2, 3), (4, 2), (3, 3)]
    n, d = 5, Fraction(85, 100)
    g = inputs.from_edges(n, [a for a, _ in edges], [b for _, b in edges])
    outd = [sum(1 for a, _ in edges if a == v) for v in range(n)]
    prev = [Fraction(k + 1, 17) for k in range(n)]
    want = [(1 - d) / n] * n
    for a, b in edges:
        want[b] += d * prev[a] / outd[a]
    pf = [float(x) for x in prev]
    got = oracle.pagerank_superstep(n, g.t_ptr, g.t_idx, g.out_degree(), pf)
    np.testing.assert_allclose(got, [float(x) for x in want], rtol=1e-15)
    parts = np.concatenate([oracle.pagerank_superstep(n, g.t_ptr, g.t_idx, g.out_degree(), pf, v_begin=a, v_end=b)
                            for a, b in ((0, 2), (2, 2), (2, 5))])
    assert np.array_equal(parts, got)


def test_pagerank_superstep_continues_the_engine():
    """From the ranks of a T - 1 run of the push-based engine, one pull-form superstep
    gives the T run (R-MAT with hubs, self-loops and dangling vertices)."""
    g = inputs.rmat_graph(11, seed=9)
    r9, _ = oracle.pagerank(g.n, g.row_ptr, g.col, T=9)
    r10, _ = oracle.pagerank(g.n, g.row_ptr, g.col, T=10)
    got = oracle.pagerank_superstep(g.n, g.t_ptr, g.t_idx, g.out_degree(), r9)
    np.testing.assert_allclose(got, r10, rtol=1e-13)
    assert (g.out_degree() == 0).any()


# ------------------------------------------------- PageRank to convergence
def _star_iterates(k, T, d=0.85):
    """Closed form of the symmetric star's iterates t = 0..T (centre, leaf)."""
    N = k + 1
    rc = (1 + d * k) / (N * (1 + d))
    rl = (1 - d) / N + d * rc / k
    ec, el = 1.0 / N - rc, 1.0 / N - rl
    out = [(rc + ec, rl + el)]
    for _ in range(T):
        ec, el = d * k * el, d * ec / k
        out.append((rc + ec, rl + el))
    return out


@pytest.mark.parametrize("k", [5, 40])
def test_pagerank_convergence_star_closed_form(k):
    """Star: the L1 change of superstep t is |c_t - c_(t-1)| + k |l_t - l_(t-1)| from
    the closed-form iterates, so the halting superstep for a tolerance eps is the
    first t >= 1 with that change below eps, and the ranks are the iterate t."""
    its = _star_iterates(k, 200)
    delta = [0.0] + [abs(its[t][0] - its[t - 1][0]) + k * abs(its[t][1] - its[t - 1][1]) for t in range(1, 201)]
    g = inputs.star(k)
    for eps in (1e-3, 1e-6, 1e-9):
        t_halt = next(t for t in range(1, 201) if delta[t] < eps)
        r, st = oracle.pagerank(g.n, g.row_ptr, g.col, T=200, tolerance=eps)
        assert st["halted"] and st["supersteps"] == t_halt + 1, (eps, st["supersteps"], t_halt)
        np.testing.assert_allclose(st["delta"][1:], delta[1:t_halt + 1], rtol=1e-9, atol=1e-14)
        np.testing.assert_allclose(r[0], its[t_halt][0], rtol=1e-13)
        np.testing.assert_allclose(r[1:], its[t_halt][1], rtol=1e-13)


def test_pagerank_convergence_cycle_halts_at_once():
    """Directed cycle: every iterate is 1/N, so the first update changes nothing and
    the run halts after superstep 1."""
    g = inputs.directed_cycle(9)
    r, st = oracle.pagerank(g.n, g.row_ptr, g.col, T=30, tolerance=1e-12)
    assert st["halted"] and st["supersteps"] == 2 and st["delta"][1] == 0.0
    np.testing.assert_allclose(r, 1.0 / 9, rtol=1e-15)


def test_pagerank_convergence_matches_dense_iteration():
    """A graph with dangling vertices and self-loops: the oracle's per-superstep L1
    change equals the dense matrix iteration's, and with the tolerance between two
    of them the run stops at the first superstep below it; T still caps the run."""
    g = inputs.rmat_graph(8, seed=3)
    A = np.zeros((g.n, g.n))
    s, t = g.edges()
    A[s, t] = 1.0
    deg = A.sum(axis=1)
    inv = np.where(deg > 0, 1.0 / np.where(deg > 0, deg, 1), 0.0)
    d, n = 0.85, g.n
    r = [np.full(n, 1.0 / n)]
    for _ in range(40):
        r.append((1 - d) / n + d * (A.T @ (inv * r[-1])))
    delta = [0.0] + [float(np.abs(r[i] - r[i - 1]).sum()) for i in range(1, 41)]
    _, st = oracle.pagerank(g.n, g.row_ptr, g.col, T=40)
    np.testing.assert_allclose(st["delta"][1:], delta[1:], rtol=1e-9)
    t_halt = 12
    eps = float(np.sqrt(delta[t_halt] * delta[t_halt - 1]))  # between supersteps 11 and 12
    assert delta[t_halt] < eps < delta[t_halt - 1]
    got, st = oracle.pagerank(g.n, g.row_ptr, g.col, T=40, tolerance=eps)
    assert st["halted"] and st["supersteps"] == t_halt + 1
    np.testing.assert_allclose(got, r[t_halt], rtol=1e-12)
    got, st = oracle.pagerank(g.n, g.row_ptr, g.col, T=5, tolerance=eps)  # the cap T comes first
    assert st["halted"] and st["supersteps"] == 6
    np.testing.assert_allclose(got, r[5], rtol=1e-12)


# ------------------------------------------------- Reliability (not in the paper)
def _f32_prob(w):
    return np.float32(w) * np.float32(1.0 / 256.0)


def _best_products_brute(n, edges, weights, source):
    """Max over all simple paths from source of the FP32 product of edge
    probabilities taken from the source outwards (depth-first enumeration)."""
    adj = {}
    for (a, b), w in zip(edges, weights):
        adj.setdefault(a, []).append((b, _f32_prob(w)))
    best = np.zeros(n, np.float32)
    best[source] = np.float32(1.0)

    def dfs(u, val, seen):
        for v, p in adj.get(u, []):
            if v in seen:
                continue
            x = np.float32(val * p)
            if x > best[v]:
                best[v] = x
            dfs(v, x, seen | {v})

    dfs(source, np.float32(1.0), {source})
    return best


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_reliability_brute_force_tiny(seed):
    rng = np.random.default_rng(seed)
    n = 8
    e = {(int(a), int(b)) for a, b in zip(rng.integers(0, n, 20), rng.integers(0, n, 20)) if a != b}
    src = [a for a, _ in sorted(e)]
    dst = [b for _, b in sorted(e)]
    g = inputs.from_edges(n, src, dst)
    w = rng.integers(1, 256, g.m).astype(np.uint32)  # per-edge weights in CSR order
    s, t = g.edges()
    want = _best_products_brute(n, list(zip(s.tolist(), t.tolist())), w.tolist(), 0)
    got, st = oracle.reliability(g.n, g.row_ptr, g.col, w, source=0)
    assert np.array_equal(got, want), (got, want)
    assert st["halted"]


def _dijkstra_max_product(g, w, source):
    """Dijkstra on the FP32 max-product order (a product never grows along an
    edge, p <= 1, and FP32 rounding keeps that order)."""
    import heapq
    best = np.zeros(g.n, np.float32)
    best[source] = np.float32(1.0)
    done = np.zeros(g.n, bool)
    heap = [(-1.0, source)]
    while heap:
        negv, u = heapq.heappop(heap)
        if done[u]:
            continue
        done[u] = True
        val = best[u]
        for k in range(int(g.row_ptr[u]), int(g.row_ptr[u + 1])):
            v = int(g.col[k])
            x = np.float32(val * _f32_prob(w[k] if w is not None else 1))
            if x > best[v]:
                best[v] = x
                heapq.heappush(heap, (-float(x), v))
    return best


@pytest.mark.parametrize("sym", [True, False])
def test_reliability_dijkstra(sym):
    g = inputs.rmat_graph(10, symmetrize=sym, weighted=True, seed=5)
    src = int(np.argmax(g.out_degree()))
    want = _dijkstra_max_product(g, g.w, src)
    got, _ = oracle.reliability(g.n, g.row_ptr, g.col, g.w, source=src)
    assert np.array_equal(got, want), int((got != want).sum())


def test_reliability_unit_weights_are_bfs_layers():
    """Without weights every edge keeps 1/256: a vertex at BFS depth d gets exactly
    2^(-8d) (exact in FP32 while representable), unreachable vertices 0, and the
    broadcasters of superstep d are the BFS layer d."""
    from scipy.sparse.csgraph import shortest_path
    g = inputs.rmat_graph(11, symmetrize=True, seed=3)
    depth = shortest_path(_csr_matrix(g), unweighted=True, indices=0)
    got, st = oracle.reliability(g.n, g.row_ptr, g.col, None, source=0)
    reach = np.isfinite(depth)
    assert depth[reach].max() <= 15
    np.testing.assert_array_equal(got[reach], np.ldexp(np.float32(1.0), (-8 * depth[reach]).astype(int)))
    assert (got[~reach] == 0).all()
    layers = np.bincount(depth[reach].astype(int))
    assert st["broadcasters"][:len(layers)].tolist() == layers.tolist()


# ------------------------------------------------- Hashmin, one superstep in C
@pytest.mark.parametrize("sym", [True, False])
def test_hashmin_superstep_iterated_is_the_engine(sym):
    """Pull-form supersteps of Hashmin, each vertex broadcasting when its label
    dropped in the superstep before (all of them in superstep 0), reproduce the push
    engine: the labels after every superstep, the recipients (active vertices) and
    the broadcasters, until no vertex broadcasts; the labels are then the union-find
    component minima on the symmetrised graph."""
    g = inputs.rmat_graph(11, symmetrize=sym, seed=6)
    label = np.arange(g.n, dtype=np.uint32)
    bcast = np.ones(g.n, np.uint8)
    _, full = oracle.hashmin(g.n, g.row_ptr, g.col)
    s = 0
    while bcast.any():
        s += 1
        new, recv = oracle.hashmin_superstep(g.n, g.t_ptr, g.t_idx, label, bcast, with_recv=True)
        got_s, st = oracle.hashmin(g.n, g.row_ptr, g.col, max_supersteps=s + 1)
        assert np.array_equal(new, got_s), s
        assert int(recv.sum()) == int(full["active"][s])
        bcast = ((new < label) & (g.out_degree() > 0)).astype(np.uint8)
        assert int((new < label).sum()) == int(full["broadcasters"][s])
        label = new
    assert s + 1 == full["supersteps"]
    if sym:
        from scipy.sparse.csgraph import connected_components
        _, comp = connected_components(_csr_matrix(g), directed=False)
        mins = np.full(comp.max() + 1, g.n, np.int64)
        np.minimum.at(mins, comp, np.arange(g.n))
        assert np.array_equal(label, mins[comp])
