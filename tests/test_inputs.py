"""Input generators: determinism, CSR/CSC consistency, symmetric weights."""
import numpy as np

import inputs


def test_rmat_deterministic_and_shaped():
    a = inputs.rmat_graph(10, seed=3)
    b = inputs.rmat_graph(10, seed=3)
    c = inputs.rmat_graph(10, seed=4)
    assert np.array_equal(a.col, b.col) and np.array_equal(a.row_ptr, b.row_ptr)
    assert not np.array_equal(a.col, c.col)
    assert a.n == 1024 and 0 < a.m <= 16 * 1024
    # rows sorted and duplicate free
    for v in range(a.n):
        row = a.col[a.row_ptr[v]:a.row_ptr[v + 1]].astype(np.int64)
        assert np.all(np.diff(row) > 0)
    # R-MAT skew: vertex 0 (all-zero bits) is the heaviest source
    assert a.out_degree().argmax() == 0


def test_csc_is_transpose():
    g = inputs.rmat_graph(9, weighted=True)
    src, dst = g.edges()
    fwd = set(zip(src.tolist(), dst.tolist(), g.w.tolist()))
    tsrc = np.repeat(np.arange(g.n), g.in_degree())
    back = set(zip(g.t_idx.tolist(), tsrc.tolist(), g.wt.tolist()))
    assert fwd == back
    for v in range(g.n):
        seg = g.t_idx[g.t_ptr[v]:g.t_ptr[v + 1]].astype(np.int64)
        assert np.all(np.diff(seg) > 0)


def test_symmetric_weights():
    g = inputs.rmat_graph(9, symmetrize=True, weighted=True)
    src, dst = g.edges()
    wmap = {(a, b): w for a, b, w in zip(src.tolist(), dst.tolist(), g.w.tolist())}
    assert all(wmap[(b, a)] == w for (a, b), w in wmap.items())
    assert g.w.min() >= 1 and g.w.max() <= 255
    assert g.t_ptr is g.row_ptr


def test_block_diagonal():
    gs = [inputs.rmat_graph(5, seed=s, symmetrize=True) for s in (1, 2, 3)]
    u, offs = inputs.block_diagonal(gs)
    assert u.n == sum(g.n for g in gs) and u.m == sum(g.m for g in gs)
    for i, g in enumerate(gs):
        lo = offs[i]
        seg = u.col[u.row_ptr[lo]:u.row_ptr[lo + g.n]] - lo
        assert np.array_equal(seg, g.col)


def test_sources_and_sizes():
    s = inputs.uniform_vertices(1000, 255, seed=1)
    assert s.shape == (255,) and s.max() < 1000
    z = inputs.loguniform_ints(1000, 1000, 100000, seed=1)
    assert z.min() >= 1000 and z.max() <= 100000
    assert np.array_equal(z, inputs.loguniform_ints(1000, 1000, 100000, seed=1))


def test_permuted_rmat_is_the_same_graph_relabelled():
    """The permuted variant is a seeded relabelling: a permutation, deterministic,
    the same degree multiset and an isomorphic edge set; the hub is no longer vertex 0."""
    p = inputs.random_permutation(1024, 7)
    assert np.array_equal(np.sort(p), np.arange(1024)) and np.array_equal(p, inputs.random_permutation(1024, 7))
    a = inputs.rmat_graph(10, seed=3)
    b = inputs.rmat_graph(10, seed=3, permute_seed=7)
    assert a.m == b.m
    assert np.array_equal(np.sort(a.out_degree()), np.sort(b.out_degree()))
    assert np.array_equal(b.out_degree()[p], a.out_degree())
    sa, ta = a.edges()
    sb, tb = b.edges()
    ka = np.sort(p[sa].astype(np.uint64) << 32 | p[ta])
    kb = np.sort(sb.astype(np.uint64) << 32 | tb)
    assert np.array_equal(ka, kb)
    assert b.out_degree().argmax() == p[0] != 0
