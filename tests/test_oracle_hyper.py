"""Pins of the hypergraph oracle (Sec. 4.4) against the explicit hypergraph
line graph: the skeleton is a subgraph with equal weights, has the same
components at every threshold, a forest of the same total weight, and the
size bound; a directed graph written as a directed hypergraph gives the
graph skeleton exactly."""
import numpy as np
import pytest

import bruteforce as bf
from oracle import oracle as O
from paper_2311_10337_gb300 import synth

INF = np.iinfo(np.int64).max
CASES = [(directed, seed) for directed in (False, True) for seed in range(14)]


def _hyper(directed, seed):
    return synth.hyper_small(20 + 9 * seed, 10 + seed % 7, 2 + seed % 9, seed, directed,
                             max_members=3 + seed % 2)


def _skel(h):
    return O.hyper_skeleton(h.t, h.n_vertices, h.s_off, h.s_vert, h.d_off, h.d_vert)


@pytest.mark.parametrize("directed,seed", CASES)
def test_hyper_weighted_connectivity(directed, seed):
    h = _hyper(directed, seed)
    E = h.n_edges
    full = bf.hyper_line_graph(h)
    u, v, w = _skel(h)
    sk = {(a, b): x for a, b, x in zip(u.tolist(), v.tolist(), w.tolist())}
    assert len(sk) == len(u)
    assert all(full[key] == x for key, x in sk.items())          # a subgraph, same weights
    for om in sorted(set(full.values())) + [INF]:
        assert np.array_equal(bf.components(E, full, om), bf.components(E, sk, om)), om
    # forest weight: Kruskal on the explicit line graph (Thm. 1 analogue)
    mu, mv, mw = O.mst(E, u, v, w)
    uf = bf.UnionFind(E)
    wf = [x for (a, b), x in sorted(full.items(), key=lambda kv: (kv[1], kv[0])) if uf.union(a, b)]
    assert wf == sorted(mw.tolist())
    # size bound: sum over vertices of (d_i - 1), d_i = incident hyperedges
    deg = np.bincount(h.s_vert, minlength=h.n_vertices)
    if directed:
        deg = deg + np.bincount(h.d_vert, minlength=h.n_vertices)
    assert len(u) <= int(np.sum(np.maximum(deg - 1, 0)))


@pytest.mark.parametrize("seed", range(8))
def test_graph_as_directed_hypergraph(seed):
    """One source and one target per hyperedge: exactly the graph skeleton,
    and Alg. 1 gives the graph's labels."""
    g = synth.random_small(40 + 13 * seed, 5 + seed % 6, 3 + seed % 8, 300 + seed)
    E = g.n_edges
    off = np.arange(E + 1, dtype=np.int64)
    hu, hv, hw = O.hyper_skeleton(g.t, g.n_vertices, off, g.src, off, g.dst)
    gu, gv, gw = O.skeleton(g.src, g.dst, g.t, g.n_vertices)
    assert np.array_equal(hu, gu) and np.array_equal(hv, gv) and np.array_equal(hw, gw)
    a = O.hyper_run(g.t, g.n_vertices, off, g.src, off, g.dst, M=3)
    b = O.run(g.src, g.dst, g.t, g.n_vertices, 3, 3)
    assert np.array_equal(a["condensed"]["labels"], b["condensed"]["labels"])


def test_undirected_path_is_local_mst():
    """At one vertex the path in time order has the weight of the clique's
    MST (points on a line: t_max - t_min)."""
    t = np.array([5, 1, 9, 1, 4], np.int64)
    off = np.arange(6, dtype=np.int64)
    vert = np.zeros(5, np.int32)                   # all five share vertex 0
    u, v, w = O.hyper_skeleton(t, 1, off, vert)
    assert sorted(w.tolist()) == [0, 1, 3, 4] and int(w.sum()) == 9 - 1
    assert sorted(zip(u.tolist(), v.tolist())) == [(0, 2), (0, 4), (1, 3), (3, 4)]


def test_hyper_validation():
    t = np.array([1, 2], np.int64)
    off = np.array([0, 2, 3], np.int64)
    with pytest.raises(ValueError):                # vertex repeated in one hyperedge
        O.hyper_skeleton(t, 4, off, np.array([1, 1, 2], np.int32))
    with pytest.raises(ValueError):                # vertex out of range
        O.hyper_skeleton(t, 2, off, np.array([0, 1, 2], np.int32))
    one = np.array([0, 1, 2], np.int64)
    with pytest.raises(ValueError):                # a vertex both source and target
        O.hyper_skeleton(t, 4, one, np.array([0, 1], np.int32), one, np.array([0, 2], np.int32))
