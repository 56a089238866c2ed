"""Pins of the mutual-reachability mode of the oracle: its graph is made of
line-graph arcs weighed by the brute-force core distances, contains the
skeleton and every kNN pair, and at k = 1 reduces exactly to the plain
method (every weight is then the arc's own |dt|)."""
import numpy as np
import pytest

import bruteforce as bf
from oracle import oracle as O
from paper_2311_10337_gb300 import synth

INF = np.iinfo(np.int64).max
GRAPHS = [synth.random_small(30 + 11 * s, 4 + s % 7, 3 + s % 9, 600 + s, zipf_s=1.2 if s % 2 else 0.0)
          for s in range(16)]


@pytest.mark.parametrize("g", GRAPHS, ids=lambda g: g.name)
@pytest.mark.parametrize("k", [1, 2, 4])
def test_mrd_graph_against_brute_force(g, k):
    u, v, w = O.mrd_graph(g.src, g.dst, g.t, g.n_vertices, k)
    full = bf.undirected_edges(g.src, g.dst, g.t)
    ids, core = bf.knn_bruteforce(g.src, g.dst, g.t, k)
    got = {(a, b): x for a, b, x in zip(u.tolist(), v.tolist(), w.tolist())}
    assert len(got) == len(u)                                  # a set
    want = {}
    su, sv, _ = O.skeleton(g.src, g.dst, g.t, g.n_vertices)
    pairs = set(zip(su.tolist(), sv.tolist()))
    for e in range(g.n_edges):
        for nb in ids[e].tolist():
            if nb >= 0:
                pairs.add((min(e, nb), max(e, nb)))
    for a, b in pairs:
        x = max(int(core[a]), int(core[b]), full[(a, b)])      # every pair is an arc of L_G
        if x != INF:
            want[(a, b)] = x
    assert got == want


@pytest.mark.parametrize("g", GRAPHS, ids=lambda g: g.name)
def test_mrd_with_k1_is_the_plain_method(g):
    a = O.mrd_run(g.src, g.dst, g.t, g.n_vertices, 1, 3)
    b = O.run(g.src, g.dst, g.t, g.n_vertices, 1, 3)
    assert sorted(a["mst"][2].tolist()) == sorted(b["mst"][2].tolist())
    assert np.array_equal(a["condensed"]["labels"], b["condensed"]["labels"])


def test_mrd_weights_dominate_plain_weights():
    g = synth.random_small(300, 25, 80, 71)
    u, v, w = O.mrd_graph(g.src, g.dst, g.t, g.n_vertices, 4)
    assert np.all(w >= np.abs(g.t[u] - g.t[v]))
