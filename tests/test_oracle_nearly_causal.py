"""Pins of the nearly-causal variant (Sec. 4.3: an arc may point up to delta
back in time, weighed |dt|) against the explicit nearly-causal line graph:
the skeleton is a subgraph with equal weights, has its components at every
threshold and a forest of the same weight; kNN lists equal enumeration;
delta = 0 is the causal method."""
import numpy as np
import pytest

import bruteforce as bf
from oracle import oracle as O
from paper_2311_10337_gb300 import synth

INF = np.iinfo(np.int64).max
GRAPHS = [synth.random_small(25 + 9 * s, 4 + s % 6, 3 + s % 12, 900 + s, zipf_s=1.3 if s % 2 else 0.0)
          for s in range(18)]


@pytest.mark.parametrize("g", GRAPHS, ids=lambda g: g.name)
@pytest.mark.parametrize("delta", [0, 1, 2, 5, 100])
def test_nearly_causal_skeleton(g, delta):
    E = g.n_edges
    full = bf.undirected_edges_nc(g.src, g.dst, g.t, delta)
    u, v, w = O.skeleton_nearly_causal(g.src, g.dst, g.t, g.n_vertices, delta)
    sk = {(a, b): x for a, b, x in zip(u.tolist(), v.tolist(), w.tolist())}
    assert len(sk) == len(u)
    assert all(full[key] == x for key, x in sk.items())
    for om in sorted(set(full.values())) + [INF]:
        assert np.array_equal(bf.components(E, full, om), bf.components(E, sk, om)), om
    mu, mv, mw = O.mst(E, u, v, w)
    uf = bf.UnionFind(E)
    wf = [x for (a, b), x in sorted(full.items(), key=lambda kv: (kv[1], kv[0])) if uf.union(a, b)]
    assert wf == sorted(mw.tolist())


@pytest.mark.parametrize("g", GRAPHS[::2], ids=lambda g: g.name)
@pytest.mark.parametrize("delta", [1, 3, 50])
@pytest.mark.parametrize("k", [1, 4])
def test_nearly_causal_knn(g, delta, k):
    ids, core = O.knn(g.src, g.dst, g.t, g.n_vertices, k, delta_nc=delta)
    bids, bcore = bf.knn_bruteforce(g.src, g.dst, g.t, k, delta_nc=delta)
    assert np.array_equal(ids, bids) and np.array_equal(core, bcore)


def test_delta_zero_is_causal():
    g = synth.random_small(300, 25, 60, 41)
    a = O.run_nearly_causal(g.src, g.dst, g.t, g.n_vertices, 4, 3, 0)
    b = O.run(g.src, g.dst, g.t, g.n_vertices, 4, 3)
    for x, y in zip(a["skeleton"], b["skeleton"]):
        assert np.array_equal(x, y)
    assert np.array_equal(a["condensed"]["labels"], b["condensed"]["labels"])
    assert all(np.array_equal(x, y) for x, y in zip(a["knn"], b["knn"]))


def test_nearly_causal_with_cutoff():
    g = synth.random_small(120, 10, 40, 43)
    full = {k: x for k, x in bf.undirected_edges_nc(g.src, g.dst, g.t, 4).items() if x <= 9}
    u, v, w = O.skeleton_nearly_causal(g.src, g.dst, g.t, g.n_vertices, 4, delta_max=9)
    sk = {(a, b): x for a, b, x in zip(u.tolist(), v.tolist(), w.tolist())}
    for om in sorted(set(full.values())) + [INF]:
        assert np.array_equal(bf.components(g.n_edges, full, om), bf.components(g.n_edges, sk, om))
