"""A wide sweep of the oracle against brute force on the explicit line graph
of Def. 1: 2,000 small random graphs with few vertices and few distinct
times, so ties, repeated pairs and reciprocal concurrent pairs are common.
Each graph is checked for Thm. 3 (components of L* and L_G at every
threshold, L* a subgraph of L_G with equal weights, each pair once), the
size bound of Sec. 2, Thm. 1 (the forest's weights are those of a minimum
spanning forest of L_G), the dendrogram's heights (the minimax distances of
L_G) and the kNN lists."""
import numpy as np

import bruteforce as bf
from oracle import oracle as O
from paper_2311_10337_gb300 import synth

INF = np.iinfo(np.int64).max
N_GRAPHS = 2000


def _graph(seed):
    rng = np.random.default_rng(seed)
    E = int(rng.integers(1, 41))
    V = int(rng.integers(2, 9))
    t_max = int(rng.integers(1, 13))
    return synth.random_small(E, V, t_max, 10_000 + seed, zipf_s=1.4 if seed % 7 == 0 else 0.0)


def _check(g):
    E = g.n_edges
    full = bf.undirected_edges(g.src, g.dst, g.t)
    u, v, w = O.skeleton(g.src, g.dst, g.t, g.n_vertices)
    sk = {(a, b): x for a, b, x in zip(u.tolist(), v.tolist(), w.tolist())}
    assert len(sk) == len(u), "a pair twice in L*"
    assert all(full.get(key) == x for key, x in sk.items()), "L* not a weighted subgraph of L_G"
    for omega in sorted(set(full.values())) + [INF]:
        assert np.array_equal(bf.components(E, full, omega), bf.components(E, sk, omega)), omega
    deg = np.bincount(g.src, minlength=g.n_vertices) + np.bincount(g.dst, minlength=g.n_vertices)
    assert len(u) <= int(np.sum(np.maximum(deg - 1, 0))), "size bound"
    mu, mv, mw = O.mst(E, u, v, w)
    uf = bf.UnionFind(E)
    kruskal = [x for (a, b), x in sorted(full.items(), key=lambda kv: (kv[1], kv[0])) if uf.union(a, b)]
    assert mw.tolist() == sorted(kruskal), "forest weights"
    a, b, _ = O.linkage(E, mu, mv)
    members = {x: [x] for x in range(E)}
    H = np.full((E, E), INF, np.int64)
    np.fill_diagonal(H, 0)
    for s in range(len(a)):
        A, B = members.pop(int(a[s])), members.pop(int(b[s]))
        for x in A:
            H[x, B] = mw[s]
            H[B, x] = mw[s]
        members[E + s] = A + B
    assert np.array_equal(H, bf.minimax(E, full)), "dendrogram heights"
    ids, core = O.knn(g.src, g.dst, g.t, g.n_vertices, 2)
    bids, bcore = bf.knn_bruteforce(g.src, g.dst, g.t, 2)
    assert np.array_equal(ids, bids) and np.array_equal(core, bcore), "kNN"


def test_oracle_sweep_against_bruteforce():
    for seed in range(N_GRAPHS):
        g = _graph(seed)
        try:
            _check(g)
        except AssertionError as ex:
            raise AssertionError(f"graph seed {seed} (E={g.n_edges}, V={g.n_vertices}): {ex}") from ex
