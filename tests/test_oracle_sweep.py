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


def _medium(seed):
    rng = np.random.default_rng(50_000 + seed)
    E = int(rng.integers(100, 301))
    V = int(rng.integers(10, 31))
    t_max = int(rng.integers(20, 201))
    return synth.random_small(E, V, t_max, 20_000 + seed, zipf_s=1.2 if seed % 3 == 0 else 0.0)


def test_condense_sweep_against_the_filtration():
    """Alg. 1's condensing and cluster extraction (the readings of HDBSCAN's
    condensed tree and excess of mass) against a restatement read directly
    off the filtration comps(L_G, w): labels, cluster count, every point's
    leaving lambda, and every cluster's birth, death, size, exact 128-bit
    stability and selection, for M = 2, 3, 4 and 5, on the small graphs and
    on 100 larger ones with deeper hierarchies."""
    graphs = [(_graph(s), 2 + s % 3) for s in range(N_GRAPHS)]
    graphs += [(_medium(s), 2 + s % 4) for s in range(100)]
    for seed, (g, M) in enumerate(graphs):
        full = bf.undirected_edges(g.src, g.dst, g.t)
        lab, ncl, fall, table = bf.condense_bruteforce(g.n_edges, full, M)
        c = O.run(g.src, g.dst, g.t, g.n_vertices, 2, M)["condensed"]
        got = sorted((int(b), int(d), int(s), (int(h) << 64) | int(lo), int(x)) for b, d, s, h, lo, x in
                     zip(c["cl_birth"], c["cl_death"], c["cl_size"], c["cl_stab_hi"], c["cl_stab_lo"],
                         c["cl_selected"]))
        where = f"graph {seed} (E={g.n_edges}, M={M})"
        assert np.array_equal(c["labels"], lab), where
        assert c["n_clusters"] == ncl, where
        assert [int(x) for x in c["fall_lambda"]] == fall, where
        assert got == table, where


def test_condense_tie_goes_to_the_parent():
    """An exact EOM tie (random graphs never give one): on the graph with
    links {0,1}, {2,3}, {4,5} at w = 2, {1,2} at 4 and {3,4} at 14, the
    lambdas are N/3, N/5, N/15 for N = 2^64 - 1 and 2 N/5 = N/3 + N/15, so
    the cluster {0..3} has exactly its children's summed stability. The
    oracle's chain and the filtration restatement both keep the parent."""
    edges = {(0, 1): 2, (2, 3): 2, (4, 5): 2, (1, 2): 4, (3, 4): 14}
    lab, ncl, _, table = bf.condense_bruteforce(6, edges, 2)
    u = np.array([a for a, _ in edges], np.int32)
    v = np.array([b for _, b in edges], np.int32)
    w = np.array(list(edges.values()), np.int64)
    mu, mv, mw = O.mst(6, u, v, w)
    a, b, s = O.linkage(6, mu, mv)
    c = O.condense(6, a, b, mw, s, 2)
    assert lab.tolist() == c["labels"].tolist() == [0, 0, 0, 0, 1, 1]
    assert ncl == c["n_clusters"] == 2
    selected = sorted(x[4] for x in table)
    assert selected == [0, 1, 1, 2, 2]                  # root, two covered children, two final


def test_discrete_condense_sweep_against_the_filtration():
    """Alg. 5 and condensing on D: with thresholds omega, D's levels are the
    filtration of L_G with every weight rounded up to the next threshold
    (links above the last one never join). The oracle's levels on L* and
    its condensing on D equal the restatement on that rounded explicit L_G:
    labels, cluster count and every cluster's birth, death, size, stability
    and selection."""
    omegas = [[0], [1, 4, 16, 64], [0, 2, 9], [0, 1, 2, 3, 5, 8, 13, 21], [2 ** i for i in range(29)]]
    for seed in range(0, N_GRAPHS, 4):
        g = _graph(seed)
        E, M = g.n_edges, 2 + seed % 3
        om = np.array(omegas[seed % len(omegas)], np.int64)
        full = bf.undirected_edges(g.src, g.dst, g.t)
        rounded = {}
        for key, x in full.items():
            i = int(np.searchsorted(om, x, side="left"))         # first threshold >= x
            if i < len(om):
                rounded[key] = int(om[i])
        lab, ncl, _, table = bf.condense_bruteforce(E, rounded, M)
        u, v, w = O.skeleton(g.src, g.dst, g.t, g.n_vertices)
        d = O.condense_levels(O.levels(E, u, v, w, om), om, M)
        got = sorted((int(b), int(dd), int(s), (int(h) << 64) | int(lo), int(x)) for b, dd, s, h, lo, x in
                     zip(d["cl_birth"], d["cl_death"], d["cl_size"], d["cl_stab_hi"], d["cl_stab_lo"],
                         d["cl_selected"]))
        where = f"graph seed {seed} (E={E}, M={M}, omega={om.tolist()})"
        assert np.array_equal(d["labels"], lab), where
        assert d["n_clusters"] == ncl, where
        assert got == table, where


def _same_condensed(c, ref, where):
    lab, ncl, fall, table = ref
    got = sorted((int(b), int(d), int(s), (int(h) << 64) | int(lo), int(x)) for b, d, s, h, lo, x in
                 zip(c["cl_birth"], c["cl_death"], c["cl_size"], c["cl_stab_hi"], c["cl_stab_lo"],
                     c["cl_selected"]))
    assert np.array_equal(c["labels"], lab), where
    assert c["n_clusters"] == ncl, where
    assert [int(x) for x in c["fall_lambda"]] == fall, where
    assert got == table, where


def test_variant_clusters_against_the_filtration():
    """The variants end to end against the restatement on their explicit
    line graphs: the time cutoff (only arcs with w <= delta, Sec. 4.3), the
    nearly-causal line graph (arcs back in time by at most delta, weighed
    |dt|, Sec. 4.3) and dynamic hypergraphs, undirected and directed
    (Sec. 4.4): labels, leaving lambdas and every cluster's birth, death,
    size, stability and selection."""
    for seed in range(0, N_GRAPHS, 5):
        g = _graph(seed)
        E, M = g.n_edges, 2 + seed % 3
        full = bf.undirected_edges(g.src, g.dst, g.t)
        delta = seed % 6
        cut = {key: x for key, x in full.items() if x <= delta}
        c = O.run(g.src, g.dst, g.t, g.n_vertices, 2, M, delta_max=delta)["condensed"]
        _same_condensed(c, bf.condense_bruteforce(E, cut, M), f"cutoff, graph seed {seed}, delta {delta}")
        dnc = 1 + seed % 4
        nc = bf.undirected_edges_nc(g.src, g.dst, g.t, dnc)
        c = O.run_nearly_causal(g.src, g.dst, g.t, g.n_vertices, 2, M, dnc)["condensed"]
        _same_condensed(c, bf.condense_bruteforce(E, nc, M), f"nearly causal, graph seed {seed}, delta {dnc}")
    for seed in range(200):
        rng = np.random.default_rng(70_000 + seed)
        mm = int(rng.integers(1, 5))                              # members per hyperedge, at most
        h = synth.hyper_small(int(rng.integers(1, 31)), int(rng.integers(2 * mm + 2, 2 * mm + 9)),
                              int(rng.integers(1, 13)), 30_000 + seed, directed=seed % 2 == 0, max_members=mm)
        M = 2 + seed % 3
        c = O.hyper_run(h.t, h.n_vertices, h.s_off, h.s_vert, h.d_off, h.d_vert, M)["condensed"]
        _same_condensed(c, bf.condense_bruteforce(h.n_edges, bf.hyper_line_graph(h), M),
                        f"hypergraph seed {seed}, directed {h.directed}")


def test_mutual_reachability_clusters_against_the_filtration():
    """The mutual-reachability mode end to end (an approximation; reading
    R-19): H = L* together with every node's kNN pairs taken by brute force
    from the explicit L_G, each pair once, weighed max(core_a, core_b, |dt|)
    with brute-force core distances, pairs with an infinite core dropped;
    the oracle's clusters equal the restatement's on that H, k = 1, 2, 3.
    The L* part of H is the oracle's own skeleton, so a skeleton defect would
    sit on both sides here: this pin relies on the separate Thm. 3 pin of
    O.skeleton against the explicit line graph; the kNN pairs and core
    distances are independent of the oracle."""
    for seed in range(0, N_GRAPHS, 7):
        g = _graph(seed)
        E, M, k = g.n_edges, 2 + seed % 3, 1 + seed % 3
        u, v, _ = O.skeleton(g.src, g.dst, g.t, g.n_vertices)
        ids, core = bf.knn_bruteforce(g.src, g.dst, g.t, k)
        pairs = set(zip(u.tolist(), v.tolist()))
        for e in range(E):
            for nb in ids[e].tolist():
                if nb >= 0:
                    pairs.add((min(e, nb), max(e, nb)))
        H = {}
        for a, b in pairs:
            x = max(int(core[a]), int(core[b]), abs(int(g.t[a]) - int(g.t[b])))
            if x != INF:
                H[(a, b)] = x
        c = O.mrd_run(g.src, g.dst, g.t, g.n_vertices, k, M)["condensed"]
        _same_condensed(c, bf.condense_bruteforce(E, H, M), f"mutual reachability, graph seed {seed}, k {k}")
