"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: brute
force on the explicit line graph (Def. 1), Thm. 1-3 of the appendix, the
size bound of Sec. 2, and the worked examples printed in the paper.
"""
import json
import os

import numpy as np
import pytest

import bruteforce as bf
from oracle import oracle as O
from paper_2311_10337_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
INF = np.iinfo(np.int64).max


def read_table(name):
    """Parse a golden table: 'edges' rows of sender receiver [day] hh:mm:ss,
    then optional 'skeleton' rows."""
    src, dst, t, sk = [], [], [], []
    mode = None
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if not line:
            continue
        if line in ("edges", "skeleton"):
            mode = line
            continue
        f = line.split()
        if mode == "edges":
            day = int(f[2]) if len(f) == 4 else 0
            h, m, s = (int(x) for x in f[-1].split(":"))
            src.append(int(f[0])); dst.append(int(f[1]))
            t.append(day * 86400 + h * 3600 + m * 60 + s)
        else:
            sk.append(tuple(int(x) for x in f))
    return (np.array(src, np.int32), np.array(dst, np.int32),
            np.array(t, np.int64), sk)


def small_graphs():
    """Tie-heavy random graphs: few vertices, few distinct times, repeated
    pairs, reciprocal concurrent pairs."""
    out = []
    for seed in range(40):
        E = 5 + (seed * 7) % 60
        V = 3 + seed % 9
        tmax = 2 + seed % 11
        out.append(synth.random_small(E, V, tmax, seed))
    for seed in range(40, 46):
        out.append(synth.random_small(120, 12, 30, seed, zipf_s=1.5))
    return out


GRAPHS = small_graphs()


def test_chain_table_skeleton():
    """The paper's chain example: the skeleton is the path of record gaps
    1708, 1977, 291, 651 s."""
    src, dst, t, want = read_table("chain_table.txt")
    u, v, w = O.skeleton(src, dst, t, 1000)
    got = sorted(zip(u.tolist(), v.tolist(), w.tolist()), key=lambda x: (x[0], x[1]))
    assert got == sorted(want)


@pytest.mark.parametrize("g", GRAPHS + ["long"], ids=lambda g: getattr(g, "name", g))
def test_thm2_local_mst_equals_kruskal(g):
    """Thm. 2: per vertex, Alg. 2's output is Kruskal's MST of L_G(i) under
    the perturbed weights B_pq = t_q - t_p + gamma q - gamma^2 p (rows and
    columns 1-based in time order), i.e. key (w, q ascending, p descending)."""
    if g == "long":
        src, dst, t, _ = read_table("long_cluster_table.txt")
        V = 1000
    else:
        src, dst, t, V = g.src, g.dst, g.t, g.n_vertices
    p_raw, q_raw, w_raw, c_raw = O.skeleton_raw(src, dst, t, V)
    for i in range(V):
        ins, outs, arcs = bf.local_arcs(src, dst, t, i)
        ins = sorted(ins.tolist(), key=lambda e: (t[e], e))
        outs = sorted(outs.tolist(), key=lambda e: (t[e], e))
        prow = {e: x + 1 for x, e in enumerate(ins)}
        qcol = {e: x + 1 for x, e in enumerate(outs)}
        arcs.sort(key=lambda a: (a[2], qcol[a[1]], -prow[a[0]]))
        nodes = {e: x for x, e in enumerate(ins + outs)}
        uf = bf.UnionFind(len(nodes))
        kr = set()
        for p, q, w in arcs:
            if uf.union(nodes[p], nodes[q]):
                kr.add((p, q, w))
        mine = {(p, q, w) for p, q, w, c in zip(p_raw.tolist(), q_raw.tolist(),
                                                 w_raw.tolist(), c_raw.tolist()) if c == i}
        assert mine == kr, f"vertex {i}"


@pytest.mark.parametrize("g", GRAPHS, ids=lambda g: g.name)
def test_thm3_weighted_connectivity(g):
    """Thm. 3: comps(L*, w) == comps(L_G, w) for every threshold w, and the
    size bound |L*| <= sum_i (|E_i| - 1) of Sec. 2."""
    E = g.n_edges
    full = bf.undirected_edges(g.src, g.dst, g.t)
    u, v, w = O.skeleton(g.src, g.dst, g.t, g.n_vertices)
    sk = {(a, b): x for a, b, x in zip(u.tolist(), v.tolist(), w.tolist())}
    assert len(sk) == len(u)                       # no pair twice
    for key, x in sk.items():                      # L* is a subgraph of L_G
        assert full[key] == x
    for omega in sorted(set(full.values())) + [INF]:
        assert np.array_equal(bf.components(E, full, omega), bf.components(E, sk, omega))
    deg = np.bincount(g.src, minlength=g.n_vertices) + np.bincount(g.dst, minlength=g.n_vertices)
    assert len(u) <= int(np.sum(np.maximum(deg - 1, 0)))


def test_long_cluster_connectivity():
    src, dst, t, _ = read_table("long_cluster_table.txt")
    full = bf.undirected_edges(src, dst, t)
    u, v, w = O.skeleton(src, dst, t, 1000)
    sk = {(a, b): x for a, b, x in zip(u.tolist(), v.tolist(), w.tolist())}
    for omega in sorted(set(full.values())):
        assert np.array_equal(bf.components(11, full, omega), bf.components(11, sk, omega))


@pytest.mark.parametrize("g", GRAPHS[::3], ids=lambda g: g.name)
@pytest.mark.parametrize("k", [1, 3, 8])
def test_knn_bruteforce(g, k):
    """kNN / core distance against enumeration of the explicit L_G."""
    ids, core = O.knn(g.src, g.dst, g.t, g.n_vertices, k)
    bids, bcore = bf.knn_bruteforce(g.src, g.dst, g.t, k)
    assert np.array_equal(ids, bids)
    assert np.array_equal(core, bcore)


def _path_max_key(adj, a, b):
    """Largest (w, u, v) key on the forest path a..b, None if disconnected."""
    stack = [(a, None)]
    prev = {a: None}
    while stack:
        x, _ = stack.pop()
        if x == b:
            break
        for y, key in adj.get(x, []):
            if y not in prev:
                prev[y] = (x, key)
                stack.append((y, key))
    if b not in prev:
        return None
    best = None
    x = b
    while prev[x] is not None:
        x, key = prev[x]
        best = key if best is None or key > best else best
    return best


@pytest.mark.parametrize("g", GRAPHS, ids=lambda g: g.name)
def test_mst_cycle_property(g):
    """Alg. 1's spanning forest on L*: the forest spans L*'s components, and every
    skeleton edge outside it is the largest (w, u, v) key on the cycle it
    closes (the cycle characterisation of the unique MSF under a strict
    order); Thm. 1: its weight multiset equals that of an MSF of L_G."""
    E = g.n_edges
    u, v, w = O.skeleton(g.src, g.dst, g.t, g.n_vertices)
    mu, mv, mw = O.mst(E, u, v, w)
    keys = list(zip(mw.tolist(), mu.tolist(), mv.tolist()))
    assert keys == sorted(keys)
    adj = {}
    for ww, a, b in keys:
        adj.setdefault(a, []).append((b, (ww, a, b)))
        adj.setdefault(b, []).append((a, (ww, a, b)))
    inmst = set(keys)
    sk = {(a, b): x for a, b, x in zip(u.tolist(), v.tolist(), w.tolist())}
    for (a, b), x in sk.items():
        if (x, a, b) in inmst:
            continue
        best = _path_max_key(adj, a, b)
        assert best is not None and best < (x, a, b)
    assert np.array_equal(bf.components(E, sk, INF),
                          bf.components(E, {(a, b): x for x, a, b in keys}, INF))
    # Thm. 1: same sorted weights as an MSF of the full line graph
    full = bf.undirected_edges(g.src, g.dst, g.t)
    uf = bf.UnionFind(E)
    wf = [x for (a, b), x in sorted(full.items(), key=lambda kv: (kv[1], kv[0])) if uf.union(a, b)]
    assert wf == sorted(mw.tolist())


@pytest.mark.parametrize("g", GRAPHS[::2], ids=lambda g: g.name)
def test_linkage_ultrametric(g):
    """Alg. 1's dendrogram: the height at which two nodes first share a cluster of
    the dendrogram equals their minimax distance in L_G (Thm. 1 + 3)."""
    E = g.n_edges
    if E > 90:
        pytest.skip("all-pairs check kept to small graphs")
    u, v, w = O.skeleton(g.src, g.dst, g.t, g.n_vertices)
    mu, mv, mw = O.mst(E, u, v, w)
    a, b, size = O.linkage(E, mu, mv)
    n = len(a)
    assert np.all(np.diff(mw) >= 0)
    leaves = {x: [x] for x in range(E)}
    H = np.full((E, E), INF, np.int64)
    np.fill_diagonal(H, 0)
    for s in range(n):
        assert a[s] < b[s]
        A, B = leaves.pop(a[s]), leaves.pop(b[s])
        assert size[s] == len(A) + len(B)
        for x in A:
            for y in B:
                H[x, y] = H[y, x] = mw[s]
        leaves[E + s] = A + B
    D = bf.minimax(E, bf.undirected_edges(g.src, g.dst, g.t))
    assert np.array_equal(H, D)


def test_condense_golden():
    cases = json.load(open(os.path.join(GOLD, "condense_cases.json")))["cases"]
    for c in cases:
        rows = np.array(c["rows"], np.int64).reshape(-1, 4)
        r = O.condense(c["n_nodes"], rows[:, 0], rows[:, 1], rows[:, 2], rows[:, 3], c["M"])
        assert r["fall_cluster"].tolist() == c["fall_cluster"], c["note"]
        assert r["fall_lambda"].tolist() == [int(x) for x in c["fall_lambda"]]
        got = [[int(r["cl_id"][x]), int(r["cl_parent"][x]), str(int(r["cl_birth"][x])),
                str(int(r["cl_death"][x])), int(r["cl_size"][x]),
                str((int(r["cl_stab_hi"][x]) << 64) | int(r["cl_stab_lo"][x])),
                int(r["cl_selected"][x])] for x in range(len(r["cl_id"]))]
        assert got == c["clusters"], c["note"]
        assert r["labels"].tolist() == c["labels"]
        assert r["n_clusters"] == c["n_clusters"]


def _partition(labels):
    """Canonical form of a labelling: noise set + set of clusters."""
    groups = {}
    for x, l in enumerate(labels.tolist()):
        groups.setdefault(l, []).append(x)
    noise = tuple(groups.pop(-1, []))
    return noise, sorted(tuple(v) for v in groups.values())


def _bursts(n_bursts, size, gap_in, gap_out, seed):
    """Relay chains a->b->c->... of `size` records, `gap_in` s apart, bursts
    `gap_out` s apart, on disjoint vertex sets."""
    src, dst, t = [], [], []
    for b in range(n_bursts):
        base = b * gap_out
        for x in range(size):
            src.append(b * 100 + x); dst.append(b * 100 + x + 1)
            t.append(base + x * gap_in + (seed * x) % 3)
    return np.array(src, np.int32), np.array(dst, np.int32), np.array(t, np.int64)


def test_two_bursts_two_clusters():
    """Two relay chains of >= M records, far apart, are the two clusters."""
    src, dst, t = _bursts(2, 8, 10, 10_000, 0)
    # link the chains weakly through a shared vertex so there is one component
    src = np.append(src, 8); dst = np.append(dst, 100); t = np.append(t, 5_000)
    r = O.run(src, dst, t, 300, 3, 5)
    labels = r["condensed"]["labels"]
    assert r["condensed"]["n_clusters"] == 2
    assert len(set(labels[:8].tolist())) == 1 and len(set(labels[8:16].tolist())) == 1
    assert labels[0] != labels[8]


@pytest.mark.parametrize("g", GRAPHS[::4], ids=lambda g: g.name)
def test_labels_invariant_time_shift_and_relabel(g):
    """Labels depend only on weighted connectivity: invariant under a time
    shift, and the partition is invariant under renumbering the edges."""
    E = g.n_edges
    M = 3
    base = O.run(g.src, g.dst, g.t, g.n_vertices, 2, M)["condensed"]["labels"]
    shifted = O.run(g.src, g.dst, g.t + 123_456_789, g.n_vertices, 2, M)["condensed"]["labels"]
    assert np.array_equal(base, shifted)
    perm = np.random.default_rng(7).permutation(E)
    r = O.run(g.src[perm], g.dst[perm], g.t[perm], g.n_vertices, 2, M)["condensed"]["labels"]
    back = np.empty(E, np.int32)
    back[perm] = r
    assert _partition(back) == _partition(base)


@pytest.mark.parametrize("g", GRAPHS[::5], ids=lambda g: g.name)
def test_labels_from_filtration(g):
    """The labels are a function of comps(L_G, w) alone: rebuilding the
    hierarchy from thresholded components of the explicit line graph and
    condensing it gives the same partition."""
    E = g.n_edges
    M = 3
    full = bf.undirected_edges(g.src, g.dst, g.t)
    # build a linkage directly from the filtration: one merge per edge of an
    # arbitrary spanning forest of L_G taken in weight order
    uf = bf.UnionFind(E)
    forest = []
    for (a, b), x in sorted(full.items(), key=lambda kv: (kv[1], kv[0][1], kv[0][0])):
        if uf.union(a, b):
            forest.append((x, a, b))
    mu = np.array([f[1] for f in forest], np.int32)
    mv = np.array([f[2] for f in forest], np.int32)
    mw = np.array([f[0] for f in forest], np.int64)
    a, b, s = O.linkage(E, mu, mv)
    alt = O.condense(E, a, b, mw, s, M)["labels"]
    ref = O.run(g.src, g.dst, g.t, g.n_vertices, 2, M)["condensed"]["labels"]
    assert _partition(alt) == _partition(ref)


def test_validation_errors():
    with pytest.raises(ValueError):
        O.csr(np.array([0], np.int32), np.array([0], np.int32), np.array([1], np.int64), 2)
    with pytest.raises(ValueError):
        O.csr(np.array([0], np.int32), np.array([5], np.int32), np.array([1], np.int64), 2)


def test_empty_graph():
    z32 = np.zeros(0, np.int32)
    r = O.run(z32, z32, np.zeros(0, np.int64), 4, 3, 5)
    assert len(r["skeleton"][0]) == 0 and r["condensed"]["n_clusters"] == 0


@pytest.mark.parametrize("g", GRAPHS[::3], ids=lambda g: g.name)
def test_discrete_levels_match_line_graph(g):
    """Alg. 5 on the skeleton gives, at every threshold, the components of
    the explicit L_G (Thm. 3), each named by its smallest member."""
    E = g.n_edges
    u, v, w = O.skeleton(g.src, g.dst, g.t, g.n_vertices)
    full = bf.undirected_edges(g.src, g.dst, g.t)
    omega = np.array(sorted(set(full.values()) | {0, 1, 2, 4, 8}), np.int64)
    lv = O.levels(E, u, v, w, omega)
    for i, om in enumerate(omega.tolist()):
        assert np.array_equal(lv[i], bf.components(E, full, om)), om


def test_discrete_levels_nested():
    """Levels are nested: a component at a lower threshold lies inside one
    component at every higher threshold (the containment tree D)."""
    g = synth.random_small(300, 20, 200, 3)
    u, v, w = O.skeleton(g.src, g.dst, g.t, g.n_vertices)
    omega = np.array([0, 1, 3, 7, 15, 31, 63, 127], np.int64)
    lv = O.levels(g.n_edges, u, v, w, omega)
    for i in range(1, len(omega)):
        parent = {}
        for x in range(g.n_edges):
            assert parent.setdefault(lv[i - 1][x], lv[i][x]) == lv[i][x]


def _cluster_rows(d):
    """Cluster table as a sorted list of (birth, death, size, stability,
    selected): ids are numbering conventions, these values are not."""
    rows = zip(d["cl_birth"].tolist(), d["cl_death"].tolist(), d["cl_size"].tolist(),
               d["cl_stab_hi"].tolist(), d["cl_stab_lo"].tolist(), d["cl_selected"].tolist())
    return sorted(rows)


def _continuous(g, M, rounding=None):
    """Alg. 1 on the skeleton; with `rounding`, every weight is first
    replaced by the smallest threshold >= it and edges above the last
    threshold are dropped."""
    E = g.n_edges
    u, v, w = O.skeleton(g.src, g.dst, g.t, g.n_vertices)
    if rounding is not None:
        om = np.asarray(rounding, np.int64)
        b = np.searchsorted(om, w, side="left")
        keep = b < len(om)
        u, v, w = u[keep], v[keep], om[b[keep]]
    mu, mv, mw = O.mst(E, u, v, w)
    a, bb, s = O.linkage(E, mu, mv)
    return O.condense(E, a, bb, mw, s, M)


@pytest.mark.parametrize("g", GRAPHS[::4], ids=lambda g: g.name)
@pytest.mark.parametrize("M", [2, 3, 5])
def test_discrete_condense_full_resolution(g, M):
    """With one threshold per distinct weight of L*, the discrete dendrogram
    loses nothing (Sec. 3): condensing it gives the continuous result."""
    u, v, w = O.skeleton(g.src, g.dst, g.t, g.n_vertices)
    if len(w) == 0:
        pytest.skip("no skeleton edges")
    omega = np.unique(w)
    lv = O.levels(g.n_edges, u, v, w, omega)
    d = O.condense_levels(lv, omega, M)
    c = _continuous(g, M)
    assert np.array_equal(d["labels"], c["labels"])
    assert d["n_clusters"] == c["n_clusters"]
    assert _cluster_rows(d) == _cluster_rows(c)


@pytest.mark.parametrize("g", GRAPHS[1::4], ids=lambda g: g.name)
@pytest.mark.parametrize("omega", [[0, 2, 9], [1, 4, 16, 64], [3], [0, 1, 2, 3, 5, 8, 13, 21]])
def test_discrete_condense_is_rounded_continuous(g, omega):
    """Coarse thresholds: the discrete dendrogram is the single-linkage
    dendrogram of weights rounded up to the next threshold (edges above the
    last one never join), so both condense to the same clusters."""
    u, v, w = O.skeleton(g.src, g.dst, g.t, g.n_vertices)
    om = np.array(omega, np.int64)
    lv = O.levels(g.n_edges, u, v, w, om)
    d = O.condense_levels(lv, om, 3)
    c = _continuous(g, 3, rounding=om)
    assert np.array_equal(d["labels"], c["labels"])
    assert _cluster_rows(d) == _cluster_rows(c)


def test_discrete_condense_one_level_closed_form():
    """One level above every weight: the clusters are the components of L*
    with >= M members (when there are two or more of them), each born at
    lambda 0 with stability |C| * lambda(omega_1)."""
    lam = lambda x: (2**64 - 1) // (x + 1)
    for seed in range(6):
        g = synth.random_small(90, 40, 50, 100 + seed)
        u, v, w = O.skeleton(g.src, g.dst, g.t, g.n_vertices)
        om = np.array([int(w.max()) + 7 if len(w) else 7], np.int64)
        lv = O.levels(g.n_edges, u, v, w, om)
        M = 4
        d = O.condense_levels(lv, om, M)
        comp = bf.components(g.n_edges, {(a, b): x for a, b, x in zip(u.tolist(), v.tolist(), w.tolist())}, INF)
        sizes = np.bincount(comp, minlength=g.n_edges)
        big = [c for c in range(g.n_edges) if sizes[c] >= M]
        want = np.full(g.n_edges, -1, np.int32)
        if len(big) >= 2:
            for r, c in enumerate(sorted(big)):      # a component's name is its smallest member
                want[comp == c] = r
            stab = [int(sizes[c]) * lam(int(om[0])) for c in big]      # exact, may pass 2^64
            rows = [(0, 0, int(sizes[c]), s >> 64, s & (2**64 - 1), 2) for c, s in zip(big, stab)]
            assert [r for r in _cluster_rows(d) if r[2] < g.n_edges] == sorted(rows)
        assert np.array_equal(d["labels"], want), seed


@pytest.mark.parametrize("g", GRAPHS[2::5], ids=lambda g: g.name)
def test_levels_tree(g):
    """D per node: x stops naming its component exactly at the first level
    whose component has a smaller member, and is then inside the component
    named merge_parent; per level the names are the nodes not yet merged."""
    u, v, w = O.skeleton(g.src, g.dst, g.t, g.n_vertices)
    omega = np.array([0, 1, 2, 4, 8, 16], np.int64)
    lv = O.levels(g.n_edges, u, v, w, omega)
    ml, mp = O.levels_tree(lv)
    full = bf.undirected_edges(g.src, g.dst, g.t)
    for i, om in enumerate(omega.tolist()):
        comp = bf.components(g.n_edges, full, om)
        names = set(int(c) for c in comp)
        assert names == {x for x in range(g.n_edges) if ml[x] == -1 or ml[x] > i}
        for x in range(g.n_edges):
            if ml[x] == i:
                assert mp[x] == comp[x] and mp[x] < x


@pytest.mark.parametrize("g", GRAPHS[::3], ids=lambda g: g.name)
@pytest.mark.parametrize("delta", [0, 1, 3, 10])
def test_cutoff_line_graph(g, delta):
    """Time cutoff of Sec. 4.3 (arcs with w <= delta_max only): the filtered
    skeleton has the components of the explicit filtered L_G at every
    threshold, its forest the weights of Kruskal on the filtered L_G, and the
    kNN lists those of enumerating the filtered L_G."""
    E = g.n_edges
    full = {k: w for k, w in bf.undirected_edges(g.src, g.dst, g.t).items() if w <= delta}
    u, v, w = O.skeleton_cutoff(g.src, g.dst, g.t, g.n_vertices, delta)
    sk = {(a, b): x for a, b, x in zip(u.tolist(), v.tolist(), w.tolist())}
    assert all(full[key] == x for key, x in sk.items())
    for om in sorted(set(full.values())) + [INF]:
        assert np.array_equal(bf.components(E, full, om), bf.components(E, sk, om))
    mu, mv, mw = O.mst(E, u, v, w)
    uf = bf.UnionFind(E)
    wf = [x for (a, b), x in sorted(full.items(), key=lambda kv: (kv[1], kv[0])) if uf.union(a, b)]
    assert wf == sorted(mw.tolist())
    for k in (1, 4):
        ids, core = O.knn(g.src, g.dst, g.t, g.n_vertices, k, delta_max=delta)
        bids, bcore = bf.knn_bruteforce(g.src, g.dst, g.t, k, delta_max=delta)
        assert np.array_equal(ids, bids) and np.array_equal(core, bcore)


def test_cutoff_above_every_weight_is_no_cutoff():
    g = synth.random_small(200, 20, 60, 31)
    a = O.run(g.src, g.dst, g.t, g.n_vertices, 4, 3)
    b = O.run(g.src, g.dst, g.t, g.n_vertices, 4, 3, delta_max=10 ** 12)
    assert np.array_equal(a["condensed"]["labels"], b["condensed"]["labels"])
    assert all(np.array_equal(x, y) for x, y in zip(a["knn"], b["knn"]))
