"""Parity at the largest configuration: the 200M-edge hub workload (10M
vertices; half the edges a Zipf(1.8) background on a 60 s grid, so the top
vertices carry tens of millions of edges and tie groups of thousands), run
through the benchmark's entry point and launch configuration (k = 8, M = 5,
the current stream).

The oracle's chain runs on the whole graph (Alg. 3's skeleton, then Alg. 1's
Kruskal forest, union-find dendrogram and condensing: minutes of single-core
C), so the skeleton set, the forest, the dendrogram rows, every
condensed-tree array and the labels are compared element by element. kNN
rows are recomputed one by one by the oracle for sampled edges, among them
edges whose tail or head is one of the largest hubs (their candidate sets
hold tens of millions of entries and their windows cross tie groups of
thousands). The
incidence lists are fixed exactly by their defining properties (offsets
from the degrees; each list a permutation sorted by (t, id)). The discrete
dendrogram's per-level component counts are checked against the forest."""
import numpy as np
import pytest

from gpu_helpers import ctx
from oracle import oracle as O
from paper_2311_10337_gb300 import synth

pytestmark = pytest.mark.gpu
POW2 = np.array([2 ** i for i in range(29)], np.int64)
CONDENSED = ["fall_cluster", "fall_lambda", "cl_id", "cl_parent", "cl_birth", "cl_death",
             "cl_stab_hi", "cl_stab_lo", "cl_size", "cl_selected"]


@pytest.fixture(scope="module")
def hub():
    import torch
    w = synth.hub(scale=1.0)
    s = torch.from_numpy(w.src).cuda()
    d = torch.from_numpy(w.dst).cuda()
    t = torch.from_numpy(w.t).cuda()
    out = ctx().run(s, d, t, w.n_vertices, w.k, w.min_cluster_size)
    names = ["out_off", "in_off", "out_t", "out_id", "in_id", "pos_out", "pos_in", "sk_u", "sk_v", "sk_w",
             "knn_id", "core", "mst_u", "mst_v", "mst_w", "link_a", "link_b", "link_size", "labels"] + CONDENSED
    r = {n: out.numpy(n) for n in names}
    r["n_clusters"] = out.n_clusters
    del out
    lv = ctx().run_levels(s, d, t, w.n_vertices, POW2, 0)
    r["n_components"] = lv.numpy("n_components")
    del s, d, t, lv
    ctx().ws = None
    torch.cuda.empty_cache()
    return w, r


@pytest.fixture(scope="module")
def chain(hub):
    """The oracle's whole clustering chain on the same graph."""
    w, _ = hub
    E = w.n_edges
    u, v, wt = O.skeleton(w.src, w.dst, w.t, w.n_vertices)       # sorted by (w, u, v)
    mu, mv, mw = O.mst(E, u, v, wt)
    a, b, s = O.linkage(E, mu, mv)
    c = O.condense(E, a, b, mw, s, w.min_cluster_size)
    return dict(skeleton=(u, v, wt), mst=(mu, mv, mw), linkage=(a, b, s), condensed=c)


def _pair_key_order(E, u, v):
    """Keys u * E + v and the permutation sorting them (torch's multi-threaded sort)."""
    import torch
    key = torch.from_numpy(u.astype(np.int64) * E + v.astype(np.int64))
    ks, o = torch.sort(key, stable=True)
    return ks.numpy(), o.numpy()


def test_incidence_lists(hub):
    w, r = hub
    E, V = w.n_edges, w.n_vertices
    for off, ids, pos, end in (("out_off", "out_id", "pos_out", w.src), ("in_off", "in_id", "pos_in", w.dst)):
        o, ids_ = r[off], r[ids]
        assert np.array_equal(o, np.concatenate([[0], np.cumsum(np.bincount(end, minlength=V))]))
        assert np.all(np.bincount(ids_, minlength=E) == 1)
        seg = np.repeat(np.arange(V, dtype=np.int32), np.diff(o))
        assert np.array_equal(end[ids_], seg)
        same = seg[1:] == seg[:-1]
        ta, tb = w.t[ids_[:-1]], w.t[ids_[1:]]
        ok = (ta < tb) | ((ta == tb) & (ids_[:-1] < ids_[1:]))
        assert np.all(ok[same]), off          # Alg. 2: each list sorted by (t, id)
        assert np.array_equal(r[pos][ids_], np.arange(E, dtype=np.int32)), pos
    assert np.array_equal(r["out_t"], w.t[r["out_id"]])


def test_skeleton(hub, chain):
    """Alg. 3's skeleton: the same set of (u, v, w) links as the oracle's."""
    w, r = hub
    E = w.n_edges
    ou, ov, ow = chain["skeleton"]
    assert len(r["sk_u"]) == len(ou)
    assert np.all(r["sk_u"] < r["sk_v"])
    gk, go = _pair_key_order(E, r["sk_u"], r["sk_v"])
    ok, oo = _pair_key_order(E, ou, ov)
    assert np.array_equal(gk, ok)
    assert np.array_equal(r["sk_w"][go], ow[oo])
    deg = np.bincount(w.src, minlength=w.n_vertices) + np.bincount(w.dst, minlength=w.n_vertices)
    assert len(ou) <= int(np.sum(np.maximum(deg - 1, 0)))      # size bound of Sec. 2


def _knn_rows(w, q):
    """The oracle's kNN rows of the query edges q, computed on the
    sub-multigraph they depend on (the queries, the in-edges of their tails,
    the out-edges of their heads; local ids keep the original id order)."""
    tails = np.zeros(w.n_vertices, bool)
    tails[w.src[q]] = True
    heads = np.zeros(w.n_vertices, bool)
    heads[w.dst[q]] = True
    keep = np.zeros(w.n_edges, bool)
    keep[q] = True
    keep |= tails[w.dst] | heads[w.src]
    sub = np.nonzero(keep)[0]
    lq = np.searchsorted(sub, q).astype(np.int32)
    ids, core = O.knn(w.src[sub], w.dst[sub], w.t[sub], w.n_vertices, w.k, lq)
    return np.where(ids >= 0, sub[np.maximum(ids, 0)], -1), core


def test_knn_sampled_light(hub):
    """1,000 sampled edges whose tail and head lists are short."""
    w, r = hub
    indeg = np.bincount(w.dst, minlength=w.n_vertices)
    outdeg = np.bincount(w.src, minlength=w.n_vertices)
    light = np.nonzero((indeg[w.src] <= 20000) & (outdeg[w.dst] <= 20000))[0]
    q = np.sort(np.random.default_rng(13).choice(light, 1000, replace=False))
    ids, core = _knn_rows(w, q)
    knn = r["knn_id"].reshape(w.n_edges, w.k)
    assert np.array_equal(knn[q], ids)
    assert np.array_equal(r["core"][q], core)


def test_knn_sampled_top_hubs(hub):
    """Edges whose tail has the largest in-list (tens of millions of
    predecessors, windows crossing tie groups of thousands on the 60 s grid)
    and edges whose head has the largest out-list."""
    w, r = hub
    indeg = np.bincount(w.dst, minlength=w.n_vertices)
    outdeg = np.bincount(w.src, minlength=w.n_vertices)
    rng = np.random.default_rng(17)
    hub_in = int(np.argmax(indeg))
    hub_out = int(np.argmax(outdeg))
    assert indeg[hub_in] > 1e7 and outdeg[hub_out] > 1e7
    q = np.concatenate([rng.choice(np.nonzero(w.src == hub_in)[0], 3, replace=False),
                        rng.choice(np.nonzero(w.dst == hub_out)[0], 3, replace=False)])
    q = np.unique(q)
    ids, core = _knn_rows(w, q)
    knn = r["knn_id"].reshape(w.n_edges, w.k)
    assert np.array_equal(knn[q], ids)
    assert np.array_equal(r["core"][q], core)


def test_forest(hub, chain):
    """Alg. 1, spanning forest: the oracle's Kruskal forest, element by element."""
    _, r = hub
    mu, mv, mw = chain["mst"]
    assert np.array_equal(r["mst_u"], mu) and np.array_equal(r["mst_v"], mv)
    assert np.array_equal(r["mst_w"], mw)


def test_dendrogram(hub, chain):
    """Alg. 1, dendrogram: the union-find replay's rows."""
    _, r = hub
    a, b, s = chain["linkage"]
    assert np.array_equal(r["link_a"], a) and np.array_equal(r["link_b"], b)
    assert np.array_equal(r["link_size"], s)


def test_condensed_tree_and_labels(hub, chain):
    """Alg. 1, condensing and extraction: every condensed-tree array, the
    stabilities and the selection, and the labels."""
    _, r = hub
    c = chain["condensed"]
    for key in CONDENSED:
        assert np.array_equal(r[key], c[key]), key
    assert np.array_equal(r["labels"], c["labels"])
    assert r["n_clusters"] == c["n_clusters"]


def test_levels_against_forest(hub, chain):
    """Alg. 5's component count at every threshold equals E minus the forest
    edges of weight <= the threshold (Thm. 1: the forest is sorted by w)."""
    w, r = hub
    mw = chain["mst"][2]
    nmst_at = np.searchsorted(mw, POW2, side="right")
    assert np.array_equal(r["n_components"], w.n_edges - nmst_at)
