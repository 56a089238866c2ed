"""Parity at the full benchmark size: the 50M-edge mid workload, run through
the same entry points and launch configuration the benchmark times (k = 8,
M = 5, the current stream; the discrete dendrogram at 2^0 .. 2^28 s).

The oracle's chain runs on the whole graph (Alg. 3's skeleton, then Alg. 1's
Kruskal forest, union-find dendrogram and condensing: a few minutes of
single-core C), so the skeleton set, the forest, the dendrogram rows, every
condensed-tree array and the labels are compared element by element. The
oracle's kNN rows are recomputed one by one for sampled edges. The incidence
lists are fixed exactly by their defining properties (offsets from the
degrees; each list a permutation sorted by (t, id)). The discrete dendrogram,
whose oracle repeats a union-find per threshold, is checked through Thm. 3 at
two thresholds against scipy's components of the skeleton and through every
level's component count against the forest."""
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
def full():
    import torch
    w = synth.mid(scale=1.0)
    s = torch.from_numpy(w.src).cuda()
    d = torch.from_numpy(w.dst).cuda()
    t = torch.from_numpy(w.t).cuda()
    out = ctx().run(s, d, t, w.n_vertices, w.k, w.min_cluster_size)
    names = ["out_off", "in_off", "out_t", "in_t", "out_id", "in_id", "pos_out", "pos_in", "sk_u", "sk_v",
             "sk_w", "knn_id", "core", "mst_u", "mst_v", "mst_w", "link_a", "link_b", "link_size",
             "labels"] + CONDENSED
    r = {n: out.numpy(n) for n in names}
    r["n_clusters"] = out.n_clusters
    lv = ctx().run_levels(s, d, t, w.n_vertices, POW2, w.min_cluster_size)
    r["merge_level"] = lv.numpy("merge_level")
    r["merge_parent"] = lv.numpy("merge_parent")
    r["n_components"] = lv.numpy("n_components")
    r["lv_labels"] = lv.numpy("labels")
    r["lv_n_clusters"] = lv.n_clusters
    del s, d, t, out, lv
    ctx().ws = None
    torch.cuda.empty_cache()
    r["n_comp"], r["comp"] = _components(w.n_edges, r["sk_u"], r["sk_v"])
    return w, r


@pytest.fixture(scope="module")
def chain(full):
    """The oracle's whole clustering chain on the same graph."""
    w, _ = full
    E = w.n_edges
    u, v, wt = O.skeleton(w.src, w.dst, w.t, w.n_vertices)       # sorted by (w, u, v)
    mu, mv, mw = O.mst(E, u, v, wt)
    a, b, s = O.linkage(E, mu, mv)
    c = O.condense(E, a, b, mw, s, w.min_cluster_size)
    return dict(skeleton=(u, v, wt), mst=(mu, mv, mw), linkage=(a, b, s), condensed=c)


def _pair_order(E, u, v):
    key = u.astype(np.int64) * E + v
    o = np.argsort(key, kind="stable")
    return key[o], o


def _csgraph(E, u, v):
    sp = pytest.importorskip("scipy.sparse")
    return sp.coo_matrix((np.ones(len(u), np.int8), (u, v)), shape=(E, E)).tocsr()


def _components(E, u, v):
    cg = pytest.importorskip("scipy.sparse.csgraph")
    n, lab = cg.connected_components(_csgraph(E, u, v), directed=False)
    return n, lab


def _min_member_names(lab):
    """Name every component by its smallest member."""
    E = len(lab)
    first = np.full(lab.max() + 1 if E else 0, E, np.int64)
    np.minimum.at(first, lab, np.arange(E))
    return first[lab].astype(np.int32)


def test_incidence_lists(full):
    w, r = full
    E, V = w.n_edges, w.n_vertices
    for off, ids, tt, pos, end in (("out_off", "out_id", "out_t", "pos_out", w.src),
                                   ("in_off", "in_id", "in_t", "pos_in", w.dst)):
        o, ids_ = r[off], r[ids]
        assert np.array_equal(o, np.concatenate([[0], np.cumsum(np.bincount(end, minlength=V))]))
        assert np.all(np.bincount(ids_, minlength=E) == 1)          # a permutation of the edges
        seg = np.repeat(np.arange(V, dtype=np.int32), np.diff(o))
        assert np.array_equal(end[ids_], seg)
        same = seg[1:] == seg[:-1]
        ta, tb = w.t[ids_[:-1]], w.t[ids_[1:]]
        ok = (ta < tb) | ((ta == tb) & (ids_[:-1] < ids_[1:]))
        assert np.all(ok[same]), off          # Alg. 2: each list sorted by (t, id)
        assert np.array_equal(r[tt], w.t[ids_]), tt
        assert np.array_equal(r[pos][ids_], np.arange(E, dtype=np.int32)), pos


def test_skeleton(full, chain):
    """Alg. 3's skeleton: the same set of (u, v, w) links as the oracle's."""
    w, r = full
    E = w.n_edges
    ou, ov, ow = chain["skeleton"]
    assert len(r["sk_u"]) == len(ou)
    assert np.all(r["sk_u"] < r["sk_v"])
    gk, go = _pair_order(E, r["sk_u"], r["sk_v"])
    ok, oo = _pair_order(E, ou, ov)
    assert np.array_equal(gk, ok)
    assert np.array_equal(r["sk_w"][go], ow[oo])


def test_knn_sampled(full):
    """kNN rows of sampled edges, by the oracle on the sub-multigraph they
    depend on: the sampled edges, the in-edges of their tails and the
    out-edges of their heads (local ids keep the original id order)."""
    w, r = full
    rng = np.random.default_rng(11)
    q = np.sort(rng.choice(w.n_edges, 3000, replace=False))
    tails = np.zeros(w.n_vertices, bool); tails[w.src[q]] = True
    heads = np.zeros(w.n_vertices, bool); heads[w.dst[q]] = True
    keep = np.zeros(w.n_edges, bool)
    keep[q] = True
    keep |= tails[w.dst] | heads[w.src]
    sub = np.nonzero(keep)[0]
    lq = np.searchsorted(sub, q).astype(np.int32)
    ids, core = O.knn(w.src[sub], w.dst[sub], w.t[sub], w.n_vertices, w.k, lq)
    ids = np.where(ids >= 0, sub[np.maximum(ids, 0)], -1)
    knn = r["knn_id"].reshape(w.n_edges, w.k)
    assert np.array_equal(knn[q], ids)
    assert np.array_equal(r["core"][q], core)


def test_forest(full, chain):
    """Alg. 1, spanning forest: the oracle's Kruskal forest, element by element, and
    one tree per component of the skeleton."""
    w, r = full
    mu, mv, mw = chain["mst"]
    assert np.array_equal(r["mst_u"], mu) and np.array_equal(r["mst_v"], mv)
    assert np.array_equal(r["mst_w"], mw)
    assert len(mu) == w.n_edges - r["n_comp"]


def test_dendrogram(full, chain):
    """Alg. 1, dendrogram: the union-find replay's rows."""
    _, r = full
    a, b, s = chain["linkage"]
    assert np.array_equal(r["link_a"], a) and np.array_equal(r["link_b"], b)
    assert np.array_equal(r["link_size"], s)


def test_condensed_tree_and_labels(full, chain):
    """Alg. 1, condensing and extraction: every condensed-tree array, the stabilities and
    the selection, and the labels."""
    _, r = full
    c = chain["condensed"]
    for key in CONDENSED:
        assert np.array_equal(r[key], c[key]), key
    assert np.array_equal(r["labels"], c["labels"])
    assert r["n_clusters"] == c["n_clusters"]


def test_labels_lie_in_components(full):
    w, r = full
    E = w.n_edges
    comp = r["comp"]
    for lab, ncl in ((r["labels"], r["n_clusters"]), (r["lv_labels"], r["lv_n_clusters"])):
        m = lab >= 0
        assert lab.max() + 1 == ncl
        # one component per cluster
        cmin = np.full(ncl, E, np.int64); cmax = np.full(ncl, -1, np.int64)
        np.minimum.at(cmin, lab[m], comp[m]); np.maximum.at(cmax, lab[m], comp[m])
        assert np.array_equal(cmin, cmax)
        # clusters numbered by their smallest member: first appearances are 0, 1, 2, ...
        _, first = np.unique(lab[m], return_index=True)
        assert np.all(np.diff(np.nonzero(m)[0][first]) > 0)
        assert np.all(np.bincount(lab[m]) >= w.min_cluster_size)


def test_levels(full):
    """Thm. 3 at two thresholds against scipy's components of the skeleton,
    and every level's component count against the forest (Thm. 1)."""
    w, r = full
    E = w.n_edges
    ml, mp = r["merge_level"], r["merge_parent"]
    merged = ml >= 0
    assert np.all(mp[merged] < np.nonzero(merged)[0]) and np.all(mp[~merged] == -1)
    nmst_at = np.searchsorted(r["mst_w"], POW2, side="right")    # the forest is sorted by w
    assert np.array_equal(r["n_components"], E - nmst_at)
    for li in (0, 10):
        keep = r["sk_w"] <= POW2[li]
        _, comp = _components(E, r["sk_u"][keep], r["sk_v"][keep])
        want = _min_member_names(comp)
        lab = np.arange(E, dtype=np.int32)
        step = (ml >= 0) & (ml <= li)
        lab[step] = mp[step]
        for _ in range(64):                      # follow D up to level li
            nxt = lab.copy()
            go = (ml[lab] >= 0) & (ml[lab] <= li)
            nxt[go] = mp[lab[go]]
            if np.array_equal(nxt, lab):
                break
            lab = nxt
        assert np.array_equal(lab, want), li
