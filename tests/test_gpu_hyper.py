"""Dynamic hypergraphs (Sec. 4.4) on the GPU against the oracle, bit for bit:
per-vertex lists, skeleton, forest, dendrogram and labels."""
import numpy as np
import pytest

from gpu_helpers import ctx, run_gpu
from oracle import oracle as O
from paper_2311_10337_gb300 import synth

pytestmark = pytest.mark.gpu


def _dev(a, dt):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dt)).cuda()


def run_hyper(h):
    import torch
    out = ctx().run_hyper(_dev(h.t, np.int64), _dev(h.s_off, np.int64), _dev(h.s_vert, np.int32),
                          h.n_vertices, h.min_cluster_size,
                          _dev(h.d_off, np.int64) if h.directed else None,
                          _dev(h.d_vert, np.int32) if h.directed else None)
    torch.cuda.synchronize()
    r = {n: out.numpy(n) for n in ("src_voff", "src_list", "dst_voff", "dst_list", "sk_u", "sk_v", "sk_w",
                                   "mst_u", "mst_v", "mst_w", "link_a", "link_b", "link_size", "labels")}
    r["n_clusters"] = out.n_clusters
    return r


def _lists(h, off, vert):
    """Per-vertex hyperedge lists in (t, id) order, written out directly."""
    V = h.n_vertices
    rows = [[] for _ in range(V)]
    for e in range(h.n_edges):
        for i in vert[off[e]:off[e + 1]].tolist():
            rows[i].append(e)
    voff = np.zeros(V + 1, np.int64)
    lst = []
    for i in range(V):
        rows[i].sort(key=lambda e: (int(h.t[e]), e))
        voff[i + 1] = voff[i] + len(rows[i])
        lst += rows[i]
    return voff, np.array(lst, np.int32)


def compare_hyper(h):
    g = run_hyper(h)
    r = O.hyper_run(h.t, h.n_vertices, h.s_off, h.s_vert, h.d_off, h.d_vert, M=h.min_cluster_size)
    voff, lst = _lists(h, h.s_off, h.s_vert)
    assert np.array_equal(g["src_voff"], voff) and np.array_equal(g["src_list"], lst), "member lists"
    if h.directed:
        voff, lst = _lists(h, h.d_off, h.d_vert)
        assert np.array_equal(g["dst_voff"], voff) and np.array_equal(g["dst_list"], lst), "target lists"
    su, sv, sw = r["skeleton"]                   # a set: compare in (u, v) order
    o, q = np.lexsort((sv, su)), np.lexsort((g["sk_v"], g["sk_u"]))
    assert np.array_equal(g["sk_u"][q], su[o]) and np.array_equal(g["sk_v"][q], sv[o]), "skeleton pairs"
    assert np.array_equal(g["sk_w"][q], sw[o]), "skeleton weights"
    mu, mv, mw = r["mst"]
    assert np.array_equal(g["mst_u"], mu) and np.array_equal(g["mst_v"], mv) and np.array_equal(g["mst_w"], mw)
    a, b, s = r["linkage"]
    assert np.array_equal(g["link_a"], a) and np.array_equal(g["link_b"], b) and np.array_equal(g["link_size"], s)
    assert np.array_equal(g["labels"], r["condensed"]["labels"]), "labels"
    assert g["n_clusters"] == r["condensed"]["n_clusters"]
    return g


@pytest.mark.parametrize("directed", [False, True])
@pytest.mark.parametrize("seed", range(12))
def test_small_tie_heavy(directed, seed):
    h = synth.hyper_small(30 + 23 * seed, 10 + seed % 9, 2 + seed % 13, 100 + seed, directed,
                          max_members=2 + seed % 4, min_cluster_size=2 + seed % 3)
    compare_hyper(h)


@pytest.mark.parametrize("directed", [False, True])
@pytest.mark.parametrize("scale", [0.0005, 0.005])
def test_mail_scaled(directed, scale):
    compare_hyper(synth.hyper(scale=scale, directed=directed))


def test_graph_as_directed_hypergraph_matches_graph_path():
    g = synth.random_small(500, 40, 60, 17)
    off = np.arange(g.n_edges + 1, dtype=np.int64)
    h = synth.HyperWorkload("g", g.t, off, g.src, off, g.dst, g.n_vertices, 3, "graph")
    a = run_hyper(h)
    b = run_gpu(g.src, g.dst, g.t, g.n_vertices, 3, 3)
    o, q = np.lexsort((b["sk_v"], b["sk_u"])), np.lexsort((a["sk_v"], a["sk_u"]))
    assert np.array_equal(a["sk_u"][q], b["sk_u"][o]) and np.array_equal(a["sk_v"][q], b["sk_v"][o])
    for key in ("mst_u", "mst_v", "mst_w", "link_a", "link_b", "labels"):
        assert np.array_equal(a[key], b[key]), key


def test_degenerate_hypergraphs():
    # one vertex shared by every hyperedge, all at one time
    E = 300
    t = np.full(E, 5, np.int64)
    off = np.arange(E + 1, dtype=np.int64)
    compare_hyper(synth.HyperWorkload("star", t, off, np.zeros(E, np.int32), None, None, 1, 4, "star"))
    # hyperedges without members, and an empty hypergraph
    t = np.array([3, 1, 4, 1, 5], np.int64)
    off = np.array([0, 2, 2, 4, 4, 5], np.int64)
    compare_hyper(synth.HyperWorkload("holes", t, off, np.array([0, 1, 1, 2, 0], np.int32), None, None, 3, 2, ""))
    z = np.zeros(1, np.int64)
    compare_hyper(synth.HyperWorkload("empty", np.zeros(0, np.int64), z, np.zeros(0, np.int32), None, None, 4, 2, ""))


def test_hyper_errors():
    from paper_2311_10337_gb300 import dgec
    t = _dev(np.array([1, 2], np.int64), np.int64)
    off = _dev(np.array([0, 2, 3], np.int64), np.int64)
    cases = [
        (dict(s_off=off, s_vert=_dev(np.array([1, 1, 2], np.int32), np.int32), n_vertices=4), 3),
        (dict(s_off=off, s_vert=_dev(np.array([0, 1, 5], np.int32), np.int32), n_vertices=4), 2),
        (dict(s_off=_dev(np.array([0, 3, 2], np.int64), np.int64),
              s_vert=_dev(np.array([0, 1, 2], np.int32), np.int32), n_vertices=4), 1),
        (dict(s_off=_dev(np.array([0, 1, 2], np.int64), np.int64), s_vert=_dev(np.array([0, 1], np.int32), np.int32),
              d_off=_dev(np.array([0, 1, 2], np.int64), np.int64), d_vert=_dev(np.array([0, 3], np.int32), np.int32),
              n_vertices=4), 3),
    ]
    for kw, status in cases:
        with pytest.raises(dgec.DgecError) as e:
            ctx().run_hyper(t, min_cluster_size=2, **kw)
        assert e.value.status == status, kw
