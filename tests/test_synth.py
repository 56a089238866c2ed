"""The seeded input generators: deterministic, every graph meets the input
assumptions of Sec. 1.2.1 (no self loops, no repeated (i, j, t) triple), and
each follows the recipe stated for it (sizes, ranges, time grids, degree
skew, member sets)."""
import numpy as np
import pytest

from paper_2311_10337_gb300 import synth

DAY = 86400


def _check_graph(src, dst, t, V):
    assert src.dtype == np.int32 and dst.dtype == np.int32 and t.dtype == np.int64
    assert len(src) == len(dst) == len(t)
    assert np.all((src >= 0) & (src < V) & (dst >= 0) & (dst < V))
    assert not np.any(src == dst)                                    # no self loops
    order = np.lexsort((t, dst, src))
    s, d, tt = src[order], dst[order], t[order]
    rep = (s[1:] == s[:-1]) & (d[1:] == d[:-1]) & (tt[1:] == tt[:-1])
    assert not np.any(rep)                                           # no repeated triple


@pytest.mark.parametrize("make", [
    lambda: synth.tiny(),
    lambda: synth.mid(scale=0.002),
    lambda: synth.hub(scale=0.001),
    lambda: synth.random_small(600, 8, 20, 3),
    lambda: synth.random_small(400, 30, 50, 4, zipf_s=1.3),
], ids=["tiny", "mid", "hub", "random", "random-zipf"])
def test_graphs_meet_the_input_assumptions(make):
    w = make()
    _check_graph(w.src, w.dst, w.t, w.n_vertices)


def test_generation_is_deterministic_per_seed():
    a, b = synth.mid(scale=0.001), synth.mid(scale=0.001)
    for x in ("src", "dst", "t"):
        assert np.array_equal(getattr(a, x), getattr(b, x)), x
    c = synth.mid(scale=0.001, seed_offset=1)
    assert not np.array_equal(a.t, c.t)


def test_sizes_and_time_ranges_follow_the_recipe():
    w = synth.tiny()
    assert (w.n_edges, w.n_vertices, w.k, w.min_cluster_size) == (20_000, 2_000, 4, 5)
    assert w.t.min() >= 0 and w.t.max() < 1_000_000 + 1_000   # U[0, 1e6), repeats moved by seconds
    m = synth.mid(scale=0.002)
    assert (m.n_edges, m.n_vertices, m.k, m.min_cluster_size) == (100_000, 2_000, 8, 5)
    assert m.t.min() >= 0 and m.t.max() < 31 * DAY               # 30-day span, bursts may run past it
    h = synth.hub(scale=0.001)
    assert (h.n_edges, h.n_vertices) == (200_000, 10_000)
    # half the edges on a 60 s grid and a tenth on an hourly one (about 60 %, less the repeats of a
    # pair in one slot that are moved by seconds), against 1/60 for uniform times
    assert np.mean(h.t % 60 == 0) > 0.5


def test_rank_zipf_endpoints_are_skewed_as_stated():
    """Rank-Zipf(2.1) over 2,000 vertices puts 1 / sum(r^-2.1) of the
    endpoint draws on the top vertex (about 64 %); self-loop resampling
    moves a little of it."""
    w = synth.tiny()
    V = w.n_vertices
    top = np.bincount(w.src, minlength=V).max() / w.n_edges
    p1 = 1.0 / np.sum(np.arange(1, V + 1, dtype=np.float64) ** -2.1)
    assert abs(p1 - 0.64) < 0.01
    assert 0.55 < top < 0.70


def test_batch_tables_and_graphs():
    b = synth.batch(24)
    eo = b.edge_off
    assert eo[0] == 0 and np.all(np.diff(eo) >= 1) and eo[-1] == len(b.src)
    sizes = np.diff(eo)
    assert np.all((sizes >= 1_000) & (sizes <= 1_000_000))
    assert np.array_equal(b.n_vertices, np.maximum(sizes // 10, 2).astype(np.int32))
    assert set(np.unique(b.k).tolist()) <= {4, 8, 16} and np.all(b.min_cluster_size == 5)
    for g in range(b.n_graphs):
        s, d, t = b.graph(g)
        _check_graph(s, d, t, int(b.n_vertices[g]))


def _check_rows(off, vert, V):
    assert off[0] == 0 and np.all(np.diff(off) >= 0) and off[-1] == len(vert)
    assert vert.dtype == np.int32 and np.all((vert >= 0) & (vert < V))
    row = np.repeat(np.arange(len(off) - 1, dtype=np.int64), np.diff(off))
    key = row * V + vert
    assert len(np.unique(key)) == len(key)                            # a vertex once per member set
    return row


@pytest.mark.parametrize("make", [
    lambda: synth.hyper(scale=0.0005, directed=True),
    lambda: synth.hyper_small(300, 12, 40, 5, directed=True),
    lambda: synth.hyper_small(300, 12, 40, 6, directed=False),
], ids=["mail", "small-directed", "small-undirected"])
def test_hypergraph_member_sets_are_valid(make):
    h = make()
    E, V = len(h.t), h.n_vertices
    assert h.t.dtype == np.int64 and len(h.s_off) == E + 1
    rs = _check_rows(h.s_off, h.s_vert, V)
    if h.directed:
        assert len(h.d_off) == E + 1
        rd = _check_rows(h.d_off, h.d_vert, V)
        both = np.intersect1d(rs * V + h.s_vert, rd * V + h.d_vert)
        assert len(both) == 0                                         # no vertex both source and target
        u = synth.undirected_of(h)
        assert np.array_equal(np.diff(u.s_off), np.diff(h.s_off) + np.diff(h.d_off))
        _check_rows(u.s_off, u.s_vert, V)


def test_broadcast_messages_have_one_sender():
    h = synth.hyper(scale=0.0005, directed=True)
    assert np.all(np.diff(h.s_off) == 1)
    nr = np.diff(h.d_off)
    assert nr.min() >= 1


@pytest.mark.parametrize("make", [lambda: synth.mid(scale=0.002), lambda: synth.hub(scale=0.001)],
                         ids=["mid", "hub"])
def test_skeleton_to_edge_ratio_is_plausible(make):
    """The paper's graphs have 1.78 (Reddit, Sec. 4.2.2) to 1.96 (e-mail,
    Sec. 4.1.2) skeleton links per edge; the synthetic stand-ins should look
    alike (about 1.9 at full size), within the bound of Sec. 2: at most
    sum_i (d_i - 1) = 2E - (vertices with an edge) links."""
    from oracle import oracle as O
    w = make()
    u, _, _ = O.skeleton(w.src, w.dst, w.t, w.n_vertices)
    deg = np.bincount(w.src, minlength=w.n_vertices) + np.bincount(w.dst, minlength=w.n_vertices)
    assert len(u) <= 2 * w.n_edges - int(np.sum(deg > 0))
    assert 1.75 < len(u) / w.n_edges < 2.0
