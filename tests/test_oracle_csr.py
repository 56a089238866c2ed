"""Pins of the oracle's incidence lists (orc_csr): the adjacency lists Alg. 3
starts from, each sorted by time as Alg. 2 sorts a vertex's edges (ties by
id, the reading used throughout).

The expected lists are built here by brute force, vertex by vertex, with a
plain Python sort of the vertex's incident edges by (t, id); the offsets are
the prefix sums of the degrees. Six arrays of the CUDA path (offsets, ids,
times and positions of both lists) are compared against this function, so a
wrong tie order here would move the GPU's expected values with it: the last
test plants exactly that mistake and shows the check catches it.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_10337_gb300 import synth
from test_oracle_pins import read_table


def _brute_lists(ends, t, V):
    """Per vertex v: the edges e with ends[e] == v, sorted by (t[e], e)."""
    E = len(ends)
    lists = [[] for _ in range(V)]
    for e in range(E):
        lists[int(ends[e])].append(e)
    off = [0]
    ids = []
    for v in range(V):
        lst = sorted(lists[v], key=lambda e: (int(t[e]), e))
        ids.extend(lst)
        off.append(len(ids))
    return np.array(off, np.int64), np.array(ids, np.int32)


def check_csr(src, dst, t, V, out_off, out_id, in_off, in_id):
    """Offsets equal the degree prefix sums; each vertex's list equals the
    brute-force (t, id) sort of its incident edges."""
    for ends, off, ids, side in ((src, out_off, out_id, "out"), (dst, in_off, in_id, "in")):
        deg = np.bincount(np.asarray(ends, np.int64), minlength=V) if len(ends) else np.zeros(V, np.int64)
        want_off = np.concatenate([[0], np.cumsum(deg)]).astype(np.int64)
        assert np.array_equal(off, want_off), f"{side}_off"
        b_off, b_ids = _brute_lists(ends, t, V)
        assert np.array_equal(b_off, want_off)
        assert np.array_equal(ids, b_ids), f"{side}_id"


def _sweep_graph(seed):
    rng = np.random.default_rng(seed)
    E = int(rng.integers(1, 41))
    V = int(rng.integers(2, 9))
    t_max = int(rng.integers(1, 13))
    return synth.random_small(E, V, t_max, 10_000 + seed, zipf_s=1.4 if seed % 7 == 0 else 0.0)


def test_csr_sweep_against_bruteforce():
    """The 2,000 tie-heavy sweep graphs (few vertices, few distinct times)."""
    for seed in range(2000):
        g = _sweep_graph(seed)
        oo, oi, io_, ii = O.csr(g.src, g.dst, g.t, g.n_vertices)
        check_csr(g.src, g.dst, g.t, g.n_vertices, oo, oi, io_, ii)


@pytest.mark.parametrize("name", ["chain_table.txt", "long_cluster_table.txt"])
def test_csr_paper_tables(name):
    """The two tables printed in the paper (Sec. 4.1.3), vertices renumbered
    densely."""
    src, dst, t, _ = read_table(name)
    verts, inv = np.unique(np.concatenate([src, dst]), return_inverse=True)
    s = inv[:len(src)].astype(np.int32)
    d = inv[len(src):].astype(np.int32)
    V = len(verts)
    oo, oi, io_, ii = O.csr(s, d, t, V)
    check_csr(s, d, t, V, oo, oi, io_, ii)


def test_csr_degenerate_inputs():
    """No edges; one vertex pair at one time; every edge at one time; a
    vertex with no edges between two that have some."""
    z32 = np.zeros(0, np.int32)
    oo, oi, io_, ii = O.csr(z32, z32, np.zeros(0, np.int64), 3)
    assert np.array_equal(oo, np.zeros(4, np.int64)) and len(oi) == 0
    check_csr(z32, z32, np.zeros(0, np.int64), 3, oo, oi, io_, ii)
    src = np.array([0, 2, 0, 2, 0], np.int32)
    dst = np.array([2, 0, 2, 0, 2], np.int32)
    t = np.array([7, 7, 7, 7, 7], np.int64)
    oo, oi, io_, ii = O.csr(src, dst, t, 3)
    check_csr(src, dst, t, 3, oo, oi, io_, ii)
    assert oi.tolist() == [0, 2, 4, 1, 3]       # ties at one time: ascending id


def test_csr_scaled_workloads():
    """The tiny workload and the three generators at small scale."""
    for g in (synth.tiny(), synth.mid(scale=0.0004), synth.hub(scale=0.0002),
              synth.random_small(3000, 40, 25, 5, zipf_s=1.2)):
        oo, oi, io_, ii = O.csr(g.src, g.dst, g.t, g.n_vertices)
        check_csr(g.src, g.dst, g.t, g.n_vertices, oo, oi, io_, ii)


def _plant_desc_id_ties(off, ids, t):
    """The oracle's lists with ties in t put in descending id order: the
    (t, -id) mistake a wrong comparator would make."""
    ids = ids.copy()
    for v in range(len(off) - 1):
        seg = ids[off[v]:off[v + 1]]
        ids[off[v]:off[v + 1]] = sorted(seg.tolist(), key=lambda e: (int(t[e]), -e))
    return ids


def _plant_id_only(off, ids, t):
    """The lists sorted by id alone (time ignored)."""
    ids = ids.copy()
    for v in range(len(off) - 1):
        ids[off[v]:off[v + 1]] = np.sort(ids[off[v]:off[v + 1]])
    return ids


@pytest.mark.parametrize("plant", [_plant_desc_id_ties, _plant_id_only], ids=["t,-id", "id-only"])
def test_planted_tie_order_is_caught(plant):
    """A mistake planted in the oracle's output (ties by descending id, or
    lists by id alone) fails the check on the sweep graphs."""
    caught = 0
    for seed in range(200):
        g = _sweep_graph(seed)
        oo, oi, io_, ii = O.csr(g.src, g.dst, g.t, g.n_vertices)
        bad_oi = plant(oo, oi, g.t)
        bad_ii = plant(io_, ii, g.t)
        if np.array_equal(bad_oi, oi) and np.array_equal(bad_ii, ii):
            continue                                # no tie (or no reorder) in this graph
        with pytest.raises(AssertionError):
            check_csr(g.src, g.dst, g.t, g.n_vertices, oo, bad_oi, io_, bad_ii)
        caught += 1
    assert caught > 100
