"""Discrete dendrogram (Alg. 5) and condensing on it: the CUDA path against
the oracle, element by element (all integer, so bit-exact)."""
import numpy as np
import pytest

from gpu_helpers import ctx, run_gpu, sorted_skeleton
from oracle import oracle as O
from paper_2311_10337_gb300 import synth

pytestmark = pytest.mark.gpu

POW2 = np.array([2 ** i for i in range(29)], np.int64)   # 1 s .. 2^28 s, as in Sec. 4.2.2


def run_levels(src, dst, t, V, omega, M=0, dense=True):
    import torch
    s = torch.from_numpy(np.ascontiguousarray(src, np.int32)).cuda()
    d = torch.from_numpy(np.ascontiguousarray(dst, np.int32)).cuda()
    tt = torch.from_numpy(np.ascontiguousarray(t, np.int64)).cuda()
    out = ctx().run_levels(s, d, tt, V, omega, M, dense)
    torch.cuda.synchronize()
    r = {n: out.numpy(n) for n in ("sk_u", "sk_v", "sk_w", "merge_level", "merge_parent",
                                   "n_components", "level_labels", "labels")}
    r["n_merges"] = out.n_merges
    r["n_clusters"] = out.n_clusters
    return r


def oracle_levels(src, dst, t, V, omega, M=0):
    E = len(src)
    u, v, w = O.skeleton(src, dst, t, V)
    lv = O.levels(E, u, v, w, omega)
    ml, mp = O.levels_tree(lv)
    ncomp = np.array([int(np.sum(lv[i] == np.arange(E))) for i in range(len(omega))], np.int64)
    out = dict(skeleton=(u, v, w), level_labels=lv, merge_level=ml, merge_parent=mp, n_components=ncomp)
    if M:
        out["condensed"] = O.condense_levels(lv, omega, M)
    return out


def compare_levels(src, dst, t, V, omega, M):
    omega = np.asarray(omega, np.int64)
    g = run_levels(src, dst, t, V, omega, M)
    r = oracle_levels(src, dst, t, V, omega, M)
    E = len(src)
    su, sv, sw = r["skeleton"]
    gu, gv, gw = sorted_skeleton(g["sk_u"], g["sk_v"], g["sk_w"])
    assert np.array_equal(gu, su) and np.array_equal(gv, sv) and np.array_equal(gw, sw), "skeleton"
    assert np.array_equal(g["level_labels"], r["level_labels"]), "level labels"
    assert np.array_equal(g["merge_level"], r["merge_level"]), "merge_level"
    assert np.array_equal(g["merge_parent"], r["merge_parent"]), "merge_parent"
    assert np.array_equal(g["n_components"], r["n_components"]), "n_components"
    assert g["n_merges"] == E - (int(r["n_components"][-1]) if E else 0)
    if M:
        c = r["condensed"]
        assert np.array_equal(g["labels"], c["labels"]), "condensed labels"
        assert g["n_clusters"] == c["n_clusters"]
    return g


def test_tiny_power_of_two_thresholds():
    w = synth.tiny()
    compare_levels(w.src, w.dst, w.t, w.n_vertices, POW2, w.min_cluster_size)


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("omega", [[0, 1, 2, 4, 8], [3], [0], [1, 10, 100, 1000], list(range(0, 64))])
def test_random_tie_heavy(seed, omega):
    g = synth.random_small(40 + 37 * seed, 4 + seed % 7, 3 + seed % 13, 500 + seed,
                           zipf_s=1.3 if seed % 2 else 0.0)
    compare_levels(g.src, g.dst, g.t, g.n_vertices, omega, 2 + seed % 3)


@pytest.mark.parametrize("scale", [0.0004, 0.002])
def test_mid_scaled(scale):
    w = synth.mid(scale=scale)
    compare_levels(w.src, w.dst, w.t, w.n_vertices, POW2, w.min_cluster_size)


def test_hub_scaled():
    w = synth.hub(scale=0.0003)
    compare_levels(w.src, w.dst, w.t, w.n_vertices, POW2, w.min_cluster_size)


def test_degenerate_cases():
    # every link has weight 0: one level joins all
    src = np.array([0, 1, 2, 0, 1], np.int32)
    dst = np.array([1, 2, 0, 2, 0], np.int32)
    t = np.full(5, 7, np.int64)
    compare_levels(src, dst, t, 3, [0], 2)
    # thresholds below every weight: nothing merges
    g = synth.random_small(80, 6, 40, 9)
    out = compare_levels(g.src, g.dst, g.t, g.n_vertices, [0], 2)
    if np.all(out["sk_w"] > 0):
        assert out["n_merges"] == 0 and np.all(out["merge_level"] == -1)
    # a single edge, and no edges
    compare_levels(np.array([0], np.int32), np.array([1], np.int32), np.array([3], np.int64), 2, POW2, 2)
    compare_levels(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64), 4, POW2, 5)
    # the largest number of thresholds
    compare_levels(g.src, g.dst, g.t, g.n_vertices, list(range(64)), 3)


def test_full_resolution_equals_continuous():
    """One threshold per distinct skeleton weight: the discrete labels are
    those of the continuous pipeline (Sec. 3: nothing is lost)."""
    for seed in range(4):
        g = synth.random_small(300, 30, 40, 700 + seed)
        cont = run_gpu(g.src, g.dst, g.t, g.n_vertices, 4, 3)
        om = np.unique(cont["sk_w"])
        assert len(om) <= 64
        lv = run_levels(g.src, g.dst, g.t, g.n_vertices, om, 3, dense=False)
        assert np.array_equal(lv["labels"], cont["labels"])
        assert lv["n_clusters"] == cont["n_clusters"]


def test_sparse_outputs_match_dense_run_and_repeat():
    w = synth.mid(scale=0.001)
    a = run_levels(w.src, w.dst, w.t, w.n_vertices, POW2, 0, dense=False)
    assert a["level_labels"] is None and a["labels"] is None
    b = run_levels(w.src, w.dst, w.t, w.n_vertices, POW2, 5, dense=True)
    c = run_levels(w.src, w.dst, w.t, w.n_vertices, POW2, 5, dense=True)
    for k in ("merge_level", "merge_parent", "n_components"):
        assert np.array_equal(a[k], b[k]), k
    for k in ("merge_level", "merge_parent", "level_labels", "labels"):
        assert np.array_equal(b[k], c[k]), k


def test_levels_errors():
    import torch
    from paper_2311_10337_gb300 import dgec
    s = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    d = torch.tensor([1, 0], dtype=torch.int32, device="cuda")
    t = torch.tensor([0, 1], dtype=torch.int64, device="cuda")
    for omega, M in (([2, 2], 0), ([3, 1], 0), ([-1, 4], 0), ([], 0), (list(range(65)), 0), ([1], 1)):
        with pytest.raises(dgec.DgecError) as e:
            ctx().run_levels(s, d, t, 2, omega, M)
        assert e.value.status == 1
    with pytest.raises(dgec.DgecError) as e:   # vertex out of range
        ctx().run_levels(s, d, t, 1, [1], 0)
    assert e.value.status == 2
