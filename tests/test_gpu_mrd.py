"""Mutual-reachability mode on the GPU against the oracle, bit for bit: the
forest, dendrogram and labels of H = L* plus kNN pairs under mutual
reachability weights; at k = 1 it is the plain method."""
import numpy as np
import pytest

from gpu_helpers import ctx, run_gpu, sorted_skeleton
from oracle import oracle as O
from paper_2311_10337_gb300 import synth

pytestmark = pytest.mark.gpu
NAMES = ["sk_u", "sk_v", "sk_w", "knn_id", "core", "mst_u", "mst_v", "mst_w", "link_a", "link_b",
         "link_size", "labels"]


def run_mrd(src, dst, t, V, k, M, delta_max=None):
    import torch
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dt)).cuda()
    out = ctx().run(dev(src, np.int32), dev(dst, np.int32), dev(t, np.int64), V, k, M,
                    delta_max=delta_max, mrd=True)
    torch.cuda.synchronize()
    r = {n: out.numpy(n) for n in NAMES}
    r["n_clusters"] = out.n_clusters
    return r


def compare_mrd(src, dst, t, V, k, M, delta_max=None):
    g = run_mrd(src, dst, t, V, k, M, delta_max)
    r = O.mrd_run(src, dst, t, V, k, M, delta_max)
    # the skeleton outputs stay L*, the kNN lists are the usual ones
    su, sv, sw = (O.skeleton(src, dst, t, V) if delta_max is None
                  else O.skeleton_cutoff(src, dst, t, V, delta_max))
    gu, gv, gw = sorted_skeleton(g["sk_u"], g["sk_v"], g["sk_w"])
    assert np.array_equal(gu, su) and np.array_equal(gv, sv) and np.array_equal(gw, sw), "skeleton"
    ids, core = O.knn(src, dst, t, V, k, None, delta_max)
    assert np.array_equal(g["knn_id"].reshape(-1), ids.reshape(-1)) and np.array_equal(g["core"], core)
    mu, mv, mw = r["mst"]
    assert np.array_equal(g["mst_u"], mu) and np.array_equal(g["mst_v"], mv), "forest"
    assert np.array_equal(g["mst_w"], mw), "forest weights"
    a, b, s = r["linkage"]
    assert np.array_equal(g["link_a"], a) and np.array_equal(g["link_b"], b) and np.array_equal(g["link_size"], s)
    assert np.array_equal(g["labels"], r["condensed"]["labels"]), "labels"
    assert g["n_clusters"] == r["condensed"]["n_clusters"]
    return g


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("k", [1, 3, 8, 16])
def test_random_tie_heavy(seed, k):
    g = synth.random_small(50 + 37 * seed, 4 + seed % 7, 3 + seed % 11, 800 + seed,
                           zipf_s=1.3 if seed % 2 else 0.0)
    compare_mrd(g.src, g.dst, g.t, g.n_vertices, k, 2 + seed % 4)


def test_mid_scaled():
    w = synth.mid(scale=0.001)
    compare_mrd(w.src, w.dst, w.t, w.n_vertices, w.k, w.min_cluster_size)


def test_tiny_with_cutoff():
    w = synth.tiny()
    compare_mrd(w.src, w.dst, w.t, w.n_vertices, w.k, w.min_cluster_size, delta_max=20000)


def test_k1_is_the_plain_method():
    w = synth.mid(scale=0.0005)
    a = run_mrd(w.src, w.dst, w.t, w.n_vertices, 1, 5)
    b = run_gpu(w.src, w.dst, w.t, w.n_vertices, 1, 5)
    assert np.array_equal(np.sort(a["mst_w"]), np.sort(b["mst_w"]))
    assert np.array_equal(a["labels"], b["labels"])


def test_empty_and_host_entry():
    z32, z64 = np.zeros(0, np.int32), np.zeros(0, np.int64)
    g = run_mrd(z32, z32, z64, 3, 4, 5)
    assert g["n_clusters"] == 0 and len(g["labels"]) == 0
    w = synth.random_small(200, 12, 40, 5)
    dev = run_mrd(w.src, w.dst, w.t, w.n_vertices, 4, 3)
    lab, ncl = ctx().run_host(w.src, w.dst, w.t, w.n_vertices, 4, 3, mrd=True)
    assert np.array_equal(lab, dev["labels"]) and ncl == dev["n_clusters"]
