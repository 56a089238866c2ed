"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

All outputs are integers, so the bar is bit-exact equality of every array:
incidence lists, skeleton (as a set), kNN ids and core distances, the
minimum spanning forest in (w, u, v) order, the dendrogram rows, the
condensed tree, stabilities and labels.
"""
import numpy as np
import pytest

from gpu_helpers import compare_all, run_gpu
from oracle import oracle as O
from paper_2311_10337_gb300 import synth

pytestmark = pytest.mark.gpu


def test_tiny_workload_all_outputs():
    w = synth.tiny()
    compare_all(w.src, w.dst, w.t, w.n_vertices, w.k, w.min_cluster_size)


@pytest.mark.parametrize("seed", range(12))
def test_random_tie_heavy(seed):
    E = [1, 2, 5, 40, 100, 333, 1000, 2047, 2048, 2049, 4500, 9000][seed]
    V = max(2, [2, 3, 4, 7, 9, 30, 50, 13, 100, 17, 300, 40][seed])
    tmax = [1, 2, 3, 10, 5, 50, 100, 7, 1000, 20, 60, 1_000_000][seed]
    w = synth.random_small(E, V, tmax, 500 + seed)
    for k, M in ((1, 2), (3, 3), (8, 5), (16, 7)):
        compare_all(w.src, w.dst, w.t, w.n_vertices, k, M)


@pytest.mark.parametrize("scale", [0.0004, 0.002])
def test_mid_scaled(scale):
    w = synth.mid(scale=scale)
    compare_all(w.src, w.dst, w.t, w.n_vertices, w.k, w.min_cluster_size)


def test_hub_scaled():
    w = synth.hub(scale=0.0003)
    rng = np.random.default_rng(1)
    q = np.sort(rng.choice(w.n_edges, 3000, replace=False)).astype(np.int32)
    compare_all(w.src, w.dst, w.t, w.n_vertices, w.k, w.min_cluster_size, knn_query=q)


def test_zipf_hubs_cross_every_sort_bin():
    """Degrees spanning the warp (<=32), CTA (<=256, <=2048) and hub (>2048)
    sort bins, with many tied timestamps."""
    w = synth.random_small(30_000, 400, 500, 77, zipf_s=1.3)
    deg = np.bincount(w.src, minlength=w.n_vertices)
    assert deg.max() > 2048 and (deg > 256).sum() > 1 and ((deg > 32) & (deg <= 256)).any()
    compare_all(w.src, w.dst, w.t, w.n_vertices, 8, 5)


def test_all_same_time():
    rng = np.random.default_rng(3)
    E, V = 3000, 60
    src = rng.integers(0, V, E).astype(np.int32)
    dst = ((src + 1 + rng.integers(0, V - 1, E)) % V).astype(np.int32)
    t = np.full(E, 42, np.int64)
    key = src.astype(np.int64) * V + dst
    _, first = np.unique(key, return_index=True)
    src, dst, t = src[first], dst[first], t[first]
    compare_all(src, dst, t, V, 4, 5)


def test_star_and_chain():
    # star: many senders into a hub, one hub reply per sender
    n = 5000
    src = np.concatenate([np.arange(1, n + 1), np.zeros(n, np.int64)]).astype(np.int32)
    dst = np.concatenate([np.zeros(n, np.int64), np.arange(1, n + 1)]).astype(np.int32)
    t = np.concatenate([np.arange(n) * 3, np.arange(n) * 3 + 1]).astype(np.int64)
    compare_all(src, dst, t, n + 1, 8, 5)
    # relay chain with increasing gaps (monotone weights along a path)
    m = 4000
    src = np.arange(m).astype(np.int32)
    dst = (np.arange(m) + 1).astype(np.int32)
    t = np.cumsum(np.arange(m)).astype(np.int64)
    compare_all(src, dst, t, m + 1, 4, 5)


def test_exact_eom_tie_goes_to_the_parent():
    """A relay chain at t = 0, 2, 6, 8, 22, 24 has the skeleton path with
    weights 2, 4, 2, 14, 2: lambdas N/3, N/5, N/15 (N = 2^64 - 1) with
    2 N/5 = N/3 + N/15, so the cluster of the first four edges has exactly
    its children's summed stability; EOM keeps the parent."""
    src = np.arange(6, dtype=np.int32)
    g, _ = compare_all(src, src + 1, np.array([0, 2, 6, 8, 22, 24], np.int64), 7, 1, 2)
    assert g["labels"].tolist() == [0, 0, 0, 0, 1, 1]
    assert sorted(g["cl_selected"].tolist()) == [0, 1, 1, 2, 2]


def test_large_timestamps_and_negative():
    w = synth.random_small(2000, 50, 1000, 9)
    compare_all(w.src, w.dst, w.t * 1_000_003 - 10**12, w.n_vertices, 4, 3)


@pytest.mark.parametrize("seed", [0, 1])
def test_wide_time_span(seed):
    """Times whose span needs more bits than fit beside the ids in one 64-bit
    sort key (nanosecond stamps over a century, negative and positive):
    stage A then sorts on the time alone with the id as the value. Ties stay
    common (few distinct times)."""
    w = synth.random_small(3000, 40, 60, 31 + seed)
    jitter = (np.arange(w.n_edges) % 3).astype(np.int64)
    t = (w.t - 30) * (np.int64(1) << 56) + jitter * (np.int64(1) << 40)
    assert int(t.max() - t.min()).bit_length() + (w.n_edges - 1).bit_length() > 64
    compare_all(w.src, w.dst, t, w.n_vertices, 4, 3)


def test_empty_and_single():
    z = np.zeros(0, np.int32)
    g = run_gpu(z, z, np.zeros(0, np.int64), 5, 4, 5)
    assert g["n_clusters"] == 0 and len(g["sk_u"]) == 0
    compare_all(np.array([0], np.int32), np.array([1], np.int32), np.array([7], np.int64), 2, 1, 2)


def test_errors_are_reported():
    import torch
    from gpu_helpers import ctx
    from paper_2311_10337_gb300 import dgec
    c = ctx()
    s = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    d = torch.tensor([1, 1], dtype=torch.int32, device="cuda")
    t = torch.tensor([0, 1], dtype=torch.int64, device="cuda")
    with pytest.raises(dgec.DgecError) as ei:
        c.run(s, d, t, 2, 4, 5)
    assert ei.value.status == 3
    d = torch.tensor([1, 9], dtype=torch.int32, device="cuda")
    with pytest.raises(dgec.DgecError) as ei:
        c.run(s, d, t, 2, 4, 5)
    assert ei.value.status == 2
    with pytest.raises(dgec.DgecError):
        c.run(s, d, t, 2, 0, 5)


def test_run_host_matches_device():
    from gpu_helpers import ctx
    w = synth.tiny(seed_offset=1)
    g = run_gpu(w.src, w.dst, w.t, w.n_vertices, w.k, w.min_cluster_size)
    lab, ncl = ctx().run_host(w.src, w.dst, w.t, w.n_vertices, w.k, w.min_cluster_size)
    assert np.array_equal(lab, g["labels"]) and ncl == g["n_clusters"]


def test_repeat_runs_identical():
    w = synth.mid(scale=0.001)
    a = run_gpu(w.src, w.dst, w.t, w.n_vertices, w.k, w.min_cluster_size)
    b = run_gpu(w.src, w.dst, w.t, w.n_vertices, w.k, w.min_cluster_size)
    for key in a:
        assert np.array_equal(np.asarray(a[key]), np.asarray(b[key])), key
