"""Time cutoff of Sec. 4.3 (only line-graph arcs with w <= delta_max): the
CUDA path against the oracle on every output, bit for bit."""
import numpy as np
import pytest

from gpu_helpers import compare_all, ctx, run_gpu
from paper_2311_10337_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("delta", [0, 1, 4, 30])
def test_random_tie_heavy(seed, delta):
    g = synth.random_small(60 + 41 * seed, 4 + seed % 6, 3 + seed % 17, 900 + seed,
                           zipf_s=1.4 if seed % 2 else 0.0)
    compare_all(g.src, g.dst, g.t, g.n_vertices, 1 + seed % 16, 2 + seed % 4, delta_max=delta)


@pytest.mark.parametrize("delta", [60, 3600, 86400])
def test_mid_scaled(delta):
    w = synth.mid(scale=0.001)
    compare_all(w.src, w.dst, w.t, w.n_vertices, w.k, w.min_cluster_size, delta_max=delta)


def test_hub_scaled():
    w = synth.hub(scale=0.0003)
    q = np.arange(0, w.n_edges, 7, dtype=np.int32)
    compare_all(w.src, w.dst, w.t, w.n_vertices, w.k, w.min_cluster_size, knn_query=q, delta_max=600)


def test_cutoff_above_every_weight_is_no_cutoff():
    w = synth.mid(scale=0.0004)
    a = run_gpu(w.src, w.dst, w.t, w.n_vertices, w.k, w.min_cluster_size)
    b = run_gpu(w.src, w.dst, w.t, w.n_vertices, w.k, w.min_cluster_size, delta_max=1 << 62)
    for key in ("sk_u", "sk_v", "knn_id", "core", "mst_w", "labels"):
        assert np.array_equal(a[key], b[key]), key


def test_cutoff_shrinks_the_skeleton_and_host_entry():
    w = synth.mid(scale=0.0004)
    g = run_gpu(w.src, w.dst, w.t, w.n_vertices, w.k, w.min_cluster_size, delta_max=300)
    assert np.all(g["sk_w"] <= 300) and np.all(g["mst_w"] <= 300)
    lab, ncl = ctx().run_host(w.src, w.dst, w.t, w.n_vertices, w.k, w.min_cluster_size, delta_max=300)
    assert np.array_equal(lab, g["labels"]) and ncl == g["n_clusters"]


def test_negative_cutoff_rejected():
    import torch
    from paper_2311_10337_gb300 import dgec
    s = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    d = torch.tensor([1, 0], dtype=torch.int32, device="cuda")
    t = torch.tensor([0, 1], dtype=torch.int64, device="cuda")
    with pytest.raises(dgec.DgecError) as e:
        ctx().run(s, d, t, 2, 4, 5, delta_max=-1)
    assert e.value.status == 1
