"""Nearly-causal line graph (Sec. 4.3: arcs up to delta back in time,
weighed |dt|) on the GPU against the oracle, bit for bit on every output."""
import numpy as np
import pytest

from gpu_helpers import ctx, run_gpu, sorted_skeleton
from oracle import oracle as O
from paper_2311_10337_gb300 import synth

pytestmark = pytest.mark.gpu
NAMES = ["out_off", "in_off", "out_id", "in_id", "sk_u", "sk_v", "sk_w", "knn_id", "core", "mst_u", "mst_v",
         "mst_w", "link_a", "link_b", "link_size", "labels"]


def run_nc(src, dst, t, V, k, M, delta, delta_max=None):
    import torch
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dt)).cuda()
    out = ctx().run(dev(src, np.int32), dev(dst, np.int32), dev(t, np.int64), V, k, M,
                    delta_max=delta_max, delta_nc=delta)
    torch.cuda.synchronize()
    r = {n: out.numpy(n) for n in NAMES}
    r["n_clusters"] = out.n_clusters
    return r


def compare_nc(src, dst, t, V, k, M, delta, delta_max=None):
    g = run_nc(src, dst, t, V, k, M, delta, delta_max)
    r = O.run_nearly_causal(src, dst, t, V, k, M, delta, delta_max)
    oo, oi, io_, ii = r["csr"]
    assert np.array_equal(g["out_off"], oo) and np.array_equal(g["out_id"], oi), "out lists"
    assert np.array_equal(g["in_off"], io_) and np.array_equal(g["in_id"], ii), "in lists"
    su, sv, sw = r["skeleton"]
    gu, gv, gw = sorted_skeleton(g["sk_u"], g["sk_v"], g["sk_w"])
    assert np.array_equal(gu, su) and np.array_equal(gv, sv) and np.array_equal(gw, sw), "skeleton"
    kid, kcore = r["knn"]
    assert np.array_equal(g["knn_id"].reshape(kid.shape), kid), "knn ids"
    assert np.array_equal(g["core"], kcore), "core"
    mu, mv, mw = r["mst"]
    assert np.array_equal(g["mst_u"], mu) and np.array_equal(g["mst_v"], mv) and np.array_equal(g["mst_w"], mw)
    a, b, s = r["linkage"]
    assert np.array_equal(g["link_a"], a) and np.array_equal(g["link_b"], b) and np.array_equal(g["link_size"], s)
    assert np.array_equal(g["labels"], r["condensed"]["labels"]), "labels"
    assert g["n_clusters"] == r["condensed"]["n_clusters"]
    return g


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("delta", [1, 2, 7, 1000])
def test_random_tie_heavy(seed, delta):
    g = synth.random_small(50 + 31 * seed, 4 + seed % 6, 3 + seed % 13, 1000 + seed,
                           zipf_s=1.3 if seed % 2 else 0.0)
    compare_nc(g.src, g.dst, g.t, g.n_vertices, 1 + (3 * seed) % 16, 2 + seed % 4, delta)


@pytest.mark.parametrize("delta", [60, 3600])
def test_mid_scaled(delta):
    w = synth.mid(scale=0.001)
    compare_nc(w.src, w.dst, w.t, w.n_vertices, w.k, w.min_cluster_size, delta)


def test_with_cutoff_and_host_entry():
    w = synth.tiny()
    compare_nc(w.src, w.dst, w.t, w.n_vertices, w.k, w.min_cluster_size, 500, delta_max=20000)
    dev = run_nc(w.src, w.dst, w.t, w.n_vertices, w.k, w.min_cluster_size, 500)
    lab, ncl = ctx().run_host(w.src, w.dst, w.t, w.n_vertices, w.k, w.min_cluster_size, delta_nc=500)
    assert np.array_equal(lab, dev["labels"]) and ncl == dev["n_clusters"]


def test_delta_zero_and_errors():
    w = synth.random_small(200, 15, 30, 3)
    a = run_nc(w.src, w.dst, w.t, w.n_vertices, 4, 3, 0)
    b = run_gpu(w.src, w.dst, w.t, w.n_vertices, 4, 3)
    for key in ("knn_id", "core", "mst_w", "labels"):
        assert np.array_equal(a[key], b[key]), key
    import torch
    from paper_2311_10337_gb300 import dgec
    s = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    d = torch.tensor([1, 0], dtype=torch.int32, device="cuda")
    t = torch.tensor([0, 1], dtype=torch.int64, device="cuda")
    for kw in (dict(delta_nc=-1), dict(delta_nc=3, mrd=True)):
        with pytest.raises(dgec.DgecError) as e:
            ctx().run(s, d, t, 2, 4, 5, **kw)
        assert e.value.status == 1
