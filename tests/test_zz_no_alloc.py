"""The allocation-free forest entry point (dgec_msf_static) against the
regular pipeline's forest, called twice in a row through the C ABI.

The paper has no counterpart to this entry point: it serves callers that
may not allocate device memory where they need the forest, so it keeps its
working memory in one fixed array inside the library. This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
import numpy as np
import pytest

from gpu_helpers import ctx
from paper_2311_10337_gb300 import dgec, synth

pytestmark = pytest.mark.gpu


def _sorted(u, v, w):
    o = np.lexsort((v, u, w))
    return u[o], v[o], w[o]


def test_static_forest_matches_pipeline_twice():
    import torch
    wl = synth.tiny(seed_offset=3)
    c = ctx()
    src = torch.from_numpy(wl.src).cuda()
    dst = torch.from_numpy(wl.dst).cuda()
    t = torch.from_numpy(wl.t).cuda()
    out = c.run(src, dst, t, wl.n_vertices, wl.k, wl.min_cluster_size)
    # copy the skeleton out of the workspace so the pipeline's memory is not touched
    u = out.tensor("sk_u").clone()
    v = out.tensor("sk_v").clone()
    w = out.tensor("sk_w").clone()
    ref = (out.numpy("mst_u"), out.numpy("mst_v"), out.numpy("mst_w"))
    E = wl.n_edges
    for _ in range(2):
        mu = torch.full((E,), -7, dtype=torch.int32, device="cuda")
        mv = torch.full((E,), -7, dtype=torch.int32, device="cuda")
        mw = torch.full((E,), -7, dtype=torch.int64, device="cuda")
        n = dgec.msf_static(u, v, w, E, mu, mv, mw)
        torch.cuda.synchronize()
        got = _sorted(mu[:n].cpu().numpy(), mv[:n].cpu().numpy(), mw[:n].cpu().numpy())
        assert n == len(ref[0])
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)


def _pipeline_forest(wl, delta_max=None):
    """The pipeline's skeleton (copied out of its workspace) and forest."""
    import torch
    c = ctx()
    src = torch.from_numpy(wl.src).cuda()
    dst = torch.from_numpy(wl.dst).cuda()
    t = torch.from_numpy(wl.t).cuda()
    out = c.run(src, dst, t, wl.n_vertices, wl.k, wl.min_cluster_size, delta_max=delta_max)
    sk = (out.tensor("sk_u").clone(), out.tensor("sk_v").clone(), out.tensor("sk_w").clone())
    ref = (out.numpy("mst_u"), out.numpy("mst_v"), out.numpy("mst_w"))
    return sk, ref


def _static(sk, n_nodes):
    import torch
    mu = torch.full((n_nodes,), -7, dtype=torch.int32, device="cuda")
    mv = torch.full((n_nodes,), -7, dtype=torch.int32, device="cuda")
    mw = torch.full((n_nodes,), -7, dtype=torch.int64, device="cuda")
    n = dgec.msf_static(*sk, n_nodes, mu, mv, mw)
    torch.cuda.synchronize()
    return _sorted(mu[:n].cpu().numpy(), mv[:n].cpu().numpy(), mw[:n].cpu().numpy())


def test_static_forest_larger_then_smaller_and_disconnected():
    """A larger call leaves its contents in the shared array; a smaller call
    after it must not see them. The smaller graph runs with a time cutoff, so
    its skeleton is disconnected and the forest has many trees."""
    big = synth.mid(scale=0.002)                       # 100,000 edges
    small = synth.tiny(seed_offset=5)                  # 20,000 edges
    sk_big, ref_big = _pipeline_forest(big)
    sk_small, ref_small = _pipeline_forest(small, delta_max=2_000)
    assert len(ref_small[0]) < small.n_edges - 100     # many trees
    for sk, ref, E in ((sk_big, ref_big, big.n_edges), (sk_small, ref_small, small.n_edges),
                       (sk_big, ref_big, big.n_edges)):
        got = _static(sk, E)
        assert len(got[0]) == len(ref[0])
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("case", ["u_ge_v", "id_out_of_range", "negative_w"])
def test_static_forest_rejects_bad_edges(case):
    import torch
    u = torch.tensor([0, 1, 2], dtype=torch.int32, device="cuda")
    v = torch.tensor([1, 2, 3], dtype=torch.int32, device="cuda")
    w = torch.tensor([5, 6, 7], dtype=torch.int64, device="cuda")
    n_nodes = 4
    if case == "u_ge_v":
        u[1], v[1] = 2, 1
    elif case == "id_out_of_range":
        n_nodes = 3
    else:
        w[2] = -1
    out32 = torch.zeros(4, dtype=torch.int32, device="cuda")
    out64 = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(dgec.DgecError) as ei:
        dgec.msf_static(u, v, w, n_nodes, out32, out32.clone(), out64)
    assert ei.value.status == 1                        # DGEC_ERR_INVALID_ARG


def test_static_forest_rejects_oversize():
    import torch
    z32 = torch.zeros(4, dtype=torch.int32, device="cuda")
    z64 = torch.zeros(4, dtype=torch.int64, device="cuda")
    n_nodes = (1 << 18) + 1                            # one node over the fixed array's limit
    o32 = torch.zeros(n_nodes, dtype=torch.int32, device="cuda")
    o64 = torch.zeros(n_nodes, dtype=torch.int64, device="cuda")
    with pytest.raises(dgec.DgecError) as ei:
        dgec.msf_static(z32, z32, z64, n_nodes, o32, o32.clone(), o64)
    assert ei.value.status == 4
