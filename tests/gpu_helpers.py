"""Shared helpers for the GPU parity tests: run the CUDA path through the
C ABI and the CPU oracle on the same seeded input, and compare."""
from __future__ import annotations

import numpy as np

from oracle import oracle as O

_CTX = None


def ctx():
    global _CTX
    if _CTX is None:
        from paper_2311_10337_gb300 import dgec
        _CTX = dgec.Context(0)
    return _CTX


def run_gpu(src, dst, t, V, k, M, delta_max=None):
    import torch
    c = ctx()
    s = torch.from_numpy(np.ascontiguousarray(src, np.int32)).cuda()
    d = torch.from_numpy(np.ascontiguousarray(dst, np.int32)).cuda()
    tt = torch.from_numpy(np.ascontiguousarray(t, np.int64)).cuda()
    out = c.run(s, d, tt, V, k, M, delta_max=delta_max)
    torch.cuda.synchronize()
    names = ["out_off", "in_off", "out_t", "in_t", "out_id", "in_id", "pos_out", "pos_in", "sk_u", "sk_v", "sk_w",
             "knn_id", "core", "mst_u", "mst_v", "mst_w", "link_a", "link_b", "link_size",
             "fall_cluster", "fall_lambda", "cl_id", "cl_parent", "cl_birth", "cl_death",
             "cl_stab_hi", "cl_stab_lo", "cl_size", "cl_selected", "labels"]
    r = {n: out.numpy(n) for n in names}
    r["n_clusters"] = out.n_clusters
    return r


def sorted_skeleton(u, v, w):
    o = np.lexsort((v, u, w))
    return u[o], v[o], w[o]


def compare_all(src, dst, t, V, k, M, knn_query=None, what=None, delta_max=None):
    """Element-wise comparison of every output array (bit-exact: all integer)."""
    g = run_gpu(src, dst, t, V, k, M, delta_max)
    r = O.run(src, dst, t, V, k, M, knn_query, delta_max)
    E = len(src)
    oo, oi, io_, ii = r["csr"]
    assert np.array_equal(g["out_off"], oo), "out_off"
    assert np.array_equal(g["in_off"], io_), "in_off"
    assert np.array_equal(g["out_id"], oi), "out_id"
    assert np.array_equal(g["in_id"], ii), "in_id"
    assert np.array_equal(g["out_t"], t[oi]), "out_t"
    assert np.array_equal(g["in_t"], t[ii]), "in_t"
    for pos, lst in (("pos_out", oi), ("pos_in", ii)):    # inverse of the list permutation
        want = np.empty(E, np.int32)
        want[lst] = np.arange(E, dtype=np.int32)
        assert np.array_equal(g[pos], want), pos
    su, sv, sw = r["skeleton"]
    gu, gv, gw = sorted_skeleton(g["sk_u"], g["sk_v"], g["sk_w"])
    assert len(gu) == len(su), f"skeleton size {len(gu)} vs {len(su)}"
    assert np.array_equal(gu, su) and np.array_equal(gv, sv) and np.array_equal(gw, sw), "skeleton"
    kid, kcore = r["knn"]
    if knn_query is None:
        assert np.array_equal(g["knn_id"], kid), "knn ids"
        assert np.array_equal(g["core"], kcore), "core"
    else:
        assert np.array_equal(g["knn_id"][knn_query], kid), "knn ids (sampled)"
        assert np.array_equal(g["core"][knn_query], kcore), "core (sampled)"
    mu, mv, mw = r["mst"]
    assert np.array_equal(g["mst_u"], mu) and np.array_equal(g["mst_v"], mv), "msf edges"
    assert np.array_equal(g["mst_w"], mw), "msf weights"
    a, b, s = r["linkage"]
    assert np.array_equal(g["link_a"], a) and np.array_equal(g["link_b"], b), "linkage rows"
    assert np.array_equal(g["link_size"], s), "linkage sizes"
    c = r["condensed"]
    assert np.array_equal(g["fall_cluster"], c["fall_cluster"]), "fall cluster"
    assert np.array_equal(g["fall_lambda"], c["fall_lambda"]), "fall lambda"
    for key in ("cl_id", "cl_parent", "cl_birth", "cl_death", "cl_size", "cl_stab_hi",
                "cl_stab_lo", "cl_selected"):
        assert np.array_equal(g[key], c[key]), key
    assert np.array_equal(g["labels"], c["labels"]), "labels"
    assert g["n_clusters"] == c["n_clusters"]
    return g, r
