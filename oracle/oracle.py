"""ctypes front end of the plain C oracle (dgec_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg; never by the product package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dgec_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libdgec_oracle.so")
_lock = threading.Lock()
_lib = None

I32P = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
I64P = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
U64P = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain C11, no arch flags)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            i64, i32 = ctypes.c_int64, ctypes.c_int32
            L.orc_validate.argtypes = [i64, i32, I32P, I32P]
            L.orc_csr.argtypes = [i64, i32, I32P, I32P, I64P, I64P, I32P, I64P, I32P]
            L.orc_skeleton_raw.argtypes = [i64, i32, I32P, I32P, I64P, I32P, I32P, I64P, I32P]
            L.orc_skeleton_raw.restype = i64
            L.orc_skeleton.argtypes = [i64, i32, I32P, I32P, I64P, I32P, I32P, I64P]
            L.orc_skeleton.restype = i64
            L.orc_knn.argtypes = [i64, i32, I32P, I32P, I64P, i32, i64, I32P, i64, i64, I32P, I64P]
            L.orc_mst.argtypes = [i64, i64, I32P, I32P, I64P, I32P, I32P, I64P]
            L.orc_mst.restype = i64
            L.orc_linkage.argtypes = [i64, i64, I32P, I32P, I32P, I32P, I64P]
            L.orc_levels.argtypes = [i64, i64, I32P, I32P, I64P, i32, I64P, I32P]
            L.orc_levels_tree.argtypes = [i64, i32, I32P, I32P, I32P]
            L.orc_hyper_skeleton.argtypes = [i64, i32, I64P, i32, I64P, I32P, I64P, I32P,
                                             I32P, I32P, I64P]
            L.orc_hyper_skeleton.restype = i64
            L.orc_condense_levels.argtypes = [i64, i32, I64P, I32P, i32, I32P,
                                              ctypes.POINTER(i32), ctypes.POINTER(i64),
                                              U64P, U64P, I64P, U64P, U64P, I32P]
            L.orc_condense.argtypes = [i64, i64, I32P, I32P, I64P, I64P, i32,
                                       I32P, U64P, I32P, I32P, U64P, U64P, I64P,
                                       U64P, U64P, I32P, I32P,
                                       ctypes.POINTER(i64), ctypes.POINTER(i32)]
            _lib = L
    return _lib


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def csr(src, dst, t, n_vertices):
    src, dst, t = _c(src, np.int32), _c(dst, np.int32), _c(t, np.int64)
    E = src.shape[0]
    out_off = np.zeros(n_vertices + 1, np.int64)
    in_off = np.zeros(n_vertices + 1, np.int64)
    out_id = np.zeros(max(E, 1), np.int32)
    in_id = np.zeros(max(E, 1), np.int32)
    rc = lib().orc_csr(E, n_vertices, src, dst, t, out_off, out_id, in_off, in_id)
    if rc:
        raise ValueError(f"oracle csr rc={rc}")
    return out_off, out_id[:E], in_off, in_id[:E]


def skeleton_raw(src, dst, t, n_vertices):
    src, dst, t = _c(src, np.int32), _c(dst, np.int32), _c(t, np.int64)
    E = src.shape[0]
    cap = 2 * E + 1
    p = np.zeros(cap, np.int32); q = np.zeros(cap, np.int32)
    w = np.zeros(cap, np.int64); c = np.zeros(cap, np.int32)
    n = lib().orc_skeleton_raw(E, n_vertices, src, dst, t, p, q, w, c)
    if n < 0:
        raise ValueError("oracle skeleton: bad input")
    return p[:n], q[:n], w[:n], c[:n]


def skeleton(src, dst, t, n_vertices):
    src, dst, t = _c(src, np.int32), _c(dst, np.int32), _c(t, np.int64)
    E = src.shape[0]
    cap = 2 * E + 1
    u = np.zeros(cap, np.int32); v = np.zeros(cap, np.int32); w = np.zeros(cap, np.int64)
    n = lib().orc_skeleton(E, n_vertices, src, dst, t, u, v, w)
    if n < 0:
        raise ValueError("oracle skeleton: bad input")
    return u[:n], v[:n], w[:n]


INT64_MAX = np.iinfo(np.int64).max


def knn(src, dst, t, n_vertices, k, query=None, delta_max=None, delta_nc=0):
    """k nearest line-graph neighbours by (w, id); with delta_max, only arcs
    with w <= delta_max exist (the cutoff of Sec. 4.3); with delta_nc > 0 an
    arc may also point up to delta_nc back in time (nearly causal, Sec. 4.3),
    weighed |dt|."""
    src, dst, t = _c(src, np.int32), _c(dst, np.int32), _c(t, np.int64)
    E = src.shape[0]
    if query is None:
        query = np.arange(E, dtype=np.int32)
    query = _c(query, np.int32)
    nq = query.shape[0]
    ids = np.zeros(max(nq * k, 1), np.int32)
    core = np.zeros(max(nq, 1), np.int64)
    dmax = INT64_MAX if delta_max is None else int(delta_max)
    rc = lib().orc_knn(E, n_vertices, src, dst, t, k, nq, query, dmax, int(delta_nc), ids, core)
    if rc:
        raise ValueError(f"oracle knn rc={rc}")
    return ids[:nq * k].reshape(nq, k), core[:nq]


def mst(n_nodes, u, v, w):
    u, v, w = _c(u, np.int32), _c(v, np.int32), _c(w, np.int64)
    n = u.shape[0]
    mu = np.zeros(max(n_nodes, 1), np.int32); mv = np.zeros(max(n_nodes, 1), np.int32)
    mw = np.zeros(max(n_nodes, 1), np.int64)
    m = lib().orc_mst(n_nodes, n, u, v, w, mu, mv, mw)
    if m < 0:
        raise MemoryError("oracle mst")
    return mu[:m], mv[:m], mw[:m]


def linkage(n_nodes, mu, mv):
    mu, mv = _c(mu, np.int32), _c(mv, np.int32)
    n = mu.shape[0]
    a = np.zeros(max(n, 1), np.int32); b = np.zeros(max(n, 1), np.int32)
    s = np.zeros(max(n, 1), np.int64)
    rc = lib().orc_linkage(n_nodes, n, mu, mv, a, b, s)
    if rc:
        raise MemoryError("oracle linkage")
    return a[:n], b[:n], s[:n]


def condense(n_nodes, a, b, w, size, M):
    a, b, w, size = _c(a, np.int32), _c(b, np.int32), _c(w, np.int64), _c(size, np.int64)
    n = a.shape[0]
    n_all = n_nodes + n + 1
    fall_cluster = np.zeros(max(n_nodes, 1), np.int32)
    fall_lambda = np.zeros(max(n_nodes, 1), np.uint64)
    cl_id = np.zeros(n_all, np.int32); cl_parent = np.zeros(n_all, np.int32)
    cl_birth = np.zeros(n_all, np.uint64); cl_death = np.zeros(n_all, np.uint64)
    cl_size = np.zeros(n_all, np.int64)
    hi = np.zeros(n_all, np.uint64); lo = np.zeros(n_all, np.uint64)
    sel = np.zeros(n_all, np.int32)
    labels = np.zeros(max(n_nodes, 1), np.int32)
    ncl = ctypes.c_int64(0); nlab = ctypes.c_int32(0)
    rc = lib().orc_condense(n_nodes, n, a, b, w, size, M, fall_cluster, fall_lambda,
                            cl_id, cl_parent, cl_birth, cl_death, cl_size, hi, lo, sel,
                            labels, ctypes.byref(ncl), ctypes.byref(nlab))
    if rc:
        raise ValueError(f"oracle condense rc={rc}")
    c = ncl.value
    return dict(fall_cluster=fall_cluster[:n_nodes], fall_lambda=fall_lambda[:n_nodes],
                cl_id=cl_id[:c], cl_parent=cl_parent[:c], cl_birth=cl_birth[:c],
                cl_death=cl_death[:c], cl_size=cl_size[:c], cl_stab_hi=hi[:c],
                cl_stab_lo=lo[:c], cl_selected=sel[:c], labels=labels[:n_nodes],
                n_clusters=nlab.value)


def skeleton_cutoff(src, dst, t, n_vertices, delta_max):
    """Skeleton of the line graph with the time cutoff of Sec. 4.3 (only arcs
    with w <= delta_max): the links of L* with w <= delta_max. By Thm. 3
    comps(L*, w) = comps(L_G, w) for every w, so for every threshold the
    filtered links have the components of the filtered line graph."""
    u, v, w = skeleton(src, dst, t, n_vertices)
    keep = w <= delta_max
    return u[keep], v[keep], w[keep]


def run(src, dst, t, n_vertices, k, M, knn_query=None, delta_max=None):
    """Alg. 4 end to end: skeleton (Alg. 3) -> Alg. 1 on it; plus kNN/core.
    With delta_max, on the cutoff line graph of Sec. 4.3."""
    E = len(src)
    out = {}
    out["csr"] = csr(src, dst, t, n_vertices)
    if delta_max is None:
        out["skeleton"] = skeleton(src, dst, t, n_vertices)
    else:
        out["skeleton"] = skeleton_cutoff(src, dst, t, n_vertices, delta_max)
    out["knn"] = knn(src, dst, t, n_vertices, k, knn_query, delta_max)
    u, v, w = out["skeleton"]
    out["mst"] = mst(E, u, v, w)
    mu, mv, mw = out["mst"]
    out["linkage"] = linkage(E, mu, mv)
    a, b, s = out["linkage"]
    out["condensed"] = condense(E, a, b, mw, s, M)
    return out


def levels(n_nodes, u, v, w, omega):
    """Alg. 5 on the graph (u, v, w): per threshold, every node's component
    named by its smallest member; shape (len(omega), n_nodes)."""
    u, v, w = _c(u, np.int32), _c(v, np.int32), _c(w, np.int64)
    om = _c(omega, np.int64)
    out = np.zeros(max(len(om) * n_nodes, 1), np.int32)
    rc = lib().orc_levels(n_nodes, len(u), u, v, w, len(om), om, out)
    if rc:
        raise MemoryError("oracle levels")
    return out[:len(om) * n_nodes].reshape(len(om), n_nodes)


def levels_tree(labels):
    """The tree D of Alg. 5 per node: (merge_level, merge_parent), -1 where a
    node names its component at every level."""
    lab = _c(labels, np.int32)
    q, n = lab.shape
    ml = np.zeros(max(n, 1), np.int32); mp = np.zeros(max(n, 1), np.int32)
    lib().orc_levels_tree(n, q, lab.reshape(-1), ml, mp)
    return ml[:n], mp[:n]


def condense_levels(labels, omega, M):
    """Condensed tree, excess of mass and labels on the discrete dendrogram
    given by per-level labels (levels() output)."""
    lab = _c(labels, np.int32)
    q, n = lab.shape
    om = _c(omega, np.int64)
    N = (q + 1) * n + 1
    out = np.zeros(max(n, 1), np.int32)
    birth = np.zeros(N, np.uint64); death = np.zeros(N, np.uint64)
    size = np.zeros(N, np.int64); hi = np.zeros(N, np.uint64); lo = np.zeros(N, np.uint64)
    sel = np.zeros(N, np.int32)
    nlab = ctypes.c_int32(0); ncl = ctypes.c_int64(0)
    rc = lib().orc_condense_levels(n, q, om, lab.reshape(-1), M, out, ctypes.byref(nlab),
                                   ctypes.byref(ncl), birth, death, size, hi, lo, sel)
    if rc:
        raise ValueError(f"oracle condense_levels rc={rc}")
    c = ncl.value
    return dict(labels=out[:n], n_clusters=nlab.value, cl_birth=birth[:c], cl_death=death[:c],
                cl_size=size[:c], cl_stab_hi=hi[:c], cl_stab_lo=lo[:c], cl_selected=sel[:c])


def hyper_skeleton(t, n_vertices, s_off, s_vert, d_off=None, d_vert=None):
    """Skeleton of a dynamic hypergraph (Sec. 4.4): undirected when d_off is
    None (members s_off/s_vert), else directed (sources s_*, targets d_*)."""
    t = _c(t, np.int64)
    E = t.shape[0]
    s_off, s_vert = _c(s_off, np.int64), _c(s_vert, np.int32)
    directed = d_off is not None
    if directed:
        d_off, d_vert = _c(d_off, np.int64), _c(d_vert, np.int32)
    else:
        d_off, d_vert = np.zeros(E + 1, np.int64), np.zeros(1, np.int32)
    if len(s_vert) == 0:
        s_vert = np.zeros(1, np.int32)
    if len(d_vert) == 0:
        d_vert = np.zeros(1, np.int32)
    cap = int(s_off[-1]) + (int(d_off[-1]) if directed else 0) + 1
    u = np.zeros(cap, np.int32); v = np.zeros(cap, np.int32); w = np.zeros(cap, np.int64)
    n = lib().orc_hyper_skeleton(E, n_vertices, t, int(directed), s_off, s_vert, d_off, d_vert, u, v, w)
    if n < 0:
        raise ValueError(f"oracle hyper_skeleton rc={-n}")
    return u[:n], v[:n], w[:n]


def hyper_run(t, n_vertices, s_off, s_vert, d_off=None, d_vert=None, M=5):
    """Alg. 1 on the hypergraph skeleton (Sec. 4.4)."""
    E = len(t)
    out = {"skeleton": hyper_skeleton(t, n_vertices, s_off, s_vert, d_off, d_vert)}
    u, v, w = out["skeleton"]
    out["mst"] = mst(E, u, v, w)
    mu, mv, mw = out["mst"]
    out["linkage"] = linkage(E, mu, mv)
    a, b, s = out["linkage"]
    out["condensed"] = condense(E, a, b, mw, s, M)
    return out


def mrd_graph(src, dst, t, n_vertices, k, delta_max=None):
    """Mutual-reachability mode (an approximation; not in the paper): the
    graph H = L* together with every edge's kNN pairs, each pair once, weighed
    max(core_a, core_b, |t_a - t_b|) (HDBSCAN's mutual reachability with the
    kNN core distances); pairs with an endpoint of infinite core (fewer than
    k neighbours) are dropped. Returns (u, v, w) with u < v, sorted by
    (u, v)."""
    src, dst, t = _c(src, np.int32), _c(dst, np.int32), _c(t, np.int64)
    E = src.shape[0]
    if delta_max is None:
        u, v, _ = skeleton(src, dst, t, n_vertices)
    else:
        u, v, _ = skeleton_cutoff(src, dst, t, n_vertices, delta_max)
    ids, core = knn(src, dst, t, n_vertices, k, None, delta_max)
    a = np.repeat(np.arange(E, dtype=np.int64), k)
    b = ids.reshape(-1).astype(np.int64)
    a, b = a[b >= 0], b[b >= 0]
    lo = np.concatenate([u.astype(np.int64), np.minimum(a, b)])
    hi = np.concatenate([v.astype(np.int64), np.maximum(a, b)])
    pairs = np.unique(lo * max(E, 1) + hi)                     # the union, as a set
    lo, hi = pairs // max(E, 1), pairs % max(E, 1)
    w = np.maximum(np.maximum(core[lo], core[hi]), np.abs(t[lo] - t[hi]))
    keep = w != INT64_MAX
    return lo[keep].astype(np.int32), hi[keep].astype(np.int32), w[keep].astype(np.int64)


def mrd_run(src, dst, t, n_vertices, k, M, delta_max=None):
    """Alg. 1 on the mutual-reachability graph H (see mrd_graph)."""
    E = len(src)
    out = {"graph": mrd_graph(src, dst, t, n_vertices, k, delta_max)}
    u, v, w = out["graph"]
    out["mst"] = mst(E, u, v, w)
    mu, mv, mw = out["mst"]
    out["linkage"] = linkage(E, mu, mv)
    a, b, s = out["linkage"]
    out["condensed"] = condense(E, a, b, mw, s, M)
    return out


def skeleton_nearly_causal(src, dst, t, n_vertices, delta_nc, delta_max=None):
    """Skeleton of the nearly-causal line graph of Sec. 4.3: an arc r -> s
    (dst r = src s) exists when t_s >= t_r - delta_nc, weighed |t_s - t_r|.
    At a vertex these arcs are the causal ones (t_r <= t_s) and the backward
    ones (t_s < t_r <= t_s + delta_nc). An MST of a union of two graphs lies
    in the union of their MSTs, Alg. 2 gives the causal part's (Thm. 2), and
    Alg. 2 on the graph with negated times gives the MST of all backward
    pairs, whose links with w <= delta_nc are the MSF of the capped family
    (Kruskal stopped at delta_nc). So the union of L*(G) and the links of
    L*(G with -t) with w <= delta_nc keeps the weighted connectivity. With
    delta_max, only links with w <= delta_max are kept. Sorted (w, u, v)."""
    u1, v1, w1 = skeleton(src, dst, t, n_vertices)
    u2, v2, w2 = skeleton(src, dst, -np.asarray(t, np.int64), n_vertices)
    keep = w2 <= delta_nc
    u = np.concatenate([u1, u2[keep]]).astype(np.int64)
    v = np.concatenate([v1, v2[keep]]).astype(np.int64)
    w = np.concatenate([w1, w2[keep]])
    E = max(len(src), 1)
    key, first = np.unique(u * E + v, return_index=True)      # the union, as a set
    u, v, w = u[first], v[first], w[first]
    if delta_max is not None:
        m = w <= delta_max
        u, v, w = u[m], v[m], w[m]
    o = np.lexsort((v, u, w))
    return u[o].astype(np.int32), v[o].astype(np.int32), w[o].astype(np.int64)


def run_nearly_causal(src, dst, t, n_vertices, k, M, delta_nc, delta_max=None):
    """Alg. 4 on the nearly-causal line graph (Sec. 4.3)."""
    E = len(src)
    out = {"csr": csr(src, dst, t, n_vertices)}
    out["skeleton"] = skeleton_nearly_causal(src, dst, t, n_vertices, delta_nc, delta_max)
    out["knn"] = knn(src, dst, t, n_vertices, k, None, delta_max, delta_nc)
    u, v, w = out["skeleton"]
    out["mst"] = mst(E, u, v, w)
    mu, mv, mw = out["mst"]
    out["linkage"] = linkage(E, mu, mv)
    a, b, s = out["linkage"]
    out["condensed"] = condense(E, a, b, mw, s, M)
    return out
