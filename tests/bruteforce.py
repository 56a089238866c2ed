"""Brute-force constructions on tiny inputs, written from the paper's
definitions and independent of both the oracle and the CUDA path.

They build the explicit increment-weighted line graph (Def. 1), which the
method itself never forms, and answer questions about it directly.
"""
from __future__ import annotations

import numpy as np


def line_graph_arcs(src, dst, t):
    """All arcs (r, s, w) of L_G (Def. 1): j_r == i_s (P1), t_r <= t_s (P2),
    w = t_s - t_r (P3)."""
    src = np.asarray(src); dst = np.asarray(dst); t = np.asarray(t, np.int64)
    r, s = np.nonzero((dst[:, None] == src[None, :]) & (t[:, None] <= t[None, :]))
    return r, s, t[s] - t[r]


def undirected_edges_nc(src, dst, t, delta_nc):
    """Undirected nearly-causal line graph (Sec. 4.3): r and s joined when
    dst r = src s and t_s >= t_r - delta_nc, weight |t_s - t_r|."""
    E = len(src)
    out = {}
    for r in range(E):
        for s in range(E):
            if r != s and dst[r] == src[s] and int(t[s]) >= int(t[r]) - delta_nc:
                out[(min(r, s), max(r, s))] = abs(int(t[s]) - int(t[r]))
    return out


def undirected_edges(src, dst, t):
    """Undirected version of L_G as a dict {(min, max): w} (weak connectivity,
    Sec. 1.2.3). Two arcs between one pair exist only for a reciprocal,
    concurrent pair; both then weigh 0."""
    r, s, w = line_graph_arcs(src, dst, t)
    out = {}
    for a, b, x in zip(r.tolist(), s.tolist(), w.tolist()):
        key = (min(a, b), max(a, b))
        if key in out:
            assert out[key] == x
        out[key] = x
    return out


def local_arcs(src, dst, t, i):
    """Arcs of the node-local line graph L_G(i) (Def. 2) read as the arcs
    that pass through vertex i: in-edge p of i, out-edge q of i, t_p <= t_q."""
    src = np.asarray(src); dst = np.asarray(dst); t = np.asarray(t, np.int64)
    ins = np.nonzero(dst == i)[0]
    outs = np.nonzero(src == i)[0]
    arcs = [(int(p), int(q), int(t[q] - t[p])) for p in ins for q in outs if t[p] <= t[q]]
    return ins, outs, arcs


class UnionFind:
    def __init__(self, n):
        self.p = list(range(n))

    def find(self, x):
        while self.p[x] != x:
            self.p[x] = self.p[self.p[x]]
            x = self.p[x]
        return x

    def union(self, a, b):
        ra, rb = self.find(a), self.find(b)
        if ra == rb:
            return False
        self.p[ra] = rb
        return True


def components(n, edges, omega):
    """comps(H, omega) (appendix): partition of range(n) by the edges with
    weight <= omega, as a canonical label array (label = smallest member)."""
    uf = UnionFind(n)
    for (a, b), w in edges.items():
        if w <= omega:
            uf.union(a, b)
    root = [uf.find(x) for x in range(n)]
    first = {}
    lab = np.empty(n, np.int64)
    for x in range(n):
        lab[x] = first.setdefault(root[x], x)
    return lab


def minimax(n, edges):
    """All-pairs minimax path weight (the smallest omega at which two nodes
    share a component of comps(H, omega)); inf where never connected."""
    INF = np.iinfo(np.int64).max
    D = np.full((n, n), INF, np.int64)
    np.fill_diagonal(D, 0)
    for (a, b), w in edges.items():
        D[a, b] = min(D[a, b], w)
        D[b, a] = min(D[b, a], w)
    for k in range(n):
        D = np.minimum(D, np.maximum(D[:, k:k + 1], D[k:k + 1, :]))
    return D


def knn_bruteforce(src, dst, t, k, delta_max=None, delta_nc=0):
    """Neighbours of each node in the undirected L_G ranked by (w, id); with
    delta_max, in the line graph keeping only arcs with w <= delta_max; with
    delta_nc, in the nearly-causal line graph."""
    E = len(src)
    und = undirected_edges(src, dst, t) if not delta_nc else undirected_edges_nc(src, dst, t, delta_nc)
    if delta_max is not None:
        und = {key: w for key, w in und.items() if w <= delta_max}
    nb = [[] for _ in range(E)]
    for (a, b), w in und.items():
        nb[a].append((w, b))
        nb[b].append((w, a))
    ids = np.full((E, k), -1, np.int32)
    core = np.full(E, np.iinfo(np.int64).max, np.int64)
    for e in range(E):
        lst = sorted(nb[e])
        for x, (w, s) in enumerate(lst[:k]):
            ids[e, x] = s
        if len(lst) >= k:
            core[e] = lst[k - 1][0]
    return ids, core


def hyper_line_graph(h):
    """Explicit line graph of a dynamic hypergraph (Sec. 4.4) as an undirected
    dict {(min, max): w}. Undirected: two hyperedges sharing a vertex, w =
    |t_r - t_s|. Directed: an arc r -> s when a target of r is a source of s
    and t_r <= t_s, w = t_s - t_r (weak connectivity as for graphs)."""
    E = h.n_edges
    src_of = {}   # vertex -> hyperedges with it as member / source
    dst_of = {}   # vertex -> hyperedges with it as target
    for e in range(E):
        for i in h.s_vert[h.s_off[e]:h.s_off[e + 1]].tolist():
            src_of.setdefault(i, []).append(e)
        if h.directed:
            for i in h.d_vert[h.d_off[e]:h.d_off[e + 1]].tolist():
                dst_of.setdefault(i, []).append(e)
    out = {}
    t = h.t.tolist()
    if not h.directed:
        for i, lst in src_of.items():
            for x in range(len(lst)):
                for y in range(x + 1, len(lst)):
                    a, b = lst[x], lst[y]
                    out[(min(a, b), max(a, b))] = abs(t[a] - t[b])
        return out
    for i, ins in dst_of.items():
        for r in ins:
            for s in src_of.get(i, []):
                if r != s and t[r] <= t[s]:
                    out[(min(r, s), max(r, s))] = t[s] - t[r]
    return out
