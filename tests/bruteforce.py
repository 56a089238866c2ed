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


def lam(w):
    """Lambda of a merge at weight w: floor((2^64 - 1) / (w + 1)), exact."""
    return ((1 << 64) - 1) // (w + 1)


def condense_bruteforce(n, edges, M):
    """Condensed tree, excess-of-mass selection and labels read directly off
    the filtration comps(H, w) of an explicit graph H (no linkage, no
    union-find replay): top down from a virtual root at w = inf (lambda 0)
    whose children are H's components; a node is a component at the
    smallest weight that connects it, and its children are its parts one
    distinct weight lower. At a node of lambda L inside cluster K: two or
    more children of size >= M end K and start one cluster each; exactly one
    continues K; the points of the other children leave K at L. Stability
    of K = sum over points leaving K of (L_p - birth) + sum over child
    clusters of size * (death - birth); EOM bottom up with ties to the
    parent, root never selected; labels by the selected ancestor, numbered
    by smallest member. Returns labels, number of clusters, each point's
    leaving lambda, and the clusters as (birth, death, size, stability,
    selected) with selected 2 final / 1 covered / 0."""
    ws = sorted(set(edges.values()))
    levels = [components(n, edges, w) for w in ws]          # levels[i]: weight <= ws[i]

    def merge_level(S, top):
        """Smallest level at which the points S form one component."""
        for i in range(top + 1):
            if len(set(levels[i][S].tolist())) == 1:
                return i
        raise AssertionError("not a component")

    def parts(S, i):
        """Components of S one distinct weight below ws[i]."""
        if i == 0:
            return [[x] for x in S]
        lab = levels[i - 1][S]
        out = {}
        for x, l in zip(S, lab.tolist()):
            out.setdefault(l, []).append(x)
        return list(out.values())

    clusters = []            # dicts: birth, death, size, points (leaving), children, members
    fall = np.zeros(n, dtype=object)
    fall_of = np.full(n, -1, np.int64)

    def new_cluster(members, birth):
        clusters.append(dict(birth=birth, death=0, size=len(members), leave=[], children=[],
                             members=list(members)))
        return len(clusters) - 1

    def leave(K, pts, L):
        for p in pts:
            clusters[K]["leave"].append(L)
            fall[p] = L
            fall_of[p] = K

    def split(K, kids, L):
        """Apply the condensing rule at one node; return (cluster, set) pairs to go on with."""
        big = [c for c in kids if len(c) >= M]
        small = [c for c in kids if len(c) < M]
        for c in small:
            leave(K, c, L)
        if len(big) >= 2:
            clusters[K]["death"] = L
            todo = []
            for c in big:
                C = new_cluster(c, L)
                clusters[K]["children"].append(C)
                todo.append((C, sorted(c)))
            return todo
        if len(big) == 1:
            return [(K, sorted(big[0]))]
        return []

    top = len(ws) - 1
    root = new_cluster(range(n), 0)
    if top >= 0:
        comps = {}
        for x, l in enumerate(levels[top].tolist()):
            comps.setdefault(l, []).append(x)
        kids = list(comps.values())
    else:
        kids = [[x] for x in range(n)]
    todo = split(root, kids, 0)
    while todo:
        K, S = todo.pop()
        i = merge_level(S, top)
        todo.extend(split(K, parts(S, i), lam(ws[i])))

    stab = []
    for c in clusters:
        s = sum(L - c["birth"] for L in c["leave"])
        s += sum(clusters[ch]["size"] * (c["death"] - c["birth"]) for ch in c["children"])
        stab.append(s)
    score = [0] * len(clusters)
    sel = [0] * len(clusters)
    for K in range(len(clusters) - 1, -1, -1):          # children are created after parents
        sumc = sum(score[ch] for ch in clusters[K]["children"])
        if K != root and stab[K] >= sumc:
            sel[K] = 1
            score[K] = stab[K]
        else:
            score[K] = sumc
    parent = {ch: K for K, c in enumerate(clusters) for ch in c["children"]}
    final = []
    for K in range(len(clusters)):
        if sel[K]:
            a, covered = parent.get(K), False
            while a is not None:
                covered |= bool(sel[a])
                a = parent.get(a)
            if not covered:
                sel[K] = 2
                final.append(K)
    final.sort(key=lambda K: min(clusters[K]["members"]))
    number = {K: x for x, K in enumerate(final)}
    labels = np.full(n, -1, np.int32)
    for p in range(n):
        a = int(fall_of[p])
        while a is not None and a >= 0:
            if sel[a] == 2:
                labels[p] = number[a]
                break
            a = parent.get(a)
    table = sorted((c["birth"], c["death"], c["size"], stab[K], sel[K]) for K, c in enumerate(clusters))
    return labels, len(final), [int(x) for x in fall], table
