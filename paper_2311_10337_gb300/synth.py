"""Seeded synthetic dynamic multigraphs (temporal edge lists).

This module only draws inputs: it holds none of the clustering arithmetic.
Both the CUDA path and the CPU oracle read the arrays it returns.

Every random number comes from a counter-based generator (splitmix64 over a
counter), so a workload is a pure function of its seed and sizes.

The workloads stand in for the paper's two datasets, which are not shipped
here: the SNAP e-mail network (Sec. 4.1) and the Reddit comment graph
(Sec. 4.2). They keep the shape the paper reports: directed edges
(i, j, t) with integer-second times, no self loops, no repeated
(i, j, t) triple (Sec. 1.2.1), many timestamp ties, bursty conversations of
5-200 records, and heavy-tailed vertex degrees.
"""
from __future__ import annotations

import dataclasses
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_MASK = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLD = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

BASE_SEED = 0x231110337


def _mix_serial(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


_CHUNK = 1 << 22


def _mix(z: np.ndarray) -> np.ndarray:
    """splitmix64's finaliser, elementwise (large arrays in parallel chunks;
    the result does not depend on the chunking)."""
    z = np.asarray(z)
    if z.size <= 2 * _CHUNK:
        return _mix_serial(z)
    out = np.empty(z.shape, np.uint64)

    def one(a):
        out[a:a + _CHUNK] = _mix_serial(z[a:a + _CHUNK])

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        list(ex.map(one, range(0, z.size, _CHUNK)))
    return out


def _argsort_u64(h: np.ndarray) -> np.ndarray:
    """Stable argsort of uint64 keys (equal to np.argsort(h, kind="stable")),
    through torch's multi-threaded CPU sort: flipping the top bit maps the
    unsigned order onto the signed one."""
    import torch
    k = (np.asarray(h, np.uint64) ^ np.uint64(1 << 63)).view(np.int64)
    return torch.sort(torch.from_numpy(k), stable=True).indices.numpy()


def _argsort_i64(k: np.ndarray) -> np.ndarray:
    """Stable argsort of int64 keys (equal to np.argsort(k, kind="stable"))."""
    import torch
    return torch.sort(torch.from_numpy(np.ascontiguousarray(k, np.int64)), stable=True).indices.numpy()


def _searchsorted_right(cdf: np.ndarray, u: np.ndarray) -> np.ndarray:
    """np.searchsorted(cdf, u, side="right") for float64 arrays, multi-threaded."""
    import torch
    return torch.searchsorted(torch.from_numpy(np.ascontiguousarray(cdf, np.float64)),
                              torch.from_numpy(np.ascontiguousarray(u, np.float64)),
                              right=True).numpy()


class Stream:
    """splitmix64 stream: value n is mix(seed_state + (n + 1) * golden)."""

    def __init__(self, seed: int, tag: int):
        with np.errstate(over="ignore"):
            s = np.array([(seed * 0x100000001B3 + tag) & 0xFFFFFFFFFFFFFFFF],
                         dtype=np.uint64)
        self.state = _mix(s + _GOLD)[0]
        self.pos = 0

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(self.pos + 1, self.pos + n + 1, dtype=np.uint64)
        self.pos += n
        with np.errstate(over="ignore"):
            return _mix(self.state + idx * _GOLD)

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) from the top 53 bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def uniform_at(self, pos: int, n: int) -> np.ndarray:
        """The n doubles a fresh stream would give from draw `pos` on (the
        stream's own position is not moved)."""
        idx = np.arange(pos + 1, pos + n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = _mix(self.state + idx * _GOLD)
        return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Integers in [lo, hi)."""
        span = hi - lo
        v = np.floor(self.uniform(n) * span).astype(np.int64)
        np.minimum(v, span - 1, out=v)
        return v + lo


@dataclasses.dataclass
class Workload:
    name: str
    src: np.ndarray   # int32[E]
    dst: np.ndarray   # int32[E]
    t: np.ndarray     # int64[E]
    n_vertices: int
    k: int
    min_cluster_size: int
    recipe: str

    @property
    def n_edges(self) -> int:
        return int(self.src.shape[0])


def _zipf_ranks(st: Stream, n: int, n_vertices: int, s: float) -> np.ndarray:
    """Rank-Zipf draw: P(rank r) proportional to r**-s, r = 1..n_vertices (0-based out)."""
    r = np.arange(1, n_vertices + 1, dtype=np.float64)
    cdf = np.cumsum(r ** (-s))
    cdf /= cdf[-1]
    u = st.uniform(n)
    idx = _searchsorted_right(cdf, u)
    return np.minimum(idx, n_vertices - 1).astype(np.int64)


def _permutation(st: Stream, n: int) -> np.ndarray:
    """Seeded random permutation (argsort of fresh 64-bit draws)."""
    return _argsort_u64(st.u64(n)).astype(np.int64)


def _zipf_endpoints(st: Stream, n: int, n_vertices: int, s: float,
                    perm: np.ndarray):
    src = perm[_zipf_ranks(st, n, n_vertices, s)]
    dst = perm[_zipf_ranks(st, n, n_vertices, s)]
    # resample self loops (the paper excludes them, Sec. 1.2.1)
    for _ in range(64):
        bad = np.nonzero(src == dst)[0]
        if bad.size == 0:
            break
        dst[bad] = perm[_zipf_ranks(st, bad.size, n_vertices, s)]
    bad = np.nonzero(src == dst)[0]
    if bad.size:
        dst[bad] = (src[bad] + 1) % n_vertices
    return src, dst


def _dedupe_triples(src, dst, t):
    """Make every (i, j, t) triple unique (Sec. 1.2.1): within each (i, j)
    pair that has a repeat, times are made strictly increasing by moving a
    repeat to one second after its predecessor. The edges are ordered by
    (pair, t, position) with two stable sorts; a pair has a repeat when two
    neighbours in that order share (pair, t). The full-size steps run as
    torch CPU ops (multi-threaded); the pairs with repeats in numpy."""
    import torch
    S = torch.from_numpy(np.ascontiguousarray(src, np.int64))
    D = torch.from_numpy(np.ascontiguousarray(dst, np.int64))
    T = torch.from_numpy(np.ascontiguousarray(t, np.int64))
    pair = (S << 32) | D
    by_t = torch.sort(T, stable=True).indices
    o = by_t[torch.sort(pair[by_t], stable=True).indices]
    pk, tt = pair[o], T[o]
    rep = (pk[1:] == pk[:-1]) & (tt[1:] == tt[:-1])
    if not bool(rep.any()):
        return t
    head = torch.ones(len(o), dtype=torch.bool)
    head[1:] = pk[1:] != pk[:-1]
    gid_all = torch.cumsum(head, 0) - 1
    bad = torch.zeros(int(gid_all[-1]) + 1, dtype=torch.bool)
    bad[gid_all[1:][rep]] = True
    sel = bad[gid_all]
    o, tt, head = o[sel].numpy(), tt[sel].numpy(), head[sel].numpy()
    gid = np.cumsum(head) - 1
    start = np.nonzero(head)[0]
    r = np.arange(len(o)) - start[gid]
    big = np.int64(1) << np.int64(40)
    v = (tt - tt.min()) - r + gid.astype(np.int64) * big
    v = np.maximum.accumulate(v)
    t = np.array(t, np.int64, copy=True)
    t[o] = v - gid.astype(np.int64) * big + r + tt.min()
    return t


def _conversations(st: Stream, n_edges: int, n_vertices: int, span: int,
                   mean_gap: float = 60.0):
    """Planted conversations: a group of U{3..20} vertices exchanges a burst of
    U{5..200} records with floor(Exp(mean_gap)) s gaps; the sender is the
    previous receiver w.p. 0.75, else a uniform member; the receiver is a
    uniform other member."""
    src = np.empty(n_edges, np.int64)
    dst = np.empty(n_edges, np.int64)
    t = np.empty(n_edges, np.int64)
    planted = np.empty(n_edges, np.int64)
    pos = 0
    conv = 0
    # draw conversations in chunks to keep this vectorised
    while pos < n_edges:
        chunk = max(1024, (n_edges - pos) // 100 + 1)
        gsize = st.integers(3, 21, chunk)
        blen = st.integers(5, 201, chunk)
        start = st.integers(0, span, chunk)
        tot = int(blen.sum())
        # members: gsize uniform vertices per conversation (repeats allowed
        # across conversations; within one, resample collisions below)
        mem_off = np.concatenate([[0], np.cumsum(gsize)])
        members = st.integers(0, n_vertices, int(mem_off[-1]))
        conv_of = np.repeat(np.arange(chunk), blen)
        step = np.arange(tot) - np.repeat(np.concatenate([[0], np.cumsum(blen)[:-1]]), blen)
        gaps = np.floor(-mean_gap * np.log1p(-st.uniform(tot))).astype(np.int64)
        gaps[step == 0] = 0
        # time = start + running sum of gaps within the burst
        csum = np.cumsum(gaps)
        first = np.concatenate([[0], np.cumsum(blen)[:-1]])
        base = np.repeat(csum[first] - gaps[first], blen)
        times = np.repeat(start, blen) + (csum - base)
        # sender / receiver chain, stepped across all bursts at once
        keep_prev = st.uniform(tot) < 0.75
        pick_s = st.integers(0, 1 << 30, tot)
        pick_r = st.integers(0, 1 << 30, tot)
        s_loc = np.empty(tot, np.int64)
        r_loc = np.empty(tot, np.int64)
        prev_r = np.zeros(chunk, np.int64)
        for x in range(int(blen.max())):
            cidx = np.nonzero(blen > x)[0]
            at = first[cidx] + x
            g = gsize[cidx]
            fresh = pick_s[at] % g
            sl = np.where((x == 0) | ~keep_prev[at], fresh, prev_r[cidx])
            rl = pick_r[at] % (g - 1)
            rl = rl + (rl >= sl)
            s_loc[at] = sl
            r_loc[at] = rl
            prev_r[cidx] = rl
        moff = np.repeat(mem_off[:-1], blen)
        s_v = members[moff + s_loc]
        r_v = members[moff + r_loc]
        take = min(tot, n_edges - pos)
        src[pos:pos + take] = s_v[:take]
        dst[pos:pos + take] = r_v[:take]
        t[pos:pos + take] = times[:take]
        planted[pos:pos + take] = conv + conv_of[:take]
        pos += take
        conv += chunk
    # two members of one group may coincide: move the receiver to a neighbour id
    same = src == dst
    dst[same] = (dst[same] + 1) % n_vertices
    return src, dst, t, planted


def tiny(seed_offset: int = 0, n_edges: int = 20_000, n_vertices: int = 2_000,
         zipf_s: float = 2.1, t_max: int = 1_000_000, k: int = 4,
         min_cluster_size: int = 5) -> Workload:
    """Endpoints rank-Zipf(2.1) by degree, t uniform integer in [0, 1e6)."""
    seed = BASE_SEED + 0 + 1000 * seed_offset
    st = Stream(seed, 1)
    perm = _permutation(Stream(seed, 2), n_vertices)
    src, dst = _zipf_endpoints(st, n_edges, n_vertices, zipf_s, perm)
    t = Stream(seed, 3).integers(0, t_max, n_edges)
    t = _dedupe_triples(src, dst, t)
    return Workload("tiny", src.astype(np.int32), dst.astype(np.int32), t,
                    n_vertices, k, min_cluster_size,
                    f"E={n_edges} V={n_vertices} zipf={zipf_s} t~U[0,{t_max})")


def mid(scale: float = 1.0, seed_offset: int = 0, k: int = 8,
        min_cluster_size: int = 5) -> Workload:
    """1M vertices, 50M edges at scale 1: 70% planted conversations over a
    30-day span, 30% Poisson background with Zipf(2.1) endpoints."""
    seed = BASE_SEED + 1 + 1000 * seed_offset
    n_edges = int(round(50_000_000 * scale))
    n_vertices = max(64, int(round(1_000_000 * scale)))
    span = 30 * 86400
    n_conv = int(round(0.7 * n_edges))
    n_bg = n_edges - n_conv
    cs, cd, ct, _ = _conversations(Stream(seed, 11), n_conv, n_vertices, span)
    perm = _permutation(Stream(seed, 12), n_vertices)
    bs, bd = _zipf_endpoints(Stream(seed, 13), n_bg, n_vertices, 2.1, perm)
    bt = Stream(seed, 14).integers(0, span, n_bg)
    src = np.concatenate([cs, bs])
    dst = np.concatenate([cd, bd])
    t = np.concatenate([ct, bt])
    order = _permutation(Stream(seed, 15), n_edges)
    src, dst, t = src[order], dst[order], t[order]
    t = _dedupe_triples(src, dst, t)
    return Workload("mid", src.astype(np.int32), dst.astype(np.int32), t,
                    n_vertices, k, min_cluster_size,
                    f"E={n_edges} V={n_vertices} span=30d conv=70% bg=30% zipf=2.1")


def hub(scale: float = 1.0, seed_offset: int = 0, k: int = 8,
        min_cluster_size: int = 5) -> Workload:
    """10M vertices, 200M edges at scale 1: 50% Zipf(1.8) background with t
    quantised to 60 s, 40% planted conversations, 10% replayed (i, j) pairs
    on an hourly grid."""
    seed = BASE_SEED + 2 + 1000 * seed_offset
    n_edges = int(round(200_000_000 * scale))
    n_vertices = max(64, int(round(10_000_000 * scale)))
    span = 30 * 86400
    n_bg = n_edges // 2
    n_conv = int(round(0.4 * n_edges))
    n_rep = n_edges - n_bg - n_conv
    perm = _permutation(Stream(seed, 21), n_vertices)
    bs, bd = _zipf_endpoints(Stream(seed, 22), n_bg, n_vertices, 1.8, perm)
    bt = Stream(seed, 23).integers(0, span // 60, n_bg) * 60
    cs, cd, ct, _ = _conversations(Stream(seed, 24), n_conv, n_vertices, span)
    # replayed pairs: a pool of pairs, each used at many hourly slots
    st = Stream(seed, 25)
    n_pairs = max(1, n_rep // 50)
    ps, pd = _zipf_endpoints(st, n_pairs, n_vertices, 1.8, perm)
    which = st.integers(0, n_pairs, n_rep)
    rs, rd = ps[which], pd[which]
    rt = st.integers(0, span // 3600, n_rep) * 3600
    src = np.concatenate([bs, cs, rs])
    dst = np.concatenate([bd, cd, rd])
    t = np.concatenate([bt, ct, rt])
    order = _permutation(Stream(seed, 26), n_edges)
    src, dst, t = src[order], dst[order], t[order]
    t = _dedupe_triples(src, dst, t)
    return Workload("hub", src.astype(np.int32), dst.astype(np.int32), t,
                    n_vertices, k, min_cluster_size,
                    f"E={n_edges} V={n_vertices} bg=50% zipf=1.8 t%60==0, conv=40%, replay=10% hourly")


def stream(scale: float = 6.0, days: int = 180, seed_offset: int = 0, k: int = 8,
           min_cluster_size: int = 5) -> Workload:
    """The serving stream: drawn as mid (70% planted conversations, 30%
    Zipf(2.1) background) at `scale` times its size -- 300M edges over 6M
    vertices at scale 6 -- over a `days`-day span, returned in (t, id)
    order (a stable sort of the drawn edges by time)."""
    seed = BASE_SEED + 4 + 1000 * seed_offset
    n_edges = int(round(50_000_000 * scale))
    n_vertices = max(64, int(round(1_000_000 * scale)))
    span = days * 86400
    n_conv = int(round(0.7 * n_edges))
    n_bg = n_edges - n_conv
    cs, cd, ct, _ = _conversations(Stream(seed, 11), n_conv, n_vertices, span)
    perm = _permutation(Stream(seed, 12), n_vertices)
    bs, bd = _zipf_endpoints(Stream(seed, 13), n_bg, n_vertices, 2.1, perm)
    bt = Stream(seed, 14).integers(0, span, n_bg)
    src = np.concatenate([cs, bs])
    del cs, bs
    dst = np.concatenate([cd, bd])
    del cd, bd
    t = np.concatenate([ct, bt])
    del ct, bt
    order = _permutation(Stream(seed, 15), n_edges)
    src, dst, t = src[order], dst[order], t[order]
    t = _dedupe_triples(src, dst, t)
    by_t = _argsort_i64(t)
    return Workload("stream", src[by_t].astype(np.int32), dst[by_t].astype(np.int32), t[by_t],
                    n_vertices, k, min_cluster_size,
                    f"E={n_edges} V={n_vertices} span={days}d conv=70% bg=30% zipf=2.1, (t, id) order")


def serve_jobs(n_jobs: int, n_stream: int, rate: float, log10_min: float = 4.0,
               log10_max: float = 7.0, seed_offset: int = 0):
    """Windowed clustering jobs over a stream of n_stream edges: window sizes
    round(10^U(log10_min, log10_max)) edges (at most the stream), uniform
    starts, Poisson arrivals at `rate` per second. Returns (starts, sizes,
    arrival times in s)."""
    st = Stream(BASE_SEED + 6 + 1000 * seed_offset, 61)
    sizes = np.round(10.0 ** (log10_min + (log10_max - log10_min) * st.uniform(n_jobs))).astype(np.int64)
    sizes = np.clip(sizes, 1, n_stream)
    starts = np.floor(st.uniform(n_jobs) * (n_stream - sizes + 1)).astype(np.int64)
    starts = np.minimum(starts, n_stream - sizes)
    gaps = -np.log1p(-st.uniform(n_jobs)) / rate
    return starts, sizes, np.cumsum(gaps)


def random_small(n_edges: int, n_vertices: int, t_max: int, seed: int,
                 zipf_s: float = 0.0) -> Workload:
    """Small tie-heavy graphs for brute-force checks (t uniform in [0, t_max))."""
    st = Stream(BASE_SEED + 77 + seed, 31)
    if zipf_s > 0:
        perm = _permutation(Stream(BASE_SEED + 77 + seed, 32), n_vertices)
        src, dst = _zipf_endpoints(st, n_edges, n_vertices, zipf_s, perm)
    else:
        src = st.integers(0, n_vertices, n_edges)
        dst = st.integers(0, n_vertices - 1, n_edges)
        dst[dst >= src] += 1
    t = Stream(BASE_SEED + 77 + seed, 33).integers(0, t_max, n_edges)
    if n_edges:
        t = _dedupe_triples(src, dst, t)
    return Workload(f"rand{seed}", src.astype(np.int32), dst.astype(np.int32),
                    t.astype(np.int64), n_vertices, 3, 3,
                    f"E={n_edges} V={n_vertices} t~U[0,{t_max})")


@dataclasses.dataclass
class Batch:
    """Independent graphs laid end to end; vertex ids are local per graph."""
    src: np.ndarray        # int32[total]
    dst: np.ndarray        # int32[total]
    t: np.ndarray          # int64[total]
    edge_off: np.ndarray   # int64[G+1]
    n_vertices: np.ndarray  # int32[G]
    k: np.ndarray          # int32[G]
    min_cluster_size: np.ndarray  # int32[G]
    recipe: str

    @property
    def n_graphs(self) -> int:
        return int(self.n_vertices.shape[0])

    def graph(self, g):
        a, b = int(self.edge_off[g]), int(self.edge_off[g + 1])
        return self.src[a:b], self.dst[a:b], self.t[a:b]


def _graph_chunks(eoff: np.ndarray, max_edges: int = 1 << 25):
    """Consecutive graph ranges [g0, g1) of at most max_edges edges each
    (a single larger graph forms a range of its own)."""
    G = len(eoff) - 1
    g0 = 0
    while g0 < G:
        g1 = int(np.searchsorted(eoff, eoff[g0] + max_edges, side="right")) - 1
        g1 = min(max(g1, g0 + 1), G)
        yield g0, g1
        g0 = g1


def batch(n_graphs: int = 4096, log10_min: float = 3.0, log10_max: float = 6.0,
          seed_offset: int = 0, t_max: int = 1_000_000, zipf_s: float = 2.1) -> Batch:
    """The batching workload: E_b = round(10^U(log10_min, log10_max)) edges,
    V_b = max(2, E_b // 10) vertices, each graph drawn like the tiny one at
    its own size (rank-Zipf(2.1) endpoints, t uniform in [0, t_max)),
    k_b uniform in {4, 8, 16}, M = 5. One inverse-CDF table serves every
    graph (a rank-Zipf law over V_b ranks is the global law conditioned on
    rank <= V_b). Draw n of a stream belongs to edge n of the batch, so the
    graphs are drawn in chunks of whole graphs with bounded host memory; a
    repeated triple can only repeat within one graph, so the repeats are
    resolved chunk by chunk."""
    seed = BASE_SEED + 3 + 1000 * seed_offset
    st = Stream(seed, 41)
    sizes = np.round(10.0 ** (log10_min + (log10_max - log10_min) * st.uniform(n_graphs)))
    sizes = np.maximum(sizes.astype(np.int64), 1)
    nv = np.maximum(sizes // 10, 2).astype(np.int64)
    k = np.array([4, 8, 16], np.int32)[st.integers(0, 3, n_graphs)]
    eoff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    total = int(eoff[-1])
    vmax = int(nv.max())
    r = np.arange(1, vmax + 1, dtype=np.float64)
    cdf = np.cumsum(r ** (-zipf_s))
    cap = cdf[nv - 1]  # mass of ranks 1..V_b
    chunks = list(_graph_chunks(eoff))

    def gid_of(g0, g1):
        return np.repeat(np.arange(g0, g1), sizes[g0:g1])

    s_src, s_dst, s_t = Stream(seed, 42), Stream(seed, 43), Stream(seed, 44)
    src = np.empty(total, np.int64)
    dst = np.empty(total, np.int64)

    def endpoints(ch):  # each chunk fills its own slice: the order of chunks does not matter
        g0, g1 = ch
        a, b = int(eoff[g0]), int(eoff[g1])
        gid = gid_of(g0, g1)
        for stream, out in ((s_src, src), (s_dst, dst)):
            u = stream.uniform_at(a, b - a) * cap[gid]
            out[a:b] = np.minimum(_searchsorted_right(cdf, u), nv[gid] - 1)

    workers = max(1, min(len(chunks), (os.cpu_count() or 1) // 2))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        list(ex.map(endpoints, chunks))
    s_src.pos = s_dst.pos = total
    # self loops are resampled; only an entry that was bad can be bad again
    bad = np.nonzero(src == dst)[0]
    for _ in range(64):
        if bad.size == 0:
            break
        gb = np.searchsorted(eoff, bad, side="right") - 1
        u = s_dst.uniform(bad.size) * cap[gb]
        dst[bad] = np.minimum(_searchsorted_right(cdf, u), nv[gb] - 1)
        bad = bad[src[bad] == dst[bad]]
    gb = np.searchsorted(eoff, bad, side="right") - 1
    dst[bad] = (src[bad] + 1) % nv[gb]
    voff = np.concatenate([[0], np.cumsum(nv)])
    t = np.empty(total, np.int64)

    def times(ch):
        g0, g1 = ch
        a, b = int(eoff[g0]), int(eoff[g1])
        v = np.floor(s_t.uniform_at(a, b - a) * t_max).astype(np.int64)
        np.minimum(v, t_max - 1, out=v)
        gid = gid_of(g0, g1)
        t[a:b] = _dedupe_triples(src[a:b] + voff[gid], dst[a:b] + voff[gid], v)

    with ThreadPoolExecutor(max_workers=workers) as ex:
        list(ex.map(times, chunks))
    return Batch(src.astype(np.int32), dst.astype(np.int32), t, eoff,
                 nv.astype(np.int32), k, np.full(n_graphs, 5, np.int32),
                 f"{n_graphs} graphs, E_b=10^U({log10_min},{log10_max}) total {total}, "
                 f"V_b=E_b/10, zipf={zipf_s}, t~U[0,{t_max}), k in {{4,8,16}}, M=5")


# ------------------------------------------------------------ hypergraphs

@dataclasses.dataclass
class HyperWorkload:
    """Dynamic hypergraph (Sec. 4.4): hyperedge e at time t[e] with members
    s_vert[s_off[e]:s_off[e+1]] (undirected), or sources there and targets
    d_vert[d_off[e]:d_off[e+1]] (directed)."""
    name: str
    t: np.ndarray
    s_off: np.ndarray
    s_vert: np.ndarray
    d_off: np.ndarray | None
    d_vert: np.ndarray | None
    n_vertices: int
    min_cluster_size: int
    recipe: str

    @property
    def n_edges(self) -> int:
        return int(self.t.shape[0])

    @property
    def directed(self) -> bool:
        return self.d_off is not None


def _distinct_rows(st: Stream, row: np.ndarray, vert: np.ndarray, fixed: np.ndarray,
                   n_vertices: int) -> np.ndarray:
    """Redraw (uniformly) members that repeat a vertex within their row;
    `fixed` marks entries that must not move (a sender)."""
    vert = vert.copy()
    for _ in range(64):
        o = np.lexsort((~fixed, vert, row))
        dup = np.zeros(len(o), bool)
        dup[1:] = (row[o][1:] == row[o][:-1]) & (vert[o][1:] == vert[o][:-1])
        bad = o[dup]
        if bad.size == 0:
            return vert
        vert[bad] = st.integers(0, n_vertices, bad.size)
    raise RuntimeError("could not draw distinct members")


def _split_rows(n_rows, sizes, vert):
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return off, vert.astype(np.int32)


def hyper_small(n_edges: int, n_vertices: int, t_max: int, seed: int, directed: bool,
                max_members: int = 4, min_cluster_size: int = 3) -> HyperWorkload:
    """Small tie-heavy hypergraphs for brute-force checks: member counts
    uniform in [1, max_members] (sources in [1, 2] when directed), members
    uniform and distinct within a hyperedge, t uniform in [0, t_max)."""
    st = Stream(BASE_SEED + 91 + seed, 41)
    assert n_vertices >= 2 * max_members + 2
    t = st.integers(0, t_max, n_edges).astype(np.int64)
    if not directed:
        sz = st.integers(1, max_members + 1, n_edges)
        row = np.repeat(np.arange(n_edges), sz)
        vert = _distinct_rows(st, row, st.integers(0, n_vertices, int(sz.sum())),
                              np.zeros(int(sz.sum()), bool), n_vertices)
        s_off, s_vert = _split_rows(n_edges, sz, vert)
        return HyperWorkload(f"hyp{seed}", t, s_off, s_vert, None, None, n_vertices,
                             min_cluster_size, f"undirected E={n_edges} V={n_vertices} t~U[0,{t_max})")
    ns = st.integers(1, 3, n_edges)
    nd = st.integers(1, max_members + 1, n_edges)
    # sources and targets of a hyperedge drawn as one distinct row, then split
    tot = ns + nd
    row = np.repeat(np.arange(n_edges), tot)
    vert = _distinct_rows(st, row, st.integers(0, n_vertices, int(tot.sum())),
                          np.zeros(int(tot.sum()), bool), n_vertices)
    first = np.concatenate([[0], np.cumsum(tot)[:-1]])
    pos = np.arange(int(tot.sum())) - np.repeat(first, tot)
    is_src = pos < np.repeat(ns, tot)
    s_off, s_vert = _split_rows(n_edges, ns, vert[is_src])
    d_off, d_vert = _split_rows(n_edges, nd, vert[~is_src])
    return HyperWorkload(f"dhyp{seed}", t, s_off, s_vert, d_off, d_vert, n_vertices,
                         min_cluster_size, f"directed E={n_edges} V={n_vertices} t~U[0,{t_max})")


def hyper(scale: float = 1.0, directed: bool = True, seed_offset: int = 0,
          min_cluster_size: int = 5) -> HyperWorkload:
    """Broadcast messages (Sec. 4.4's single sender, many receivers): 20M
    hyperedges over 1M vertices at scale 1, a 30-day span. 70% in planted
    groups of U{3..12} members exchanging bursts of U{5..100} messages with
    Exp(60 s) gaps: the sender a uniform member, the receivers the next
    1 + Geom(1/2) members after it (cyclically, capped at the group). 30%
    background: sender rank-Zipf(2.1), 1 + Geom(1/2) receivers (at most 8)
    rank-Zipf(2.1) and distinct, t uniform. Undirected: members = sender and
    receivers together."""
    seed = BASE_SEED + 5 + 1000 * seed_offset
    n_edges = int(round(20_000_000 * scale))
    n_vertices = max(64, int(round(1_000_000 * scale)))
    span = 30 * 86400
    st = Stream(seed, 51)
    n_conv = int(round(0.7 * n_edges))
    n_bg = n_edges - n_conv
    # planted groups
    snd, rcv_cnt, t_parts, rcv_parts = [], [], [], []
    pos = 0
    while pos < n_conv:
        chunk = max(1024, (n_conv - pos) // 50 + 1)
        g = st.integers(3, 13, chunk)
        blen = st.integers(5, 101, chunk)
        start = st.integers(0, span, chunk)
        mem_off = np.concatenate([[0], np.cumsum(g)])
        members = st.integers(0, n_vertices, int(mem_off[-1]))
        row = np.repeat(np.arange(chunk), g)
        members = _distinct_rows(st, row, members, np.zeros(len(members), bool), n_vertices)
        tot = int(blen.sum())
        conv_of = np.repeat(np.arange(chunk), blen)
        first = np.concatenate([[0], np.cumsum(blen)[:-1]])
        gaps = np.floor(-60.0 * np.log1p(-st.uniform(tot))).astype(np.int64)
        gaps[first] = 0
        csum = np.cumsum(gaps)
        times = np.repeat(start, blen) + csum - np.repeat(csum[first], blen)
        gg = g[conv_of]
        sl = st.integers(0, 1 << 30, tot) % gg
        geo = np.floor(np.log1p(-st.uniform(tot)) / np.log(0.5)).astype(np.int64)
        nr = np.minimum(1 + geo, gg - 1)
        take = min(tot, n_conv - pos)
        sl, nr, gg, times, conv_of = sl[:take], nr[:take], gg[:take], times[:take], conv_of[:take]
        base = mem_off[conv_of]
        snd.append(members[base + sl])
        rcv_cnt.append(nr)
        x = np.arange(int(nr.sum())) - np.repeat(np.concatenate([[0], np.cumsum(nr)[:-1]]), nr)
        rl = (np.repeat(sl, nr) + 1 + x) % np.repeat(gg, nr)
        rcv_parts.append(members[np.repeat(base, nr) + rl])
        t_parts.append(times)
        pos += take
    perm = _permutation(Stream(seed, 52), n_vertices)
    bs = perm[_zipf_ranks(st, n_bg, n_vertices, 2.1)]
    geo = np.floor(np.log1p(-st.uniform(n_bg)) / np.log(0.5)).astype(np.int64)
    bn = np.minimum(1 + geo, 8)
    brow = np.repeat(np.arange(n_bg), bn + 1)
    bv = np.empty(int((bn + 1).sum()), np.int64)
    bfirst = np.concatenate([[0], np.cumsum(bn + 1)[:-1]])
    bv[:] = perm[_zipf_ranks(st, len(bv), n_vertices, 2.1)]
    bv[bfirst] = bs
    fixed = np.zeros(len(bv), bool)
    fixed[bfirst] = True
    bv = _distinct_rows(st, brow, bv, fixed, n_vertices)
    brcv = np.delete(bv, bfirst)
    bt = st.integers(0, span, n_bg)
    snd.append(bs); rcv_cnt.append(bn); rcv_parts.append(brcv); t_parts.append(bt)
    sender = np.concatenate(snd)
    nr = np.concatenate(rcv_cnt)
    rcv = np.concatenate(rcv_parts)
    t = np.concatenate(t_parts).astype(np.int64)
    # hyperedges in a seeded random order
    order = _permutation(Stream(seed, 53), n_edges)
    r_off = np.concatenate([[0], np.cumsum(nr)]).astype(np.int64)
    nr_o = nr[order]
    idx = np.repeat(r_off[order], nr_o) + (np.arange(int(nr_o.sum())) -
                                           np.repeat(np.concatenate([[0], np.cumsum(nr_o)[:-1]]), nr_o))
    rcv_o = rcv[idx]
    sender, t = sender[order], t[order]
    recipe = (f"E={n_edges} V={n_vertices} span=30d groups=70% (U3..12 members, bursts U5..100, "
              f"Exp(60s) gaps) bg=30% zipf=2.1, receivers 1+Geom(1/2)")
    if directed:
        s_off = np.arange(n_edges + 1, dtype=np.int64)
        d_off = np.concatenate([[0], np.cumsum(nr_o)]).astype(np.int64)
        return HyperWorkload("mail", t, s_off, sender.astype(np.int32), d_off, rcv_o.astype(np.int32),
                             n_vertices, min_cluster_size, "directed " + recipe)
    sz = nr_o + 1
    m_off = np.concatenate([[0], np.cumsum(sz)]).astype(np.int64)
    mv = np.empty(int(m_off[-1]), np.int64)
    mv[m_off[:-1]] = sender
    rest = np.ones(len(mv), bool)
    rest[m_off[:-1]] = False
    mv[rest] = rcv_o
    return HyperWorkload("mail_u", t, m_off, mv.astype(np.int32), None, None, n_vertices,
                         min_cluster_size, "undirected " + recipe)


def undirected_of(h: HyperWorkload) -> HyperWorkload:
    """The same hyperedges with sources and targets merged into one member
    set (sources first)."""
    E = h.n_edges
    ns, nd = np.diff(h.s_off), np.diff(h.d_off)
    m_off = np.concatenate([[0], np.cumsum(ns + nd)]).astype(np.int64)
    first_d = np.repeat(m_off[:-1] + ns, nd) + (np.arange(int(nd.sum())) - np.repeat(h.d_off[:-1], nd))
    first_s = np.repeat(m_off[:-1], ns) + (np.arange(int(ns.sum())) - np.repeat(h.s_off[:-1], ns))
    mv = np.empty(int(m_off[-1]), np.int32)
    mv[first_s] = h.s_vert
    mv[first_d] = h.d_vert
    return HyperWorkload(h.name + "_u", h.t, m_off, mv, None, None, h.n_vertices, h.min_cluster_size,
                         "undirected of " + h.recipe)
