"""Benchmark: temporal edges/s of the whole edge-clustering path (Alg. 4:
incidence lists, skeleton, kNN + core distances, minimum spanning forest,
dendrogram, condensed tree, labels) on the largest single-GPU workload, the
synthetic 'hub' graph (10M vertices, 200M edges, k = 8, M = 5).

One step = one full pass of the path over the 200M edges, inputs resident
in HBM. Prints one JSON line (rank 0). Multi-GPU runs are independent
replicas (one graph per rank, no collective on the data path).

Side reports in the same line: the 50M-edge 'mid' graph (the path, the
discrete dendrogram, the variants and hypergraphs), the tiny graph's
latency, the batched form on 4,096 graphs against one run per graph, and
the served form (20,000 windowed jobs over a 300M-edge stream). The two
large side workloads are drawn by a spawned helper process while the GPU
measures the headline.

--impl reference times the CPU oracle (the reference arm for this path) on
a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import shutil
import subprocess
import sys
import tempfile
import threading
import time
from concurrent.futures import ProcessPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "temporal edges/s end-to-end (kNN+MST+dendrogram)"
UNIT = "edges/s"


# Algorithmic bytes per input edge of each stage at k neighbours (what the
# method must move; the quadratic line graph is never formed):
#   A  incidence lists: read the edge 16 B, write the lists 24 B;
#   B  skeleton + kNN: read the lists 24 B, write the skeleton (<= 2 links,
#      16 B each) 32 B, the kNN ids 4k B and the core distance 8 B;
#   C  forest: read the skeleton 32 B, write the forest 16 B;
#   D  dendrogram + condensed tree + labels: read the forest 16 B, write the
#      dendrogram rows 24 B, the points' condensed rows 20 B, the labels 4 B.
def stage_bytes_per_edge(k: int) -> dict:
    return {"A": 40, "B": 24 + 32 + 4 * k + 8, "C": 48, "D": 64}


def pipeline_bytes_per_edge(k: int) -> int:
    return sum(stage_bytes_per_edge(k).values())


# Algorithmic bytes per edge of the kNN kernel (stage B's list reads and the
# kNN output): the lists read once (24 B), k ids (4k B), the core distance
# (8 B). Window re-reads and offset lookups are access overhead, not counted.
def knn_bytes_per_edge(k: int) -> int:
    return 24 + 4 * k + 8


# DRAM bytes (read + write) per edge of the kNN step at k = 8, by kNN form
# (the launch configuration's knn_packed), each from one ncu capture on the
# hub graph at scale 0.02 (4M edges), scaled to a full step by the edges it
# processes. Form 1, the per-edge packed kernel: 312.6 MB read + 212.7 MB
# written (profiles/k_knn32_hub_small.md). Form 2, the two list-order passes:
# 139.0 + 427.7 MB read, 218.1 + 216.4 MB written
# (profiles/k_knn_list_order_hub_small.md). A form without a capture of its
# current kernels, or whose kernels changed since, maps to None.
KNN_TRAFFIC_BYTES_PER_EDGE_K8 = {
    1: (312_571_904 + 212_684_800) / 4_000_000,
    2: (139_018_240 + 218_062_336 + 427_675_136 + 216_392_960) / 4_000_000,
}

CPU_SAMPLE_MINUTES = {"hub": 25.0, "mid": 150.0, "tiny": 1e9}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dgec", choices=["dgec", "reference"])
    ap.add_argument("--workload", default="hub", choices=["hub", "mid", "tiny"])
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--roofline-kernel", default="k_knn",
                    help="kernel timed live for the roofline object")
    ap.add_argument("--cpu-sample-minutes", type=float, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mid", action="store_true", help="skip the 50M-edge side reports")
    ap.add_argument("--mid-scale", type=float, default=1.0)
    ap.add_argument("--batch-graphs", type=int, default=4096,
                    help="graphs in the batched-vs-plain comparison (0 = skip)")
    ap.add_argument("--serve-jobs", type=int, default=20000,
                    help="jobs in the serving measurement (0 = skip)")
    ap.add_argument("--serve-stream-scale", type=float, default=6.0,
                    help="serving stream size in units of 50M edges")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="Poisson arrivals per second")
    ap.add_argument("--serve-lanes", type=int, default=3)
    ap.add_argument("--serve-pool-gb", type=float, default=150.0)
    ap.add_argument("--hyper-scale", type=float, default=1.0,
                    help="scale of the hypergraph (broadcast message) measurement; 0 = skip")
    ap.add_argument("--nc-delta", type=int, default=60,
                    help="tolerance (s) of the nearly-causal measurement; < 0 = skip")
    ap.add_argument("--no-mrd", action="store_true",
                    help="skip the mutual-reachability mode measurement")
    ap.add_argument("--no-levels", action="store_true",
                    help="skip the discrete-dendrogram (Alg. 5) measurement")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the library's default launch configuration (no autotuning)")
    ap.add_argument("--no-breakdown", action="store_true",
                    help="skip the per-kernel breakdown step (one extra untimed pass)")
    return ap.parse_args()


def max_over_ranks(x: float, world: int, device) -> float:
    """The slowest rank's value (timings are max over ranks); x itself at N = 1."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: int, seconds: float) -> float:
    """Whole-job throughput of N replicas: every rank's units over the slowest
    rank's time (weak scaling: each rank runs its own graph)."""
    return world * units_per_rank / seconds


def make_workload(name, scale, rank):
    """Rank r's graph: the same recipe and size, its own seed."""
    from paper_2311_10337_gb300 import synth
    if name == "mid":
        return synth.mid(scale=scale, seed_offset=rank)
    if name == "hub":
        return synth.hub(scale=scale, seed_offset=rank)
    return synth.tiny(seed_offset=rank)


def time_window_sample(w, minutes):
    """Bounded sample for the CPU oracle: the edges of the first `minutes`
    of the workload's time span (a sub-window of the same stream)."""
    tmax = int(w.t.min()) + int(minutes * 60)
    sel = np.nonzero(w.t < tmax)[0]
    return w.src[sel], w.dst[sel], w.t[sel]


def cpu_model() -> str:
    """The host CPU's model name as lscpu prints it (machine type if unknown)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine() or "unknown"


def cpu_baseline(w, minutes):
    from oracle import oracle as O
    O.build()
    s, d, t = time_window_sample(w, minutes)
    t0 = time.perf_counter()
    O.run(s, d, t, w.n_vertices, w.k, w.min_cluster_size)
    dt = time.perf_counter() - t0
    return {"value": len(s) / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {minutes:g} min of the {w.name} stream: {len(s)} edges "
                      f"(of {w.n_edges}), single-threaded C oracle, {dt:.2f} s",
            "host": f"{cpu_model()}, {os.cpu_count()} cores, 1 used"}


class Clocks:
    """Sample nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def knn_roofline(timed, steps, E, k, knn_form, peak, peak_kind, breakdown, prefix="k_knn"):
    """Roofline object of the kNN step from the kernel timers of the timed
    steps. `timed` maps each kernel name timed (every name starting with
    `prefix`: one launch a pass in the per-edge forms, the two passes
    k_knn_pred and k_knn in the list-order form) to (total ms, launches).
    The unit of work is the kNN step of one pass over the E edges, so
    `achieved` is its algorithmic bytes (64 B/edge at k = 8)
    over its device time per pass. `breakdown` (name -> (ms, launches)) of
    one pass with every launch timed gives the step's share and the top
    kernels. Returns (roofline dict, top kernels or None)."""
    tot_ms = sum(v[0] for v in timed.values())
    tot_n = sum(v[1] for v in timed.values())
    kb = knn_bytes_per_edge(k)
    per_pass = tot_ms / steps if tot_n else None
    achieved = (kb * E) / (per_pass / 1000.0) / 1e9 if per_pass else None
    per_edge = KNN_TRAFFIC_BYTES_PER_EDGE_K8.get(knn_form) if prefix == "k_knn" and k == 8 else None
    traffic = per_edge * E if per_edge else None
    share = None
    top = None
    if breakdown:
        tot = sum(v[0] for v in breakdown.values())
        mine = sum(v[0] for n_, v in breakdown.items() if n_.startswith(prefix))
        if mine > 0 and tot > 0:
            share = mine / tot
        if tot > 0:
            top = [[n, round(v[0], 3), v[1], round(v[0] / tot, 4)] for n, v in
                   sorted(breakdown.items(), key=lambda kv: -kv[1][0])[:12]]
    roof = {"bound": "hbm", "kernel": prefix, "achieved": achieved, "peak": peak,
            "peak_kind": peak_kind, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": traffic,
            "traffic_over_algorithmic": (traffic / (kb * E)) if traffic else None,
            "algorithmic_bytes_per_edge": kb, "algorithmic_bytes_per_launch": kb * E,
            "ms_per_pass": per_pass,
            "avg_launch_ms": (tot_ms / tot_n) if tot_n else None,
            "share_of_step": share,
            "kernels": sorted(timed), "launches_per_step": tot_n / steps, "knn_form": knn_form}
    return roof, top


def stage_report(stages, E, k, peak):
    """Per-stage device time of one pass (CUDA events at the stage boundaries,
    from the library) against the stage's algorithmic bytes; D = D1 + D2."""
    by = stage_bytes_per_edge(k)
    ms = {"A": 0.0, "B": 0.0, "C": 0.0, "D": 0.0}
    for name, t in stages:
        key = "D" if name.startswith("D") else name[:1]
        if key in ms:
            ms[key] += t
    out = {}
    for key, t in ms.items():
        if t <= 0:
            continue
        gbs = by[key] * E / (t / 1000.0) / 1e9
        out[key] = {"ms": round(t, 3), "bytes_per_edge": by[key], "achieved_gbs": round(gbs, 1),
                    "frac": round(gbs / peak, 4)}
    return out


# ------------------------------------------------------- side workloads

def _gen_to_files(kind: str, arg: float, outdir: str) -> str:
    """Runs in a spawned helper process: draw a large side workload and save
    its arrays as .npy files under outdir/kind."""
    sys.path.insert(0, ROOT)
    from paper_2311_10337_gb300 import synth
    d = os.path.join(outdir, kind)
    os.makedirs(d, exist_ok=True)
    if kind == "batch":
        b = synth.batch(int(arg))
        for f in ("src", "dst", "t", "edge_off", "n_vertices", "k", "min_cluster_size"):
            np.save(os.path.join(d, f + ".npy"), getattr(b, f))
        with open(os.path.join(d, "recipe.txt"), "w") as fh:
            fh.write(b.recipe)
    else:
        w = synth.stream(scale=arg)
        for f in ("src", "dst", "t"):
            np.save(os.path.join(d, f + ".npy"), getattr(w, f))
        with open(os.path.join(d, "meta.json"), "w") as fh:
            json.dump({"n_vertices": w.n_vertices, "k": w.k, "M": w.min_cluster_size,
                       "recipe": w.recipe}, fh)
    return d


def _load(d, names):
    return {n: np.load(os.path.join(d, n + ".npy")) for n in names}


def tiny_latency(ctx, runs):
    """Latency of one whole pass on the 20,000-edge tiny graph, which sits in
    L2 and is bound by launches and host round trips rather than bandwidth:
    CUDA events around each call on the launching stream, after a warm-up."""
    import torch
    from paper_2311_10337_gb300 import synth
    w = synth.tiny()
    s, d, t = (torch.from_numpy(x).cuda() for x in (w.src, w.dst, w.t))
    stream = torch.cuda.current_stream()
    ctx.run(s, d, t, w.n_vertices, w.k, w.min_cluster_size)
    torch.cuda.synchronize()
    ms = []
    for _ in range(runs):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.run(s, d, t, w.n_vertices, w.k, w.min_cluster_size)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return {"edges": w.n_edges, "k": w.k, "runs": runs, "latency_ms_p50": float(np.median(ms)),
            "latency_ms_min": float(np.min(ms)), "launches": ctx.launches()}


def timed_runs(ctx, fn, steps):
    """CUDA-event time of `steps` calls of fn() on the current stream after
    one warm-up call; returns (ms per call, launches per call, last result)."""
    import torch
    out = fn()
    launches = ctx.launches()
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, launches, out


def mid_reports(ctx, args, steps, peak):
    """The 50M-edge mid graph: the whole path, then the discrete dendrogram,
    the mutual-reachability mode and the nearly-causal variant on it."""
    import torch
    w = make_workload("mid", args.mid_scale, 0)
    src, dst, tt = (torch.from_numpy(x).cuda() for x in (w.src, w.dst, w.t))
    E, V, k, M = w.n_edges, w.n_vertices, w.k, w.min_cluster_size
    ms, launches, out = timed_runs(ctx, lambda: ctx.run(src, dst, tt, V, k, M), steps)
    res = {"workload": f"{w.name}: {w.recipe}, k={k}, M={M}", "edges": E,
           "edges_per_s": E / (ms / 1000.0), "ms": ms, "gpu_launches_per_run": launches,
           "n_clusters": out.n_clusters, "stages": stage_report(ctx.stage_timing(), E, k, peak)}
    del out
    if not args.no_levels:
        res["discrete_dendrogram"] = discrete_levels(ctx, src, dst, tt, w, steps)
    if not args.no_mrd:
        ms, launches, out = timed_runs(ctx, lambda: ctx.run(src, dst, tt, V, k, M, mrd=True), steps)
        res["mutual_reachability"] = {"edges_per_s": E / (ms / 1000.0), "ms": ms, "forest_edges": out.n_mst,
                                      "n_clusters": out.n_clusters, "gpu_launches_per_run": launches}
        del out
    if args.nc_delta >= 0:
        ms, launches, out = timed_runs(
            ctx, lambda: ctx.run(src, dst, tt, V, k, M, delta_nc=args.nc_delta), steps)
        res["nearly_causal"] = {"edges_per_s": E / (ms / 1000.0), "ms": ms, "delta_s": args.nc_delta,
                                "skeleton_links": out.n_skeleton, "forest_edges": out.n_mst,
                                "n_clusters": out.n_clusters, "gpu_launches_per_run": launches}
        del out
    del src, dst, tt
    ctx.ws = None
    torch.cuda.empty_cache()
    return res


def discrete_levels(ctx, src, dst, tt, w, steps):
    """Edges/s of the discrete-dendrogram path (Alg. 5: incidence lists,
    skeleton, components at omega = 2^0 .. 2^28 s and the tree D), alone
    and with condensing on D (M of the workload); inputs resident."""
    omega = np.array([2 ** i for i in range(29)], np.int64)
    E, V, M = w.n_edges, w.n_vertices, w.min_cluster_size
    res = {"thresholds": "2^0 .. 2^28 (29 levels)"}
    for name, m in (("levels", 0), ("levels_condensed", M)):
        ms, launches, out = timed_runs(ctx, lambda: ctx.run_levels(src, dst, tt, V, omega, m), steps)
        res[name] = {"edges_per_s": E / (ms / 1000.0), "ms": ms, "gpu_launches_per_run": launches}
        if m:
            res[name]["n_clusters"] = out.n_clusters
        else:
            nc = out.numpy("n_components")
            res["n_merges"] = out.n_merges
            res["components_at"] = {"1s": int(nc[0]), "2^10s": int(nc[10]), "2^20s": int(nc[20]),
                                    "2^28s": int(nc[28])}
        del out
    return res


def hypergraphs(ctx, scale, steps):
    """Hyperedges/s of Alg. 1 on the dynamic-hypergraph skeleton (Sec. 4.4):
    the broadcast-message workload, directed (one sender, receivers) and
    the same hyperedges undirected; inputs resident, CUDA events."""
    import torch
    from paper_2311_10337_gb300 import synth
    hd = synth.hyper(scale=scale, directed=True)
    res = {"recipe": hd.recipe, "hyperedges": hd.n_edges}
    for name, h in (("directed", hd), ("undirected", synth.undirected_of(hd))):
        dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dt)).cuda()
        args = (dev(h.t, np.int64), dev(h.s_off, np.int64), dev(h.s_vert, np.int32), h.n_vertices,
                h.min_cluster_size)
        kw = dict(d_off=dev(h.d_off, np.int64), d_vert=dev(h.d_vert, np.int32)) if h.directed else {}
        ms, launches, out = timed_runs(ctx, lambda: ctx.run_hyper(*args, **kw), steps)
        memb = int(h.s_off[-1]) + (int(h.d_off[-1]) if h.directed else 0)
        res[name] = {"hyperedges_per_s": h.n_edges / (ms / 1000.0), "ms": ms, "memberships": memb,
                     "skeleton_links": out.n_skeleton, "n_clusters": out.n_clusters,
                     "gpu_launches_per_run": launches}
        del args, kw, out
    ctx.ws = None
    torch.cuda.empty_cache()
    return res


def batched_vs_plain(ctx, d, max_edges, tune_it=True):
    """Aggregate edges/s of the batched form over every graph of the batching
    workload (passes of at most max_edges edges) against one run per graph,
    on the same GPU, same graphs, identical output (every label compared)."""
    import torch
    b = _load(d, ("src", "dst", "t", "edge_off", "n_vertices", "k", "min_cluster_size"))
    recipe = open(os.path.join(d, "recipe.txt")).read()
    eo, nv, kk, mm = b["edge_off"], b["n_vertices"], b["k"], b["min_cluster_size"]
    G, total = len(nv), int(eo[-1])
    s = torch.from_numpy(b["src"]).cuda()
    dd = torch.from_numpy(b["dst"]).cuda()
    t = torch.from_numpy(b["t"]).cuda()
    del b
    lab_b = torch.empty(total, dtype=torch.int32, device="cuda")
    # launch configuration tuned on the first 64 graphs as one batch (cached per GPU model)
    tuned = None
    if tune_it:
        from paper_2311_10337_gb300 import tune
        z = int(eo[64])
        tuned = tune.tune(ctx, lambda: ctx.run_batch(s[:z], dd[:z], t[:z], eo[:65], nv[:64], kk[:64], mm[:64]),
                          f"batch-first64:{recipe}", steps=2)
        ctx.ws = None
        torch.cuda.empty_cache()
    # warm-up pass over the first graphs only, then the timed passes over all
    ctx.run_batch_passes(s[:int(eo[8])], dd[:int(eo[8])], t[:int(eo[8])], eo[:9], nv[:8], kk[:8], mm[:8],
                         max_edges, lab_b[:int(eo[8])])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ncl_b, passes = ctx.run_batch_passes(s, dd, t, eo, nv, kk, mm, max_edges, lab_b)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    ctx.ws = None
    torch.cuda.empty_cache()
    # one launch sequence per graph, inputs already resident
    lab_p = torch.empty(total, dtype=torch.int32, device="cuda")
    ncl_p = np.zeros(G, np.int32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g in range(G):
        a, z = int(eo[g]), int(eo[g + 1])
        o = ctx.run(s[a:z], dd[a:z], t[a:z], int(nv[g]), int(kk[g]), int(mm[g]))
        lab_p[a:z].copy_(o.tensor("labels"))
        ncl_p[g] = o.n_clusters
    torch.cuda.synchronize()
    tp = time.perf_counter() - t0
    same = bool(torch.equal(lab_b, lab_p)) and bool(np.array_equal(ncl_b, ncl_p))
    sizes = np.diff(eo)
    del s, dd, t, lab_b, lab_p
    ctx.ws = None
    torch.cuda.empty_cache()
    return {"graphs": G, "edges": total, "recipe": recipe, "edges_min": int(sizes.min()),
            "edges_max": int(sizes.max()), "passes": passes, "max_edges_per_pass": int(max_edges),
            "batched_edges_per_s": total / tb, "batched_s": tb,
            "one_run_per_graph_edges_per_s": total / tp, "one_run_per_graph_s": tp,
            "speedup": tp / tb, "identical_labels_all_graphs": same, "launch_config": tuned}


def serving(d, args):
    """Served form: windowed clustering jobs over a resident edge stream in
    (t, id) order, Poisson arrivals, window sizes log-uniform in [1e4, 1e7]
    edges, k = 8, M = 5. Latency = submission to labels ready; throughput =
    window edges / makespan. A sample of jobs (the largest windows among
    them) is re-run alone and must give identical labels."""
    import torch
    from paper_2311_10337_gb300 import dgec, synth
    arr = _load(d, ("src", "dst", "t"))
    meta = json.load(open(os.path.join(d, "meta.json")))
    S = torch.from_numpy(arr["src"]).cuda()
    D = torch.from_numpy(arr["dst"]).cuda()
    T = torch.from_numpy(arr["t"]).cuda()
    del arr
    E = int(S.shape[0])
    V, k, M = int(meta["n_vertices"]), int(meta["k"]), int(meta["M"])
    srv = dgec.Server(int(args.serve_pool_gb * (1 << 30)), args.serve_lanes, V, max_jobs_per_batch=64)
    cap = srv.lane_capacity()
    n_jobs = args.serve_jobs
    starts, sizes, arrivals = synth.serve_jobs(n_jobs, E, args.serve_rate)
    sizes = np.minimum(sizes, cap)
    # re-checked alone afterwards: the 8 largest windows and 24 others
    rng = np.random.default_rng(0x5E7E)
    check = set(np.argsort(-sizes, kind="stable")[:8].tolist()) | set(rng.choice(n_jobs, 24, replace=False).tolist())
    kept = {}
    lat = np.zeros(n_jobs)
    status = np.zeros(n_jobs, np.int32)
    tickets = [None] * n_jobs
    outs = [None] * n_jobs
    ready = threading.Semaphore(0)

    def waiter():
        for x in range(n_jobs):
            ready.acquire()
            rc, _, ms = srv.wait(tickets[x], 900_000)
            status[x], lat[x] = rc, ms
            if x in check:
                kept[x] = outs[x].cpu()
            outs[x] = None                     # the output buffer returns to the allocator

    th = threading.Thread(target=waiter, daemon=True)
    torch.cuda.synchronize()
    th.start()
    t0 = time.perf_counter()
    for x in range(n_jobs):
        delay = t0 + arrivals[x] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        a, n = int(starts[x]), int(sizes[x])
        outs[x] = torch.empty(n, dtype=torch.int32, device="cuda")
        tickets[x] = srv.submit(S[a:a + n], D[a:a + n], T[a:a + n], k, M, outs[x])
        ready.release()
    th.join()
    torch.cuda.synchronize()
    makespan = time.perf_counter() - t0
    srv.close()
    del srv
    torch.cuda.empty_cache()
    ctx = dgec.Context(0)
    same = True
    for x in sorted(check):
        a, n = int(starts[x]), int(sizes[x])
        o = ctx.run(S[a:a + n], D[a:a + n], T[a:a + n], V, k, M)
        same &= bool(torch.equal(o.tensor("labels").cpu(), kept[x]))
    ctx.close()
    del S, D, T
    torch.cuda.empty_cache()
    return {"jobs": n_jobs, "failed": int(np.sum(status != 0)), "arrivals_per_s": args.serve_rate,
            "lanes": args.serve_lanes, "pool_gb": args.serve_pool_gb, "lane_capacity_edges": cap,
            "window_edges_total": int(sizes.sum()), "window_edges_max": int(sizes.max()),
            "makespan_s": makespan, "edges_per_s": float(sizes.sum() / makespan),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "identical_to_alone": same, "alone_checked_jobs": len(check),
            "stream": f"{meta['recipe']}: {E} edges, {V} vertices"}


def reference_sample_minutes(args, workload) -> float:
    """Window of the reference arm's per-step sample. Unless one is given,
    it shrinks as warm-up + timed steps grow, so that the whole run stays
    within a few minutes of one core."""
    if args.cpu_sample_minutes is not None:
        return args.cpu_sample_minutes
    base = CPU_SAMPLE_MINUTES[workload]
    n = args.warmup + args.steps
    return base if n <= 10 else base * 0.8 if n <= 20 else base * 0.6 if n <= 40 else base * 0.4


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle, as it stands, on a bounded sample."""
    if rank != 0:
        return
    w = make_workload(args.workload, args.scale, 0)
    minutes = reference_sample_minutes(args, args.workload)
    per_step = []
    info = None
    for i in range(args.warmup + args.steps):
        info = cpu_baseline(w, minutes)
        if i >= args.warmup:
            per_step.append(info["value"])
    v = float(np.median(per_step))
    n_sample = int(info["sample"].split(": ")[1].split(" ")[0])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * n_sample / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": f"{w.name}: {w.recipe}, k={w.k}, M={w.min_cluster_size}",
                       "sample": info["sample"]},
            "cpu_baseline": dict(info, value=v),
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    # the large side workloads are drawn by a spawned helper while the GPU works
    gen, futs, tmp = None, {}, None
    if rank == 0 and (args.batch_graphs > 0 or args.serve_jobs > 0):
        tmp = tempfile.mkdtemp(prefix="dgec_bench_")
        gen = ProcessPoolExecutor(max_workers=1, mp_context=mp.get_context("spawn"))
        if args.batch_graphs > 0:
            futs["batch"] = gen.submit(_gen_to_files, "batch", args.batch_graphs, tmp)
        if args.serve_jobs > 0:
            futs["stream"] = gen.submit(_gen_to_files, "stream", args.serve_stream_scale, tmp)
    try:
        run(args, rank, world, local, futs)
    finally:
        if gen is not None:
            gen.shutdown(wait=False, cancel_futures=True)
        if tmp:
            shutil.rmtree(tmp, ignore_errors=True)


def run(args, rank, world, local, futs):
    import torch
    import torch.distributed as dist
    from paper_2311_10337_gb300 import dgec
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    peak, peak_kind = peaks()
    w = make_workload(args.workload, args.scale, rank)
    E, V, k, M = w.n_edges, w.n_vertices, w.k, w.min_cluster_size
    recipe = w.recipe
    ctx = dgec.Context(local)
    src = torch.from_numpy(w.src).cuda()
    dst = torch.from_numpy(w.dst).cuda()
    tt = torch.from_numpy(w.t).cuda()
    stream = torch.cuda.current_stream()
    tuned = None
    if not args.no_tune:
        from paper_2311_10337_gb300 import tune
        tuned = tune.tune(ctx, lambda: ctx.run(src, dst, tt, V, k, M),
                          f"{args.workload}:E={E}:V={V}:k={k}:M={M}", steps=1)
    for _ in range(args.warmup):
        out = ctx.run(src, dst, tt, V, k, M)
    launches = ctx.launches()
    bd = None
    if not args.no_breakdown:
        ctx.set_kernel_timing(2)
        ctx.run(src, dst, tt, V, k, M)
        bd = ctx.kernel_timing()
        ctx.set_kernel_timing(0)
    ctx.set_kernel_timing(3, args.roofline_kernel)  # every kernel of the step: k_knn, or k_knn_pred + k_knn
    clocks = Clocks(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        out = ctx.run(src, dst, tt, V, k, M)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    stages = ctx.stage_timing()           # the last timed step, from the library's stage events
    dom_by = ctx.kernel_timing()
    knn_form = ctx.launch_config()[2]
    ctx.set_kernel_timing(0)
    ms = max_over_ranks(ms, world, "cuda")
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    n_clusters = out.n_clusters
    del out
    # end to end through the host entry point: pinned host inputs in, labels out
    e2e = None
    if not args.no_e2e:
        ctx.ws = None
        torch.cuda.empty_cache()
        hs = torch.from_numpy(w.src).pin_memory().numpy()
        hd = torch.from_numpy(w.dst).pin_memory().numpy()
        ht = torch.from_numpy(w.t).pin_memory().numpy()
        lab = torch.empty(E, dtype=torch.int32).pin_memory().numpy()
        ctx.run_host(hs, hd, ht, V, k, M, labels_out=lab)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.run_host(hs, hd, ht, V, k, M, labels_out=lab)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.steps
        e2e_s = max_over_ranks(e2e_s, world, "cuda")
        e2e = {"value": job_rate(world, E, e2e_s), "unit": UNIT, "h2d_bytes_per_step": 16 * E,
               "d2h_bytes_per_step": 4 * E}
        del hs, hd, ht, lab
    del src, dst, tt
    ctx.ws = None
    torch.cuda.empty_cache()
    side = {}
    if rank == 0:
        roof, top = knn_roofline(dom_by, args.steps, E, k, knn_form, peak, peak_kind, bd, args.roofline_kernel)
        roof.update({
                "stages": stage_report(stages, E, k, peak),
                "pipeline": {"bytes_per_edge": pipeline_bytes_per_edge(k),
                             "achieved": pipeline_bytes_per_edge(k) * E / (ms / 1000.0) / 1e9,
                             "frac": pipeline_bytes_per_edge(k) * E / (ms / 1000.0) / 1e9 / peak}})
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            try:
                cpu = cpu_baseline(w, args.cpu_sample_minutes or CPU_SAMPLE_MINUTES[args.workload])
            except Exception as ex:  # the baseline is a report, never the product path
                cpu = {"error": str(ex)[:200]}
        del w
        steps_side = max(1, min(args.steps, 3))
        for name, fn in (("tiny", lambda: tiny_latency(ctx, max(10, args.steps))),
                         ("mid", (lambda: mid_reports(ctx, args, steps_side, peak)) if not args.no_mid else None),
                         ("hypergraph", (lambda: hypergraphs(ctx, args.hyper_scale, steps_side))
                          if args.hyper_scale > 0 else None)):
            if fn is None:
                continue
            try:
                side[name] = fn()
            except Exception as ex:  # a side report: never costs the main line
                side[name] = {"error": str(ex)[:300]}
            ctx.ws = None
            torch.cuda.empty_cache()
        if "batch" in futs:
            try:
                side["batch"] = batched_vs_plain(ctx, futs["batch"].result(), max_edges=150_000_000,
                                                 tune_it=not args.no_tune)
            except Exception as ex:
                side["batch"] = {"error": str(ex)[:300]}
            ctx.ws = None
            torch.cuda.empty_cache()
        if "stream" in futs:
            try:
                side["serve"] = serving(futs["stream"].result(), args)
            except Exception as ex:
                side["serve"] = {"error": str(ex)[:300]}
        line = {"metric": METRIC, "value": job_rate(world, E, ms / 1000.0), "unit": UNIT,
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                "config": {"workload": f"{args.workload}: {recipe}, k={k}, M={M}",
                           "edges_per_gpu": E, "parallelism": "replicas only",
                           "l2": "inputs (16 B/edge = %.0f MB) exceed L2; no flush" % (16 * E / 1e6),
                           "n_clusters": n_clusters},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches * args.steps, "clocks": clk, "launch_config": tuned,
                "kernel_top": top, **side}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
