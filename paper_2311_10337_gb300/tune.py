"""Autotuner of the launch configuration (dgec_set_launch_config).

Two parameters change speed and never results: the kNN kernel's threads per
CTA and the CTA count of the grid-stride streaming kernels. For one GPU
model and one workload shape the tuner times the whole path (CUDA events on
the launching stream, after a warm-up) for each candidate, one parameter at
a time, keeps the fastest, and caches the choice in a JSON file keyed by the
GPU's name and the workload signature, so that later runs on the same model
skip the search.
"""
from __future__ import annotations

import json
import os
import threading

KNN_BLOCKS = (64, 128, 256)
_lock = threading.Lock()


def stream_cta_candidates(num_sms: int) -> tuple:
    """Multiples of the SM count (resident CTAs per SM of 256 threads: up to
    8) and the library's default."""
    return tuple(sorted({num_sms * 8, num_sms * 32, num_sms * 128, 65536}))


def cache_path() -> str:
    return os.environ.get("DGEC_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "dgec", "launch_config.json"))


def _read_cache(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _write_cache(path, data):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_ms(run, steps):
    import torch
    run()
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def tune(ctx, run, signature: str, steps: int = 2, use_cache: bool = True) -> dict:
    """Pick (knn_block, stream_ctas) for `run` (a callable making one call
    on ctx) and leave ctx configured with it. Returns the choice, the
    timings of every candidate tried, and whether it came from the cache."""
    import torch
    gpu = torch.cuda.get_device_name(ctx.device)
    path = cache_path()
    if use_cache:
        with _lock:
            hit = _read_cache(path).get(gpu, {}).get(signature)
        if hit:
            ctx.set_launch_config(int(hit["knn_block"]), int(hit["stream_ctas"]))
            return dict(hit, cached=True)
    sms = torch.cuda.get_device_properties(ctx.device).multi_processor_count
    kb, sc = ctx.launch_config()
    trials = []
    best_sc, best = sc, None
    for cand in stream_cta_candidates(sms):
        ctx.set_launch_config(kb, cand)
        ms = _time_ms(run, steps)
        trials.append({"knn_block": kb, "stream_ctas": cand, "ms": round(ms, 3)})
        if best is None or ms < best:
            best, best_sc = ms, cand
    best_kb = kb
    for cand in KNN_BLOCKS:
        if cand == kb:
            continue
        ctx.set_launch_config(cand, best_sc)
        ms = _time_ms(run, steps)
        trials.append({"knn_block": cand, "stream_ctas": best_sc, "ms": round(ms, 3)})
        if ms < best:
            best, best_kb = ms, cand
    ctx.set_launch_config(best_kb, best_sc)
    choice = {"knn_block": best_kb, "stream_ctas": best_sc, "ms": round(best, 3), "gpu": gpu,
              "signature": signature}
    with _lock:
        data = _read_cache(path)
        data.setdefault(gpu, {})[signature] = choice
        try:
            _write_cache(path, data)
        except OSError:
            pass  # a read-only home: the choice still applies to this context
    return dict(choice, cached=False, trials=trials)
