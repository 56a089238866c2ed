"""Autotuner of the launch configuration (dgec_set_launch_config).

Three parameters change speed and never results: the kNN kernel's threads
per CTA, the CTA count of the grid-stride streaming kernels and the form of
the kNN kernel's candidates (packed 64-bit keys or not). For one GPU
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
    """Pick (knn_block, stream_ctas, knn_packed) for `run` (a callable making
    one call on ctx) and leave ctx configured with it, one parameter at a
    time. Returns the choice, the timings of every candidate tried, and
    whether it came from the cache."""
    import torch
    gpu = torch.cuda.get_device_name(ctx.device)
    path = cache_path()
    if use_cache:
        with _lock:
            hit = _read_cache(path).get(gpu, {}).get(signature)
        if hit:
            ctx.set_launch_config(int(hit["knn_block"]), int(hit["stream_ctas"]), int(hit.get("knn_packed", 0)))
            return dict(hit, cached=True)
    sms = torch.cuda.get_device_properties(ctx.device).multi_processor_count
    cfg = list(ctx.launch_config())
    best = _time_ms(run, steps)  # the starting configuration
    trials = [{"knn_block": cfg[0], "stream_ctas": cfg[1], "knn_packed": cfg[2], "ms": round(best, 3)}]
    for dim, cands in ((1, stream_cta_candidates(sms)), (0, KNN_BLOCKS), (2, (0, 1, 2))):
        best_v = cfg[dim]
        for cand in cands:
            if cand == cfg[dim]:
                continue  # the current value is timed already
            trial = list(cfg)
            trial[dim] = cand
            ctx.set_launch_config(*trial)
            ms = _time_ms(run, steps)
            trials.append({"knn_block": trial[0], "stream_ctas": trial[1], "knn_packed": trial[2],
                           "ms": round(ms, 3)})
            if ms < best:
                best, best_v = ms, cand
        cfg[dim] = best_v
    ctx.set_launch_config(*cfg)
    choice = {"knn_block": cfg[0], "stream_ctas": cfg[1], "knn_packed": cfg[2], "ms": round(best, 3),
              "gpu": gpu, "signature": signature}
    with _lock:
        data = _read_cache(path)
        data.setdefault(gpu, {})[signature] = choice
        try:
            _write_cache(path, data)
        except OSError:
            pass  # a read-only home: the choice still applies to this context
    return dict(choice, cached=False, trials=trials)
