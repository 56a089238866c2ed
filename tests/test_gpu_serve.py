"""Serving loop: jobs submitted while others run are batched by the lanes
(continuous batching); every job's labels equal those of the job alone."""
import numpy as np
import pytest

from gpu_helpers import run_gpu
from oracle import oracle as O
from paper_2311_10337_gb300 import dgec, synth

pytestmark = pytest.mark.gpu


def _stream(scale=0.004):
    w = synth.mid(scale=scale)
    order = np.lexsort((np.arange(w.n_edges), w.t))   # the stream in (t, id) order
    return w.src[order], w.dst[order], w.t[order], w.n_vertices


def test_served_jobs_equal_alone():
    import threading
    import time
    import torch
    src, dst, t, V = _stream()
    E = len(src)
    S, D, T = (torch.from_numpy(x).cuda() for x in (src, dst, t))
    rng = np.random.default_rng(11)
    jobs = []
    for _ in range(36):
        n = int(min(E, round(10 ** rng.uniform(2.5, 4.8))))
        a = int(rng.integers(0, E - n + 1))
        jobs.append((a, n, int(rng.choice([4, 8, 16])), int(rng.choice([2, 5]))))
    srv = dgec.Server(pool_bytes=3 << 30, n_lanes=3, vertex_bound=V, max_jobs_per_batch=8)
    outs = [torch.full((n,), -9, dtype=torch.int32, device="cuda") for (_, n, _, _) in jobs]
    tickets = [None] * len(jobs)

    def submitter(lo, hi, gap):
        for x in range(lo, hi):
            a, n, k, M = jobs[x]
            tickets[x] = srv.submit(S[a:a + n], D[a:a + n], T[a:a + n], k, M, outs[x])
            time.sleep(gap)
    # two producers, one bursty and one paced, so jobs arrive while lanes are busy
    th = [threading.Thread(target=submitter, args=(0, 18, 0.0)),
          threading.Thread(target=submitter, args=(18, 36, 0.002))]
    for x in th:
        x.start()
    for x in th:
        x.join()
    res = [srv.wait(tk, 60_000) for tk in tickets]
    torch.cuda.synchronize()
    served = [o.cpu().numpy() for o in outs]
    srv.close()
    for x, (a, n, k, M) in enumerate(jobs):
        rc, ncl, lat = res[x]
        assert rc == 0 and lat > 0, (x, rc)
        alone = run_gpu(src[a:a + n], dst[a:a + n], t[a:a + n], V, k, M)
        assert np.array_equal(served[x], alone["labels"]), x
        assert ncl == alone["n_clusters"]
    a, n, k, M = jobs[0]
    r = O.run(src[a:a + n], dst[a:a + n], t[a:a + n], V, k, M)
    assert np.array_equal(served[0], r["condensed"]["labels"])


def test_served_bad_and_oversize_jobs():
    import torch
    srv = dgec.Server(pool_bytes=256 << 20, n_lanes=1, vertex_bound=1000, max_jobs_per_batch=4)
    cap = srv.lane_capacity()
    assert cap > 1000
    s = torch.tensor([0, 3, 4], dtype=torch.int32, device="cuda")
    d = torch.tensor([1, 3, 0], dtype=torch.int32, device="cuda")   # a self loop
    t = torch.tensor([1, 2, 3], dtype=torch.int64, device="cuda")
    lab = torch.empty(3, dtype=torch.int32, device="cuda")
    bad = srv.submit(s, d, t, 4, 5, lab)
    n = cap + 1
    big = torch.zeros(n, dtype=torch.int32, device="cuda")
    bt = torch.zeros(n, dtype=torch.int64, device="cuda")
    blab = torch.empty(n, dtype=torch.int32, device="cuda")
    over = srv.submit(big, big + 1, bt, 4, 5, blab)
    ok_s = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    ok_d = torch.tensor([1, 2], dtype=torch.int32, device="cuda")
    ok_t = torch.tensor([5, 6], dtype=torch.int64, device="cuda")
    ok_lab = torch.empty(2, dtype=torch.int32, device="cuda")
    good = srv.submit(ok_s, ok_d, ok_t, 4, 2, ok_lab)
    assert srv.wait(bad, 30_000)[0] == 3        # DGEC_ERR_SELF_LOOP
    assert srv.wait(over, 30_000)[0] == 8       # DGEC_ERR_ADMISSION
    rc, ncl, _ = srv.wait(good, 30_000)
    assert rc == 0
    srv.close()
