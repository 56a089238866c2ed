"""The launch configuration changes speed, never results: every candidate
the autotuner may pick gives the same outputs as the default, and the
tuner's choice is cached per GPU model and workload signature."""
import numpy as np
import pytest

from gpu_helpers import ctx, run_gpu
from paper_2311_10337_gb300 import synth

pytestmark = pytest.mark.gpu


def test_every_launch_config_gives_identical_outputs():
    from paper_2311_10337_gb300 import tune
    w = synth.mid(scale=0.002)
    c = ctx()
    default = c.launch_config()
    ref = run_gpu(w.src, w.dst, w.t, w.n_vertices, w.k, w.min_cluster_size)
    try:
        for kb in tune.KNN_BLOCKS:
            for sc in (152, 2432, 65536):
                for packed in (0, 1, 2):
                    c.set_launch_config(kb, sc, packed)
                    got = run_gpu(w.src, w.dst, w.t, w.n_vertices, w.k, w.min_cluster_size)
                    for key in ref:
                        assert np.array_equal(np.asarray(got[key]), np.asarray(ref[key])), (kb, sc, packed, key)
    finally:
        c.set_launch_config(*default)


def test_bad_launch_config_is_rejected():
    from paper_2311_10337_gb300 import dgec
    c = ctx()
    default = c.launch_config()
    for kb, sc, pk in ((96, 1000, 0), (128, 0, 0), (128, (1 << 20) + 1, 0), (128, 1000, 3), (128, 1000, -1)):
        with pytest.raises(dgec.DgecError) as ei:
            c.set_launch_config(kb, sc, pk)
        assert ei.value.status == 1
    assert c.launch_config() == default


def test_tuner_picks_a_candidate_and_caches_it(tmp_path, monkeypatch):
    import torch
    from paper_2311_10337_gb300 import tune
    monkeypatch.setenv("DGEC_TUNE_CACHE", str(tmp_path / "cfg.json"))
    w = synth.tiny()
    s, d, t = (torch.from_numpy(x).cuda() for x in (w.src, w.dst, w.t))
    c = ctx()
    default = c.launch_config()
    try:
        run = lambda: c.run(s, d, t, w.n_vertices, w.k, w.min_cluster_size)
        first = tune.tune(c, run, "tiny-test", steps=1)
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        assert not first["cached"] and first["knn_block"] in tune.KNN_BLOCKS
        assert first["stream_ctas"] in tune.stream_cta_candidates(sms)
        assert first["knn_packed"] in (0, 1, 2)
        chosen = (first["knn_block"], first["stream_ctas"], first["knn_packed"])
        assert c.launch_config() == chosen
        c.set_launch_config(*default)
        again = tune.tune(c, run, "tiny-test", steps=1)
        assert again["cached"] and (again["knn_block"], again["stream_ctas"], again["knn_packed"]) == chosen
        assert c.launch_config() == chosen
    finally:
        c.set_launch_config(*default)
