"""The bench's kNN roofline object, built from kernel timers on the host: the
unit of work is the kNN step of one pass whichever form ran (one launch in
the per-edge forms, the two list-order passes otherwise), the DRAM traffic
comes from the capture of the form that ran, and the step's share of the
pass sums every kernel of the step."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402

E = 200_000_000
PEAK = 6702.2


def test_list_order_form_counts_both_passes_per_pass():
    timed = {"k_knn_pred": (5 * 10.0, 5), "k_knn": (5 * 33.0, 5)}  # five timed passes
    roof, _ = bench.knn_roofline(timed, 5, E, 8, 2, PEAK, "measured", None)
    assert roof["ms_per_pass"] == pytest.approx(43.0)
    assert roof["avg_launch_ms"] == pytest.approx(21.5)
    assert roof["launches_per_step"] == 2
    assert roof["kernels"] == ["k_knn", "k_knn_pred"]
    assert roof["algorithmic_bytes_per_edge"] == 64  # lists 24 + ids 4k + core 8 at k = 8
    assert roof["achieved"] == pytest.approx(64 * E / 0.043 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / PEAK)
    per_edge = bench.KNN_TRAFFIC_BYTES_PER_EDGE_K8[2]
    assert roof["traffic"] == pytest.approx(per_edge * E)
    assert roof["traffic_over_algorithmic"] == pytest.approx(per_edge / 64)


def test_per_edge_form_uses_its_own_capture():
    roof, _ = bench.knn_roofline({"k_knn": (3 * 43.5, 3)}, 3, E, 8, 1, PEAK, "measured", None)
    assert roof["ms_per_pass"] == pytest.approx(43.5)
    assert roof["avg_launch_ms"] == pytest.approx(43.5)
    assert roof["launches_per_step"] == 1
    assert roof["traffic"] == pytest.approx(bench.KNN_TRAFFIC_BYTES_PER_EDGE_K8[1] * E)


def test_no_capture_means_no_traffic():
    # form 0 has no capture, and the captures hold for k = 8 only
    for form, k in ((0, 8), (2, 16), (1, 4)):
        roof, _ = bench.knn_roofline({"k_knn": (10.0, 1)}, 1, E, k, form, PEAK, "measured", None)
        assert roof["traffic"] is None and roof["traffic_over_algorithmic"] is None
        assert roof["algorithmic_bytes_per_edge"] == 24 + 4 * k + 8


def test_share_sums_every_kernel_of_the_step():
    bd = {"k_knn_pred": (10.0, 1), "k_knn": (30.0, 1), "k_radix_scatter": (40.0, 96), "k_c_cpar": (20.0, 1)}
    roof, top = bench.knn_roofline({"k_knn": (30.0, 1), "k_knn_pred": (10.0, 1)}, 1, E, 8, 2, PEAK,
                                   "measured", bd)
    assert roof["share_of_step"] == pytest.approx(0.4)
    assert [t[0] for t in top] == ["k_radix_scatter", "k_knn", "k_c_cpar", "k_knn_pred"]
    assert top[0][3] == pytest.approx(0.4)


def test_nothing_timed_gives_empty_figures():
    roof, top = bench.knn_roofline({}, 5, E, 8, 2, PEAK, "measured", None)
    assert roof["achieved"] is None and roof["frac"] is None and roof["ms_per_pass"] is None
    assert roof["launches_per_step"] == 0 and top is None
