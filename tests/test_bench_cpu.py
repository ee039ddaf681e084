"""The benchmark's roofline arithmetic on synthetic counters (no GPU): the dominant pass,
its bound, achieved rate and fraction follow from the per-pair and per-byte counts, and the
measured DRAM traffic is reported only when it was captured from the current sources."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6781.1, "sm_max_mhz": 2070.0}
GEOM = {"sms": 152, "pixels": 3840 * 2160, "K": 16, "N": 10_000_000, "params": 590_000_000, "sort_passes": 2,
        "flat_backward": True}


def _prof(stages, counters):
    return {"stages": stages, "counters": counters}


def test_blend_backward_is_alu_bound_and_its_fraction_follows_the_counts():
    cnt = {"bwd_pairs": 2e9, "bwd_contrib": 1.9e9, "fwd_instances_staged": 2e7, "visible": 6e6}
    prof = _prof({"blend_bwd": (8.0, 2), "adam": (5.0, 2)}, cnt)
    rl = bench.roofline(prof, PEAKS, "measured", {}, {}, GEOM)
    assert rl["kernel"] == "blend_bwd" and rl["bound"] == "alu" and rl["unit"] == "TFLOP/s"
    peak = 152 * bench.FP32_LANES_PER_SM * 2 * 2070e6
    flops = 70 * 1e9                       # per launch: 70 FP32 operations per evaluated pair
    assert rl["algorithmic_flops"] == pytest.approx(flops)
    assert rl["achieved"] == pytest.approx(flops / 4e-3 / 1e12)
    assert rl["peak"] == pytest.approx(peak / 1e12)
    assert rl["frac"] == pytest.approx(rl["achieved"] / rl["peak"])
    # bytes per launch: 24 B per pixel, 36 B per staged record and per visible splat
    assert rl["algorithmic_bytes"] == pytest.approx(24 * GEOM["pixels"] + 36 * 1e7 + 36 * 3e6)
    assert rl["traffic"] is None           # no capture given
    assert set(rl["next"]) == {"adam"} and rl["next"]["adam"]["bound"] == "hbm"
    assert rl["next"]["adam"]["achieved"] == pytest.approx(28 * GEOM["params"] / 2.5e-3 / 1e9)


def test_traffic_is_reported_only_for_the_sources_it_was_captured_from():
    cnt = {"bwd_pairs": 2e9, "bwd_contrib": 1.9e9, "fwd_instances_staged": 2e7, "visible": 6e6}
    prof = _prof({"blend_bwd": (8.0, 2)}, cnt)
    table = {"blend_bwd": {"dram_bytes_per_launch": 250_000_000, "source": "raster.cu", "source_sha": "abc",
                           "workload": "city-10M-3840x2160-K16"}}
    hit = bench.roofline(prof, PEAKS, "measured", {"raster.cu": "abc"}, table, GEOM, "city-10M-3840x2160-K16")
    assert hit["traffic"] == 250_000_000
    stale = bench.roofline(prof, PEAKS, "measured", {"raster.cu": "def"}, table, GEOM, "city-10M-3840x2160-K16")
    assert stale["traffic"] is None
    other = bench.roofline(prof, PEAKS, "measured", {"raster.cu": "abc"}, table, GEOM, "object-1M-1600x1060-K8")
    assert other["traffic"] is None


def test_adam_is_hbm_bound_at_28_bytes_per_parameter():
    prof = _prof({"adam": (5.0, 2)}, {})
    rl = bench.roofline(prof, PEAKS, "measured", {}, {}, GEOM)
    assert rl["kernel"] == "adam" and rl["bound"] == "hbm" and rl["unit"] == "GB/s"
    assert rl["algorithmic_bytes"] == pytest.approx(28 * GEOM["params"])
    assert rl["frac"] == pytest.approx(rl["achieved"] / PEAKS["hbm_gbs"])
