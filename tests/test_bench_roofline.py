"""The benchmark's roofline object, computed from a synthetic profile: the entry
with the largest estimated share of the step among those with algorithmic bytes
(sampled entries count PROFILE_PERIOD times), achieved bandwidth from bytes and
time per launch, the measured peak or the fallback, and ncu traffic reported
only while the kernel sources match its capture."""
import pytest

import bench

PROF = {
    "pressure_spmv": (10, 0.5, 1.0e9),   # sampled: share 0.5 x period
    "visc_spmv": (5, 1.0, 2.0e9),        # sampled: share 1.0 x period
    "advect": (3, 2.0, 3.0e8),           # timed at every launch: share 2.0
    "mg_vcycle_v": (5, 9.0, 0.0),        # no byte count: never the roofline entry
    "all_kernels": (100, 0.0, 0.0),
}


def test_picks_the_largest_share_with_bytes():
    r = bench.roofline_of(PROF, {"hbm_gbs": 5000.0}, "h", traffic_table={})
    assert r["kernel"] == "visc_spmv"
    assert r["achieved"] == pytest.approx((2.0e9 / 5) / (1.0e-3 / 5) / 1e9)   # 2000 GB/s
    assert r["frac"] == pytest.approx(r["achieved"] / 5000.0)
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(4.0e8)
    assert r["avg_launch_us"] == pytest.approx(200.0)
    assert r["peak_source"].endswith("(of measured)") and r["traffic"] is None


def test_traffic_only_for_the_matching_sources():
    table = {"visc_spmv": {"bytes_per_launch": 123, "source": "abc"}}
    assert bench.roofline_of(PROF, None, "abc", traffic_table=table)["traffic"] == 123
    assert bench.roofline_of(PROF, None, "xyz", traffic_table=table)["traffic"] is None


def test_fallback_peak_and_empty_profile():
    r = bench.roofline_of(PROF, None, "h", traffic_table={})
    assert r["peak"] == 6800.0 and r["peak_source"] == "fallback"
    assert bench.roofline_of({"all_kernels": (3, 0.0, 0.0)}, None, "h", traffic_table={}) is None
    assert bench.roofline_of({}, None, "h", traffic_table={}) is None


def test_unsampled_entry_wins_when_its_time_is_larger():
    prof = dict(PROF, advect=(3, 9.0, 3.0e8))   # 9.0 > 1.0 x period = 8.0
    assert bench.roofline_of(prof, None, "h", traffic_table={})["kernel"] == "advect"
