"""The benchmark's roofline objects, computed from synthetic profiles: the single
kernel with the largest estimated share of the step (mean duration times the
launches that did work) among those with algorithmic bytes, achieved bandwidth
from bytes and time per launch, the measured peak or the fallback, ncu traffic
reported only while the kernel sources match its capture; aggregates of several
kernels (a V-cycle) never win; the level-0 multigrid family sums its kernels."""
import pytest

import bench

# name: (timed launches, total ms, bytes of the timed launches, launches that did work)
PROF = {
    "pressure_spmv": (10, 0.5, 1.0e9, 80),   # mean 0.05 ms x 80 = 4.0
    "visc_spmv": (5, 1.0, 2.0e9, 40),        # mean 0.2 ms x 40 = 8.0
    "advect": (3, 2.0, 3.0e8, 3),            # 2.0
    "mg_vcycle_v": (5, 9.0, 1.0e9, 40),      # an aggregate: never the roofline entry
    "all_kernels": (100, 0.0, 0.0),
}


def test_picks_the_largest_share_with_bytes():
    r = bench.roofline_of(PROF, {"hbm_gbs": 5000.0}, "h", traffic_table={})
    assert r["kernel"] == "visc_spmv"
    assert r["achieved"] == pytest.approx((2.0e9 / 5) / (1.0e-3 / 5) / 1e9)   # 2000 GB/s
    assert r["frac"] == pytest.approx(r["achieved"] / 5000.0)
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(4.0e8)
    assert r["avg_launch_us"] == pytest.approx(200.0)
    assert r["launches_all"] == 40
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


def test_launch_counts_decide_the_share():
    # a kernel timed at every launch but launched rarely loses to a sampled one launched often
    prof = dict(PROF, advect=(3, 9.0, 3.0e8, 3))          # 9.0 > 8.0
    assert bench.roofline_of(prof, None, "h", traffic_table={})["kernel"] == "advect"
    prof = dict(PROF, advect=(3, 6.0, 3.0e8, 3))          # 6.0 < 8.0
    assert bench.roofline_of(prof, None, "h", traffic_table={})["kernel"] == "visc_spmv"
    # a three-field profile (no launch count) counts its timed launches
    old = {k: v[:3] for k, v in PROF.items()}
    assert bench.roofline_of(old, None, "h", traffic_table={})["kernel"] == "advect"


def test_kernel_table_and_family():
    prof = {"mg0_smooth2": (4, 0.2, 4.0e8, 32), "mg0_residual": (4, 0.2, 2.0e8, 32), "mg_coarse": (4, 0.1, 0.0, 16),
            "all_kernels": (500, 0.0, 0.0)}
    t = bench.kernel_table(prof, step_ms=10.0, steps=2, hbm=4000.0)
    assert set(t) == {"mg0_smooth2", "mg0_residual", "mg_coarse"}
    assert t["mg0_smooth2"]["est_share_of_step"] == pytest.approx(0.05 * 32 / 20.0)
    assert t["mg0_smooth2"]["achieved_gbs"] == pytest.approx(2000.0)
    assert t["mg0_smooth2"]["frac_of_hbm"] == pytest.approx(0.5)
    assert "achieved_gbs" not in t["mg_coarse"]
    fam = bench.family_roofline(prof, {"hbm_gbs": 4000.0})
    assert fam["achieved"] == pytest.approx((6.0e8) / (0.4e-3) / 1e9)      # 1500 GB/s
    assert fam["frac"] == pytest.approx(1500.0 / 4000.0)
    assert bench.family_roofline({"all_kernels": (1, 0.0, 0.0)}, None) is None


def test_traffic_entry_with_its_own_files():
    # an entry that names its files is matched against their hash, not the global one
    good = bench.source_hash(("fs_mg.cu", "fs_mask.cu"))
    prof = {"mg0_smooth2": (3, 0.09, 3 * 6.7e7, 100)}
    table = {"mg0_smooth2": {"bytes_per_launch": 5, "source": good, "files": ("fs_mg.cu", "fs_mask.cu")}}
    assert bench.roofline_of(prof, None, "other", traffic_table=table)["traffic"] == 5
    table["mg0_smooth2"]["source"] = "0" * 16
    assert bench.roofline_of(prof, None, good, traffic_table=table)["traffic"] is None
