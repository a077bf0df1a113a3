"""The roofline arithmetic of bench.py, without a GPU: each job's bound is the
slower of the write ceiling and its integer ALU bound, the committed ncu
summaries are read only while they match the current sources, and the fused
kernel's bound is the slowest of its three ceilings."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_job_roofline_takes_the_slower_bound():
    # 20 T lane-ops/s over 25 ALU lane-ops per value = 0.8 T values/s = 6.4 TB/s of 8-byte values
    r = bench.job_rooflines({("g", "f64"): 8.0, ("h", "u64"): 8.0}, 7800.0, 20e12, {("g", "f64"): 25.0,
                                                                                       ("h", "u64"): 10.0})
    assert r[("g", "f64")]["bound"] == "alu" and r[("g", "f64")]["roofline_gbs"] == pytest.approx(6400.0)
    assert r[("h", "u64")]["bound"] == "hbm" and r[("h", "u64")]["roofline_gbs"] == 7800.0
    # without a recorded count the write ceiling is the bound
    r = bench.job_rooflines({("x", "u32"): 4.0}, 7800.0, 20e12, {})
    assert r[("x", "u32")]["bound"] == "hbm" and r[("x", "u32")]["alu_bound_gbs"] is None


def test_committed_summaries_match_the_current_sources():
    """The ALU-ops, traffic, fused-kernel and Berlekamp-Massey summaries under
    profiles/ were taken on the current kernel sources (their recorded hashes match), so the
    bench applies them."""
    ops = bench.recorded_alu_ops()
    assert len(ops) == 36 and all(v > 0 for v in ops.values())
    t = bench.recorded_traffic()
    assert t is not None and 0.9 < t["bytes_per_launch"] / t["algorithmic_bytes_per_launch"] <= 1.0
    f = bench.recorded_fused_counts()
    assert f is not None and f["alu_lane_ops_per_stream"] > 1000 and f["shared_wavefronts_per_stream"] > 16
    lc = bench.recorded_lc_alu_ops()
    assert lc is not None and lc > 1e10


def test_fused_roofline_is_the_slowest_ceiling(monkeypatch):
    """2^24 streams x 64 u64: with 1529 ALU lane-ops and 23.7 wavefronts per
    stream at 20 T lane-ops/s and 152 SMs x 2.07 GHz, the ALU bound (1.28 ms)
    is above the shared-memory bound (1.26 ms) and the HBM bound (1.10 ms)."""
    import types
    monkeypatch.setattr(bench, "recorded_fused_counts",
                        lambda: {"alu_lane_ops_per_stream": 1529.25, "shared_wavefronts_per_stream": 23.7})
    fake_torch = types.SimpleNamespace(cuda=types.SimpleNamespace(
        current_device=lambda: 0, get_device_properties=lambda d: types.SimpleNamespace(multi_processor_count=152)))
    monkeypatch.setitem(sys.modules, "torch", fake_torch)
    r = bench.fused_roofline(1 << 24, 64, 1.615, {"write_peak_gbs": 7800.0}, {"alu_lane_ops_per_s": 20.05e12})
    assert r["bound"] == "alu"
    assert r["alu_ms"] == pytest.approx((1 << 24) * 1529.25 / 20.05e12 * 1e3)
    assert r["l1_ms"] == pytest.approx((1 << 24) * 23.7 / (152 * 2.07e9) * 1e3)
    assert r["hbm_ms"] < r["l1_ms"] < r["alu_ms"]
    assert r["frac"] == pytest.approx(r["alu_ms"] / 1.615)
