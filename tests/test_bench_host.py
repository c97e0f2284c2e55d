"""bench.py's host-side arithmetic on synthetic inputs (no GPU): the roofline
fractions it reports, and the DRAM-traffic figure that goes null when the
workload size or the measured kernel's sources differ."""
import math

import pytest

import bench


def test_df64_roofline_arithmetic():
    # 1e7 x 50 event-points of 273 FP32-pipe operations in 5.21 ms
    r = bench.df64_roofline(5.21e-3, 1e7 * 50, None, 2070.0)
    peak = 152 * 128 * 2 * 2070e6 / 1e12
    achieved = 273 * 5e8 * 2 / 5.21e-3 / 1e12
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert math.isclose(r["peak"], peak, rel_tol=1e-12) and math.isclose(r["peak"], 80.54784, rel_tol=1e-9)
    assert math.isclose(r["achieved"], achieved, rel_tol=1e-12)
    assert math.isclose(r["frac"], achieved / peak, rel_tol=1e-12)
    # a kernel at exactly the unit rate reads 1.0
    t_peak = 273 * 5e8 / (152 * 128 * 2070e6)
    assert math.isclose(bench.df64_roofline(t_peak, 5e8, None, 2070.0)["frac"], 1.0, rel_tol=1e-12)


def test_fp64_roofline_and_equivalent():
    rates = {"n_sm": 152, "dfma_per_s": 6.26e11, "exp_per_s": 2.6e10, "log_per_s": 1.7e10, "rcp_per_s": 7.9e10}
    slots = 17 + 2 * 6.26e11 / 2.6e10 + 6.26e11 / 1.7e10 + 6.26e11 / 7.9e10
    peak_dfma = 152 * 2 * 2070e6
    r = bench.fp64_roofline(72.7e-3, 5e8, rates, 2070.0)
    assert math.isclose(r["frac"], slots * 5e8 / 72.7e-3 / peak_dfma, rel_tol=1e-12)
    e = bench.fp64_equivalent(5.21e-3, 5e8, rates, 2070.0, bench.MIX_OPS)
    assert math.isclose(e["fp64_bound_ms"], slots * 5e8 / peak_dfma * 1e3, rel_tol=1e-12)
    assert math.isclose(e["frac"], e["fp64_bound_ms"] / 5.21, rel_tol=1e-12)


def test_traffic_is_null_for_other_sizes_or_sources(tmp_path):
    rec = dict(bench.DF64_MIX_TRAFFIC)
    assert bench._traffic_if_current(rec, bench.N_EVENTS + 1, bench.N_POINTS) is None
    assert bench._traffic_if_current(rec, bench.N_EVENTS, bench.N_POINTS - 1) is None
    stale = dict(rec, sources_sha256_16="0" * 16)
    assert bench._traffic_if_current(stale, bench.N_EVENTS, bench.N_POINTS) is None
    assert bench._traffic_if_current(rec, bench.N_EVENTS, bench.N_POINTS) in (None, rec["bytes"])
