"""bench.py's host-side arithmetic on synthetic inputs (no GPU): the roofline
fractions it reports, the ncu records that go null when the workload size
or the measured kernel's sources differ, the parity metric, the stratified
estimate of the plain path's time, and the (bin, Gaussian) count of the 2-D
kernels' culling."""
import math

import numpy as np
import pytest

import bench


def test_fp64_roofline_arithmetic():
    # 1e7 x 50 event-points of 33 FP64-pipe instructions in 31.5 ms (arithmetic only)
    r = bench.roofline_fp64("k", 33, 5e8, 31.5e-3, 2070.0)
    peak = 152 * 2 * 2 * 2070e6 / 1e12
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert math.isclose(r["peak"], peak, rel_tol=1e-12) and math.isclose(r["peak"], 1.258560, rel_tol=1e-6)
    assert math.isclose(r["achieved"], 33 * 5e8 * 2 / 31.5e-3 / 1e12, rel_tol=1e-12)
    assert math.isclose(r["frac"], r["achieved"] / peak, rel_tol=1e-12)
    # a kernel that issues its counted instructions at exactly the unit rate reads 1.0
    t_peak = 33 * 5e8 / (152 * 2 * 2070e6)
    assert math.isclose(bench.roofline_fp64("k", 33, 5e8, t_peak, 2070.0)["frac"], 1.0, rel_tol=1e-12)
    # the probe's figure is reported beside the peak, not in place of it
    r = bench.roofline_fp64("k", 33, 5e8, t_peak, 2070.0, {"n_sm": 152, "dfma_per_s": 6.26e11, "ffma_per_s": 1})
    assert math.isclose(r["probe_fp64_tflops"], 1.252, rel_tol=1e-9) and math.isclose(r["frac"], 1.0)


def test_df64_roofline_arithmetic():
    r = bench.roofline_df64("k", 273, 5e8, 5.21e-3, 2070.0)
    peak = 152 * 128 * 2 * 2070e6 / 1e12
    assert math.isclose(r["peak"], peak, rel_tol=1e-12) and math.isclose(r["peak"], 80.54784, rel_tol=1e-9)
    assert math.isclose(r["frac"], 273 * 5e8 * 2 / 5.21e-3 / 1e12 / peak, rel_tol=1e-12)
    assert "issue efficiency" in r["work_per_unit"]


def test_instruction_counts_add_up():
    # the per-unit FP64 counts are the sums spelled out next to them
    exp2, rcp, log = 7, 3, 13
    assert bench.FP64_INSTR["mix"] == 1 + 1 + 1 + 1 + exp2 + 1 + rcp + 1 + 1 + 1 + 3   # lean ratio form
    # a peak: d, c2 d, exp2 of the product c2 d x d (fexp2_prod), the model's FMA
    assert bench.FP64_INSTR["gp1_c1"] == 1 + (1 + 1 + exp2 + 1) + 3 + 5 + 2 + 5 / 4
    assert bench.FP64_INSTR["fit_c4"] == 2 + 3 + 2 + (1 + 1 + exp2 + 1) + 3 + 5 + 4
    assert bench.FP64_INSTR["fit_c5"] == 2 + 1 + 3 * (1 + 1 + exp2 + 1) + log + rcp + 2 + 1 + 15 + 2
    assert bench.FP64_INSTR["rg2_gauss"] == 1 + 4 + exp2 + 1 + 2 + 3   # column form
    assert bench.FP64_INSTR["rg2_bin"] == 2 + log + rcp + 4
    # row recurrence: dy, e R, R + R (q - 1), model, adjoints; per run the exponent at
    # both ends (dy, u', v', v'^2, FMA each), two exp2, the ratio's exponent (two FMAs)
    assert bench.FP64_INSTR["rg2_gauss_rec"] == 1 + 1 + 1 + 1 + 2 + 3
    assert bench.FP64_INSTR["rg2_run_rec"] == 2 * 5 + 2 * exp2 + 2


def test_ncu_records_are_null_for_other_sizes_or_sources(monkeypatch):
    rec = {"sources": bench.FP64_SOURCES, "sources_sha256_16": bench.sources_hash(bench.FP64_SOURCES),
           "workload": [bench.N_EVENTS, bench.N_POINTS], "dram_bytes": 8.1e7, "fp64_pipe_pct": 86.0}
    monkeypatch.setitem(bench.NCU_RECORDS, "k_test", rec)
    assert bench.ncu_record("k_test", bench.N_EVENTS, bench.N_POINTS)["dram_bytes"] == 8.1e7
    assert bench.ncu_record("k_test", bench.N_EVENTS + 1, bench.N_POINTS) is None
    assert bench.ncu_record("k_test", bench.N_EVENTS, bench.N_POINTS - 1) is None
    monkeypatch.setitem(bench.NCU_RECORDS, "k_test", dict(rec, sources_sha256_16="0" * 16))
    assert bench.ncu_record("k_test", bench.N_EVENTS, bench.N_POINTS) is None
    assert bench.ncu_record("k_absent") is None


class _R:
    def __init__(self, value, grad, scale):
        self.value, self.grad, self.scale = value, np.asarray(grad, float), np.asarray(scale, float)


def test_parity_metric():
    # e_k = |g - o| / max(|o|, 1e-6 S): a component near zero is judged against its scale
    refs = [_R(10.0, [1.0, 0.0], [5.0, 1e3])]
    p = bench.parity([10.0], [[1.0 + 1e-11, 1e-8]], refs)
    assert math.isclose(p["max_grad_rel_err"], 1e-8 / 1e-3, rel_tol=1e-6) and not p["ok"]
    p = bench.parity([10.0 * (1 + 5e-11)], [[1.0 + 5e-11, 5e-14]], refs)
    assert p["ok"] and p["max_grad_rel_err"] <= 1e-10 and math.isclose(p["max_value_rel_err"], 5e-11, rel_tol=1e-3)


def test_stratified_estimate():
    rng = np.random.default_rng(0)
    pop = [rng.uniform(1, 2, 100), rng.uniform(10, 20, 50)]
    # every unit sampled: the exact total and no sampling error
    est, se = bench.stratified_estimate([(len(p), p) for p in pop])
    assert math.isclose(est, sum(p.sum() for p in pop)) and se == 0.0
    # a sample: the formula, term by term
    s = [pop[0][:10], pop[1][:5]]
    est, se = bench.stratified_estimate([(100, s[0]), (50, s[1])])
    assert math.isclose(est, 100 * s[0].mean() + 50 * s[1].mean())
    v = 100 ** 2 * s[0].var(ddof=1) / 10 * 0.9 + 50 ** 2 * s[1].var(ddof=1) / 5 * 0.9
    assert math.isclose(se, math.sqrt(v))
    # the strata partition the histograms
    sizes = rng.integers(64, 65536, 1000)
    st = bench._strata(sizes, 8, 24)
    allp = np.concatenate([p for p, _ in st])
    assert sorted(allp.tolist()) == list(range(1000)) and all(set(i) <= set(p) for p, i in st)
    assert all(sizes[st[k][0]].max() <= sizes[st[k + 1][0]].min() for k in range(7))


def test_culled_pair_count_of_the_2d_kernels():
    # one wide Gaussian reaches every tile; a narrow one only the tiles near its centre
    wide = np.array([100.0, 0.5, 0.5, 1.0, 1.0, 0.0, 5.0])
    assert bench._c3_active_pairs(wide, K=1, nx=256, ny=256) == 256 * 256
    narrow = np.array([100.0, 0.5, 0.5, 0.001, 0.001, 0.0, 5.0])
    # r^2 / (2 s^2) <= 80: r <= 0.0126, inside the 2 x 2 tiles of 64 / 1024 around the centre
    assert bench._c3_active_pairs(narrow, K=1, nx=1024, ny=1024) == 4 * 64 * 64
    # split by the tiles' kept counts (the recurrence takes tiles of at most 5): same total
    assert bench._c3_active_pairs(narrow, K=1, nx=1024, ny=1024, by_kept=True) == [0, 4 * 64 * 64]
    # elongated along y: the exponent reaches -80 within 0.0126 of the centre in x but
    # everywhere in y (0.5^2 / (2 0.05^2) = 50), so 2 x 16 tiles of 1024^2; rotated by
    # 90 degrees, 16 x 2; the isotropic bound max(sx, sy) would keep far more
    long_y = np.array([100.0, 0.5, 0.5, 0.001, 0.05, 0.0, 5.0])
    assert bench._c3_active_pairs(long_y, K=1, nx=1024, ny=1024) == 2 * 16 * 64 * 64
    long_x = long_y.copy()
    long_x[5] = np.pi / 2
    assert bench._c3_active_pairs(long_x, K=1, nx=1024, ny=1024) == 2 * 16 * 64 * 64
