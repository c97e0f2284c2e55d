"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bar: max over components of |g - g_oracle| / max(|g_oracle|, 1e-6 S_k) and
the relative error of the value both <= 1e-10 in FP64 (S_k = sum over
elements of |dT_i/dtheta_k|, from the oracle).  Inputs come from the seeded
generators in paper_2203_06139_gb300.synth.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2203_06139_gb300 import cg, synth
from tests._metrics import max_rel_err, value_rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-10

OBJ_MAP = {cg.OBJ_CHI2: oracle.CHI2, cg.OBJ_POISSON: oracle.POISSON, cg.OBJ_POISSON_BC: oracle.POISSON_BC}


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def check(v, g, ref, tol=TOL):
    g = g.detach().cpu().numpy() if isinstance(g, torch.Tensor) else g
    v = float(v)
    assert ref.rc == oracle.OK
    e = max_rel_err(g, ref.grad, ref.scale)
    ev = value_rel_err(v, ref.value)
    assert e <= tol and ev <= tol, (e, ev, g, ref.grad, v, ref.value)
    return e, ev


# --------------------------------------------------------------------------
# 1-D binned, Gaussian peaks + polynomial
# --------------------------------------------------------------------------
CASES_1D = [(1, 1, 0), (0, 2, 1), (2, 2, 1), (3, 1, 0), (4, 3, 1), (1, -1, 0), (2, 0, 0)]


@pytest.mark.parametrize("obj", [cg.OBJ_CHI2, cg.OBJ_POISSON, cg.OBJ_POISSON_BC])
@pytest.mark.parametrize("K,D,pm", CASES_1D)
def test_gauss_poly_small(dev, obj, K, D, pm):
    n = 3001  # several tiles and a ragged tail
    p = synth.random_gauss_poly(max(K, 1), D, n, lo=-2.0, hi=3.0, poly_mode=pm, seed=10 * K + D + pm)
    if K == 0:
        th0 = p["theta"][3:].copy()
        th0[0] = abs(th0[0]) + 50.0
        y = np.random.default_rng(4).poisson(np.maximum(
            synth.expected_counts_1d(0, D, pm, -2.0, 3.0, n, th0), 1.0)).astype(float)
        thetas = np.stack([th0, th0 * 1.03, th0 * 0.97])
    else:
        y = p["y"]
        thetas = np.stack([p["theta"], p["truth"] * 1.02, p["truth"]])
    pb = cg.Problem.gauss_poly(torch.tensor(y, device=dev), -2.0, 3.0, K, D, obj, poly_mode=pm)
    v, g = cg.batch_gradient(pb, torch.tensor(thetas, device=dev))
    assert pb.status(len(thetas)) == cg.OK
    for i in range(len(thetas)):
        ref = oracle.binned1d(K, D, pm, OBJ_MAP[obj], y, -2.0, 3.0, thetas[i])
        check(v[i], g[i], ref)


def test_gauss_poly_single_point_calls(dev):
    p = synth.random_gauss_poly(2, 1, 777, seed=5)
    pb = cg.Problem.gauss_poly(torch.tensor(p["y"], device=dev), 0.0, 1.0, 2, 1, cg.OBJ_POISSON)
    th = torch.tensor(p["theta"], device=dev)
    v, g = cg.gradient(pb, th)
    v2 = cg.objective(pb, th)
    ref = oracle.binned1d(2, 1, 0, oracle.POISSON, p["y"], 0.0, 1.0, p["theta"])
    check(v, g, ref)
    assert float(v2) == float(v)


def test_gauss_poly_explicit_centres_and_unaligned(dev):
    n = 2049
    p = synth.random_gauss_poly(1, 2, n + 1, seed=8)
    centres = np.sort(np.random.default_rng(3).uniform(0.0, 1.0, n + 1))
    y = p["y"]
    yt = torch.tensor(y, device=dev)
    ct = torch.tensor(centres, device=dev)
    # explicit centres, aligned
    pb = cg.Problem.gauss_poly(yt, 0.0, 1.0, 1, 2, cg.OBJ_CHI2, centres=ct)
    v, g = cg.gradient(pb, torch.tensor(p["theta"], device=dev))
    check(v, g, oracle.binned1d(1, 2, 0, oracle.CHI2, y, 0.0, 1.0, p["theta"], centres=centres))
    # views starting one element in: 8-byte aligned only, scalar-load path
    pb2 = cg.Problem.gauss_poly(yt[1:], 0.0, 1.0, 1, 2, cg.OBJ_CHI2, centres=ct[1:])
    assert pb2.data.data_ptr() % 16 == 8
    v, g = cg.gradient(pb2, torch.tensor(p["theta"], device=dev))
    check(v, g, oracle.binned1d(1, 2, 0, oracle.CHI2, y[1:], 0.0, 1.0, p["theta"], centres=centres[1:]))


@pytest.mark.parametrize("n", [1, 2, 3, 255, 256, 257, 511, 512, 513, 4096, 4097])
def test_gauss_poly_sizes(dev, n):
    p = synth.random_gauss_poly(1, 1, n, seed=n)
    pb = cg.Problem.gauss_poly(torch.tensor(p["y"], device=dev), 0.0, 1.0, 1, 1, cg.OBJ_POISSON_BC)
    v, g = cg.gradient(pb, torch.tensor(p["theta"], device=dev))
    check(v, g, oracle.binned1d(1, 1, 0, oracle.POISSON_BC, p["y"], 0.0, 1.0, p["theta"]))


def test_empty_histogram(dev):
    y = torch.zeros(0, dtype=torch.float64, device=dev)
    pb = cg.Problem.gauss_poly(y, 0.0, 1.0, 1, 1, cg.OBJ_CHI2)
    v, g = cg.gradient(pb, torch.tensor([1.0, 0.5, 0.1, 1.0, 0.0], dtype=torch.float64, device=dev))
    assert float(v) == 0.0 and torch.all(g == 0)
    assert pb.status() == cg.OK


def test_domain_errors_are_reported_and_cleared(dev):
    p = synth.random_gauss_poly(1, 0, 1000, seed=2)
    pb = cg.Problem.gauss_poly(torch.tensor(p["y"], device=dev), 0.0, 1.0, 1, 0, cg.OBJ_POISSON)
    bad = p["theta"].copy()
    bad[3] = -1e4  # background far below zero: log of a negative model value
    cg.gradient(pb, torch.tensor(bad, device=dev))
    assert pb.status() == cg.ERR_DOMAIN
    zero_w = p["theta"].copy()
    zero_w[2] = 0.0
    cg.gradient(pb, torch.tensor(zero_w, device=dev))
    assert pb.status() == cg.ERR_DOMAIN
    cg.gradient(pb, torch.tensor(p["theta"], device=dev))
    assert pb.status() == cg.OK


def test_invalid_arguments_raise(dev):
    y = torch.ones(10, dtype=torch.float64, device=dev)
    with pytest.raises(cg.CgError):
        cg.Problem.gauss_poly(y, 0.0, 1.0, 5, 1).n_params
    with pytest.raises(cg.CgError):
        cg.Problem.gauss_poly(y.float(), 0.0, 1.0, 1, 1)
    pb = cg.Problem.gauss_poly(y, 1.0, 1.0, 1, 1)
    with pytest.raises(cg.CgError):
        cg.gradient(pb, torch.ones(5, dtype=torch.float64, device=dev))


def test_deterministic_repeats(dev):
    h = synth.c1_histogram()
    pb = cg.Problem.gauss_poly(torch.tensor(h["y"], device=dev), 0.0, 10.0, 1, 1, cg.OBJ_CHI2)
    th = torch.tensor(synth.c1_theta_points(), device=dev)
    v0, g0 = cg.batch_gradient(pb, th)
    v0, g0 = v0.clone(), g0.clone()
    for _ in range(20):
        v, g = cg.batch_gradient(pb, th)
        assert torch.equal(v, v0) and torch.equal(g, g0)


def test_c1_full_size_all_points(dev):
    """10,000 bins x 100 parameter points, in the launch the bench times."""
    h = synth.c1_histogram()
    th = synth.c1_theta_points()
    pb = cg.Problem.gauss_poly(torch.tensor(h["y"], device=dev), 0.0, 10.0, 1, 1, cg.OBJ_CHI2)
    v, g = cg.batch_gradient(pb, torch.tensor(th, device=dev))
    refs = oracle.many(oracle.binned1d, th, K=1, D=1, poly_mode=0, obj=oracle.CHI2, y=h["y"], lo=0.0, hi=10.0)
    g = g.cpu().numpy()
    for i, ref in enumerate(refs):
        check(v[i], g[i], ref)


# --------------------------------------------------------------------------
# unbinned mixture
# --------------------------------------------------------------------------
def test_mixture_small(dev):
    x = synth.c2_events(100003)
    th = synth.c2_theta_points(5)
    pm = cg.Problem.mixture(torch.tensor(x, device=dev), 0.0, 10.0)
    v, g = cg.batch_gradient(pm, torch.tensor(th, device=dev))
    for i in range(5):
        check(v[i], g[i], oracle.unbinned_mix(x, 0.0, 10.0, th[i]))


def test_mixture_weighted_and_other_range(dev):
    x = synth.c2_events(50001, truth=np.array([0.6, 3.0, 0.8, 0.3]), lo=1.0, hi=7.5)
    w = np.random.default_rng(9).uniform(0.2, 2.0, x.size)
    th = np.array([0.55, 3.1, 0.75, 0.33])
    pm = cg.Problem.mixture(torch.tensor(x, device=dev), 1.0, 7.5, weights=torch.tensor(w, device=dev))
    v, g = cg.gradient(pm, torch.tensor(th, device=dev))
    check(v, g, oracle.unbinned_mix(x, 1.0, 7.5, th, weights=w))


# Points that take each form of the FP64 mixture element: the lean ratio
# form (a, b > 0, the exponential's share well above 1/16), the
# two-exponential form (a = 0 at f = 0), a ratio form whose
# Gaussian-to-exponential ratio exceeds 2^1021 for the events near a steep
# exponential's far end (those take the per-event fallback), and fractions
# next to 1 (log2(a/b) near 23: the exponential's share is so small that its
# sums taken as differences would cancel, and the tiles are summed again in
# the full ratio form).
MIX_FORM_POINTS = np.array([[0.3, 2.0, 0.3, 0.5],
                            [0.0, 2.0, 0.3, 0.5],
                            [0.3, 9.0, 0.5, 100.0],
                            [0.9999999, 2.1, 0.28, 0.45],
                            [0.999, 0.5, 0.05, 9.0]])


@pytest.mark.parametrize("weighted", [False, True])
def test_mixture_fp64_both_forms_in_one_launch(dev, weighted):
    x = np.concatenate([synth.c2_events(40001), np.array([9.99, 9.999, 9.0, 0.0, 1e-12, 5.0])])
    w = np.random.default_rng(11).uniform(0.2, 2.0, x.size) if weighted else None
    wt = torch.tensor(w, device=dev) if weighted else None
    pm = cg.Problem.mixture(torch.tensor(x, device=dev), 0.0, 10.0, weights=wt)
    v, g = cg.batch_gradient(pm, torch.tensor(MIX_FORM_POINTS, device=dev))
    assert pm.status(len(MIX_FORM_POINTS)) == cg.OK
    for i, th in enumerate(MIX_FORM_POINTS):
        check(v[i], g[i], oracle.unbinned_mix(x, 0.0, 10.0, th, weights=w))


@pytest.mark.slow
def test_c2_full_size_sampled_points(dev):
    """10^7 events x 50 points in the bench's launch; the oracle checks a sample of points."""
    x = synth.c2_events()
    th = synth.c2_theta_points()
    pm = cg.Problem.mixture(torch.tensor(x, device=dev), 0.0, 10.0)
    v, g = cg.batch_gradient(pm, torch.tensor(th, device=dev))
    assert pm.status(50) == cg.OK
    idx = [0, 17, 33, 49]
    refs = oracle.many(oracle.unbinned_mix, th[idx], x=x, lo=0.0, hi=10.0)
    g = g.cpu().numpy()
    for i, ref in zip(idx, refs):
        check(v[i], g[i], ref)


# --------------------------------------------------------------------------
# 2-D rotated Gaussians
# --------------------------------------------------------------------------
@pytest.mark.parametrize("K,nx,ny", [(1, 31, 17), (3, 67, 45), (8, 129, 97)])
def test_rotgauss2d_small(dev, K, nx, ny):
    truth = synth.c3_truth(K)
    counts = np.random.default_rng(K).poisson(synth.expected_counts_2d(truth, K, nx, ny)).astype(float)
    th = truth * (1 + np.random.default_rng(K + 1).uniform(-0.05, 0.05, truth.size))
    p2 = cg.Problem.rotgauss2d(torch.tensor(counts, device=dev), K)
    v, g = cg.gradient(p2, torch.tensor(th, device=dev))
    check(v, g, oracle.binned2d(K, counts, 0.0, 1.0, 0.0, 1.0, th))


def test_rotgauss2d_elongated_culling(dev):
    """Narrow, elongated Gaussians at 30 and 120 degrees across many 64 x 64
    tiles of a ragged 333 x 301 grid (and one centred outside the grid): the
    tiles' culling by the exact maximum of the exponent over each box keeps
    the result at the oracle's, which has no culling."""
    th = np.array([300.0, 0.4, 0.55, 0.004, 0.08, np.pi / 6,
                   200.0, 0.7, 0.3, 0.06, 0.003, 2 * np.pi / 3,
                   150.0, 1.05, 0.5, 0.01, 0.02, 0.3,
                   2.0])
    K, nx, ny = 3, 333, 301
    counts = np.random.default_rng(21).poisson(synth.expected_counts_2d(th, K, nx, ny)).astype(float)
    p2 = cg.Problem.rotgauss2d(torch.tensor(counts, device=dev), K)
    for t in (th, th * (1 + np.random.default_rng(22).uniform(-0.03, 0.03, th.size))):
        v, g = cg.gradient(p2, torch.tensor(t, device=dev))
        check(v, g, oracle.binned2d(K, counts, 0.0, 1.0, 0.0, 1.0, t))


@pytest.mark.slow
def test_c3_full_size(dev):
    """4096 x 4096 bins, 8 rotated Gaussians + constant, one parameter point."""
    h = synth.c3_histogram()
    th = synth.c3_theta_point(h["truth"])[0]
    p2 = cg.Problem.rotgauss2d(torch.tensor(h["counts"], device=dev), 8)
    v, g = cg.gradient(p2, torch.tensor(th, device=dev))
    check(v, g, oracle.binned2d(8, h["counts"], 0.0, 1.0, 0.0, 1.0, th))


# --------------------------------------------------------------------------
# double-float (FP32-pipe) path: same bar against the oracle, and its error
# against the FP64 path is recorded
# --------------------------------------------------------------------------
def test_mixture_df64_small(dev):
    x = synth.c2_events(100003)
    th = synth.c2_theta_points(5)
    pm = cg.Problem.mixture(torch.tensor(x, device=dev), 0.0, 10.0, precision=cg.PREC_DF64)
    v, g = cg.batch_gradient(pm, torch.tensor(th, device=dev))
    assert pm.status(5) == cg.OK
    for i in range(5):
        check(v[i], g[i], oracle.unbinned_mix(x, 0.0, 10.0, th[i]))


def test_mixture_df64_weighted_other_range(dev):
    x = synth.c2_events(50001, truth=np.array([0.6, 3.0, 0.8, 0.3]), lo=1.0, hi=7.5)
    w = np.random.default_rng(9).uniform(0.2, 2.0, x.size)
    th = np.array([0.55, 3.1, 0.75, 0.33])
    pm = cg.Problem.mixture(torch.tensor(x, device=dev), 1.0, 7.5, weights=torch.tensor(w, device=dev),
                            precision=cg.PREC_DF64)
    v, g = cg.gradient(pm, torch.tensor(th, device=dev))
    check(v, g, oracle.unbinned_mix(x, 1.0, 7.5, th, weights=w))


def test_mixture_df64_tails_fall_back(dev):
    """Events deep in both tails (both exponentials below 1e-30 of their
    coefficients) take the FP64 fallback; results still match the oracle."""
    x = np.concatenate([synth.c2_events(4001), np.array([9.99, 9.999, 0.0, 1e-12])])
    th = np.array([0.999, 0.5, 0.05, 9.0])   # narrow Gaussian, steep exponential
    pm = cg.Problem.mixture(torch.tensor(x, device=dev), 0.0, 10.0, precision=cg.PREC_DF64)
    v, g = cg.gradient(pm, torch.tensor(th, device=dev))
    check(v, g, oracle.unbinned_mix(x, 0.0, 10.0, th))


@pytest.mark.slow
def test_c2_df64_full_size_and_error_vs_fp64(dev, record_property):
    x = synth.c2_events()
    th = synth.c2_theta_points()
    xt, tt = torch.tensor(x, device=dev), torch.tensor(th, device=dev)
    p64 = cg.Problem.mixture(xt, 0.0, 10.0)
    pdf = cg.Problem.mixture(xt, 0.0, 10.0, precision=cg.PREC_DF64)
    v64, g64 = cg.batch_gradient(p64, tt)
    vdf, gdf = cg.batch_gradient(pdf, tt)
    assert pdf.status(50) == cg.OK
    idx = [0, 17, 33, 49]
    refs = oracle.many(oracle.unbinned_mix, th[idx], x=x, lo=0.0, hi=10.0)
    for i, ref in zip(idx, refs):
        check(vdf[i], gdf[i], ref)
    # stated error of the double-float path against the FP64 path, all 50 points
    gv = (gdf - g64).abs() / g64.abs()
    vv = (vdf - v64).abs() / v64.abs()
    err_g, err_v = float(gv.max()), float(vv.max())
    record_property("df64_vs_fp64_max_rel_grad", err_g)
    record_property("df64_vs_fp64_max_rel_value", err_v)
    print("df64 vs fp64: max rel grad %.3e, value %.3e" % (err_g, err_v))
    assert err_g < 1e-11 and err_v < 1e-12


@pytest.mark.parametrize("obj", [cg.OBJ_CHI2, cg.OBJ_POISSON, cg.OBJ_POISSON_BC])
@pytest.mark.parametrize("K,D,pm", [(1, 1, 0), (2, 2, 1), (3, 1, 0), (4, 3, 1), (0, 2, 1), (1, -1, 0)])
def test_gauss_poly_df64_small(dev, obj, K, D, pm):
    n = 3001
    p = synth.random_gauss_poly(max(K, 1), D, n, lo=-2.0, hi=3.0, poly_mode=pm, seed=10 * K + D + pm)
    if K == 0:
        th0 = p["theta"][3:].copy()
        th0[0] = abs(th0[0]) + 50.0
        y = np.random.default_rng(4).poisson(np.maximum(
            synth.expected_counts_1d(0, D, pm, -2.0, 3.0, n, th0), 1.0)).astype(float)
        thetas = np.stack([th0, th0 * 1.03])
    else:
        y = p["y"]
        thetas = np.stack([p["theta"], p["truth"] * 1.02])
    pb = cg.Problem.gauss_poly(torch.tensor(y, device=dev), -2.0, 3.0, K, D, obj, poly_mode=pm,
                               precision=cg.PREC_DF64)
    v, g = cg.batch_gradient(pb, torch.tensor(thetas, device=dev))
    assert pb.status(len(thetas)) == cg.OK
    for i in range(len(thetas)):
        check(v[i], g[i], oracle.binned1d(K, D, pm, OBJ_MAP[obj], y, -2.0, 3.0, thetas[i]))


def test_c1_df64_full_size_all_points(dev):
    h = synth.c1_histogram()
    th = synth.c1_theta_points()
    pb = cg.Problem.gauss_poly(torch.tensor(h["y"], device=dev), 0.0, 10.0, 1, 1, cg.OBJ_CHI2, precision=cg.PREC_DF64)
    v, g = cg.batch_gradient(pb, torch.tensor(th, device=dev))
    refs = oracle.many(oracle.binned1d, th, K=1, D=1, poly_mode=0, obj=oracle.CHI2, y=h["y"], lo=0.0, hi=10.0)
    g = g.cpu().numpy()
    for i, ref in enumerate(refs):
        check(v[i], g[i], ref)


@pytest.mark.parametrize("obj", [cg.OBJ_CHI2, cg.OBJ_POISSON_BC])
def test_value_only_matches_gradient_value(dev, obj):
    p = synth.random_gauss_poly(3, 1, 5001, seed=77)
    pb = cg.Problem.gauss_poly(torch.tensor(p["y"], device=dev), 0.0, 1.0, 3, 1, obj, precision=cg.PREC_DF64)
    th = torch.tensor(np.stack([p["theta"], p["truth"]]), device=dev)
    v, _ = cg.batch_gradient(pb, th)
    vo = cg.batch_objective(pb, th)
    for i in range(2):
        ref = oracle.binned1d(3, 1, 0, OBJ_MAP[obj], p["y"], 0.0, 1.0, th[i].cpu().numpy())
        assert abs(float(vo[i]) - ref.value) <= 1e-10 * abs(ref.value)
    torch.testing.assert_close(vo, v, rtol=1e-13, atol=0)


@pytest.mark.parametrize("K,nx,ny", [(1, 31, 17), (3, 130, 70), (8, 200, 129)])
def test_rotgauss2d_df64_small(dev, K, nx, ny):
    truth = synth.c3_truth(K)
    counts = np.random.default_rng(K).poisson(synth.expected_counts_2d(truth, K, nx, ny)).astype(float)
    th = truth * (1 + np.random.default_rng(K + 1).uniform(-0.05, 0.05, truth.size))
    p2 = cg.Problem.rotgauss2d(torch.tensor(counts, device=dev), K, precision=cg.PREC_DF64)
    v, g = cg.gradient(p2, torch.tensor(th, device=dev))
    assert p2.status() == cg.OK
    check(v, g, oracle.binned2d(K, counts, 0.0, 1.0, 0.0, 1.0, th))


@pytest.mark.slow
def test_c3_df64_full_size(dev):
    h = synth.c3_histogram()
    th = synth.c3_theta_point(h["truth"])[0]
    p2 = cg.Problem.rotgauss2d(torch.tensor(h["counts"], device=dev), 8, precision=cg.PREC_DF64)
    v, g = cg.gradient(p2, torch.tensor(th, device=dev))
    check(v, g, oracle.binned2d(8, h["counts"], 0.0, 1.0, 0.0, 1.0, th))
