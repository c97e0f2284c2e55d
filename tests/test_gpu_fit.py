"""Fitters on the GPU: the batched persistent fitter (warp / CTA / cluster
units, graph replay), the plain per-histogram path and the batched
per-histogram gradient, against the oracle (gradients to 1e-10, fitted
minima to 1e-6 relative in objective value)."""
import numpy as np
import pytest
import torch

import oracle
from oracle.fit import bfgs_fit
from paper_2203_06139_gb300 import cg, synth
from paper_2203_06139_gb300.fit import BatchFitter, HistBatch, SingleFitter, TileMap, autotune
from tests._metrics import max_rel_err

pytestmark = pytest.mark.gpu
OBJ_MAP = {cg.OBJ_CHI2: oracle.CHI2, cg.OBJ_POISSON: oracle.POISSON, cg.OBJ_POISSON_BC: oracle.POISSON_BC}


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def small_c4(H=48, max_bins=20000, seed_index=3):
    d = synth.c4_batch(H=H, min_bins=64, max_bins=max_bins, index=seed_index)
    return d


def oracle_fit(y, K, D, pm, obj, lo, hi, th0, max_iter=200):
    fg = lambda t: (lambda r: (r.value, r.grad))(oracle.binned1d(K, D, pm, obj, y, lo, hi, t))
    gn = lambda t: oracle.binned1d_gn(K, D, pm, obj, y, lo, hi, t)
    return bfgs_fit(fg, gn, th0, max_iter=max_iter, tol=1e-12)


def test_batch_gradient_per_histogram(dev):
    d = small_c4(H=24)
    b = HistBatch(d["y"], d["offsets"], d["lo"], d["hi"], 1, 2, cg.OBJ_CHI2, poly_mode=1)
    th = torch.tensor(d["start"], device=dev)
    v, g = b.gradient(th)
    g = g.cpu().numpy()
    for h in range(d["H"]):
        y = d["y"][d["offsets"][h]:d["offsets"][h + 1]]
        ref = oracle.binned1d(1, 2, 1, oracle.CHI2, y, 0.0, 1.0, d["start"][h])
        assert max_rel_err(g[h], ref.grad, ref.scale) <= 1e-10
        assert abs(float(v[h]) - ref.value) <= 1e-10 * abs(ref.value)


def test_init_matches_oracle_gn_and_gradient(dev):
    d = small_c4(H=16)
    b = HistBatch(d["y"], d["offsets"], d["lo"], d["hi"], 1, 2, cg.OBJ_CHI2, poly_mode=1)
    f = BatchFitter(b, TileMap(1024, 8192, 256, 2))
    st = f.init(torch.tensor(d["start"], device=dev))
    h0 = st.d[:, 168:168 + 6].cpu().numpy()
    for h in range(d["H"]):
        y = d["y"][d["offsets"][h]:d["offsets"][h + 1]]
        gn = oracle.binned1d_gn(1, 2, 1, oracle.CHI2, y, 0.0, 1.0, d["start"][h])
        np.testing.assert_allclose(1.0 / h0[h], gn, rtol=1e-10)
    assert torch.all(st.status == cg.FIT_RUNNING)


@pytest.mark.parametrize("tmap", [TileMap(1 << 30, 1 << 30, 256, 1), TileMap(0, 1 << 30, 256, 1),
                                  TileMap(0, 0, 128, 2), TileMap(1024, 8192, 256, 4), TileMap(512, 4096, 128, 8)],
                         ids=["all-warp", "all-cta", "all-cluster2", "mixed-c4", "mixed-c8"])
def test_batched_fit_reaches_oracle_minimum(dev, tmap):
    d = small_c4(H=40)
    b = HistBatch(d["y"], d["offsets"], d["lo"], d["hi"], 1, 2, cg.OBJ_CHI2, poly_mode=1)
    f = BatchFitter(b, tmap)
    f.init(torch.tensor(d["start"], device=dev))
    st = f.step(n_steps=200, tol=1e-12)
    torch.cuda.synchronize()
    F = st.f.cpu().numpy()
    status = st.status.cpu().numpy()
    assert np.all(status == cg.FIT_CONVERGED) or np.all(np.isin(status, [cg.FIT_CONVERGED, cg.FIT_LINESEARCH_FAILED]))
    for h in range(0, d["H"], 3):
        y = d["y"][d["offsets"][h]:d["offsets"][h + 1]]
        ref = oracle_fit(y, 1, 2, 1, oracle.CHI2, 0.0, 1.0, d["start"][h])
        assert abs(F[h] - ref["F"]) <= 1e-6 * abs(ref["F"]), (h, F[h], ref["F"], status[h])


def test_mappings_agree(dev):
    d = small_c4(H=32, max_bins=40000)
    b = HistBatch(d["y"], d["offsets"], d["lo"], d["hi"], 1, 2, cg.OBJ_CHI2, poly_mode=1)
    res = []
    for m in [TileMap(1 << 30, 1 << 30, 256, 1), TileMap(0, 1 << 30, 512, 1), TileMap(256, 2048, 256, 8)]:
        f = BatchFitter(b, m)
        f.init(torch.tensor(d["start"], device=dev))
        res.append(f.step(200, 1e-12).f.cpu().numpy())
    for r in res[1:]:
        np.testing.assert_allclose(r, res[0], rtol=1e-8)


def test_graph_replay_equals_eager(dev):
    d = small_c4(H=24)
    b = HistBatch(d["y"], d["offsets"], d["lo"], d["hi"], 1, 2, cg.OBJ_CHI2, poly_mode=1)
    m = TileMap(1024, 8192, 256, 4)
    f1 = BatchFitter(b, m)
    f1.init(torch.tensor(d["start"], device=dev))
    eager = f1.step(3, 1e-12).raw.clone()
    f2 = BatchFitter(b, m)
    f2.init(torch.tensor(d["start"], device=dev))
    f2.capture(3, 1e-12)
    f2.replay()
    torch.cuda.synchronize()
    assert torch.equal(f2.states.raw, eager)


@pytest.mark.parametrize("obj", [cg.OBJ_POISSON, cg.OBJ_POISSON_BC])
def test_batched_fit_poisson_three_peaks(dev, obj):
    d = synth.c5_batch(H=12, n_bins=2048)
    b = HistBatch(d["y"], d["offsets"], d["lo"], d["hi"], 3, 1, obj, poly_mode=0)
    start = d["truth"] * np.random.default_rng(1).uniform(0.97, 1.03, d["truth"].shape)
    f = BatchFitter(b, TileMap(4096, 1 << 30, 256, 1))
    f.init(torch.tensor(start, device=dev))
    st = f.step(200, 1e-12)
    F = st.f.cpu().numpy()
    for h in range(0, 12, 4):
        y = d["y"][d["offsets"][h]:d["offsets"][h + 1]]
        ref = oracle_fit(y, 3, 1, 0, OBJ_MAP[obj], 0.0, 1.0, start[h], max_iter=400)
        assert abs(F[h] - ref["F"]) <= 1e-6 * abs(ref["F"]), (h, F[h], ref["F"])


def test_single_path_full_c1_fit(dev):
    """The plain per-histogram path on 10,000 bins, to the oracle's minimum."""
    h = synth.c1_histogram()
    pb = cg.Problem.gauss_poly(torch.tensor(h["y"], device=dev), 0.0, 10.0, 1, 1, cg.OBJ_CHI2)
    th0 = synth.c1_theta_points(1)[0]
    sf = SingleFitter(pb)
    st = sf.fit(torch.tensor(th0, device=dev), max_iter=200, tol=1e-12)
    ref = oracle_fit(h["y"], 1, 1, 0, oracle.CHI2, 0.0, 10.0, th0)
    assert int(st.status[0]) == cg.FIT_CONVERGED
    assert abs(float(st.f[0]) - ref["F"]) <= 1e-6 * abs(ref["F"])


def test_autotuner_returns_a_valid_map(dev, tmp_path, monkeypatch):
    monkeypatch.setenv("CG_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    d = small_c4(H=64, max_bins=65536)
    b = HistBatch(d["y"], d["offsets"], d["lo"], d["hi"], 1, 2, cg.OBJ_CHI2, poly_mode=1)
    best, timings = autotune(b, torch.tensor(d["start"], device=dev), n_steps=2)
    assert len(timings) >= 4 and isinstance(best, TileMap)
    best2, _ = autotune(b, torch.tensor(d["start"], device=dev), n_steps=2)
    assert best2.as_dict() == best.as_dict()


@pytest.mark.parametrize("obj,K,D,pm", [(cg.OBJ_CHI2, 1, 2, 1), (cg.OBJ_POISSON_BC, 3, 1, 0)])
def test_batched_fit_df64_reaches_oracle_minimum(dev, obj, K, D, pm):
    if K == 1:
        d = small_c4(H=24)
        start = d["start"]
    else:
        d = synth.c5_batch(H=12, n_bins=2048)
        start = d["truth"] * np.random.default_rng(1).uniform(0.97, 1.03, d["truth"].shape)
    b = HistBatch(d["y"], d["offsets"], d["lo"], d["hi"], K, D, obj, poly_mode=pm, precision=cg.PREC_DF64)
    f = BatchFitter(b, TileMap(1024, 8192, 256, 4))
    f.init(torch.tensor(start, device=dev))
    F = f.step(200, 1e-12).f.cpu().numpy()
    for h in range(0, d["H"], 3):
        y = d["y"][d["offsets"][h]:d["offsets"][h + 1]]
        ref = oracle_fit(y, K, D, pm, OBJ_MAP[obj], 0.0, 1.0, start[h], max_iter=400)
        assert abs(F[h] - ref["F"]) <= 1e-6 * abs(ref["F"]), (h, F[h], ref["F"])
