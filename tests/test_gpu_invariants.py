"""Invariants of the CUDA path that hold without a reference value.

Noise-free data: counts equal to the truth density (drawn from the
generator's own evaluation of the model, not from either gradient code)
make every residual zero, so the exact gradient vanishes at the truth; on
the GPU every per-bin term is then rounding noise, bounded here as for the
oracle: |g_k| <= 1e-12 S_k with S_k the oracle's per-component scale 1 %
away from the truth.  Checked for the 1-D models of the single-histogram
and batched workloads (chi2, Poisson, Baker-Cousins) and the 2-D model, on
the FP64 and the double-float paths.

Determinism: a result depends only on the problem and the reduction tree,
which the problem size, the number of parameter points and the tile map fix;
repeats on other streams, from CUDA graphs, and under tile maps that keep a
histogram in the same kind of unit are bitwise equal.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2203_06139_gb300 import cg, synth
from paper_2203_06139_gb300.fit import BatchFitter, HistBatch, TileMap

pytestmark = pytest.mark.gpu
PRECS = [cg.PREC_FP64, cg.PREC_DF64]
ORC = {cg.OBJ_CHI2: oracle.CHI2, cg.OBJ_POISSON: oracle.POISSON, cg.OBJ_POISSON_BC: oracle.POISSON_BC}


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("obj", [cg.OBJ_CHI2, cg.OBJ_POISSON, cg.OBJ_POISSON_BC])
def test_noise_free_gradient_vanishes_1d(obj, prec):
    h = synth.c1_histogram(n_bins=10000, noise=False)
    y = torch.tensor(h["y"], device="cuda")
    pb = cg.Problem.gauss_poly(y, 0.0, 10.0, 1, 1, obj, precision=prec)
    v, g = cg.gradient(pb, torch.tensor(h["truth"], device="cuda"))
    torch.cuda.synchronize()
    assert pb.status() == cg.OK
    ref = oracle.binned1d(1, 1, 0, ORC[obj], h["y"], 0.0, 10.0, h["truth"] * 1.01)
    assert np.all(np.abs(g.cpu().numpy()) <= 1e-12 * ref.scale)
    assert np.all(np.abs(ref.grad) > 1e-3 * ref.scale)     # the bound is not vacuous


@pytest.mark.parametrize("prec", PRECS)
def test_noise_free_gradient_vanishes_2d(prec):
    truth = synth.c3_truth(8)
    counts = synth.expected_counts_2d(truth, 8, 512, 384)
    pb = cg.Problem.rotgauss2d(torch.tensor(counts, device="cuda"), 8, precision=prec)
    v, g = cg.gradient(pb, torch.tensor(truth, device="cuda"))
    torch.cuda.synchronize()
    assert pb.status() == cg.OK
    ref = oracle.binned2d(8, counts, 0.0, 1.0, 0.0, 1.0, truth * 1.01)
    assert np.all(np.abs(g.cpu().numpy()) <= 1e-12 * ref.scale)


@pytest.mark.parametrize("prec", PRECS)
def test_noise_free_gradient_vanishes_batched(prec):
    """Gaussian + quadratic (in t = 2x - 1) histograms of the batched workload,
    chi2, through the batched gradient call."""
    d = synth.c4_batch(H=12, max_bins=20000)
    offs, truth = d["offsets"], d["truth"]
    y = np.concatenate([synth.expected_counts_1d(1, 2, 1, 0.0, 1.0, int(offs[h + 1] - offs[h]), truth[h])
                        for h in range(12)])
    b = HistBatch(y, offs, d["lo"], d["hi"], 1, 2, cg.OBJ_CHI2, poly_mode=1, precision=prec)
    v, g = b.gradient(torch.tensor(truth, device="cuda"))
    g = g.cpu().numpy()
    for h in range(12):
        ref = oracle.binned1d(1, 2, 1, oracle.CHI2, y[offs[h]:offs[h + 1]], 0.0, 1.0, truth[h] * 1.01)
        assert np.all(np.abs(g[h]) <= 1e-12 * ref.scale), h


def test_bitwise_across_streams_and_graphs():
    """The same call eagerly on the current stream, on a side stream, and
    replayed from a CUDA graph: bitwise the same values and gradients."""
    x = torch.tensor(synth.c2_events(300007), device="cuda")
    th = torch.tensor(synth.c2_theta_points(7), device="cuda")
    hy = torch.tensor(synth.c1_histogram()["y"], device="cuda")
    thy = torch.tensor(synth.c1_theta_points(9), device="cuda")
    for pb, t in ((cg.Problem.mixture(x, 0.0, 10.0), th),
                  (cg.Problem.mixture(x, 0.0, 10.0, precision=cg.PREC_DF64), th),
                  (cg.Problem.gauss_poly(hy, 0.0, 10.0, 1, 1, cg.OBJ_CHI2), thy)):
        v0, g0 = cg.batch_gradient(pb, t)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            v1, g1 = cg.batch_gradient(pb, t)
        torch.cuda.current_stream().wait_stream(s)
        v2 = torch.empty_like(v0)
        g2 = torch.empty_like(g0)
        with torch.cuda.stream(s):
            cg.batch_gradient(pb, t, v2, g2)   # warm the capture stream
        torch.cuda.current_stream().wait_stream(s)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            cg.batch_gradient(pb, t, v2, g2)
        v2.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for a, b in ((v0, v1), (g0, g1), (v0, v2), (g0, g2)):
            assert torch.equal(a, b)


@pytest.mark.parametrize("prec", PRECS)
def test_fits_bitwise_across_maps_that_keep_the_unit(prec):
    """Two tile maps that differ only in the warp/CTA threshold: histograms in
    the same kind of unit under both (warp below 512 bins, CTA of 256 threads
    above 2048) follow the same reduction tree and end bitwise equal, whatever
    else the maps move between units."""
    d = synth.c4_batch(H=64, max_bins=8192)
    sizes = np.diff(d["offsets"])
    th0 = torch.tensor(d["start"], device="cuda")
    b = HistBatch(d["y"], d["offsets"], d["lo"], d["hi"], 1, 2, cg.OBJ_CHI2, poly_mode=1, precision=prec)
    out = []
    for m in (TileMap(512, 1 << 30, 256, 1), TileMap(2048, 1 << 30, 256, 1)):
        f = BatchFitter(b, m)
        f.init(th0)
        st = f.step(20, 1e-9)
        torch.cuda.synchronize()
        out.append((st.theta.clone(), st.f.clone()))
    keep = torch.tensor((sizes <= 512) | (sizes > 2048), device="cuda")
    assert int(keep.sum()) >= 32
    assert torch.equal(out[0][0][keep], out[1][0][keep]) and torch.equal(out[0][1][keep], out[1][1][keep])
    assert bool(torch.isfinite(out[0][1]).all()) and bool(torch.isfinite(out[1][1]).all())
