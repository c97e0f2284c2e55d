"""Second-order fits on the GPU: the Gauss-Newton matrix of every histogram
of a df64 batch against the oracle's, and Levenberg-Marquardt fits against
the oracle's minima.

The matrix is accumulated in FP32 (products h r_a r_b of the raw Jacobian
factors, summed per thread, then in df64 across threads): with m bins per
thread each entry's error is below about (m + 8) 2^-24 sum_i |h r_a r_b|
<= (m + 8) 2^-24 sqrt(GN_aa GN_bb) (Cauchy-Schwarz), so with at most 20000
bins over 256 threads (m <= 79) the bound below is 1e-5 of
sqrt(GN_aa GN_bb).  Value and gradient are the df64 ones (1e-10)."""
import numpy as np
import pytest
import torch

import oracle
from oracle.fit import CONVERGED, bfgs_fit, lm_fit
from paper_2203_06139_gb300 import cg, synth
from paper_2203_06139_gb300.fit import _H, _H0, HistBatch, LMFitter
from tests._metrics import max_rel_err

pytestmark = pytest.mark.gpu
OBJ_MAP = {cg.OBJ_CHI2: oracle.CHI2, cg.OBJ_POISSON: oracle.POISSON, cg.OBJ_POISSON_BC: oracle.POISSON_BC}
GN_TOL = 1e-5


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def _narrow_peak_batch(ns, seed=5):
    """A narrow Gaussian and no background: far from the peak the df64
    exponential underflows and those bins take the FP64 fallback."""
    rng = np.random.default_rng(seed)
    ys, starts = [], []
    for n in ns:
        th = np.array([rng.uniform(200.0, 2000.0), rng.uniform(0.4, 0.6), rng.uniform(0.01, 0.03)])
        ys.append(rng.poisson(synth.expected_counts_1d(1, -1, 0, 0.0, 1.0, n, th)).astype(float))
        starts.append(th * rng.uniform(0.95, 1.05, 3))
    offsets = np.concatenate([[0], np.cumsum([len(y) for y in ys])]).astype(np.int64)
    H = len(ns)
    return dict(y=np.concatenate(ys), offsets=offsets, lo=np.zeros(H), hi=np.ones(H), start=np.stack(starts), H=H)


def _case(name):
    if name == "chi2_K1_D2":
        d = synth.c4_batch(H=12, min_bins=64, max_bins=20000, index=3)
        return d, cg.OBJ_CHI2, 1, 2, 1
    if name == "bc_K3_D1":
        d = synth.c5_batch(H=6, n_bins=2048)
        d["start"] = d["truth"] * np.random.default_rng(1).uniform(0.97, 1.03, d["truth"].shape)
        return d, cg.OBJ_POISSON_BC, 3, 1, 0
    if name == "bc_K1_D3":
        ps = [synth.random_gauss_poly(1, 3, n, poly_mode=1, seed=30 + i) for i, n in enumerate([500, 7000])]
        y = np.concatenate([p["y"] for p in ps])
        offs = np.concatenate([[0], np.cumsum([p["n"] for p in ps])]).astype(np.int64)
        d = dict(y=y, offsets=offs, lo=np.zeros(2), hi=np.ones(2), start=np.stack([p["theta"] for p in ps]), H=2)
        return d, cg.OBJ_POISSON_BC, 1, 3, 1
    if name == "poisson_K2_D0":
        ps = [synth.random_gauss_poly(2, 0, n, seed=20 + i) for i, n in enumerate([100, 1500, 9000])]
        y = np.concatenate([p["y"] for p in ps])
        offs = np.concatenate([[0], np.cumsum([p["n"] for p in ps])]).astype(np.int64)
        d = dict(y=y, offsets=offs, lo=np.zeros(3), hi=np.ones(3), start=np.stack([p["theta"] for p in ps]), H=3)
        return d, cg.OBJ_POISSON, 2, 0, 0
    d = _narrow_peak_batch([100, 700, 3000, 12000])
    return d, (cg.OBJ_POISSON if name == "poisson_narrow_peak" else cg.OBJ_POISSON_BC), 1, -1, 0


CASES = ["chi2_K1_D2", "bc_K3_D1", "bc_K1_D3", "poisson_K2_D0", "poisson_narrow_peak", "bc_narrow_peak"]


@pytest.mark.parametrize("name", CASES)
def test_gauss_newton_matrix_matches_the_oracle(dev, name):
    d, obj, K, D, pm = _case(name)
    b = HistBatch(d["y"], d["offsets"], d["lo"], d["hi"], K, D, obj, poly_mode=pm, precision=cg.PREC_DF64)
    th = d["start"]
    v, g, G = (t.cpu().numpy() for t in b.gauss_newton(torch.tensor(th, device=dev)))
    v2, g2, G2 = (t.cpu().numpy() for t in b.gauss_newton(torch.tensor(th, device=dev)))
    assert np.array_equal(G, G2) and np.array_equal(g, g2)          # deterministic
    vb, gb = (t.cpu().numpy() for t in b.gradient(torch.tensor(th, device=dev)))
    for h in range(d["H"]):
        y = d["y"][d["offsets"][h]:d["offsets"][h + 1]]
        r = oracle.binned1d(K, D, pm, OBJ_MAP[obj], y, d["lo"][h], d["hi"][h], th[h])
        assert abs(v[h] - r.value) <= 1e-10 * abs(r.value), (h, v[h], r.value)
        assert max_rel_err(g[h], r.grad, r.scale) <= 1e-10
        ref = oracle.binned1d_gnmat(K, D, pm, OBJ_MAP[obj], y, d["lo"][h], d["hi"][h], th[h])
        dd = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
        err = np.max(np.abs(G[h] - ref) / np.where(dd > 0, dd, 1.0))
        assert err <= GN_TOL, (h, err)
        assert np.array_equal(G[h], G[h].T)
    # the same value and gradient as the first-order call
    assert np.array_equal(v, vb) or np.max(np.abs(v - vb) / np.abs(vb)) <= 1e-15


@pytest.mark.parametrize("name", ["chi2_K1_D2", "bc_K3_D1", "bc_K1_D3", "poisson_narrow_peak"])
def test_lm_fit_reaches_the_oracle_minimum(dev, name):
    """Every fit converges; its objective equals the oracle's BFGS minimum
    (and the oracle's LM minimum) to 1e-6 relative."""
    d, obj, K, D, pm = _case(name)
    b = HistBatch(d["y"], d["offsets"], d["lo"], d["hi"], K, D, obj, poly_mode=pm, precision=cg.PREC_DF64)
    f = LMFitter(b)
    f.init(torch.tensor(d["start"], device=dev), tol=1e-12)
    st = f.step(100, 1e-12)
    F, status, th = st.f.cpu().numpy(), st.status.cpu().numpy(), st.theta.cpu().numpy()
    assert np.all(status == CONVERGED), status
    o = OBJ_MAP[obj]
    for h in range(d["H"]):
        y = d["y"][d["offsets"][h]:d["offsets"][h + 1]]
        lo, hi = d["lo"][h], d["hi"][h]
        fg = lambda t: (lambda q: (q.value, q.grad))(oracle.binned1d(K, D, pm, o, y, lo, hi, t))
        gn = lambda t: oracle.binned1d_gn(K, D, pm, o, y, lo, hi, t)
        ref = bfgs_fit(fg, gn, d["start"][h], max_iter=400, tol=1e-12)
        assert abs(F[h] - ref["F"]) <= 1e-6 * abs(ref["F"]), (h, F[h], ref["F"])
        fgh = lambda t: fg(t) + (oracle.binned1d_gnmat(K, D, pm, o, y, lo, hi, t),)
        rl = lm_fit(fgh, d["start"][h], max_evals=101, tol=1e-12)
        assert abs(F[h] - rl["F"]) <= 1e-6 * abs(rl["F"])


def test_lm_first_steps_follow_the_oracle(dev):
    """Five evaluations from the same start: the same accept / reject
    decisions (iterations and damping) as the oracle's LM, and the same point
    to the accuracy of the FP32 matrix."""
    d, obj, K, D, pm = _case("chi2_K1_D2")
    b = HistBatch(d["y"], d["offsets"], d["lo"], d["hi"], K, D, obj, poly_mode=pm, precision=cg.PREC_DF64)
    f = LMFitter(b)
    f.init(torch.tensor(d["start"], device=dev), tol=0.0)
    st = f.step(4, 0.0)
    th, iters, lam = st.theta.cpu().numpy(), st.iters.cpu().numpy(), st.d[:, _H0].cpu().numpy()
    for h in range(d["H"]):
        y = d["y"][d["offsets"][h]:d["offsets"][h + 1]]
        fg = lambda t: (lambda q: (q.value, q.grad))(oracle.binned1d(K, D, pm, oracle.CHI2, y, 0.0, 1.0, t))
        fgh = lambda t: fg(t) + (oracle.binned1d_gnmat(K, D, pm, oracle.CHI2, y, 0.0, 1.0, t),)
        rl = lm_fit(fgh, d["start"][h], max_evals=5, tol=0.0)
        assert iters[h] == rl["iters"] and lam[h] == rl["lam"], (h, iters[h], rl["iters"], lam[h], rl["lam"])
        np.testing.assert_allclose(th[h], rl["theta"], rtol=1e-4, atol=1e-6 * np.abs(rl["theta"]).max())


def test_lm_graph_replay_equals_eager(dev):
    d, obj, K, D, pm = _case("chi2_K1_D2")
    b = HistBatch(d["y"], d["offsets"], d["lo"], d["hi"], K, D, obj, poly_mode=pm, precision=cg.PREC_DF64)
    start = torch.tensor(d["start"], device=dev)
    f1 = LMFitter(b)
    f1.init(start, tol=1e-10)
    e = f1.step(30, 1e-10).raw.clone()
    f2 = LMFitter(b)
    f2.capture(start, n_steps=30, tol=1e-10)
    f2.states.raw.zero_()
    r = f2.replay().raw
    torch.cuda.synchronize()
    assert torch.equal(e, r)


def test_lm_needs_a_df64_batch(dev):
    d, obj, K, D, pm = _case("chi2_K1_D2")
    b = HistBatch(d["y"], d["offsets"], d["lo"], d["hi"], K, D, obj, poly_mode=pm, precision=cg.PREC_FP64)
    with pytest.raises(cg.CgError):
        b.gauss_newton(torch.tensor(d["start"], device=dev))
    with pytest.raises(cg.CgError):
        LMFitter(b)


def test_lm_tiles_span_histograms_with_a_ragged_tail(dev):
    """Histograms of 3 full tiles + 17 bins, exactly one tile, one tile + 1
    bin and 300 bins: the state after init holds the tiled evaluation at the
    start point (value and gradient to 1e-10, GN within the FP32 bound), and
    the fits reach the oracle's minima."""
    ns = [3 * 16384 + 17, 16384, 16385, 300]
    ps = [synth.random_gauss_poly(1, 1, n, poly_mode=1, seed=40 + i) for i, n in enumerate(ns)]
    y = np.concatenate([p["y"] for p in ps])
    offs = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    start = np.stack([p["theta"] for p in ps])
    H = len(ns)
    b = HistBatch(y, offs, np.zeros(H), np.ones(H), 1, 1, cg.OBJ_POISSON, poly_mode=1, precision=cg.PREC_DF64)
    f = LMFitter(b)
    st = f.init(torch.tensor(start, device=dev), tol=1e-12)
    F0, g0 = st.f.cpu().numpy(), st.grad.cpu().numpy()
    G0 = st.d[:, _H:_H + 144].cpu().numpy().reshape(H, 12, 12)[:, :5, :5]
    for h in range(H):
        yy = y[offs[h]:offs[h + 1]]
        r = oracle.binned1d(1, 1, 1, oracle.POISSON, yy, 0.0, 1.0, start[h])
        assert abs(F0[h] - r.value) <= 1e-10 * abs(r.value)
        assert max_rel_err(g0[h], r.grad, r.scale) <= 1e-10
        ref = oracle.binned1d_gnmat(1, 1, 1, oracle.POISSON, yy, 0.0, 1.0, start[h])
        dd = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
        assert np.max(np.abs(G0[h] - ref) / dd) <= GN_TOL
    st = f.step(80, 1e-12)
    F, status = st.f.cpu().numpy(), st.status.cpu().numpy()
    assert np.all(status == CONVERGED), status
    for h in range(H):
        yy = y[offs[h]:offs[h + 1]]
        fg = lambda t: (lambda q: (q.value, q.grad))(oracle.binned1d(1, 1, 1, oracle.POISSON, yy, 0.0, 1.0, t))
        gn = lambda t: oracle.binned1d_gn(1, 1, 1, oracle.POISSON, yy, 0.0, 1.0, t)
        ref = bfgs_fit(fg, gn, start[h], max_iter=400, tol=1e-12)
        assert abs(F[h] - ref["F"]) <= 1e-6 * abs(ref["F"]), (h, F[h], ref["F"])


def test_lm_edge_cases_in_one_batch(dev):
    """An empty histogram (value 0, converged at the start), a 1-bin histogram
    (rank-one matrix: the fit may not converge, but F never increases), a
    start with a zero width (CG_FIT_DOMAIN, start kept) and an ordinary
    histogram (the oracle's minimum) in one batch."""
    p = synth.random_gauss_poly(1, 2, 700, poly_mode=1, seed=61)
    ys = [np.zeros(0), np.array([37.0]), p["y"].copy(), p["y"]]
    offs = np.concatenate([[0], np.cumsum([len(y) for y in ys])]).astype(np.int64)
    start = np.stack([p["theta"]] * 4)
    start[2, 2] = 0.0
    H = 4
    b = HistBatch(np.concatenate(ys), offs, np.zeros(H), np.ones(H), 1, 2, cg.OBJ_CHI2, poly_mode=1,
                  precision=cg.PREC_DF64)
    f = LMFitter(b)
    st = f.init(torch.tensor(start, device=dev), tol=1e-12)
    F0 = st.f.cpu().numpy().copy()
    assert st.status[2].item() == 4 and np.array_equal(st.theta[2].cpu().numpy(), start[2])
    st = f.step(60, 1e-12)
    F, status = st.f.cpu().numpy(), st.status.cpu().numpy()
    assert status[0] == CONVERGED and F[0] == 0.0
    assert F[1] <= F0[1] and status[1] in (0, 1, 3)
    assert status[2] == 4
    assert status[3] == CONVERGED
    fg = lambda t: (lambda q: (q.value, q.grad))(oracle.binned1d(1, 2, 1, oracle.CHI2, ys[3], 0.0, 1.0, t))
    gn = lambda t: oracle.binned1d_gn(1, 2, 1, oracle.CHI2, ys[3], 0.0, 1.0, t)
    ref = bfgs_fit(fg, gn, start[3], max_iter=400, tol=1e-12)
    assert abs(F[3] - ref["F"]) <= 1e-6 * abs(ref["F"])
