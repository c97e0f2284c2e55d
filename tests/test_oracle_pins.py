"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test checks the tape-AD oracle (oracle/cg_oracle.c) against one of:
closed-form derivatives derived by hand (written independently below),
central finite differences of its own value, invariants that hold exactly
(vanishing gradient at noise-free data, the normalisation of a pdf, the
linear-least-squares sub-problem), library routines (numpy.linalg.lstsq,
scipy.integrate.quad, Gauss-Legendre nodes) and brute-force expansion of
tiny cases.  The objective definitions follow the histogram-fitting use of
AD gradients in Sec. 4 (Fig. 3) of the paper and the Gaussian of Listing 1.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle.fit import CONVERGED, bfgs_fit, lm_fit
from paper_2203_06139_gb300 import synth
from tests._metrics import max_rel_err

OBJS = [oracle.CHI2, oracle.POISSON, oracle.POISSON_BC]


# --------------------------------------------------------------------------
# hand-derived closed forms (independent of the tape)
# --------------------------------------------------------------------------
def closed_form_binned1d(K, D, poly_mode, obj, y, lo, hi, theta):
    """Value and gradient of a 1-D binned objective from derivatives taken by
    hand: dG/dA = e, dG/dmu = A e (x-mu)/s^2, dG/ds = A e (x-mu)^2/s^3,
    df/dc_j = u^j; dT/df = -2 w (y-f) (chi2), 1 - y/f (Poisson),
    2 (1 - y/f) (Baker-Cousins)."""
    n = y.size
    x = lo + (np.arange(n) + 0.5) * ((hi - lo) / n)
    u = x if poly_mode == 0 else (2 * x - lo - hi) / (hi - lo)
    P = 3 * K + D + 1
    J = np.zeros((n, P))
    f = np.zeros(n)
    for k in range(K):
        A, mu, s = theta[3 * k:3 * k + 3]
        e = np.exp(-(x - mu) ** 2 / (2 * s * s))
        f += A * e
        J[:, 3 * k] = e
        J[:, 3 * k + 1] = A * e * (x - mu) / s ** 2
        J[:, 3 * k + 2] = A * e * (x - mu) ** 2 / s ** 3
    for j in range(D + 1):
        f += theta[3 * K + j] * u ** j
        J[:, 3 * K + j] = u ** j
    if obj == oracle.CHI2:
        w = 1.0 / np.maximum(y, 1.0)
        T = w * (y - f) ** 2
        dT = -2 * w * (y - f)
    elif obj == oracle.POISSON:
        T = f - np.where(y > 0, y * np.log(np.where(y > 0, f, 1.0)), 0.0)
        dT = 1 - y / f
    else:
        ylog = np.where(y > 0, y * np.log(np.where(y > 0, y / f, 1.0)), 0.0)
        T = 2 * (f - y + ylog)
        dT = 2 * (1 - y / f)
    return math.fsum(T), np.array([math.fsum(dT * J[:, k]) for k in range(P)])


@pytest.mark.parametrize("obj", OBJS)
@pytest.mark.parametrize("K,D,poly_mode", [(1, 1, 0), (2, 2, 1), (3, 1, 0), (1, -1, 0), (0, 3, 1)])
def test_binned1d_matches_hand_derivatives(obj, K, D, poly_mode):
    p = synth.random_gauss_poly(max(K, 1) if K else 1, D, 301, lo=-1.0, hi=2.0,
                                poly_mode=poly_mode, seed=7 * K + D + 3)
    if K == 0:
        theta = p["theta"][3:]
        y = np.maximum(p["y"], 0.0)
        mean = synth.expected_counts_1d(0, D, poly_mode, -1.0, 2.0, 301, theta)
        y = np.random.default_rng(1).poisson(np.maximum(mean, 1.0)).astype(float)
        theta = theta.copy()
        theta[0] = abs(theta[0]) + 50.0
    else:
        theta, y = p["theta"], p["y"]
    r = oracle.binned1d(K, D, poly_mode, obj, y, -1.0, 2.0, theta)
    assert r.rc == oracle.OK
    v, g = closed_form_binned1d(K, D, poly_mode, obj, y, -1.0, 2.0, theta)
    assert abs(r.value - v) <= 1e-13 * abs(v)
    assert max_rel_err(r.grad, g, r.scale, floor=1e-9) <= 1e-12


def test_brute_force_four_bins():
    """Four bins of one Gaussian on a constant, expanded term by term."""
    y = np.array([3.0, 0.0, 7.0, 2.0])
    th = np.array([5.0, 0.45, 0.2, 1.5])   # A, mu, s, c0
    xs = [0.125, 0.375, 0.625, 0.875]
    val = 0.0
    grad = np.zeros(4)
    for xi, yi in zip(xs, y):
        e = math.exp(-((xi - 0.45) ** 2) / (2 * 0.04))
        f = 5.0 * e + 1.5
        w = 1.0 / max(yi, 1.0)
        val += w * (yi - f) ** 2
        c = -2.0 * w * (yi - f)
        grad += c * np.array([e, 5.0 * e * (xi - 0.45) / 0.04, 5.0 * e * (xi - 0.45) ** 2 / 0.008, 1.0])
    r = oracle.binned1d(1, 0, 0, oracle.CHI2, y, 0.0, 1.0, th)
    assert abs(r.value - val) <= 1e-14 * val
    np.testing.assert_allclose(r.grad, grad, rtol=1e-13, atol=0)


def test_peak_height_convention():
    """Amplitude is the peak height ("gaus" of Fig. 3a): f(mu) = A + background."""
    th = np.array([123.0, 0.3, 0.05, 7.0, 2.0])
    f = oracle.gauss_poly_eval(1, 1, 0, 0.0, 1.0, np.array([0.3, 0.35]), th)
    assert abs(f[0] - (123.0 + 7.0 + 0.6)) < 1e-12
    assert abs(f[1] - (123.0 * math.exp(-0.5) + 7.0 + 0.7)) < 1e-12


@pytest.mark.parametrize("obj", OBJS)
def test_binned1d_central_fd(obj):
    p = synth.random_gauss_poly(2, 1, 500, seed=11)
    th = p["theta"]
    r = oracle.binned1d(2, 1, 0, obj, p["y"], 0.0, 1.0, th)
    fd = np.zeros_like(th)
    for k in range(th.size):
        h = 1e-6 * max(abs(th[k]), 1e-3)
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd[k] = (oracle.binned1d(2, 1, 0, obj, p["y"], 0.0, 1.0, tp).value
                 - oracle.binned1d(2, 1, 0, obj, p["y"], 0.0, 1.0, tm).value) / (2 * h)
    assert max_rel_err(r.grad, fd, r.scale) <= 1e-5


@pytest.mark.parametrize("obj", OBJS)
def test_noise_free_gradient_vanishes(obj):
    """Counts equal to the truth density (from the generator, not the oracle)
    make every residual zero, so the gradient vanishes at the truth."""
    h = synth.c1_histogram(n_bins=2000, noise=False)
    r = oracle.binned1d(1, 1, 0, obj, h["y"], 0.0, 10.0, h["truth"])
    assert r.rc == oracle.OK
    # at the truth every per-bin term is rounding noise; measure it against
    # the per-component scale 1% away from the truth
    ref = oracle.binned1d(1, 1, 0, obj, h["y"], 0.0, 10.0, h["truth"] * 1.01)
    assert np.all(np.abs(r.grad) <= 1e-12 * ref.scale)
    assert np.all(np.abs(ref.grad) > 1e-3 * ref.scale)
    if obj == oracle.CHI2 or obj == oracle.POISSON_BC:
        assert abs(r.value) <= 1e-9 * h["y"].sum()


def test_linear_least_squares_subproblem():
    """At fixed (mu, s), chi2 is linear least squares in (A, c0, c1); at the
    numpy.linalg.lstsq solution the oracle's gradient in those is zero."""
    h = synth.c1_histogram(n_bins=3000)
    x = synth.uniform_centres(3000, 0.0, 10.0)
    mu, s = 5.02, 0.49
    e = np.exp(-(x - mu) ** 2 / (2 * s * s))
    sw = np.sqrt(1.0 / np.maximum(h["y"], 1.0))
    X = np.stack([e, np.ones_like(x), x], 1) * sw[:, None]
    coef = np.linalg.lstsq(X, h["y"] * sw, rcond=None)[0]
    th = np.array([coef[0], mu, s, coef[1], coef[2]])
    r = oracle.binned1d(1, 1, 0, oracle.CHI2, h["y"], 0.0, 10.0, th)
    for k in (0, 3, 4):
        assert abs(r.grad[k]) <= 1e-9 * r.scale[k]
    assert abs(r.grad[1]) > 1e-6 * r.scale[1]


def test_gauss_newton_diagonal():
    p = synth.random_gauss_poly(2, 2, 400, poly_mode=1, seed=3)
    th = p["theta"]
    for obj in OBJS:
        gn = oracle.binned1d_gn(2, 2, 1, obj, p["y"], 0.0, 1.0, th)
        x = synth.uniform_centres(400, 0.0, 1.0)
        t = 2 * x - 1
        J = []
        f = np.zeros(400)
        for k in range(2):
            A, mu, s = th[3 * k:3 * k + 3]
            e = np.exp(-(x - mu) ** 2 / (2 * s * s))
            f += A * e
            J += [e, A * e * (x - mu) / s ** 2, A * e * (x - mu) ** 2 / s ** 3]
        for j in range(3):
            f += th[6 + j] * t ** j
            J.append(t ** j)
        J = np.array(J)
        y = p["y"]
        hh = {oracle.CHI2: 2 / np.maximum(y, 1), oracle.POISSON: y / f ** 2,
              oracle.POISSON_BC: 2 * y / f ** 2}[obj]
        np.testing.assert_allclose(gn, (hh[None, :] * J ** 2).sum(1), rtol=1e-12)


def _hand_jacobian(K, D, poly_mode, lo, hi, n, theta):
    """f and df/dtheta [n, P] of the 1-D family from derivatives taken by hand."""
    x = lo + (np.arange(n) + 0.5) * ((hi - lo) / n)
    u = x if poly_mode == 0 else (2 * x - lo - hi) / (hi - lo)
    P = 3 * K + D + 1
    J = np.zeros((n, P))
    f = np.zeros(n)
    for k in range(K):
        A, mu, s = theta[3 * k:3 * k + 3]
        e = np.exp(-(x - mu) ** 2 / (2 * s * s))
        f += A * e
        J[:, 3 * k], J[:, 3 * k + 1], J[:, 3 * k + 2] = e, A * e * (x - mu) / s ** 2, A * e * (x - mu) ** 2 / s ** 3
    for j in range(D + 1):
        f += theta[3 * K + j] * u ** j
        J[:, 3 * K + j] = u ** j
    return f, J


@pytest.mark.parametrize("K,D,pm", [(1, 2, 1), (2, 1, 0), (3, 1, 0), (1, -1, 0)])
def test_gauss_newton_matrix_hand_jacobian(K, D, pm):
    """GN_ab = sum_i h_i J_ia J_ib with J from the hand derivatives and h the
    curvature of each bin term; symmetric, diagonal = the GN diagonal."""
    p = synth.random_gauss_poly(K, D, 500, poly_mode=pm, seed=4 + K)
    th, y = p["theta"], p["y"]
    f, J = _hand_jacobian(K, D, pm, 0.0, 1.0, 500, th)
    for obj in OBJS:
        G = oracle.binned1d_gnmat(K, D, pm, obj, y, 0.0, 1.0, th)
        fs = np.where(y > 0, f, 1.0)
        hh = {oracle.CHI2: 2 / np.maximum(y, 1), oracle.POISSON: np.where(y > 0, y / fs ** 2, 0.0),
              oracle.POISSON_BC: np.where(y > 0, 2 * y / fs ** 2, 0.0)}[obj]
        ref = (J * hh[:, None]).T @ J
        d = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
        assert np.max(np.abs(G - ref) / d) <= 1e-12
        assert np.array_equal(G, G.T)
        np.testing.assert_allclose(np.diag(G), oracle.binned1d_gn(K, D, pm, obj, y, 0.0, 1.0, th), rtol=1e-13)


@pytest.mark.parametrize("obj", OBJS)
def test_gauss_newton_matrix_is_the_hessian_at_zero_residual(obj):
    """Where y = f(theta) exactly (noise-free, non-integer counts) the dropped
    term (dT/df) d2f/dtheta2 vanishes for all three objectives, so GN equals
    the Hessian: central differences of the oracle's exact gradient."""
    K, D, pm = 2, 1, 1
    p = synth.random_gauss_poly(K, D, 800, poly_mode=pm, seed=9, noise=False)
    th, y = p["truth"], p["y"]
    G = oracle.binned1d_gnmat(K, D, pm, obj, y, 0.0, 1.0, th)
    P = th.size
    Hs = np.zeros((P, P))
    for b in range(P):
        h = 1e-5 * max(abs(th[b]), 1e-2)
        tp, tm = th.copy(), th.copy()
        tp[b] += h
        tm[b] -= h
        Hs[:, b] = (oracle.binned1d(K, D, pm, obj, y, 0.0, 1.0, tp).grad
                    - oracle.binned1d(K, D, pm, obj, y, 0.0, 1.0, tm).grad) / (2 * h)
    d = np.sqrt(np.outer(np.diag(G), np.diag(G)))
    assert np.max(np.abs(G - Hs) / d) <= 1e-6


def test_empty_bins_where_the_model_underflows():
    """One narrow peak without background: far from it the model underflows
    to exactly 0 in FP64 and the bins are empty.  An empty bin's Poisson term
    is T = f (2 f for Baker-Cousins), so it adds dT/df = 1 (2) times the
    Jacobian to the gradient and nothing to the Gauss-Newton diagonal; the
    oracle matches that closed form rather than producing 0/0."""
    n = 2000
    th = np.array([800.0, 0.5, 0.01])
    x = synth.uniform_centres(n, 0.0, 1.0)
    y = np.random.default_rng(2).poisson(th[0] * np.exp(-(x - th[1]) ** 2 / (2 * th[2] ** 2))).astype(float)
    A, mu, s = t = th * np.array([1.02, 1.0, 0.97])
    e = np.exp(-(x - mu) ** 2 / (2 * s * s))
    f = A * e
    assert np.any(f == 0.0) and np.all(y[f == 0.0] == 0.0)
    J = np.array([e, A * e * (x - mu) / s ** 2, A * e * (x - mu) ** 2 / s ** 3])
    fs = np.where(f > 0.0, f, 1.0)
    for obj, c in ((oracle.POISSON, 1.0), (oracle.POISSON_BC, 2.0)):
        with np.errstate(divide="ignore", invalid="ignore"):   # discarded branch: fs**2 may underflow
            gi = np.where(y > 0.0, c * (1.0 - y / fs), c)
            hh = np.where(y > 0.0, c * y / fs ** 2, 0.0)
        r = oracle.binned1d(1, -1, 0, obj, y, 0.0, 1.0, t)
        gref = (gi[None, :] * J).sum(1)
        assert np.all(np.isfinite(r.grad))
        np.testing.assert_allclose(r.grad, gref, rtol=1e-9, atol=1e-12 * np.abs(J).sum())
        gn = oracle.binned1d_gn(1, -1, 0, obj, y, 0.0, 1.0, t)
        np.testing.assert_allclose(gn, (hh[None, :] * J ** 2).sum(1), rtol=1e-12)


# --------------------------------------------------------------------------
# unbinned mixture
# --------------------------------------------------------------------------
def test_unbinned_pdf_normalised():
    """exp(-NLL) of one event is p(x); its integral over [lo, hi] is 1 for any
    parameters (scipy quad), and separately for each component."""
    for th in ([0.3, 2.0, 0.3, 0.5], [0.7, 9.5, 1.7, 2.2], [1.0, 4.0, 0.8, 0.1], [0.0, 4.0, 0.8, 0.9]):
        def p(x):
            return math.exp(-oracle.unbinned_mix(np.array([x]), 0.0, 10.0, np.array(th)).value)
        val, _ = integrate.quad(p, 0.0, 10.0, points=[th[1]], limit=200, epsabs=1e-13, epsrel=1e-12)
        assert abs(val - 1.0) < 1e-9


def test_unbinned_hand_derivatives():
    x = synth.c2_events(2000)
    th = np.array([0.35, 2.1, 0.27, 0.55])
    f, mu, s, lam = th
    lo, hi = 0.0, 10.0
    Phi = lambda z: 0.5 * math.erfc(-z / math.sqrt(2))
    phi = lambda z: math.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)
    a, b = (lo - mu) / s, (hi - mu) / s
    ZG = Phi(b) - Phi(a)
    ZE = math.exp(-lam * lo) - math.exp(-lam * hi)
    g = np.exp(-0.5 * ((x - mu) / s) ** 2) / (s * math.sqrt(2 * math.pi)) / ZG
    e = lam * np.exp(-lam * x) / ZE
    p = f * g + (1 - f) * e
    # dZG/dmu = (phi(a) - phi(b))/s ; dZG/ds = (a phi(a) - b phi(b))/s
    dZG_mu = (phi(a) - phi(b)) / s
    dZG_s = (a * phi(a) - b * phi(b)) / s
    dg_mu = g * ((x - mu) / s ** 2 - dZG_mu / ZG)
    dg_s = g * ((x - mu) ** 2 / s ** 3 - 1 / s - dZG_s / ZG)
    dZE_lam = -lo * math.exp(-lam * lo) + hi * math.exp(-lam * hi)
    de_lam = e * (1 / lam - x - dZE_lam / ZE)
    grad = -np.array([math.fsum((g - e) / p), math.fsum(f * dg_mu / p), math.fsum(f * dg_s / p),
                      math.fsum((1 - f) * de_lam / p)])
    r = oracle.unbinned_mix(x, lo, hi, th)
    assert abs(r.value + math.fsum(np.log(p))) <= 1e-13 * abs(r.value)
    assert max_rel_err(r.grad, grad, r.scale, floor=1e-9) <= 1e-11


def test_unbinned_asimov_gradient_vanishes():
    """Weighted events at Gauss-Legendre nodes with weights w_j p(x_j; theta*)
    integrate the NLL against the true pdf; its gradient at theta* is
    -grad of the integral of p, which is zero because p stays normalised."""
    th = np.array([0.3, 2.0, 0.3, 0.5])
    nodes, wts = np.polynomial.legendre.leggauss(64)
    xs, ws = [], []
    edges = np.concatenate([np.linspace(0.0, 4.0, 81), np.linspace(4.0, 10.0, 13)[1:]])
    for a, b in zip(edges[:-1], edges[1:]):
        xs.append(0.5 * (b - a) * nodes + 0.5 * (a + b))
        ws.append(0.5 * (b - a) * wts)
    xs = np.concatenate(xs)
    ws = np.concatenate(ws)
    px = np.array([math.exp(-oracle.unbinned_mix(np.array([xx]), 0.0, 10.0, th).value) for xx in xs])
    assert abs(np.dot(ws, px) - 1.0) < 1e-12
    r = oracle.unbinned_mix(xs, 0.0, 10.0, th, weights=ws * px)
    assert np.all(np.abs(r.grad) <= 1e-11 * r.scale), (r.grad, r.scale)
    # and it does not vanish away from the truth
    r2 = oracle.unbinned_mix(xs, 0.0, 10.0, th * 1.05, weights=ws * px)
    assert np.all(np.abs(r2.grad) > 1e-5 * r2.scale)


def test_unbinned_gradient_at_truth_shrinks_like_one_over_sqrt_n():
    """Events drawn from the model at its truth: the score has mean zero, so
    the summed gradient grows like sqrt(N) while the sum of per-event |terms|
    S_k grows like N.  |g_k| <= 5 S_k / sqrt(N) at N = 1e4, 1e5, 1e6 (a
    normalisation or sampling mistake leaves |g_k| of order S_k)."""
    truth = synth.C2_TRUTH
    for n in (10 ** 4, 10 ** 5, 10 ** 6):
        x = synth.c2_events(n)
        r = oracle.unbinned_mix(x, 0.0, 10.0, truth)
        assert np.all(np.abs(r.grad) <= 5.0 * r.scale / math.sqrt(n)), (n, r.grad, r.scale)


def test_unbinned_central_fd():
    x = synth.c2_events(5000)
    th = np.array([0.28, 1.9, 0.33, 0.47])
    r = oracle.unbinned_mix(x, 0.0, 10.0, th)
    for k in range(4):
        h = 1e-6 * abs(th[k])
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (oracle.unbinned_mix(x, 0.0, 10.0, tp).value - oracle.unbinned_mix(x, 0.0, 10.0, tm).value) / (2 * h)
        assert abs(fd - r.grad[k]) <= 1e-5 * max(abs(r.grad[k]), 1e-6 * r.scale[k])


# --------------------------------------------------------------------------
# 2-D rotated Gaussians
# --------------------------------------------------------------------------
def closed_form_2d(K, counts, theta):
    ny, nx = counts.shape
    X = synth.uniform_centres(nx, 0.0, 1.0)[None, :]
    Y = synth.uniform_centres(ny, 0.0, 1.0)[:, None]
    mu = np.full(counts.shape, theta[6 * K])
    parts = []
    for k in range(K):
        A, mx, my, sx, sy, ph = theta[6 * k:6 * k + 6]
        c, s = math.cos(ph), math.sin(ph)
        dx, dy = X - mx, Y - my
        u = c * dx + s * dy
        v = -s * dx + c * dy
        e = np.exp(-0.5 * (u * u / sx ** 2 + v * v / sy ** 2))
        mu = mu + A * e
        # d/d(mu_x): A e (u c/sx^2 - v s/sy^2); d/d(mu_y): A e (u s/sx^2 + v c/sy^2)
        # d/d(sx): A e u^2/sx^3; d/d(sy): A e v^2/sy^3; d/d(phi): -A e u v (1/sx^2 - 1/sy^2)
        parts += [e, A * e * (u * c / sx ** 2 - v * s / sy ** 2), A * e * (u * s / sx ** 2 + v * c / sy ** 2),
                  A * e * u * u / sx ** 3, A * e * v * v / sy ** 3, -A * e * u * v * (1 / sx ** 2 - 1 / sy ** 2)]
    parts.append(np.ones(counts.shape))
    dT = 1 - counts / mu
    T = mu - np.where(counts > 0, counts * np.log(mu), 0.0)
    return math.fsum(T.ravel()), np.array([math.fsum((dT * p).ravel()) for p in parts])


def test_binned2d_hand_derivatives():
    K = 3
    truth = synth.c3_truth(K)
    th = truth * (1 + np.random.default_rng(5).uniform(-0.05, 0.05, truth.size))
    counts = np.random.default_rng(6).poisson(synth.expected_counts_2d(truth, K, 37, 29)).astype(float)
    r = oracle.binned2d(K, counts, 0.0, 1.0, 0.0, 1.0, th)
    v, g = closed_form_2d(K, counts, th)
    assert abs(r.value - v) <= 1e-13 * abs(v)
    assert max_rel_err(r.grad, g, r.scale, floor=1e-9) <= 1e-11


def test_binned2d_noise_free_vanishes_and_fd():
    K = 2
    truth = synth.c3_truth(K)
    mean = synth.expected_counts_2d(truth, K, 40, 33)
    r0 = oracle.binned2d(K, mean, 0.0, 1.0, 0.0, 1.0, truth)
    th = truth * 1.02
    r = oracle.binned2d(K, mean, 0.0, 1.0, 0.0, 1.0, th)
    assert np.all(np.abs(r0.grad) <= 1e-12 * r.scale)
    for k in range(th.size):
        h = 1e-6 * max(abs(th[k]), 1e-3)
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (oracle.binned2d(K, mean, 0.0, 1.0, 0.0, 1.0, tp).value
              - oracle.binned2d(K, mean, 0.0, 1.0, 0.0, 1.0, tm).value) / (2 * h)
        assert abs(fd - r.grad[k]) <= 1e-5 * max(abs(r.grad[k]), 1e-6 * r.scale[k])


# --------------------------------------------------------------------------
# Listing 1
# --------------------------------------------------------------------------
def test_listing1_gauss():
    for x, p, s in [(0.3, 0.1, 2.0), (-1.0, 0.5, 0.7), (4.0, 4.0, 1.3)]:
        v, dx, dp = oracle.listing1_gauss(x, p, s)
        ref = (2 * math.pi) ** -0.5 * s ** -0.5 * math.exp(-(x - p) ** 2 / (2 * s * s))
        assert abs(v - ref) <= 1e-15 * ref
        assert abs(dx - (-(x - p) / s ** 2 * ref)) <= 1e-14 * max(abs(ref), 1e-300)
        assert abs(dp - ((x - p) / s ** 2 * ref)) <= 1e-14 * max(abs(ref), 1e-300)


# --------------------------------------------------------------------------
# oracle fit
# --------------------------------------------------------------------------
def test_oracle_fit_reaches_lstsq_consistent_minimum():
    """The BFGS fit of one histogram ends at a point where the linear
    parameters are the weighted least-squares solution for its (mu, s), and
    chi2/ndf is statistically sane."""
    n = 2000
    h = synth.c1_histogram(n_bins=n)
    y = h["y"]
    fg = lambda t: (lambda r: (r.value, r.grad))(oracle.binned1d(1, 1, 0, oracle.CHI2, y, 0.0, 10.0, t))
    gn = lambda t: oracle.binned1d_gn(1, 1, 0, oracle.CHI2, y, 0.0, 10.0, t)
    res = bfgs_fit(fg, gn, h["truth"] * np.array([1.15, 0.97, 1.2, 0.85, 1.1]), max_iter=200, tol=1e-12)
    assert res["status"] == CONVERGED
    th = res["theta"]
    x = synth.uniform_centres(n, 0.0, 10.0)
    e = np.exp(-(x - th[1]) ** 2 / (2 * th[2] ** 2))
    sw = np.sqrt(1 / np.maximum(y, 1))
    coef = np.linalg.lstsq(np.stack([e, np.ones(n), x], 1) * sw[:, None], y * sw, rcond=None)[0]
    np.testing.assert_allclose([th[0], th[3], th[4]], coef, rtol=1e-6)
    ndf = n - 5
    assert abs(res["F"] / ndf - 1) < 5 * math.sqrt(2 / ndf)
    assert abs(th[1] - 5.0) < 0.01


def test_oracle_lm_solves_linear_least_squares():
    """With no peak (K = 0) chi2 is linear least squares and GN its exact
    Hessian: LM ends at numpy.linalg.lstsq's solution."""
    n, D = 3000, 3
    r = np.random.default_rng(2)
    x = synth.uniform_centres(n, 0.0, 1.0)
    u = 2 * x - 1
    y = r.poisson(50 + 20 * u - 10 * u ** 2 + 5 * u ** 3).astype(float)
    fgh = lambda t: (lambda q: (q.value, q.grad, oracle.binned1d_gnmat(0, D, 1, oracle.CHI2, y, 0.0, 1.0, t)))(
        oracle.binned1d(0, D, 1, oracle.CHI2, y, 0.0, 1.0, t))
    res = lm_fit(fgh, np.array([1.0, 0.0, 0.0, 0.0]), tol=1e-14)
    assert res["status"] == CONVERGED
    sw = np.sqrt(1 / np.maximum(y, 1))
    X = np.stack([u ** j for j in range(D + 1)], 1)
    coef = np.linalg.lstsq(X * sw[:, None], y * sw, rcond=None)[0]
    chi2_min = np.sum(sw ** 2 * (y - X @ coef) ** 2)
    # the stop rule bounds EDM (tol |F|), i.e. F - F_min, not the parameters directly
    assert abs(res["F"] - chi2_min) <= 1e-12 * chi2_min
    np.testing.assert_allclose(res["theta"], coef, rtol=1e-6, atol=1e-6 * np.abs(coef).max())


@pytest.mark.parametrize("obj", OBJS)
def test_oracle_lm_reaches_the_bfgs_minimum(obj):
    """The second-order fit and the gradient-only fit end at the same minimum
    (objective to 1e-9 relative), LM in fewer evaluations."""
    p = synth.random_gauss_poly(1, 2, 2000, poly_mode=1, seed=12)
    y = p["y"]
    th0 = p["truth"] * np.array([1.1, 0.98, 1.15, 0.9, 1.1, 0.9])
    fg = lambda t: (lambda q: (q.value, q.grad))(oracle.binned1d(1, 2, 1, obj, y, 0.0, 1.0, t))
    gn = lambda t: oracle.binned1d_gn(1, 2, 1, obj, y, 0.0, 1.0, t)
    fgh = lambda t: fg(t) + (oracle.binned1d_gnmat(1, 2, 1, obj, y, 0.0, 1.0, t),)
    ref = bfgs_fit(fg, gn, th0, max_iter=400, tol=1e-14)
    lm = lm_fit(fgh, th0, max_evals=200, tol=1e-14)
    assert ref["status"] == CONVERGED and lm["status"] == CONVERGED
    assert abs(lm["F"] - ref["F"]) <= 1e-9 * abs(ref["F"])
    np.testing.assert_allclose(lm["theta"], ref["theta"], rtol=1e-5, atol=1e-6 * np.abs(ref["theta"]).max())
    assert lm["evals"] < ref["evals"]


def check_lm_steps_on_a_separable_quadratic(lm_fit):
    """F = sum_i a_i (theta_i - t_i)^2 has GN = diag(2a) = its Hessian, so
    the damped step is -(theta - t) / (1 + lambda): after accepted steps with
    lambda_j = 1e-3 / 10^j, theta_k - t = (theta_0 - t) prod_j lambda_j /
    (1 + lambda_j).  Three steps from the start, checked to rounding."""
    a = np.array([3.0, 0.5, 20.0])
    t = np.array([1.0, -2.0, 0.25])
    th0 = np.array([4.0, 1.0, -1.0])
    fgh = lambda th: (float(np.sum(a * (th - t) ** 2)), 2 * a * (th - t), np.diag(2 * a))
    one = lm_fit(fgh, th0, max_evals=2, tol=0.0)
    np.testing.assert_allclose(one["theta"] - t, (th0 - t) * (1e-3 / (1 + 1e-3)), rtol=1e-10)
    res = lm_fit(fgh, th0, max_evals=4, tol=0.0)
    factor = np.prod([l / (1 + l) for l in (1e-3, 1e-4, 1e-5)])
    # theta - t is ~1e-12 here: compare theta itself, to a few units of its rounding
    np.testing.assert_allclose(res["theta"], t + (th0 - t) * factor, rtol=0, atol=4e-16 * np.abs(t).max() * 4)
    assert res["iters"] == 3 and res["evals"] == 4
    assert res["lam"] == max(1e-3 * 0.1 * 0.1 * 0.1, 1e-12)
    assert abs(res["edm"] - float(np.sum(a * (res["theta"] - t) ** 2))) <= 1e-12 * res["edm"]


def test_oracle_lm_steps_on_a_separable_quadratic():
    check_lm_steps_on_a_separable_quadratic(lm_fit)


def check_bfgs_first_step_is_newton(bfgs_fit):
    """With H_0 = diag(1 / GN) and GN the exact (diagonal) Hessian, the first
    direction is the Newton step, accepted at alpha = 1 (Armijo holds with
    F = 0): one iteration, two evaluations, theta = t to rounding."""
    a = np.array([3.0, 0.5, 20.0, 7.0])
    t = np.array([1.0, -2.0, 0.25, 3.0])
    fg = lambda th: (float(np.sum(a * (th - t) ** 2)), 2 * a * (th - t))
    res = bfgs_fit(fg, lambda th: 2 * a, np.array([4.0, 1.0, -1.0, 0.0]), tol=1e-12)
    assert res["status"] == CONVERGED and res["iters"] == 1 and res["evals"] == 2
    np.testing.assert_allclose(res["theta"], t, rtol=0, atol=1e-15 * 4)


def test_oracle_bfgs_first_step_is_newton_on_a_separable_quadratic():
    check_bfgs_first_step_is_newton(bfgs_fit)


def check_bfgs_secant(bfgs_fit):
    """After one iteration on F = (theta - t)^T A (theta - t) with a full SPD
    A, the updated inverse Hessian maps the gradient change to the step
    (H y = s) and stays symmetric."""
    r = np.random.default_rng(8)
    Q = r.normal(size=(5, 5))
    A = Q @ Q.T + 5 * np.eye(5)
    t = r.normal(size=5)
    fg = lambda th: (float((th - t) @ A @ (th - t)), 2 * A @ (th - t))
    th0 = t + r.normal(size=5)
    res = bfgs_fit(fg, lambda th: 2 * np.diag(A), th0, max_iter=1, tol=0.0)
    s = res["theta"] - th0
    y = res["g"] - fg(th0)[1]
    np.testing.assert_allclose(res["H"] @ y, s, rtol=1e-10, atol=1e-12 * np.abs(s).max())
    np.testing.assert_allclose(res["H"], res["H"].T, rtol=1e-12, atol=1e-15)


def test_oracle_bfgs_update_satisfies_the_secant_condition():
    check_bfgs_secant(bfgs_fit)


def test_fig3a_fit_recovers_the_generating_gaussian():
    """Fig. 3a's histogram (1000 bins on [-5, 5], 10^5 draws of a Gaussian of
    mean 1 and width 3 within the range): the oracle's fits return the
    generating shape.  Peak height per bin = 10^5 x 0.01 x phi(0) / 3 / P(range)
    = 150.1; mu and s within 5 standard errors (s / sqrt(N) and s / sqrt(2N));
    the Baker-Cousins (maximum-likelihood) height within 2 %, the chi2 one
    within 4 % (the 1/max(y, 1) weights pull it low); chi2 / ndf sane."""
    from scipy.special import ndtr
    h = synth.fig3a_histogram()
    y = h["y"]
    mass = ndtr(4.0 / 3.0) - ndtr(-2.0)
    A_true = 1e5 * 0.01 / (3.0 * math.sqrt(2 * math.pi)) / mass
    n_eff = y.sum()
    for obj, tolA in ((oracle.CHI2, 0.04), (oracle.POISSON_BC, 0.02)):
        fg = lambda t: (lambda q: (q.value, q.grad))(oracle.binned1d(1, -1, 0, obj, y, -5.0, 5.0, t))
        gn = lambda t: oracle.binned1d_gn(1, -1, 0, obj, y, -5.0, 5.0, t)
        res = bfgs_fit(fg, gn, np.array([120.0, 0.5, 2.5]), max_iter=200, tol=1e-12)
        assert res["status"] == CONVERGED
        A, mu, sg = res["theta"]
        assert abs(mu - 1.0) <= 5 * 3.0 / math.sqrt(n_eff)
        assert abs(abs(sg) - 3.0) <= 5 * 3.0 / math.sqrt(2 * n_eff)
        assert abs(A - A_true) <= tolA * A_true, (obj, A, A_true)
        if obj == oracle.CHI2:
            ndf = y.size - 3
            assert abs(res["F"] / ndf - 1) < 5 * math.sqrt(2 / ndf)


def test_compensated_sum_of_identical_terms():
    """10^6 identical events: the NLL is N times one event's term to a few
    ulps (a plain running sum drifts by ~N eps / 2 relative)."""
    N = 10 ** 6
    th = np.array([0.3, 2.0, 0.3, 0.5])
    one = oracle.unbinned_mix(np.array([2.345]), 0.0, 10.0, th)
    r = oracle.unbinned_mix(np.full(N, 2.345), 0.0, 10.0, th)
    eps = np.finfo(float).eps
    assert abs(r.value - N * one.value) <= 4 * eps * abs(N * one.value)
    np.testing.assert_allclose(r.grad, N * one.grad, rtol=4 * eps)


# --------------------------------------------------------------------------
# Hand-written closed-form gradients (cg_closed.c) against the tape
# --------------------------------------------------------------------------
def _rel(g, ref, scale, floor):
    return float(np.max(np.abs(g - ref) / np.maximum(np.abs(ref), floor * scale)))


def test_closed_form_mixture_matches_the_tape():
    """Two independent statements of the unbinned-NLL gradient (the tape's
    recorded partials, the derivatives written out by hand) agree to 1e-13 at
    parameter points away from the minimum, and the central-difference
    gradient to the accuracy finite differences allow."""
    x = synth.c2_events(100000)
    for th in synth.c2_theta_points(4):
        r = oracle.unbinned_mix(x, 0.0, 10.0, th)
        v, g = oracle.closed_mix(x, 0.0, 10.0, th, threads=4)
        assert abs(v - r.value) <= 1e-13 * abs(r.value)
        assert _rel(g, r.grad, r.scale, 1e-3) <= 1e-13
        fd = oracle.closed_mix_fd(x, 0.0, 10.0, th, threads=4)
        assert _rel(fd, r.grad, r.scale, 1e-6) <= 1e-5


@pytest.mark.parametrize("K,D,pm", [(1, 1, 0), (2, 2, 1), (3, 0, 1)])
def test_closed_form_chi2_matches_the_tape(K, D, pm):
    p = synth.random_gauss_poly(K, D, 3001, lo=0.0, hi=10.0, poly_mode=pm, seed=20 + K)
    for th in (p["theta"], p["truth"] * 1.03):
        r = oracle.binned1d(K, D, pm, oracle.CHI2, p["y"], 0.0, 10.0, th)
        v, g = oracle.closed_gauss_poly_chi2(K, D, pm, p["y"], 0.0, 10.0, th, threads=3)
        assert abs(v - r.value) <= 1e-13 * abs(r.value)
        assert _rel(g, r.grad, r.scale, 1e-3) <= 1e-13


def test_closed_form_sums_are_deterministic_per_thread_count():
    x = synth.c2_events(50000)
    th = synth.c2_theta_points(1)[0]
    a = oracle.closed_mix(x, 0.0, 10.0, th, threads=5)
    b = oracle.closed_mix(x, 0.0, 10.0, th, threads=5)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])
