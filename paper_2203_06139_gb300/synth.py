"""Seeded synthetic inputs for the fit workloads.

This module draws data only: histograms (Poisson counts around a stated truth
density), unbinned event samples, truth vectors and parameter points.  It
computes no objective and no gradient, and is the one module that both the
CUDA path's callers (tests, bench) and the CPU oracle's callers use for
inputs.  numpy's PCG64 generator with seed 2203061390 + workload index is
used throughout; parameter points use that seed + 1000.

Workloads (sizes are the defaults; every generator takes smaller sizes too):
  0  single 1-D histogram, 10,000 bins on [0, 10], Gaussian (A=1000, mu=5,
     s=0.5) + linear background (50 - 2x), chi-square; 100 parameter points
     at U(0.8, 1.2) x truth.
  1  10^7 unbinned events from 0.3 N(2, 0.3) + 0.7 Exp(rate 0.5), each
     component truncated to [0, 10] and sampled by its exact inverse CDF;
     50 parameter points at U(0.8, 1.2) x truth, fraction kept in [0.05, 0.95].
  2  4096 x 4096 histogram on [0, 1]^2 of 8 rotated 2-D Gaussians (A in
     U(50, 500), means in U(0.1, 0.9), widths in U(0.01, 0.05), angle in
     U(0, pi)) + constant 5, Poisson counts.
  3  4096 1-D histograms on [0, 1], bin counts round(exp(U(ln 64, ln 65536))),
     Gaussian (A in U(100, 5000), mu in U(0.2, 0.8), s in U(0.01, 0.1)) +
     quadratic background b0 + b1 t + b2 t^2, t = 2x - 1, b0 in U(1, 100),
     b1, b2 in U(-0.3, 0.3) b0; starts at U(0.8, 1.2) x truth.
  4  2048-bin histograms on [0, 1] of 3 Gaussians (A in U(100, 5000), mu in
     U(0.05, 0.95), s in U(0.005, 0.05), sorted by mu) + linear background
     whose end values lie in U(10, 200).
  fig3a: 1000 bins on [-5, 5] filled with 100,000 draws of the "gaus" shape
     with (A, mu, s) = (100, 1, 3) restricted to the histogram range (Fig. 3a).
"""
import math

import numpy as np
from scipy.special import ndtr, ndtri

SEED_BASE = 2203061390
THETA_SEED_OFFSET = 1000


def rng(index, offset=0):
    return np.random.Generator(np.random.PCG64(SEED_BASE + index + offset))


def uniform_centres(n, lo, hi):
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * ((hi - lo) / n)


def _peaks_plus_poly(x, theta, K, D, poly_mode, lo, hi):
    """Expected counts of the data-generating density: K Gaussian peaks
    (amplitude = peak height) plus a polynomial of degree D in x or in
    t = (2x - lo - hi)/(hi - lo)."""
    out = np.zeros_like(x)
    for k in range(K):
        A, mu, s = theta[3 * k:3 * k + 3]
        out += A * np.exp(-0.5 * ((x - mu) / s) ** 2)
    u = x if poly_mode == 0 else (2.0 * x - lo - hi) / (hi - lo)
    for j in range(D + 1):
        out += theta[3 * K + j] * u ** j
    return out


def expected_counts_1d(K, D, poly_mode, lo, hi, n, theta):
    """Noise-free expected counts at the uniform bin centres (truth density)."""
    return _peaks_plus_poly(uniform_centres(n, lo, hi), np.asarray(theta, np.float64),
                            K, D, poly_mode, lo, hi)


# ----------------------------------------------------------------------------
# workload 0: one histogram, 100 parameter points
# ----------------------------------------------------------------------------
C1_TRUTH = np.array([1000.0, 5.0, 0.5, 50.0, -2.0])


def c1_histogram(n_bins=10000, lo=0.0, hi=10.0, noise=True):
    mean = expected_counts_1d(1, 1, 0, lo, hi, n_bins, C1_TRUTH)
    y = rng(0).poisson(mean).astype(np.float64) if noise else mean
    return dict(K=1, D=1, poly_mode=0, lo=lo, hi=hi, n=n_bins, y=y, truth=C1_TRUTH.copy())


def c1_theta_points(n_points=100):
    r = rng(0, THETA_SEED_OFFSET)
    return C1_TRUTH[None, :] * r.uniform(0.8, 1.2, size=(n_points, C1_TRUTH.size))


# ----------------------------------------------------------------------------
# workload 1: unbinned mixture events, 50 parameter points
# ----------------------------------------------------------------------------
C2_TRUTH = np.array([0.3, 2.0, 0.3, 0.5])   # (fraction, mu, s, lambda)
C2_RANGE = (0.0, 10.0)


def c2_events(n_events=10 ** 7, truth=C2_TRUTH, lo=0.0, hi=10.0, index=1):
    frac, mu, s, lam = truth
    r = rng(index)
    is_gauss = r.random(n_events) < frac
    u = r.random(n_events)
    # truncated normal by its inverse CDF
    a, b = ndtr((lo - mu) / s), ndtr((hi - mu) / s)
    xg = mu + s * ndtri(a + u * (b - a))
    # truncated exponential by its inverse CDF
    xe = lo - np.log1p(-u * (-math.expm1(-lam * (hi - lo)))) / lam
    x = np.where(is_gauss, xg, xe)
    return np.clip(x, lo, hi)


def c2_theta_points(n_points=50):
    r = rng(1, THETA_SEED_OFFSET)
    th = C2_TRUTH[None, :] * r.uniform(0.8, 1.2, size=(n_points, 4))
    th[:, 0] = np.clip(th[:, 0], 0.05, 0.95)
    return th


# ----------------------------------------------------------------------------
# workload 2: 2-D histogram of rotated Gaussians + constant
# ----------------------------------------------------------------------------
def c3_truth(K=8, index=2):
    r = rng(index)
    th = np.zeros(6 * K + 1)
    for k in range(K):
        th[6 * k + 0] = r.uniform(50.0, 500.0)
        th[6 * k + 1] = r.uniform(0.1, 0.9)
        th[6 * k + 2] = r.uniform(0.1, 0.9)
        th[6 * k + 3] = r.uniform(0.01, 0.05)
        th[6 * k + 4] = r.uniform(0.01, 0.05)
        th[6 * k + 5] = r.uniform(0.0, math.pi)
    th[6 * K] = 5.0
    return th


def expected_counts_2d(theta, K, nx, ny, lx=0.0, hx=1.0, ly=0.0, hy=1.0, rows=None):
    """Noise-free means at the bin centres, shape (ny, nx), row-major (x fastest)."""
    xc = uniform_centres(nx, lx, hx)
    yc = uniform_centres(ny, ly, hy)
    rows = range(ny) if rows is None else rows
    out = np.empty((ny, nx))
    step = max(1, (1 << 22) // max(nx, 1))
    for j0 in range(0, ny, step):
        j1 = min(ny, j0 + step)
        X = xc[None, :]
        Y = yc[j0:j1, None]
        mu = np.full((j1 - j0, nx), theta[6 * K])
        for k in range(K):
            A, mx, my, sx, sy, phi = theta[6 * k:6 * k + 6]
            c, s = math.cos(phi), math.sin(phi)
            u = c * (X - mx) + s * (Y - my)
            v = -s * (X - mx) + c * (Y - my)
            mu += A * np.exp(-0.5 * ((u / sx) ** 2 + (v / sy) ** 2))
        out[j0:j1] = mu
    return out


def c3_histogram(nx=4096, ny=4096, K=8, noise=True):
    truth = c3_truth(K)
    mean = expected_counts_2d(truth, K, nx, ny)
    counts = rng(2, 7).poisson(mean).astype(np.float64) if noise else mean
    return dict(K=K, nx=nx, ny=ny, lx=0.0, hx=1.0, ly=0.0, hy=1.0, counts=counts, truth=truth)


def c3_theta_point(truth, n_points=1):
    r = rng(2, THETA_SEED_OFFSET)
    return truth[None, :] * (1.0 + r.uniform(-0.05, 0.05, size=(n_points, truth.size)))


# ----------------------------------------------------------------------------
# workload 3: many uneven 1-D histograms (Gaussian + quadratic in t)
# ----------------------------------------------------------------------------
def c4_batch(H=4096, min_bins=64, max_bins=65536, index=3):
    r = rng(index)
    n = np.rint(np.exp(r.uniform(math.log(min_bins), math.log(max_bins), size=H))).astype(np.int64)
    truth = np.zeros((H, 6))
    truth[:, 0] = r.uniform(100.0, 5000.0, H)
    truth[:, 1] = r.uniform(0.2, 0.8, H)
    truth[:, 2] = r.uniform(0.01, 0.10, H)
    truth[:, 3] = r.uniform(1.0, 100.0, H)
    truth[:, 4] = r.uniform(-0.3, 0.3, H) * truth[:, 3]
    truth[:, 5] = r.uniform(-0.3, 0.3, H) * truth[:, 3]
    offsets = np.zeros(H + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(n)
    y = np.empty(int(offsets[-1]))
    rp = rng(index, 7)
    for h in range(H):
        mean = expected_counts_1d(1, 2, 1, 0.0, 1.0, int(n[h]), truth[h])
        y[offsets[h]:offsets[h + 1]] = rp.poisson(mean)
    start = truth * rng(index, THETA_SEED_OFFSET).uniform(0.8, 1.2, size=truth.shape)
    return dict(K=1, D=2, poly_mode=1, H=H, offsets=offsets, y=y, lo=np.zeros(H), hi=np.ones(H),
                truth=truth, start=start)


# ----------------------------------------------------------------------------
# workload 4: 2048-bin histograms of 3 peaks + linear background
# ----------------------------------------------------------------------------
def c5_truth(H, index=4, chunk=0):
    r = rng(index, 100 * chunk)
    A = r.uniform(100.0, 5000.0, (H, 3))
    mu = r.uniform(0.05, 0.95, (H, 3))
    s = r.uniform(0.005, 0.05, (H, 3))
    order = np.argsort(mu, axis=1)
    A = np.take_along_axis(A, order, 1)
    mu = np.take_along_axis(mu, order, 1)
    s = np.take_along_axis(s, order, 1)
    b0 = r.uniform(10.0, 200.0, H)
    b1 = r.uniform(10.0, 200.0, H) - b0
    th = np.zeros((H, 11))
    th[:, 0:9:3], th[:, 1:9:3], th[:, 2:9:3] = A, mu, s
    th[:, 9], th[:, 10] = b0, b1
    return th


def c5_batch(H=65536, n_bins=2048, index=4, chunk=0):
    truth = c5_truth(H, index, chunk)
    x = uniform_centres(n_bins, 0.0, 1.0)
    mean = np.empty((H, n_bins))
    step = 4096
    for h0 in range(0, H, step):
        t = truth[h0:h0 + step]
        m = t[:, 9:10] + t[:, 10:11] * x[None, :]
        for k in range(3):
            m = m + t[:, 3 * k:3 * k + 1] * np.exp(
                -0.5 * ((x[None, :] - t[:, 3 * k + 1:3 * k + 2]) / t[:, 3 * k + 2:3 * k + 3]) ** 2)
        mean[h0:h0 + step] = m
    y = rng(index, 100 * chunk + 7).poisson(mean).astype(np.float64)
    offsets = np.arange(H + 1, dtype=np.int64) * n_bins
    return dict(K=3, D=1, poly_mode=0, H=H, n_bins=n_bins, offsets=offsets, y=y.reshape(-1),
                lo=np.zeros(H), hi=np.ones(H), truth=truth)


# ----------------------------------------------------------------------------
# Fig. 3a: TH1D(1000 bins, [-5, 5]) filled with 100,000 draws of gaus(100, 1, 3)
# ----------------------------------------------------------------------------
def fig3a_histogram(index=5):
    lo, hi, n = -5.0, 5.0, 1000
    mu, s = 1.0, 3.0
    r = rng(index)
    a, b = ndtr((lo - mu) / s), ndtr((hi - mu) / s)
    x = mu + s * ndtri(a + r.random(100000) * (b - a))
    y = np.histogram(x, bins=n, range=(lo, hi))[0].astype(np.float64)
    return dict(K=1, D=-1, poly_mode=0, lo=lo, hi=hi, n=n, y=y)


# ----------------------------------------------------------------------------
# small random problems for parity tests
# ----------------------------------------------------------------------------
def random_gauss_poly(K, D, n, lo=0.0, hi=1.0, poly_mode=0, seed=0, noise=True):
    """A histogram with K well-separated peaks + positive background and a
    parameter point near its truth."""
    r = np.random.Generator(np.random.PCG64(SEED_BASE + 50000 + seed))
    th = np.zeros(3 * K + D + 1)
    span = hi - lo
    for k in range(K):
        th[3 * k] = r.uniform(50.0, 2000.0)
        th[3 * k + 1] = lo + span * (k + 0.5 + r.uniform(-0.2, 0.2)) / max(K, 1)
        th[3 * k + 2] = span * r.uniform(0.01, 0.08)
    if D >= 0:
        th[3 * K] = r.uniform(20.0, 100.0)
        for j in range(1, D + 1):
            scale = 1.0 if poly_mode == 1 else (1.0 / max(abs(hi), abs(lo), 1e-9)) ** j
            th[3 * K + j] = r.uniform(-0.2, 0.2) * th[3 * K] * scale
    mean = expected_counts_1d(K, D, poly_mode, lo, hi, n, th)
    y = r.poisson(np.maximum(mean, 0.0)).astype(np.float64) if noise else mean
    theta = th * r.uniform(0.9, 1.1, size=th.size)
    return dict(K=K, D=D, poly_mode=poly_mode, lo=lo, hi=hi, n=n, y=y, truth=th, theta=theta)


def c5_batch_device(H, n_bins=2048, index=4, chunk=0, device="cuda"):
    """Workload-4 histograms drawn on the GPU (for the 10^6-histogram training
    set): truth from c5_truth (numpy PCG64), expected counts at the bin
    centres, Poisson counts from a torch generator seeded with the same base
    seed.  Returns the batch as a dict whose "y" holds the counts as a device
    tensor [H * n_bins]."""
    import torch
    truth = c5_truth(H, index, chunk)
    t = torch.tensor(truth, device=device)
    x = torch.tensor(uniform_centres(n_bins, 0.0, 1.0), device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(SEED_BASE + index + 100 * chunk + 7)
    y = torch.empty((H, n_bins), dtype=torch.float64, device=device)
    step = 8192
    for h0 in range(0, H, step):
        tt = t[h0:h0 + step]
        m = tt[:, 9:10] + tt[:, 10:11] * x[None, :]
        for k in range(3):
            m = m + tt[:, 3 * k:3 * k + 1] * torch.exp(
                -0.5 * ((x[None, :] - tt[:, 3 * k + 1:3 * k + 2]) / tt[:, 3 * k + 2:3 * k + 3]) ** 2)
        y[h0:h0 + step] = torch.poisson(m, generator=gen)
    offsets = np.arange(H + 1, dtype=np.int64) * n_bins
    return dict(K=3, D=1, poly_mode=0, H=H, n_bins=n_bins, offsets=offsets, y=y.reshape(-1),
                lo=np.zeros(H), hi=np.ones(H), truth=truth)
