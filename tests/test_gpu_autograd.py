"""torch.autograd.Function over the fused kernel: gradients against central
finite differences (h = 1e-6 relative) of the kernel's own value and against
the CPU oracle, on the 2-D rotated-Gaussian Poisson NLL."""
import numpy as np
import pytest
import torch

import oracle
from paper_2203_06139_gb300 import cg, synth
from paper_2203_06139_gb300.autograd import fit_objective
from tests._metrics import max_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def _fd_ok(g, fd, F, th, scale):
    """Central differences at h_k = 1e-6 |theta_k| agree with g to 1e-5 (relative,
    floored at 1e-6 S_k) plus their own rounding error: F is known to an ulp or
    so at each point, so the difference quotient carries ~8 eps |F| / h_k."""
    h = 1e-6 * np.maximum(np.abs(th), 1e-3)
    allowed = 1e-5 * np.maximum(np.abs(g), 1e-6 * scale) + 8 * np.finfo(float).eps * abs(F) / h
    return np.all(np.abs(g - fd) <= allowed), np.max(np.abs(g - fd) / allowed)


def _fd(pb, th):
    g = np.zeros(th.numel())
    base = th.detach().cpu().numpy()
    for k in range(base.size):
        h = 1e-6 * max(abs(base[k]), 1e-3)
        tp, tm = base.copy(), base.copy()
        tp[k] += h
        tm[k] -= h
        fp = float(cg.objective(pb, torch.tensor(tp, device=th.device)))
        fm = float(cg.objective(pb, torch.tensor(tm, device=th.device)))
        g[k] = (fp - fm) / (2 * h)
    return g


@pytest.mark.parametrize("K,nx,ny", [(3, 96, 80), (8, 512, 512)])
def test_autograd_matches_fd_and_oracle(dev, K, nx, ny):
    truth = synth.c3_truth(K)
    counts = np.random.default_rng(K).poisson(synth.expected_counts_2d(truth, K, nx, ny)).astype(float)
    th0 = truth * (1 + np.random.default_rng(11).uniform(-0.05, 0.05, truth.size))
    pb = cg.Problem.rotgauss2d(torch.tensor(counts, device=dev), K)
    theta = torch.tensor(th0, device=dev, requires_grad=True)
    F = fit_objective(theta, pb)
    F.backward()
    g = theta.grad.detach().cpu().numpy()
    ref = oracle.binned2d(K, counts, 0.0, 1.0, 0.0, 1.0, th0)
    assert max_rel_err(g, ref.grad, ref.scale) <= 1e-10
    assert abs(float(F.detach()) - ref.value) <= 1e-10 * abs(ref.value)
    ok, worst = _fd_ok(g, _fd(pb, theta), ref.value, th0, ref.scale)
    assert ok, worst


def test_autograd_chain_rule_and_batch(dev):
    """Adjoint scaling through a downstream expression, and the batched form."""
    h = synth.c1_histogram(n_bins=2000)
    pb = cg.Problem.gauss_poly(torch.tensor(h["y"], device=dev), 0.0, 10.0, 1, 1, cg.OBJ_CHI2)
    th = torch.tensor(synth.c1_theta_points(4), device=dev, requires_grad=True)
    vals = fit_objective(th, pb)
    (3.0 * vals.sum() + vals[1] ** 2).backward()
    _, g = cg.batch_gradient(pb, th.detach())
    expect = 3.0 * g
    expect[1] += 2 * vals[1].detach() * g[1]
    torch.testing.assert_close(th.grad, expect, rtol=1e-14, atol=0)


@pytest.mark.slow
def test_autograd_c3_full_size(dev):
    """4096 x 4096 bins, 49 parameters: autograd gradient vs central FD."""
    hh = synth.c3_histogram()
    th0 = synth.c3_theta_point(hh["truth"])[0]
    pb = cg.Problem.rotgauss2d(torch.tensor(hh["counts"], device=dev), 8)
    theta = torch.tensor(th0, device=dev, requires_grad=True)
    F = fit_objective(theta, pb)
    F.backward()
    g = theta.grad.detach().cpu().numpy()
    fd = _fd(pb, theta)
    ok, worst = _fd_ok(g, fd, float(F.detach()), th0, np.abs(g))
    assert ok, worst
