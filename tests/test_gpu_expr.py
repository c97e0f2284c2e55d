"""Expression programs on the GPU: the generated forward + reverse kernels
against the oracle's expression interpreter (1e-10, the parity bar of the
hand-written kernels), values only, several parameter points, determinism."""
import numpy as np
import pytest
import torch

import oracle
from paper_2203_06139_gb300 import cg, synth
from paper_2203_06139_gb300 import expr as E
from tests._metrics import max_rel_err
from tests.test_expr_cpu import _odd_expression, chi2_gauss_linear, mixture_nll

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def _check(prog, nl, n_params, inputs, thetas, dev):
    ins = [torch.tensor(a, device=dev) for a in inputs]
    tt = torch.tensor(thetas, device=dev)
    v, g = prog.gradient(ins, tt)
    v2 = prog.objective(ins, tt)
    v3, g3 = prog.gradient(ins, tt)
    torch.cuda.synchronize()
    v, g, v2 = v.cpu().numpy(), g.cpu().numpy(), v2.cpu().numpy()
    assert np.array_equal(v, v3.cpu().numpy()) and np.array_equal(g, g3.cpu().numpy())   # deterministic
    assert np.array_equal(v, v2)
    for h in range(len(thetas)):
        r = oracle.expr(nl, n_params, inputs, thetas[h])
        assert r.rc == oracle.OK
        assert abs(v[h] - r.value) <= 1e-10 * abs(r.value), (h, v[h], r.value)
        assert max_rel_err(g[h], r.grad, r.scale) <= 1e-10, (h, g[h], r.grad)


def test_generated_chi2_matches_the_oracle(dev):
    p = synth.c1_histogram()
    root = chi2_gauss_linear(0.0, 10.0, 10000)
    prog = E.compile(root, 5, 1)
    assert "cgx_tiles" in prog.source and prog.num_acc >= 2
    _check(prog, E.nodes(root), 5, [p["y"]], synth.c1_theta_points(6), dev)


def test_generated_mixture_with_normalisations_matches_the_oracle(dev):
    x = synth.c2_events(300001)
    root = mixture_nll(0.0, 10.0)
    prog = E.compile(root, 4, 1)
    th = synth.c2_theta_points(5)
    _check(prog, E.nodes(root), 4, [x], th, dev)
    # and the hand-built oracle of the same objective
    v, g = prog.gradient([torch.tensor(x, device=dev)], torch.tensor(th, device=dev))
    for h in range(len(th)):
        r = oracle.unbinned_mix(x, 0.0, 10.0, th[h])
        assert max_rel_err(g[h].cpu().numpy(), r.grad, r.scale) <= 1e-10


def test_generated_odd_expression_matches_the_oracle(dev):
    rng = np.random.default_rng(11)
    u, w = rng.uniform(0.5, 2.0, 7777), rng.uniform(-1.0, 1.0, 7777)
    root = _odd_expression()
    prog = E.compile(root, 3, 2)
    th = np.array([[0.7, 1.3, 0.4], [1.1, 0.9, -0.3], [0.2, 2.0, 1.5]])
    _check(prog, E.nodes(root), 3, [u, w], th, dev)


def test_single_element_and_many_points(dev):
    root = chi2_gauss_linear(0.0, 1.0, 1)
    prog = E.compile(root, 5, 1)
    y = np.array([7.0])
    th = np.tile(np.array([3.0, 0.5, 0.2, 1.0, 0.5]), (300, 1)) * np.linspace(0.9, 1.1, 300)[:, None]
    _check(prog, E.nodes(root), 5, [y], th, dev)


def test_malformed_program_raises(dev):
    with pytest.raises(cg.CgError):
        E.compile(E.param(0) * 2.0, 1, 0)   # no element dependence


def test_generated_eight_peaks_matches_the_oracle(dev):
    """A program with 26 parameters (8 Gaussians + line): the sweep of the
    Fig. 3b comparison uses such programs."""
    K, n = 8, 20000
    p = synth.random_gauss_poly(K, 1, n, seed=77)
    x = (E.index() + 0.5) * (1.0 / n)
    f = E.param(3 * K) + E.param(3 * K + 1) * x
    for k in range(K):
        f = f + E.param(3 * k) * E.exp(-(x - E.param(3 * k + 1)) ** 2 / (2.0 * E.param(3 * k + 2) ** 2))
    y = E.inp(0)
    root = (y - f) ** 2 / E.maximum(y, 1.0)
    prog = E.compile(root, 3 * K + 2, 1)
    th = np.stack([p["theta"], p["truth"] * 1.02])
    _check(prog, E.nodes(root), 3 * K + 2, [p["y"]], th, dev)
    vo = E.compile(root, 3 * K + 2, 1, value_only=True)
    v = vo.objective([torch.tensor(p["y"], device=dev)], torch.tensor(th, device=dev)).cpu().numpy()
    for h in range(2):
        r = oracle.expr(E.nodes(root), 3 * K + 2, [p["y"]], th[h])
        assert abs(v[h] - r.value) <= 1e-10 * abs(r.value)
    with pytest.raises(cg.CgError):
        vo.gradient([torch.tensor(p["y"], device=dev)], torch.tensor(th, device=dev))



def test_generated_thirty_two_peaks_matches_the_oracle(dev):
    """98 parameters (32 Gaussians + line): 99 per-thread accumulators, past
    the register file (they spill); the largest program of the Fig. 3b sweep."""
    K, n = 32, 3000
    p = synth.random_gauss_poly(K, 1, n, seed=432)
    x = (E.index() + 0.5) * (1.0 / n)
    f = E.param(3 * K) + E.param(3 * K + 1) * x
    for k in range(K):
        f = f + E.param(3 * k) * E.exp(-(x - E.param(3 * k + 1)) ** 2 / (2.0 * E.param(3 * k + 2) ** 2))
    y = E.inp(0)
    root = (y - f) ** 2 / E.maximum(y, 1.0)
    prog = E.compile(root, 3 * K + 2, 1)
    assert prog.num_acc > 64
    _check(prog, E.nodes(root), 3 * K + 2, [p["y"]], np.stack([p["theta"], p["truth"]]), dev)
