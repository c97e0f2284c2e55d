"""Failure detection on the GPU without a fault: the kernels' bounded wait
(the GEMM pipelines' mbarrier waits) run on a barrier that nothing
completes gives up after its limit, reports through the status word, and
leaves the context usable for the next calls."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2203_06139_gb300 import cg, synth
from tests._metrics import max_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def test_a_wait_that_nothing_completes_gives_up_and_reports(dev):
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cg.check_wait_timeout(err)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert int(err.item()) == 1
    assert 0.2 < dt < 20.0, dt   # the limit is about 2e9 clock cycles
    # the context is still usable: a GEMM on the tensor cores and a gradient
    g = torch.Generator(device="cuda").manual_seed(3)
    A = torch.randn((300, 256), generator=g, device=dev).to(torch.bfloat16)
    B = torch.randn((256, 256), generator=g, device=dev).to(torch.bfloat16)
    C = torch.empty((300, 256), dtype=torch.float32, device=dev)
    err2 = torch.zeros(1, dtype=torch.int32, device=dev)
    cg.gemm_bf16(A, B, 300, 256, 256, Cf=C, err=err2)
    ref = A.float() @ B.float().t()
    assert int(err2.item()) == 0
    assert float((C - ref).abs().max() / ref.abs().max()) < 1e-5
    p = synth.random_gauss_poly(1, 1, 2001, seed=4)
    pb = cg.Problem.gauss_poly(torch.tensor(p["y"], device=dev), 0.0, 1.0, 1, 1, cg.OBJ_CHI2)
    v, gr = cg.gradient(pb, torch.tensor(p["theta"], device=dev))
    r = oracle.binned1d(1, 1, 0, oracle.CHI2, p["y"], 0.0, 1.0, p["theta"])
    assert max_rel_err(gr.cpu().numpy(), r.grad, r.scale) <= 1e-10
    assert pb.status() == cg.OK


def test_the_check_refuses_a_bad_status_word(dev):
    with pytest.raises(cg.CgError):
        cg.check_wait_timeout(torch.zeros(1, dtype=torch.int64, device=dev))
