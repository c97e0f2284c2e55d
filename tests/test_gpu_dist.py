"""The element-sharded gradient on a real NCCL process group.

This pool gives one GPU per process, so the group has one rank: the shard is
the whole sample and the exchange is NCCL's all-gather of the (1 + P)
device-resident partial sums, whose result must equal the unsharded call
bit for bit.  The multi-rank arithmetic (rank-ordered sums, uneven shards,
a rank that leaves) is covered by the gloo tests in test_dist.py.
"""
import os
import socket

import pytest
import torch

pytestmark = pytest.mark.gpu


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_sharded_mixture_gradient_over_nccl():
    import torch.distributed as dist
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_06139_gb300 import cg, synth
    from paper_2203_06139_gb300 import dist as cgdist
    assert not dist.is_initialized()
    dist.init_process_group("nccl", init_method="tcp://127.0.0.1:%d" % _port(), rank=0, world_size=1,
                            device_id=torch.device("cuda:0"))
    try:
        x = torch.tensor(synth.c2_events(100003), device="cuda")
        th = torch.tensor(synth.c2_theta_points(1)[0], device="cuda")
        v, g = cgdist.sharded_mixture_gradient(x, 0.0, 10.0, th)
        assert v.is_cuda and g.is_cuda and g.shape == (4,)
        v1, g1 = cg.gradient(cg.Problem.mixture(x, 0.0, 10.0), th)
        torch.cuda.synchronize()
        assert float(v) == float(v1) and torch.equal(g, g1)
    finally:
        dist.destroy_process_group()
