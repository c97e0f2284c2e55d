"""Multi-rank host logic on CPU (gloo, world size 2): sharding, the
rank-ordered combination of partial sums, max-over-ranks timing, and a rank
that leaves before the exchange.  The per-shard partial sums come from the
CPU oracle (these processes have no GPU)."""
import datetime
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2203_06139_gb300 import dist as cgdist


def test_shard_partitions_exactly():
    for n in (0, 1, 7, 1000, 10 ** 7 + 3):
        for world in (1, 2, 3, 8):
            rs = [cgdist.shard(n, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            for (a, b), (c, d) in zip(rs, rs[1:]):
                assert b == c
            sizes = [b - a for a, b in rs]
            assert max(sizes) - min(sizes) <= 1


def test_shard_batch_balances_bins():
    rng = np.random.default_rng(4)
    for H in (1, 2, 7, 4096):
        n = np.rint(np.exp(rng.uniform(np.log(64), np.log(65536), H))).astype(np.int64)
        offs = np.concatenate([[0], np.cumsum(n)])
        for world in (1, 2, 3, 8):
            rs = [cgdist.shard_batch(offs, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == H
            for (a, b), (c, d) in zip(rs, rs[1:]):
                assert b == c
            bins = [int(offs[b] - offs[a]) for a, b in rs]
            assert max(abs(x - offs[-1] / world) for x in bins) <= n.max()


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, x, theta, out_dir, mode):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    import oracle
    try:
        if mode == "leave" and rank == 1:
            return   # leaves between steps: no collective in flight
        a, b = cgdist.shard(x.size, rank, world)
        r = oracle.unbinned_mix(x[a:b], 0.0, 10.0, theta)
        try:
            v, g = cgdist.combine(torch.tensor(r.value, dtype=torch.float64), torch.tensor(r.grad, dtype=torch.float64))
            t = cgdist.max_over_ranks(0.5 + rank)
            np.save(os.path.join(out_dir, "r%d.npy" % rank), np.concatenate([[float(v)], g.numpy(), [t]]))
        except Exception as e:   # the peer is gone: the collective must fail, not hang
            open(os.path.join(out_dir, "err%d.txt" % rank), "w").write(type(e).__name__ + ": " + str(e)[:200])
    finally:
        if not (mode == "leave" and rank == 1):
            try:
                dist.destroy_process_group()
            except Exception:
                pass


def _batch_worker(rank, world, port, ys, offs, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    import oracle
    try:
        h0, h1 = cgdist.shard_batch(offs, rank, world)
        th = np.array([1000.0, 0.5, 0.05, 50.0, 2.0, -1.0])
        rs = [oracle.binned1d(1, 2, 1, oracle.CHI2, ys[offs[h]:offs[h + 1]], 0.0, 1.0, th) for h in range(h0, h1)]
        v = torch.tensor([r.value for r in rs], dtype=torch.float64)
        g = torch.tensor(np.array([r.grad for r in rs], dtype=np.float64).reshape(-1, 6), dtype=torch.float64)
        V, G = cgdist.gather_batch(v, g, h0, len(offs) - 1, 6)
        np.save(os.path.join(out_dir, "b%d.npy" % rank), np.concatenate([V.numpy(), G.numpy().reshape(-1)]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_batch_equals_single_process(tmp_path):
    """Histograms split by bins over two gloo ranks, each evaluating its own
    (CPU oracle here), gathered: bit-identical to one process."""
    import oracle
    from paper_2203_06139_gb300 import synth
    d = synth.c4_batch(H=9, max_bins=3000)
    ys, offs = d["y"], d["offsets"]
    mp.start_processes(_batch_worker, args=(2, _port(), ys, offs, str(tmp_path)), nprocs=2, start_method="spawn")
    b0, b1 = np.load(tmp_path / "b0.npy"), np.load(tmp_path / "b1.npy")
    assert np.array_equal(b0, b1)
    th = np.array([1000.0, 0.5, 0.05, 50.0, 2.0, -1.0])
    ref = [oracle.binned1d(1, 2, 1, oracle.CHI2, ys[offs[h]:offs[h + 1]], 0.0, 1.0, th) for h in range(9)]
    assert np.array_equal(b0[:9], np.array([r.value for r in ref]))
    assert np.array_equal(b0[9:].reshape(9, 6), np.array([r.grad for r in ref]))


def test_two_ranks_sum_equals_single_process(tmp_path):
    from paper_2203_06139_gb300 import synth
    import oracle
    x = synth.c2_events(20001)
    th = synth.c2_theta_points(1)[0]
    mp.start_processes(_worker, args=(2, _port(), x, th, str(tmp_path), "ok"), nprocs=2, start_method="spawn")
    r0, r1 = np.load(tmp_path / "r0.npy"), np.load(tmp_path / "r1.npy")
    assert np.array_equal(r0, r1)                     # every rank holds the same result
    ref = oracle.unbinned_mix(x, 0.0, 10.0, th)
    assert abs(r0[0] - ref.value) <= 1e-12 * abs(ref.value)
    np.testing.assert_allclose(r0[1:5], ref.grad, rtol=1e-11)
    assert r0[5] == 1.5                               # max over ranks of 0.5 + rank


def test_rank_leaving_makes_the_exchange_fail_not_hang(tmp_path):
    from paper_2203_06139_gb300 import synth
    x = synth.c2_events(1001)
    th = synth.c2_theta_points(1)[0]
    mp.start_processes(_worker, args=(2, _port(), x, th, str(tmp_path), "leave"), nprocs=2, start_method="spawn")
    assert (tmp_path / "err0.txt").exists(), "rank 0 should see the exchange fail"
    assert not (tmp_path / "r0.npy").exists()


def test_a_rank_without_histograms_still_gathers(tmp_path):
    """One histogram over two ranks: the second rank owns none, passes empty
    results, and both ranks still assemble the same [H], [H, P] arrays."""
    import oracle
    from paper_2203_06139_gb300 import synth
    d = synth.c4_batch(H=1, max_bins=3000)
    ys, offs = d["y"], d["offsets"]
    assert cgdist.shard_batch(offs, 1, 2) == (1, 1)
    mp.start_processes(_batch_worker, args=(2, _port(), ys, offs, str(tmp_path)), nprocs=2, start_method="spawn")
    b0, b1 = np.load(tmp_path / "b0.npy"), np.load(tmp_path / "b1.npy")
    assert np.array_equal(b0, b1) and b0.size == 1 + 6
    th = np.array([1000.0, 0.5, 0.05, 50.0, 2.0, -1.0])
    ref = oracle.binned1d(1, 2, 1, oracle.CHI2, ys, 0.0, 1.0, th)
    assert b0[0] == ref.value and np.array_equal(b0[1:], ref.grad)
