"""One objective sharded over ranks (one process per GPU).

The objective is a sum of independent per-element terms, so a large problem
splits into contiguous element ranges: every rank evaluates its range with
the fused kernel and the ranks exchange one (1 + P)-vector per evaluation,
gathered and summed in rank order so the result is the same on every rank
and on every run.  For the unbinned mixture the per-range value and gradient
are exactly additive (the epilogue is linear in the accumulators), so the
sum equals the single-process result up to summation order.
"""
import torch
import torch.distributed as dist


def shard(n, rank, world):
    """Contiguous range [lo, hi) of n elements for `rank` of `world` (balanced)."""
    base, rem = divmod(int(n), int(world))
    lo = rank * base + min(rank, rem)
    return lo, lo + base + (1 if rank < rem else 0)


def combine(value, grad, group=None):
    """All-gather every rank's (value, grad) and sum them in rank order.

    One exchange of (1 + P) doubles per rank, on the device the tensors live
    on (CUDA tensors under NCCL, CPU tensors under gloo); the rank-ordered
    sum makes the result the same on every rank and on every run."""
    vec = torch.cat([value.reshape(1).double(), grad.reshape(-1).double()])
    world = dist.get_world_size(group)
    bufs = [torch.empty_like(vec) for _ in range(world)]
    dist.all_gather(bufs, vec, group=group)
    tot = bufs[0].clone()
    for b in bufs[1:]:
        tot += b
    return tot[0], tot[1:]


def shard_batch(offsets, rank, world):
    """Histograms [h0, h1) of `rank` for a batch with CSR bin offsets
    (offsets[H] + 1 entries): contiguous ranges cut where the running bin count
    first reaches r / world of the total, so every rank's bins are within one
    histogram's size of total / world."""
    import numpy as np
    offsets = np.asarray(offsets, dtype=np.int64)
    H = len(offsets) - 1
    total = int(offsets[-1] - offsets[0])

    def cut(r):
        if r <= 0:
            return 0
        if r >= world:
            return H
        return int(np.searchsorted(offsets, offsets[0] + total * r / world, side="left"))

    lo = cut(rank)
    return lo, max(lo, cut(rank + 1))


def gather_batch(values, grads, h0, H, P, group=None):
    """Every rank's per-histogram results (values [h1 - h0], grads [h1 - h0, P]
    of its histograms from h0; a rank with no histograms passes empty
    tensors) assembled into [H] and [H, P] on every rank: one all-reduce of
    zero-padded arrays of H (1 + P) doubles, exact (each entry is one rank's
    number plus zeros).  P is passed, not read from grads, so that every rank
    reduces the same length whatever it holds."""
    n = values.numel()
    if grads.numel() != n * P:
        raise ValueError("grads must hold P = %d values per histogram" % P)
    full = torch.zeros(H * (1 + P), dtype=torch.float64, device=values.device)
    full[h0:h0 + n] = values.double()
    if P and n:
        full[H + h0 * P:H + (h0 + n) * P] = grads.double().reshape(-1)
    dist.all_reduce(full, op=dist.ReduceOp.SUM, group=group)
    return full[:H], full[H:].reshape(H, P)


def max_over_ranks(seconds, group=None, device="cpu"):
    """The slowest rank's time (the job's time)."""
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sharded_mixture_gradient(x, lo, hi, theta, group=None, precision=None):
    """Unbinned-mixture NLL and gradient of all events x (device tensor, the full
    sample on every rank), with this rank evaluating its contiguous shard on
    its GPU (FP64 unless another precision is asked for) and the (1 + 4)
    partial sums exchanged on the device by combine()."""
    from . import cg
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    a, b = shard(x.numel(), rank, world)
    pb = cg.Problem.mixture(x[a:b].contiguous(), lo, hi,
                            precision=cg.PREC_FP64 if precision is None else precision)
    v, g = cg.gradient(pb, theta)
    return combine(v, g, group)
