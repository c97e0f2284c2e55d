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
    """All-gather every rank's (value, grad) and sum them in rank order."""
    vec = torch.cat([value.reshape(1).double(), grad.reshape(-1).double()])
    world = dist.get_world_size(group)
    bufs = [torch.empty_like(vec) for _ in range(world)]
    dist.all_gather(bufs, vec, group=group)
    tot = bufs[0].clone()
    for b in bufs[1:]:
        tot += b
    return tot[0], tot[1:]


def max_over_ranks(seconds, group=None, device="cpu"):
    """The slowest rank's time (the job's time)."""
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sharded_mixture_gradient(x, lo, hi, theta, group=None, precision=None):
    """Unbinned-mixture NLL and gradient of all events x (device tensor, the full
    sample on every rank or this rank's slice of it when `x` is already local),
    with this rank evaluating its shard on its GPU."""
    from . import cg
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    a, b = shard(x.numel(), rank, world)
    pb = cg.Problem.mixture(x[a:b].contiguous(), lo, hi,
                            precision=cg.PREC_DF64 if precision is None else precision)
    v, g = cg.gradient(pb, theta)
    vv, gg = combine(v.cpu(), g.cpu(), group)
    return vv, gg
