"""Running the path on several GPUs, one process per GPU (torch.distributed).

Two ways to use more GPUs, both over the member partition of Section III-D
(members are independent for fitness):

* independent populations: every rank evolves its own population(s) from its
  own seed; nothing crosses ranks on the data path, only the timing is reduced
  (`rank_seed`, `max_over_ranks`);
* one population split by members: every rank applies the operators of a
  generation to the same population (the draws are counter-based, so all
  ranks produce the same children), evaluates a contiguous slice of the
  children and the int64 fitness slices are all-gathered
  (`sharded_generation`).

The functions take the process group as an argument and work with any backend
whose tensors they are given (NCCL with device tensors, gloo with host tensors).
"""
from __future__ import annotations


def shard_bounds(total: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous slice [lo, hi) of `total` units owned by `rank`; sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def rank_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank`'s independent population."""
    return (seed + rank) & (2**64 - 1)


def _world(group):
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized():
        return 1, 0
    return dist.get_world_size(group), dist.get_rank(group)


def max_over_ranks(value: float, group=None, device=None) -> float:
    """The largest `value` over the ranks (the timing rule: the slowest rank decides)."""
    import torch
    import torch.distributed as dist

    world, _ = _world(group)
    if world == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def _group_active(group) -> bool:
    import torch.distributed as dist

    return dist.is_available() and dist.is_initialized()


def gather_slices(full, lo: int, hi: int, group=None):
    """Every rank owns full[lo:hi] of the 1-D tensor `full` (bounds from shard_bounds);
    afterwards every rank holds all slices.  With NCCL and device tensors the copies and the
    collective are ordered on torch's current stream (no host synchronisation).  Without a
    process group this is a no-op; with one, the collective runs even for a single rank."""
    import torch
    import torch.distributed as dist

    if not _group_active(group):
        return full
    world, _ = _world(group)
    total = full.numel()
    width = -(-total // world)
    mine = torch.zeros(width, dtype=full.dtype, device=full.device)
    mine[: hi - lo] = full[lo:hi]
    parts = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    for r, part in enumerate(parts):
        a, b = shard_bounds(total, world, r)
        full[a:b] = part[: b - a]
    return full


def sharded_generation(ctx, cfg, g: int, pop_in, fit_in, pop_out, fit_out, group=None):
    """One generation of a population split by members: the operators on every rank
    (identical children), the fitness of this rank's slice of the s-1 children, then an
    all-gather of the int64 fitness.  `ctx` needs offspring() and fitness() (Context).

    Everything is ordered on the context's stream: the kernels run there, and the all-gather
    is issued with that stream as torch's current stream, so NCCL waits for the slice's fitness
    and the next generation's kernels wait for the gathered values without any host
    synchronisation.  A context without a CUDA stream (a host stand-in) is synchronised
    instead."""
    world, rank = _world(group)
    if not _group_active(group):  # one process: the plain generation
        return ctx.generation(cfg, g, pop_in, fit_in, pop_out, fit_out)
    ctx.offspring(cfg, g, pop_in, fit_in, pop_out, fit_out)
    children = cfg.pop - 1
    lo, hi = shard_bounds(children, world, rank)
    if hi > lo:
        ctx.fitness(pop_out[1 + lo:1 + hi], out=fit_out[1 + lo:1 + hi])
    stream = getattr(ctx, "stream", None)
    if stream is None:
        ctx.sync()
        gather_slices(fit_out[1:], lo, hi, group)
    else:
        import torch

        with torch.cuda.stream(stream):
            gather_slices(fit_out[1:], lo, hi, group)
    return pop_out, fit_out
