"""Host-side helpers for runs with one process per GPU.

Particles are independent units of Algorithm 1, so a multi-GPU run needs no
exchange on the data path: every rank holds its own replica of the mesh and
locates its own particles. The only collectives are the reductions of the
measurement (slowest rank's time, total particle count). The paper's
subdomain decomposition with particle migration (Sec. 1, Sec. 3) is not used.
"""


def shard_range(n, rank, world):
    """Contiguous slice [lo, hi) of n particles owned by `rank` of `world`.

    The first n % world ranks take one extra particle, so the slices cover
    [0, n) exactly once and differ in size by at most one.
    """
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("shard_range: bad n/rank/world (%r, %r, %r)" % (n, rank, world))
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def _reduce(value, op, device=None):
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return t.item()


def max_over_ranks(value, device=None):
    """The largest value over all ranks (the slowest rank's time); the value
    itself without an initialised process group. `device` is where the
    reduction buffer lives: a CUDA device under NCCL, None (CPU) under gloo."""
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.MAX, device)


def sum_over_ranks(value, device=None):
    """The sum over all ranks (e.g. particles located by the whole job)."""
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.SUM, device)
