"""Partition of one batch of subproblems over several GPUs, one process per GPU.

The subproblems of a batch (boxes, properties, branch-and-bound subdomains) are independent: the
solvers batch them along one axis (Sec. 6.1) and never mix them. A job over several GPUs therefore
gives each rank a contiguous slice of the batch, replicates the network on every rank, bounds the
slices with no exchange between ranks, and gathers the bounds once at the end. Host-side plumbing
only: the bounding itself runs in each rank's own context.
"""
from __future__ import annotations


def shard_batch(S: int, world: int, rank: int) -> tuple[int, int]:
    """[start, stop) of rank's contiguous slice of S subproblems; slices differ in size by at most
    one, the larger ones first, and cover 0 .. S - 1 in rank order."""
    if S < 0 or world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad partition: S={S}, world={world}, rank={rank}")
    base, extra = divmod(S, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def gather_bounds(local, S: int, dist, device=None):
    """Every rank's slice of the bounds, gathered in batch order on every rank (one all_gather of
    slices padded to the largest one; the only collective of a bounding job). local: the rank's
    bounds, a 1-D float64 tensor of its slice's length; with one process (dist None or not
    initialised) it is returned as is."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return local
    world, rank = dist.get_world_size(), dist.get_rank()
    width = -(-S // world)
    buf = torch.zeros(width, dtype=torch.float64, device=device if device is not None else local.device)
    buf[:local.numel()] = local
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    out = []
    for r, p in enumerate(parts):
        a, b = shard_batch(S, world, r)
        out.append(p[:b - a])
    return torch.cat(out)
