"""The all-pair histogram of Sec. 2.3 split over several processes, one GPU each.

A handle's pair work list is deterministic and its units are independent, so rank r of W
evaluates the contiguous unit range shard_range(n_units, r, W) and one integer SUM
all-reduce combines the partial histograms. Integer counts make the result identical,
bit for bit, to the one-process histogram whatever the split.

Monte Carlo chains do not shard (every move depends on the one before it): several ranks
run independent replicas instead, and replica_seed gives each its own Philox key.
"""
from __future__ import annotations


def shard_range(n_units: int, rank: int, world: int) -> tuple[int, int]:
    """[t0, t1) of rank `rank` among `world`: contiguous, disjoint, covering [0, n_units),
    sizes differing by at most one (the first n_units mod world ranks take one more)."""
    if world < 1 or not 0 <= rank < world or n_units < 0:
        raise ValueError(f"bad split: n_units={n_units} rank={rank} world={world}")
    base, extra = divmod(n_units, world)
    t0 = rank * base + min(rank, extra)
    return t0, t0 + base + (1 if rank < extra else 0)


def replica_seed(seed: int, rank: int) -> int:
    """Philox key of rank `rank`'s replica chain (distinct for distinct ranks)."""
    return (int(seed) + int(rank)) & 0xFFFFFFFFFFFFFFFF


def partial_gr_sharded(box, hist, group=None, stream=None) -> tuple[int, int]:
    """Accumulate this rank's share of box's pair histogram into `hist` (int64, on the
    rank's GPU, `box.hist_len` entries) and SUM-all-reduce it over `group`.

    Every rank must pass a histogram that starts from zero: the all-reduce adds whatever it
    held before the call on every rank. The histogram kernels run on `stream` (the current
    torch stream when None); the all-reduce is ordered after them on torch's current stream.
    Returns the unit range this rank evaluated.
    """
    import torch
    import torch.distributed as dist

    world, rank = dist.get_world_size(group), dist.get_rank(group)
    t0, t1 = shard_range(box.epsr_partial_gr_tiles(), rank, world)
    if t1 > t0:
        box.epsr_partial_gr_range(t0, t1, hist, stream=stream)
    if hist.is_cuda and stream is not None:
        ext = stream if isinstance(stream, torch.cuda.Stream) else \
            torch.cuda.ExternalStream(int(stream), device=hist.device)
        torch.cuda.current_stream(hist.device).wait_stream(ext)
    dist.all_reduce(hist, op=dist.ReduceOp.SUM, group=group)
    return t0, t1
