"""Channel sharding across ranks (one process per GPU).

Fine channels are independent correlation problems (paper Sec. 2: each
baseline carries 768 channels, each correlated on its own), so a job splits
into contiguous channel ranges with no exchange between ranks; the output of
rank r is the visibility block of its channels, and concatenating the
blocks in rank order gives the single-GPU result."""
from __future__ import annotations


def channel_range(n_chan: int, rank: int, world: int) -> tuple[int, int]:
    """[c0, c1) of rank ``rank``: contiguous, sizes differ by at most one,
    lower ranks take the extra channels."""
    if world < 1 or not 0 <= rank < world or n_chan < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n_chan, world)
    c0 = rank * base + min(rank, extra)
    return c0, c0 + base + (1 if rank < extra else 0)


def all_ranges(n_chan: int, world: int) -> list[tuple[int, int]]:
    return [channel_range(n_chan, r, world) for r in range(world)]
