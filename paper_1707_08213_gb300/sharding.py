"""Splitting one transform over several GPUs (one process per GPU) with no data exchange.

Windows are independent (Section 4.1, Eq. 2), so rank k of W computes a contiguous band of
window rows [q_begin, q_end) through the plan's band support; it reads input rows
[q_begin, q_end + n0 - 1) (an n0 - 1 row halo) and writes a disjoint slab of the output.
The only collectives are for timing (a barrier and a max-reduction); gathering the slabs,
if wanted, is the caller's choice.
"""
from __future__ import annotations

from typing import Tuple


def band_for_rank(P0: int, rank: int, world: int) -> Tuple[int, int]:
    """Window rows [begin, end) of `rank`: as equal as possible, earlier ranks get the
    remainder.  Every row is covered exactly once; a rank may get an empty band when
    world > P0."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    base, extra = divmod(P0, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def input_rows_for_band(begin: int, end: int, n0: int) -> Tuple[int, int]:
    """Input rows a band reads: its windows' rows plus the n0 - 1 row halo."""
    return begin, (end + n0 - 1) if end > begin else begin


def max_over_ranks(value: float, dist=None) -> float:
    """Slowest rank's time (the job's time) via an all-reduce, or the value itself."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
