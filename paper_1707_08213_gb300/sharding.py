"""Splitting work over several GPUs (one process per GPU) with no data exchange.

Windows are independent (Section 4.1, Eq. 2), so rank k of W computes a contiguous band of
window rows [q_begin, q_end) through the plan's band support; it reads input rows
[q_begin, q_end + n0 - 1) (an n0 - 1 row halo) and writes a disjoint slab of the output.
A batch of independent images is split by whole images instead (`assign_images`: longest
processing time first on output bytes, the transform's dominant cost).  The only
collectives are for timing (a barrier and a max-reduction); gathering the results, if
wanted, is the caller's choice.
"""
from __future__ import annotations

import heapq
from typing import List, Optional, Sequence, Tuple


def band_for_rank(P0: int, rank: int, world: int) -> Tuple[int, int]:
    """Window rows [begin, end) of `rank`: as equal as possible, earlier ranks get the
    remainder.  Every row is covered exactly once; a rank may get an empty band when
    world > P0."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    base, extra = divmod(P0, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def plan_bands(P0: int, rank: int, world: int) -> Optional[List[Tuple[int, int]]]:
    """The `bands` argument of a one-array Transform (swdft2d_shape's row_begin/row_end, in
    window-start coordinates) for this rank's share of one transform: None (every window row)
    on a single rank, else [band_for_rank(P0, rank, world)]."""
    return None if world == 1 else [band_for_rank(P0, rank, world)]


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


def output_bytes(N0: int, N1: int, n0: int, n1: int) -> int:
    """Bytes of one image's output, P0 * P1 * n0 * n1 complex64: the work the transform's
    memory-bound passes scale with."""
    return 8 * (N0 - n0 + 1) * (N1 - n1 + 1) * n0 * n1


def assign_images(costs: Sequence[float], world: int) -> List[List[int]]:
    """Images per rank by longest processing time first: images in decreasing cost order,
    each to the rank with the least assigned cost so far (lowest rank on ties).  Every
    image goes to exactly one rank; the largest load is at most 4/3 - 1/(3 world) times the
    best possible.  Deterministic, so every rank computes the same assignment locally."""
    if world < 1:
        raise ValueError("bad world")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    out: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    for lst in out:
        lst.sort()
    return out
