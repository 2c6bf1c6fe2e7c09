"""The pipelined persistent batch launch (csrc/batch_pipe.cuh, build_pipe in csrc/api.cpp),
replayed on the CPU.

A pipelined kernel takes tiles of one window shape (n0, n1) in ticket order: row tiles (a
block of z rows x a chunk of window columns, Eq. rowfswft2d) and column tiles (32 channels x
a chunk of window rows, Eq. colfswft2d).  A finished row tile raises its flag; a column tile
waits until the flags of the row tiles holding its z rows and window columns are up.  These
tests rebuild the host's tile order (same geometry rules as pipe_geom, same ordering as
build_pipe) for the batch shapes the library sees and check, without a GPU:

* every z row x window column is written by exactly one row tile, and every (window row,
  channel) is computed by exactly one column tile;
* the row tiles a column tile waits for hold every z value it reads, and all have earlier
  tickets (the wait can only be on work that has already started);
* an event simulation with a few resident blocks, each holding its tile and the prefetched
  next ticket, with random tile durations, always finishes (no deadlock), and a column tile
  never starts before every z value it reads is written.
"""
import heapq
import random

import numpy as np
import pytest

SM = 152
MAXN = 64


def bfu_threads(m0):
    return 256 if m0 >= 6 else 128


def bfu_B(m0):
    return 3 if m0 >= 6 else (m0 if m0 < 2 else 2)


def bfu_groups(m0):
    return 1 if m0 >= 6 else (4 >> bfu_B(m0))


def pipe_row_B(m1):
    return 3 if m1 >= 5 else (m1 if m1 < 3 else 3)


def rows_per_tile(m0, m1):
    return bfu_threads(m0) >> pipe_row_B(m1)


def default_row_chunk(P1, zrows, threads_per_row, n1):
    t = zrows * threads_per_row
    nc = max(1, (64 << 10) // max(t, 1))
    chunk = (P1 + nc - 1) // nc
    return min(max(chunk, max(1, n1 // 2)), P1)


def default_col_nchunks(nch, fused_small=False):
    groups = (nch + 31) // 32
    want = (4 * SM + groups - 1) // groups
    return min(max(want, 16 if fused_small else 8), 65535)


def default_col_chunk(rows, n0, nchunks):
    chunk = (rows + nchunks - 1) // nchunks
    return min(max(chunk, 2 * n0), rows)


def col_rows(ck, chunk, rows_out, n0):
    """z rows [lo, hi) column chunk ck reads (look-back n0/2 rows; padding rows not waited for)."""
    qa = ck * chunk
    qb = min(qa + chunk, rows_out)
    look = n0 // 2 if n0 >= 2 else 0
    return max(qa - look, 0), qb + n0 - 1


def geom(N0, N1, n0, n1):
    m0, m1 = n0.bit_length() - 1, n1.bit_length() - 1
    P0, P1 = N0 - n0 + 1, N1 - n1 + 1
    zrows = P0 + n0 - 1
    g = dict(m0=m0, m1=m1, n0=n0, n1=n1, P0=P0, P1=P1, zrows=zrows)
    g["rpb"] = rows_per_tile(m0, m1)
    g["row_chunk"] = default_row_chunk(P1, zrows, 1 << pipe_row_B(m1), n1)
    g["row_chunks"] = -(-P1 // g["row_chunk"])
    g["row_blocks"] = -(-zrows // g["rpb"])
    g["col_chunk"] = default_col_chunk(P0, n0, default_col_nchunks(P1 * n1))
    g["col_chunks"] = -(-P0 // g["col_chunk"])
    per_block = 32 * bfu_groups(m0)
    g["col_blocks"] = -(-(P1 * n1) // per_block)
    return g


Z_AHEAD = 48 << 20


def build(shapes, slots=1216):
    """Item list of one class: stages (per array, largest first, per column chunk: the row
    tiles first needed by the chunk, then its column tiles), each stage's column tiles held
    back until `slots` tickets follow its last row tile, later stages' row tiles filling the
    gap (the next stage's always, more up to Z_AHEAD bytes of z written ahead; build_pipe)."""
    gs = [geom(*s) for s in shapes]
    order = sorted(range(len(gs)), key=lambda i: -gs[i]["P0"] * gs[i]["P1"] * gs[i]["n0"] * gs[i]["n1"])
    st = []
    for i in order:
        g = gs[i]
        nxt = 0
        for ck in range(g["col_chunks"]):
            lo, hi = col_rows(ck, g["col_chunk"], g["P0"], g["n0"])
            rb1 = max(nxt, (hi - 1) // g["rpb"] + 1)
            rows = min(rb1 * g["rpb"], g["zrows"]) - min(nxt * g["rpb"], g["zrows"])
            st.append((i, nxt, rb1, ck, rows * g["P1"] * g["n1"] * 8))
            nxt = rb1
    items, dep_end = [], [0] * len(st)
    z_ahead, r = 0, 0

    def emit_rows(k):
        nonlocal z_ahead
        i, rb0, rb1, _, zb = st[k]
        for rb in range(rb0, rb1):
            for rc in range(gs[i]["row_chunks"]):
                items.append((i, "row", rb, rc))
        dep_end[k] = len(items)
        z_ahead += zb

    for k in range(len(st)):
        while r <= k + 1 and r < len(st):
            emit_rows(r)
            r += 1
        while r < len(st) and len(items) - dep_end[k] < slots and z_ahead + st[r][4] <= Z_AHEAD:
            emit_rows(r)
            r += 1
        i, _, _, ck, zb = st[k]
        for cb in range(gs[i]["col_blocks"]):
            items.append((i, "col", ck, cb))
        z_ahead -= zb
    return gs, items


def waits_for(g, ck, cb):
    """(row block, row chunk) flags a column tile polls: its z rows' blocks x the row chunks
    of its window columns (batch_pipe_kernel)."""
    lo, hi = col_rows(ck, g["col_chunk"], g["P0"], g["n0"])
    ch = 32 * bfu_groups(g["m0"])
    ch_lo = cb * ch
    ch_hi = min(ch_lo + ch, g["P1"] * g["n1"]) - 1
    rc_lo, rc_hi = (ch_lo >> g["m1"]) // g["row_chunk"], (ch_hi >> g["m1"]) // g["row_chunk"]
    return [(rb, rc) for rb in range(lo // g["rpb"], (hi - 1) // g["rpb"] + 1)
            for rc in range(rc_lo, rc_hi + 1)]


def reads(g, ck, cb):
    """z values (row, window column) a column tile reads that exist (rows >= 0)."""
    lo, hi = col_rows(ck, g["col_chunk"], g["P0"], g["n0"])
    ch = 32 * bfu_groups(g["m0"])
    ch_lo = cb * ch
    ch_hi = min(ch_lo + ch, g["P1"] * g["n1"]) - 1
    return lo, hi, ch_lo >> g["m1"], (ch_hi >> g["m1"]) + 1


# shapes of one window class each (the two-pass arrays of a persistent plan: n0 n1 > 64 or
# n1 = 64): the 256-image batch's sides and windows, then small and ragged edge cases
CLASSES = [
    [(1024, 1024, 64, 16), (128, 512, 64, 16), (256, 128, 64, 16)],
    [(512, 1024, 32, 32), (1024, 128, 32, 32)],
    [(1024, 256, 8, 32), (128, 128, 8, 32)],
    [(256, 1024, 16, 16), (16, 16, 16, 16), (17, 40, 16, 16)],
    [(70, 50, 8, 32), (40, 33, 8, 32)],
    [(64, 64, 64, 16), (65, 17, 64, 16)],
    [(40, 80, 2, 64), (9, 200, 2, 64)],
    [(9, 200, 1, 64), (3, 64, 1, 64)],
    [(300, 9, 64, 8), (64, 8, 64, 8)],
]


@pytest.mark.parametrize("shapes", CLASSES)
@pytest.mark.parametrize("slots", [1, 304, 1216])
def test_tiles_cover_every_z_row_and_output_once(shapes, slots):
    gs, items = build(shapes, slots)
    for i, g in enumerate(gs):
        rows = np.zeros((g["zrows"], g["P1"]), np.int32)
        outs = np.zeros((g["P0"], g["P1"] * g["n1"]), np.int32)
        for (j, kind, a, b) in items:
            if j != i:
                continue
            if kind == "row":
                r0, r1 = a * g["rpb"], min((a + 1) * g["rpb"], g["zrows"])
                c0, c1 = b * g["row_chunk"], min((b + 1) * g["row_chunk"], g["P1"])
                rows[r0:r1, c0:c1] += 1
            else:
                q0, q1 = a * g["col_chunk"], min((a + 1) * g["col_chunk"], g["P0"])
                ch = 32 * bfu_groups(g["m0"])
                outs[q0:q1, b * ch:min((b + 1) * ch, g["P1"] * g["n1"])] += 1
        assert (rows == 1).all(), "a z row x window column is written by no or several row tiles"
        assert (outs == 1).all(), "a window row x channel is computed by no or several column tiles"


def check_order(gs, items):
    """The flags a column tile polls cover every z value it reads, and their row tiles have
    earlier tickets."""
    ticket = {it: t for t, it in enumerate(items)}
    for t, (i, kind, a, b) in enumerate(items):
        if kind != "col":
            continue
        g = gs[i]
        flags = waits_for(g, a, b)
        lo, hi, q_lo, q_hi = reads(g, a, b)
        assert 0 <= lo < hi <= g["zrows"] and 0 <= q_lo < q_hi <= g["P1"]
        covered = np.zeros((hi - lo, q_hi - q_lo), bool)
        for rb, rc in flags:
            assert ticket[(i, "row", rb, rc)] < t, "a column tile waits on a later row tile"
            r0, r1 = max(rb * g["rpb"], lo), min((rb + 1) * g["rpb"], hi)
            c0, c1 = max(rc * g["row_chunk"], q_lo), min((rc + 1) * g["row_chunk"], q_hi)
            covered[r0 - lo:r1 - lo, c0 - q_lo:c1 - q_lo] = True
        assert covered.all(), "a column tile reads z values no awaited row tile writes"


@pytest.mark.parametrize("shapes", CLASSES)
@pytest.mark.parametrize("slots", [1, 304, 1216])
def test_column_tiles_wait_for_every_value_they_read_and_only_on_earlier_tiles(shapes, slots):
    check_order(*build(shapes, slots))


def _simulate(gs, items, blocks, seed, waits=waits_for):
    """Blocks take tickets in order (each holding its tile and the prefetched next ticket);
    a row tile finishes after a random time and raises its flag; a column tile starts when
    the flags it polls are up, and must then find every z value it reads written."""
    rng = random.Random(seed)
    n = len(items)
    flag = set()       # (i, rb, rc) of finished row tiles
    nxt = 0
    t_now = 0.0
    events = []        # (time, block, ticket) completions
    waiting = {}       # block -> ticket waiting for its flags
    held = {}          # block -> prefetched ticket

    def try_start(blk, t):
        i, kind, a, b = items[t]
        if kind == "col":
            g = gs[i]
            if any((i, rb, rc) not in flag for rb, rc in waits(g, a, b)):
                waiting[blk] = t
                return
            lo, hi, q_lo, q_hi = reads(g, a, b)
            for r in range(lo, hi):
                for q in (q_lo, q_hi - 1):
                    assert (i, r // g["rpb"], q // g["row_chunk"]) in flag, "column tile reads unwritten z"
        heapq.heappush(events, (t_now + rng.uniform(0.5, 2.0), blk, t))

    for blk in range(blocks):
        if nxt < n:
            cur, nxt = nxt, nxt + 1
            if nxt < n:
                held[blk], nxt = nxt, nxt + 1
            try_start(blk, cur)
    finished = 0
    while finished < n:
        if not events:
            raise AssertionError(f"deadlock: {len(waiting)} blocks waiting, {finished}/{n} tiles done")
        t_now, blk, t = heapq.heappop(events)
        i, kind, a, b = items[t]
        if kind == "row":
            flag.add((i, a, b))
        finished += 1
        for wb, wt in list(waiting.items()):
            del waiting[wb]
            try_start(wb, wt)
        if blk in held:
            cur = held.pop(blk)
            if nxt < n:
                held[blk], nxt = nxt, nxt + 1
            try_start(blk, cur)


@pytest.mark.parametrize("shapes", CLASSES)
@pytest.mark.parametrize("blocks", [1, 3, 40])
def test_pipelined_schedule_always_finishes(shapes, blocks):
    gs, items = build(shapes, slots=blocks)
    for seed in range(3):
        _simulate(gs, items, blocks, seed)


def test_planted_mistakes_are_caught():
    """A column tile moved before the row tiles it reads, or a column tile that polls one row
    chunk too few (its last window column's z unwritten): the checks fail."""
    gs, items = build(CLASSES[0])
    first_col = next(t for t, it in enumerate(items) if it[1] == "col")
    moved = [items[first_col]] + items[:first_col] + items[first_col + 1:]
    with pytest.raises(AssertionError):
        check_order(gs, moved)

    def short(g, ck, cb):
        f = waits_for(g, ck, cb)
        last = max(rc for _, rc in f)
        return [x for x in f if x[1] != last] if last > 0 else f[:-1]
    with pytest.raises(AssertionError):
        for seed in range(5):
            _simulate(gs, items, 40, seed, waits=short)
