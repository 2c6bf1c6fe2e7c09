"""The GPU trees' per-thread schedules, executed step by step on the CPU.

The sliding tree of Section 4.2 along one axis runs on the GPU as a walk over window-end
positions p in which every level keeps a FIFO of the values it needs again s_v steps later,
optionally split over 2^B threads by node residue (tree_core.cuh, SlidingTree), and its
transpose walks p downwards (adjoint_core.cuh, SlidingTreeAdjoint); the ternary tree of
windows 3^M splits by residue mod 3 (tree3_core.cuh, SlidingTree3Split).  These tests replay
exactly those schedules -- the same FIFO depths, slot indices (step index modulo the FIFO
depth), node residues and twiddle indices -- in plain Python for every window length
2^M <= 64 and split B <= min(M, 3) (and 3^M <= 27), and compare with numpy's FFT of every window (forward)
and with the explicit overlap-add of every window's inverse DFT (adjoint).  They pin the
index arithmetic of the kernels' register schedules without a GPU.

The later tests replay whole passes block by block, with each block's shared-memory staging:
the two adjoint passes (cp.async staging of G into a ring in a bank-conflict-free layout,
chunking of window rows and columns, the side rows two column chunks share and the fold that
adds them) for every window side they build, and
the forward passes (row_tile into z; col_tile_impl with its ring of z rows fed by copies of z
or by the fused form's shuffled row DFTs), and the ternary passes (row_tree3_kernel's staged
run write-back; col_tree3_kernel's ring and its staged copy-out).
"""
import numpy as np
import pytest


def held(B, u):
    """Nodes of level u one thread of a 2^B split holds."""
    return 1 if u <= B else 1 << (u - B)


def fifo_depth(M, u):
    """Steps a level-u value waits before level u + 1 reads it again (s_{u+1} = 2^(M-u-1))."""
    return 1 << (M - u - 1)


def tw_offset(B, v):
    """First twiddle of level v in a thread's table (levels 1..v-1 before it)."""
    return sum(1 if w <= B else held(B, w - 1) for w in range(1, v))


def forward_tree(M, B, c, feeds, j0=0):
    """Thread c of the sliding tree (tree_core.cuh, SlidingTree) over the steps j = j0, j0 + 1, ..:
    feeds[j - j0] = (x at the window's end position, x n/2 positions earlier), values or arrays
    over independent lanes; returns the thread's level-M nodes k = c + 2^B t at every step.
    The FIFOs start at zero, as the kernels' do."""
    n = 1 << M
    om = np.exp(-2j * np.pi * np.arange(n) / n)
    tw = [0j] * max(1, tw_offset(B, M + 1))
    cb = c & ((1 << B) - 1)
    for v in range(1, M + 1):
        base = tw_offset(B, v)
        if v <= B:
            tw[base] = om[(c & ((1 << v) - 1)) << (M - v)]
        else:
            for t in range(held(B, v - 1)):
                tw[base + t] = om[(cb + (t << B)) << (M - v)]
    fifos = {u: [[0j] * held(B, u) for _ in range(fifo_depth(M, u))] for u in range(1, M)}
    period = 1 << (M - 2) if M >= 2 else 1  # the kernels' unroll period
    outs = []
    for i, (xp, xs) in enumerate(feeds):
        J = (j0 + i) % period
        cur = [xp] + [0j] * (held(B, M) - 1)
        for v in range(1, M + 1):
            hp = held(B, v - 1)
            if v == 1:
                old = [xs]  # level 0 is re-read, no FIFO
            else:
                slot = J % fifo_depth(M, v - 1)
                old = list(fifos[v - 1][slot])
                fifos[v - 1][slot] = cur[:hp]
            tb = tw_offset(B, v)
            if v <= B:
                cur[0] = old[0] + tw[tb] * cur[0]
            else:
                for t in range(hp):
                    prod = tw[tb + t] * cur[t]
                    cur[t + hp] = old[t] - prod
                    cur[t] = old[t] + prod
        outs.append(cur[:held(B, M)])
    return outs


def forward_walk(M, B, c, x):
    """Thread c's outputs (nodes k = c + 2^B t of level M) at every position p of x."""
    n = 1 << M
    feeds = [(x[p], x[max(p - n // 2, 0)] if M >= 1 else 0j) for p in range(len(x))]
    return forward_tree(M, B, c, feeds)


def adjoint_tree(M, B, c, feeds, tail_from=None):
    """Thread c of the transposed tree (adjoint_core.cuh, SlidingTreeAdjoint) over the steps
    j = 0, 1, ..: feeds[j] = its held level-M inputs (k = c + 2^B t) at step j, each a value
    or an array over independent lanes; returns the thread's partial output at every step.
    From step tail_from on the output is the level-1 FIFO slot alone (SlidingTreeAdjoint::tail),
    with no tree evaluated."""
    n = 1 << M
    om = np.exp(-2j * np.pi * np.arange(n) / n)
    cb = c & ((1 << B) - 1)
    tw = {}
    for v in range(1, M + 1):
        if v > B:
            tw[v] = [np.conj(om[(cb + (t << B)) << (M - v)]) for t in range(held(B, v - 1))]
        else:
            tw[v] = [np.conj(om[(c & ((1 << v) - 1)) << (M - v)])]
    rings = {v: [[0j] * (held(B, v - 1) if v > B else 1) for _ in range(1 << (M - v))]
             for v in range(1, M + 1)}
    period = 1 << (M - 1) if M >= 1 else 1
    outs = []
    for j, feed in enumerate(feeds):
        J = j % period
        if tail_from is not None and j >= tail_from:
            outs.append(rings[1][J % (1 << (M - 1))][0])
            continue
        cur = list(feed)
        for v in range(M, 0, -1):
            slot = J % (1 << (M - v))
            if v > B:
                hp = held(B, v - 1)
                for t in range(hp):
                    d = cur[t] - cur[t + hp]
                    s = cur[t] + cur[t + hp]
                    old = rings[v][slot][t]
                    rings[v][slot][t] = s
                    cur[t] = tw[v][t] * d + old
            else:
                old = rings[v][slot][0]
                rings[v][slot][0] = cur[0]
                cur[0] = tw[v][0] * cur[0] + old
        outs.append(cur[0])
    return outs


def adjoint_walk(M, B, c, G, N):
    """Thread c's partial of y[p] = sum_j sum_k G[p-j][k] w_n^{+jk}, p = N-1 .. 0."""
    n = 1 << M
    cb = c & ((1 << B) - 1)
    ks = [cb + (t << B) for t in range(held(B, M))]
    feeds = []
    for p in range(N - 1, -1, -1):
        q = p - (n - 1)
        feeds.append([G[q][k] if 0 <= q < len(G) else 0j for k in ks])
    return np.array(adjoint_tree(M, B, c, feeds))[::-1]


SPLITS = [(M, B) for M in range(0, 7) for B in range(0, min(M, 3) + 1)]


@pytest.mark.parametrize("M,B", SPLITS)
def test_forward_schedule_gives_every_windows_dft(M, B):
    n = 1 << M
    rng = np.random.default_rng(10 * M + B)
    x = rng.standard_normal(n + 21) + 1j * rng.standard_normal(n + 21)
    for c in range(1 << B):
        outs = forward_walk(M, B, c, x)
        ks = [(c & ((1 << B) - 1)) + (t << B) for t in range(held(B, M))]
        for p in range(n - 1, len(x)):
            ref = np.fft.fft(x[p - n + 1:p + 1])
            np.testing.assert_allclose(outs[p], ref[ks], atol=1e-9)


def row_walk_start(M):
    """First step of a row-pass chunk's walk (row_tile): level 1 reads level 0 n/2 positions back
    from memory, so the output at step n - 1 needs level 1 from step n - 1 - (n/2 - 1) = n/2 on
    (the FIFO depths of levels 1 .. M-1 add up to n/2 - 1); steps before it are never needed."""
    return (1 << M) // 2


def col_walk_start(M, group_aligned=True):
    """First step of a column tile's walk (col_tile_impl): n/2, rounded down to whole step groups
    for the TMA stage, whose every fetch must start on a group."""
    half = (1 << M) // 2
    return (half // col_group(M)) * col_group(M) if group_aligned else half


def late_walk(M, B, c, x, j0):
    n = 1 << M
    feeds = [(x[p], x[p - n // 2] if M >= 1 else 0j) for p in range(j0, len(x))]
    return forward_tree(M, B, c, feeds, j0)


@pytest.mark.parametrize("M,B", SPLITS)
def test_walk_started_at_half_a_window_gives_every_windows_dft(M, B):
    """Zeroed FIFOs and a walk that starts at the row or column pass's first step: every
    complete window (end position >= n - 1) is still exact."""
    n = 1 << M
    rng = np.random.default_rng(900 + 10 * M + B)
    x = rng.standard_normal(n + 21) + 1j * rng.standard_normal(n + 21)
    for j0 in sorted({row_walk_start(M), col_walk_start(M)}):
        assert j0 % (1 << (M - 2) if M >= 2 else 1) == 0  # FIFO slots keep their step residues
        for c in range(1 << B):
            outs = late_walk(M, B, c, x, j0)
            ks = [(c & ((1 << B) - 1)) + (t << B) for t in range(held(B, M))]
            for p in range(n - 1, len(x)):
                np.testing.assert_allclose(outs[p - j0], np.fft.fft(x[p - n + 1:p + 1])[ks], atol=1e-9)


@pytest.mark.parametrize("M", [2, 3, 4, 5, 6])
def test_walk_started_one_period_too_late_is_caught(M):
    """Planted mistake: a walk that starts one unroll period after n/2 leaves a zero in a FIFO
    that the first complete window reads."""
    n, period = 1 << M, 1 << (M - 2)
    rng = np.random.default_rng(950 + M)
    x = rng.standard_normal(n + 5) + 1j * rng.standard_normal(n + 5)
    j0 = n // 2 + period
    first = np.array(late_walk(M, 0, 0, x, j0)[n - 1 - j0])
    assert np.abs(first - np.fft.fft(x[:n])).max() > 1e-3


@pytest.mark.parametrize("M,B", SPLITS)
def test_adjoint_schedule_gives_the_overlap_add_of_inverse_dfts(M, B):
    n = 1 << M
    N = n + 13
    P = N - n + 1
    rng = np.random.default_rng(100 + 10 * M + B)
    G = rng.standard_normal((P, n)) + 1j * rng.standard_normal((P, n))
    ref = np.zeros(N, complex)
    for q in range(P):
        ref[q:q + n] += np.fft.ifft(G[q]) * n  # sum_k G[q][k] w^{+jk}
    y = sum(adjoint_walk(M, B, c, G, N) for c in range(1 << B))
    np.testing.assert_allclose(y, ref, atol=1e-9)


@pytest.mark.parametrize("M,B", [(M, B) for (M, B) in SPLITS if M >= 1])
def test_adjoint_walk_ends_with_level_one_fifo_readout(M, B):
    """A chunk's walk ends with n - 1 steps past its last window (zero inputs).  In the last
    n/2 of them no window reaches the position through level 1 (its support is n/2 - 1 steps
    deep), so every thread's partial is its level-1 FIFO slot: the walk with that readout equals
    the full walk at every step.  Planted mistake: starting the readout one step earlier loses
    the level-1 node of the first readout step."""
    n = 1 << M
    nwin = n + 5
    rng = np.random.default_rng(1200 + 10 * M + B)
    G = rng.standard_normal((nwin, n)) + 1j * rng.standard_normal((nwin, n))
    cb = lambda c: c & ((1 << B) - 1)
    feeds = {c: [[G[j][cb(c) + (t << B)] for t in range(held(B, M))] if j < nwin else [0j] * held(B, M)
                 for j in range(nwin + n - 1)] for c in range(1 << B)}
    full = sum(np.array(adjoint_tree(M, B, c, feeds[c])) for c in range(1 << B))
    tail = sum(np.array(adjoint_tree(M, B, c, feeds[c], nwin + n // 2 - 1)) for c in range(1 << B))
    np.testing.assert_allclose(tail, full, atol=1e-12)
    early = sum(np.array(adjoint_tree(M, B, c, feeds[c], nwin + n // 2 - 2)) for c in range(1 << B))
    assert np.abs(early - full).max() > 1e-6


def ternary_tree(M, c, feeds, j0=0):
    """Thread c (< 3) of the ternary tree split by residue mod 3 (tree3_core.cuh) over the
    steps j = j0, j0 + 1, ..: feeds[j - j0] = (x at the window end p, x at p - s_1, x at p - 2 s_1),
    s_1 = 3^(M-1), values or lane arrays; returns its level-M nodes c + 3u, u < 3^(M-1)."""
    w27 = np.exp(-2j * np.pi * np.arange(27) / 27)

    def held_t(t):  # level-t nodes one thread holds
        return 1 if t <= 1 else 3 ** (t - 1)

    tw = {t: [(w27[(ip * (27 // 3 ** t)) % 27], w27[(2 * ip * (27 // 3 ** t)) % 27])
              for ip in (c + 3 * a for a in range(3 ** (t - 2)))] for t in range(2, M + 1)}
    # level t-1 is read s_t and 2 s_t steps back: a FIFO of 2 s_t slots
    fifos = {t: [[0j] * held_t(t - 1) for _ in range(2 * 3 ** (M - t))] for t in range(2, M + 1)}
    period = 2 * 3 ** (M - 2) if M >= 2 else 1
    w3 = np.exp(-2j * np.pi / 3)
    outs = []
    for i, (xp, xs1, xs2) in enumerate(feeds):
        J = (j0 + i) % period
        cur = [xs2 + w3 ** c * xs1 + w3 ** (2 * c) * xp]  # level 1, node c
        for t in range(2, M + 1):
            s = 3 ** (M - t)
            D = 2 * s
            hp = held_t(t - 1)
            nxt = [0j] * (3 * hp)
            for a in range(hp):
                a2 = cur[a]
                a1 = fifos[t][(J + s) % D][a]
                a0 = fifos[t][J % D][a]
                fifos[t][J % D][a] = a2
                b1 = tw[t][a][0] * a1
                b2 = tw[t][a][1] * a2
                for k in range(3):
                    nxt[a + k * hp] = a0 + w3 ** k * b1 + w3 ** (2 * k) * b2
            cur = nxt
        outs.append(cur)
    return outs


def mixed_split(n):
    """n = 3^B3 2^A2: (B3, A2), or None."""
    b = a = 0
    while n % 3 == 0:
        n //= 3
        b += 1
    while n % 2 == 0:
        n //= 2
        a += 1
    return (b, a) if n == 1 else None


def mixed_period(B3, A2):
    """The unroll period of SlidingTreeMixed: the depth of level 2's FIFO."""
    n = 3 ** B3 * 2 ** A2
    if B3 + A2 < 2:
        return 1
    r2 = 3 if B3 >= 2 else 2
    N2 = 3 * r2
    return (r2 - 1) * (n // N2)


def mixed_tree(B3, A2, c, feeds, j0=0, scale=1.0):
    """Thread c (< 3) of the mixed-radix tree split by residue mod 3 (tree3_core.cuh,
    SlidingTreeMixed: B3 radix-3 levels, then A2 radix-2 levels) over the steps j = j0, j0 + 1, ..:
    feeds[j - j0] = (x at p, x at p - s_1, x at p - 2 s_1), s_1 = n / 3; returns its level-L
    nodes c + 3u, u < n / 3.  FIFO depths, slots (step index modulo the depth, within the
    unroll period) and twiddle indices as the kernel has them; `scale` multiplies every output,
    folded into level 1 as the column kernel folds it."""
    n = 3 ** B3 * 2 ** A2
    L = B3 + A2
    om = np.exp(-2j * np.pi * np.arange(n) / n)

    def rad(t):
        return 3 if t <= B3 else 2

    def Nt(t):
        return 3 ** t if t <= B3 else 3 ** B3 * 2 ** (t - B3)

    def held(t):
        return 1 if t <= 1 else Nt(t) // 3

    def depth(t):
        return (rad(t) - 1) * (n // Nt(t))

    period = mixed_period(B3, A2)
    assert all(period % depth(t) == 0 for t in range(2, L + 1))
    s1 = n // 3
    tw1 = (scale * om[(c * s1) % n], scale * om[(2 * c * s1) % n])
    tw = {t: [[om[((c + 3 * a) * d * (n // Nt(t))) % n] for d in range(1, rad(t))]
              for a in range(held(t - 1))] for t in range(2, L + 1)}
    fifos = {t: [[0j] * held(t - 1) for _ in range(depth(t))] for t in range(2, L + 1)}
    w3 = np.exp(-2j * np.pi / 3)
    outs = []
    for i, (xp, xs1, xs2) in enumerate(feeds):
        J = (j0 + i) % period
        cur = [scale * xs2 + tw1[0] * xs1 + tw1[1] * xp]  # level 1, node c
        for t in range(2, L + 1):
            s, D, hp = n // Nt(t), depth(t), held(t - 1)
            nxt = [0j] * (rad(t) * hp)
            for a in range(hp):
                if rad(t) == 3:
                    a2, a1, a0 = cur[a], fifos[t][(J + s) % D][a], fifos[t][J % D][a]
                    fifos[t][J % D][a] = a2
                    b1, b2 = tw[t][a][0] * a1, tw[t][a][1] * a2
                    for k in range(3):
                        nxt[a + k * hp] = a0 + w3 ** k * b1 + w3 ** (2 * k) * b2
                else:
                    a1, a0 = cur[a], fifos[t][J % D][a]
                    fifos[t][J % D][a] = a1
                    b = tw[t][a][0] * a1
                    nxt[a], nxt[a + hp] = a0 + b, a0 - b
            cur = nxt
        outs.append(cur)
    return outs


MIXED_SHAPES = [(b, a) for b in (1, 2, 3) for a in range(0, 5) if 3 ** b * 2 ** a <= 64]


@pytest.mark.parametrize("B3,A2", MIXED_SHAPES)
def test_mixed_schedule_gives_every_windows_dft(B3, A2):
    n = 3 ** B3 * 2 ** A2
    rng = np.random.default_rng(700 + n)
    x = rng.standard_normal(n + 19) + 1j * rng.standard_normal(n + 19)
    s1 = n // 3
    feeds = [(x[p], x[p - s1] if p - s1 >= 0 else 0j, x[p - 2 * s1] if p - 2 * s1 >= 0 else 0j)
             for p in range(len(x))]
    for c in range(3):
        outs = mixed_tree(B3, A2, c, feeds)
        for p in range(n - 1, len(x)):
            ref = np.fft.fft(x[p - n + 1:p + 1])
            np.testing.assert_allclose(outs[p], ref[c::3], atol=1e-9)


def walk3_start(n):
    """First step of a ternary or mixed chunk's walk (row_tree3_kernel, col_tree3_kernel): level 1
    reads level 0 s_1 and 2 s_1 back from memory, and the FIFO depths of levels 1 .. L-1 add up
    to n - 1 - 2 s_1, so the output at step n - 1 needs level 1 from step 2 s_1 = 2n/3 on."""
    return 2 * (n // 3) if n % 3 == 0 else 0


@pytest.mark.parametrize("B3,A2", MIXED_SHAPES)
def test_mixed_walk_started_at_two_thirds_gives_every_windows_dft(B3, A2):
    n = 3 ** B3 * 2 ** A2
    s1, period, j0 = n // 3, mixed_period(B3, A2), walk3_start(n)
    assert j0 % period == 0
    rng = np.random.default_rng(760 + n)
    x = rng.standard_normal(n + 19) + 1j * rng.standard_normal(n + 19)
    feeds = [(x[p], x[p - s1], x[p - 2 * s1]) for p in range(j0, len(x))]
    for c in range(3):
        outs = mixed_tree(B3, A2, c, feeds, j0)
        for p in range(n - 1, len(x)):
            np.testing.assert_allclose(outs[p - j0], np.fft.fft(x[p - n + 1:p + 1])[c::3], atol=1e-9)
    # planted mistake: one period later, the first complete window reads a zeroed FIFO slot
    if B3 + A2 >= 2:
        late = [(x[p], x[p - s1], x[p - 2 * s1]) for p in range(j0 + period, len(x))]
        bad = max(np.abs(np.array(mixed_tree(B3, A2, c, late, j0 + period)[n - 1 - j0 - period]) -
                         np.fft.fft(x[:n])[c::3]).max() for c in range(3))
        assert bad > 1e-3


def ternary_walk(M, c, x):
    """Thread c's level-M nodes at every position p of x (zero before the array)."""
    s1 = 3 ** (M - 1)
    feeds = [(x[p], x[p - s1] if p - s1 >= 0 else 0j, x[p - 2 * s1] if p - 2 * s1 >= 0 else 0j)
             for p in range(len(x))]
    return ternary_tree(M, c, feeds)


@pytest.mark.parametrize("M", [1, 2, 3])
def test_ternary_schedule_gives_every_windows_dft(M):
    n = 3 ** M
    rng = np.random.default_rng(500 + M)
    x = rng.standard_normal(n + 17) + 1j * rng.standard_normal(n + 17)
    for c in range(3):
        outs = ternary_walk(M, c, x)
        ks = [c + 3 * u for u in range(3 ** (M - 1))]
        for p in range(n - 1, len(x)):
            ref = np.fft.fft(x[p - n + 1:p + 1])
            np.testing.assert_allclose(outs[p], ref[ks], atol=1e-9)


# ---------------------------------------------------------------------------------------------
# The two adjoint passes (adjoint_kernels.cuh, adjoint.cu) with their shared-memory staging,
# chunking and side-row fold, replayed block by block: every staged value a thread reads is
# checked against the operand it stands for, every output is written exactly once, and the
# result equals the explicit overlap-add of every window's inverse DFT (A^H G, scale 1).

def adj_col_B(M):
    return M if M < 1 else (1 if M <= 4 else M - 3)


def adj_row_B(M):
    return 3 if M >= 4 else (M if M < 2 else 2)


def adj_col_chunk(rows_out, n, requested):
    chunk = requested if requested > 0 else rows_out
    chunk = max(chunk, n - 1)
    return max(1, min(chunk, rows_out))


# adj_col_ring_kernel (adjoint_kernels.cuh): each step's runs of G are staged in a ring of
# ADJ_STAGES stages of adj_col_gs(M) steps by all 128 threads (16-byte cp.async pieces, 8-byte
# when G is not 16-byte aligned or n0 = 1); lanes hold the residue in their high bits; the
# host picks the staging layout (adj_col_layout, as in adjoint_kernels.cuh).

ADJ_STAGES = 2


def adj_col_gs(M):
    return 2 if M >= 4 else 32 >> M


def adj_col_conflicts(M, B, L):
    """Most distinct 8-byte words one half-warp's read maps to one bank pair (warp 0)."""
    mode, lw, gs, ks, slot = L
    R, CPW, n, W = 1 << B, 32 >> B, 1 << M, 1 << lw
    worst = 1
    for t in range(n // R):
        for h in range(2):
            per_bank = {}
            for l in range(16):
                lane = 16 * h + l
                c, ch = lane // CPW, lane % CPW
                a = (ch >> lw) * gs + (ch & (W - 1)) + (c + R * t) * ks
                per_bank.setdefault(a & 15, set()).add(a)
            worst = max(worst, max(len(v) for v in per_bank.values()))
    return worst


def adj_col_layout(M, B, m1):
    """(mode, lw, gs, ks, slot): fewest conflicts, then fewest runs per step, then smallest
    slot; padded q1 groups (mode 1) only when one run would read with more than 2-way conflicts."""
    n, n1, CH = 1 << M, 1 << m1, 128 >> B
    best, key = None, None

    def consider(L, runs):  # strict improvement only: the first of equals wins, as in the host code
        nonlocal best, key
        k = (adj_col_conflicts(M, B, L), runs, L[4])
        if key is None or k < key:
            best, key = L, k
    if n1 <= CH:
        consider((0, m1, n * n1, n1, CH * n), 1)
    if n1 < CH and key[0] > 2:
        for pad in range(2, 31, 2):
            consider((1, m1, n * n1 + pad, n1, (CH >> m1) * (n * n1 + pad)), CH >> m1)
    if n1 >= CH:
        lw = CH.bit_length() - 1
        for pad in range(0, 31, 2):
            consider((2, lw, 0, CH + pad, n * (CH + pad)), n)
    return best


def emulate_adj_col_ring(G, n0, n1, chunk_req, q16=True):
    """adj_col_ring_kernel over its grid, then adj_fold_kernel: the ring, layout and lanes
    above, filled by all 128 threads with 16-byte (q16) or 8-byte cp.async pieces.  Every
    piece is checked to be aligned to its size at both ends, to land inside its step's part of
    its ring slot and to read inside G; the pieces of a step cover its runs exactly once; a
    slot is refilled (stage g + ADJ_STAGES - 1, after the block barrier of stage g) only once
    the stage in it was read; every staged value a thread reads is the G value it stands for."""
    rows_out, P1 = G.shape[0], G.shape[1]
    M, m1 = n0.bit_length() - 1, n1.bit_length() - 1
    B = adj_col_B(M)
    R, n, CH, CPW = 1 << B, n0, 128 >> B, 32 >> B
    GS, NS = adj_col_gs(M), ADJ_STAGES
    mode, lw, gs, ks, slot = adj_col_layout(M, B, m1)
    q16 = q16 and m1 >= 1  # channel pairs need n1 >= 2
    assert 128 + 8 * NS * GS * slot <= 227 * 1024
    nch = P1 * n1
    Gf = G.reshape(-1)
    grow = nch * n
    chunk = adj_col_chunk(rows_out, n, chunk_req)
    nchunks = -(-rows_out // chunk)
    gz = np.full((rows_out + n - 1) * nch, np.nan, complex)
    side = np.full(max(nchunks - 1, 0) * (n - 1) * nch, np.nan, complex)
    tid = np.arange(128)
    warp, lane = tid >> 5, tid & 31
    c_of, chl_of = lane // CPW, warp * CPW + (lane & (CPW - 1))
    tbase = (chl_of >> lw) * gs + (chl_of & ((1 << lw) - 1)) + c_of * ks
    tstride = R * ks
    for bx in range(-(-nch // CH)):
        ch0 = bx * CH
        chv = min(CH, nch - ch0)
        assert chv % min(n1, CH) == 0
        gbase = (ch0 >> m1) * n * n1 + (ch0 & (n1 - 1))
        runs = 1 if mode == 0 else (chv >> m1 if mode == 1 else n)
        run_vals = chv * n if mode == 0 else (n * n1 if mode == 1 else CH)
        # copies: thread i owns channel pair cl (one channel with 8-byte pieces) and the
        # k0 = k0f + KS t of every step
        qv = 2 if q16 else 1
        NP = CH // qv
        KS = 128 // NP
        for by in range(nchunks):
            qa = by * chunk
            qb = min(qa + chunk, rows_out)
            last = qb == rows_out
            p_hi, nwin = qb + n - 2, qb - qa
            steps = nwin + n - 1
            ngroups = -(-nwin // GS)
            ring = np.full(NS * GS * slot, np.nan, complex)
            in_slot = [None] * NS
            read = set()

            def piece(src, dst, vals, step0):
                assert (8 * src) % (8 * vals) == 0 and (128 + 8 * dst) % (8 * vals) == 0
                assert step0 <= dst and dst + vals <= step0 + slot, "piece leaves its step's slot"
                assert 0 <= src and src + vals <= Gf.size, "piece reads outside G"
                assert np.isnan(ring[dst:dst + vals]).all(), "piece written twice in one stage"
                ring[dst:dst + vals] = Gf[src:src + vals]

            def fetch(g):
                if g >= ngroups:
                    return
                sl = g % NS
                assert in_slot[sl] is None or in_slot[sl] in read, "slot refilled before it was read"
                in_slot[sl] = g
                ring[sl * GS * slot:(sl + 1) * GS * slot] = np.nan
                j0 = g * GS
                cnt = min(GS, nwin - j0)
                dst0 = sl * GS * slot
                for t in range(128):
                    cl, k0f = (t % NP) * qv, t // NP
                    if not (cl < chv and k0f < n):
                        continue
                    gsrc = gbase + (cl >> m1) * n * n1 + (cl & (n1 - 1)) + k0f * n1
                    sdst = (cl >> lw) * gs + (cl & ((1 << lw) - 1)) + k0f * ks
                    for st in range(cnt):
                        step0 = dst0 + st * slot
                        src = gsrc + (qb - 1 - (j0 + st)) * grow
                        for u in range(max(1, -(-(n - k0f) // KS))):
                            if k0f + KS * u >= n:
                                break
                            piece(src + u * KS * n1, step0 + sdst + u * KS * ks, qv, step0)
                for st in range(cnt):  # the pieces cover exactly each step's runs
                    step0 = dst0 + st * slot
                    assert (~np.isnan(ring[step0:step0 + slot])).sum() == runs * run_vals

            for g in range(NS - 1):
                fetch(g)
            feeds = {c: [] for c in range(R)}
            for j in range(steps):
                g = j // GS
                if j % GS == 0:
                    if g >= 1:
                        read.add(g - 1)  # the block barrier: every thread has read stage g - 1
                    fetch(g + NS - 1)
                if j < nwin:
                    assert in_slot[g % NS] == g
                    base = (g % NS) * GS * slot + (j % GS) * slot
                    addrs = base + tbase[:, None] + tstride * np.arange(held(B, M))[None, :]
                    assert (addrs >= base).all() and (addrs < base + slot).all()
                    u = ring[addrs]
                    chg = ch0 + chl_of
                    ok = chg < nch
                    chc = np.minimum(chg, nch - 1)
                    k0 = c_of[:, None] + R * np.arange(held(B, M))[None, :]
                    want = G[qb - 1 - j, (chc >> m1)[:, None], k0, (chc & (n1 - 1))[:, None]]
                    np.testing.assert_array_equal(u[ok], want[ok])
                else:
                    u = np.zeros((128, held(B, M)), complex)
                for c in range(R):
                    sel = np.nonzero(c_of == c)[0]
                    feeds[c].append([u[sel, t] for t in range(held(B, M))])
            part = np.zeros((steps, 128), complex)
            # for n0 = 16 and 64 the last n/2 steps read the level-1 FIFO alone (no window
            # reaches them through level 1)
            tail = nwin + n // 2 - 1 if M in (4, 6) else None
            for c in range(R):
                part[:, np.nonzero(c_of == c)[0]] = np.array(adjoint_tree(M, B, c, feeds[c], tail))
            off = CPW
            while off < 32:
                part = part + part[:, (warp << 5) | (lane ^ off)]
                off <<= 1
            y = np.zeros((steps, CH), complex)
            y[:, chl_of[c_of == 0]] = part[:, c_of == 0]
            for j in range(steps):
                r = p_hi - j
                for chl in range(CH):
                    ch = ch0 + chl
                    if ch >= nch:
                        continue
                    if r >= qb and not last:
                        i = by * (n - 1) * nch + (r - qb) * nch + ch
                        assert np.isnan(side[i]), "side value written twice"
                        side[i] = y[j, chl]
                    else:
                        assert np.isnan(gz[r * nch + ch]), "gz value written twice"
                        gz[r * nch + ch] = y[j, chl]
    per_row = (n - 1) * nch
    for i in range(side.size):
        b = i // per_row + 1
        gz[b * chunk * nch + (i - (b - 1) * per_row)] += side[i]
    assert not np.isnan(gz).any(), "a gz value was never written"
    return gz.reshape(rows_out + n - 1, nch)


RING_CASES = [(1, 64), (1, 1), (2, 64), (2, 1), (4, 16), (8, 8), (16, 16), (16, 4), (16, 1),
              (32, 32), (32, 2), (64, 16), (64, 64), (64, 1)]


@pytest.mark.parametrize("n0,n1", RING_CASES)
def test_adj_col_ring_staging_replayed(n0, n1):
    rows_out, P1 = 19, 5
    N0, N1 = rows_out + n0 - 1, P1 + n1 - 1
    rng = np.random.default_rng(13 * n0 + n1)
    G = rng.standard_normal((rows_out, P1, n0, n1)) + 1j * rng.standard_normal((rows_out, P1, n0, n1))
    want = np.zeros((rows_out + n0 - 1, P1, n1), complex)
    for q0 in range(rows_out):
        want[q0:q0 + n0] += np.fft.ifft(G[q0], axis=1).transpose(1, 0, 2) * n0
    want = want.reshape(rows_out + n0 - 1, -1)
    for q16 in (True, False):  # G 16-byte aligned, or not
        for col_chunk in (0, max(n0 - 1, 1), 7):
            gz = emulate_adj_col_ring(G, n0, n1, col_chunk, q16)
            np.testing.assert_allclose(gz, want, atol=1e-9)
    gx = emulate_adj_row(want, N1, n1, N1)
    np.testing.assert_allclose(gx, overlap_add_of_inverse_dfts(G, N0, N1), atol=1e-8)


@pytest.mark.parametrize("M", range(0, 7))
def test_adj_col_layouts_stay_aligned_and_inside_the_ring(M):
    """For every window side 2^M >= 2 and every n1 = 1..64, the staging layout the host picks
    keeps runs 16-byte aligned, fits the ring in shared memory, and reads free of bank
    conflicts in the cases the workloads use (16x16, 32x32, 64x16 windows)."""
    B = adj_col_B(M)
    CH = 128 >> B
    for m1 in range(0, 7):
        mode, lw, gs, ks, slot = adj_col_layout(M, B, m1)
        # runs start 16-byte aligned: steps (slot), q1 groups (gs, mode 1), k0 runs (ks, mode 2)
        assert slot % 2 == 0 and (mode != 1 or gs % 2 == 0) and (mode != 2 or ks % 2 == 0)
        assert 128 + 8 * ADJ_STAGES * adj_col_gs(M) * slot <= 227 * 1024
        if mode == 2:
            assert (1 << m1) >= CH
        else:
            assert (1 << m1) <= CH
    assert adj_col_conflicts(4, 1, adj_col_layout(4, 1, 4)) == 1
    assert adj_col_conflicts(5, 2, adj_col_layout(5, 2, 5)) == 1
    assert adj_col_conflicts(6, 3, adj_col_layout(6, 3, 4)) == 1
    assert adj_col_layout(4, 1, 4)[0] == 0  # 16x16: one contiguous run per step


def emulate_adj_row(gz, N1, n1, chunk):
    """adj_row_kernel over its grid (row blocks x column chunks) with its cp.async staging.
    gz: (zrows, P1 * n1).  Returns gx (zrows, N1), complex (the real path stores .real)."""
    zrows = gz.shape[0]
    M = n1.bit_length() - 1
    B = adj_row_B(M)
    R, n = 1 << B, n1
    kRows = 128 >> B
    GS = min(16, max(1, 2048 // (kRows * n)))
    kRow = GS * n + R
    kPiece = 2 if n >= 2 else 1
    kPerRow = GS * n // kPiece
    assert kPerRow <= 128 and 128 % kPerRow == 0 and (kPiece == 1 or kRow % 2 == 0)
    kRowStep = 128 // kPerRow
    kCopies = kRows // kRowStep
    P1 = N1 - n + 1
    rowlen = P1 * n
    gzf = gz.reshape(-1)
    chunk = min(chunk, N1)
    gx = np.full((zrows, N1), np.nan, complex)
    for bx in range(-(-zrows // kRows)):
        row0 = bx * kRows
        for by in range(-(-N1 // chunk)):
            pa = by * chunk
            pb = min(pa + chunk, N1)
            p_hi = min(pb + n - 2, N1 - 1)
            steps = p_hi - pa + 1
            q1_top = p_hi - (n - 1)
            sz = np.full(2 * kRows * kRow, np.nan, complex)

            def fetch(j0, b):
                q1lo = q1_top - j0 - (GS - 1)
                for tid in range(128):
                    off_f = (tid % kPerRow) * kPiece
                    rl_f = tid // kPerRow
                    q = q1lo + off_f // n
                    qok = 0 <= q < P1
                    goff = q1lo * n + off_f
                    dst = (b * kRows + rl_f) * kRow + off_f
                    for t in range(kCopies):
                        r = row0 + rl_f + t * kRowStep
                        ok = qok and r < zrows
                        d = dst + t * kRowStep * kRow
                        if kPiece == 2:  # 16-byte copies: both ends 16-byte aligned
                            assert d % 2 == 0 and (not ok or (r * rowlen + goff) % 2 == 0)
                        for e in range(kPiece):
                            sz[d + e] = gzf[r * rowlen + goff + e] if ok else 0

            fetch(0, 0)
            lanes = np.arange(kRows)
            rows = row0 + lanes
            feeds = [[] for _ in range(R)]
            for j in range(steps):
                if j % GS == 0 and j + GS < steps:
                    fetch(j + GS, (j // GS + 1) & 1)
                q1 = q1_top - j
                for c in range(R):
                    base = (((j // GS) & 1) * kRows + lanes) * kRow + (GS - 1 - j % GS) * n + c
                    u = [sz[base + t * R] for t in range(held(B, M))]
                    for t, ut in enumerate(u):  # gz[row][q1][k1 = c + R t], 0 outside
                        valid = (rows < zrows) & (0 <= q1 < P1)
                        want = np.where(valid, gz[np.minimum(rows, zrows - 1),
                                                  min(max(q1, 0), P1 - 1) * n + c + R * t], 0)
                        np.testing.assert_array_equal(ut, want)
                    feeds[c].append(u)
            y = sum(np.array(adjoint_tree(M, B, c, feeds[c])) for c in range(R))  # (steps, kRows)
            for j in range(steps):
                p1 = p_hi - j
                if p1 >= pb:
                    continue
                for rl in range(kRows):
                    if row0 + rl < zrows:
                        assert np.isnan(gx[row0 + rl, p1]), "gx value written twice"
                        gx[row0 + rl, p1] = y[j, rl]
    assert not np.isnan(gx).any(), "a gx value was never written"
    return gx


def overlap_add_of_inverse_dfts(G, N0, N1):
    """A^H G at scale 1: every window's sum_k G[q][k] w^{+j.k} added at its position."""
    P0, P1, n0, n1 = G.shape
    out = np.zeros((N0, N1), complex)
    for q0 in range(P0):
        for q1 in range(P1):
            out[q0:q0 + n0, q1:q1 + n1] += np.fft.ifft2(G[q0, q1]) * (n0 * n1)
    return out


ADJ_CASES = [(1, 64), (2, 32), (4, 16), (8, 8), (16, 4), (32, 2), (64, 1)]


@pytest.mark.parametrize("n0,n1", ADJ_CASES)
def test_adjoint_passes_with_staging_chunks_and_fold(n0, n1):
    rows_out, P1 = 21, 5
    N0, N1 = rows_out + n0 - 1, P1 + n1 - 1
    rng = np.random.default_rng(7 * n0 + n1)
    G = rng.standard_normal((rows_out, P1, n0, n1)) + 1j * rng.standard_normal((rows_out, P1, n0, n1))
    ref = overlap_add_of_inverse_dfts(G, N0, N1)
    ref_z = None
    for col_chunk in (0, 1, 5, 8):  # one chunk; the n0 - 1 minimum; ragged chunks
        gz = emulate_adj_col_ring(G, n0, n1, col_chunk)
        if ref_z is None:
            ref_z = gz
        else:
            np.testing.assert_allclose(gz, ref_z, atol=1e-9)
    for row_chunk in (N1, n1, 3):  # one chunk; the n1 minimum; chunks shorter than a window
        gx = emulate_adj_row(ref_z, N1, n1, row_chunk)
        np.testing.assert_allclose(gx, ref, atol=1e-8)


# ---------------------------------------------------------------------------------------------
# The forward passes (tree_kernels.cuh) replayed block by block: row_tile (two-pass form, row
# levels into z), col_tile_impl with its shared-memory ring of z rows filled one step group
# ahead by either stage -- ZStageLoad (cp.async copies of z, with the n0/2 padding rows in
# front of z that only incomplete border trees read) or ZStageRowDft (the fused form's row
# levels by warp shuffles) -- and the scaled stores of every window's coefficients.

def tg_period(M):
    return 1 << (M - 2) if M >= 2 else 1


def col_group(M):
    return max(tg_period(M), 8)


def col_ring_rows(M, ahead=1):
    look = (1 << (M - 1)) if M >= 1 else 0
    if ahead >= 2:  # TMA: the look-back rounded up to whole groups
        look = -(-look // col_group(M)) * col_group(M)
    need = look + (1 + ahead) * col_group(M)
    r = 1
    while r < need:
        r <<= 1
    return r


def emulate_row_pass(x, n1, B, chunk, pad):
    """row_tree_kernel over (row blocks of 128 >> B rows) x (chunks of window columns): returns
    z with `pad` padding rows (NaN: never written by the row pass) in front."""
    rows, N1 = x.shape
    M = n1.bit_length() - 1
    R, P1 = 1 << B, N1 - n1 + 1
    z = np.full((pad + rows, P1 * n1), np.nan, complex)
    for qa in range(0, P1, chunk):
        qb = min(qa + chunk, P1)
        steps = (qb - qa) + (n1 - 1)
        assert qb + n1 - 2 <= N1 - 1  # last column read
        j0 = row_walk_start(M)
        assert qa + j0 - n1 // 2 >= qa  # no look-back before the chunk's first window
        feeds = [(x[:, qa + j], x[:, max(qa + j - n1 // 2, 0)] if M >= 1 else 0j) for j in range(j0, steps)]
        for c in range(R):
            outs = forward_tree(M, B, c, feeds, j0)
            for j in range(n1 - 1, steps):
                q1 = qa + j - (n1 - 1)
                for t, o in enumerate(outs[j - j0]):
                    col = q1 * n1 + c + (t << B)
                    assert np.isnan(z[pad:, col]).all(), "z value written twice"
                    z[pad:, col] = o
    return z


class LoadStage:
    """ZStageLoad: ring rows from z (band row rr is z row pad + rr), zero for channels past nch."""

    def __init__(self, z, pad, nch):
        self.z, self.pad, self.nch = z, pad, nch

    def fetch(self, ring, r_lo, r_hi, CH, ch0, RD):
        for rr in range(r_lo, r_hi):
            assert 0 <= self.pad + rr < self.z.shape[0]  # every copy source inside z
            cc = np.arange(CH)
            ok = ch0 + cc < self.nch
            ring[(rr & (RD - 1)) * CH + cc] = np.where(ok, self.z[self.pad + rr, np.minimum(ch0 + cc, self.nch - 1)], 0)
        return {rr & (RD - 1) for rr in range(r_lo, r_hi)}

    def check(self, got, zr, ch):  # a copy: bit for bit (NaN for padding rows)
        ok = ch < self.nch
        np.testing.assert_array_equal(got, np.where(ok, self.z[self.pad + zr, np.minimum(ch, self.nch - 1)], 0))

    def wait(self):
        pass


class TmaStage(LoadStage):
    """ZStageTma: thread 0 loads each ring row as one TMA box of CH channels x 1 row of the
    2D tensor [pad + rows][nch] (8-byte elements; zero past nch and past the last row), the
    loads of fetch f completing on mbarrier f mod 3 (the tile runs two groups ahead); wait()
    completes the oldest fetch in flight.  Checks the TMA rules (inner coordinate x 8 bytes a
    multiple of 16, the box's inner extent a multiple of 16 bytes and at most 256 elements, a
    non-negative row) and that a barrier is never re-armed before its phase was waited for."""
    AHEAD = 2
    NB = AHEAD + 1

    def __init__(self, z, pad, nch):
        super().__init__(z, pad, nch)
        self.k, self.w = 0, 0
        self.armed, self.phase = [False] * self.NB, [0] * self.NB

    def __call__(self, kP):
        self.kP = kP
        return self

    def fetch(self, ring, r_lo, r_hi, CH, ch0, RD):
        kP = self.kP
        assert (8 * ch0) % 16 == 0 and (8 * CH) % 16 == 0 and CH <= 256 and kP <= 256
        assert RD % kP == 0
        b = self.k % self.NB
        assert not self.armed[b], "barrier re-armed before its phase was waited for"
        self.armed[b] = True
        g0, g1 = r_lo // kP, -(-r_hi // kP)  # whole groups (floor, ceil)
        rows = set()
        for g in range(g0, g1):  # one box of CH channels x kP rows, zero outside z
            dst = ((g * kP) & (RD - 1)) * CH
            assert 0 <= dst and dst + kP * CH <= RD * CH  # inside the ring, no wrap
            for i in range(kP):
                y = self.pad + g * kP + i
                cc = ch0 + np.arange(CH)
                ok = (cc < self.nch) & (0 <= y) & (y < self.z.shape[0])
                ring[dst + i * CH:dst + (i + 1) * CH] = np.where(
                    ok, self.z[min(max(y, 0), self.z.shape[0] - 1), np.minimum(cc, self.nch - 1)], 0)
                rows.add((g * kP + i) & (RD - 1))
        self.k += 1
        return rows

    def wait(self):
        if self.w >= self.k:
            return
        f = self.w
        self.w += 1
        b = f % self.NB
        assert self.armed[b] and self.phase[b] == f // self.NB
        self.armed[b] = False
        self.phase[b] += 1


class RowDftStage:
    """ZStageRowDft: each warp computes the n1-point DFTs of 32 channels of one input row by
    shuffles; lane (i, d) holds node i at position p - d."""

    def __init__(self, x, n1):
        self.x, self.n1 = x, n1
        self.M1 = n1.bit_length() - 1
        self.zrows, N1 = x.shape
        self.P1 = N1 - n1 + 1
        self.om64 = np.exp(-2j * np.pi * np.arange(64) / 64)

    def row_dft(self, r, ch0):
        M1, n1 = self.M1, self.n1
        lane = np.arange(32)
        l = lane & (n1 - 1)
        base = lane - l
        q1 = (ch0 >> M1) + (lane >> M1)
        v = np.zeros(32, complex)
        valid = (0 <= r < self.zrows) & (q1 < self.P1)
        col = q1 + n1 - 1 - l
        if valid.any():
            assert col[valid].max() < self.x.shape[1]
            v[valid] = self.x[r, col[valid]]
        for t in range(1, M1 + 1):
            i, d = l >> (M1 - t), l & ((1 << (M1 - t)) - 1)
            src = base + ((i & ((1 << (t - 1)) - 1)) << (M1 - t + 1)) + d
            assert ((src >= base) & (src + (1 << (M1 - t)) < base + n1)).all()  # own window's lanes
            v = v[src + (1 << (M1 - t))] + self.om64[i << (6 - t)] * v[src]
        return v

    def row_dft64(self, r, q1):
        """n1 = 64: one warp evaluates the whole window column q1; value e of lane L is flat
        index l = 2 L + e of the (i, d) layout, so levels 1..5 take both operands from register
        e of the source lanes, and level 6 (nodes L and 32 + L) from the lane's own two
        registers.  Returns (lo, hi) per lane."""
        lane = np.arange(32)
        v = np.zeros((2, 32), complex)
        if 0 <= r < self.zrows and q1 < self.P1:
            p = q1 + 63
            v[0] = self.x[r, p - 2 * lane]
            v[1] = self.x[r, p - 2 * lane - 1]
        for t in range(1, 6):
            nv = np.zeros_like(v)
            for e in range(2):
                l = 2 * lane + e
                i, d = l >> (6 - t), l & ((1 << (6 - t)) - 1)
                assert ((d & 1) == e).all()  # an operand's register is the value's own
                lc = ((i & ((1 << (t - 1)) - 1)) << (7 - t)) | d
                ls = lc + (1 << (6 - t))
                assert ((lc & 1) == e).all() and ((ls & 1) == e).all()
                assert ((lc >> 1) + (1 << (5 - t)) == ls >> 1).all()
                nv[e] = v[e][ls >> 1] + self.om64[i << (6 - t)] * v[e][lc >> 1]
            v = nv
        return v[1] + self.om64[lane] * v[0], v[1] + self.om64[32 + lane] * v[0]

    def fetch(self, ring, r_lo, r_hi, CH, ch0, RD):
        for rr in range(r_lo, r_hi):
            if self.n1 == 64:  # whole window columns
                assert CH % 64 == 0 and ch0 % 64 == 0
                for wc in range(CH >> 6):
                    lo, hi = self.row_dft64(rr, (ch0 >> 6) + wc)
                    base = (rr & (RD - 1)) * CH + wc * 64
                    ring[base + np.arange(32)] = lo
                    ring[base + 32 + np.arange(32)] = hi
            else:
                for g in range(CH >> 5):
                    ring[(rr & (RD - 1)) * CH + g * 32 + np.arange(32)] = self.row_dft(rr, ch0 + g * 32)
        return {rr & (RD - 1) for rr in range(r_lo, r_hi)}

    def check(self, got, zr, ch):  # the n1-point DFT of the window's row (0 outside x)
        q1, k1 = ch >> self.M1, ch & (self.n1 - 1)
        want = np.zeros(len(ch), complex)
        if 0 <= zr < self.zrows:
            for i in np.nonzero(q1 < self.P1)[0]:
                want[i] = np.fft.fft(self.x[zr, q1[i]:q1[i] + self.n1])[k1[i]]
        np.testing.assert_allclose(got, want, atol=1e-12)

    def wait(self):
        pass


def emulate_col_pass(stage, n0, B, groups, m1, P1, rows_out, chunk, scale):
    """col_tile_impl over (blocks of 32 * groups channels) x (chunks of window rows); returns
    the output (rows_out, P1, n0, n1), every value written exactly once."""
    M = n0.bit_length() - 1
    R, n, n1 = 1 << B, n0, 1 << m1
    AHEAD = getattr(stage, "AHEAD", 1)  # step groups fetched ahead of the one computed
    kP, kH, RD = col_group(M), n0 // 2, col_ring_rows(M, AHEAD)
    assert kP % tg_period(M) == 0 and RD >= kH + (AHEAD + 1) * kP
    if isinstance(stage, TmaStage):
        stage = stage(kP)
        assert chunk % kP == 0  # launch_col_tree takes TMA only for chunks of whole groups
    CH, nch = 32 * groups, P1 << m1
    out = np.full((rows_out, P1, n0, n1), np.nan, complex)
    my = np.arange(CH)
    for ch0 in range(0, nch, CH):
        ch = ch0 + my
        active = ch < nch
        for qa in range(0, rows_out, chunk):
            qb = min(qa + chunk, rows_out)
            steps, zr_end = (qb - qa) + (n - 1), qb + n - 1
            j0 = col_walk_start(M, isinstance(stage, TmaStage))
            ring = np.full(RD * CH, np.nan, complex)
            stage.fetch(ring, qa + j0 - kH, min(qa + j0 + kP, zr_end), CH, ch0, RD)
            inflight = []  # ring rows of each fetch still in flight, oldest first
            for a in range(1, AHEAD):
                if j0 + a * kP < steps:
                    lo, hi = qa + j0 + a * kP, min(qa + j0 + (a + 1) * kP, zr_end)
                    inflight.append(stage.fetch(ring, lo, hi, CH, ch0, RD))
            stage.wait()
            feeds = []
            for jb in range(j0, steps, kP):
                if jb + AHEAD * kP < steps:
                    lo, hi = qa + jb + AHEAD * kP, min(qa + jb + (AHEAD + 1) * kP, zr_end)
                    inflight.append(stage.fetch(ring, lo, hi, CH, ch0, RD))
                busy = set().union(*inflight) if inflight else set()
                for j in range(jb, min(jb + kP, steps)):
                    zr = qa + j
                    # no row this group reads is one the fetch in flight writes
                    assert (zr & (RD - 1)) not in busy and ((zr - kH) & (RD - 1)) not in busy
                    assert j0 < kH or zr - kH >= qa  # a walk from n/2 reads no padding row
                    xp = ring[(zr & (RD - 1)) * CH + my]
                    xs = ring[((zr - kH) & (RD - 1)) * CH + my] if M >= 1 else 0j
                    stage.check(xp, zr, ch)
                    if M >= 1:
                        stage.check(xs, zr - kH, ch)
                    feeds.append((xp, xs))
                stage.wait()
                if inflight:
                    inflight.pop(0)
            for c in range(R):
                outs = forward_tree(M, B, c, feeds, j0)
                for j in range(n - 1, steps):
                    q0 = qa + j - (n - 1)
                    for t, o in enumerate(outs[j - j0]):
                        k0 = c + R * t
                        for i in np.nonzero(active)[0]:
                            q1, k1 = ch[i] >> m1, ch[i] & (n1 - 1)
                            assert np.isnan(out[q0, q1, k0, k1]), "output written twice"
                            out[q0, q1, k0, k1] = scale * o[i]
    assert not np.isnan(out).any(), "an output was never written"
    return out


def every_window_dft(x, n0, n1, scale):
    N0, N1 = x.shape
    P0, P1 = N0 - n0 + 1, N1 - n1 + 1
    ref = np.empty((P0, P1, n0, n1), complex)
    for q0 in range(P0):
        for q1 in range(P1):
            ref[q0, q1] = np.fft.fft2(x[q0:q0 + n0, q1:q1 + n1]) * scale
    return ref


def col_split(m0):
    return 3 if m0 >= 6 else min(m0, 2)


FWD_CASES = [  # (n0, n1, rows_out, P1, groups, column chunks)
    (1, 8, 5, 7, 1, (5, 2)),
    (2, 4, 6, 9, 2, (6, 4)),
    (4, 16, 7, 3, 1, (7, 3)),
    (8, 2, 9, 19, 2, (9, 4)),
    (16, 1, 11, 37, 1, (11, 5)),
    (32, 4, 6, 10, 1, (6, 4)),
    (64, 1, 5, 33, 1, (5, 2)),
]


TMA_CASES = [  # chunks of whole step groups (8 rows; 16 for n0 = 64), ragged last chunks
    (1, 8, 21, 7, 1, (8, 16)),
    (4, 16, 19, 3, 1, (8,)),
    (8, 2, 25, 19, 2, (8, 16)),
    (16, 4, 20, 9, 1, (8, 16)),
    (32, 4, 18, 10, 1, (8,)),
    (64, 2, 40, 6, 1, (16, 32)),
]


@pytest.mark.parametrize("n0,n1,rows_out,P1,groups,chunks", TMA_CASES)
def test_two_pass_forward_with_tma_boxes(n0, n1, rows_out, P1, groups, chunks):
    rng = np.random.default_rng(3000 + n0 * 64 + n1)
    N0, N1 = rows_out + n0 - 1, P1 + n1 - 1
    x = rng.standard_normal((N0, N1)) + 1j * rng.standard_normal((N0, N1))
    ref = every_window_dft(x, n0, n1, 1.0)
    m1 = n1.bit_length() - 1
    pad = n0 // 2
    z = emulate_row_pass(x, n1, min(m1, 3), P1, pad)
    for chunk in chunks:
        out = emulate_col_pass(TmaStage(z, pad, P1 * n1), n0, col_split(n0.bit_length() - 1),
                               groups, m1, P1, rows_out, chunk, 1.0)
        np.testing.assert_allclose(out, ref, atol=1e-9)


@pytest.mark.parametrize("n0,n1,rows_out,P1,groups,chunks", FWD_CASES)
def test_two_pass_forward_with_ring_staging(n0, n1, rows_out, P1, groups, chunks):
    rng = np.random.default_rng(1000 + n0 * 64 + n1)
    N0, N1 = rows_out + n0 - 1, P1 + n1 - 1
    x = rng.standard_normal((N0, N1)) + 1j * rng.standard_normal((N0, N1))
    scale = 1 / np.sqrt(n0 * n1)
    ref = every_window_dft(x, n0, n1, scale)
    m1 = n1.bit_length() - 1
    pad = n0 // 2
    for row_chunk in (P1, max(1, n1 // 2)):
        z = emulate_row_pass(x, n1, min(m1, 3), row_chunk, pad)
        for chunk in chunks:
            for Stage in (LoadStage, TmaStage):  # cp.async copies, or TMA boxes
                # (TMA: z rows of an even number of channels, chunks of whole step groups)
                if Stage is TmaStage and ((P1 * n1) % 2 or chunk % col_group(n0.bit_length() - 1)):
                    continue
                out = emulate_col_pass(Stage(z, pad, P1 * n1), n0, col_split(n0.bit_length() - 1),
                                       groups, m1, P1, rows_out, chunk, scale)
                np.testing.assert_allclose(out, ref, atol=1e-9)


FUSED64_CASES = [(16, 64, 7, 5, 1, (7, 3)), (1, 64, 4, 6, 2, (4, 3)), (32, 64, 5, 3, 2, (5, 2))]


@pytest.mark.parametrize("n0,n1,rows_out,P1,groups,chunks",
                         [c for c in FWD_CASES if c[1] <= 32] + FUSED64_CASES)
def test_fused_forward_with_row_dfts_by_shuffles(n0, n1, rows_out, P1, groups, chunks):
    rng = np.random.default_rng(2000 + n0 * 64 + n1)
    N0, N1 = rows_out + n0 - 1, P1 + n1 - 1
    x = rng.standard_normal((N0, N1))
    ref = every_window_dft(x, n0, n1, 1.0)
    m1 = n1.bit_length() - 1
    if n1 == 64:  # launch_fused_tree: tiles of whole window columns
        groups = max(2, groups & ~1)
    for chunk in chunks:
        out = emulate_col_pass(RowDftStage(x, n1), n0, col_split(n0.bit_length() - 1), groups, m1,
                               P1, rows_out, chunk, 1.0)
        np.testing.assert_allclose(out, ref, atol=1e-9)


# ---------------------------------------------------------------------------------------------
# The ternary passes (tree3.cu) replayed block by block: row_tree3_kernel with its output
# stage [row][step][k1] written back in runs, and col_tree3_kernel with its ring of z rows
# (look-backs s_1 and 2 s_1 rows up, 2 n0 / 3 padding rows in front of z) and, when n1 is not
# a multiple of 4, its double-buffered output stage copied out by consecutive threads.

def row3_unr(period):
    return 6 if period <= 6 and 6 % period == 0 else (8 if period <= 8 and 8 % period == 0 else 12)


def col3_group(period):
    return 8 if period <= 8 and 8 % period == 0 else (6 if period == 6 else 12)


def tree3_outs(n, feeds, j0=0, scale=1.0):
    """Every residue thread's outputs from step j0 on, scaled (the mixed tree; n = 1: the data
    itself)."""
    B3, A2 = mixed_split(n)
    if B3 == 0:
        return {0: [[scale * f[0]] for f in feeds]}
    return {c: mixed_tree(B3, A2, c, feeds, j0, scale) for c in range(3)}


def emulate_row_pass3(x, n1, chunk, pad):
    rows, N1 = x.shape
    B3, A2 = mixed_split(n1)
    n, R, OUT = n1, (3 if B3 >= 1 else 1), (n1 // 3 if B3 >= 1 else 1)
    S1 = n1 // 3 if B3 >= 1 else 0
    UNR = row3_unr(mixed_period(B3, A2) if B3 >= 1 else 1)
    assert B3 == 0 or UNR % mixed_period(B3, A2) == 0
    P1 = N1 - n + 1
    zrow = P1 * n
    z = np.full((pad + rows) * zrow, np.nan, complex)
    written = np.zeros(z.shape, int)
    for row0 in range(0, rows, 32):
        nrows = min(32, rows - row0)
        lanes = np.arange(32)
        xr = x[np.minimum(row0 + lanes, rows - 1)]  # lanes past the last row re-read row0's
        xr[row0 + lanes >= rows] = x[row0]
        for qa in range(0, P1, chunk):
            qb = min(qa + chunk, P1)
            steps = (qb - qa) + (n - 1)
            stage = np.full(32 * UNR * n, np.nan, complex)
            w0 = walk3_start(n)
            assert w0 - 2 * S1 >= 0  # no look-back before the chunk's first window
            feeds = [(xr[:, qa + j], xr[:, max(qa + j - S1, 0)], xr[:, max(qa + j - 2 * S1, 0)])
                     for j in range(w0, steps)]
            outs = tree3_outs(n, feeds, w0)
            for jb in range(w0, steps, UNR):
                for j in range(jb, min(jb + UNR, steps)):
                    if j >= n - 1:
                        for c in range(R):
                            for u in range(OUT):
                                stage[(lanes * UNR + (j - jb)) * n + c + 3 * u] = outs[c][j - w0][u]
                j0, j1 = max(jb, n - 1), min(jb + UNR, steps)
                if j1 > j0:
                    run, q, sofs = (j1 - j0) * n, qa + j0 - (n - 1), (j0 - jb) * n
                    for r in range(nrows):
                        zq = (pad + row0 + r) * zrow + q * n
                        sq = sofs + r * UNR * n
                        assert q * n + run <= zrow  # inside the row
                        z[zq:zq + run] = stage[sq:sq + run]
                        written[zq:zq + run] += 1
    assert (written[pad * zrow:] == 1).all(), "z value not written exactly once"
    return z.reshape(pad + rows, zrow)


def emulate_col_pass3(z, pad, n0, n1, P1, rows_out, chunk, scale):
    B3, A2 = mixed_split(n0)
    M = B3  # 0: a window of one row
    n, R, OUT = n0, (3 if B3 >= 1 else 1), (n0 // 3 if B3 >= 1 else 1)
    S1 = n0 // 3 if B3 >= 1 else 0
    W = 64
    G = col3_group(mixed_period(B3, A2) if B3 >= 1 else 1)
    assert B3 == 0 or G % mixed_period(B3, A2) == 0
    need = (2 * S1 if B3 >= 1 else 0) + 2 * G
    RD = 1 << (need - 1).bit_length()
    T = max(1, W // n1)
    CH = T * n1
    nch = P1 * n1
    orow_len = nch * n
    staged = n1 % 4 != 0
    out = np.full(rows_out * orow_len, np.nan, complex)
    written = np.zeros(out.shape, int)
    my = np.arange(W)
    for bx in range(-(-P1 // T)):
        q1_0 = bx * T
        ch0 = q1_0 * n1
        ch = ch0 + my
        active = (my < CH) & (ch < nch)
        tile_elems = min(T, nch // n1 - q1_0) * n * n1
        q1l, k1 = my // n1, my % n1
        for qa in range(0, rows_out, chunk):
            qb = min(qa + chunk, rows_out)
            steps, zr_end = (qb - qa) + (n - 1), qb + n - 1
            ring = np.full(RD * W, np.nan, complex)

            def fetch(r_lo, r_hi):
                for rr in range(r_lo, r_hi):
                    assert 0 <= pad + rr < z.shape[0]
                    cc = np.arange(CH)
                    ok = ch0 + cc < nch
                    ring[(rr & (RD - 1)) * W + cc] = np.where(ok, z[pad + rr, np.minimum(ch0 + cc, nch - 1)], 0)

            w0 = walk3_start(n)
            fetch(qa + w0 - 2 * S1, min(qa + w0 + G, zr_end))
            feeds = []
            for jb in range(w0, steps, G):
                if jb + G < steps:
                    fetch(qa + jb + G, min(qa + jb + 2 * G, zr_end))
                for j in range(jb, min(jb + G, steps)):
                    zr = qa + j
                    assert zr - 2 * S1 >= qa  # the shortened walk reads no padding row
                    f = tuple(ring[((zr - d) & (RD - 1)) * W + my] for d in (0, S1, 2 * S1))
                    for d, v in zip((0, S1, 2 * S1), f):  # the live lanes read z rows zr - d
                        if M >= 1 or d == 0:
                            np.testing.assert_array_equal(v[active], z[pad + zr - d, ch[active]])
                    feeds.append(f)
            outs = tree3_outs(n, feeds, w0, scale)  # the scale folded into level 1
            orow = qa * orow_len + q1_0 * n * n1
            stage = [np.full(W * n, np.nan, complex) for _ in range(2)]
            buf = 0
            for j in range(n - 1, steps):
                if staged:
                    st = stage[buf]
                    for c in range(R):
                        for u in range(OUT):
                            idx = q1l * n * n1 + c * n1 + k1 + 3 * u * n1
                            st[idx[my < CH]] = outs[c][j - w0][u][my < CH]
                    e = np.arange(tile_elems)
                    # one bulk copy (16-byte aligned ends, a multiple of 16 bytes) where the run
                    # allows it, else per-thread copies: the same values either way
                    bulk = orow_len % 2 == 0 and (q1_0 * n * n1) % 2 == 0 and tile_elems % 2 == 0
                    if bulk:
                        assert orow % 2 == 0 and (RD * W + buf * W * n) % 2 == 0 and (8 * tile_elems) % 16 == 0
                    out[orow + e] = st[e]
                    written[orow + e] += 1
                    buf ^= 1
                else:
                    for c in range(R):
                        for u in range(OUT):
                            idx = orow + q1l * n * n1 + c * n1 + k1 + 3 * u * n1
                            out[idx[active]] = outs[c][j - w0][u][active]
                            written[idx[active]] += 1
                orow += orow_len
    assert (written == 1).all(), "output not written exactly once"
    return out.reshape(rows_out, P1, n0, n1)


TERNARY_CASES = [  # (n0, n1, rows_out, P1, column chunks); n1 of 2^k comes from the binary row pass
    (1, 9, 5, 9, (5, 2)),
    (3, 3, 7, 30, (7, 3)),
    (9, 1, 8, 70, (8, 5)),
    (9, 4, 6, 21, (6, 4)),
    (27, 2, 5, 40, (5, 3)),
    (3, 27, 6, 5, (6, 4)),
    (27, 27, 3, 4, (3, 2)),
    (3, 64, 4, 3, (4, 3)),
    # mixed radices within an axis: 3^b 2^a
    (6, 6, 6, 11, (6, 4)),
    (12, 2, 5, 30, (5, 3)),
    (1, 12, 5, 9, (5, 2)),
    (24, 8, 4, 6, (4, 3)),
    (48, 1, 3, 40, (3, 2)),
    (18, 36, 3, 3, (3, 2)),
    (54, 3, 3, 5, (3, 2)),
    (9, 48, 4, 2, (4, 3)),
    (36, 16, 3, 4, (3, 2)),
]


@pytest.mark.parametrize("n0,n1,rows_out,P1,chunks", TERNARY_CASES)
def test_ternary_passes_with_staging(n0, n1, rows_out, P1, chunks):
    rng = np.random.default_rng(3000 + n0 * 64 + n1)
    N0, N1 = rows_out + n0 - 1, P1 + n1 - 1
    x = rng.standard_normal((N0, N1)) + 1j * rng.standard_normal((N0, N1))
    scale = 1 / np.sqrt(n0 * n1)
    ref = every_window_dft(x, n0, n1, scale)
    pad = 2 * n0 // 3
    for row_chunk in (P1, 4):
        if n1 % 3 == 0 or n1 == 1:
            z = emulate_row_pass3(x, n1, min(row_chunk, P1), pad)
        else:
            m1 = n1.bit_length() - 1
            z = emulate_row_pass(x, n1, min(m1, 3), min(row_chunk, P1), pad)
        for chunk in chunks:
            out = emulate_col_pass3(z, pad, n0, n1, P1, rows_out, chunk, scale)
            np.testing.assert_allclose(out, ref, atol=1e-9)
