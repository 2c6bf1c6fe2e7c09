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


def forward_walk(M, B, c, x):
    """Thread c's outputs (nodes k = c + 2^B t of level M) at every position p."""
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
    for j, p in enumerate(range(len(x))):
        J = j % period
        cur = [x[p]] + [0j] * (held(B, M) - 1)
        look_back = x[max(p - n // 2, 0)] if M >= 1 else 0j  # level 0 is re-read, no FIFO
        for v in range(1, M + 1):
            hp = held(B, v - 1)
            if v == 1:
                old = [look_back]
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


def adjoint_walk(M, B, c, G, N):
    """Thread c's partial of y[p] = sum_j sum_k G[p-j][k] w_n^{+jk}, p = N-1 .. 0."""
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
    y = np.zeros(N, complex)
    for j, p in enumerate(range(N - 1, -1, -1)):
        J = j % period
        q = p - (n - 1)
        ks = [cb + (t << B) for t in range(held(B, M))]
        cur = [G[q][k] if 0 <= q < len(G) else 0j for k in ks]
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
        y[p] = cur[0]
    return y


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


def ternary_walk(M, c, x):
    """Thread c (< 3) of the ternary tree split by residue mod 3 (tree3_core.cuh): its
    level-M nodes c + 3u, u < 3^(M-1), at every position p."""
    n = 3 ** M
    w27 = np.exp(-2j * np.pi * np.arange(27) / 27)
    s1 = 3 ** (M - 1)

    def held_t(t):  # level-t nodes one thread holds
        return 1 if t <= 1 else 3 ** (t - 1)

    tw = {t: [(w27[(ip * (27 // 3 ** t)) % 27], w27[(2 * ip * (27 // 3 ** t)) % 27])
              for ip in (c + 3 * a for a in range(3 ** (t - 2)))] for t in range(2, M + 1)}
    # level t-1 is read s_t and 2 s_t steps back: a FIFO of 2 s_t slots
    fifos = {t: [[0j] * held_t(t - 1) for _ in range(2 * 3 ** (M - t))] for t in range(2, M + 1)}
    period = 2 * 3 ** (M - 2) if M >= 2 else 1
    w3 = np.exp(-2j * np.pi / 3)
    outs = []
    for j, p in enumerate(range(len(x))):
        J = j % period
        xs1 = x[p - s1] if p - s1 >= 0 else 0j
        xs2 = x[p - 2 * s1] if p - 2 * s1 >= 0 else 0j
        cur = [xs2 + w3 ** c * xs1 + w3 ** (2 * c) * x[p]]  # level 1, node c
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
