"""The mixed-radix adjoint's per-window inverse FFT (csrc/adjoint3.cu, ifft_rec / ifft_pos),
replayed on the CPU with the kernel's own index arithmetic: radix 3 while the length has a
factor 3 above 3, then radix 2; the R interleaved subsequences transformed in place, then per
j' one R-point butterfly twiddled by w_N^{+j' d} (none for j' = 0), output a stored over input
d; X[j] read back at ifft_pos(N, j).  The butterflies are the kernel's: a sum and a difference
for R = 2, and for R = 3 X0 = t0 + s, X1 = m + i h d, X2 = m - i h d (s = t1 + t2,
d = t1 - t2, m = t0 - s/2, h = sin(pi/3) from the table).  Checked against numpy's inverse FFT
(times N) for every window length the adjoint takes; planted mistakes (the twiddle taken at
the top length, the rotation's sign flipped) must fail."""
import numpy as np
import pytest


def ifft_radix(n):
    return 3 if (n % 3 == 0 and n > 3) else (2 if (n % 2 == 0 and n > 2) else n)


def ifft_pos(n, j):
    if n <= 3:
        return j
    r = ifft_radix(n)
    m = n // r
    return r * ifft_pos(m, j % m) + j // m


def bfly(t, h, sign=1):
    """The kernel's inverse 2- and 3-point butterflies (ibfly3 for three inputs)."""
    if len(t) == 1:
        return t
    if len(t) == 2:
        return [t[0] + t[1], t[0] - t[1]]
    s, d = t[1] + t[2], t[1] - t[2]
    m = t[0] - 0.5 * s
    return [t[0] + s, m + sign * 1j * h * d, m - sign * 1j * h * d]


def ifft_rec(v, ntop, n, stride, off, w, sub_twiddle=True, sign=1):
    """w[k] = w_ntop^{-k}; conj(w[x ntop / n]) = w_n^{+x}."""
    h = -w[ntop // 3].imag if ntop % 3 == 0 else 0.0
    if n <= 3:
        x = bfly([v[off + stride * k] for k in range(n)], h, sign)
        for a in range(n):
            v[off + stride * a] = x[a]
        return
    r = ifft_radix(n)
    m = n // r
    for d in range(r):
        ifft_rec(v, ntop, m, stride * r, off + stride * d, w, sub_twiddle, sign)
    for jp in range(m):
        base = off + stride * r * ifft_pos(m, jp)
        step = (ntop // n) if sub_twiddle else 1
        t = [v[base + stride * d] if (d == 0 or jp == 0) else np.conj(w[(jp * d * step) % ntop]) * v[base + stride * d]
             for d in range(r)]
        x = bfly(t, h, sign)
        for a in range(r):
            v[base + stride * a] = x[a]


LENGTHS = [1, 2, 3, 6, 9, 12, 18, 24, 27, 36, 48, 54]


@pytest.mark.parametrize("n", LENGTHS)
def test_inverse_fft_matches_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    w = np.exp(-2j * np.pi * np.arange(n) / n)
    v = list(x)
    ifft_rec(v, n, n, 1, 0, w)
    got = np.array([v[ifft_pos(n, j)] for j in range(n)])
    assert sorted(ifft_pos(n, j) for j in range(n)) == list(range(n))  # a permutation
    assert np.abs(got - np.fft.ifft(x) * n).max() < 1e-9 * max(1, n)


@pytest.mark.parametrize("mistake", ["top-length twiddle", "rotation sign"])
def test_planted_mistakes_fail(mistake):
    n = 27
    rng = np.random.default_rng(1)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    w = np.exp(-2j * np.pi * np.arange(n) / n)
    v = list(x)
    if mistake == "top-length twiddle":
        ifft_rec(v, n, n, 1, 0, w, sub_twiddle=False)
    else:
        ifft_rec(v, n, n, 1, 0, w, sign=-1)
    got = np.array([v[ifft_pos(n, j)] for j in range(n)])
    assert np.abs(got - np.fft.ifft(x) * n).max() > 1e-3
