"""The mixed-radix adjoint's per-window inverse FFT (csrc/adjoint3.cu, ifft_rec / ifft_pos),
replayed on the CPU with the kernel's own index arithmetic: radix 3 while the length has a
factor 3 above 3, then radix 2; the R interleaved subsequences transformed in place, then per
j' one R-point butterfly twiddled by w_N^{+j' d}, output a stored over input d; X[j] read back
at ifft_pos(N, j).  Checked against numpy's inverse FFT (times N) for every window length the
adjoint takes, and a planted mistake (the twiddle taken at the top length) must fail."""
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


def ifft_rec(v, ntop, n, stride, off, w, sub_twiddle=True):
    """w[k] = w_ntop^{-k}; conj(w[x ntop / n]) = w_n^{+x}."""
    if n <= 3:
        x = [v[off + stride * k] for k in range(n)]
        for a in range(n):
            v[off + stride * a] = sum(np.conj(w[(a * d * (ntop // n)) % ntop]) * x[d] for d in range(n))
        return
    r = ifft_radix(n)
    m = n // r
    for d in range(r):
        ifft_rec(v, ntop, m, stride * r, off + stride * d, w, sub_twiddle)
    for jp in range(m):
        base = off + stride * r * ifft_pos(m, jp)
        step = (ntop // n) if sub_twiddle else 1
        t = [v[base] if d == 0 else np.conj(w[(jp * d * step) % ntop]) * v[base + stride * d] for d in range(r)]
        for a in range(r):
            v[base + stride * a] = sum(np.conj(w[(a * d * (ntop // r)) % ntop]) * t[d] for d in range(r))


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


def test_planted_twiddle_mistake_fails():
    n = 27
    rng = np.random.default_rng(1)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    w = np.exp(-2j * np.pi * np.arange(n) / n)
    v = list(x)
    ifft_rec(v, n, n, 1, 0, w, sub_twiddle=False)
    got = np.array([v[ifft_pos(n, j)] for j in range(n)])
    assert np.abs(got - np.fft.ifft(x) * n).max() > 1e-3
