"""Pins for the FP64 oracle: each checks it against something other than itself.

Pins used (arXiv 1707.08213):
* library routine: every window equals numpy.fft.fft2 of its patch times the scale
  (Section 4.1, Eq. 2: a 2D DFT per window);
* brute force: Eq. 2 as nested loops with their own exponentials on arrays up to 12 x 12,
  every pair of window sides in {1, 2, 4, 8};
* closed forms: a pure 2D complex exponential gives one bin of known magnitude and phase;
  a real cosine gives two; the DC bin is the scaled window sum;
* invariants: per-window Parseval (unitary scale), linearity, the sliding shift identity
  between neighbouring windows, transposition symmetry (non-square windows);
* special cases: n0 = 1 reduces to the 1D SWDFT of Eq. 1 (with its 1/n scale); n = 2 is the
  length-two DFT of Section 4.2's level one; the first window is a plain 2D DFT;
* printed values: the output-size example of Section 4.3 (tests/golden);
* the paper's tree (Section 4.2) reproduces the definition to FP64 rounding (Section 4.6),
  with 2(n0 n1 - 1) node operations per tree (Eq. windowops) and the level invariant.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

SHAPES = [
    # (N0, N1, n0, n1)
    (1, 1, 1, 1), (5, 7, 1, 1), (6, 9, 2, 1), (6, 9, 1, 2), (9, 13, 4, 8), (12, 11, 8, 4),
    (8, 8, 8, 8), (11, 12, 2, 4), (10, 10, 4, 4), (7, 16, 1, 16), (16, 5, 16, 1),
]


def _rand(seed, N0, N1, cplx=True):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((N0, N1))
    if cplx:
        x = x + 1j * rng.standard_normal((N0, N1))
    return x


def _fft2_windows(x, n0, n1):
    N0, N1 = x.shape
    P0, P1 = N0 - n0 + 1, N1 - n1 + 1
    out = np.empty((P0, P1, n0, n1), dtype=np.complex128)
    for q0 in range(P0):
        for q1 in range(P1):
            out[q0, q1] = np.fft.fft2(x[q0:q0 + n0, q1:q1 + n1])
    return out


@pytest.mark.parametrize("method", ["direct", "separable"])
@pytest.mark.parametrize("N0,N1,n0,n1", SHAPES)
@pytest.mark.parametrize("cplx", [False, True])
def test_every_window_is_numpy_fft2(oracle_lib, method, N0, N1, n0, n1, cplx):
    x = _rand(N0 * 100 + N1, N0, N1, cplx)
    ref = _fft2_windows(x, n0, n1) / math.sqrt(n0 * n1)
    a = oracle_lib.swdft2d(x, n0, n1, norm="unitary", method=method)
    assert a.shape == (N0 - n0 + 1, N1 - n1 + 1, n0, n1)
    np.testing.assert_allclose(a, ref, rtol=0, atol=1e-13 * max(1.0, np.abs(x).max() * n0 * n1))


@pytest.mark.parametrize("n0", [1, 2, 4, 8])
@pytest.mark.parametrize("n1", [1, 2, 4, 8])
def test_brute_force_loops(oracle_lib, n0, n1):
    """Eq. 2 as plain nested loops with their own exponentials (no numpy FFT, no matrices),
    on arrays of at most 12 x 12, every pair of window sides in {1, 2, 4, 8}."""
    N0, N1 = min(12, n0 + 3), min(12, n1 + 4)
    x = _rand(7 * n0 + n1, N0, N1)
    a = oracle_lib.swdft2d(x, n0, n1, norm="none", method="direct")
    worst = 0.0
    for q0 in range(N0 - n0 + 1):
        for q1 in range(N1 - n1 + 1):
            for k0 in range(n0):
                for k1 in range(n1):
                    acc = 0j
                    for j0 in range(n0):
                        for j1 in range(n1):
                            ang = -2.0 * math.pi * (j0 * k0 / n0 + j1 * k1 / n1)
                            acc += x[q0 + j0, q1 + j1] * complex(math.cos(ang), math.sin(ang))
                    worst = max(worst, abs(a[q0, q1, k0, k1] - acc))
    assert worst <= 1e-12 * n0 * n1


@pytest.mark.parametrize("norm,scale", [("none", lambda n0, n1: 1.0),
                                        ("unitary", lambda n0, n1: 1 / math.sqrt(n0 * n1)),
                                        ("inv_n", lambda n0, n1: 1.0 / (n0 * n1))])
def test_first_window_is_plain_2d_dft(oracle_lib, norm, scale):
    x = _rand(3, 12, 20)
    a = oracle_lib.swdft2d(x, 4, 8, norm=norm)
    np.testing.assert_allclose(a[0, 0], np.fft.fft2(x[:4, :8]) * scale(4, 8), atol=1e-12)


@pytest.mark.parametrize("n0,n1,k0,k1", [(4, 8, 1, 3), (8, 4, 7, 0), (8, 8, 0, 5), (2, 16, 1, 9)])
def test_pure_exponential_gives_one_bin(oracle_lib, n0, n1, k0, k1):
    N0, N1 = 13, 21
    r = np.arange(N0)[:, None]
    c = np.arange(N1)[None, :]
    x = np.exp(2j * np.pi * (k0 * r / n0 + k1 * c / n1))
    a = oracle_lib.swdft2d(x, n0, n1, norm="unitary", method="direct")
    P0, P1 = N0 - n0 + 1, N1 - n1 + 1
    q0 = np.arange(P0)[:, None]
    q1 = np.arange(P1)[None, :]
    expect_bin = math.sqrt(n0 * n1) * np.exp(2j * np.pi * (k0 * q0 / n0 + k1 * q1 / n1))
    np.testing.assert_allclose(a[:, :, k0, k1], expect_bin, atol=1e-12)
    mask = np.ones((n0, n1), bool)
    mask[k0, k1] = False
    assert np.abs(a[:, :, mask]).max() < 1e-12


def test_real_cosine_gives_two_bins(oracle_lib):
    n0, n1, k0, k1 = 8, 8, 2, 3
    r = np.arange(16)[:, None]
    c = np.arange(16)[None, :]
    x = np.cos(2 * np.pi * (k0 * r / n0 + k1 * c / n1))
    a = oracle_lib.swdft2d(x, n0, n1, norm="none")
    mag = np.abs(a)
    assert np.allclose(mag[:, :, k0, k1], n0 * n1 / 2, atol=1e-11)
    assert np.allclose(mag[:, :, n0 - k0, n1 - k1], n0 * n1 / 2, atol=1e-11)
    mag[:, :, k0, k1] = 0
    mag[:, :, n0 - k0, n1 - k1] = 0
    assert mag.max() < 1e-11


@pytest.mark.parametrize("method", ["direct", "separable"])
def test_parseval_per_window(oracle_lib, method):
    x = _rand(11, 14, 19)
    for n0, n1 in [(4, 8), (8, 2), (1, 16), (8, 8)]:
        a = oracle_lib.swdft2d(x, n0, n1, method=method)
        lhs = np.sum(np.abs(a) ** 2, axis=(2, 3))
        rhs = workloads.window_sq_norms(x, n0, n1)
        np.testing.assert_allclose(lhs, rhs, rtol=1e-12)


def test_dc_bin_is_scaled_window_sum(oracle_lib):
    x = _rand(12, 15, 17)
    n0, n1 = 4, 8
    a = oracle_lib.swdft2d(x, n0, n1, norm="unitary")
    P0, P1 = 15 - n0 + 1, 17 - n1 + 1
    sums = np.array([[x[i:i + n0, j:j + n1].sum() for j in range(P1)] for i in range(P0)])
    np.testing.assert_allclose(a[:, :, 0, 0], sums / math.sqrt(n0 * n1), atol=1e-12)


def test_linearity(oracle_lib):
    x, y = _rand(1, 10, 12), _rand(2, 10, 12)
    al, be = 0.7 - 0.2j, -1.3 + 0.5j
    lhs = oracle_lib.swdft2d(al * x + be * y, 4, 4)
    rhs = al * oracle_lib.swdft2d(x, 4, 4) + be * oracle_lib.swdft2d(y, 4, 4)
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)


@pytest.mark.parametrize("n0,n1", [(4, 8), (8, 4), (2, 16)])
def test_sliding_shift_identity(oracle_lib, n0, n1):
    """A[q0,q1+1,k] = w1^{+k1} (A[q0,q1,k] + DFT_j0(x[q0+j0,q1+n1] - x[q0+j0,q1])[k0]),
    and the same along q0, with A unnormalised."""
    x = _rand(21, 17, 23)
    A = oracle_lib.swdft2d(x, n0, n1, norm="none")
    P0, P1 = A.shape[:2]
    w1 = np.exp(2j * np.pi * np.arange(n1) / n1)
    w0 = np.exp(2j * np.pi * np.arange(n0) / n0)
    for q0 in range(P0):
        for q1 in range(P1 - 1):
            d = np.fft.fft(x[q0:q0 + n0, q1 + n1] - x[q0:q0 + n0, q1])    # over j0 -> k0
            pred = w1[None, :] * (A[q0, q1] + d[:, None])
            np.testing.assert_allclose(A[q0, q1 + 1], pred, atol=1e-11)
    for q0 in range(P0 - 1):
        for q1 in range(P1):
            d = np.fft.fft(x[q0 + n0, q1:q1 + n1] - x[q0, q1:q1 + n1])    # over j1 -> k1
            pred = w0[:, None] * (A[q0, q1] + d[None, :])
            np.testing.assert_allclose(A[q0 + 1, q1], pred, atol=1e-11)


def test_transposition_symmetry(oracle_lib):
    x = _rand(31, 11, 19)
    a = oracle_lib.swdft2d(x, 4, 8)
    b = oracle_lib.swdft2d(x.T.copy(), 8, 4)
    np.testing.assert_allclose(b, a.transpose(1, 0, 3, 2), atol=1e-12)


def test_one_dimensional_reduction_is_eq1(oracle_lib):
    """n0 = 1 with the 1/n scale is Eq. 1's 1D SWDFT of each row."""
    x = _rand(41, 3, 30)
    n = 8
    a = oracle_lib.swdft2d(x, 1, n, norm="inv_n")
    for r in range(3):
        for q in range(30 - n + 1):
            np.testing.assert_allclose(a[r, q, 0], np.fft.fft(x[r, q:q + n]) / n, atol=1e-13)


def test_level_one_is_length_two_dft(oracle_lib):
    with open(os.path.join(GOLDEN, "paper_printed_values.json")) as f:
        assert "level_one" in json.load(f)
    x = _rand(51, 4, 9)
    a = oracle_lib.swdft2d(x, 1, 2, norm="none")
    np.testing.assert_allclose(a[:, :, 0, 0], x[:, :-1] + x[:, 1:], atol=1e-14)
    np.testing.assert_allclose(a[:, :, 0, 1], x[:, :-1] - x[:, 1:], atol=1e-14)


def test_windows_subset_matches_full(oracle_lib):
    x = _rand(61, 20, 18)
    full = oracle_lib.swdft2d(x, 8, 4)
    q0s = [0, 12, 5, 12, 0]
    q1s = [0, 14, 7, 0, 14]
    for method in ("direct", "separable"):
        sub = oracle_lib.swdft2d_windows(x, 8, 4, q0s, q1s, method=method)
        np.testing.assert_allclose(sub, full[q0s, q1s], atol=1e-13)


def test_output_size_example_from_paper():
    """Section 4.3 prints the output size for P0=P1=400, n0=n1=32 in complex128."""
    with open(os.path.join(GOLDEN, "paper_printed_values.json")) as f:
        ex = json.load(f)["output_size_example"]
    n = ex["P0"] * ex["P1"] * ex["n0"] * ex["n1"]
    assert n == ex["complex_numbers"]
    assert n * ex["bytes_per_complex"] == ex["bytes"]
    # the oracle's output for such an array has that many elements (shape only, small rows)
    N1 = ex["P1"] + ex["n1"] - 1
    assert (32 - 32 + 1) * (N1 - 32 + 1) * 32 * 32 * ex["P0"] == ex["complex_numbers"]


# ---------------------------------------------------------------- the paper's tree (FP64)

@pytest.mark.parametrize("N0,N1,n0,n1", SHAPES + [(20, 24, 16, 8), (33, 40, 32, 32)])
def test_tree_reproduces_definition(oracle_lib, N0, N1, n0, n1):
    x = _rand(N0 + 7 * N1, N0, N1)
    ref = oracle_lib.swdft2d(x, n0, n1, method="separable")
    out, ops, _ = oracle_lib.tree2d(x, n0, n1)
    nrm = np.sqrt(workloads.window_sq_norms(x, n0, n1))
    err = np.abs(out - ref).max(axis=(2, 3)) / nrm
    assert err.max() < 1e-13


def test_tree_opcount_matches_eq_windowops(oracle_lib):
    with open(os.path.join(GOLDEN, "paper_printed_values.json")) as f:
        cases = json.load(f)["window_ops"]["cases"]
    for n0, n1, c_each in cases:
        assert 2 * (n0 * n1 - 1) == c_each
        if n0 * n1 > 256:
            continue
        N0, N1 = n0 + 2, n1 + 3
        _, ops, _ = oracle_lib.tree2d(_rand(1, N0, N1), n0, n1)
        assert ops == N0 * N1 * c_each


def test_tree_level_invariant(oracle_lib):
    """Row level t node i1 at p is the 2^t-point DFT of x[p0, p1-(2^t-1-j)s_t], j<2^t;
    column level v node (i0,i1) is the 2^(v-m1)-point DFT along p0 (stride s_v) of the
    n1-point row DFTs, for complete positions."""
    N0, N1, n0, n1 = 12, 14, 4, 8
    m0, m1 = 2, 3
    x = _rand(71, N0, N1)
    for t in range(1, m1 + 1):
        _, _, dump = oracle_lib.tree2d(x, n0, n1, norm="none", dump_level=t)
        s = 2 ** (m1 - t)
        L = 2 ** t
        for p0 in range(N0):
            for p1 in range((L - 1) * s, N1):
                seq = x[p0, [p1 - (L - 1 - j) * s for j in range(L)]]
                np.testing.assert_allclose(dump[p0, p1, :L], np.fft.fft(seq), atol=1e-12)
    for v in range(m1 + 1, m1 + m0 + 1):
        _, _, dump = oracle_lib.tree2d(x, n0, n1, norm="none", dump_level=v)
        s = 2 ** (m0 + m1 - v)
        L = 2 ** (v - m1)
        for p0 in range((L - 1) * s, N0):
            for p1 in range(n1 - 1, N1):
                rows = [p0 - (L - 1 - j) * s for j in range(L)]
                z = np.stack([np.fft.fft(x[r, p1 - n1 + 1:p1 + 1]) for r in rows])  # (L, n1)
                got = dump[p0, p1, :L * n1].reshape(L, n1)
                np.testing.assert_allclose(got, np.fft.fft(z, axis=0), atol=1e-11)


def test_tree_f32_close_to_definition(oracle_lib):
    x = workloads.small_uniform_64().images[0]
    ref = oracle_lib.swdft2d(x, 8, 8)
    out, _, _ = oracle_lib.tree2d(x, 8, 8, precision="f32")
    nrm = np.sqrt(workloads.window_sq_norms(x, 8, 8))
    e, _ = workloads.normalised_error(out, ref, nrm ** 2)
    assert e < 1e-5


# ---------------------------------------------------------------- adjoint

@pytest.mark.parametrize("n0,n1", [(4, 8), (8, 4), (1, 4), (4, 1), (2, 2), (3, 6), (9, 4), (12, 1), (1, 12),
                                   (6, 9), (27, 3)])
def test_adjoint_dot_product(oracle_lib, n0, n1):
    """<A x, G> = <x, A^H G> for both adjoint methods, power-of-two and mixed-radix windows."""
    N0, N1 = max(11, n0 + 4), max(13, n1 + 5)
    x = _rand(81, N0, N1)
    rng = np.random.default_rng(82)
    G = rng.standard_normal((N0 - n0 + 1, N1 - n1 + 1, n0, n1)) + 1j * rng.standard_normal(
        (N0 - n0 + 1, N1 - n1 + 1, n0, n1))
    ax = oracle_lib.swdft2d(x, n0, n1)
    for method in ("direct", "separable"):
        ahg = oracle_lib.swdft2d_adjoint(G, N0, N1, method=method)
        lhs = np.vdot(ax, G)          # <A x, G>
        rhs = np.vdot(x, ahg)         # <x, A^H G>
        assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(lhs))


def test_adjoint_pixels_match_full(oracle_lib):
    N0, N1, n0, n1 = 14, 12, 4, 8
    rng = np.random.default_rng(90)
    G = rng.standard_normal((N0 - n0 + 1, N1 - n1 + 1, n0, n1)) + 0.5j
    full = oracle_lib.swdft2d_adjoint(G, N0, N1)
    rs = [0, 13, 7, 0, 13, 5]
    cs = [0, 11, 6, 11, 0, 2]
    np.testing.assert_allclose(oracle_lib.swdft2d_adjoint_pixels(G, N0, N1, rs, cs),
                               full[rs, cs], atol=1e-12)


def test_adjoint_equals_finite_differences_of_loss(oracle_lib):
    """L(x) = sum w |A x|^2 for real x: dL/dx = Re(A^H (2 w A x)) (central differences)."""
    N0, N1, n0, n1 = 8, 9, 4, 4
    rng = np.random.default_rng(91)
    x = rng.standard_normal((N0, N1))
    w = rng.uniform(size=(N0 - n0 + 1, N1 - n1 + 1, n0, n1))

    def loss(v):
        return float(np.sum(w * np.abs(oracle_lib.swdft2d(v, n0, n1)) ** 2))

    a = oracle_lib.swdft2d(x, n0, n1)
    grad = oracle_lib.swdft2d_adjoint(2 * w * a, N0, N1).real
    h = 1e-6
    for r, c in itertools.product(range(N0), range(N1)):
        e = np.zeros_like(x)
        e[r, c] = h
        fd = (loss(x + e) - loss(x - e)) / (2 * h)
        assert abs(fd - grad[r, c]) < 1e-6 * max(1.0, abs(fd))
