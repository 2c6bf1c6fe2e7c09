"""Pins for the k-dimensional oracle (Section 4.4: the 2D transform of Eq. 2 with one sum per
dimension; the tree of Eq. kdfswft).  Each check ties the oracle to something other than
itself: numpy's FFT of every window, a brute-force loop with its own exponentials, a closed
form, Parseval, the 2D and 1D oracles as special cases, and the tree of Eq. kdfswft with its
node count.  A second group plants mistakes in a copy of the C source and checks that the
library-routine pin rejects each of them."""
import cmath
import itertools
import math
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

import oracle

ORACLE_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                          "oracle", "swdftkd_oracle.c")


def _rand(seed, shape, cplx=True):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(shape)
    if cplx:
        x = x + 1j * rng.standard_normal(shape)
    return x


def _fftn_windows(x, n):
    P = [a - b + 1 for a, b in zip(x.shape, n)]
    out = np.empty(tuple(P) + tuple(n), dtype=np.complex128)
    for q in itertools.product(*[range(p) for p in P]):
        sl = tuple(slice(a, a + b) for a, b in zip(q, n))
        out[q] = np.fft.fftn(x[sl]) / math.sqrt(int(np.prod(n)))
    return out


KD_CASES = [
    ((9,), (4,)), ((7, 9, 6), (4, 2, 4)), ((5, 6, 7), (1, 4, 2)), ((6, 5, 4), (2, 1, 4)),
    ((4, 5, 6), (4, 4, 4)), ((8, 3, 5), (8, 2, 1)), ((3, 4, 5, 6), (2, 2, 4, 2)),
    ((5, 4, 3, 4), (1, 4, 2, 4)),
]


@pytest.mark.parametrize("method", ["direct", "separable"])
@pytest.mark.parametrize("shape,n", KD_CASES)
def test_every_window_equals_fftn(shape, n, method):
    for cplx in (False, True):
        x = _rand(len(shape) * 10 + sum(shape), shape, cplx)
        got = oracle.swdftkd(x, n, method=method)
        assert got.shape == tuple(a - b + 1 for a, b in zip(shape, n)) + tuple(n)
        assert np.abs(got - _fftn_windows(x, n)).max() < 1e-12


def test_brute_force_three_dimensions():
    """Six nested loops with exponentials from cmath, no tables, tiny sizes."""
    x = _rand(3, (4, 3, 4))
    n = (2, 2, 4)
    got = oracle.swdftkd(x, n, norm="none")
    P = [a - b + 1 for a, b in zip(x.shape, n)]
    for q0, q1, q2 in itertools.product(range(P[0]), range(P[1]), range(P[2])):
        for k0, k1, k2 in itertools.product(range(n[0]), range(n[1]), range(n[2])):
            s = 0j
            for j0, j1, j2 in itertools.product(range(n[0]), range(n[1]), range(n[2])):
                s += x[q0 + j0, q1 + j1, q2 + j2] * cmath.exp(
                    -2j * math.pi * (j0 * k0 / n[0] + j1 * k1 / n[1] + j2 * k2 / n[2]))
            assert abs(got[q0, q1, q2, k0, k1, k2] - s) < 1e-12


def test_closed_form_single_bin():
    """x = exp(2 pi i sum_d kappa_d r_d / n_d): one nonzero bin kappa in every window, of
    magnitude sqrt(prod n) on the unitary scale and phase 2 pi sum_d kappa_d q_d / n_d."""
    shape, n, kappa = (10, 9, 12), (4, 8, 2), (3, 5, 1)
    r = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    x = np.exp(2j * math.pi * sum(k * ri / nd for k, ri, nd in zip(kappa, r, n)))
    a = oracle.swdftkd(x, n, method="separable")
    P = a.shape[:3]
    mask = np.zeros(n, dtype=bool)
    mask[kappa] = True
    assert np.abs(a[..., ~mask]).max() < 1e-11
    qs = np.meshgrid(*[np.arange(p) for p in P], indexing="ij")
    expect = math.sqrt(np.prod(n)) * np.exp(2j * math.pi * sum(k * q / nd for k, q, nd in zip(kappa, qs, n)))
    assert np.abs(a[..., kappa[0], kappa[1], kappa[2]] - expect).max() < 1e-11


def test_parseval_every_window():
    x = _rand(5, (9, 8, 10))
    n = (4, 4, 8)
    a = oracle.swdftkd(x, n, method="separable")
    e = (np.abs(a) ** 2).sum(axis=(3, 4, 5))
    P = a.shape[:3]
    for q in itertools.product(*[range(p) for p in P]):
        w = x[q[0]:q[0] + 4, q[1]:q[1] + 4, q[2]:q[2] + 8]
        assert abs(e[q] - (np.abs(w) ** 2).sum()) < 1e-10 * max(1.0, e[q])


def test_reduces_to_the_2d_and_1d_oracles():
    x2 = _rand(6, (11, 13))
    a2 = oracle.swdft2d(x2, 4, 8)
    assert np.abs(oracle.swdftkd(x2, (4, 8)) - a2).max() < 1e-13
    # a leading dimension of extent 1 with a window of 1 is the 2D transform of the slice
    a3 = oracle.swdftkd(x2[None], (1, 4, 8), method="separable")
    assert np.abs(a3[0, :, :, 0] - a2).max() < 1e-13
    # one dimension: the 1D sliding DFT, numpy FFT of every window
    x1 = _rand(7, (20,))
    a1 = oracle.swdftkd(x1, (8,), norm="none")
    ref = np.stack([np.fft.fft(x1[q:q + 8]) for q in range(13)])
    assert np.abs(a1 - ref).max() < 1e-12


@pytest.mark.parametrize("shape,n", KD_CASES)
def test_tree_eq_kdfswft_matches_definition_and_counts_nodes(shape, n):
    """Eq. kdfswft reproduces every window's DFT (to FP64 rounding), and a tree over
    prod n coefficients costs 2 (prod n - 1) node evaluations at every position."""
    x = _rand(99 + sum(shape), shape)
    t, ops = oracle.treekd(x, n)
    assert np.abs(t - oracle.swdftkd(x, n)).max() < 1e-13
    assert ops == int(np.prod(shape)) * 2 * (int(np.prod(n)) - 1)


def test_selected_windows_match_full_output():
    x = _rand(8, (10, 9, 12))
    n = (4, 2, 8)
    full = oracle.swdftkd(x, n)
    rng = np.random.default_rng(1)
    P = full.shape[:3]
    q = np.stack([rng.integers(0, p, 40) for p in P], axis=1)
    for method in ("direct", "separable"):
        got = oracle.swdftkd_windows(x, n, q, method=method)
        assert np.abs(got - full[q[:, 0], q[:, 1], q[:, 2]]).max() < 1e-13


def test_rejects_bad_shapes():
    with pytest.raises(ValueError):
        oracle.swdftkd(np.zeros((4, 4, 4)), (8, 2, 2))
    with pytest.raises(ValueError):
        oracle.swdftkd(np.zeros((2, 2, 2, 2, 2)), (1, 1, 1, 1, 1))
    with pytest.raises(ValueError):
        oracle.treekd(np.zeros((6, 6, 6)), (3, 2, 2))  # the tree needs powers of two
    with pytest.raises(ValueError):
        oracle.swdftkd_windows(np.zeros((6, 6, 6)), (2, 2, 2), [[5, 0, 0]])


# (name, original text, mutated text): plausible mistakes, each caught by the fftn pin
MUTANTS = [
    ("exponent_sign", "w[2 * j + 1] = -sin(ang);", "w[2 * j + 1] = sin(ang);"),
    ("direct_dropped_dimension_offset", "off += jj[d] * g->xstride[d];\n            }",
     "if (d > 0) off += jj[d] * g->xstride[d];\n            }"),
    ("direct_kernel_product_sign", "const double tr = er * e[0] - ei * e[1];",
     "const double tr = er * e[0] + ei * e[1];"),
    ("separable_transposed_axes", "const int64_t st = g->kstride[d];\n        for (int64_t start",
     "const int64_t st = g->kstride[g->K - 1 - d];\n        for (int64_t start"),
    ("input_strides_swapped", "g->xstride[d] = g->xstride[d + 1] * N[d + 1];",
     "g->xstride[d] = g->xstride[d + 1] * N[d];"),
    ("missing_scale", "for (int64_t i = 0; i < 2 * g->nn; ++i) out[i] *= c;", ""),
]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name,orig,mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_kd_mutant(tmp_path, name, orig, mut):
    src = open(ORACLE_SRC).read()
    assert src.count(orig) == 1, f"mutation site for {name} not found exactly once"
    mpath = tmp_path / "mutant.c"
    mpath.write_text(src.replace(orig, mut))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-o", str(so), str(mpath), "-lm"],
                   check=True, capture_output=True)
    # the mutant runs in a child process: a mutant that corrupts memory is caught by its
    # crash instead of taking the test run down with it
    shape, n = (6, 5, 10), (4, 2, 8)  # distinct lengths, so no axis can stand in for another
    x = np.ascontiguousarray(_rand(17, shape))
    ref_path = tmp_path / "ref.npy"
    np.save(ref_path, _fftn_windows(x, n))
    x_path = tmp_path / "x.npy"
    np.save(x_path, x)
    child = f"""
import ctypes, math, numpy as np
lib = ctypes.CDLL({str(so)!r})
P = ctypes.c_void_p
lib.swo_swdftkd.argtypes = [P, ctypes.c_int, P, P, ctypes.c_double, ctypes.c_int, ctypes.c_int, P]
x = np.load({str(x_path)!r}); ref = np.load({str(ref_path)!r})
N = np.array(x.shape, dtype=np.int64); nw = np.array({n!r}, dtype=np.int32)
ok = True
for method in (0, 1):
    out = np.zeros(ref.shape, dtype=np.complex128)
    rc = lib.swo_swdftkd(x.ctypes.data, 3, N.ctypes.data, nw.ctypes.data,
                         1 / math.sqrt(int(np.prod(nw))), method, 1, out.ctypes.data)
    ok = ok and rc == 0 and bool(np.abs(out - ref).max() < 1e-12)
print("PASSED_PIN" if ok else "CAUGHT")
"""
    res = subprocess.run([sys.executable, "-c", child], capture_output=True, text=True, timeout=120)
    caught = "PASSED_PIN" not in res.stdout
    assert caught, f"mutant {name} passed the fftn pin"
