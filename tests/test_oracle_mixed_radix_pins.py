"""Pins for mixed-radix windows (n = 2^a 3^b samples along one axis): the tree with a radix
chosen per level (oracle/swdft_radix_tree.c, swt_tree2d_mixed_f64), which extends the
paper's binary tree (Section 4.2) and the ternary trees Section 5 mentions.

The recurrence was derived for this library (the paper gives none), so it is tied to things
outside itself: the definition oracle (Eq. 2) is first pinned to numpy's fft2 at these
lengths; then every order of a window's radices must reproduce that definition to FP64
rounding, with the node count the recurrence implies; a pure complex exponential must give
one bin of known magnitude and phase in every window; a constant radix must agree bit for bit
with the radix-2 / radix-3 tree; and planted mistakes in the C source must fail."""
import math
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

import oracle

# (radices of dimension 0, radices of dimension 1), level order; every mixed length to 54
CASES = [
    ((3, 2), (2, 3)),            # 6 x 6, radix 3 first along one axis, radix 2 first along the other
    ((3, 2, 2), (2,)),           # 12 x 2
    ((2, 3, 2), (2, 2)),         # 12 x 4, interleaved
    ((2,), (3, 2, 2)),           # 2 x 12
    ((3, 3, 2), ()),             # 18 x 1
    ((2, 3, 3), (3,)),           # 18 x 3
    ((3, 2, 2, 2), (2,)),        # 24 x 2
    ((2, 2, 2, 3), (3, 2)),      # 24 x 6
    ((3, 3, 2, 2), ()),          # 36 x 1
    ((), (2, 3, 2, 3)),          # 1 x 36
    ((3, 2, 2, 2, 2), (2,)),     # 48 x 2
    ((2,), (2, 2, 3, 2, 2)),     # 2 x 48
    ((3, 3, 3, 2), ()),          # 54 x 1
    ((), (2, 3, 3, 3)),          # 1 x 54
    ((3, 2), (3, 3, 2, 2)),      # 6 x 36
]


def _n(rads):
    return int(np.prod(rads)) if rads else 1


def _x(seed, N0, N1):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((N0, N1)) + 1j * rng.standard_normal((N0, N1))


def _fft2_windows(x, n0, n1):
    P0, P1 = x.shape[0] - n0 + 1, x.shape[1] - n1 + 1
    return np.stack([[np.fft.fft2(x[i:i + n0, j:j + n1]) for j in range(P1)]
                     for i in range(P0)]) / math.sqrt(n0 * n1)


def _nodes(rads):
    """Nodes of one 1D tree: level t has N_t = r_1 .. r_t nodes."""
    total, size = 0, 1
    for r in rads:
        size *= r
        total += size
    return total


@pytest.mark.parametrize("r0,r1", CASES)
def test_definition_at_mixed_lengths_equals_fft2(r0, r1):
    n0, n1 = _n(r0), _n(r1)
    x = _x(n0 * 131 + n1, n0 + 4, n1 + 3)
    ref = _fft2_windows(x, n0, n1)
    for method in ("direct", "separable"):
        assert np.abs(oracle.swdft2d(x, n0, n1, method=method) - ref).max() < 1e-12


@pytest.mark.parametrize("r0,r1", CASES)
def test_mixed_tree_matches_definition_and_counts_nodes(r0, r1):
    n0, n1 = _n(r0), _n(r1)
    N0, N1 = n0 + 5, n1 + 6
    x = _x(7 * n0 + n1, N0, N1)
    t, ops = oracle.tree2d_mixed(x, r0, r1)
    assert np.abs(t - oracle.swdft2d(x, n0, n1, method="separable")).max() < 1e-12
    assert ops == N0 * N1 * (_nodes(r1) + n1 * _nodes(r0))


@pytest.mark.parametrize("rads", [(3, 2, 2, 2), (2, 3, 2, 2), (2, 2, 3, 2), (2, 2, 2, 3)])
def test_every_order_of_the_radices_gives_the_same_windows(rads):
    """24 = 3 * 2^3 in all four orders: the same window DFTs (to FP64 rounding)."""
    x = _x(24, 5, 30)
    ref = _fft2_windows(x, 1, 24)
    t, _ = oracle.tree2d_mixed(x, (), rads)
    assert np.abs(t - ref).max() < 1e-12


def test_one_complex_exponential_gives_one_bin():
    """x = exp(2 pi i (k0 r / n0 + k1 c / n1)): window q has the single bin (k0, k1) of
    magnitude sqrt(n0 n1) (unitary scale) and phase 2 pi (k0 q0 / n0 + k1 q1 / n1)."""
    r0, r1 = (3, 2, 2), (2, 3)  # 12 x 6
    n0, n1 = 12, 6
    k0, k1 = 5, 4
    N0, N1 = 20, 15
    r, c = np.meshgrid(np.arange(N0), np.arange(N1), indexing="ij")
    x = np.exp(2j * np.pi * (k0 * r / n0 + k1 * c / n1))
    t, _ = oracle.tree2d_mixed(x, r0, r1)
    want = np.zeros_like(t)
    q0, q1 = np.meshgrid(np.arange(N0 - n0 + 1), np.arange(N1 - n1 + 1), indexing="ij")
    want[:, :, k0, k1] = math.sqrt(n0 * n1) * np.exp(2j * np.pi * (k0 * q0 / n0 + k1 * q1 / n1))
    assert np.abs(t - want).max() < 1e-11


def test_constant_radix_is_the_radix_2_and_radix_3_tree():
    x = _x(5, 30, 20)
    for (r0, r1) in (((2, 2, 2), (2, 2)), ((3, 3), (3,)), ((3, 3, 3), (2, 2))):
        a, ops_a = oracle.tree2d_mixed(x, r0, r1)
        b, ops_b = oracle.tree2d_radix(x, _n(r0), _n(r1))
        assert ops_a == ops_b
        assert np.array_equal(a, b)


RADIX_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                         "swdft_radix_tree.c")
FN = "int swt_tree2d_mixed_f64("

MUTANTS = [
    ("reversed_shift", "const int64_t q = p0 - (int64_t)(r - 1 - d) * s;", "const int64_t q = p0 - (int64_t)d * s;"),
    ("twiddle_without_stride", "const double *w = om1 + 2 * ((i * d * s) % n1);", "const double *w = om1 + 2 * ((i * d) % n1);"),
    ("parent_mod_size", "(i0 % prev_size) * n1 + i1);", "(i0 % size) * n1 + i1);"),
    ("twiddle_on_parent_index", "const double *w = om1 + 2 * ((i * d * s) % n1);",
     "const double *w = om1 + 2 * (((i % prev_size) * d * s) % n1);"),
]


@pytest.mark.parametrize("name,orig,mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_mixed_tree_mutant(tmp_path, name, orig, mut):
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    src = open(RADIX_SRC).read()
    head, fn = src[:src.index(FN)], src[src.index(FN):]
    assert fn.count(orig) == 1, f"mutation site for {name} not found exactly once"
    (tmp_path / "m.c").write_text(head + fn.replace(orig, mut))
    so = tmp_path / "libm.so"
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-o", str(so), str(tmp_path / "m.c"), "-lm"],
                   check=True, capture_output=True)
    x = _x(31, 17, 16)
    np.save(tmp_path / "x.npy", x)
    np.save(tmp_path / "ref.npy", _fft2_windows(x, 12, 6))
    child = f"""
import ctypes, math, numpy as np
lib = ctypes.CDLL({str(so)!r}); P = ctypes.c_void_p
lib.swt_tree2d_mixed_f64.argtypes = [P, ctypes.c_int64, ctypes.c_int64, P, ctypes.c_int, P, ctypes.c_int, ctypes.c_double, P, P]
x = np.ascontiguousarray(np.load({str(tmp_path / 'x.npy')!r})); ref = np.load({str(tmp_path / 'ref.npy')!r})
r0 = np.array([3, 2, 2], dtype=np.int32); r1 = np.array([2, 3], dtype=np.int32)
out = np.zeros(ref.shape, dtype=np.complex128)
rc = lib.swt_tree2d_mixed_f64(x.ctypes.data, 17, 16, r0.ctypes.data, 3, r1.ctypes.data, 2, 1 / math.sqrt(72), out.ctypes.data, None)
print("PASSED_PIN" if rc == 0 and np.abs(out - ref).max() < 1e-12 else "CAUGHT")
"""
    res = subprocess.run([sys.executable, "-c", child], capture_output=True, text=True, timeout=120)
    assert "PASSED_PIN" not in res.stdout, f"mutant {name} passed the pin"
