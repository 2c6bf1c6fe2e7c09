"""Pins for radix-3 windows (the ternary trees Section 5 mentions without equations).

The definition oracle takes any window length; here it is tied to numpy's fft2 at lengths
3, 9 and 27 (and mixed with powers of two), and the derived ternary recurrence (the tree in
oracle/swdft_radix_tree.c) is checked against that definition to FP64 rounding, with its
node count, and against the paper's binary tree where both apply."""
import math

import numpy as np
import pytest

import oracle

CASES = [(3, 3), (9, 3), (3, 9), (27, 1), (1, 27), (9, 9), (27, 9), (9, 16), (8, 27), (3, 2), (4, 3),
         (2, 4), (16, 8)]


def _x(seed, N0, N1):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((N0, N1)) + 1j * rng.standard_normal((N0, N1))


def _fft2_windows(x, n0, n1):
    P0, P1 = x.shape[0] - n0 + 1, x.shape[1] - n1 + 1
    return np.stack([[np.fft.fft2(x[i:i + n0, j:j + n1]) for j in range(P1)]
                     for i in range(P0)]) / math.sqrt(n0 * n1)


def _nodes(n):
    """Nodes per 1D tree of n = r^m samples: sum_t r^t = r (n - 1) / (r - 1)."""
    if n == 1:
        return 0
    r = 3 if n % 3 == 0 else 2
    return r * (n - 1) // (r - 1)


@pytest.mark.parametrize("n0,n1", CASES)
def test_definition_at_radix3_lengths_equals_fft2(n0, n1):
    x = _x(n0 * 100 + n1, n0 + 5, n1 + 4)
    ref = _fft2_windows(x, n0, n1)
    for method in ("direct", "separable"):
        assert np.abs(oracle.swdft2d(x, n0, n1, method=method) - ref).max() < 1e-12


@pytest.mark.parametrize("n0,n1", CASES)
def test_ternary_tree_matches_definition_and_counts_nodes(n0, n1):
    N0, N1 = n0 + 6, n1 + 7
    x = _x(n0 + 7 * n1, N0, N1)
    t, ops = oracle.tree2d_radix(x, n0, n1)
    assert np.abs(t - oracle.swdft2d(x, n0, n1, method="separable")).max() < 1e-12
    assert ops == N0 * N1 * (_nodes(n1) + n1 * _nodes(n0))


def test_binary_case_agrees_with_the_papers_tree():
    x = _x(5, 20, 24)
    a, ops_a = oracle.tree2d_radix(x, 8, 16)
    b, ops_b, _ = oracle.tree2d(x, 8, 16)
    assert ops_a == ops_b
    assert np.abs(a - b).max() < 1e-13


def test_ternary_level_one_is_the_three_point_dft():
    """n = 3 along dimension 1: the first level at p is the 3-point DFT of x[p-2..p]."""
    x = _x(9, 1, 12)
    a, _ = oracle.tree2d_radix(x, 1, 3, norm="none")
    for q in range(10):
        w = x[0, q:q + 3]
        expect = [sum(w[j] * np.exp(-2j * np.pi * j * k / 3) for j in range(3)) for k in range(3)]
        assert np.abs(a[0, q, 0] - np.array(expect)).max() < 1e-13


def test_rejects_other_radices():
    with pytest.raises(ValueError):
        oracle.tree2d_radix(_x(1, 10, 10), 5, 2)
    with pytest.raises(ValueError):
        oracle.tree2d_radix(_x(1, 10, 10), 6, 2)


RADIX_SRC = __import__("os").path.join(__import__("os").path.dirname(__import__("os").path.dirname(
    __import__("os").path.abspath(__file__))), "oracle", "swdft_radix_tree.c")

MUTANTS = [
    ("reversed_shift", "const int64_t q = p1 - (int64_t)(r1 - 1 - d) * s;", "const int64_t q = p1 - (int64_t)d * s;"),
    ("twiddle_without_stride", "const double *w = om0 + 2 * ((i0 * d * s) % n0);", "const double *w = om0 + 2 * ((i0 * d) % n0);"),
    ("wrong_parent_node", "(i0 % half) * n1 + i1);", "(i0 % size) * n1 + i1);"),
]


@pytest.mark.parametrize("name,orig,mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_radix_tree_mutant(tmp_path, name, orig, mut):
    import shutil
    import subprocess
    import sys
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    src = open(RADIX_SRC).read()
    # the constant-radix tree only (the mixed-radix function after it shares some lines)
    cut = src.index("int swt_tree2d_mixed_f64(") if "int swt_tree2d_mixed_f64(" in src else len(src)
    body, tail = src[:cut], src[cut:]
    assert body.count(orig) == 1, f"mutation site for {name} not found exactly once"
    (tmp_path / "m.c").write_text(body.replace(orig, mut) + tail)
    so = tmp_path / "libm.so"
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-o", str(so), str(tmp_path / "m.c"), "-lm"],
                   check=True, capture_output=True)
    x = _x(31, 15, 14)
    np.save(tmp_path / "x.npy", x)
    np.save(tmp_path / "ref.npy", _fft2_windows(x, 9, 3))
    child = f"""
import ctypes, math, numpy as np
lib = ctypes.CDLL({str(so)!r}); P = ctypes.c_void_p
lib.swt_tree2d_radix_f64.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_double, P, P]
x = np.ascontiguousarray(np.load({str(tmp_path / 'x.npy')!r})); ref = np.load({str(tmp_path / 'ref.npy')!r})
out = np.zeros(ref.shape, dtype=np.complex128)
rc = lib.swt_tree2d_radix_f64(x.ctypes.data, 15, 14, 9, 3, 1 / math.sqrt(27), out.ctypes.data, None)
print("PASSED_PIN" if rc == 0 and np.abs(out - ref).max() < 1e-12 else "CAUGHT")
"""
    res = subprocess.run([sys.executable, "-c", child], capture_output=True, text=True, timeout=120)
    assert "PASSED_PIN" not in res.stdout, f"mutant {name} passed the pin"
