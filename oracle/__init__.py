"""FP64 CPU oracle for the 2D sliding window DFT (arXiv 1707.08213, Section 4.1, Eq. 2).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the cpu_baseline
leg of ``bench.py`` import this package.  The GPU library shares no code with it.

Contents (plain C in ``swdft2d_oracle.c`` / ``swdft2d_tree_ref.c``, loaded through ctypes):

* :func:`swdft2d` -- every window by the definition (``method="direct"``, the double sum
  of Eq. 2) or by the row-column factorisation of Section 4.2 (``method="separable"``,
  the same sum reordered).
* :func:`swdft2d_windows` -- selected windows only (for full-size parity by sampling).
* :func:`swdft2d_adjoint` / :func:`swdft2d_adjoint_pixels` -- the explicit adjoint A^H.
* :func:`tree2d` -- the paper's tree (Section 4.2 equations, Section 4.3 loop order) in
  FP64 or FP32, with the node-operation count of Eq. windowops and level dumps.
* :func:`swdftkd` / :func:`swdftkd_windows` -- the k-dimensional transform of Section 4.4
  (k <= 4) by its definition, direct or axis by axis (``swdftkd_oracle.c``).
* :func:`treekd` -- the tree of Eq. kdfswft in FP64, with its node-operation count.
* :func:`tree2d_radix` -- the 2D tree with radix-2 or radix-3 levels per axis (the ternary
  trees Section 5 mentions; recurrence derived in ``swdft_radix_tree.c``), FP64.
* :func:`tree2d_mixed` -- the same tree with a radix chosen per level (2 or 3, any order),
  for windows of 2^a 3^b samples along an axis, FP64.

Arrays are numpy; outputs are complex128 with layout [q0][q1][k0][k1], where window q
covers rows q0..q0+n0-1 and columns q1..q1+n1-1 (the paper's window end p = q + n - 1).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["swdft2d_oracle.c", "swdft2d_tree_ref.c", "swdftkd_oracle.c", "swdft_radix_tree.c"]
_lib = None

NORMS = ("unitary", "none", "inv_n")


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the C oracle into ``oracle/_build/liboracle.so`` with gcc (OpenMP if present)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(s) for s in srcs)):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp] + srcs + ["-lm"]
    for extra in (["-fopenmp"], []):
        cmd = base[:2] + extra + base[2:]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode == 0:
            os.replace(tmp, _LIB_PATH)
            if verbose:
                print(" ".join(cmd))
            return _LIB_PATH
    raise RuntimeError("oracle build failed:\n" + res.stderr)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
    P = ctypes.c_void_p
    lib.swo_swdft2d.argtypes = [P, i64, i64, i32, i32, d, i32, i32, P]
    lib.swo_swdft2d_windows.argtypes = [P, i64, i64, i32, i32, d, i32, i64, P, P, i32, P]
    lib.swo_swdft2d_adjoint.argtypes = [P, i64, i64, i32, i32, d, i32, P]
    lib.swo_swdft2d_adjoint_pixels.argtypes = [P, i64, i64, i32, i32, d, i64, P, P, i32, P]
    lib.swt_tree2d_f64.argtypes = [P, i64, i64, i32, i32, d, P, P, i32, P, i32]
    lib.swt_tree2d_f32.argtypes = [P, i64, i64, i32, i32, ctypes.c_float, P, P, i32, P, i32]
    lib.swo_swdftkd.argtypes = [P, i32, P, P, d, i32, i32, P]
    lib.swo_swdftkd_windows.argtypes = [P, i32, P, P, d, i32, i64, P, i32, P]
    lib.swt_treekd_f64.argtypes = [P, i32, P, P, d, P, P]
    lib.swt_tree2d_radix_f64.argtypes = [P, i64, i64, i32, i32, d, P, P]
    lib.swt_tree2d_mixed_f64.argtypes = [P, i64, i64, P, i32, P, i32, d, P, P]
    for f in ("swo_swdft2d", "swo_swdft2d_windows", "swo_swdft2d_adjoint",
              "swo_swdft2d_adjoint_pixels", "swt_tree2d_f64", "swt_tree2d_f32",
              "swo_openmp_available", "swo_swdftkd", "swo_swdftkd_windows", "swt_treekd_f64",
              "swt_tree2d_radix_f64", "swt_tree2d_mixed_f64"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def openmp_available() -> bool:
    return bool(_load().swo_openmp_available())


def scale_for(norm: str, n0: int, n1: int) -> float:
    """Output scale: Eq. 2's 1/sqrt(n0 n1) ("unitary"), 1 ("none"), 1/(n0 n1) ("inv_n")."""
    if norm == "unitary":
        return 1.0 / math.sqrt(n0 * n1)
    if norm == "none":
        return 1.0
    if norm == "inv_n":
        return 1.0 / (n0 * n1)
    raise ValueError(f"unknown normalisation {norm!r}")


def _as_c128(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x), dtype=np.complex128)


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


_METHODS = {"direct": 0, "separable": 1}


def swdft2d(x, n0: int, n1: int, norm: str = "unitary", method: str = "direct",
            threads: int = 1) -> np.ndarray:
    """All windows of a 2D array, (P0, P1, n0, n1) complex128."""
    xs = _as_c128(x)
    N0, N1 = xs.shape
    P0, P1 = N0 - n0 + 1, N1 - n1 + 1
    if P0 < 1 or P1 < 1 or n0 < 1 or n1 < 1:
        raise ValueError("window larger than the array")
    out = np.empty((P0, P1, n0, n1), dtype=np.complex128)
    _check(_load().swo_swdft2d(_ptr(xs), N0, N1, n0, n1, scale_for(norm, n0, n1),
                               _METHODS[method], threads, _ptr(out)), "swdft2d")
    return out


def swdft2d_windows(x, n0: int, n1: int, q0s: Sequence[int], q1s: Sequence[int],
                    norm: str = "unitary", method: str = "separable",
                    threads: int = 1) -> np.ndarray:
    """Selected windows (q0s[i], q1s[i]) -> (len, n0, n1) complex128."""
    xs = _as_c128(x)
    N0, N1 = xs.shape
    a = np.ascontiguousarray(q0s, dtype=np.int64)
    b = np.ascontiguousarray(q1s, dtype=np.int64)
    if a.shape != b.shape:
        raise ValueError("q0s and q1s differ in length")
    out = np.empty((a.size, n0, n1), dtype=np.complex128)
    _check(_load().swo_swdft2d_windows(_ptr(xs), N0, N1, n0, n1, scale_for(norm, n0, n1),
                                       _METHODS[method], a.size, _ptr(a), _ptr(b), threads,
                                       _ptr(out)), "swdft2d_windows")
    return out


def swdft2d_adjoint(G, N0: int, N1: int, norm: str = "unitary",
                    method: str = "separable") -> np.ndarray:
    """A^H G for G of shape (P0, P1, n0, n1) -> (N0, N1) complex128."""
    Gs = _as_c128(G)
    P0, P1, n0, n1 = Gs.shape
    if (P0, P1) != (N0 - n0 + 1, N1 - n1 + 1):
        raise ValueError("G does not match the array shape")
    g = np.empty((N0, N1), dtype=np.complex128)
    _check(_load().swo_swdft2d_adjoint(_ptr(Gs), N0, N1, n0, n1, scale_for(norm, n0, n1),
                                       _METHODS[method], _ptr(g)), "swdft2d_adjoint")
    return g


def swdft2d_adjoint_pixels(G, N0: int, N1: int, rs, cs, norm: str = "unitary",
                           threads: int = 1) -> np.ndarray:
    """(A^H G)[rs[i], cs[i]] by the direct conjugate sum -> (len,) complex128."""
    Gs = _as_c128(G)
    P0, P1, n0, n1 = Gs.shape
    if (P0, P1) != (N0 - n0 + 1, N1 - n1 + 1):
        raise ValueError("G does not match the array shape")
    a = np.ascontiguousarray(rs, dtype=np.int64)
    b = np.ascontiguousarray(cs, dtype=np.int64)
    out = np.empty(a.size, dtype=np.complex128)
    _check(_load().swo_swdft2d_adjoint_pixels(_ptr(Gs), N0, N1, n0, n1,
                                              scale_for(norm, n0, n1), a.size, _ptr(a),
                                              _ptr(b), threads, _ptr(out)),
           "swdft2d_adjoint_pixels")
    return out


def tree2d(x, n0: int, n1: int, norm: str = "unitary", precision: str = "f64",
           dump_level: Optional[int] = None, threads: int = 1):
    """The paper's tree.  Returns (out, opcount, dump).

    out: (P0, P1, n0, n1) complex (complex128 for f64, complex64 for f32);
    opcount: node evaluations (complex multiply + add each);
    dump: the (N0, N1, n0*n1) buffer of level ``dump_level`` or None.
    """
    if precision == "f64":
        xs = _as_c128(x)
        ctype, fn = np.complex128, _load().swt_tree2d_f64
        c = ctypes.c_double(scale_for(norm, n0, n1))
    elif precision == "f32":
        xs = np.ascontiguousarray(np.asarray(x), dtype=np.complex64)
        ctype, fn = np.complex64, _load().swt_tree2d_f32
        c = ctypes.c_float(scale_for(norm, n0, n1))
    else:
        raise ValueError(precision)
    N0, N1 = xs.shape
    out = np.empty((N0 - n0 + 1, N1 - n1 + 1, n0, n1), dtype=ctype)
    ops = ctypes.c_int64(0)
    dump = None
    if dump_level is not None:
        dump = np.empty((N0, N1, n0 * n1), dtype=ctype)
    rc = fn(_ptr(xs), N0, N1, n0, n1, c, _ptr(out), ctypes.byref(ops),
            -1 if dump_level is None else int(dump_level),
            None if dump is None else _ptr(dump), threads)
    _check(rc, "tree2d")
    return out, int(ops.value), dump


# ------------------------------------------------------------------ k dimensions (Section 4.4)

MAX_DIMS = 4


def scale_for_kd(norm: str, n: Sequence[int]) -> float:
    """Eq. 2's scale in k dimensions: 1/sqrt(prod n) ("unitary"), 1, or 1/prod n."""
    nn = int(np.prod(n))
    return {"unitary": 1.0 / math.sqrt(nn), "none": 1.0, "inv_n": 1.0 / nn}[norm]


def _kd_args(x, n):
    xs = _as_c128(x)
    K = xs.ndim
    if K < 1 or K > MAX_DIMS or len(n) != K:
        raise ValueError("need 1..4 dimensions and one window length per dimension")
    N = np.ascontiguousarray(xs.shape, dtype=np.int64)
    nw = np.ascontiguousarray(n, dtype=np.int32)
    if np.any(nw < 1) or np.any(nw > N):
        raise ValueError("window larger than the array")
    return xs, K, N, nw


def swdftkd(x, n: Sequence[int], norm: str = "unitary", method: str = "direct",
            threads: int = 1) -> np.ndarray:
    """All windows of a k-dimensional array: (P_0..P_{k-1}, n_0..n_{k-1}) complex128."""
    xs, K, N, nw = _kd_args(x, n)
    P = tuple(int(a - b + 1) for a, b in zip(N, nw))
    out = np.empty(P + tuple(int(v) for v in nw), dtype=np.complex128)
    _check(_load().swo_swdftkd(_ptr(xs), K, _ptr(N), _ptr(nw), scale_for_kd(norm, nw),
                               _METHODS[method], threads, _ptr(out)), "swdftkd")
    return out


def swdftkd_windows(x, n: Sequence[int], qs, norm: str = "unitary", method: str = "separable",
                    threads: int = 1) -> np.ndarray:
    """Selected windows, qs of shape (count, k) first samples -> (count, n_0..) complex128."""
    xs, K, N, nw = _kd_args(x, n)
    q = np.ascontiguousarray(qs, dtype=np.int64).reshape(-1, K)
    out = np.empty((q.shape[0],) + tuple(int(v) for v in nw), dtype=np.complex128)
    _check(_load().swo_swdftkd_windows(_ptr(xs), K, _ptr(N), _ptr(nw), scale_for_kd(norm, nw),
                                       _METHODS[method], q.shape[0], _ptr(q), threads,
                                       _ptr(out)), "swdftkd_windows")
    return out


def treekd(x, n: Sequence[int], norm: str = "unitary"):
    """The tree of Eq. kdfswft in FP64.  Returns (out, opcount) like :func:`swdftkd`."""
    xs, K, N, nw = _kd_args(x, n)
    P = tuple(int(a - b + 1) for a, b in zip(N, nw))
    out = np.empty(P + tuple(int(v) for v in nw), dtype=np.complex128)
    ops = ctypes.c_int64(0)
    _check(_load().swt_treekd_f64(_ptr(xs), K, _ptr(N), _ptr(nw), scale_for_kd(norm, nw),
                                  _ptr(out), ctypes.byref(ops)), "treekd")
    return out, int(ops.value)


def tree2d_radix(x, n0: int, n1: int, norm: str = "unitary"):
    """The 2D tree with radix-2 or radix-3 levels per axis (n_i a power of 2 or of 3), FP64.
    Returns (out (P0, P1, n0, n1) complex128, nodes evaluated)."""
    xs = _as_c128(x)
    N0, N1 = xs.shape
    out = np.empty((N0 - n0 + 1, N1 - n1 + 1, n0, n1), dtype=np.complex128)
    ops = ctypes.c_int64(0)
    _check(_load().swt_tree2d_radix_f64(_ptr(xs), N0, N1, n0, n1, scale_for(norm, n0, n1),
                                        _ptr(out), ctypes.byref(ops)), "tree2d_radix")
    return out, int(ops.value)


def tree2d_mixed(x, radices0: Sequence[int], radices1: Sequence[int], norm: str = "unitary"):
    """The 2D tree with per-level radices (each 2 or 3, in level order) along each axis: the
    windows are n0 = prod(radices0) by n1 = prod(radices1), FP64.  Returns (out (P0, P1, n0,
    n1) complex128, nodes evaluated)."""
    xs = _as_c128(x)
    N0, N1 = xs.shape
    r0 = np.ascontiguousarray(list(radices0) or [0], dtype=np.int32)
    r1 = np.ascontiguousarray(list(radices1) or [0], dtype=np.int32)
    n0, n1 = int(np.prod(radices0)) if radices0 else 1, int(np.prod(radices1)) if radices1 else 1
    out = np.empty((N0 - n0 + 1, N1 - n1 + 1, n0, n1), dtype=np.complex128)
    ops = ctypes.c_int64(0)
    _check(_load().swt_tree2d_mixed_f64(_ptr(xs), N0, N1, _ptr(r0), len(radices0), _ptr(r1), len(radices1),
                                        scale_for(norm, n0, n1), _ptr(out), ctypes.byref(ops)), "tree2d_mixed")
    return out, int(ops.value)

