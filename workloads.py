"""Seeded synthetic inputs for the 2D sliding window DFT, plus the error metric.

This module is shared by the FP64 oracle's tests and by the GPU path's tests and bench.
It holds no DFT arithmetic: it only draws arrays and compares results.

Every workload is drawn with ``numpy.random.default_rng(seed)`` (PCG64) in float64 and
rounded to float32; complex arrays draw their real and imaginary parts as one array of
shape (2, N0, N1).  The paper (arXiv 1707.08213) measures only "a 100x100 array" with no
value distribution (Section 4.5, Fig. 4), so the shapes below are the five workloads the
hot path is specified on, each named for what it is:

=========================  ===========================================================
``small_uniform_64``       64x64 float32 U[-1,1), seed 0; 8x8 windows
``sinusoids_512``          512x512 float32 N(0,1), seed 1, plus three 2D sinusoids;
                           32x32 windows (the benchmarked workload)
``complex_1024x2048``      1024x2048 complex64, re/im N(0,1), seed 2; 16x64 windows
``uneven_batch_256``       256 float32 images, sides from {128,256,512,1024}, U[-1,1),
                           seed 3; window per image from six shapes
``adjoint_batch_8``        8x256x256 float32 N(0,1), seed 4; 16x16 windows; loss mask
                           w ~ U[0,1) over (position, k0, k1) drawn after the images
``volume_128``             128x128x128 float32 N(0,1), seed 5; 8x8x8 windows (the
                           k-dimensional transform of Section 4.4, k = 3)
=========================  ===========================================================
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Tuple

import numpy as np

# window shapes the uneven batch draws from (n0, n1)
UNEVEN_WINDOWS: Tuple[Tuple[int, int], ...] = ((4, 4), (8, 8), (16, 16), (32, 32), (8, 32), (64, 16))
UNEVEN_SIDES: Tuple[int, ...] = (128, 256, 512, 1024)


@dataclasses.dataclass
class Workload:
    """One array (or a batch of arrays) and its window shape(s)."""
    name: str
    images: List[np.ndarray]          # each (N0, N1) float32 or complex64
    windows: List[Tuple[int, int]]    # (n0, n1) per image
    note: str = ""

    @property
    def batch(self) -> int:
        return len(self.images)

    def output_coeffs(self) -> int:
        tot = 0
        for x, (n0, n1) in zip(self.images, self.windows):
            tot += (x.shape[0] - n0 + 1) * (x.shape[1] - n1 + 1) * n0 * n1
        return tot


def _real(rng: np.random.Generator, shape, dist: str) -> np.ndarray:
    if dist == "uniform":
        return rng.uniform(-1.0, 1.0, size=shape)
    if dist == "normal":
        return rng.standard_normal(size=shape)
    raise ValueError(dist)


def random_array(seed: int, N0: int, N1: int, complex_input: bool = False,
                 dist: str = "normal") -> np.ndarray:
    """Generic seeded array used by the parity tests (float32 or complex64)."""
    rng = np.random.default_rng(seed)
    if complex_input:
        v = _real(rng, (2, N0, N1), dist)
        return (v[0] + 1j * v[1]).astype(np.complex64)
    return _real(rng, (N0, N1), dist).astype(np.float32)


def random_array_kd(seed: int, shape, complex_input: bool = False,
                    dist: str = "normal") -> np.ndarray:
    """Seeded array of any rank (complex: real and imaginary parts as one (2, *shape) draw)."""
    rng = np.random.default_rng(seed)
    shape = tuple(int(v) for v in shape)
    if complex_input:
        v = _real(rng, (2,) + shape, dist)
        return (v[0] + 1j * v[1]).astype(np.complex64)
    return _real(rng, shape, dist).astype(np.float32)


VOLUME_SHAPE = (128, 128, 128)
VOLUME_WINDOW = (8, 8, 8)


def volume_128() -> Tuple[np.ndarray, Tuple[int, int, int]]:
    """128x128x128 float32 N(0,1) (seed 5) and its 8x8x8 window: 121^3 positions x 512
    coefficients = 9.07e8 complex64 outputs (7.26 GB)."""
    return random_array_kd(5, VOLUME_SHAPE), VOLUME_WINDOW


def small_uniform_64() -> Workload:
    rng = np.random.default_rng(0)
    x = rng.uniform(-1.0, 1.0, size=(64, 64)).astype(np.float32)
    return Workload("small_uniform_64", [x], [(8, 8)], "64x64 f32 U[-1,1) seed 0, 8x8 windows")


def sinusoids_512() -> Workload:
    """N(0,1) noise plus three sinusoids A*cos(2*pi*(f0*r/N0 + f1*c/N1) + phi).

    Draw order: the noise, then per sinusoid (f0, f1, A, phi) with f0, f1 integers uniform
    in [1, N/2-1], A uniform in [0.5, 2], phi uniform in [0, 2*pi).
    """
    N = 512
    rng = np.random.default_rng(1)
    x = rng.standard_normal(size=(N, N))
    r = np.arange(N, dtype=np.float64)[:, None]
    c = np.arange(N, dtype=np.float64)[None, :]
    for _ in range(3):
        f0 = int(rng.integers(1, N // 2))
        f1 = int(rng.integers(1, N // 2))
        amp = float(rng.uniform(0.5, 2.0))
        phi = float(rng.uniform(0.0, 2.0 * math.pi))
        x = x + amp * np.cos(2.0 * math.pi * (f0 * r / N + f1 * c / N) + phi)
    return Workload("sinusoids_512", [x.astype(np.float32)], [(32, 32)],
                    "512x512 f32 N(0,1) seed 1 + 3 sinusoids, 32x32 windows")


def complex_1024x2048() -> Workload:
    rng = np.random.default_rng(2)
    v = rng.standard_normal(size=(2, 1024, 2048))
    x = (v[0] + 1j * v[1]).astype(np.complex64)
    return Workload("complex_1024x2048", [x], [(16, 64)],
                    "1024x2048 c64 re/im N(0,1) seed 2, 16x64 windows")


def uneven_batch_shapes(count: int = 256, seed: int = 3):
    """(sides, window indices) of the uneven batch, drawn before any pixel value."""
    rng = np.random.default_rng(seed)
    sides = rng.choice(np.array(UNEVEN_SIDES), size=(count, 2))
    widx = rng.integers(0, len(UNEVEN_WINDOWS), size=count)
    return rng, sides, widx


def uneven_batch_256(count: int = 256, seed: int = 3) -> Workload:
    rng, sides, widx = uneven_batch_shapes(count, seed)
    images, windows = [], []
    for i in range(count):
        N0, N1 = int(sides[i, 0]), int(sides[i, 1])
        images.append(rng.uniform(-1.0, 1.0, size=(N0, N1)).astype(np.float32))
        windows.append(UNEVEN_WINDOWS[int(widx[i])])
    return Workload("uneven_batch_256", images, windows,
                    f"{count} f32 images, sides in {UNEVEN_SIDES}, U[-1,1) seed {seed}, "
                    f"windows drawn from {UNEVEN_WINDOWS}")


def uneven_batch_output_coeffs(count: int = 256, seed: int = 3) -> int:
    """Output size of the uneven batch without drawing the pixels."""
    _, sides, widx = uneven_batch_shapes(count, seed)
    tot = 0
    for i in range(count):
        n0, n1 = UNEVEN_WINDOWS[int(widx[i])]
        tot += (int(sides[i, 0]) - n0 + 1) * (int(sides[i, 1]) - n1 + 1) * n0 * n1
    return tot


def adjoint_batch_8():
    """Images (8,256,256) f32 and the loss mask w (P0,P1,n0,n1) f32, both from seed 4."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal(size=(8, 256, 256)).astype(np.float32)
    n0 = n1 = 16
    P0 = P1 = 256 - 16 + 1
    w = rng.uniform(0.0, 1.0, size=(P0, P1, n0, n1)).astype(np.float32)
    return x, w, (n0, n1)


def paper_fig4_shapes():
    """The paper's only speed workload: a 100x100 array, square windows 4..64 (Fig. 4)."""
    return [(100, 100, n, n) for n in (4, 8, 16, 32, 64)]


# --------------------------------------------------------------------------------------
# error metric: max_k |a - ref| / ||x_w||_2 per window, on the unitary scale
# --------------------------------------------------------------------------------------

def window_sq_norms(x: np.ndarray, n0: int, n1: int) -> np.ndarray:
    """||x_w||_2^2 for every window (P0, P1), in float64 via 2D prefix sums."""
    a = np.abs(np.asarray(x, dtype=np.complex128)) ** 2
    S = np.zeros((a.shape[0] + 1, a.shape[1] + 1), dtype=np.float64)
    S[1:, 1:] = np.cumsum(np.cumsum(a, axis=0), axis=1)
    P0, P1 = a.shape[0] - n0 + 1, a.shape[1] - n1 + 1
    return (S[n0:n0 + P0, n1:n1 + P1] - S[:P0, n1:n1 + P1]
            - S[n0:n0 + P0, :P1] + S[:P0, :P1]).clip(min=0.0)


def window_sq_norms_at(x: np.ndarray, n0: int, n1: int, q0s, q1s) -> np.ndarray:
    xs = np.asarray(x, dtype=np.complex128)
    return np.array([np.sum(np.abs(xs[a:a + n0, b:b + n1]) ** 2) for a, b in zip(q0s, q1s)])


def window_sq_norms_kd(x: np.ndarray, n) -> np.ndarray:
    """||x_w||_2^2 for every window of a k-dimensional array (shape P_0..P_{k-1}), float64,
    by a sliding sum along each axis in turn."""
    a = np.abs(np.asarray(x, dtype=np.complex128)) ** 2
    for ax, w in enumerate(n):
        c = np.cumsum(a, axis=ax)
        zero = np.zeros_like(np.take(c, [0], axis=ax))
        c = np.concatenate([zero, c], axis=ax)
        L = a.shape[ax] - w + 1
        a = np.take(c, range(w, w + L), axis=ax) - np.take(c, range(0, L), axis=ax)
    return a.clip(min=0.0)


def window_sq_norms_kd_at(x: np.ndarray, n, qs) -> np.ndarray:
    xs = np.asarray(x, dtype=np.complex128)
    out = []
    for q in np.asarray(qs).reshape(-1, xs.ndim):
        sl = tuple(slice(int(a), int(a) + int(b)) for a, b in zip(q, n))
        out.append(np.sum(np.abs(xs[sl]) ** 2))
    return np.array(out)


def normalised_error(a: np.ndarray, ref: np.ndarray, sq_norms: np.ndarray,
                     to_unitary: float = 1.0):
    """(max_w e_w, rms) with e_w = max_k |a-ref| / ||x_w||_2 (unitary scale).

    ``a`` and ``ref`` have shape (..., n0, n1) with the leading axes matching ``sq_norms``.
    ``to_unitary`` rescales outputs computed in another normalisation.  A window of zero
    norm must be exactly zero: its error is the absolute difference (never divided).
    """
    d = np.abs(np.asarray(a, dtype=np.complex128) - np.asarray(ref, dtype=np.complex128))
    d = d * to_unitary
    flat = d.reshape(sq_norms.shape + (-1,))
    nrm = np.sqrt(sq_norms)[..., None]
    safe = np.where(nrm > 0, nrm, 1.0)
    rel = np.where(nrm > 0, flat / safe, flat)
    return float(rel.max(initial=0.0)), float(math.sqrt(np.mean(rel ** 2)) if rel.size else 0.0)


def adjoint_pixel_norms(G: np.ndarray, N0: int, N1: int) -> np.ndarray:
    """sqrt(sum over windows w containing pixel (r,c) of ||G_w||_2^2), shape (N0, N1).

    With the unitary scale, each window adds at most ||G_w||_2 to |(A^H G)[r,c]|, so this is
    the natural per-pixel scale of an adjoint's error (the analogue of ||x_w||_2 forward).
    """
    Gs = np.asarray(G)
    P0, P1, n0, n1 = Gs.shape
    e = np.sum(np.abs(Gs.astype(np.complex128)) ** 2, axis=(2, 3))
    S = np.zeros((P0 + 1, P1 + 1))
    S[1:, 1:] = np.cumsum(np.cumsum(e, axis=0), axis=1)
    r = np.arange(N0)
    c = np.arange(N1)
    r_lo = np.clip(r - n0 + 1, 0, P0)[:, None]
    r_hi = np.clip(r + 1, 0, P0)[:, None]
    c_lo = np.clip(c - n1 + 1, 0, P1)[None, :]
    c_hi = np.clip(c + 1, 0, P1)[None, :]
    box = S[r_hi, c_hi] - S[r_lo, c_hi] - S[r_hi, c_lo] + S[r_lo, c_lo]
    return np.sqrt(np.clip(box, 0.0, None))


def adjoint_error(g: np.ndarray, ref: np.ndarray, pixel_norms: np.ndarray) -> float:
    """max over pixels of |g - ref| / pixel norm (absolute where the norm is 0)."""
    d = np.abs(np.asarray(g, dtype=np.complex128) - np.asarray(ref, dtype=np.complex128))
    return float(np.max(np.where(pixel_norms > 0, d / np.where(pixel_norms > 0, pixel_norms, 1), d)))
