"""GB300-native 2D Tree Sliding Window DFT (Richardson & Eddy, arXiv 1707.08213).

For an N0 x N1 array and n0 x n1 windows (powers of two) this computes the 2D DFT of every
window position (Section 4.1, Eq. 2) with the paper's tree of radix-2 butterflies shared
between overlapping windows (Section 4.2), in hand-written sm_103a CUDA kernels behind the
C ABI of ``include/swdft2d.h``.  PyTorch supplies device memory and streams only.

    import torch, paper_1707_08213_gb300 as sw
    a = sw.swdft2d(x_cuda, 32, 32)        # (P0, P1, n0, n1) complex64

Output layout is [q0][q1][k0][k1] with q_i the window's first row/column; the default
scale is Eq. 2's 1/sqrt(n0 n1).  ``TransformKD`` / ``swdftkd`` give the k-dimensional
transform of Section 4.4 (k <= 4) through ``include/swdftkd.h``; ``SlidingStream`` the
streaming form (rows pushed over time, ``include/swdftstream.h``).
"""
from __future__ import annotations

from typing import Dict, Sequence, Tuple

import torch

from . import _native
from ._native import (ALGOS, C64, FLAG_AUTOTUNE, FLAG_GRAPH, FLAG_HOST_IO, FLAG_PERSISTENT, NORMS, R32, Plan,
                      PlanKD, StreamPlan, SwdftError, status_string, version)

__all__ = ["swdft2d", "swdft2d_adjoint", "Transform", "Plan", "SwdftError", "SWDFT2dFunction",
           "status_string", "version", "FLAG_AUTOTUNE", "FLAG_GRAPH", "FLAG_HOST_IO", "FLAG_PERSISTENT",
           "TransformKD", "PlanKD", "swdftkd", "SlidingStream", "StreamPlan"]


def _dtype_code(x: torch.Tensor) -> int:
    if x.dtype == torch.float32:
        return R32
    if x.dtype == torch.complex64:
        return C64
    raise TypeError(f"input must be float32 or complex64, got {x.dtype}")


def _stream_ptr(device: torch.device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


class Transform:
    """A plan for a fixed list of input shapes plus its workspace on one CUDA device."""

    def __init__(self, shapes: Sequence[Tuple[int, int, int, int, int]], norm: str = "unitary",
                 algo: str = "tree", flags: int = 0, device=None,
                 bands: Sequence[Tuple[int, int]] = None, pos: str = "start"):
        """shapes: (N0, N1, n0, n1, dtype_code) per array; bands: optional (row_begin,
        row_end) of output window rows per array, in the ``pos`` convention."""
        spec = []
        for i, (N0, N1, n0, n1, dt) in enumerate(shapes):
            d = dict(N0=N0, N1=N1, n0=n0, n1=n1, dtype=dt)
            if bands is not None and bands[i] is not None:
                d["row_begin"], d["row_end"] = bands[i]
            spec.append(d)
        self.plan = Plan(spec, norm=norm, pos=pos, algo=algo, flags=flags)
        self.shapes = [tuple(s) for s in shapes]
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        ws = self.plan.workspace_size()
        self.workspace = torch.empty(max(ws, 1), dtype=torch.uint8, device=self.device)
        self._ws_ptr = self.workspace.data_ptr() if ws > 0 else 0

    def output_shapes(self):
        return [self.plan.output_shape(i) for i in range(len(self.shapes))]

    def empty_outputs(self):
        return [torch.empty(s, dtype=torch.complex64, device=self.device)
                for s in self.output_shapes()]

    def _check_inputs(self, xs):
        if len(xs) != len(self.shapes):
            raise ValueError("wrong number of arrays")
        for x, (N0, N1, _, _, dt) in zip(xs, self.shapes):
            if not x.is_cuda or x.device != self.device:
                raise ValueError("inputs must be CUDA tensors on the plan's device")
            if tuple(x.shape) != (N0, N1) or _dtype_code(x) != dt or not x.is_contiguous():
                raise ValueError("input does not match the planned shape/dtype or is not contiguous")

    def forward(self, xs, outs=None):
        self._check_inputs(xs)
        outs = self.empty_outputs() if outs is None else outs
        self.plan.execute([x.data_ptr() for x in xs], [o.data_ptr() for o in outs],
                          self._ws_ptr, _stream_ptr(self.device))
        return outs

    def adjoint(self, gouts, gins=None):
        if gins is None:
            gins = [torch.empty((N0, N1), dtype=torch.float32 if dt == R32 else torch.complex64,
                                device=self.device) for (N0, N1, _, _, dt) in self.shapes]
        self.plan.execute_adjoint([g.data_ptr() for g in gouts], [g.data_ptr() for g in gins],
                                  self._ws_ptr, _stream_ptr(self.device))
        return gins

    def autotune(self, xs, outs=None):
        self._check_inputs(xs)
        outs = self.empty_outputs() if outs is None else outs
        self.plan.autotune([x.data_ptr() for x in xs], [o.data_ptr() for o in outs],
                           self._ws_ptr, _stream_ptr(self.device))
        return outs


_CACHE: Dict[tuple, Transform] = {}


def _transform_for(x: torch.Tensor, n0: int, n1: int, norm: str, algo: str) -> Transform:
    key = (x.device, tuple(x.shape), x.dtype, n0, n1, norm, algo)
    t = _CACHE.get(key)
    if t is None:
        t = Transform([(x.shape[0], x.shape[1], n0, n1, _dtype_code(x))], norm=norm,
                      algo=algo, device=x.device)
        _CACHE[key] = t
    return t


def swdft2d(x: torch.Tensor, n0: int, n1: int, norm: str = "unitary",
            algo: str = "tree") -> torch.Tensor:
    """2D sliding window DFT of one CUDA array -> (P0, P1, n0, n1) complex64."""
    if x.dim() != 2:
        raise ValueError("x must be 2D")
    x = x.contiguous()
    return _transform_for(x, n0, n1, norm, algo).forward([x])[0]


def swdft2d_adjoint(g: torch.Tensor, N0: int, N1: int, complex_input: bool = False,
                    norm: str = "unitary") -> torch.Tensor:
    """A^H g for g of shape (P0, P1, n0, n1) complex64 -> (N0, N1) float32 (real input's
    gradient, Re A^H g) or complex64."""
    n0, n1 = int(g.shape[2]), int(g.shape[3])
    proto = torch.empty((N0, N1), dtype=torch.complex64 if complex_input else torch.float32,
                        device=g.device)
    t = _transform_for(proto, n0, n1, norm, "tree")
    return t.adjoint([g.contiguous()])[0]


class SWDFT2dFunction(torch.autograd.Function):
    """y = swdft2d(x); backward applies the hand-written adjoint kernel A^H."""

    @staticmethod
    def forward(ctx, x, n0: int, n1: int, norm: str = "unitary"):
        ctx.shape = (x.shape[0], x.shape[1], x.is_complex(), n0, n1, norm)
        return swdft2d(x, n0, n1, norm)

    @staticmethod
    def backward(ctx, grad):
        N0, N1, cplx, n0, n1, norm = ctx.shape
        return swdft2d_adjoint(grad, N0, N1, complex_input=cplx, norm=norm), None, None, None


class TransformKD:
    """A k-dimensional plan (Section 4.4, k <= 4) plus its workspace on one CUDA device."""

    def __init__(self, N: Sequence[int], n: Sequence[int], dtype: int = R32,
                 norm: str = "unitary", device=None):
        self.plan = PlanKD(N, n, dtype=dtype, norm=norm)
        self.N, self.n, self.dtype = tuple(int(v) for v in N), tuple(int(v) for v in n), dtype
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        ws = self.plan.workspace_size()
        self.workspace = torch.empty(max(ws, 1), dtype=torch.uint8, device=self.device)
        self._ws_ptr = self.workspace.data_ptr() if ws > 0 else 0

    def output_shape(self):
        return self.plan.output_shape()

    def empty_output(self):
        return torch.empty(self.output_shape(), dtype=torch.complex64, device=self.device)

    def forward(self, x: torch.Tensor, out: torch.Tensor = None) -> torch.Tensor:
        if not x.is_cuda or x.device != self.device or tuple(x.shape) != self.N \
                or _dtype_code(x) != self.dtype or not x.is_contiguous():
            raise ValueError("input does not match the planned shape/dtype/device or is not contiguous")
        out = self.empty_output() if out is None else out
        if tuple(out.shape) != self.output_shape() or out.dtype != torch.complex64 \
                or not out.is_contiguous() or out.device != self.device:
            raise ValueError("output must be a contiguous complex64 tensor of the output shape")
        self.plan.execute(x.data_ptr(), out.data_ptr(), self._ws_ptr, _stream_ptr(self.device))
        return out


_CACHE_KD: Dict[tuple, TransformKD] = {}


def swdftkd(x: torch.Tensor, n: Sequence[int], norm: str = "unitary") -> torch.Tensor:
    """k-dimensional sliding window DFT of one CUDA array (k = x.dim() <= 4)
    -> (P_0, .., P_{k-1}, n_0, .., n_{k-1}) complex64."""
    x = x.contiguous()
    key = (x.device, tuple(x.shape), x.dtype, tuple(n), norm)
    t = _CACHE_KD.get(key)
    if t is None:
        t = TransformKD(tuple(x.shape), n, dtype=_dtype_code(x), norm=norm, device=x.device)
        _CACHE_KD[key] = t
    return t.forward(x)


class SlidingStream:
    """Rows of an N1-wide array pushed over time; each push returns the window rows they
    complete, (rows, P1, n0, n1) complex64, identical to the same rows of one transform of
    everything pushed so far (Section 4.3's real-time order)."""

    def __init__(self, N1: int, n0: int, n1: int, dtype: int = R32, norm: str = "unitary",
                 max_rows: int = 64, device=None):
        self.plan = StreamPlan(N1, n0, n1, dtype=dtype, norm=norm, max_rows=max_rows)
        self.N1, self.n0, self.n1, self.dtype, self.max_rows = N1, n0, n1, dtype, max_rows
        self.P1 = N1 - n1 + 1
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        self.state = torch.empty(max(self.plan.state_size(), 1), dtype=torch.uint8, device=self.device)

    def push(self, rows: torch.Tensor, out: torch.Tensor = None):
        """rows: (R, N1) float32 / complex64 on the stream's device.  Returns (q0 of the first
        window row, tensor (rows_out, P1, n0, n1))."""
        if rows.dim() != 2 or rows.shape[1] != self.N1 or _dtype_code(rows) != self.dtype \
                or not rows.is_cuda or rows.device != self.device or rows.stride(1) != 1:
            raise ValueError("rows must be (R, N1) on the stream's device with the planned dtype")
        R = int(rows.shape[0])
        seen = self.plan.rows_seen()
        hist = min(seen, self.n0 - 1)
        nout = max(0, hist + R - (self.n0 - 1))
        if out is None:
            out = torch.empty((nout, self.P1, self.n0, self.n1), dtype=torch.complex64, device=self.device)
        elif tuple(out.shape) != (nout, self.P1, self.n0, self.n1) or not out.is_contiguous():
            raise ValueError("out must be a contiguous (rows_out, P1, n0, n1) complex64 tensor")
        n, first = self.plan.push(rows.data_ptr(), R, rows.stride(0), out.data_ptr() if nout else 0,
                                  self.state.data_ptr(), _stream_ptr(self.device))
        assert n == nout
        return first, out

    def reset(self):
        self.plan.reset()
