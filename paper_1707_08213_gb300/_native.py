"""ctypes binding of the C ABI in include/swdft2d.h, include/swdftkd.h and
include/swdftstream.h (argument marshalling only).

Every step of the transform runs in the CUDA library ``_lib/libswdft2d.so``; this module
only converts Python values to the plain pointers and sizes the ABI takes.  There is no
CPU fallback: if the library is missing, importing it raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libswdft2d.so")

# status codes (swdft_status)
OK = 0
ERR_INVALID_ARG = -1
ERR_NOT_POW2 = -2
ERR_WINDOW_TOO_LARGE = -3
ERR_UNSUPPORTED = -4
ERR_OOM = -5
ERR_CUDA = -6
ERR_DEVICE_TIMEOUT = -7
ERR_WORKSPACE = -8

R32, C64 = 0, 1
NORMS = {"unitary": 0, "none": 1, "inv_n": 2}
POS = {"start": 0, "end": 1}
ALGOS = {"auto": 0, "tree": 1, "tc_bf16x3": 2, "tc_bf16": 3, "tc_f16_scaled": 4, "tc_f16": 5}
ALGO_NAMES = {v: k for k, v in ALGOS.items()}
FLAG_GRAPH, FLAG_HOST_IO, FLAG_PERSISTENT, FLAG_AUTOTUNE = 1, 2, 4, 8
FORM_NAMES = {0: "pipelined", 1: "fused_group", 2: "per_array"}

# every symbol include/*.h declare
EXPORTS = (
    "swdft2d_plan", "swdft2d_output_shape", "swdft2d_workspace_size", "swdft2d_get_algo",
    "swdft2d_get_form",
    "swdft2d_execute", "swdft2d_execute_adjoint", "swdft2d_execute_host", "swdft2d_autotune",
    "swdft2d_launch_count", "swdft2d_destroy", "swdft2d_status_string", "swdft2d_version",
    "swdft2d_load_tuning",
    "swdft2d_execute_stage", "swdft2d_set_tree_config", "swdft2d_execute_static_scratch",
    "swdft2d_check_device", "swdft2d_inject_alloc_failure", "swdft2d_selftest_wait_timeout",
    "swdft2d_debug_batch_wait",
    "swdftkd_plan", "swdftkd_output_shape", "swdftkd_workspace_size", "swdftkd_launch_count",
    "swdftkd_execute", "swdftkd_destroy",
    "swdft2d_stream_create", "swdft2d_stream_state_size", "swdft2d_stream_push",
    "swdft2d_stream_rows_seen", "swdft2d_stream_reset", "swdft2d_stream_destroy",
)
KD_MAX_DIMS = 4


class SwdftError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


class Shape(ctypes.Structure):
    _fields_ = [("N0", ctypes.c_int64), ("N1", ctypes.c_int64), ("ld", ctypes.c_int64),
                ("n0", ctypes.c_int32), ("n1", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("row_begin", ctypes.c_int64),
                ("row_end", ctypes.c_int64)]


class ShapeKD(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("N", ctypes.c_int64 * KD_MAX_DIMS), ("n", ctypes.c_int32 * KD_MAX_DIMS)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} is missing "
                          "(run __graft_entry__.build() or paper_1707_08213_gb300/build.py)")
    lib = ctypes.CDLL(LIB_PATH)
    P, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "swdft2d_plan": ([ctypes.POINTER(P), i32, ctypes.POINTER(Shape), i32, i32, i32, u32], i32),
        "swdft2d_output_shape": ([P, i32, ctypes.POINTER(i64)], i32),
        "swdft2d_workspace_size": ([P, ctypes.POINTER(ctypes.c_size_t)], i32),
        "swdft2d_get_algo": ([P, ctypes.POINTER(i32)], i32),
        "swdft2d_get_form": ([P, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)], i32),
        "swdft2d_execute": ([P, PP, PP, P, P], i32),
        "swdft2d_execute_adjoint": ([P, PP, PP, P, P], i32),
        "swdft2d_execute_host": ([P, PP, PP, P], i32),
        "swdft2d_autotune": ([P, PP, PP, P, P], i32),
        "swdft2d_launch_count": ([P, i32, ctypes.POINTER(i32)], i32),
        "swdft2d_load_tuning": ([P, ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(i32)], i32),
        "swdft2d_execute_stage": ([P, i32, PP, PP, P, P], i32),
        "swdft2d_set_tree_config": ([P, i32, i32, i64, i32, i64, i32, i32], i32),
        "swdft2d_execute_static_scratch": ([P, i64, i64, i64, i32, i32, i32, i32, P, P], i32),
        "swdft2d_check_device": ([], i32),
        "swdft2d_inject_alloc_failure": ([i64], i32),
        "swdft2d_selftest_wait_timeout": ([i32, P], i32),
        "swdft2d_debug_batch_wait": ([i64, i32], i32),
        "swdft2d_destroy": ([P], i32),
        "swdft2d_status_string": ([i32], ctypes.c_char_p),
        "swdft2d_version": ([], i32),
        "swdftkd_plan": ([ctypes.POINTER(P), ctypes.POINTER(ShapeKD), i32, u32], i32),
        "swdftkd_output_shape": ([P, ctypes.POINTER(i64)], i32),
        "swdftkd_workspace_size": ([P, ctypes.POINTER(ctypes.c_size_t)], i32),
        "swdftkd_launch_count": ([P, ctypes.POINTER(i32)], i32),
        "swdftkd_execute": ([P, P, P, P, P], i32),
        "swdftkd_destroy": ([P], i32),
        "swdft2d_stream_create": ([ctypes.POINTER(P), i64, i32, i32, i32, i32, i64], i32),
        "swdft2d_stream_state_size": ([P, ctypes.POINTER(ctypes.c_size_t)], i32),
        "swdft2d_stream_push": ([P, P, i64, i64, P, P, ctypes.POINTER(i64), ctypes.POINTER(i64), P], i32),
        "swdft2d_stream_rows_seen": ([P, ctypes.POINTER(i64)], i32),
        "swdft2d_stream_reset": ([P], i32),
        "swdft2d_stream_destroy": ([P], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


lib = _load()


def status_string(status: int) -> str:
    return lib.swdft2d_status_string(int(status)).decode()


def _check(status: int, what: str):
    if status != OK:
        raise SwdftError(status, what)


def _ptr_array(ptrs: Sequence[int]):
    arr = (ctypes.c_void_p * len(ptrs))()
    for i, p in enumerate(ptrs):
        arr[i] = ctypes.c_void_p(int(p)) if p else None
    return arr


class Plan:
    """An owned swdft2d plan handle (one or more arrays)."""

    def __init__(self, shapes: Sequence[dict], norm: str = "unitary", pos: str = "start",
                 algo: str = "tree", flags: int = 0):
        arr = (Shape * len(shapes))()
        for i, s in enumerate(shapes):
            arr[i] = Shape(int(s["N0"]), int(s["N1"]), int(s.get("ld", 0)), int(s["n0"]),
                           int(s["n1"]), int(s.get("dtype", R32)), 0,
                           int(s.get("row_begin", 0)), int(s.get("row_end", 0)))
        h = ctypes.c_void_p()
        _check(lib.swdft2d_plan(ctypes.byref(h), len(shapes), arr, NORMS[norm], POS[pos],
                                ALGOS[algo], int(flags)), "swdft2d_plan")
        self._h = h
        self.batch = len(shapes)
        self.norm = norm
        self.flags = flags

    @property
    def handle(self):
        if self._h is None or not self._h.value:
            raise ValueError("plan destroyed")
        return self._h

    def output_shape(self, i: int = 0):
        out = (ctypes.c_int64 * 4)()
        _check(lib.swdft2d_output_shape(self.handle, i, out), "swdft2d_output_shape")
        return tuple(int(v) for v in out)

    def workspace_size(self) -> int:
        v = ctypes.c_size_t()
        _check(lib.swdft2d_workspace_size(self.handle, ctypes.byref(v)), "swdft2d_workspace_size")
        return int(v.value)

    def algo(self) -> str:
        v = ctypes.c_int32()
        _check(lib.swdft2d_get_algo(self.handle, ctypes.byref(v)), "swdft2d_get_algo")
        return ALGO_NAMES[int(v.value)]

    def form(self, i: int):
        """(algorithm name, form name) array i runs in: form "pipelined" / "fused_group" (a
        persistent plan's shared kernels) or "per_array"."""
        a, f = ctypes.c_int32(), ctypes.c_int32()
        _check(lib.swdft2d_get_form(self.handle, int(i), ctypes.byref(a), ctypes.byref(f)), "swdft2d_get_form")
        return ALGO_NAMES[int(a.value)], FORM_NAMES[int(f.value)]

    def launch_count(self, adjoint: bool = False) -> int:
        v = ctypes.c_int32()
        _check(lib.swdft2d_launch_count(self.handle, int(adjoint), ctypes.byref(v)),
               "swdft2d_launch_count")
        return int(v.value)

    def load_tuning(self, path: str, gpu_name: str = None) -> int:
        """Apply the tuning-cache records of `path` made on `gpu_name` (None: this device);
        returns the number of arrays set."""
        n = ctypes.c_int32()
        _check(lib.swdft2d_load_tuning(self.handle, str(path).encode(),
                                       None if gpu_name is None else gpu_name.encode(), ctypes.byref(n)),
               "swdft2d_load_tuning")
        return int(n.value)

    def execute(self, in_ptrs, out_ptrs, ws_ptr: int, stream: int = 0):
        _check(lib.swdft2d_execute(self.handle, _ptr_array(in_ptrs), _ptr_array(out_ptrs),
                                   ctypes.c_void_p(ws_ptr or None), ctypes.c_void_p(stream or None)),
               "swdft2d_execute")

    def execute_stage(self, stage: int, in_ptrs, out_ptrs, ws_ptr: int, stream: int = 0):
        _check(lib.swdft2d_execute_stage(self.handle, int(stage), _ptr_array(in_ptrs),
                                         _ptr_array(out_ptrs), ctypes.c_void_p(ws_ptr or None),
                                         ctypes.c_void_p(stream or None)), "swdft2d_execute_stage")

    def set_tree_config(self, i: int, row_B: int, row_chunk: int, col_B: int, col_chunk: int,
                        col_groups: int, fused: int = -1):
        _check(lib.swdft2d_set_tree_config(self.handle, int(i), int(row_B), int(row_chunk),
                                           int(col_B), int(col_chunk), int(col_groups), int(fused)),
               "swdft2d_set_tree_config")

    def execute_adjoint(self, gout_ptrs, gin_ptrs, ws_ptr: int, stream: int = 0):
        _check(lib.swdft2d_execute_adjoint(self.handle, _ptr_array(gout_ptrs),
                                           _ptr_array(gin_ptrs), ctypes.c_void_p(ws_ptr or None),
                                           ctypes.c_void_p(stream or None)),
               "swdft2d_execute_adjoint")

    def execute_host(self, h_in_ptrs, h_out_ptrs, stream: int = 0):
        _check(lib.swdft2d_execute_host(self.handle, _ptr_array(h_in_ptrs),
                                        _ptr_array(h_out_ptrs), ctypes.c_void_p(stream or None)),
               "swdft2d_execute_host")

    def autotune(self, in_ptrs, out_ptrs, ws_ptr: int, stream: int = 0):
        _check(lib.swdft2d_autotune(self.handle, _ptr_array(in_ptrs), _ptr_array(out_ptrs),
                                    ctypes.c_void_p(ws_ptr or None), ctypes.c_void_p(stream or None)),
               "swdft2d_autotune")

    def destroy(self):
        if self._h is not None and self._h.value:
            lib.swdft2d_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def check_device() -> int:
    """SWDFT_OK, or ERR_DEVICE_TIMEOUT if a bounded device wait gave up since the last call."""
    return int(lib.swdft2d_check_device())


def selftest_wait_timeout(polls: int, stream: int = 0) -> None:
    """Enqueue one block whose bounded device wait runs out on purpose (at most `polls` polls
    of about 1 ms); the next check_device() then reports ERR_DEVICE_TIMEOUT."""
    _check(lib.swdft2d_selftest_wait_timeout(int(polls), ctypes.c_void_p(stream or None)),
           "swdft2d_selftest_wait_timeout")


def debug_batch_wait(budget_cycles: int, poison: int) -> None:
    """Set the clock64 budget of the pipelined batch kernels' waits (0: the default, about a
    second) and the test hook that makes array 0's column tiles wait for `poison` row tiles
    that never run; used by the next persistent launch enqueued or captured."""
    _check(lib.swdft2d_debug_batch_wait(int(budget_cycles), int(poison)), "swdft2d_debug_batch_wait")


def inject_alloc_failure(after: int) -> None:
    """Let the library's next `after` allocations succeed and fail every later one with
    SWDFT_ERR_OOM; after < 0 turns injection off."""
    _check(lib.swdft2d_inject_alloc_failure(int(after)), "swdft2d_inject_alloc_failure")


def version() -> int:
    return int(lib.swdft2d_version())


def raw_plan(shapes: Sequence[dict], norm: int, pos: int, algo: int, flags: int):
    """Call swdft2d_plan with raw enum values; returns (status, handle or None)."""
    arr = (Shape * max(1, len(shapes)))()
    for i, s in enumerate(shapes):
        arr[i] = Shape(int(s["N0"]), int(s["N1"]), int(s.get("ld", 0)), int(s["n0"]),
                       int(s["n1"]), int(s.get("dtype", R32)), 0, int(s.get("row_begin", 0)),
                       int(s.get("row_end", 0)))
    h = ctypes.c_void_p()
    st = lib.swdft2d_plan(ctypes.byref(h), len(shapes), arr, norm, pos, algo, flags)
    return st, (h if h.value else None)


def raw_plan_kd(N: Sequence[int], n: Sequence[int], dtype: int = R32, norm: int = 0,
                flags: int = 0, k: Optional[int] = None):
    """Call swdftkd_plan with raw values; returns (status, handle or None)."""
    sh = ShapeKD()
    sh.k = len(N) if k is None else int(k)
    sh.dtype = int(dtype)
    for d in range(min(len(N), KD_MAX_DIMS)):
        sh.N[d] = int(N[d])
        sh.n[d] = int(n[d])
    h = ctypes.c_void_p()
    st = lib.swdftkd_plan(ctypes.byref(h), ctypes.byref(sh), int(norm), int(flags))
    return st, (h if h.value else None)


class PlanKD:
    """Owns one swdftkd plan (Section 4.4: the k-dimensional transform, k <= 4)."""

    def __init__(self, N: Sequence[int], n: Sequence[int], dtype: int = R32,
                 norm: str = "unitary"):
        if len(N) != len(n) or not 1 <= len(N) <= KD_MAX_DIMS:
            raise ValueError("need 1..4 dimensions and one window length per dimension")
        st, h = raw_plan_kd(N, n, dtype, NORMS[norm])
        _check(st, "swdftkd_plan")
        self._h = h
        self.k = len(N)

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("plan destroyed")
        return self._h

    def output_shape(self):
        out = (ctypes.c_int64 * (2 * KD_MAX_DIMS))()
        _check(lib.swdftkd_output_shape(self.handle, out), "swdftkd_output_shape")
        return tuple(int(v) for v in out[:2 * self.k])

    def workspace_size(self) -> int:
        v = ctypes.c_size_t()
        _check(lib.swdftkd_workspace_size(self.handle, ctypes.byref(v)), "swdftkd_workspace_size")
        return int(v.value)

    def launch_count(self) -> int:
        v = ctypes.c_int32()
        _check(lib.swdftkd_launch_count(self.handle, ctypes.byref(v)), "swdftkd_launch_count")
        return int(v.value)

    def execute(self, in_ptr: int, out_ptr: int, ws_ptr: int, stream: int = 0):
        _check(lib.swdftkd_execute(self.handle, ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr),
                                   ctypes.c_void_p(ws_ptr or None), ctypes.c_void_p(stream or None)),
               "swdftkd_execute")

    def destroy(self):
        if self._h is not None and self._h.value:
            lib.swdftkd_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def raw_stream(N1: int, n0: int, n1: int, dtype: int = R32, norm: int = 0, max_rows: int = 1):
    """Call swdft2d_stream_create with raw values; returns (status, handle or None)."""
    h = ctypes.c_void_p()
    st = lib.swdft2d_stream_create(ctypes.byref(h), int(N1), int(n0), int(n1), int(dtype),
                                   int(norm), int(max_rows))
    return st, (h if h.value else None)


class StreamPlan:
    """Owns one swdft2d_stream object (rows pushed over time, windows emitted as completed)."""

    def __init__(self, N1: int, n0: int, n1: int, dtype: int = R32, norm: str = "unitary",
                 max_rows: int = 1):
        st, h = raw_stream(N1, n0, n1, dtype, NORMS[norm], max_rows)
        _check(st, "swdft2d_stream_create")
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("stream destroyed")
        return self._h

    def state_size(self) -> int:
        v = ctypes.c_size_t()
        _check(lib.swdft2d_stream_state_size(self.handle, ctypes.byref(v)), "swdft2d_stream_state_size")
        return int(v.value)

    def push(self, rows_ptr: int, nrows: int, ld: int, out_ptr: int, state_ptr: int, stream: int = 0):
        """Returns (window rows written, index q0 of the first)."""
        n, first = ctypes.c_int64(), ctypes.c_int64()
        _check(lib.swdft2d_stream_push(self.handle, ctypes.c_void_p(rows_ptr or None), int(nrows), int(ld),
                                       ctypes.c_void_p(out_ptr or None), ctypes.c_void_p(state_ptr or None),
                                       ctypes.byref(n), ctypes.byref(first), ctypes.c_void_p(stream or None)),
               "swdft2d_stream_push")
        return int(n.value), int(first.value)

    def rows_seen(self) -> int:
        v = ctypes.c_int64()
        _check(lib.swdft2d_stream_rows_seen(self.handle, ctypes.byref(v)), "swdft2d_stream_rows_seen")
        return int(v.value)

    def reset(self):
        _check(lib.swdft2d_stream_reset(self.handle), "swdft2d_stream_reset")

    def destroy(self):
        if self._h is not None and self._h.value:
            lib.swdft2d_stream_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
