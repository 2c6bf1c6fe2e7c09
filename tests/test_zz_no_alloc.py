"""The allocation-free entry point, swdft2d_execute_static_scratch, against the planned one.

Some callers may not allocate device memory at all (plug-ins handed only their buffers,
code running after a framework has claimed the device memory, real-time paths).  For them
the library keeps the intermediate z rows in a fixed device array of its own and needs no
plan or workspace.  This test calls that entry point through the C ABI twice in a row on
different shapes (one of them needing several bands) and checks each result against
swdft2d_execute with the parity tolerance of the other GPU tests (max |difference| / window
norm <= 1e-5).  It lives in its own file, collected last, and passes alone or after the
rest of the suite.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def sw():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1707_08213_gb300 as sw
    return sw


def _static_call(nat, xd, N0, N1, n0, n1, dtype, out, ld=0, norm=0):
    return nat.lib.swdft2d_execute_static_scratch(
        ctypes.c_void_p(xd.data_ptr()), N0, N1, ld, n0, n1, dtype, norm,
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _max_normalised_diff(out, ref, x, n0, n1, scale_to_unitary=1.0):
    d = (out - ref).abs().amax(dim=(2, 3)).double().cpu().numpy() * scale_to_unitary
    nrm = np.sqrt(workloads.window_sq_norms(x, n0, n1))
    return float(np.max(np.where(nrm > 0, d / np.where(nrm > 0, nrm, 1), d)))


def test_static_scratch_matches_planned_entry_twice(sw):
    from paper_1707_08213_gb300 import _native as nat
    cases = [
        (workloads.sinusoids_512().images[0], 32, 32),                           # several bands
        (workloads.random_array(31, 300, 257, complex_input=True), 16, 64),      # complex input
        (workloads.random_array(32, 97, 61), 8, 4),                               # one band
    ]
    for rep in range(2):
        for x, n0, n1 in cases:
            N0, N1 = x.shape
            dtype = 1 if np.iscomplexobj(x) else 0
            xd = torch.from_numpy(x).cuda()
            ref = sw.Transform([(N0, N1, n0, n1, dtype)]).forward([xd])[0]
            out = torch.full_like(ref, float("nan"))
            st = _static_call(nat, xd, N0, N1, n0, n1, dtype, out)
            assert st == 0, nat.status_string(st)
            torch.cuda.synchronize()
            err = _max_normalised_diff(out, ref, x, n0, n1)
            assert err <= TOL, f"call {rep}, {x.shape} {n0}x{n1}: max normalised diff {err:.3e}"


def test_static_scratch_row_stride_norms_and_edge_windows(sw):
    """Rows further apart than N1 (ld > N1), the NONE and 1/(n0 n1) scales, and the window
    sides 1 and 64, each against the planned transform of the same (contiguous) array.
    Differences are compared on the unitary scale."""
    from paper_1707_08213_gb300 import _native as nat
    cases = [  # (seed, N0, N1, ld, n0, n1, complex, norm)
        (41, 150, 120, 136, 16, 8, False, "unitary"),
        (42, 90, 70, 77, 8, 8, True, "unitary"),
        (43, 200, 100, 0, 64, 16, False, "none"),
        (44, 64, 300, 301, 1, 8, False, "inv_n"),
        (45, 130, 90, 96, 8, 1, True, "none"),
        (46, 80, 200, 0, 16, 64, False, "inv_n"),
    ]
    for rep in range(2):
        for seed, N0, N1, ld, n0, n1, cplx, norm in cases:
            x = workloads.random_array(seed, N0, N1, complex_input=cplx)
            dtype = 1 if cplx else 0
            xd = torch.from_numpy(x).cuda()
            if ld:
                wide = torch.full((N0, ld), float("nan"), dtype=xd.dtype, device="cuda")
                wide[:, :N1] = xd
                src = wide
            else:
                src = xd
            ref = sw.Transform([(N0, N1, n0, n1, dtype)], norm=norm).forward([xd])[0]
            out = torch.full_like(ref, float("nan"))
            st = _static_call(nat, src, N0, N1, n0, n1, dtype, out, ld=ld, norm=nat.NORMS[norm])
            assert st == 0, nat.status_string(st)
            torch.cuda.synchronize()
            to_unitary = {"unitary": 1.0, "none": 1 / np.sqrt(n0 * n1), "inv_n": np.sqrt(n0 * n1)}[norm]
            err = _max_normalised_diff(out, ref, x, n0, n1, to_unitary)
            assert err <= TOL, f"call {rep}, {(N0, N1, ld)} {n0}x{n1} {norm}: max normalised diff {err:.3e}"


def test_static_scratch_rejects_oversized_and_bad_args(sw):
    from paper_1707_08213_gb300 import _native as nat
    x = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    out = torch.zeros((1, 1, 8, 8), dtype=torch.complex64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # a one-row band of a 64x64-window transform over 6000 columns needs
    # 96 * 5937 * 64 * 8 bytes of z, beyond the 32 MiB array: rejected before any launch
    st = nat.lib.swdft2d_execute_static_scratch(ctypes.c_void_p(x.data_ptr()), 64, 6000, 0, 64,
                                                64, 0, 0, ctypes.c_void_p(out.data_ptr()), s)
    assert st == nat.ERR_WORKSPACE
    assert nat.lib.swdft2d_execute_static_scratch(None, 8, 8, 0, 8, 8, 0, 0,
                                                  ctypes.c_void_p(out.data_ptr()), s) == nat.ERR_INVALID_ARG
    # ternary and mixed-radix windows (which plans accept) are not offered by this radix-2 entry point
    assert nat.lib.swdft2d_execute_static_scratch(ctypes.c_void_p(x.data_ptr()), 8, 8, 0, 3, 8, 0,
                                                  0, ctypes.c_void_p(out.data_ptr()), s) == nat.ERR_UNSUPPORTED
    assert nat.lib.swdft2d_execute_static_scratch(ctypes.c_void_p(x.data_ptr()), 9, 9, 0, 8, 9, 0,
                                                  0, ctypes.c_void_p(out.data_ptr()), s) == nat.ERR_UNSUPPORTED
    assert nat.lib.swdft2d_execute_static_scratch(ctypes.c_void_p(x.data_ptr()), 12, 8, 0, 12, 8, 0,
                                                  0, ctypes.c_void_p(out.data_ptr()), s) == nat.ERR_UNSUPPORTED
    assert nat.lib.swdft2d_execute_static_scratch(ctypes.c_void_p(x.data_ptr()), 8, 8, 0, 5, 8, 0,
                                                  0, ctypes.c_void_p(out.data_ptr()), s) == nat.ERR_NOT_POW2
