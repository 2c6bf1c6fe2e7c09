"""Parity of the k-dimensional transform (Section 4.4, Eq. kdfswft; through the C ABI of
include/swdftkd.h) with the FP64 k-dimensional oracle.

Bar as for 2D: max over coefficients of |a_gpu - a_oracle| / ||x_w||_2 <= 1e-5 per window on
the unitary scale.  Small arrays are compared on every coefficient (shapes that span
several 32-channel tiles and row chunks, with ragged tails and windows of 1 and 64 along
some axes); the 128^3 volume and a 32^4 complex array on sampled windows plus per-window
Parseval over all windows.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-5
THREADS = 8


@pytest.fixture(scope="module")
def sw():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1707_08213_gb300 as sw
    return sw


def run_kd(sw, x, n, norm="unitary"):
    t = sw.TransformKD(x.shape, n, dtype=1 if np.iscomplexobj(x) else 0, norm=norm)
    a = t.forward(torch.from_numpy(np.ascontiguousarray(x)).cuda())
    torch.cuda.synchronize()
    return a, t


def check(a, x, n, norm="unitary"):
    ref = oracle.swdftkd(x, n, norm=norm, method="separable", threads=THREADS)
    to_unitary = oracle.scale_for_kd("unitary", n) / oracle.scale_for_kd(norm, n)
    got = a.cpu().numpy()
    assert got.shape == ref.shape
    err, rms = workloads.normalised_error(got, ref, workloads.window_sq_norms_kd(x, n), to_unitary)
    assert err <= TOL, f"{x.shape} {n}: max normalised error {err:.3e} (rms {rms:.3e})"
    return err


KD_SHAPES = [
    ((9, 10, 11), (2, 4, 8)), ((17, 13, 40), (4, 8, 32)), ((33, 20, 12), (16, 4, 2)),
    ((10, 70, 9), (1, 64, 1)), ((70, 5, 6), (64, 1, 2)), ((12, 12, 12), (8, 8, 8)),
    ((5, 9, 70), (4, 2, 64)), ((40, 3, 3), (32, 2, 2)), ((1, 1, 1), (1, 1, 1)),
    ((6, 7, 8, 9), (2, 4, 2, 8)), ((3, 20, 5, 7), (2, 16, 1, 4)), ((4, 4, 4, 4), (4, 4, 4, 4)),
]


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("shape,n", KD_SHAPES)
def test_every_coefficient(sw, shape, n, cplx):
    x = workloads.random_array_kd(sum(shape) * 7 + len(shape), shape, complex_input=cplx)
    a, t = run_kd(sw, x, n)
    assert t.plan.launch_count() == len(shape)
    check(a, x, n)


@pytest.mark.parametrize("norm", ["none", "inv_n"])
def test_normalisations(sw, norm):
    x = workloads.random_array_kd(41, (14, 15, 16), complex_input=True)
    a, _ = run_kd(sw, x, (4, 2, 8), norm=norm)
    check(a, x, (4, 2, 8), norm=norm)


def test_one_and_two_dimensions_are_the_2d_path(sw):
    x2 = workloads.random_array(42, 50, 70)
    a2 = sw.swdft2d(torch.from_numpy(x2).cuda(), 16, 8)
    b2, _ = run_kd(sw, x2, (16, 8))
    assert torch.equal(a2, b2)
    x1 = workloads.random_array_kd(43, (300,), complex_input=True)
    b1, _ = run_kd(sw, x1, (32,))
    check(b1, x1, (32,))
    a1 = sw.swdft2d(torch.from_numpy(x1[None]).cuda(), 1, 32)
    assert torch.equal(a1.reshape(b1.shape), b1)


def test_leading_window_of_one_equals_2d_of_each_slice(sw):
    """n_0 = 1: dimension 0's pass only scales, so every slice q0 is exactly the 2D
    transform of input slice q0 (the same node arithmetic, bit for bit)."""
    x = workloads.random_array_kd(44, (3, 40, 36))
    a, _ = run_kd(sw, x, (1, 8, 16))
    for s in range(3):
        b = sw.swdft2d(torch.from_numpy(np.ascontiguousarray(x[s])).cuda(), 8, 16)
        assert torch.equal(a[s, :, :, 0], b)


def test_deterministic(sw):
    x = workloads.random_array_kd(45, (20, 30, 40))
    a, t = run_kd(sw, x, (8, 4, 16))
    b = t.forward(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_volume_128_full_size(sw):
    """128^3 float32, 8x8x8 windows (7.26 GB of output): 4096 sampled windows plus the eight
    corners against the oracle, and Parseval on every window."""
    x, n = workloads.volume_128()
    a, _ = run_kd(sw, x, n)
    P = a.shape[:3]
    rng = np.random.default_rng(15)
    q = np.stack([rng.integers(0, p, 4096) for p in P], axis=1)
    corners = np.array([[i * (P[0] - 1), j * (P[1] - 1), k * (P[2] - 1)]
                        for i in (0, 1) for j in (0, 1) for k in (0, 1)])
    q = np.concatenate([q, corners])
    qd = torch.from_numpy(q).cuda()
    got = a[qd[:, 0], qd[:, 1], qd[:, 2]].cpu().numpy()
    ref = oracle.swdftkd_windows(x, n, q, threads=THREADS)
    err, _ = workloads.normalised_error(got, ref, workloads.window_sq_norms_kd_at(x, n, q))
    assert err <= TOL, f"sampled windows: {err:.3e}"
    sq = torch.from_numpy(workloads.window_sq_norms_kd(x, n)).cuda()
    worst = 0.0
    for r in range(0, P[0], 16):
        e = torch.view_as_real(a[r:r + 16]).pow(2).sum(dim=(3, 4, 5, 6)).double()
        worst = max(worst, float(((e - sq[r:r + 16]).abs() / sq[r:r + 16]).max()))
    assert worst <= 1e-5, f"Parseval relative error {worst:.3e}"
    del a
    torch.cuda.empty_cache()


def test_four_dimensions_full_size(sw):
    """32^4 complex, 4x4x4x4 windows (29^4 x 256 coefficients, 1.45 GB): sampled windows
    against the oracle plus Parseval on every window."""
    x = workloads.random_array_kd(46, (32, 32, 32, 32), complex_input=True)
    n = (4, 4, 4, 4)
    a, t = run_kd(sw, x, n)
    assert t.plan.launch_count() == 4
    P = a.shape[:4]
    rng = np.random.default_rng(47)
    q = np.stack([rng.integers(0, p, 2048) for p in P], axis=1)
    q = np.concatenate([q, np.zeros((1, 4), np.int64), np.array([[p - 1 for p in P]])])
    qd = torch.from_numpy(q).cuda()
    got = a[qd[:, 0], qd[:, 1], qd[:, 2], qd[:, 3]].cpu().numpy()
    ref = oracle.swdftkd_windows(x, n, q, threads=THREADS)
    err, _ = workloads.normalised_error(got, ref, workloads.window_sq_norms_kd_at(x, n, q))
    assert err <= TOL, f"sampled windows: {err:.3e}"
    sq = torch.from_numpy(workloads.window_sq_norms_kd(x, n)).cuda()
    worst = 0.0
    for r in range(0, P[0], 8):
        e = torch.view_as_real(a[r:r + 8]).pow(2).sum(dim=(4, 5, 6, 7, 8)).double()
        worst = max(worst, float(((e - sq[r:r + 8]).abs() / sq[r:r + 8]).max()))
    assert worst <= 1e-5, f"Parseval {worst:.3e}"
    del a
    torch.cuda.empty_cache()
