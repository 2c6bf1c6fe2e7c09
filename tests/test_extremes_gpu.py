"""Shapes at the edges of what the kernels take, against the FP64 oracle (Section 4.1, Eq. 2;
per-window error / window norm <= 1e-5): a 2^20-sample row and a 2^20-row column with
64-point windows (grid limits, 64-bit offsets), the largest windows (64 x 64), arrays that
hold exactly one window, windows of one sample, a persistent batch of many tiny arrays, and
the adjoint (per-pixel error / pixel norm <= 1e-5) on a 2^20-sample row and a 2^17-row
column."""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def sw():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1707_08213_gb300 as sw
    return sw


def _sampled(sw, x, n0, n1, count, seed):
    N0, N1 = x.shape
    t = sw.Transform([(N0, N1, n0, n1, 1 if np.iscomplexobj(x) else 0)])
    a = t.forward([torch.from_numpy(np.ascontiguousarray(x)).cuda()])[0]
    torch.cuda.synchronize()
    P0, P1 = N0 - n0 + 1, N1 - n1 + 1
    rng = np.random.default_rng(seed)
    q0 = np.concatenate([rng.integers(0, P0, count), [0, P0 - 1, 0, P0 - 1]])
    q1 = np.concatenate([rng.integers(0, P1, count), [0, 0, P1 - 1, P1 - 1]])
    got = a[torch.from_numpy(q0).cuda(), torch.from_numpy(q1).cuda()].cpu().numpy()
    ref = oracle.swdft2d_windows(x, n0, n1, q0, q1, threads=8)
    err, _ = workloads.normalised_error(got, ref, workloads.window_sq_norms_at(x, n0, n1, q0, q1))
    assert err <= TOL, f"{x.shape} {n0}x{n1}: {err:.3e}"
    # Parseval on every window, in slabs
    sq = torch.from_numpy(workloads.window_sq_norms(x, n0, n1)).cuda()
    worst = 0.0
    step = max(1, (1 << 22) // (P1 * n0 * n1))
    for r in range(0, P0, step):
        e = torch.view_as_real(a[r:r + step]).pow(2).sum(dim=(2, 3, 4)).double()
        s = sq[r:r + step]
        worst = max(worst, float(((e - s).abs() / s.clamp_min(1e-30)).max()))
    assert worst <= 1e-5, f"Parseval {worst:.3e}"
    del a
    torch.cuda.empty_cache()


def test_long_row(sw):
    x = workloads.random_array(101, 1, 1 << 20)
    _sampled(sw, x, 1, 64, 4096, 1)


def test_tall_column(sw):
    x = workloads.random_array(102, 1 << 20, 8, complex_input=True)
    _sampled(sw, x, 64, 8, 4096, 2)


def test_largest_windows(sw):
    x = workloads.random_array(103, 300, 400)
    _sampled(sw, x, 64, 64, 2048, 3)


@pytest.mark.parametrize("n0,n1,cplx", [(64, 64, False), (32, 1, True), (1, 1, False), (16, 8, True)])
def test_array_holding_exactly_one_window(sw, n0, n1, cplx):
    x = workloads.random_array(104 + n0 + n1, n0, n1, complex_input=cplx)
    a = sw.swdft2d(torch.from_numpy(x).cuda(), n0, n1)
    torch.cuda.synchronize()
    assert tuple(a.shape) == (1, 1, n0, n1)
    ref = np.fft.fft2(x.astype(np.complex128)) / np.sqrt(n0 * n1)
    assert np.abs(a.cpu().numpy()[0, 0] - ref).max() <= TOL * np.linalg.norm(x)


def test_one_sample_windows_are_the_scaled_input(sw):
    x = workloads.random_array(105, 70, 90, complex_input=True)
    a = sw.swdft2d(torch.from_numpy(x).cuda(), 1, 1)
    torch.cuda.synchronize()
    assert torch.equal(a[:, :, 0, 0], torch.from_numpy(x).cuda())


def test_persistent_batch_of_many_tiny_arrays(sw):
    rng = np.random.default_rng(106)
    shapes = []
    for i in range(300):
        n0, n1 = int(2 ** rng.integers(0, 3)), int(2 ** rng.integers(0, 3))
        shapes.append((n0 + int(rng.integers(0, 5)), n1 + int(rng.integers(0, 5)), n0, n1, int(i % 2)))
    xs = [workloads.random_array(1000 + i, s[0], s[1], complex_input=bool(s[4])) for i, s in enumerate(shapes)]
    t = sw.Transform(shapes, flags=sw.FLAG_PERSISTENT | sw.FLAG_GRAPH)
    xd = [torch.from_numpy(x).cuda() for x in xs]
    outs = t.empty_outputs()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        for _ in range(2):
            t.forward(xd, outs)
    st.synchronize()
    per = sw.Transform(shapes).forward(xd)
    torch.cuda.synchronize()
    for o, p, x, (N0, N1, n0, n1, c) in zip(outs, per, xs, shapes):
        assert torch.equal(o, p)
        ref = oracle.swdft2d(x, n0, n1, method="direct")
        err, _ = workloads.normalised_error(o.cpu().numpy(), ref, workloads.window_sq_norms(x, n0, n1))
        assert err <= TOL


def _adjoint_sampled(sw, N0, N1, n0, n1, cplx, count, seed):
    P0, P1 = N0 - n0 + 1, N1 - n1 + 1
    rng = np.random.default_rng(seed)
    G = (rng.standard_normal((P0, P1, n0, n1), dtype=np.float32)
         + 1j * rng.standard_normal((P0, P1, n0, n1), dtype=np.float32)).astype(np.complex64)
    t = sw.Transform([(N0, N1, n0, n1, int(cplx))])
    g = t.adjoint([torch.from_numpy(G).cuda()])[0]
    torch.cuda.synchronize()
    rs = np.concatenate([rng.integers(0, N0, count), [0, N0 - 1, 0, N0 - 1]])
    cs = np.concatenate([rng.integers(0, N1, count), [0, 0, N1 - 1, N1 - 1]])
    got = g[torch.from_numpy(rs).cuda(), torch.from_numpy(cs).cuda()].cpu().numpy()
    ref = oracle.swdft2d_adjoint_pixels(G, N0, N1, rs, cs, threads=8)
    if not cplx:
        ref = ref.real
    norms = workloads.adjoint_pixel_norms(G, N0, N1)[rs, cs]
    err = workloads.adjoint_error(got, ref, norms)
    assert err <= TOL, f"adjoint {N0}x{N1} {n0}x{n1}: {err:.3e}"
    del g
    torch.cuda.empty_cache()


def test_adjoint_long_row(sw):
    _adjoint_sampled(sw, 1, 1 << 20, 1, 64, False, 4096, 11)


def test_adjoint_tall_column(sw):
    _adjoint_sampled(sw, 1 << 17, 8, 64, 8, True, 4096, 12)
