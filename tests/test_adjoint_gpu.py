"""Parity of the hand-written adjoint kernels (transposed tree, through the C ABI and
torch.autograd) with the FP64 oracle's explicit adjoint A^H, the dot-product identity, and
central finite differences of an FP64 loss.

Bar: max over pixels of |g_gpu - g_oracle| / sqrt(sum over windows w containing the pixel of
||G_w||^2) <= 1e-5 (the adjoint's analogue of the forward's window-norm metric).
"""
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


def _G(seed, P0, P1, n0, n1):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((P0, P1, n0, n1)) + 1j * rng.standard_normal((P0, P1, n0, n1))
            ).astype(np.complex64)


def gpu_adjoint(sw, G, N0, N1, cplx, norm="unitary", band=None, pos="start"):
    n0, n1 = G.shape[2], G.shape[3]
    t = sw.Transform([(N0, N1, n0, n1, 1 if cplx else 0)], norm=norm,
                     bands=None if band is None else [band], pos=pos)
    g = t.adjoint([torch.from_numpy(G).cuda()])[0]
    torch.cuda.synchronize()
    return g.cpu().numpy()


SHAPES = [(1, 1, 1, 1), (9, 9, 8, 8), (37, 53, 4, 8), (64, 77, 8, 16), (23, 300, 1, 64),
          (300, 23, 64, 1), (100, 100, 32, 32), (130, 90, 64, 16), (45, 45, 2, 32), (50, 70, 16, 8),
          (80, 120, 32, 64), (130, 100, 64, 64), (60, 70, 16, 16), (40, 33, 16, 1), (33, 40, 2, 1),
          (100, 33, 4, 1)]  # seven column chunks over an odd number of channels: the fold's one-value path


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("N0,N1,n0,n1", SHAPES)
def test_adjoint_matches_oracle(sw, N0, N1, n0, n1, cplx):
    P0, P1 = N0 - n0 + 1, N1 - n1 + 1
    G = _G(N0 + 3 * N1, P0, P1, n0, n1)
    g = gpu_adjoint(sw, G, N0, N1, cplx)
    ref = oracle.swdft2d_adjoint(G, N0, N1)
    if not cplx:
        ref = ref.real
    assert g.shape == (N0, N1)
    err = workloads.adjoint_error(g, ref, workloads.adjoint_pixel_norms(G, N0, N1))
    assert err <= TOL, f"adjoint max normalised error {err:.3e}"


@pytest.mark.parametrize("norm", ["none", "inv_n"])
def test_adjoint_normalisations(sw, norm):
    N0, N1, n0, n1 = 40, 50, 8, 16
    G = _G(5, N0 - n0 + 1, N1 - n1 + 1, n0, n1)
    g = gpu_adjoint(sw, G, N0, N1, True, norm=norm)
    ref = oracle.swdft2d_adjoint(G, N0, N1, norm=norm)
    scale = oracle.scale_for("unitary", n0, n1) / oracle.scale_for(norm, n0, n1)
    err = workloads.adjoint_error(g * scale, ref * scale, workloads.adjoint_pixel_norms(G, N0, N1))
    assert err <= TOL


def test_adjoint_of_band_zeroes_untouched_rows(sw):
    N0, N1, n0, n1 = 60, 40, 8, 4
    P0, P1 = N0 - n0 + 1, N1 - n1 + 1
    G = _G(6, P0, P1, n0, n1)
    Gb = np.zeros_like(G)
    Gb[10:30] = G[10:30]
    g = gpu_adjoint(sw, np.ascontiguousarray(G[10:30]), N0, N1, False, band=(10, 30))
    ref = oracle.swdft2d_adjoint(Gb, N0, N1).real
    err = workloads.adjoint_error(g, ref, workloads.adjoint_pixel_norms(Gb, N0, N1))
    assert err <= TOL
    assert np.all(g[:10] == 0) and np.all(g[30 + n0 - 1:] == 0)


def test_dot_product_identity_full_size(sw):
    """<A x, G> = <x, A^H G> on the 8 x 256x256, 16x16-window differentiation workload."""
    xs, w, (n0, n1) = workloads.adjoint_batch_8()
    N0, N1 = xs.shape[1:]
    t = sw.Transform([(N0, N1, n0, n1, 0)] * len(xs))
    xd = [torch.from_numpy(x).cuda() for x in xs]
    a = t.forward(xd)
    rng = np.random.default_rng(44)
    Gs = [torch.from_numpy(_G(100 + i, N0 - n0 + 1, N1 - n1 + 1, n0, n1)).cuda() for i in range(len(xs))]
    g = t.adjoint(Gs)
    torch.cuda.synchronize()
    lhs = sum(torch.vdot(ai.flatten().to(torch.complex128), Gi.flatten().to(torch.complex128))
              for ai, Gi in zip(a, Gs))
    rhs = sum(torch.vdot(xi.flatten().to(torch.complex128), gi.flatten().to(torch.complex128))
              for xi, gi in zip(xd, g))
    # x is real: <x, A^H G> uses Re(A^H G), so compare real parts
    assert abs(lhs.real - rhs.real) <= 1e-5 * abs(lhs.real) + 1e-3, (lhs, rhs)


def test_autograd_gradient_full_size_against_oracle(sw):
    """loss = sum w |A x|^2 per image of the 8-image batch; torch's grad via the adjoint
    kernel vs the oracle's explicit adjoint (image 0 in full, sampled pixels of the rest)."""
    xs, w, (n0, n1) = workloads.adjoint_batch_8()
    N0, N1 = xs.shape[1:]
    wd = torch.from_numpy(w).cuda()
    rng = np.random.default_rng(45)
    for i, x in enumerate(xs):
        xd = torch.from_numpy(x).cuda().requires_grad_(True)
        a = sw.SWDFT2dFunction.apply(xd, n0, n1)
        loss = (wd * a.abs() ** 2).sum()
        loss.backward()
        g = xd.grad.cpu().numpy()
        a_np = a.detach().cpu().numpy()
        Gup = 2 * w * a_np                                  # torch's gradient w.r.t. a
        if i == 0:
            ref = oracle.swdft2d_adjoint(Gup, N0, N1).real
            err = workloads.adjoint_error(g, ref, workloads.adjoint_pixel_norms(Gup, N0, N1))
        else:
            rs = rng.integers(0, N0, 256)
            cs = rng.integers(0, N1, 256)
            ref = oracle.swdft2d_adjoint_pixels(Gup, N0, N1, rs, cs, threads=8).real
            err = workloads.adjoint_error(g[rs, cs], ref,
                                          workloads.adjoint_pixel_norms(Gup, N0, N1)[rs, cs])
        assert err <= TOL, f"image {i}: {err:.3e}"


@pytest.mark.parametrize("n", [4, 8, 16])
def test_autograd_gradient_matches_fp64_finite_differences(sw, n):
    """The 16x16 top-left crop of image 0 with n x n windows; mask = the first P0 x P1 x n x n
    entries of the workload's mask; central differences (h = 1e-6) of the FP64 oracle loss."""
    xs, w_full, _ = workloads.adjoint_batch_8()
    x = np.ascontiguousarray(xs[0, :16, :16])
    P = 16 - n + 1
    w = np.ascontiguousarray(w_full[:P, :P, :n, :n]).astype(np.float64)
    xd = torch.from_numpy(x).cuda().requires_grad_(True)
    a = sw.SWDFT2dFunction.apply(xd, n, n)
    loss = (torch.from_numpy(w).cuda().float() * a.abs() ** 2).sum()
    loss.backward()
    g = xd.grad.cpu().numpy().astype(np.float64)

    def L(v):
        return float(np.sum(w * np.abs(oracle.swdft2d(v, n, n)) ** 2))

    x64 = x.astype(np.float64)
    h = 1e-6
    fd = np.empty_like(x64)
    for r in range(16):
        for c in range(16):
            e = np.zeros_like(x64)
            e[r, c] = h
            fd[r, c] = (L(x64 + e) - L(x64 - e)) / (2 * h)
    scale = np.abs(fd).max()
    assert np.abs(g - fd).max() <= 1e-5 * scale + 1e-6, (np.abs(g - fd).max(), scale)


def test_adjoint_of_persistent_batch_plan(sw):
    """A persistent plan's adjoint runs its arrays on several streams; each array needs its
    own gz region.  Results must equal the per-array plan's and the oracle's."""
    shapes = [(70, 50, 8, 16, 0), (64, 64, 16, 4, 1), (90, 40, 32, 8, 0), (33, 60, 4, 32, 1),
              (50, 50, 16, 16, 0), (41, 77, 2, 8, 1)]
    Gs = [_G(70 + i, N0 - n0 + 1, N1 - n1 + 1, n0, n1) for i, (N0, N1, n0, n1, _) in enumerate(shapes)]
    Gd = [torch.from_numpy(G).cuda() for G in Gs]
    a = sw.Transform(shapes).adjoint(Gd)
    b = sw.Transform(shapes, flags=sw.FLAG_PERSISTENT).adjoint(Gd)
    torch.cuda.synchronize()
    for u, v, G, (N0, N1, n0, n1, c) in zip(a, b, Gs, shapes):
        assert torch.equal(u, v)
        ref = oracle.swdft2d_adjoint(G, N0, N1)
        if not c:
            ref = ref.real
        err = workloads.adjoint_error(v.cpu().numpy(), ref, workloads.adjoint_pixel_norms(G, N0, N1))
        assert err <= TOL, f"{(N0, N1, n0, n1)}: {err:.3e}"


@pytest.mark.parametrize("cplx", [False, True])
def test_adjoint_of_same_shape_arrays_in_grouped_launches(sw, cplx):
    """Eleven arrays of one shape: the adjoint runs them as a group of eight and a group of
    three per launch; each result equals its one-array plan's bit for bit and the oracle's."""
    N0, N1, n0, n1 = 120, 45, 8, 8  # two column chunks of at most 6 n0 rows: the fold launch runs too
    band = (5, 99)
    P1 = N1 - n1 + 1
    Gs = [_G(200 + i, band[1] - band[0], P1, n0, n1) for i in range(11)]
    Gd = [torch.from_numpy(G).cuda() for G in Gs]
    t = sw.Transform([(N0, N1, n0, n1, int(cplx))] * 11, bands=[band] * 11)
    assert t.plan.launch_count(adjoint=True) == 6  # per group: column pass, fold, row pass
    got = t.adjoint(Gd)
    torch.cuda.synchronize()
    for i, (G, g) in enumerate(zip(Gs, got)):
        one = sw.Transform([(N0, N1, n0, n1, int(cplx))], bands=[band]).adjoint([Gd[i]])[0]
        torch.cuda.synchronize()
        assert torch.equal(g, one)
        full = np.zeros((N0 - n0 + 1, P1, n0, n1), np.complex64)
        full[band[0]:band[1]] = G
        ref = oracle.swdft2d_adjoint(full, N0, N1)
        if not cplx:
            ref = ref.real
        err = workloads.adjoint_error(g.cpu().numpy(), ref, workloads.adjoint_pixel_norms(full, N0, N1))
        assert err <= TOL, f"array {i}: {err:.3e}"


@pytest.mark.parametrize("N0,N1,n0,n1", [(60, 70, 16, 16), (100, 100, 32, 32), (130, 90, 64, 16),
                                         (50, 70, 16, 8), (40, 33, 16, 1), (45, 45, 2, 32)])
def test_bulk_and_cp_async_staging_agree_bit_for_bit(sw, N0, N1, n0, n1):
    """The column adjoint stages G by bulk copies when G is 16-byte aligned and by 8-byte
    cp.async otherwise (a G that starts 8 bytes into a buffer).  Both sum the residues of a
    channel in the same order, so the two gradients are equal bit for bit; and no bounded
    wait of the bulk kernel gave up (swdft2d_check_device)."""
    from paper_1707_08213_gb300 import _native as nat
    P0, P1 = N0 - n0 + 1, N1 - n1 + 1
    G = torch.from_numpy(_G(7 * N0 + N1, P0, P1, n0, n1)).cuda()
    buf = torch.empty(G.numel() + 1, dtype=torch.complex64, device="cuda")
    Gm = buf[1:].view(G.shape)
    Gm.copy_(G)
    assert G.data_ptr() % 16 == 0 and Gm.data_ptr() % 16 == 8
    t = sw.Transform([(N0, N1, n0, n1, 0)])
    a = t.adjoint([G])[0].clone()
    b = t.adjoint([Gm])[0]
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert nat.check_device() == 0

