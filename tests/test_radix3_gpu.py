"""Ternary and mixed-radix trees on the GPU (windows of 3, 9 or 27 along an axis -- the
radix-3 trees Section 5 mentions -- and of 3^b 2^a samples, radix-3 levels then radix-2
levels within one axis) against the FP64 oracle's definition: max over a window's
coefficients of |a - a_oracle| / ||x_w||_2 <= 1e-5 on the unitary scale, every coefficient
of small arrays (ragged sizes, radices mixed within and across the axes), and 512x512
arrays with 27x27 and 48x24 windows on sampled windows plus per-window Parseval."""
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


def run(sw, x, n0, n1, norm="unitary", flags=0, band=None):
    t = sw.Transform([(x.shape[0], x.shape[1], n0, n1, 1 if np.iscomplexobj(x) else 0)], norm=norm,
                     flags=flags, bands=None if band is None else [band])
    a = t.forward([torch.from_numpy(np.ascontiguousarray(x)).cuda()])[0]
    torch.cuda.synchronize()
    return a, t


def check(a, x, n0, n1, norm="unitary"):
    ref = oracle.swdft2d(x, n0, n1, norm=norm, method="separable", threads=8)
    to_unitary = oracle.scale_for("unitary", n0, n1) / oracle.scale_for(norm, n0, n1)
    err, _ = workloads.normalised_error(a.cpu().numpy(), ref, workloads.window_sq_norms(x, n0, n1), to_unitary)
    assert err <= TOL, f"{x.shape} {n0}x{n1}: {err:.3e}"


SHAPES = [(3, 3), (9, 9), (27, 27), (27, 1), (1, 27), (9, 3), (3, 27), (9, 16), (27, 64), (3, 2),
          (1, 3), (27, 8),
          # mixed radices within an axis (3^b 2^a): every length to 54
          (6, 6), (12, 12), (24, 6), (48, 4), (6, 48), (18, 18), (36, 12), (54, 6), (9, 54),
          (12, 1), (1, 48), (48, 48), (24, 36), (54, 64)]


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n0,n1", SHAPES)
def test_every_coefficient(sw, n0, n1, cplx):
    N0, N1 = n0 + 37, n1 + 151  # several 128-channel tiles and row chunks, ragged tails
    x = workloads.random_array(n0 * 31 + n1, N0, N1, complex_input=cplx)
    a, t = run(sw, x, n0, n1)
    assert tuple(a.shape) == (N0 - n0 + 1, N1 - n1 + 1, n0, n1)
    assert t.plan.launch_count() == 2
    check(a, x, n0, n1)


@pytest.mark.parametrize("norm", ["none", "inv_n"])
def test_normalisations(sw, norm):
    x = workloads.random_array(77, 60, 90, complex_input=True)
    a, _ = run(sw, x, 9, 27, norm=norm)
    check(a, x, 9, 27, norm=norm)
    a, _ = run(sw, x, 12, 18, norm=norm)
    check(a, x, 12, 18, norm=norm)


def test_band_graph_and_host_buffers_match(sw):
    x = workloads.random_array(78, 120, 100)
    full, _ = run(sw, x, 27, 9)
    band, _ = run(sw, x, 27, 9, band=(20, 61))
    assert torch.equal(band, full[20:61])
    t = sw.Transform([(120, 100, 27, 9, 0)], flags=sw.FLAG_GRAPH)
    xd = torch.from_numpy(x).cuda()
    out = t.empty_outputs()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(3):
            out[0].zero_()
            t.forward([xd], out)
    s.synchronize()
    assert torch.equal(out[0], full)
    th = sw.Transform([(120, 100, 27, 9, 0)], flags=sw.FLAG_HOST_IO)
    h_in = torch.from_numpy(x).pin_memory()
    h_out = torch.empty(tuple(full.shape), dtype=torch.complex64).pin_memory()
    th.plan.execute_host([h_in.data_ptr()], [h_out.data_ptr()], torch.cuda.current_stream().cuda_stream)
    assert torch.equal(h_out, full.cpu())


ADJ_SHAPES = [(40, 40, 9, 9), (60, 70, 27, 9), (50, 80, 12, 16), (20, 90, 1, 27), (70, 60, 6, 48),
              (100, 120, 54, 36), (33, 31, 3, 3), (90, 64, 24, 18), (64, 80, 36, 4)]


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("N0,N1,n0,n1", ADJ_SHAPES)
def test_adjoint_matches_oracle(sw, N0, N1, n0, n1, cplx):
    """Ternary and mixed-radix windows: the adjoint (per-window inverse DFTs overlap-added
    per axis; a power-of-two row window through the transposed radix-2 tree) against the
    FP64 oracle's explicit A^H (Section 4.1's map transposed), every pixel, per-pixel bar
    max |g - g_oracle| / (sum of ||G_w||^2 over the windows covering it)^(1/2) <= 1e-5."""
    P0, P1 = N0 - n0 + 1, N1 - n1 + 1
    rng = np.random.default_rng(N0 * 7 + n0 * 3 + n1)
    G = (rng.standard_normal((P0, P1, n0, n1)) + 1j * rng.standard_normal((P0, P1, n0, n1))).astype(np.complex64)
    t = sw.Transform([(N0, N1, n0, n1, 1 if cplx else 0)])
    g = t.adjoint([torch.from_numpy(G).cuda()])[0]
    torch.cuda.synchronize()
    assert sw._native.check_device() == 0
    ref = oracle.swdft2d_adjoint(G, N0, N1)
    if not cplx:
        ref = ref.real
    assert tuple(g.shape) == (N0, N1)
    err = workloads.adjoint_error(g.cpu().numpy(), ref, workloads.adjoint_pixel_norms(G, N0, N1))
    assert err <= 1e-5, f"adjoint max normalised error {err:.3e}"


def test_adjoint_band_norm_and_dot_product(sw):
    """A band of window rows (rows outside its reach get 0), the 1/(n0 n1) normalisation,
    and <A x, G> = <x, A^H G> on a 27x18 window."""
    N0, N1, n0, n1 = 120, 100, 27, 18
    x = workloads.random_array(5, N0, N1)
    band = (30, 61)
    t = sw.Transform([(N0, N1, n0, n1, 0)], norm="inv_n", bands=[band])
    a = t.forward([torch.from_numpy(x).cuda()])[0]
    rng = np.random.default_rng(6)
    G = (rng.standard_normal(tuple(a.shape)) + 1j * rng.standard_normal(tuple(a.shape))).astype(np.complex64)
    g = t.adjoint([torch.from_numpy(G).cuda()])[0].cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    lhs = np.vdot(a.cpu().numpy().astype(np.complex128), G.astype(np.complex128)).real
    rhs = float(np.dot(x.astype(np.float64).ravel(), g.ravel()))
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)
    assert not g[:band[0]].any() and not g[band[1] + n0 - 1:].any()
    full = np.zeros((N0 - n0 + 1, N1 - n1 + 1, n0, n1), np.complex64)
    full[band[0]:band[1]] = G
    ref = oracle.swdft2d_adjoint(full, N0, N1, norm="inv_n").real
    scale = oracle.scale_for("unitary", n0, n1) / oracle.scale_for("inv_n", n0, n1)
    err = workloads.adjoint_error(g * scale, ref * scale, workloads.adjoint_pixel_norms(full, N0, N1))
    assert err <= 1e-5


@pytest.mark.parametrize("n0,n1", [(27, 27), (48, 24)])
def test_512_full_size(sw, n0, n1):
    x = workloads.random_array(79, 512, 512)
    a, _ = run(sw, x, n0, n1)
    P0, P1 = a.shape[:2]
    rng = np.random.default_rng(80)
    q0 = np.concatenate([rng.integers(0, P0, 2048), [0, 0, P0 - 1, P0 - 1]])
    q1 = np.concatenate([rng.integers(0, P1, 2048), [0, P1 - 1, 0, P1 - 1]])
    got = a[torch.from_numpy(q0).cuda(), torch.from_numpy(q1).cuda()].cpu().numpy()
    ref = oracle.swdft2d_windows(x, n0, n1, q0, q1, threads=8)
    err, _ = workloads.normalised_error(got, ref, workloads.window_sq_norms_at(x, n0, n1, q0, q1))
    assert err <= TOL, f"sampled windows: {err:.3e}"
    sq = torch.from_numpy(workloads.window_sq_norms(x, n0, n1)).cuda()
    worst = 0.0
    for r in range(0, P0, 64):
        e = torch.view_as_real(a[r:r + 64]).pow(2).sum(dim=(2, 3, 4)).double()
        worst = max(worst, float(((e - sq[r:r + 64]).abs() / sq[r:r + 64]).max()))
    assert worst <= 1e-5, f"Parseval relative error {worst:.3e}"
    del a
    torch.cuda.empty_cache()
