"""The persistent batched launch (SWDFT_FLAG_PERSISTENT): many arrays of uneven sizes and
window shapes in persistent kernels per window group (row, column and fused groups),
optionally replayed from a CUDA graph, against the FP64 oracle (Section 4.1, Eq. 2;
per-window error / window norm <= 1e-5)."""
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


MIXED = [(70, 50, 8, 32, False), (33, 90, 16, 4, True), (130, 64, 64, 16, False),
         (20, 20, 4, 4, False), (1, 1, 1, 1, True), (128, 128, 32, 32, False),
         (45, 300, 2, 64, True), (300, 9, 64, 1, False), (64, 64, 8, 8, True)]


def _inputs():
    return [workloads.random_array(50 + i, N0, N1, complex_input=c)
            for i, (N0, N1, _, _, c) in enumerate(MIXED)]


def _check(out, x, n0, n1):
    ref = oracle.swdft2d(x, n0, n1, method="separable", threads=8)
    err, _ = workloads.normalised_error(out.cpu().numpy(), ref, workloads.window_sq_norms(x, n0, n1))
    assert err <= TOL, f"{x.shape} {n0}x{n1}: {err:.3e}"


@pytest.mark.parametrize("flags", ["persistent", "persistent+graph"])
def test_persistent_batch_of_mixed_shapes(sw, flags):
    xs = _inputs()
    f = sw.FLAG_PERSISTENT | (sw.FLAG_GRAPH if "graph" in flags else 0)
    t = sw.Transform([(N0, N1, n0, n1, int(c)) for (N0, N1, n0, n1, c) in MIXED], flags=f)
    # one persistent kernel per row-window group and per column-window group of the two-pass
    # arrays, and one per (n0, n1) group of the fused arrays (small windows, n0 n1 <= 64)
    fused = [(n0, n1) for _, _, n0, n1, _ in MIXED if n0 * n1 <= 64]
    two = [(n0, n1) for _, _, n0, n1, _ in MIXED if (n0, n1) not in fused]
    assert t.plan.launch_count() == len({b for _, b in two}) + len({a for a, _ in two}) + len(set(fused))
    assert t.plan.launch_count() == 12
    xd = [torch.from_numpy(x).cuda() for x in xs]
    outs = t.empty_outputs()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(3):          # the graph is captured on the first call and replayed
            for o in outs:
                o.fill_(float("nan"))
            t.forward(xd, outs)
    s.synchronize()
    for o, x, (N0, N1, n0, n1, c) in zip(outs, xs, MIXED):
        _check(o, x, n0, n1)


def test_persistent_matches_per_array_launches(sw):
    xs = _inputs()
    shapes = [(N0, N1, n0, n1, int(c)) for (N0, N1, n0, n1, c) in MIXED]
    xd = [torch.from_numpy(x).cuda() for x in xs]
    a = sw.Transform(shapes).forward(xd)
    b = sw.Transform(shapes, flags=sw.FLAG_PERSISTENT).forward(xd)
    torch.cuda.synchronize()
    for u, v in zip(a, b):
        assert torch.equal(u, v)


def test_uneven_batch_256_full_size(sw):
    """256 float32 images, sides in {128..1024}, windows from six shapes, one persistent
    launch pair: >= 256 sampled windows per image against the oracle, and per-window
    Parseval on every window of every image."""
    wl = workloads.uneven_batch_256()
    shapes = [(x.shape[0], x.shape[1], n0, n1, 0) for x, (n0, n1) in zip(wl.images, wl.windows)]
    t = sw.Transform(shapes, flags=sw.FLAG_PERSISTENT | sw.FLAG_GRAPH)
    xd = [torch.from_numpy(x).cuda() for x in wl.images]
    outs = t.empty_outputs()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        t.forward(xd, outs)
    s.synchronize()
    rng = np.random.default_rng(33)
    worst, worst_parseval = 0.0, 0.0
    for i, (x, (n0, n1), o) in enumerate(zip(wl.images, wl.windows, outs)):
        P0, P1 = x.shape[0] - n0 + 1, x.shape[1] - n1 + 1
        q0 = np.concatenate([rng.integers(0, P0, 252), [0, 0, P0 - 1, P0 - 1]])
        q1 = np.concatenate([rng.integers(0, P1, 252), [0, P1 - 1, 0, P1 - 1]])
        got = o[torch.from_numpy(q0).cuda(), torch.from_numpy(q1).cuda()].cpu().numpy()
        ref = oracle.swdft2d_windows(x, n0, n1, q0, q1, threads=8)
        err, _ = workloads.normalised_error(got, ref, workloads.window_sq_norms_at(x, n0, n1, q0, q1))
        worst = max(worst, err)
        sq = torch.from_numpy(workloads.window_sq_norms(x, n0, n1)).cuda()
        e = torch.view_as_real(o).pow(2).sum(dim=(2, 3, 4)).double()
        worst_parseval = max(worst_parseval, float(((e - sq).abs() / sq).max()))
    assert worst <= TOL, f"sampled windows: {worst:.3e}"
    assert worst_parseval <= 1e-5, f"Parseval: {worst_parseval:.3e}"
    total = sum(o.numel() for o in outs)
    assert total == workloads.uneven_batch_output_coeffs()
    del outs, xd, t
    torch.cuda.empty_cache()
