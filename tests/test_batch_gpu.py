"""The persistent batched launch (SWDFT_FLAG_PERSISTENT): many arrays of uneven sizes and
window shapes in one persistent kernel per window shape (a pipelined row+column kernel for
the two-pass arrays, a fused kernel for small windows), optionally replayed from a CUDA
graph, against the FP64 oracle (Section 4.1, Eq. 2; per-window error / window norm <= 1e-5);
the pipelined kernels' bounded waits made to run out through the test hook."""
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
    # one pipelined kernel per (n0, n1) of the two-pass arrays, one fused kernel per (n0, n1)
    # of the fused arrays (small windows: n0 n1 <= 64, n1 < 64)
    fused = [(n0, n1) for _, _, n0, n1, _ in MIXED if n0 * n1 <= 64 and n1 < 64]
    two = [(n0, n1) for _, _, n0, n1, _ in MIXED if (n0, n1) not in fused]
    assert t.plan.launch_count() == len(set(two)) + len(set(fused))
    assert t.plan.launch_count() == 9
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


def test_persistent_bands_match_per_array_launches(sw):
    """Bands of window rows (row_begin/row_end) in a persistent plan: the pipelined and fused
    kernels start at the band's first input row, bit for bit the per-array result."""
    shapes = [(300, 90, 32, 32, 0), (200, 70, 16, 64, 1), (150, 40, 8, 8, 0), (260, 33, 64, 16, 0)]
    bands = [(37, 211), (0, 5), (100, 0), (1, 2)]
    xs = [workloads.random_array(70 + i, s[0], s[1], complex_input=bool(s[4])) for i, s in enumerate(shapes)]
    xd = [torch.from_numpy(x).cuda() for x in xs]
    a = sw.Transform(shapes, bands=bands).forward(xd)
    b = sw.Transform(shapes, bands=bands, flags=sw.FLAG_PERSISTENT).forward(xd)
    torch.cuda.synchronize()
    assert sw._native.check_device() == 0
    for u, v in zip(a, b):
        assert torch.equal(u, v)


def test_pipelined_wait_gives_up_then_the_next_launch_is_clean(sw):
    """The test hook makes array 0's column tiles wait for a row tile that never runs: the
    bounded wait (about 1 ms of clock64 cycles) gives up, every block of the launch stops,
    check_device reports the time-out; with the hook off the same plan runs clean and
    matches the per-array result bit for bit."""
    nat = sw._native
    shapes = [(130, 64, 64, 16, 0), (70, 50, 8, 32, 0), (20, 20, 4, 4, 0)]
    xs = [workloads.random_array(80 + i, s[0], s[1]) for i, s in enumerate(shapes)]
    xd = [torch.from_numpy(x).cuda() for x in xs]
    want = sw.Transform(shapes).forward(xd)
    t = sw.Transform(shapes, flags=sw.FLAG_PERSISTENT)
    torch.cuda.synchronize()
    assert nat.check_device() == 0
    try:
        nat.debug_batch_wait(2_000_000, 1)
        t.forward(xd)
        torch.cuda.synchronize()
        assert nat.check_device() == -7
    finally:
        nat.debug_batch_wait(0, 0)
    got = t.forward(xd)
    torch.cuda.synchronize()
    assert nat.check_device() == 0
    for u, v in zip(want, got):
        assert torch.equal(u, v)


def test_persistent_tensor_core_arrays_match_per_array_launches(sw):
    """A persistent plan made with the split-bf16 tensor-core form runs each array through the
    per-array tensor-core launches beside the persistent kernels: bit for bit the per-array
    plan's result, within the 1e-5 bar of the oracle."""
    shapes = [(70, 140, 16, 64, 0), (100, 90, 32, 32, 1), (150, 60, 64, 8, 0)]
    xs = [workloads.random_array(60 + i, s[0], s[1], complex_input=bool(s[4])) for i, s in enumerate(shapes)]
    xd = [torch.from_numpy(x).cuda() for x in xs]
    a = sw.Transform(shapes, algo="tc_bf16x3").forward(xd)
    t = sw.Transform(shapes, algo="tc_bf16x3", flags=sw.FLAG_PERSISTENT | sw.FLAG_GRAPH)
    assert t.plan.launch_count() == 2 * len(shapes)
    b = t.forward(xd)
    b = t.forward(xd)  # replayed from the graph
    torch.cuda.synchronize()
    assert sw._native.check_device() == 0
    for u, v, x, s in zip(a, b, xs, shapes):
        assert torch.equal(u, v)
        _check(v, x, s[2], s[3])


def test_persistent_plan_with_ternary_and_mixed_radix_arrays(sw):
    """Ternary and mixed-radix windows in a persistent plan run on their own launches beside
    the pipelined and fused kernels: bit for bit the per-array plan's result, also after the
    autotuner (which leaves them on their own)."""
    shapes = [(90, 80, 27, 9, 0), (70, 100, 12, 16, 1), (130, 64, 64, 16, 0), (40, 40, 4, 4, 0),
              (60, 75, 6, 48, 0)]
    xs = [workloads.random_array(40 + i, s[0], s[1], complex_input=bool(s[4])) for i, s in enumerate(shapes)]
    xd = [torch.from_numpy(x).cuda() for x in xs]
    want = sw.Transform(shapes).forward(xd)
    t = sw.Transform(shapes, flags=sw.FLAG_PERSISTENT | sw.FLAG_GRAPH)
    assert [t.plan.form(i)[1] for i in range(len(shapes))] == ["per_array", "per_array", "pipelined",
                                                              "fused_group", "per_array"]
    got = t.forward(xd)
    got = t.forward(xd)
    tuned = sw.Transform(shapes, algo="auto", flags=sw.FLAG_PERSISTENT)
    out_t = tuned.autotune(xd)
    tuned.forward(xd, out_t)
    torch.cuda.synchronize()
    assert sw._native.check_device() == 0
    for i, (u, v, w) in enumerate(zip(want, got, out_t)):
        assert torch.equal(u, v)
        if i in (0, 1, 4):
            assert tuned.plan.form(i)[1] == "per_array"
            assert torch.equal(u, w)
        _check(v, xs[i], shapes[i][2], shapes[i][3])


def test_persistent_autotuned_batch_of_mixed_shapes(sw):
    """algo="auto" with a persistent plan: the autotuner times each window shape's arrays in
    the pipelined kernel, the fused kernel, per-array tree launches and per-array split-bf16
    launches, and keeps the fastest per shape; whatever it keeps, every array meets the 1e-5
    bar, also replayed from a graph."""
    xs = _inputs()
    shapes = [(N0, N1, n0, n1, int(c)) for (N0, N1, n0, n1, c) in MIXED]
    xd = [torch.from_numpy(x).cuda() for x in xs]
    t = sw.Transform(shapes, algo="auto", flags=sw.FLAG_PERSISTENT | sw.FLAG_GRAPH)
    outs = t.autotune(xd)
    assert t.plan.launch_count() >= 1
    for _ in range(2):
        for o in outs:
            o.fill_(float("nan"))
        t.forward(xd, outs)
    torch.cuda.synchronize()
    assert sw._native.check_device() == 0
    for o, x, (N0, N1, n0, n1, c) in zip(outs, xs, MIXED):
        _check(o, x, n0, n1)


def test_uneven_batch_256_full_size(sw):
    """256 float32 images, sides in {128..1024}, windows from six shapes, one persistent
    kernel per window shape: >= 256 sampled windows per image against the oracle, and
    per-window Parseval on every window of every image."""
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
