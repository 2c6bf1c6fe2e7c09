"""Guard-region tests: every entry point writes only inside the buffers it is given.

Each device buffer handed to the library (output, workspace, stream state, and the input,
which must stay unchanged) sits between two 4 KiB guard regions filled with a sentinel byte;
after the call the guards must hold the sentinel still, and the result must equal the same
call on the library's usual (unguarded) buffers bit for bit.  The sentinel 0xA5 reads as a
small negative float32, never a NaN, so regions the kernels read but never need (z's padding
rows) stay harmless.  The helper itself is checked on CPU tensors.
"""
import numpy as np
import pytest
import torch

import workloads

GUARD = 4096  # bytes on each side; keeps every view 256-byte aligned
FILL = 0xA5


class Guarded:
    """nbytes of device memory with GUARD sentinel bytes on each side."""

    def __init__(self, nbytes, device="cuda"):
        self.n = int(nbytes)
        self.raw = torch.full((self.n + 2 * GUARD,), FILL, dtype=torch.uint8, device=device)

    def ptr(self):
        return self.raw.data_ptr() + GUARD

    def view(self, dtype, shape):
        return self.raw[GUARD:GUARD + self.n].view(dtype).view(shape)

    def intact(self):
        return bool((self.raw[:GUARD] == FILL).all()) and bool((self.raw[GUARD + self.n:] == FILL).all())


def guarded_copy(t):
    """A guarded buffer holding a copy of tensor t (same dtype and shape)."""
    g = Guarded(t.numel() * t.element_size(), device=t.device)
    g.view(t.dtype, t.shape).copy_(t)
    return g


def test_guard_helper_detects_writes_outside_the_view():
    g = Guarded(64, device="cpu")
    v = g.view(torch.complex64, (2, 4))
    v.fill_(1 + 2j)
    assert g.intact()
    assert (g.ptr() - g.raw.data_ptr()) % 256 == 0
    g.raw[GUARD + 64] = 0  # one byte past the end
    assert not g.intact()
    h = Guarded(16, device="cpu")
    h.raw[GUARD - 1] = 7   # one byte before the start
    assert not h.intact()
    c = guarded_copy(torch.arange(6, dtype=torch.float32).reshape(2, 3))
    assert torch.equal(c.view(torch.float32, (2, 3)), torch.arange(6, dtype=torch.float32).reshape(2, 3))
    assert c.intact()


# ------------------------------------------------------------------------------- GPU cases

@pytest.fixture(scope="module")
def sw():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1707_08213_gb300 as sw
    return sw


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _dtype(x):
    return torch.complex64 if np.iscomplexobj(x) else torch.float32


FORWARD = [  # (N0, N1, n0, n1, complex, algo)
    (40, 33, 4, 4, False, "tree"),        # fused form
    (64, 77, 8, 16, False, "tree"),
    (70, 50, 8, 32, True, "tree"),
    (100, 100, 64, 64, False, "tree"),
    (150, 60, 64, 8, True, "tree"),
    (512, 512, 32, 32, False, "tree"),    # the bench's shape
    (60, 61, 27, 27, False, "tree"),      # ternary trees
    (50, 41, 9, 4, True, "tree"),
    (100, 90, 32, 32, False, "tc_bf16x3"),
    (70, 140, 16, 64, True, "tc_bf16x3"),
    (300, 41, 64, 16, False, "tc_bf16"),
]


@pytest.mark.gpu
@pytest.mark.parametrize("N0,N1,n0,n1,cplx,algo", FORWARD)
def test_forward_writes_only_its_output_and_workspace(sw, N0, N1, n0, n1, cplx, algo):
    x = workloads.random_array(N0 * 7 + N1, N0, N1, complex_input=cplx)
    xd = torch.from_numpy(x).cuda()
    t = sw.Transform([(N0, N1, n0, n1, 1 if cplx else 0)], algo=algo)
    ref = t.forward([xd])[0]
    shape = t.output_shapes()[0]
    gx = guarded_copy(xd)
    gout = Guarded(ref.numel() * 8)
    gws = Guarded(t.plan.workspace_size())
    t.plan.execute([gx.ptr()], [gout.ptr()], gws.ptr(), _stream())
    torch.cuda.synchronize()
    assert gx.intact() and gout.intact() and gws.intact()
    assert torch.equal(gx.view(_dtype(x), (N0, N1)), xd), "the input changed"
    assert torch.equal(gout.view(torch.complex64, shape), ref)


@pytest.mark.gpu
def test_batch_forms_write_only_their_buffers(sw):
    shapes = [(70, 50, 8, 32, 0), (33, 90, 16, 4, 1), (64, 64, 64, 16, 0), (20, 20, 4, 4, 0)]
    xs = [torch.from_numpy(workloads.random_array(40 + i, s[0], s[1], complex_input=bool(s[4]))).cuda()
          for i, s in enumerate(shapes)]
    for flags in (0, sw.FLAG_GRAPH, sw.FLAG_PERSISTENT, sw.FLAG_PERSISTENT | sw.FLAG_GRAPH):
        t = sw.Transform(shapes, flags=flags)
        refs = t.forward(xs)
        gxs = [guarded_copy(x) for x in xs]
        gouts = [Guarded(r.numel() * 8) for r in refs]
        gws = Guarded(t.plan.workspace_size())
        for _ in range(2):  # graph plans capture on the first call and replay on the second
            t.plan.execute([g.ptr() for g in gxs], [g.ptr() for g in gouts], gws.ptr(), _stream())
        torch.cuda.synchronize()
        assert all(g.intact() for g in gxs + gouts) and gws.intact(), f"flags {flags}"
        for g, r in zip(gouts, refs):
            assert torch.equal(g.view(torch.complex64, r.shape), r), f"flags {flags}"


@pytest.mark.gpu
@pytest.mark.parametrize("N0,N1,n0,n1,cplx,count", [
    (64, 77, 8, 16, False, 1),
    (256, 256, 16, 16, False, 8),   # grouped launches, chunks with side rows and the fold
    (40, 300, 4, 64, True, 3),
    (300, 20, 64, 2, False, 1),
])
def test_adjoint_writes_only_its_gradient_and_workspace(sw, N0, N1, n0, n1, cplx, count):
    t = sw.Transform([(N0, N1, n0, n1, 1 if cplx else 0)] * count)
    P0, P1 = N0 - n0 + 1, N1 - n1 + 1
    rng = np.random.default_rng(N0 + N1 + count)
    gs = [torch.from_numpy((rng.standard_normal((P0, P1, n0, n1)) +
                            1j * rng.standard_normal((P0, P1, n0, n1))).astype(np.complex64)).cuda()
          for _ in range(count)]
    refs = t.adjoint(gs)
    ggs = [guarded_copy(g) for g in gs]
    gouts = [Guarded(r.numel() * r.element_size()) for r in refs]
    gws = Guarded(t.plan.workspace_size())
    t.plan.execute_adjoint([g.ptr() for g in ggs], [g.ptr() for g in gouts], gws.ptr(), _stream())
    torch.cuda.synchronize()
    assert all(g.intact() for g in ggs + gouts) and gws.intact()
    for gg, g in zip(ggs, gs):
        assert torch.equal(gg.view(torch.complex64, g.shape), g), "the upstream gradient changed"
    for go, r in zip(gouts, refs):
        assert torch.equal(go.view(r.dtype, r.shape), r)


@pytest.mark.gpu
@pytest.mark.parametrize("N,n", [((20, 24, 28), (4, 8, 2)), ((9, 10, 11, 12), (2, 4, 1, 8))])
def test_kd_writes_only_its_output_and_workspace(sw, N, n):
    x = torch.from_numpy(np.random.default_rng(sum(N)).standard_normal(N).astype(np.float32)).cuda()
    t = sw.TransformKD(N, n)
    ref = t.forward(x)
    gx = guarded_copy(x)
    gout = Guarded(ref.numel() * 8)
    gws = Guarded(t.plan.workspace_size())
    t.plan.execute(gx.ptr(), gout.ptr(), gws.ptr(), _stream())
    torch.cuda.synchronize()
    assert gx.intact() and gout.intact() and gws.intact()
    assert torch.equal(gx.view(torch.float32, N), x)
    assert torch.equal(gout.view(torch.complex64, ref.shape), ref)


@pytest.mark.gpu
@pytest.mark.parametrize("N1,n0,n1,max_rows,pieces", [
    (64, 8, 4, 16, [1, 3, 16, 16, 2, 9]),     # kept input rows, fused launches
    (80, 8, 64, 5, [1, 5, 5, 2, 5, 5, 5]),    # kept z rows, row and column passes
    (50, 32, 1, 40, [31, 1, 40, 7]),
])
def test_stream_writes_only_its_output_and_state(sw, N1, n0, n1, max_rows, pieces):
    N0 = sum(pieces)
    x = torch.from_numpy(workloads.random_array(N0 + N1, N0, N1)).cuda()
    ref_stream = sw.SlidingStream(N1, n0, n1, max_rows=max_rows)
    plan = sw.StreamPlan(N1, n0, n1, max_rows=max_rows)
    gstate = Guarded(plan.state_size())
    gx = guarded_copy(x)
    base = gx.view(torch.float32, (N0, N1))
    r = 0
    for R in pieces:
        _, want = ref_stream.push(x[r:r + R])
        gout = Guarded(want.numel() * 8)
        n, _ = plan.push(base[r:r + R].data_ptr(), R, N1, gout.ptr() if want.numel() else 0,
                         gstate.ptr(), _stream())
        torch.cuda.synchronize()
        assert n == want.shape[0]
        assert gout.intact() and gstate.intact() and gx.intact()
        assert torch.equal(gout.view(torch.complex64, want.shape), want)
        r += R
    assert torch.equal(base, x)
