"""The streaming form (include/swdftstream.h): rows pushed over time in pieces of any size;
the window rows each push emits must be the same rows of one transform of the whole array
(bit for bit: the same node arithmetic, whether the kept rows are input rows (n1 <= 32 and
pushes of at most 4 n0 rows) or z rows), and within 1e-5 of the FP64 oracle (Section 4.1 Eq. 2, per-window error /
window norm)."""
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


def stream_all(sw, x, n0, n1, pieces, max_rows, norm="unitary", ld_pad=0):
    N0, N1 = x.shape
    cplx = np.iscomplexobj(x)
    st = sw.SlidingStream(N1, n0, n1, dtype=1 if cplx else 0, norm=norm, max_rows=max_rows)
    wide = np.zeros((N0, N1 + ld_pad), dtype=x.dtype)
    wide[:, :N1] = x
    xd = torch.from_numpy(wide).cuda()
    outs, r, expect_first = [], 0, 0
    for R in pieces:
        R = min(R, N0 - r)
        first, o = st.push(xd[r:r + R, :N1])
        assert first == expect_first
        expect_first += o.shape[0]
        outs.append(o)
        r += R
        if r == N0:
            break
    assert r == N0
    torch.cuda.synchronize()
    return torch.cat(outs), st


def check(sw, x, n0, n1, got, norm="unitary"):
    N0, N1 = x.shape
    full = sw.Transform([(N0, N1, n0, n1, 1 if np.iscomplexobj(x) else 0)], norm=norm).forward(
        [torch.from_numpy(x).cuda()])[0]
    torch.cuda.synchronize()
    assert got.shape == full.shape
    assert torch.equal(got, full)
    ref = oracle.swdft2d(x, n0, n1, norm=norm, method="separable", threads=8)
    to_unitary = oracle.scale_for("unitary", n0, n1) / oracle.scale_for(norm, n0, n1)
    err, _ = workloads.normalised_error(got.cpu().numpy(), ref, workloads.window_sq_norms(x, n0, n1),
                                        to_unitary)
    assert err <= TOL, f"{err:.3e}"


@pytest.mark.parametrize("N0,N1,n0,n1,cplx,pieces,max_rows", [
    (150, 77, 16, 8, False, [1, 3, 16, 5, 1, 1, 40, 7, 2, 40, 40], 40),
    (90, 64, 8, 32, True, [1] * 90, 1),                 # one row per push: many history moves
    (70, 50, 1, 16, False, [2, 5, 9, 30, 30], 30),      # n0 = 1: no history (z rows kept)
    (200, 40, 64, 4, True, [10, 63, 1, 64, 64], 64),    # the longest column tree
    (41, 33, 32, 1, False, [31, 1, 9], 31),             # n1 = 1, first window after 32 rows
    (60, 100, 8, 64, False, [1, 5, 20, 20, 14], 20),    # n1 = 64: kept rows are z rows
    (50, 90, 16, 64, True, [1] * 50, 1),                # the same, one row per push
])
def test_pieces_match_one_transform(sw, N0, N1, n0, n1, cplx, pieces, max_rows):
    x = workloads.random_array(N0 + N1 + n0, N0, N1, complex_input=cplx)
    got, _ = stream_all(sw, x, n0, n1, pieces, max_rows)
    check(sw, x, n0, n1, got)


def test_strided_rows_and_normalisation(sw):
    x = workloads.random_array(61, 60, 45, complex_input=True)
    got, _ = stream_all(sw, x, 8, 8, [7] * 9, 7, norm="inv_n", ld_pad=13)
    check(sw, x, 8, 8, got, norm="inv_n")


def test_reset_starts_a_new_array(sw):
    a = workloads.random_array(62, 40, 30)
    b = workloads.random_array(63, 50, 30)
    st = sw.SlidingStream(30, 8, 4, max_rows=16)
    for x in (a, b):
        st.reset()
        xd = torch.from_numpy(x).cuda()
        outs = [st.push(xd[i:i + 16])[1] for i in range(0, x.shape[0], 16)]
        torch.cuda.synchronize()
        check(sw, x, 8, 4, torch.cat(outs))
