"""Failure injection on the host (no GPU fault): device allocations made to fail one after the
other through swdft2d_inject_alloc_failure return SWDFT_ERR_OOM, and the same call repeated
once injection is off completes with the expected result (each call keeps what it did
allocate and resumes from there)."""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1707_08213_gb300 as sw
    return sw


def _stream():
    return torch.cuda.current_stream().cuda_stream


def test_host_buffer_path_fails_at_each_device_buffer_then_recovers(sw):
    nat = sw._native
    x = workloads.random_array(77, 90, 70)
    want = sw.Transform([(90, 70, 8, 16, 0)]).forward([torch.from_numpy(x).cuda()])[0].cpu()
    t = sw.Transform([(90, 70, 8, 16, 0)], flags=sw.FLAG_HOST_IO)
    h_in = torch.from_numpy(x).pin_memory()
    h_out = torch.zeros(tuple(want.shape), dtype=torch.complex64).pin_memory()
    try:
        # input, workspace, then the two output bands: each attempt gets one more of them
        for after in (0, 1, 1, 1):
            nat.inject_alloc_failure(after)
            with pytest.raises(nat.SwdftError) as e:
                t.plan.execute_host([h_in.data_ptr()], [h_out.data_ptr()], _stream())
            assert e.value.status == -5
    finally:
        nat.inject_alloc_failure(-1)
    t.plan.execute_host([h_in.data_ptr()], [h_out.data_ptr()], _stream())
    torch.cuda.synchronize()
    assert torch.equal(h_out, want)


def test_persistent_plan_fails_at_each_descriptor_table_then_recovers(sw):
    nat = sw._native
    shapes = [(70, 50, 8, 32, 0), (20, 20, 4, 4, 0), (64, 64, 64, 16, 0)]
    xs = [torch.from_numpy(workloads.random_array(90 + i, s[0], s[1])).cuda() for i, s in enumerate(shapes)]
    want = sw.Transform(shapes).forward(xs)
    t = sw.Transform(shapes, flags=sw.FLAG_PERSISTENT)
    outs = t.empty_outputs()
    try:
        # pinned staging, device copy, graph copy of the descriptors, then the pipelined
        # kernels' tile table: each attempt gets one more of them
        for after in (0, 1, 1, 1):
            nat.inject_alloc_failure(after)
            with pytest.raises(nat.SwdftError) as e:
                t.forward(xs, outs)
            assert e.value.status == -5
    finally:
        nat.inject_alloc_failure(-1)
    t.forward(xs, outs)
    torch.cuda.synchronize()
    for o, w in zip(outs, want):
        assert torch.equal(o, w)


def test_bounded_device_wait_times_out_and_reports(sw):
    """A device wait that runs out (an mbarrier nothing arrives on, 64 polls of at most
    about 1 ms) is recorded in the device status word, read and reset by check_device; the
    context stays usable for the tensor-core kernels that use the same bounded waits."""
    nat = sw._native
    nat.check_device()  # clear any earlier record
    nat.selftest_wait_timeout(64, _stream())
    torch.cuda.synchronize()
    assert nat.check_device() == -7
    assert nat.check_device() == 0
    x = workloads.random_array(5, 100, 90)
    xd = torch.from_numpy(x).cuda()
    a = sw.Transform([(100, 90, 32, 32, 0)], algo="tc_bf16x3").forward([xd])[0]
    b = sw.Transform([(100, 90, 32, 32, 0)]).forward([xd])[0]
    torch.cuda.synchronize()
    assert nat.check_device() == 0
    # per window, |difference| / window norm: the split form's 1e-5 bar
    d = (a - b).abs().amax(dim=(2, 3)).cpu().numpy()
    assert float((d / np.sqrt(workloads.window_sq_norms(x, 32, 32))).max()) <= 1e-5
