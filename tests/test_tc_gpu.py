"""The tensor-core (tcgen05) form: row levels on the tree, column DFT as a UMMA product
against the n0-point DFT matrix, against the FP64 oracle.

Bar (Section 4.1, Eq. 2; per-window max error / ||x_w||_2): <= 1e-5 for the 3-term split
bf16 form; plain bf16 and fp16 (with and without the per-image scale) are measured and
reported, and checked only against loose sanity bounds.
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
    assert sw._native.check_device() == 0
    return sw


def run(sw, x, n0, n1, algo, chunk=None):
    N0, N1 = x.shape
    t = sw.Transform([(N0, N1, n0, n1, 1 if np.iscomplexobj(x) else 0)], algo=algo)
    a = t.forward([torch.from_numpy(np.ascontiguousarray(x)).cuda()])[0]
    torch.cuda.synchronize()
    assert sw._native.check_device() == 0, "a tensor-core kernel timed out"
    return a


def err_vs_oracle(a, x, n0, n1):
    ref = oracle.swdft2d(x, n0, n1, method="separable", threads=8)
    return workloads.normalised_error(a.cpu().numpy(), ref, workloads.window_sq_norms(x, n0, n1))


SHAPES = [(64, 64, 16, 16), (100, 90, 32, 32), (70, 140, 16, 64), (150, 60, 64, 8), (80, 200, 32, 8),
          (47, 33, 16, 32), (300, 41, 64, 16)]


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("N0,N1,n0,n1", SHAPES)
def test_split_bf16_meets_tolerance(sw, N0, N1, n0, n1, cplx):
    x = workloads.random_array(N0 + N1, N0, N1, complex_input=cplx)
    a = run(sw, x, n0, n1, "tc_bf16x3")
    err, rms = err_vs_oracle(a, x, n0, n1)
    assert err <= TOL, f"split bf16: max {err:.3e} rms {rms:.3e}"


@pytest.mark.parametrize("algo,bound", [("tc_bf16", 2e-2), ("tc_f16", 5e-3), ("tc_f16_scaled", 5e-3)])
def test_single_term_forms_are_sane(sw, algo, bound):
    x = workloads.random_array(5, 100, 90, complex_input=True)
    a = run(sw, x, 32, 32, algo)
    err, rms = err_vs_oracle(a, x, 32, 32)
    print(f"{algo}: max {err:.3e} rms {rms:.3e}")
    assert err <= bound


def test_fp16_scale_rescues_large_inputs(sw):
    x = workloads.random_array(6, 80, 80) * np.float32(1e4)
    plain = run(sw, x, 32, 32, "tc_f16")
    scaled = run(sw, x, 32, 32, "tc_f16_scaled")
    e_plain, _ = err_vs_oracle(plain, x, 32, 32)
    e_scaled, _ = err_vs_oracle(scaled, x, 32, 32)
    assert e_scaled <= 5e-3
    assert not (e_plain <= 5e-3)  # unscaled fp16 overflows (|z| > 65504)


def test_tc_rejects_small_windows(sw):
    with pytest.raises(sw.SwdftError) as e:
        sw.Transform([(64, 64, 8, 8, 0)], algo="tc_bf16x3")
    assert e.value.status == -4


def _sample_windows(P0, P1, count, seed):
    """count seeded random windows, then every window of the four edges and the centre."""
    rng = np.random.default_rng(seed)
    q0 = [rng.integers(0, P0, count), np.zeros(P1, np.int64), np.full(P1, P0 - 1),
          np.arange(P0), np.arange(P0), [P0 // 2]]
    q1 = [rng.integers(0, P1, count), np.arange(P1), np.arange(P1),
          np.zeros(P0, np.int64), np.full(P0, P1 - 1), [P1 // 2]]
    return np.concatenate(q0).astype(np.int64), np.concatenate(q1).astype(np.int64)


_REF = {}


def _sampled_ref(x, n0, n1, count, seed):
    """The oracle on the sample, computed once per (array, window, sample)."""
    key = (id(x), n0, n1, count, seed)
    if key not in _REF:
        q0, q1 = _sample_windows(x.shape[0] - n0 + 1, x.shape[1] - n1 + 1, count, seed)
        _REF[key] = (q0, q1, oracle.swdft2d_windows(x, n0, n1, q0, q1, threads=8),
                     workloads.window_sq_norms_at(x, n0, n1, q0, q1))
    return _REF[key]


def _full(sw, x, n0, n1, algo, count, seed):
    N0, N1 = x.shape
    P0, P1 = N0 - n0 + 1, N1 - n1 + 1
    a = run(sw, x, n0, n1, algo)
    q0, q1, ref, nrm = _sampled_ref(x, n0, n1, count, seed)
    got = a[torch.from_numpy(q0).cuda(), torch.from_numpy(q1).cuda()].cpu().numpy()
    err, rms = workloads.normalised_error(got, ref, nrm)
    sq = torch.from_numpy(workloads.window_sq_norms(x, n0, n1)).cuda()
    worst = 0.0
    for r in range(0, P0, 64):
        e = torch.view_as_real(a[r:r + 64]).pow(2).sum(dim=(2, 3, 4)).double()
        worst = max(worst, float(((e - sq[r:r + 64]).abs() / sq[r:r + 64]).max()))
    del a
    torch.cuda.empty_cache()
    return err, rms, worst


def test_split_bf16_sinusoids_512_full_size(sw):
    x = workloads.sinusoids_512().images[0]
    err, rms, parseval = _full(sw, x, 32, 32, "tc_bf16x3", 2048, 21)
    assert err <= TOL, (err, rms)
    assert parseval <= 1e-5


_C3 = {}


@pytest.mark.parametrize("algo", ["tc_bf16x3", "tc_f16_scaled"])
def test_complex_1024x2048_full_size(sw, algo):
    """The tree's sample of the 1024x2048 complex workload: 65,536 seeded windows, every
    window of the four edges and the centre."""
    if "x" not in _C3:
        _C3["x"] = workloads.complex_1024x2048().images[0]
    x = _C3["x"]
    err, rms, parseval = _full(sw, x, 16, 64, algo, 65536, 12)
    print(f"{algo}: max {err:.3e} rms {rms:.3e} parseval {parseval:.3e}")
    if algo == "tc_bf16x3":
        assert err <= TOL and parseval <= 1e-5
    else:
        assert err <= 5e-3
