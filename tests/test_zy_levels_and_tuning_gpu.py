"""GPU checks of the tree's level m1 and of the tuning cache's round trip.

* The row levels alone (stage 0, Eq. rowfswft2d) leave in z level m1 of every complete row
  tree: the oracle tree's level dump (the level invariant of Section 4.2).
* The autotuner appends one record per tuned array to SWDFT_TUNE_CACHE and, on a later plan,
  applies this GPU's record without timing.

Collected after the parity files (each file here stands alone).
"""
import json
import math

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


def _dt(x):
    return 1 if np.iscomplexobj(x) else 0


def assert_close_to_oracle(a_gpu, x, n0, n1):
    ref = oracle.swdft2d(x, n0, n1, method="separable", threads=8)
    err, rms = workloads.normalised_error(a_gpu.cpu().numpy(), ref, workloads.window_sq_norms(x, n0, n1))
    assert err <= TOL, f"max normalised error {err:.3e} (rms {rms:.3e})"


@pytest.mark.parametrize("N0,N1,n0,n1,cplx", [(40, 70, 8, 16, False), (36, 90, 4, 64, True),
                                              (50, 45, 32, 2, False)])
def test_row_pass_leaves_level_m1_of_every_tree(sw, N0, N1, n0, n1, cplx):
    """The row levels alone (stage 0, Eq. rowfswft2d) leave in z level m1 of the tree at every
    position whose row tree is complete: the oracle tree's level-m1 dump T[p0][p1][0][k1] at
    p1 = q1 + n1 - 1 (the level invariant: the n1-point DFT of x[p0][p1-n1+1 .. p1]), per row
    window within 1e-5 of its norm."""
    x = workloads.random_array(700 + n1, N0, N1, complex_input=cplx)
    t = sw.Transform([(N0, N1, n0, n1, _dt(x))])
    t.plan.set_tree_config(0, 2, 0, 2, 0, 1, 0)  # two passes: z goes through the workspace
    xd = torch.from_numpy(x).cuda()
    out = t.empty_outputs()
    t.plan.execute_stage(0, [xd.data_ptr()], [out[0].data_ptr()], t._ws_ptr,
                         torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    P1, pad = N1 - n1 + 1, n0 // 2
    z = t.workspace.view(torch.complex64)[pad * P1 * n1:(pad + N0) * P1 * n1].reshape(N0, P1, n1)
    z = z.cpu().numpy()
    _, _, dump = oracle.tree2d(x, n0, n1, norm="none", dump_level=int(math.log2(n1)))
    ref = dump[:, n1 - 1:, :n1]
    sq = np.abs(x) ** 2
    c = np.concatenate([np.zeros((N0, 1)), np.cumsum(sq, axis=1)], axis=1)
    norms = np.sqrt(c[:, n1:] - c[:, :P1])  # ||x[r][q1 .. q1+n1-1]||
    err = (np.abs(z - ref).max(axis=2) / np.maximum(norms, 1e-30)).max()
    assert err <= TOL, f"level m1 vs the oracle's dump: {err:.3e}"


def test_autotune_takes_this_gpus_cached_records(sw, tmp_path, monkeypatch):
    """With SWDFT_TUNE_CACHE holding a record for this GPU and array, autotune applies it
    without timing (nothing appended) and the plan makes the same choice; another GPU's
    record is not applied."""
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("SWDFT_TUNE_CACHE", str(cache))
    x = workloads.random_array(660, 120, 100)
    xd = torch.from_numpy(x).cuda()
    t = sw.Transform([(120, 100, 16, 16, 0)], algo="auto")
    t.autotune([xd])
    first = cache.read_text()
    assert len(first.strip().splitlines()) == 1
    rec = json.loads(first)
    assert rec["gpu"] == torch.cuda.get_device_name()
    t2 = sw.Transform([(120, 100, 16, 16, 0)], algo="auto")
    t2.autotune([xd])
    assert cache.read_text() == first
    assert t2.plan.algo() == t.plan.algo() and t2.plan.launch_count() == t.plan.launch_count()
    a = t2.forward([xd])[0]
    torch.cuda.synchronize()
    assert_close_to_oracle(a, x, 16, 16)
    rec["gpu"] = "another GPU"
    other = tmp_path / "other.jsonl"
    other.write_text(json.dumps(rec) + "\n")
    assert sw.Transform([(120, 100, 16, 16, 0)], algo="auto").plan.load_tuning(str(other)) == 0
    assert sw.Transform([(120, 100, 16, 16, 0)], algo="auto").plan.load_tuning(str(cache)) == 1
