"""The multi-GPU split on the CPU: two gloo ranks each take a band of window rows (one
process per GPU in production), and the concatenation of their bands equals the unsplit
transform (Section 4.1, Eq. 2, by the FP64 oracle); two ranks split a batch of images by
longest processing time and together cover it.  Also the band arithmetic, the image
assignment's balance bound and the max-over-ranks timing reduction."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _load_sharding():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_swdft_sharding", os.path.join(ROOT, "paper_1707_08213_gb300", "sharding.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_bands_cover_every_row_once():
    sh = _load_sharding()
    for P0 in (1, 2, 7, 57, 481):
        for world in (1, 2, 3, 8, 600):
            rows = []
            for r in range(world):
                b, e = sh.band_for_rank(P0, r, world)
                assert 0 <= b <= e <= P0
                rows.extend(range(b, e))
            assert rows == list(range(P0))
    assert sh.input_rows_for_band(10, 20, 8) == (10, 27)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, outdir):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import oracle
    import workloads
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sh = _load_sharding()
    x = workloads.random_array(77, 40, 30, complex_input=True)
    n0, n1 = 8, 4
    P0 = x.shape[0] - n0 + 1
    b, e = sh.band_for_rank(P0, rank, world)
    r0, r1 = sh.input_rows_for_band(b, e, n0)
    band = oracle.swdft2d(x[r0:r1], n0, n1) if e > b else np.zeros((0,), np.complex128)
    np.save(os.path.join(outdir, f"band{rank}.npy"), band)
    t = sh.max_over_ranks(1.0 + rank, dist)
    np.save(os.path.join(outdir, f"max{rank}.npy"), np.array([t]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_band_split_equals_unsplit(tmp_path):
    import oracle
    import workloads
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    x = workloads.random_array(77, 40, 30, complex_input=True)
    full = oracle.swdft2d(x, 8, 4)
    parts = [np.load(tmp_path / f"band{r}.npy") for r in range(world)]
    assert np.array_equal(np.concatenate(parts, axis=0), full)
    for r in range(world):
        assert float(np.load(tmp_path / f"max{r}.npy")[0]) == 2.0



def _plan_band_worker(rank, world, port, outdir):
    """Each rank builds the plan a multi-GPU bench run builds for its band (host only: plan
    creation makes no CUDA call) and records what the library made of the band."""
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import __graft_entry__
    __graft_entry__.build()
    from paper_1707_08213_gb300 import _native as nat
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sh = _load_sharding()
    N0, N1, n0, n1 = 512, 512, 32, 32
    P0 = N0 - n0 + 1
    bands = sh.plan_bands(P0, rank, world)
    assert bands == [sh.band_for_rank(P0, rank, world)]
    spec = {"N0": N0, "N1": N1, "n0": n0, "n1": n1, "dtype": nat.R32}
    spec["row_begin"], spec["row_end"] = bands[0]
    plan = nat.Plan([spec])
    np.save(os.path.join(outdir, f"plan{rank}.npy"), np.array([*bands[0], *plan.output_shape(0)]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_plans_take_the_ranks_bands(tmp_path):
    """The bands handed to swdft2d_shape (row_begin/row_end) are band_for_rank's, and the
    plans' outputs (P0 rows split between the ranks) tile the transform's window rows."""
    world = 2
    mp.spawn(_plan_band_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    sh = _load_sharding()
    rows = []
    for r in range(world):
        b, e, p0, p1, k0, k1 = (int(v) for v in np.load(tmp_path / f"plan{r}.npy"))
        assert (b, e) == sh.band_for_rank(481, r, world)
        assert (p0, p1, k0, k1) == (e - b, 481, 32, 32)
        rows.extend(range(b, e))
    assert rows == list(range(481))
    assert sh.plan_bands(481, 0, 1) is None


def test_image_assignment_covers_and_balances():
    sh = _load_sharding()
    rng = np.random.default_rng(3)
    sides = rng.choice([128, 256, 512, 1024], size=(256, 2))
    wins = [(4, 4), (8, 8), (16, 16), (32, 32), (8, 32), (64, 16)]
    costs = [sh.output_bytes(int(a), int(b), *wins[int(k)]) for (a, b), k in zip(sides, rng.integers(0, 6, 256))]
    for world in (1, 2, 3, 4, 8, 300):
        parts = sh.assign_images(costs, world)
        assert len(parts) == world
        assert sorted(i for p in parts for i in p) == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        lower = max(max(costs), sum(costs) / world)  # no split can beat this
        assert max(loads) <= (4 / 3 - 1 / (3 * world)) * lower * (1 + 1e-12) + 1e-9 or max(loads) == max(costs)
    assert sh.assign_images([5, 5, 4, 3, 3], 2) == [[0, 2], [1, 3, 4]]  # loads 9 and 11
    assert sh.assign_images([], 3) == [[], [], []]


def _batch_worker(rank, world, port, outdir):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import oracle
    import workloads
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sh = _load_sharding()
    shapes = [(20, 30, 4, 8), (40, 16, 8, 2), (12, 12, 4, 4), (33, 21, 16, 8), (25, 25, 2, 2)]
    mine = sh.assign_images([sh.output_bytes(*s) for s in shapes], world)[rank]
    for i in mine:
        N0, N1, n0, n1 = shapes[i]
        x = workloads.random_array(90 + i, N0, N1)
        np.save(os.path.join(outdir, f"img{i}_rank{rank}.npy"), oracle.swdft2d(x, n0, n1))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_image_split_covers_the_batch(tmp_path):
    import oracle
    import workloads
    world = 2
    mp.spawn(_batch_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    shapes = [(20, 30, 4, 8), (40, 16, 8, 2), (12, 12, 4, 4), (33, 21, 16, 8), (25, 25, 2, 2)]
    files = sorted(os.listdir(tmp_path))
    assert len(files) == len(shapes)  # each image computed by exactly one rank
    for i, (N0, N1, n0, n1) in enumerate(shapes):
        got = [f for f in files if f.startswith(f"img{i}_")]
        assert len(got) == 1
        ref = oracle.swdft2d(workloads.random_array(90 + i, N0, N1), n0, n1)
        assert np.array_equal(np.load(tmp_path / got[0]), ref)
