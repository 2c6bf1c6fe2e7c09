"""The multi-GPU split on the CPU: two gloo ranks each take a band of window rows (one
process per GPU in production), and the concatenation of their bands equals the unsplit
transform (Section 4.1, Eq. 2, by the FP64 oracle).  Also the band arithmetic and the
max-over-ranks timing reduction."""
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
