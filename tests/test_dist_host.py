"""The multi-process host logic of bench.py on CPU with the gloo backend and
two ranks: photon ranges per rank are disjoint and together give exactly the
single-process run (the oracle stands in for the kernel here), and the job
rate takes the slowest rank's time and the summed steps."""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_PER_RANK = 3000


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    import oracle
    off, n = bench.photon_range(rank, N_PER_RANK)
    r = oracle.walk(mu_s=3.0 / 45.0, phase="hg", hg_g=0.8, n_photons=n, photon_offset=off, nx=16, nz=16,
                    n_threads=1)
    img = torch.tensor(r["image"])
    dist.all_reduce(img, op=dist.ReduceOp.SUM)
    rate, t_max, total = bench.job_rate(1.0 + rank, r["steps"], ws, torch.device("cpu"))
    if rank == 0:
        np.save(os.path.join(out_dir, "img.npy"), img.numpy())
        np.save(os.path.join(out_dir, "rate.npy"), np.array([rate, t_max, total]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_one_run(tmp_path, oracle_mod):
    import torch.multiprocessing as mp
    ws = 2
    mp.spawn(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    img = np.load(tmp_path / "img.npy")
    rate, t_max, total = np.load(tmp_path / "rate.npy")
    one = oracle_mod.walk(mu_s=3.0 / 45.0, phase="hg", hg_g=0.8, n_photons=ws * N_PER_RANK, nx=16, nz=16,
                          n_threads=1)
    np.testing.assert_allclose(img, one["image"], rtol=1e-12, atol=1e-15)
    assert t_max == 2.0                     # the slower rank
    assert total == one["steps"]            # steps summed over ranks
    assert rate == pytest.approx(one["steps"] / 2.0)


def test_photon_ranges_partition():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    spans = [bench.photon_range(r, 1000) for r in range(8)]
    assert spans[0] == (0, 1000)
    for (a, n), (b, _) in zip(spans, spans[1:]):
        assert a + n == b
