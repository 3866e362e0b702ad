"""Multi-process path on CPU: two gloo ranks each sweep their shard of the start
vectors (the oracle stands in for the GPU sweep here) and combine once; the
result equals the single-process sweep over all vectors."""
import os
import socket

import numpy as np
import pytest

from paper_1308_5467_gb300.shard import combine_moments, torch_all_reduce, vector_shard


def test_vector_shard_partition():
    for n, world in ((64, 2), (65, 4), (3, 8), (1000, 7)):
        spans = [vector_shard(n, world, r) for r in range(world)]
        covered = [i for off, cnt in spans for i in range(off, off + cnt)]
        assert covered == list(range(n))
        assert max(c for _, c in spans) - min(c for _, c in spans) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n_v_total, out_path):
    import torch.distributed as dist

    from oracle import kpm
    from synthetic import laplacian_2d
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A = laplacian_2d(20)
    off, cnt = vector_shard(n_v_total, world, rank)
    mu_local = kpm.kpm_moments(A, -0.1, 8.1, 60, cnt, seed=3, vec_offset=off, nthreads=1)
    mu = combine_moments(mu_local, cnt, n_v_total, torch_all_reduce())
    if rank == 0:
        np.save(out_path, mu)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("n_v_total", [8, 9])
def test_two_gloo_ranks_equal_single_process(tmp_path, n_v_total):
    import torch.multiprocessing as mp

    from oracle import kpm
    from synthetic import laplacian_2d
    out = str(tmp_path / "mu.npy")
    mp.spawn(_worker, args=(2, _free_port(), n_v_total, out), nprocs=2, join=True)
    mu = np.load(out)
    ref = kpm.kpm_moments(laplacian_2d(20), -0.1, 8.1, 60, n_v_total, seed=3)
    assert np.abs(mu - ref).max() < 1e-14
