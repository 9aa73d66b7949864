"""Host logic of the multi-GPU (replicas) path on CPU with 2 gloo ranks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2602_20097_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 10.0 + 5.0 * rank                # rank 1 is the slow one
        ms_max = replicas.max_over_ranks(ms_local)
        owned = list(replicas.shard(96, rank, world))
        results[rank] = (ms_max, owned, replicas.rank_seed(2, rank))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_partition():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    results = mgr.dict()
    mp.spawn(_worker, args=(world, port, results), nprocs=world, join=True)
    assert results[0][0] == results[1][0] == 15.0
    covered = sorted(results[0][1] + results[1][1])
    assert covered == list(range(96))
    assert results[0][2] != results[1][2]
    gbs = replicas.whole_job_gbs(4 * 512 ** 3, world, results[0][0])
    assert gbs == pytest.approx(4 * 512 ** 3 * 2 / 15e-3 / 1e9)


@pytest.mark.parametrize("n,world", [(96, 1), (96, 5), (7, 8), (0, 3)])
def test_shard_is_a_partition(n, world):
    parts = [list(replicas.shard(n, r, world)) for r in range(world)]
    assert sorted(sum(parts, [])) == list(range(n))
    sizes = [len(p) for p in parts]
    assert max(sizes) - min(sizes) <= 1


def test_max_over_ranks_without_group():
    assert replicas.max_over_ranks(3.5) == 3.5
