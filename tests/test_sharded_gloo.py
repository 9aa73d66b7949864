"""The sharded orchestration (Section VII-B) on CPU, no GPU.

Two gloo processes run ``sharded.run_rank`` with the oracle-backed host stages
of ``shard_stages_cpu`` (same interface as the CUDA stages): slabs, ghost
planes, bands and every all-to-all are the product code; each process's
result slab must equal the oracle's whole-field result (exact strategy), its
approximate strategy, or Algorithm 4 per slab, bit for bit. More process
counts run as threads over the in-process hub.
"""
import os
import socket
import threading
import zlib

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2602_20097_gb300 import sharded
from tests import oracle_checks as oc
from tests.shard_stages_cpu import CpuStages

FIELDS = [((10, 9, 8), "smooth", 0.01), ((12, 15), "sparse", 0.05), ((9, 7, 6), "step", 0.02),
          ((16, 11), "smooth", 0.01), ((8, 10), "top", 0.1)]


def _field(shape, kind):
    if kind == "top":   # boundaries in the first slab only: the strategies differ
        q = np.zeros(shape, np.int32)
        q[:2] = 1
        return q
    rng = np.random.default_rng(zlib.crc32(repr((shape, kind)).encode()))
    return oc.random_index_field(rng, shape, kind)


def _expected(q, eb, strategy, nparts):
    if strategy == "exact":
        return oracle.mitigate(q, eb, debug=False)["out"]
    if strategy == "approximate":
        return oracle.mitigate_approx(q, eb, nparts)["out"]
    return oracle.mitigate_independent(q, eb, nparts)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        comm = sharded.TorchComm()
        for i, (shape, kind, eb) in enumerate(FIELDS):
            q = _field(shape, kind)
            b, e = sharded.slab_bounds(shape[0], world)[rank]
            for strategy in sharded.STRATEGIES:
                out = sharded.run_rank(CpuStages(), comm, torch.from_numpy(q[b:e].copy()), shape, eb, strategy)
                results[(rank, i, strategy)] = out.numpy()
    finally:
        dist.destroy_process_group()


def test_two_gloo_processes_reproduce_the_oracle():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    results = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), results), nprocs=world, join=True)
    differs = 0
    for i, (shape, kind, eb) in enumerate(FIELDS):
        q = _field(shape, kind)
        for strategy in sharded.STRATEGIES:
            got = np.concatenate([results[(r, i, strategy)] for r in range(world)])
            want = _expected(q, eb, strategy, world)
            np.testing.assert_array_equal(got, want, err_msg=f"{shape} {kind} {strategy}")
        differs += int((oracle.mitigate_approx(q, eb, world)["out"] != oracle.mitigate(q, eb)["out"]).sum())
    assert differs > 0   # the approximate strategy departs somewhere on these fields


def run_threads(stages_fn, q, dims, eb, P, strategy):
    hub = sharded.LoopbackHub(P, timeout=120)
    res, errs = [None] * P, []
    slabs = sharded.slab_bounds(dims[0], P)

    def work(r):
        try:
            b, e = slabs[r]
            res[r] = sharded.run_rank(stages_fn(), hub.comm(r), q[b:e].contiguous(), dims, eb, strategy)
        except BaseException as ex:  # noqa: BLE001 - re-raised below
            errs.append(ex)
            hub.barrier.abort()

    ts = [threading.Thread(target=work, args=(r,)) for r in range(P)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if errs:
        raise errs[0]
    return torch.cat(res)


@pytest.mark.parametrize("P", [1, 3, 4])
@pytest.mark.parametrize("shape,kind", [((10, 9, 8), "smooth"), ((9, 2, 7), "noisy"), ((7, 5, 6), "sparse"),
                                        ((20, 24), "smooth"), ((8, 3), "step")], ids=str)
def test_thread_processes_reproduce_the_oracle(P, shape, kind):
    q = _field(shape, kind)
    for strategy in sharded.STRATEGIES:
        got = run_threads(CpuStages, torch.from_numpy(q), shape, 0.02, P, strategy).numpy()
        np.testing.assert_array_equal(got, _expected(q, 0.02, strategy, P), err_msg=strategy)


def test_plan_covers_every_plane_and_band():
    for dims, P in [((10, 9, 8), 3), ((9, 2, 7), 3), ((5, 4), 5)]:
        plans = [sharded._Plan(dims, P, r) for r in range(P)]
        assert sum(p.own(p.r) for p in plans) == dims[0]
        assert sum(plans[0].band_width(k) for k in range(P)) == dims[1]
        for p in plans:
            assert p.lo[p.r] == (1 if p.slabs[p.r][0] > 0 else 0)
            assert p.hi[p.r] == (1 if p.slabs[p.r][1] < dims[0] else 0)


@pytest.mark.parametrize("dims,P,msg", [((10,), 1, "rank-2 or rank-3"), ((1, 9, 8), 1, "extent"),
                                        ((3, 9, 8), 4, "planes")])
def test_bad_layouts_are_rejected(dims, P, msg):
    hub = sharded.LoopbackHub(1)
    q = torch.zeros(dims, dtype=torch.int32)
    comm = hub.comm(0)
    comm.size = P
    with pytest.raises(ValueError, match=msg):
        sharded.run_rank(CpuStages(), comm, q, dims, 0.1, "exact")
