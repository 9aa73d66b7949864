"""Sharded forms (Section VII-B) on the GPU through the C ABI (needs a GB300).

Emulated processes share one device: host threads over the in-process hub
(every kernel is launched on the one default stream, so none waits on
another), or two real processes over gloo with host copies. The exact form
must give the one-process call's bits; the approximate form must match the
oracle's approximate strategy within the parity tolerance (1e-6 of the value
range); the independent form must give per-slab calls' bits.
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
from paper_2602_20097_gb300 import qai, sharded, synth
from tests import oracle_checks as oc

pytestmark = pytest.mark.gpu


def _stages():
    return sharded.CudaStages(qai.default_params())


def run_threads(q, eb, P, strategy):
    dims = tuple(q.shape)
    hub = sharded.LoopbackHub(P, timeout=300)
    res, errs = [None] * P, []
    slabs = sharded.slab_bounds(dims[0], P)

    def work(r):
        try:
            b, e = slabs[r]
            res[r] = sharded.run_rank(_stages(), hub.comm(r), q[b:e].contiguous(), dims, eb, strategy)
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
    out = torch.cat(res)
    torch.cuda.synchronize()
    return out


def _tol(q, eb):
    return 1e-6 * 2.0 * eb * max(1, int(q.max()) - int(q.min()))


def _check(q, eb, P):
    qn = q.cpu().numpy()
    one = qai.mitigate(q, eb)
    ex = run_threads(q, eb, P, "exact")
    assert torch.equal(ex, one), "exact form differs from the one-process call"
    ref = oracle.mitigate(qn, eb, debug=False)["out"]
    assert np.max(np.abs(ex.cpu().numpy().astype(np.float64) - ref)) <= _tol(qn, eb)
    ap = run_threads(q, eb, P, "approximate").cpu().numpy().astype(np.float64)
    want = oracle.mitigate_approx(qn, eb, P)["out"]
    err = np.abs(ap - want)
    assert err.max() <= _tol(qn, eb), f"approximate form: {err.max():.3e} at {np.unravel_index(err.argmax(), err.shape)}"
    ind = run_threads(q, eb, P, "independent")
    for b, e in sharded.slab_bounds(q.shape[0], P):
        assert torch.equal(ind[b:e], qai.mitigate(q[b:e].contiguous(), eb))
    return int((want != ref).sum())


@pytest.mark.parametrize("P", [1, 2, 3, 4])
@pytest.mark.parametrize("shape,kind", [((10, 9, 8), "smooth"), ((9, 2, 7), "noisy"), ((33, 17, 65), "smooth"),
                                        ((20, 24), "sparse"), ((64, 100), "smooth"), ((8, 3), "step")], ids=str)
def test_small_fields(shape, kind, P):
    rng = np.random.default_rng(zlib.crc32(repr((shape, kind)).encode()))
    q = torch.from_numpy(oc.random_index_field(rng, shape, kind)).cuda()
    _check(q, 0.01, P)


@pytest.mark.parametrize("name,shape,rel_eb,P", [("grf", (96, 128, 160), 1e-2, 4), ("front", (64, 200, 72), 1e-2, 3),
                                                 ("front", (300, 500), 1e-2, 2), ("grf", (128, 128, 128), 1e-3, 8)],
                         ids=str)
def test_real_fields(name, shape, rel_eb, P):
    x = (synth.grf(shape, slope=11.0 / 3.0, seed=21, device="cuda") if name == "grf"
         else synth.grf_front(shape, seed=21, device="cuda"))
    eb = rel_eb * synth.value_range(x)
    q = synth.quantize(x, eb)
    differs = _check(q, eb, P)
    if name == "front":
        assert differs > 0   # sparse boundaries: the approximate strategy departs


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q, eb, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        comm = sharded.HostCopyComm()
        b, e = sharded.slab_bounds(q.shape[0], world)[rank]
        qd = torch.from_numpy(q[b:e].copy()).cuda()
        for strategy in ("exact", "approximate"):
            out = sharded.mitigate(qd, q.shape, eb, strategy=strategy, comm=comm)
            torch.cuda.synchronize()
            results[(rank, strategy)] = out.cpu().numpy()
    finally:
        dist.destroy_process_group()


def test_two_processes_over_gloo_with_host_copies():
    x = synth.grf_front((40, 120, 96), seed=5, device="cpu")
    eb = 1e-2 * synth.value_range(x)
    q = synth.quantize(x, eb).numpy()
    mgr = mp.get_context("spawn").Manager()
    results = mgr.dict()
    mp.spawn(_worker, args=(2, _free_port(), q, eb, results), nprocs=2, join=True)
    ex = np.concatenate([results[(r, "exact")] for r in range(2)]).astype(np.float64)
    ap = np.concatenate([results[(r, "approximate")] for r in range(2)]).astype(np.float64)
    assert np.max(np.abs(ex - oracle.mitigate(q, eb, debug=False)["out"])) <= _tol(q, eb)
    assert np.max(np.abs(ap - oracle.mitigate_approx(q, eb, 2)["out"])) <= _tol(q, eb)
