"""qai_mitigate_host: the method end to end from host memory (needs a GB300).

For 3-D fields with rows of 16-byte multiples and page-locked, device-mapped
host buffers the call pipelines: q goes to the device in z-slabs, step A runs
on each slab as it lands, each slab of D'' goes back while later slabs
arrive, and the outputs that later kernels change (the queries of the second
EDT, or everything after a fallback pass) are written into the host buffer
by a last kernel. Every case must give the device entry point's bits.
"""
import numpy as np
import pytest
import torch

from paper_2602_20097_gb300 import qai, synth

pytestmark = pytest.mark.gpu


def _both(q, eb, pinned_out=True):
    dev = qai.mitigate(q, eb)
    qh = q.cpu().pin_memory()
    out = torch.full(tuple(q.shape), float("nan"), dtype=torch.float32)
    if pinned_out:
        out = out.pin_memory()
    host = qai.mitigate_host(qh, eb, out_host=out)
    torch.cuda.synchronize()
    return dev.cpu(), host


@pytest.mark.parametrize("shape,rel_eb", [((96, 128, 160), 1e-3), ((96, 128, 160), 1e-2), ((64, 72, 80), 3e-3),
                                          ((17, 33, 68), 1e-2)], ids=str)
def test_pipelined_host_call_matches_the_device_call(shape, rel_eb):
    x = synth.grf(shape, slope=11.0 / 3.0, seed=51, device="cuda")
    eb = rel_eb * synth.value_range(x)
    q = synth.quantize(x, eb)
    dev, host = _both(q, eb)
    assert torch.equal(dev, host)


def test_host_call_after_the_separable_first_edt():
    """A step across x: the points at x = 0 are four cells from B1, beyond
    the bounded search, so the separable first EDT rewrites the outputs after
    step A's slabs went back (the last kernel copies every output)."""
    qn = np.zeros((24, 20, 12), np.int32)
    qn[:, :, 5:] = 1
    dev, host = _both(torch.from_numpy(qn).cuda(), 0.05)
    assert torch.equal(dev, host)


def test_host_call_with_indices_outside_the_fast_range():
    """|q| near 2^30: the exact step A redoes the fast one after its slabs
    went back."""
    rng = np.random.default_rng(5)
    qn = (rng.integers(-3, 4, size=(32, 40, 48)) + (1 << 30)).astype(np.int32)
    dev, host = _both(torch.from_numpy(qn).cuda(), 0.01)
    assert torch.equal(dev, host)


def test_host_call_into_pageable_memory_takes_the_plain_copies():
    x = synth.grf((48, 64, 80), slope=3.0, seed=52, device="cuda")
    eb = 2e-3 * synth.value_range(x)
    q = synth.quantize(x, eb)
    dev, host = _both(q, eb, pinned_out=False)
    assert torch.equal(dev, host)


def test_host_calls_back_to_back_on_one_workspace():
    x = synth.grf((64, 96, 128), slope=11.0 / 3.0, seed=53, device="cuda")
    ws = qai.alloc_workspace(qai.workspace_size_host((64, 96, 128)))
    outs = []
    for rel in (1e-3, 1e-2, 1e-3):
        eb = rel * synth.value_range(x)
        q = synth.quantize(x, eb)
        qh = q.cpu().pin_memory()
        oh = torch.empty(tuple(q.shape), dtype=torch.float32).pin_memory()
        qai.mitigate_host(qh, eb, out_host=oh, workspace=ws)
        outs.append((oh, qh, qai.mitigate(q, eb)))   # qh stays alive until the copies ran
    torch.cuda.synchronize()
    for oh, _, dev in outs:
        assert torch.equal(oh, dev.cpu())
