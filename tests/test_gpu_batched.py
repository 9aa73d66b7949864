"""The batched form (persistent grouped launches over all fields, in one
cached CUDA graph; per-field sequences on forked streams inside a caller's
capture) against single qai_mitigate calls (bit-identical: the same kernel
bodies on the same data) and against the FP64 oracle on a subset."""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_20097_gb300 import qai, synth

pytestmark = pytest.mark.gpu

SHAPES = [(5000,), (257,), (64, 100), (37, 1025), (180, 361), (500, 500),
          (16, 16, 16), (9, 130, 47), (33, 17, 65), (40, 64, 96), (7, 9, 33), (64, 64, 64)]


def _fields(shapes, seed0=100):
    qs, ebs, xs = [], [], []
    for i, shp in enumerate(shapes):
        x = synth.grf_front(shp, seed=seed0 + i, device="cuda") if len(shp) > 1 else \
            torch.from_numpy(synth.sinusoids(shp, seed=seed0 + i)).cuda()
        eb = (10 ** (-3 + (i % 3) * 0.5)) * synth.value_range(x)
        qs.append(synth.quantize(x, eb))
        ebs.append(eb)
        xs.append(x)
    return qs, ebs, xs


@pytest.mark.parametrize("kw", [{}, {"sign_rule": 1, "b2_rule": 1}, {"eta": 0.6, "idw_power": 1.5}], ids=str)
def test_batched_equals_single_calls(kw):
    qs, ebs, _ = _fields(SHAPES)
    batch = qai.Batch(qs, ebs)
    outs = qai.mitigate_batched(batch, **kw)
    torch.cuda.synchronize()
    first = [o.clone() for o in outs]
    qai.mitigate_batched(batch, **kw)            # replay of the cached graph
    torch.cuda.synchronize()
    for q, eb, o, f in zip(qs, ebs, outs, first):
        ref = qai.mitigate(q, eb, **kw)
        torch.cuda.synchronize()
        assert torch.equal(o, ref), q.shape
        assert torch.equal(f, ref), q.shape


def test_batched_matches_oracle_and_autotune_keeps_results():
    qs, ebs, xs = _fields(SHAPES, seed0=300)
    batch = qai.Batch(qs, ebs)
    choice = qai.autotune_batched(batch)
    assert set(choice) <= {1, 2, 3} and all(v["ms"] > 0 for v in choice.values())
    assert choice[1]["streams"] == 1 and not choice[1]["grouped"]
    for r in (2, 3):
        c = choice[r]
        assert c["grouped"] and c["launches"] >= 10 and c["points_per_block"] in (1 << k for k in range(14, 19))
        assert (c["tile_w"], c["rows_per_band"]) in {(0, 0), (8, 32), (16, 32), (32, 32), (8, 16), (16, 16),
                                                     (16, 64), (32, 64)}
    outs = qai.mitigate_batched(batch)
    torch.cuda.synchronize()
    for q, eb, x, o in zip(qs, ebs, xs, outs):
        ref = oracle.mitigate(q.cpu().numpy(), eb, debug=False)["out"]
        rng = synth.value_range(x)
        assert np.max(np.abs(o.cpu().numpy().astype(np.float64) - ref)) <= 1e-6 * rng, q.shape


def test_ninety_six_uneven_fields():
    specs = synth.batch_specs()
    qs, ebs = [], []
    for sp in specs:
        x = synth.grf(sp["shape"], slope=sp["slope"], seed=sp["seed"], device="cuda")
        eb = sp["rel_eb"] * synth.value_range(x)
        qs.append(synth.quantize(x, eb))
        ebs.append(eb)
    batch = qai.Batch(qs, ebs)
    qai.autotune_batched(batch)
    outs = qai.mitigate_batched(batch)
    torch.cuda.synchronize()
    for i, (q, eb, o) in enumerate(zip(qs, ebs, outs)):
        ref = qai.mitigate(q, eb)
        torch.cuda.synchronize()
        assert torch.equal(o, ref), (i, q.shape)
    for i in (0, 1, 2, 3, 50, 95):           # a subset against the oracle
        ref = oracle.mitigate(qs[i].cpu().numpy(), ebs[i], debug=False)["out"]
        rng = 2 * ebs[i] * (int(qs[i].max()) - int(qs[i].min()) + 1)
        assert np.max(np.abs(outs[i].cpu().numpy().astype(np.float64) - ref)) <= 1e-6 * rng


def test_batched_inside_a_caller_graph():
    qs, ebs, _ = _fields([(64, 100), (16, 16, 16), (9, 130, 47)], seed0=500)
    batch = qai.Batch(qs, ebs)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        qai.mitigate_batched(batch)           # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    expect = [o.clone() for o in batch.outs]
    for o in batch.outs:
        o.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        qai.mitigate_batched(batch)
    g.replay()
    torch.cuda.synchronize()
    for o, e in zip(batch.outs, expect):
        assert torch.equal(o, e)


def test_batched_argument_errors():
    q = torch.zeros((8, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(qai.QAIError):
        qai.Batch([q], [0.1, 0.2])
    batch = qai.Batch([q], [0.1])
    batch.ebs[0] = -1.0
    with pytest.raises(qai.QAIError):
        qai.mitigate_batched(batch)


def test_more_fields_than_one_launch_holds():
    """70 fields of one shape share every kernel: the launches split at 64
    fields; the fronts at eb 1e-2 of the range take the fallbacks."""
    qs, ebs = [], []
    for i in range(70):
        x = synth.grf_front((40, 96), seed=700 + i, device="cuda")
        eb = (1e-2 if i % 2 else 1e-3) * synth.value_range(x)
        qs.append(synth.quantize(x, eb))
        ebs.append(eb)
    batch = qai.Batch(qs, ebs)
    outs = qai.mitigate_batched(batch)
    torch.cuda.synchronize()
    for i, (q, eb, o) in enumerate(zip(qs, ebs, outs)):
        assert torch.equal(o, qai.mitigate(q, eb)), i
