"""Adjoint of step E on the GPU (dL/dD', dL/deta, dL/dp with the EDT
assignment fixed) vs the FP64 oracle gradient, whose own pin is finite
differences of the FP64 forward (test_oracle_adjoint.py)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_20097_gb300 import qai, synth

pytestmark = pytest.mark.gpu


def _case(name, shape, seed, rel):
    if name == "sinusoids":
        x = torch.from_numpy(synth.sinusoids(shape, seed=seed)).cuda()
    elif name == "grf":
        x = synth.grf(shape, slope=11.0 / 3.0, seed=seed, device="cuda")
    else:
        x = synth.grf_front(shape, seed=seed, device="cuda")
    eb = rel * synth.value_range(x)
    return x, synth.quantize(x, eb), eb


def _grad_out(x, q, eb, eta, p):
    out = qai.mitigate(q, eb, eta=eta, idw_power=p)
    return (out.double() - x.double()).float()


CASES = [("sinusoids", (64, 64, 64), 1, 1e-2, 0.9, 1.0), ("sinusoids", (40, 50, 60), 2, 3e-2, 0.7, 1.7),
         ("front", (96, 128), 3, 1e-2, 0.9, 0.6), ("grf", (48, 56, 64), 4, 1e-2, 1.1, 2.0),
         ("front", (30, 70, 90), 5, 5e-3, 0.9, 1.0)]


@pytest.mark.parametrize("name,shape,seed,rel,eta,p", CASES, ids=lambda v: str(v))
@pytest.mark.parametrize("stored", [True, False], ids=["stored", "recompute"])
def test_gradient_matches_fp64_oracle(name, shape, seed, rel, eta, p, stored):
    x, q, eb = _case(name, shape, seed, rel)
    g = _grad_out(x, q, eb, eta, p)
    saved = qai.mitigate_save(q, eb, eta=eta, idw_power=p)[1] if stored else None
    gd, gp = qai.mitigate_backward(q, eb, g, saved=saved, eta=eta, idw_power=p)
    torch.cuda.synchronize()
    assert torch.equal(gd, g)
    ref = oracle.grad_params(q.cpu().numpy(), eb, g.cpu().numpy().astype(np.float64), eta=eta, idw_power=p)
    got = gp.cpu().numpy()
    scale = float(torch.sum(torch.abs(g.double()))) * eb   # magnitude of the summed terms
    for k in range(2):
        assert abs(got[k] - ref[k]) <= 1e-5 * abs(ref[k]) + 1e-7 * scale, (k, got[k], ref[k])


@pytest.mark.parametrize("shape", [(64, 80, 96), (200, 300), (3000,)], ids=str)
def test_modes_agree_and_each_is_deterministic(shape):
    x, q, eb = _case("grf" if len(shape) > 1 else "sinusoids", shape, 6, 1e-2)
    g = _grad_out(x, q, eb, 0.9, 1.0)
    saved = qai.mitigate_save(q, eb)[1]
    a = [qai.mitigate_backward(q, eb, g, saved=saved, want_grad_dprime=False)[1] for _ in range(2)]
    b = [qai.mitigate_backward(q, eb, g, saved=None)[1] for _ in range(2)]
    torch.cuda.synchronize()
    assert torch.equal(a[0], a[1]) and torch.equal(b[0], b[1])
    scale = float(torch.sum(torch.abs(g.double()))) * eb
    # the modes group the fp32 partial sums differently: agreement to rounding
    assert torch.allclose(a[0], b[0], rtol=1e-6, atol=1e-8 * scale)


def test_crops_of_a_larger_field():
    x, _, _ = _case("grf", (128, 128, 128), 7, 1e-3)
    for (z, y, w) in [(0, 0, 0), (40, 70, 96), (96, 96, 96)]:
        xc = x[z:z + 32, y:y + 32, w:w + 32].contiguous()
        eb = 1e-2 * synth.value_range(xc)
        qc = synth.quantize(xc, eb)
        g = _grad_out(xc, qc, eb, 0.9, 1.0)
        _, gp = qai.mitigate_backward(qc, eb, g, want_grad_dprime=False)
        ref = oracle.grad_params(qc.cpu().numpy(), eb, g.cpu().numpy().astype(np.float64))
        scale = float(torch.sum(torch.abs(g.double()))) * eb
        got = gp.cpu().numpy()
        for k in range(2):
            assert abs(got[k] - ref[k]) <= 1e-5 * abs(ref[k]) + 1e-7 * scale


def test_output_c_is_the_compensation():
    x, q, eb = _case("sinusoids", (32, 40, 48), 8, 2e-2)
    full = qai.mitigate(q, eb)
    comp = qai.mitigate(q, eb, output_c=True)
    dprime = (q.double() * 2 * eb).float()
    torch.cuda.synchronize()
    assert float(torch.max(torch.abs(dprime + comp - full))) <= 2e-7 * float(torch.max(torch.abs(full))) + 1e-9
    assert float(torch.max(torch.abs(comp))) <= 0.9 * eb * (1 + 1e-6)
    # the library's D' is float(q) * float(2 eps), and D' + C from the library
    # is that D' plus the compensation, one fp32 add
    dq = qai.dequantize(q, eb)
    assert torch.equal(dq, q.float() * torch.tensor(2 * eb, dtype=torch.float32, device="cuda"))
    added = qai.mitigate_add(q, dq, eb)
    assert torch.equal(added, dq + comp)
    assert float(torch.max(torch.abs(added - full))) <= 2e-7 * float(torch.max(torch.abs(full))) + 1e-9


def test_autograd_function_and_tuning():
    x, q, eb = _case("sinusoids", (48, 48, 48), 9, 2e-2)
    dprime = (q.double() * 2 * eb).float()
    for stored in (True, False):
        e = torch.tensor(0.8, dtype=torch.float64, device="cuda", requires_grad=True)
        p = torch.tensor(1.2, dtype=torch.float64, device="cuda", requires_grad=True)
        dp = dprime.clone().requires_grad_(True)
        out = qai.QAIFunction.apply(dp, e, p, q, eb, stored)
        loss = 0.5 * torch.sum((out.double() - x.double()) ** 2)
        loss.backward()
        g = (out.detach().double() - x.double()).float()
        _, ref = qai.mitigate_backward(q, eb, g, eta=0.8, idw_power=1.2)
        assert torch.allclose(dp.grad, g)
        assert torch.allclose(torch.stack([e.grad, p.grad]), ref, rtol=1e-6)
    hist = qai.tune(q, eb, x, eta=0.5, p=1.0, steps=8, lr=0.02)
    assert hist[-1][2] < hist[0][2]
