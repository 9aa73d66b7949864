"""Pins of the oracle's adjoint of step E (dL/deta, dL/dp with the EDT
assignment fixed) against central finite differences of the FP64 forward."""
import numpy as np
import pytest

import oracle
from paper_2602_20097_gb300 import synth


def _loss(q, eb, x, eta, p):
    r = oracle.mitigate(q, eb, eta=eta, idw_power=p, debug=False)["out"]
    return 0.5 * float(np.sum((r - x) ** 2))


@pytest.mark.parametrize("field,shape,rel,eta,p", [
    ("sinusoids", (12, 14, 16), 0.02, 0.9, 1.0),
    ("sinusoids", (10, 11, 13), 0.05, 0.7, 1.6),
    ("front", (40, 50), 0.01, 0.9, 0.6),
    ("front", (7, 19, 23), 0.03, 1.1, 2.0),
])
def test_adjoint_matches_central_differences(field, shape, rel, eta, p):
    x = synth.sinusoids(shape, seed=7) if field == "sinusoids" else synth.grf_front(shape, seed=8).numpy()
    x = x.astype(np.float64)
    eb = rel * synth.value_range(x)
    q = synth.quantize(x, eb)
    r = oracle.mitigate(q, eb, eta=eta, idw_power=p, debug=False)["out"]
    ge, gp = oracle.grad_params(q, eb, r - x, eta=eta, idw_power=p)
    h = 1e-3
    fe = (_loss(q, eb, x, eta + h, p) - _loss(q, eb, x, eta - h, p)) / (2 * h)
    h = 1e-4
    fp = (_loss(q, eb, x, eta, p + h) - _loss(q, eb, x, eta, p - h)) / (2 * h)
    assert ge == pytest.approx(fe, rel=1e-7, abs=1e-12)
    assert gp == pytest.approx(fp, rel=1e-5, abs=1e-10)


def test_eta_gradient_is_linear_in_grad_out():
    x = synth.sinusoids((9, 10, 11), seed=9)
    eb = 0.02 * synth.value_range(x)
    q = synth.quantize(x, eb)
    rng = np.random.default_rng(1)
    g1, g2 = rng.normal(size=q.shape), rng.normal(size=q.shape)
    a = np.array(oracle.grad_params(q, eb, g1))
    b = np.array(oracle.grad_params(q, eb, g2))
    c = np.array(oracle.grad_params(q, eb, 2.0 * g1 - 3.0 * g2))
    np.testing.assert_allclose(c, 2.0 * a - 3.0 * b, rtol=1e-10, atol=1e-12)


def test_fields_without_signs_have_zero_parameter_gradients():
    # constant field: no boundary at all; a steep ramp (3 indices per cell):
    # every interior point is a boundary whose sign the fast-varying rule
    # zeroes (|q[+1] - q[-1]| = 6); S = 0 everywhere
    g = np.random.default_rng(2).normal(size=(9, 10, 11))
    for q in (np.full((9, 10, 11), 7, np.int32), (3 * np.indices((9, 10, 11))[2]).astype(np.int32)):
        ge, gp = oracle.grad_params(q, 0.1, g)
        assert ge == 0.0 and gp == 0.0


def test_eta_gradient_of_the_hand_worked_ramp():
    # D'' - D' = S w eta eps, so with G = 1 everywhere dL/deta = sum (D'' - D') / eta,
    # taken from the hand-derived V1 values (tests/golden/V1_ramp.json)
    import json
    import os
    fx = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "V1_ramp.json")))
    q = np.array(fx["q"], np.int32)
    dprime = 2 * fx["eb"] * q
    want = float(np.sum(np.array(fx["expect"]["out"]) - dprime)) / fx["eta"]
    ge, gp = oracle.grad_params(q, fx["eb"], np.ones(q.shape), eta=fx["eta"])
    assert ge == pytest.approx(want, rel=1e-12, abs=1e-12)
