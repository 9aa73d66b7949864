"""Pins of the CPU oracle against things other than itself (no GPU needed).

* hand-worked vectors from the paper's definitions (tests/golden/*.json);
* Eq. 2 by brute force: squared EDT and nearest index (R5 tie rule);
* Algorithms 2 and 3 and step E re-stated independently in numpy;
* the error-bound invariant |x - D''| <= (1 + eta) eps (Sec. VIII-C, Table II);
* symmetries (q -> -q, q -> q + c), special cases (constant, checkerboard),
  and the squeeze of extent-1 axes (R1).
"""
import glob
import json
import os
import zlib

import numpy as np
import pytest

import oracle
from paper_2602_20097_gb300 import synth
from tests import oracle_checks as oc

GOLDEN = sorted(glob.glob(os.path.join(os.path.dirname(__file__), "golden", "V*.json")))


@pytest.mark.parametrize("path", GOLDEN, ids=[os.path.basename(p)[:-5] for p in GOLDEN])
def test_golden_vectors(path):
    fx = json.load(open(path))
    q = np.array(fx["q"], np.int32)
    p = fx["params"]
    r = oracle.mitigate(q, fx["eb"], eta=fx["eta"], grad_threshold=p["grad_threshold"],
                        sign_rule=p["sign_rule"], b2_rule=p["b2_rule"])
    for key, val in fx["expect"].items():
        exp = np.array(val)
        if key == "out":
            np.testing.assert_allclose(r["out"], exp, rtol=0, atol=1e-12, err_msg=key)
        else:
            np.testing.assert_array_equal(r[key], exp.astype(r[key].dtype), err_msg=key)
    if "original_x" in fx:
        x = np.array(fx["original_x"])
        assert np.array_equal(synth.quantize(x, fx["eb"]), q)
        assert np.max(np.abs(x - r["out"])) <= (1 + fx["eta"]) * fx["eb"] + 1e-12


EDT_SHAPES = [(1,), (2,), (7,), (40,), (1, 9), (5, 1), (3, 4), (9, 9), (6, 11),
              (2, 2, 2), (3, 5, 7), (7, 8, 9), (9, 4, 6), (1, 6, 5), (4, 1, 6)]


@pytest.mark.parametrize("shape", EDT_SHAPES, ids=str)
@pytest.mark.parametrize("density", [0.0, -1, 0.05, 0.3, 1.0])
def test_edt_matches_brute_force(shape, density):
    rng = np.random.default_rng(zlib.crc32(repr((shape, density)).encode()))
    for _ in range(3):
        if density == -1:                              # exactly one site
            m = np.zeros(shape, bool)
            m.flat[rng.integers(m.size)] = True
        else:
            m = rng.random(shape) < density
        d, i = oracle.edt(m)
        bd, bi = oc.brute_edt(m)
        np.testing.assert_array_equal(d, bd)
        np.testing.assert_array_equal(i, bi)


def test_edt_tie_rule_prefers_smallest_linear_index():
    # (1,1) is at distance 1 from (1,2) [index 7] and (2,1) [index 11]: R5 picks 7.
    m = np.zeros((5, 5), bool)
    m[1, 2] = m[2, 1] = True
    d, i = oracle.edt(m)
    assert d[1, 1] == 1 and i[1, 1] == 7
    assert d[2, 2] == 1 and i[2, 2] == 7


KINDS = ["smooth", "noisy", "sparse", "constant", "checker", "step", "extreme"]
STEP_SHAPES = [(13,), (1, 17), (6, 9), (12, 10), (5, 6, 7), (9, 8, 11), (3, 10, 4), (1, 5, 6)]


@pytest.mark.parametrize("shape", STEP_SHAPES, ids=str)
@pytest.mark.parametrize("kind", KINDS)
def test_steps_match_independent_restatement(shape, kind):
    rng = np.random.default_rng(zlib.crc32(repr((shape, kind)).encode()))
    q = oc.random_index_field(rng, shape, kind)
    for sign_rule in (0, 1):
        for thr in (2, 3):
            b1, sb = oracle.boundary_and_sign(q, grad_threshold=thr, sign_rule=sign_rule)
            eb1, esb = oc.boundary_and_sign(q, grad_threshold=thr, sign_rule=sign_rule)
            np.testing.assert_array_equal(b1, eb1)
            np.testing.assert_array_equal(sb, esb)
    for b2_rule in (0, 1):
        r = oracle.mitigate(q, 0.01, eta=0.9, b2_rule=b2_rule)
        d1, i1 = oc.brute_edt(r["b1"] == 1)
        np.testing.assert_array_equal(r["dist1"], d1)
        np.testing.assert_array_equal(r["idx1"], i1)
        s, b2 = oc.propagate_and_b2(q, r["b1"], r["sb"], r["idx1"], b2_rule=b2_rule)
        np.testing.assert_array_equal(r["s"], s)
        np.testing.assert_array_equal(r["b2"], b2)
        d2, _ = oc.brute_edt(r["b2"] == 1)
        np.testing.assert_array_equal(r["dist2"], d2)
        out, comp = oc.compensate(q, r["dist1"], r["dist2"], r["s"], 0.01, 0.9)
        np.testing.assert_allclose(r["comp"], comp, rtol=0, atol=1e-15)
        np.testing.assert_allclose(r["out"], out, rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("p", [0.5, 1.0, 2.0])
def test_idw_power_closed_form(p):
    rng = np.random.default_rng(5)
    q = oc.random_index_field(rng, (9, 10, 11), "smooth")
    r = oracle.mitigate(q, 0.02, eta=0.7, idw_power=p)
    out, comp = oc.compensate(q, r["dist1"], r["dist2"], r["s"], 0.02, 0.7, idw_power=p)
    np.testing.assert_allclose(r["comp"], comp, rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("field", ["sinusoids", "grf", "front2d"])
def test_error_bound_invariant(field):
    if field == "sinusoids":
        x = synth.sinusoids((24, 28, 20), seed=11)
    elif field == "grf":
        x = synth.grf((20, 24, 28), seed=12).numpy()
    else:
        x = synth.grf_front((60, 90), seed=13).numpy()
    for rel in (1e-3, 1e-2, 5e-2):
        eb = rel * synth.value_range(x)
        q = synth.quantize(x, eb)
        r = oracle.mitigate(q, eb, eta=0.9)
        dprime = 2.0 * q.astype(np.float64) * eb
        assert np.max(np.abs(x - dprime)) <= eb * (1 + 1e-12)
        assert np.max(np.abs(r["comp"])) <= 0.9 * eb * (1 + 1e-12)
        assert np.max(np.abs(x - r["out"])) <= 1.9 * eb * (1 + 1e-12)


def test_symmetries_and_special_cases():
    rng = np.random.default_rng(3)
    q = oc.random_index_field(rng, (8, 9, 10), "smooth")
    a = oracle.mitigate(q, 0.05)
    neg = oracle.mitigate(-q, 0.05)
    np.testing.assert_array_equal(neg["s"], -a["s"])
    np.testing.assert_allclose(neg["comp"], -a["comp"], atol=0)
    shifted = oracle.mitigate(q + 37, 0.05)
    np.testing.assert_allclose(shifted["comp"], a["comp"], atol=0)
    const = oracle.mitigate(np.full((6, 7, 8), -3, np.int32), 0.1)
    assert not const["b1"].any() and np.all(const["comp"] == 0)
    assert np.all(const["dist1"] == oc.INF32) and np.all(const["idx1"] == -1)
    # checkerboard: every interior point is a boundary, central differences are 0,
    # so signs survive: low cells pull up by eta*eps, high cells pull down.
    cb = oc.random_index_field(rng, (6, 7, 8), "checker")
    r = oracle.mitigate(cb, 0.1)
    inner = oc._interior_mask(cb.shape)
    assert np.all(r["b1"][inner] == 1) and not r["b2"].any()
    np.testing.assert_allclose(r["comp"][inner], np.where(cb[inner] == 0, 0.09, -0.09))


def test_squeeze_extent_one_axes():
    rng = np.random.default_rng(4)
    q2 = oc.random_index_field(rng, (11, 13), "smooth")
    ref = oracle.mitigate(q2, 0.03)
    for shp in [(1, 11, 13), (11, 1, 13), (11, 13, 1)]:
        r = oracle.mitigate(q2.reshape(shp), 0.03)
        for k in ("b1", "sb", "s", "b2", "dist1", "dist2", "idx1"):
            np.testing.assert_array_equal(r[k].reshape(q2.shape), ref[k], err_msg=str((shp, k)))
        np.testing.assert_array_equal(r["out"].reshape(q2.shape), ref["out"])
