"""Pins of the oracle's sharded strategies (Section VII-B), no GPU.

``oracle.mitigate_approx`` is checked against an independent restatement
built from the numpy helpers of ``oracle_checks`` (Algorithm 2 by slicing,
the EDT by exhaustive search, Algorithm 3, step E by its case split), against
Algorithm 4 itself where the strategy reduces to it (one slab), and against
the invariants the strategy implies: each slab sees a subset of the sites, so
Dist1 can only grow, and it stays the whole-field value wherever the nearest
boundary lies in the point's own slab.
"""
import zlib

import numpy as np
import pytest

import oracle
from tests import oracle_checks as oc

INF32 = oc.INF32


def restated_approx(q, eb, nparts, eta=0.9, idw_power=1.0):
    """The approximate strategy from its description: whole-field B1 and S_B
    (ghost planes make the stencil exact), EDTs inside each slab, GetBoundary
    on the whole field's S (ghost planes of S)."""
    b1, sb = oc.boundary_and_sign(q)
    n0 = q.shape[0]
    dist1 = np.empty(q.shape, np.int32)
    idx1 = np.empty(q.shape, np.int64)
    plane = int(np.prod(q.shape[1:]))
    for b, e in oracle.slab_bounds(n0, nparts):
        d, i = oc.brute_edt(b1[b:e])
        dist1[b:e] = d
        idx1[b:e] = np.where(i >= 0, i.astype(np.int64) + b * plane, -1)
    s, b2 = oc.propagate_and_b2(q, b1, sb, idx1)
    dist2 = np.empty(q.shape, np.int32)
    for b, e in oracle.slab_bounds(n0, nparts):
        dist2[b:e] = oc.brute_edt(b2[b:e])[0]
    out, _ = oc.compensate(q, dist1, dist2, s, eb, eta, idw_power)
    return dict(out=out, dist1=dist1, idx1=idx1.astype(np.int32), s=s, b2=b2, dist2=dist2)


CASES = [((9, 8, 7), "smooth"), ((9, 8, 7), "sparse"), ((12, 15), "smooth"), ((12, 15), "noisy"),
         ((11, 6, 5), "step"), ((16, 9), "sparse"), ((6, 10, 9), "checker")]


@pytest.mark.parametrize("shape,kind", CASES, ids=str)
@pytest.mark.parametrize("nparts", [1, 2, 3, 5])
def test_approx_matches_restatement(shape, kind, nparts):
    rng = np.random.default_rng(zlib.crc32(repr((shape, kind, nparts)).encode()))
    q = oc.random_index_field(rng, shape, kind)
    eb = 0.01
    ref = restated_approx(q, eb, nparts)
    got = oracle.mitigate_approx(q, eb, nparts)
    for k in ("dist1", "idx1", "s", "b2", "dist2"):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    np.testing.assert_allclose(got["out"], ref["out"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("shape,kind", CASES, ids=str)
def test_one_slab_is_algorithm_4(shape, kind):
    rng = np.random.default_rng(zlib.crc32(repr((shape, kind)).encode()))
    q = oc.random_index_field(rng, shape, kind)
    a, m = oracle.mitigate_approx(q, 0.02, 1), oracle.mitigate(q, 0.02)
    for k in ("out", "dist1", "idx1", "s", "b2", "dist2"):
        np.testing.assert_array_equal(a[k], m[k], err_msg=k)


@pytest.mark.parametrize("nparts", [2, 3, 4])
def test_local_sites_only_raise_dist1(nparts):
    rng = np.random.default_rng(100 + nparts)
    q = oc.random_index_field(rng, (12, 11, 10), "sparse")
    a, m = oracle.mitigate_approx(q, 0.01, nparts), oracle.mitigate(q, 0.01)
    assert np.all(a["dist1"] >= m["dist1"])
    # where the whole-field nearest boundary lies in the point's own slab,
    # the slab finds it (and the same one among equals: the smallest index)
    slab_of = np.empty(12, int)
    for k, (b, e) in enumerate(oracle.slab_bounds(12, nparts)):
        slab_of[b:e] = k
    z = np.indices(q.shape)[0]
    plane = 11 * 10
    inside = (m["idx1"] >= 0) & (slab_of[np.clip(m["idx1"], 0, None) // plane] == slab_of[z])
    assert inside.any() and (~inside).any()
    for k in ("dist1", "idx1", "s"):
        np.testing.assert_array_equal(a[k][inside], m[k][inside], err_msg=k)


def test_slab_without_boundary_keeps_dequantized_values():
    """q = 1 on rows 0-1, 0 below: B1 is rows 1 (S_B = -1) and 2 (S_B = +1),
    both in the first slab. The whole-field method propagates S = +1 down to
    every row below and, with no B2 (the S change sits on a q change), adds
    C = eta eps there; the approximate strategy's second slab sees no B1
    point, so S = 0 and D'' = D' = 0 on it, and the slab interface turns into
    a sign-flipping boundary."""
    q = np.zeros((8, 10), np.int32)
    q[:2] = 1
    eb, eta = 0.1, 0.9
    a, m = oracle.mitigate_approx(q, eb, 2), oracle.mitigate(q, eb)
    assert np.all(a["dist1"][4:] == INF32) and np.all(a["s"][4:] == 0)
    np.testing.assert_array_equal(a["out"][4:], np.zeros((4, 10)))
    np.testing.assert_allclose(m["out"][4:], eta * eb, rtol=0, atol=1e-15)
    # and the S change at the slab interface (same q, S +1 above, 0 below)
    # becomes a B2 line that the whole field does not have
    assert not m["b2"].any()
    assert np.all(a["b2"][3, 1:-1] == 1) and np.all(a["b2"][4, 1:-1] == 1)
    assert np.all(a["dist2"][3] <= 1) and np.all(m["dist2"] == INF32)


def test_independent_strategy_runs_algorithm_4_per_slab():
    rng = np.random.default_rng(7)
    q = oc.random_index_field(rng, (10, 9, 8), "smooth")
    out = oracle.mitigate_independent(q, 0.01, 3)
    for b, e in oracle.slab_bounds(10, 3):
        np.testing.assert_array_equal(out[b:e], oracle.mitigate(q[b:e], 0.01)["out"])


def test_slab_bounds_partition():
    for n0, p in [(10, 3), (7, 7), (512, 8), (5, 1)]:
        bs = oracle.slab_bounds(n0, p)
        assert bs[0][0] == 0 and bs[-1][1] == n0
        assert all(bs[k][1] == bs[k + 1][0] for k in range(p - 1))
        sizes = [e - b for b, e in bs]
        assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1


def test_new_entry_points_match_definitions():
    rng = np.random.default_rng(3)
    q = oc.random_index_field(rng, (7, 8, 9), "smooth")
    m = oracle.mitigate(q, 0.05)
    # GetBoundary(S) restated against the oracle's, for the oracle's own S
    _, b2 = oc.propagate_and_b2(q, m["b1"], m["sb"], m["idx1"])
    np.testing.assert_array_equal(oracle.boundary_of_s(q, m["s"]), b2)
    out, _ = oc.compensate(q, m["dist1"], m["dist2"], m["s"], 0.05)
    np.testing.assert_allclose(oracle.compensate(q, m["dist1"], m["dist2"], m["s"], 0.05), out, atol=1e-12, rtol=0)
    np.testing.assert_array_equal(oracle.compensate(q, m["dist1"], m["dist2"], m["s"], 0.05), m["out"])
