"""The signed-point route of the second EDT, through the C ABI (needs a GB300).

A plain qai_mitigate call (no per-step outputs) computes Dist2 only where step
E uses it -- points with S != 0 off B1 (Sec. VI-E: elsewhere C = 0 or the
weight is 1) -- by an exact shell search, then a search over every B2 site for
the points the shell search leaves, and hands the field to the dense second
EDT only when a list overflows. A debug call runs the dense second EDT
everywhere (its maps are checked bit for bit against the FP64 oracle in
test_gpu_parity.py). Every route must give the debug call's bits, and D''
within the parity tolerance of the oracle.
"""
import zlib

import numpy as np
import pytest
import torch

import oracle
from paper_2602_20097_gb300 import qai, synth
from tests import oracle_checks as oc

pytestmark = pytest.mark.gpu

ROUTES = ["auto", "brute", "dense", "off"]


def _plain_and_debug(q, eb, route, first_edt="local", **kw):
    ws = qai.alloc_workspace(qai.workspace_size(tuple(q.shape)))
    plain = qai.mitigate(q, eb, workspace=ws, route=route, first_edt=first_edt, **kw)
    counts = qai.route_counts(ws, tuple(q.shape)) if route != "off" and _rank(q) >= 2 else None
    full, maps = qai.mitigate(q, eb, debug=True, **kw)
    torch.cuda.synchronize()
    return plain, full, maps, counts


def _rank(q):
    return sum(1 for n in q.shape if n > 1)


def _field(name, shape, seed):
    if name == "grf":
        return synth.grf(shape, slope=11.0 / 3.0, seed=seed, device="cuda")
    return synth.grf_front(shape, seed=seed, device="cuda")


@pytest.mark.parametrize("first_edt", ["local", "separable"])
@pytest.mark.parametrize("route", ROUTES)
@pytest.mark.parametrize("name,shape,rel_eb", [("grf", (96, 128, 160), 1e-3), ("grf", (96, 128, 160), 1e-2),
                                               ("front", (64, 200, 72), 1e-3), ("front", (300, 500), 1e-3),
                                               ("grf", (700, 900), 1e-2), ("front", (40, 1, 64), 3e-3)],
                         ids=str)
def test_routes_match_the_dense_evaluation(route, first_edt, name, shape, rel_eb):
    x = _field(name, tuple(n for n in shape if n > 1), 31).reshape(shape)
    eb = rel_eb * synth.value_range(x)
    q = synth.quantize(x, eb).contiguous()
    plain, full, maps, counts = _plain_and_debug(q, eb, route, first_edt)
    assert torch.equal(plain, full), f"{route}: {(plain != full).sum().item()} points differ"
    plain_c, full_c, _, _ = _plain_and_debug(q, eb, route, first_edt, output_c=True)
    assert torch.equal(plain_c, full_c)
    if counts is not None and first_edt == "separable":
        assert not counts["separable_first_edt"]
    if counts is not None:
        want = int(((maps["s"] != 0) & (maps["dist1"] > 0)).sum().item())
        if route == "dense":
            assert counts["dense"]
        elif not counts["dense"]:
            assert counts["queries"] == want
            if route == "brute":
                assert counts["list_searched"] == want


@pytest.mark.parametrize("rel_eb", [1e-3, 1e-2])
def test_near_items_from_the_counter_match_the_dense_evaluation(rel_eb):
    """640 x 256 x 64: 40 960 items of four rows for the bounded nearest-site
    search, more than eight per warp of a resident grid on a 152-SM GB300, so
    the warps take their items from the route counter in the strided order
    (the fixed split runs below that). The plain call must give the bits of
    the debug call's dense evaluation."""
    shape = (640, 256, 64)
    x = synth.grf(shape, slope=11.0 / 3.0, seed=77, device="cuda")
    eb = rel_eb * synth.value_range(x)
    q = synth.quantize(x, eb).contiguous()
    plain, full, maps, counts = _plain_and_debug(q, eb, "auto")
    assert torch.equal(plain, full), f"{(plain != full).sum().item()} points differ"
    if rel_eb == 1e-3:
        assert not counts["separable_first_edt"]  # the search's own output stands
    if not counts["dense"]:
        assert counts["queries"] == int(((maps["s"] != 0) & (maps["dist1"] > 0)).sum().item())


@pytest.mark.parametrize("route", ["auto", "brute"])
@pytest.mark.parametrize("shape", [(17, 33), (64, 100), (180, 360), (3, 4, 5), (7, 9, 33), (16, 16, 16),
                                   (33, 17, 65), (20, 70, 31), (9, 130, 47)], ids=str)
@pytest.mark.parametrize("kind", ["smooth", "noisy", "sparse", "checker", "step", "extreme"])
def test_routes_on_index_fields_match_the_oracle(route, shape, kind):
    rng = np.random.default_rng(zlib.crc32(repr((shape, kind, "route")).encode()))
    qn = oc.random_index_field(rng, shape, kind)
    q = torch.from_numpy(qn).cuda()
    plain, full, _, _ = _plain_and_debug(q, 0.01, route)
    assert torch.equal(plain, full)
    ref = oracle.mitigate(qn, 0.01)["out"]
    rng_q = 2.0 * 0.01 * max(1, int(qn.max()) - int(qn.min()))
    tol = 1e-6 * rng_q + 4.0 * np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(plain.cpu().numpy().astype(np.float64) - ref) <= tol)


@pytest.mark.parametrize("kw", [dict(sign_rule=1), dict(b2_rule=1), dict(grad_threshold=3),
                                dict(idw_power=2.0), dict(eta=0.0), dict(idw_power=0.7, b2_rule=1)], ids=str)
@pytest.mark.parametrize("route", ["auto", "brute", "dense"])
def test_routes_under_rule_variants(kw, route):
    x = synth.grf((48, 64, 80), slope=3.0, seed=41, device="cuda")
    eb = 3e-3 * synth.value_range(x)
    q = synth.quantize(x, eb)
    plain, full, _, _ = _plain_and_debug(q, eb, route, **kw)
    assert torch.equal(plain, full)


@pytest.mark.parametrize("shape", [(5, 7), (17, 33), (3, 4, 5), (2, 2, 2), (7, 9, 33), (33, 17, 65), (4, 4, 4096),
                                   (2, 3, 16383), (4096, 2, 3), (37, 1025)], ids=str)
@pytest.mark.parametrize("kind", ["noisy", "extreme", "checker"])
def test_local_first_edt_on_index_fields(shape, kind):
    """Dense B1 (noise, |q| near 2^31, a checkerboard): the bounded search
    decides every point; edges, odd extents and the 64-bit stencil path."""
    rng = np.random.default_rng(zlib.crc32(repr((shape, kind, "local")).encode()))
    qn = oc.random_index_field(rng, shape, kind)
    q = torch.from_numpy(qn).cuda()
    plain, full, _, counts = _plain_and_debug(q, 0.01, "auto")
    assert torch.equal(plain, full)
    ref = oracle.mitigate(qn, 0.01)["out"]
    rng_q = 2.0 * 0.01 * max(1, int(qn.max()) - int(qn.min()))
    tol = 1e-6 * rng_q + 4.0 * np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(plain.cpu().numpy().astype(np.float64) - ref) <= tol)


def test_step_field_without_b2_takes_the_list_search_with_no_sites():
    """One quantization step across x: every point off the two boundary planes
    is a query, and B2 is empty (each q region has a single sign), so Dist2 is
    INF and the weight 1 (the limit of Sec. VI-E's weights)."""
    qn = np.zeros((8, 9, 10), np.int32)
    qn[:, :, 5:] = 1
    q = torch.from_numpy(qn).cuda()
    plain, full, maps, counts = _plain_and_debug(q, 0.05, "auto")
    assert torch.equal(plain, full)
    assert counts["separable_first_edt"]          # x = 0 is 4 cells from B1: beyond the bounded search
    assert not counts["dense"] and counts["b2_sites"] == 0
    assert counts["queries"] == counts["list_searched"] > 0
    assert int((maps["b2"] != 0).sum().item()) == 0
    ref = oracle.mitigate(qn, 0.05)["out"]
    np.testing.assert_allclose(plain.cpu().numpy(), ref, atol=1e-7)


def test_many_queries_hand_the_field_to_the_dense_second_edt():
    """A smooth ramp: large regions of one sign, queries far above the list
    capacity (N / 32 + 1024 for a 3-D field) -- the dense second EDT must
    take over."""
    zz, yy, xx = np.meshgrid(np.arange(40), np.arange(64), np.arange(96), indexing="ij")
    qn = ((xx + 0.5 * yy + 0.25 * zz) // 9).astype(np.int32)
    q = torch.from_numpy(qn).cuda()
    plain, full, maps, counts = _plain_and_debug(q, 0.01, "auto")
    assert torch.equal(plain, full)
    assert counts["dense"]
    assert int(((maps["s"] != 0) & (maps["dist1"] > 0)).sum().item()) > qn.size // 32 + 1024


@pytest.mark.parametrize("shape,patch", [((600, 700), (slice(100, 160), slice(200, 260))),
                                         ((40, 240, 260), (slice(5, 35), slice(100, 110), slice(40, 80)))],
                         ids=["2d", "3d"])
def test_a_dense_cluster_of_queries_spills_past_the_tile_buffer(shape, patch):
    """Random indices (every boundary fast-varying, so S = 0) around a gentle
    ramp patch (signs kept): thousands of queries in a few tiles of the last
    EDT1 pass, more than one tile buffers, far fewer than the list holds."""
    rng = np.random.default_rng(7)
    qn = rng.integers(0, 1000, size=shape).astype(np.int32)
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    ramp = (grids[-1] // 7 + grids[-2] // 11).astype(np.int32)
    qn[patch] = ramp[patch]
    q = torch.from_numpy(qn).cuda()
    plain, full, maps, counts = _plain_and_debug(q, 0.01, "auto")
    assert torch.equal(plain, full)
    want = int(((maps["s"] != 0) & (maps["dist1"] > 0)).sum().item())
    assert not counts["dense"] and counts["queries"] >= want > 1000


def test_grf_512_eb_1e3_stays_on_the_signed_route():
    """The 512^3 k^-11/3 field at eb = 1e-3 x range: few queries, most of them
    far from B2 (the list search finds them); no dense second EDT."""
    x = synth.grf((512, 512, 512), slope=11.0 / 3.0, seed=2, device="cuda")
    eb = 1e-3 * synth.value_range(x)
    q = synth.quantize(x, eb)
    del x
    ws = qai.alloc_workspace(qai.workspace_size(tuple(q.shape)))
    plain = qai.mitigate(q, eb, workspace=ws)
    counts = qai.route_counts(ws, tuple(q.shape))
    assert not counts["dense"] and counts["queries"] > 0 and not counts["separable_first_edt"]
    dense = qai.mitigate(q, eb, workspace=ws, route="off")
    torch.cuda.synchronize()
    assert torch.equal(plain, dense)
