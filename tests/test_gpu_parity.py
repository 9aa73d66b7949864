"""CUDA path vs the FP64 oracle, through the C ABI (needs a GB300).

Bar: B1, S_B, Dist1, I1 (smallest index on ties), S, B2 and Dist2 bit-exact;
D'' within 1e-6 of the value range (fp32 kernels vs FP64 oracle: the fp32
rounding of q * 2 eps and of the weights is ~1e-7 of |D''| for fields in
[0, 1], so 1e-6 * range leaves an order of magnitude of margin); and the
relaxed error bound |x - D''| <= (1 + eta) eps on every point where the
original field is known.
"""
import zlib

import numpy as np
import pytest
import torch

import oracle
from paper_2602_20097_gb300 import qai, synth
from tests import oracle_checks as oc

pytestmark = pytest.mark.gpu

MAPS = ("b1", "sb", "dist1", "idx1", "s", "b2", "dist2")


def tolerance(q, eb, ref_out, x_range=None):
    """1e-6 of the value range. For the synthetic index fields (no original
    field, |q| up to 2^31) add 4 fp32 ulps of |D''|: no fp32 output is closer
    than half an ulp to the FP64 value, and the kernel rounds q, 2 eps, their
    product and the final add once each."""
    if x_range is not None:
        return 1e-6 * x_range
    rng = 2.0 * eb * max(1, int(q.max()) - int(q.min()))
    return 1e-6 * rng + 4.0 * np.spacing(np.abs(ref_out).astype(np.float32)).astype(np.float64)


def gpu_run(q, eb, **kw):
    qt = torch.from_numpy(np.ascontiguousarray(q)).cuda()
    out, maps = qai.mitigate(qt, eb, debug=True, **kw)
    torch.cuda.synchronize()
    return out.cpu().numpy(), {k: v.cpu().numpy() for k, v in maps.items()}


def assert_parity(q, eb, x_range=None, **kw):
    ref = oracle.mitigate(q, eb, **kw)
    out, maps = gpu_run(q, eb, **kw)
    for k in MAPS:
        bad = np.flatnonzero(maps[k].ravel() != ref[k].ravel())
        assert bad.size == 0, (f"{k}: {bad.size} mismatches, first at {bad[:5]}: "
                               f"gpu {maps[k].ravel()[bad[:5]]} oracle {ref[k].ravel()[bad[:5]]}")
    err = np.abs(out.astype(np.float64) - ref["out"])
    tol = tolerance(q, eb, ref["out"], x_range)
    worst = np.argmax(err - tol)
    assert np.all(err <= tol), (f"|D''_gpu - D''_oracle| = {err.ravel()[worst]:.3e} > "
                                f"{np.broadcast_to(tol, err.shape).ravel()[worst]:.3e} at {worst}")
    return ref, out


SHAPES = [(1,), (2,), (3,), (13,), (100,), (1000,), (5003,),
          (1, 17), (3, 3), (5, 7), (17, 33), (64, 100), (100, 64), (180, 360), (37, 1025),
          (2, 2, 2), (3, 4, 5), (7, 9, 33), (16, 16, 16), (33, 17, 65), (20, 70, 31), (9, 130, 47)]
KINDS = ["smooth", "noisy", "sparse", "constant", "checker", "step", "extreme"]


@pytest.mark.parametrize("shape", SHAPES, ids=str)
@pytest.mark.parametrize("kind", KINDS)
def test_parity_shapes_and_kinds(shape, kind):
    rng = np.random.default_rng(zlib.crc32(repr((shape, kind)).encode()))
    q = oc.random_index_field(rng, shape, kind)
    assert_parity(q, 0.01)


@pytest.mark.parametrize("kw", [dict(sign_rule=1), dict(b2_rule=1), dict(grad_threshold=3),
                                dict(idw_power=2.0), dict(eta=0.5), dict(idw_power=0.7, b2_rule=1)],
                         ids=str)
@pytest.mark.parametrize("shape", [(501,), (61, 77), (23, 31, 45)], ids=str)
def test_parity_rule_variants(shape, kw):
    rng = np.random.default_rng(zlib.crc32(repr((shape, sorted(kw.items()))).encode()))
    q = oc.random_index_field(rng, shape, "smooth")
    assert_parity(q, 0.02, **kw)


@pytest.mark.parametrize("shape", [(32768,), (4096, 3), (3, 4096), (5, 16383), (4096, 2, 3),
                                   (3, 4096, 5), (2, 3, 16383), (1, 1, 32768)], ids=str)
def test_parity_maximum_extents(shape):
    rng = np.random.default_rng(zlib.crc32(repr(shape).encode()))
    q = oc.random_index_field(rng, shape, "smooth")
    assert_parity(q, 0.01)


def test_golden_vectors_on_gpu():
    import glob, json, os
    for path in sorted(glob.glob(os.path.join(os.path.dirname(__file__), "golden", "V*.json"))):
        fx = json.load(open(path))
        p = fx["params"]
        out, maps = gpu_run(np.array(fx["q"], np.int32), fx["eb"], eta=fx["eta"],
                            grad_threshold=p["grad_threshold"], sign_rule=p["sign_rule"],
                            b2_rule=p["b2_rule"])
        for k, v in fx["expect"].items():
            if k == "out":
                np.testing.assert_allclose(out, np.array(v), atol=1e-6, err_msg=fx["name"])
            else:
                np.testing.assert_array_equal(maps[k], np.array(v).astype(maps[k].dtype),
                                              err_msg=f"{fx['name']}:{k}")


def _field(name, shape, seed):
    if name == "sinusoids":
        return torch.from_numpy(synth.sinusoids(shape, seed=seed)).cuda()
    if name == "grf":
        return synth.grf(shape, slope=11.0 / 3.0, seed=seed, device="cuda")
    return synth.grf_front(shape, seed=seed, device="cuda")


def _real_field_parity(name, shape, seed, rel_eb):
    x = _field(name, shape, seed)
    xr = synth.value_range(x)
    eb = rel_eb * xr
    q = synth.quantize(x, eb)
    ref, out = assert_parity(q.cpu().numpy(), eb, x_range=xr)
    err = np.abs(x.cpu().numpy().astype(np.float64) - out.astype(np.float64))
    assert err.max() <= 1.9 * eb + 1e-6 * xr, f"error bound violated: {err.max() / eb:.6f} eps"
    return ref, out


def test_config_64cube_sinusoids():
    _real_field_parity("sinusoids", (64, 64, 64), 1, 1e-2)


@pytest.mark.parametrize("rel_eb", [1e-3, 1e-2])
def test_config_512cube_grf_full_size(rel_eb):
    _real_field_parity("grf", (512, 512, 512), 2, rel_eb)


@pytest.mark.parametrize("shape,seed", [((100, 500, 500), 3), ((256, 384, 384), 4),
                                        ((98, 1200, 1200), 5), ((1800, 3600), 6)], ids=str)
def test_config_anisotropic_full_size(shape, seed):
    _real_field_parity("front", shape, seed, 1e-3)


def test_host_entry_point_matches_device_entry_point():
    x = synth.grf((40, 50, 60), seed=9, device="cuda")
    eb = 1e-3
    q = synth.quantize(x, eb)
    dev = qai.mitigate(q, eb)
    qh = q.cpu().pin_memory()
    host = qai.mitigate_host(qh, eb)
    torch.cuda.synchronize()
    assert torch.equal(dev.cpu(), host)


def test_repeat_calls_and_workspace_reuse_are_deterministic():
    x = synth.grf((64, 80, 96), seed=10, device="cuda")
    q = synth.quantize(x, 2e-3)
    ws = qai.alloc_workspace(qai.workspace_size(tuple(q.shape)))
    a = qai.mitigate(q, 2e-3, workspace=ws)
    b = qai.mitigate(q, 2e-3, workspace=ws)
    c = qai.mitigate(q, 2e-3)             # library-allocated workspace
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(a, c)


def test_profile_and_launch_count():
    q = synth.quantize(synth.grf((32, 32, 32), seed=1, device="cuda"), 1e-2)
    qai.profile_read()
    qai.profile_enable(True)
    n0 = qai.launch_count()
    qai.mitigate(q, 1e-2)
    torch.cuda.synchronize()
    stats = qai.profile_read()
    qai.profile_enable(False)
    names = {"detect", "near", "rowpass1", "colpass1_y", "colpass1_z_final", "pack_s", "b2sparse", "brute_sparse",
             "b2map", "signed_query", "signed_query_mid", "b2list", "signed_brute", "expand", "rowpass2",
             "colpass2_y", "colpass2_z_final"}
    # one launch each, and step A's exact pass (gated, run behind the fast one)
    assert qai.launch_count() - n0 == len(names) + 1
    assert set(stats) == names
    assert all(v[0] == 1 and v[1] > 0 for v in stats.values())


@pytest.mark.parametrize("name,shape,rel_eb", [("grf", (96, 128, 160), 1e-3), ("front", (64, 200, 72), 1e-3),
                                               ("front", (300, 500), 1e-3), ("sinusoids", (40, 64, 64), 3e-3)],
                         ids=str)
def test_flat_tiles_equal_full_evaluation(name, shape, rel_eb):
    """Tiles whose columns hold no S != 0 stream D'' = D' in the last pass; the
    debug path evaluates every point. Both must give the same bits, and the
    field must have columns of both kinds."""
    x = _field(name, shape, 11)
    eb = rel_eb * synth.value_range(x)
    q = synth.quantize(x, eb)
    fast = qai.mitigate(q, eb)
    fast_c = qai.mitigate(q, eb, output_c=True)
    full, maps = qai.mitigate(q, eb, debug=True)
    full_c, _ = qai.mitigate(q, eb, debug=True, output_c=True)
    torch.cuda.synchronize()
    assert torch.equal(fast, full) and torch.equal(fast_c, full_c)
    col_has = (maps["s"] != 0).any(dim=0)             # columns of the last pass
    assert bool(col_has.any()) and not bool(col_has.all())
