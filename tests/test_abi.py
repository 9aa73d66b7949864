"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/qai.h declares; host-side argument checks return status codes without
launching anything (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2602_20097_gb300 import build, qai

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qai.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qai_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    return qai.load()


def test_library_builds_in_tree():
    path = build.build()
    assert os.path.exists(path) and path.startswith(os.path.join(ROOT, "paper_2602_20097_gb300"))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "qai_mitigate" in names and len(names) >= 8
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(qai.SIGNATURES), "binding and header disagree"


def test_default_params(lib):
    p = qai.default_params()
    assert (p.eta, p.idw_power, p.grad_threshold, p.sign_rule, p.b2_rule, p.flags) == (0.9, 1.0, 2, 0, 0, 0)


def _ws(shape, flags=0):
    n = ctypes.c_size_t()
    rc = qai.load().qai_workspace_size(len(shape), qai._dims(shape), flags, ctypes.byref(n))
    return rc, n.value


def test_workspace_sizes():
    rc, n3 = _ws((512, 512, 512))
    assert rc == 0 and n3 >= 512 ** 3 * 12
    rc, n3i = _ws((512, 512, 512), qai.WS_INDEX)
    assert rc == 0 and n3i >= n3 + 512 ** 3 * 4
    rc, n2 = _ws((1800, 3600))
    assert rc == 0 and n2 >= 1800 * 3600 * 8
    # squeezing: a 1 x ny x nx field needs the 2-D workspace
    assert _ws((1, 1800, 3600))[1] == n2


@pytest.mark.parametrize("shape,code", [((0, 4, 4), 2), ((4, 4, 20000), 2), ((5000, 4, 4), 2),
                                        ((40000,), 2), ((2048, 2048, 1024), 2), ((3,) * 4, 2)])
def test_unsupported_shapes(shape, code):
    rc, _ = _ws(shape)
    assert rc == code


def _call(q=1, out=1, shape=(8, 8, 8), eb=0.1, params=None, ws=None, wsb=0):
    lib = qai.load()
    return lib.qai_mitigate(ctypes.c_void_p(q) if q else None, ctypes.c_void_p(out) if out else None,
                            len(shape), qai._dims(shape), eb,
                            ctypes.byref(params) if params is not None else None,
                            ctypes.c_void_p(ws) if ws else None, wsb, None, None)


def test_argument_errors_return_status():
    lib = qai.load()
    assert _call(q=0) == 1
    assert _call(out=0) == 1
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        assert _call(eb=bad) == 1
    for field, val in (("eta", float("nan")), ("eta", -1.0), ("idw_power", 0.0),
                       ("grad_threshold", 0), ("sign_rule", 2), ("b2_rule", -1), ("flags", 2)):
        p = qai.default_params()
        setattr(p, field, val)
        assert _call(params=p) == 1, field
    assert _call(shape=(8, 0, 8)) == 2
    # a workspace that is too small or misaligned is rejected before any launch
    assert _call(ws=256, wsb=16) == 1
    assert _call(ws=257, wsb=1 << 30) == 1
    assert lib.qai_status_string(1) == b"QAI_ERR_INVALID_ARG"
    assert b"workspace" in lib.qai_last_error()


def test_profile_counters_start_empty():
    assert qai.profile_read() == {}
    assert qai.launch_count() >= 0


def test_adjoint_sizes_and_argument_errors():
    lib = qai.load()
    assert qai.saved_size((64, 64, 64)) >= 64 ** 3 * 9
    assert 0 < qai.workspace_size_backward((64, 64, 64), False) <= 64 * 1024
    # recompute mode: the forward workspace, D'' and Dist2 arrays, the partials
    fwd = qai.workspace_size((64, 64, 64))
    assert fwd + 8 * 64 ** 3 < qai.workspace_size_backward((64, 64, 64), True) < fwd + 8 * 64 ** 3 + 64 * 1024
    assert qai.workspace_size_backward((5000,), True) >= qai.workspace_size((5000,)) + 2 * 4 * 5000
    shape = (8, 8, 8)
    rc = lib.qai_mitigate_backward(ctypes.c_void_p(16), None, None, ctypes.c_void_p(16), 3, qai._dims(shape),
                                   0.1, None, None, None, 0, None)
    assert rc == 1                                     # NULL grad_out
    rc = lib.qai_mitigate_backward(ctypes.c_void_p(16), ctypes.c_void_p(16), None, ctypes.c_void_p(16), 3,
                                   qai._dims(shape), 0.1, None, None, None, 0, None)
    assert rc == 1 and b"workspace" in lib.qai_last_error()   # no workspace
    rc = lib.qai_mitigate_save(ctypes.c_void_p(16), ctypes.c_void_p(16), 3, qai._dims(shape), 0.1, None,
                               ctypes.c_void_p(257), None, 0, None)
    assert rc == 1                                     # misaligned saved state


def test_quality_sizes_and_argument_errors():
    lib = qai.load()
    assert 0 < qai.workspace_size_quality((512, 512, 512)) < 1 << 20
    assert qai.workspace_size_quality((1800, 3600), 7, 2) > 0
    n = ctypes.c_size_t()
    for w, s in ((0, 2), (12, 2), (7, 0), (7, 5)):
        assert lib.qai_workspace_size_quality(3, qai._dims((8, 8, 8)), w, s, ctypes.byref(n)) == 1
    shape = (8, 8, 8)
    rc = lib.qai_quality(None, ctypes.c_void_p(256), 3, qai._dims(shape), 7, 2, ctypes.c_void_p(256), None,
                         ctypes.c_void_p(256), 1 << 20, None)
    assert rc == 1                                        # NULL x
    rc = lib.qai_quality(ctypes.c_void_p(256), ctypes.c_void_p(256), 3, qai._dims(shape), 7, 2,
                         ctypes.c_void_p(256), None, ctypes.c_void_p(256), 8, None)
    assert rc == 1 and b"workspace" in lib.qai_last_error()


def test_shard_entry_points_check_arguments_before_launching():
    lib = qai.load()
    fake = 4096        # never dereferenced: every call below fails its checks first
    dims = qai._dims((4, 5, 6))
    ws, wb = ctypes.c_size_t(), ctypes.c_int()
    assert lib.qai_shard_sizes(3, dims, ctypes.byref(ws), ctypes.byref(wb)) == 0
    assert ws.value >= 4 * 5 * 6 * 2 and wb.value == 4
    assert lib.qai_shard_sizes(2, qai._dims((4, 5)), ctypes.byref(ws), ctypes.byref(wb)) == 0
    assert ws.value == 0 and wb.value == 2
    assert lib.qai_shard_sizes(1, qai._dims((4,)), ctypes.byref(ws), ctypes.byref(wb)) == 2
    assert lib.qai_shard_sizes(3, qai._dims((4, 5000, 6)), ctypes.byref(ws), ctypes.byref(wb)) == 2
    assert lib.qai_shard_rows(3, 3, dims, fake, None, fake, fake, fake, 1 << 20, None, None) == 1
    assert lib.qai_shard_rows(2, 3, dims, fake, None, fake, fake, fake, 1 << 20, None, None) == 1  # no S
    assert lib.qai_shard_rows(1, 3, dims, fake, None, fake, fake, fake, 1, None, None) == 1        # workspace
    assert lib.qai_shard_lines(1, 3, qai._dims((5, 5, 6)), dims, fake, None, fake, fake, fake, None, 0.1,
                               None, None) == 2                                                    # band > field
    assert lib.qai_shard_lines(2, 3, dims, dims, fake, fake, fake, fake, fake, fake, -1.0, None, None) == 1
    assert lib.qai_shard_copy(fake, 4, fake, 8, 16, 2, None) == 1                                 # pitch < width
    assert lib.qai_shard_copy(None, 16, None, 16, 0, 2, None) == 0                                # nothing to copy
