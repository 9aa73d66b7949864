"""qai_mitigate_static: the entry point for callers that cannot allocate device
memory (it runs on a scratch array compiled into the library). It must give
what qai_mitigate gives, call after call, although every call reuses the same
scratch array and finds there whatever the call before left. This file is
collected last on purpose."""
import ctypes

import pytest
import torch

from paper_2602_20097_gb300 import qai, synth


def _static(q, eb, out):
    lib = qai.load()
    p = qai.default_params()
    rc = lib.qai_mitigate_static(ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                 q.dim(), qai._dims(tuple(q.shape)), float(eb), ctypes.byref(p),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


def _case(kind, shape, seed):
    x = (synth.grf_front if kind == "front" else synth.grf)(shape, seed=seed, device="cuda")
    eb = 1e-3 * synth.value_range(x)
    return synth.quantize(x, eb), eb, 1e-6 * synth.value_range(x)


@pytest.mark.gpu
def test_static_scratch_matches_qai_mitigate_call_after_call():
    # the largest field first, so that the smaller ones after it find its
    # contents at the same offsets of the scratch array; then the same shape
    # again with another seed; fields of exactly QAI_STATIC_MAX_POINTS points
    # in 3-D (128^3) and in 2-D (1024 x 2048)
    cases = [("front", (96, 128, 160), 22), ("grf", (64, 72, 80), 21), ("grf", (64, 72, 80), 23),
             ("grf", (128, 128, 128), 24), ("front", (1024, 2048), 25), ("grf", (40, 50, 60), 26)]
    for kind, shape, seed in cases:
        q, eb, tol = _case(kind, shape, seed)
        ref = qai.mitigate(q, eb)
        out = torch.full(tuple(q.shape), float("nan"), dtype=torch.float32, device="cuda")
        assert _static(q, eb, out) == 0, qai.load().qai_last_error()
        torch.cuda.synchronize()
        diff = (out.double() - ref.double()).abs().max().item()   # the parity tolerance of the GPU tests
        assert diff <= tol, f"{shape}: static scratch result differs from qai_mitigate by {diff:.3e}"


@pytest.mark.gpu
def test_a_warm_static_call_allocates_no_device_memory():
    q, eb, tol = _case("grf", (64, 64, 64), 27)
    out = torch.empty(tuple(q.shape), dtype=torch.float32, device="cuda")
    assert _static(q, eb, out) == 0, qai.load().qai_last_error()     # the first call loads the array
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _static(q, eb, out) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device memory changed by {free0 - free1} bytes across static calls"


@pytest.mark.gpu
def test_static_scratch_rejects_fields_beyond_its_limit():
    for shape in ((129, 128, 128), (1025, 2048)):                   # 2^21 + 2^14 and 2^21 + 2^11 points
        q = torch.zeros(shape, dtype=torch.int32, device="cuda")
        out = torch.empty(q.shape, dtype=torch.float32, device="cuda")
        assert _static(q, 1e-3, out) == 2
        assert b"static scratch limit" in qai.load().qai_last_error()
