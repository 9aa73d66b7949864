"""qai_mitigate_static: the entry point for callers that cannot allocate device
memory (it runs on a scratch array compiled into the library). It must give
what qai_mitigate gives, call after call, although every call reuses the same
scratch array. This file is collected last on purpose."""
import ctypes

import numpy as np
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


@pytest.mark.gpu
def test_static_scratch_matches_qai_mitigate_on_two_calls_in_a_row():
    fields = [synth.grf((64, 72, 80), seed=21, device="cuda"),      # 368,640 points
              synth.grf_front((96, 128, 160), seed=22, device="cuda")]  # 1,966,080 points
    for x in fields:
        eb = 1e-3 * synth.value_range(x)
        q = synth.quantize(x, eb)
        ref = qai.mitigate(q, eb)
        out = torch.full(tuple(q.shape), float("nan"), dtype=torch.float32, device="cuda")
        assert _static(q, eb, out) == 0, qai.load().qai_last_error()
        torch.cuda.synchronize()
        tol = 1e-6 * synth.value_range(x)           # the parity tolerance of the GPU tests
        diff = (out.double() - ref.double()).abs().max().item()
        assert diff <= tol, f"static scratch result differs from qai_mitigate by {diff:.3e}"


@pytest.mark.gpu
def test_static_scratch_rejects_fields_beyond_its_limit():
    q = torch.zeros((129, 128, 128), dtype=torch.int32, device="cuda")   # 2,113,536 points
    out = torch.empty(q.shape, dtype=torch.float32, device="cuda")
    assert _static(q, 1e-3, out) == 2
    assert b"static scratch limit" in qai.load().qai_last_error()
