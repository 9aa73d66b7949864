"""Python binding of ``libqai.so`` (ctypes; argument marshalling only).

Every step of the method runs in the library's CUDA kernels; this module only
passes device pointers, sizes and the current CUDA stream. PyTorch provides the
device memory and the stream. There is no CPU fallback: if the library cannot
be loaded, :func:`load` raises :class:`QAIError`.

Names follow the C ABI in ``include/qai.h``:

* :func:`mitigate` -- Algorithm 4 on a CUDA int32 tensor, returns D'' (float32);
  ``debug=True`` also returns the per-step maps B1, S_B, Dist1, I1, S, B2, Dist2.
* :func:`mitigate_host` -- the same from/to host (pinned) tensors, with the
  copies made by the library on the stream.
* :func:`workspace_size`, :func:`route_counts`, :func:`profile_enable`,
  :func:`profile_read`, :func:`launch_count`.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

P = ctypes.c_void_p
_lock = threading.Lock()
_lib = None

SIGN_SUM, SIGN_FIRST = 0, 1
B2_SAME_Q, B2_LITERAL = 0, 1
WS_INDEX = 1
FLAG_OUTPUT_C = 1
# route selection bits of qai_params.flags (testing and measurement only: every
# route gives the same output bits)
FLAG_EDT2_DENSE = 0x10
FLAG_EDT2_HANDOVER = 0x20
FLAG_EDT2_LIST = 0x40
FLAG_EDT1_SEPARABLE = 0x80
ROUTE_FLAGS = {"auto": 0, "off": FLAG_EDT2_DENSE, "dense": FLAG_EDT2_HANDOVER, "brute": FLAG_EDT2_LIST}
INF32 = 2 ** 31 - 1


class QAIError(RuntimeError):
    pass


class Params(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_double), ("idw_power", ctypes.c_double),
                ("grad_threshold", ctypes.c_int32), ("sign_rule", ctypes.c_int32),
                ("b2_rule", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class DebugOut(ctypes.Structure):
    _fields_ = [("b1", P), ("sb", P), ("dist1", P), ("idx1", P), ("s", P), ("b2", P), ("dist2", P)]


class BatchChoice(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int32), ("fields", ctypes.c_int32), ("streams", ctypes.c_int32),
                ("order", ctypes.c_int32), ("ms", ctypes.c_float), ("grouped", ctypes.c_int32),
                ("tile_w", ctypes.c_int32), ("rows_per_band", ctypes.c_int32),
                ("points_per_block", ctypes.c_int32), ("launches", ctypes.c_int32)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double), ("algo_bytes", ctypes.c_double)]


# name -> (restype, argtypes) of every symbol include/qai.h declares
SIGNATURES = {
    "qai_default_params": (None, [ctypes.POINTER(Params)]),
    "qai_workspace_size": (ctypes.c_int, [ctypes.c_int, P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_size_t)]),
    "qai_mitigate": (ctypes.c_int, [P, P, ctypes.c_int, P, ctypes.c_double, ctypes.POINTER(Params),
                                    P, ctypes.c_size_t, P, ctypes.POINTER(DebugOut)]),
    "qai_route_counts": (ctypes.c_int, [P, ctypes.c_int, P, P, P]),
    "qai_workspace_size_host": (ctypes.c_int, [ctypes.c_int, P, ctypes.POINTER(ctypes.c_size_t)]),
    "qai_mitigate_host": (ctypes.c_int, [P, P, ctypes.c_int, P, ctypes.c_double, ctypes.POINTER(Params),
                                         P, ctypes.c_size_t, P]),
    "qai_mitigate_static": (ctypes.c_int, [P, P, ctypes.c_int, P, ctypes.c_double,
                                           ctypes.POINTER(Params), P]),
    "qai_dequantize": (ctypes.c_int, [P, P, ctypes.c_int64, ctypes.c_double, P]),
    "qai_mitigate_add": (ctypes.c_int, [P, P, P, ctypes.c_int, P, ctypes.c_double, ctypes.POINTER(Params),
                                        P, P, ctypes.c_size_t, P]),
    "qai_saved_size": (ctypes.c_int, [ctypes.c_int, P, ctypes.POINTER(ctypes.c_size_t)]),
    "qai_mitigate_save": (ctypes.c_int, [P, P, ctypes.c_int, P, ctypes.c_double, ctypes.POINTER(Params),
                                         P, P, ctypes.c_size_t, P]),
    "qai_workspace_size_backward": (ctypes.c_int, [ctypes.c_int, P, ctypes.c_int,
                                                   ctypes.POINTER(ctypes.c_size_t)]),
    "qai_mitigate_backward": (ctypes.c_int, [P, P, P, P, ctypes.c_int, P, ctypes.c_double,
                                             ctypes.POINTER(Params), P, P, ctypes.c_size_t, P]),
    "qai_workspace_size_batched": (ctypes.c_int, [ctypes.c_int, P, P, ctypes.POINTER(ctypes.c_size_t)]),
    "qai_mitigate_batched": (ctypes.c_int, [ctypes.c_int, P, P, P, P, P, ctypes.POINTER(Params), P,
                                            ctypes.c_size_t, P]),
    "qai_autotune_batched": (ctypes.c_int, [ctypes.c_int, P, P, P, P, P, ctypes.POINTER(Params), P,
                                            ctypes.c_size_t, P, ctypes.POINTER(BatchChoice)]),
    "qai_shard_sizes": (ctypes.c_int, [ctypes.c_int, P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_int)]),
    "qai_shard_rows": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, P, P, P, P, P, P, ctypes.c_size_t,
                                      ctypes.POINTER(Params), P]),
    "qai_shard_lines": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, P, P, P, P, P, P, P, P, ctypes.c_double,
                                       ctypes.POINTER(Params), P]),
    "qai_shard_copy": (ctypes.c_int, [P, ctypes.c_int64, P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, P]),
    "qai_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "qai_profile_read": (ctypes.c_int, [ctypes.POINTER(KernelStat), ctypes.c_int]),
    "qai_profile_select": (ctypes.c_int, [ctypes.c_char_p]),
    "qai_workspace_size_quality": (ctypes.c_int, [ctypes.c_int, P, ctypes.c_int, ctypes.c_int,
                                                  ctypes.POINTER(ctypes.c_size_t)]),
    "qai_quality": (ctypes.c_int, [P, P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, P, P, P,
                                   ctypes.c_size_t, P]),
    "qai_launch_count": (ctypes.c_int64, []),
    "qai_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "qai_last_error": (ctypes.c_char_p, []),
}


def load(build_if_missing: bool = True):
    """Load ``libqai.so`` (building it with nvcc first if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and _build.stale():
            try:
                _build.build()
            except Exception as e:  # noqa: BLE001 - re-raised with context
                raise QAIError(f"libqai.so could not be built: {e}") from e
        if not os.path.exists(path):
            raise QAIError(f"libqai.so not found at {path}; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def library_path() -> str:
    return _build.LIB


def _check(rc):
    if rc != 0:
        lib = load()
        raise QAIError(f"{lib.qai_status_string(rc).decode()}: {lib.qai_last_error().decode()}")


def default_params(**kw) -> Params:
    p = Params()
    load().qai_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if v is not None:
            setattr(p, k, v)
    return p


def _dims(shape):
    arr = (ctypes.c_int64 * len(shape))(*[int(s) for s in shape])
    return arr


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def workspace_size(shape, with_index: bool = False) -> int:
    n = ctypes.c_size_t()
    _check(load().qai_workspace_size(len(shape), _dims(shape), WS_INDEX if with_index else 0,
                                     ctypes.byref(n)))
    return int(n.value)


def workspace_size_host(shape) -> int:
    n = ctypes.c_size_t()
    _check(load().qai_workspace_size_host(len(shape), _dims(shape), ctypes.byref(n)))
    return int(n.value)


def alloc_workspace(nbytes: int, device=None) -> torch.Tensor:
    """A device byte buffer of ``nbytes`` (the caching allocator aligns to 512 B)."""
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device or "cuda")


def route_flags(route: str = "auto", first_edt: str = "local") -> int:
    """qai_params.flags bits of a route choice: ``route`` = "auto" (default),
    "off" (dense second EDT alone), "dense" (the route hands over to the dense
    second EDT), "brute" (no shell search); ``first_edt`` = "local" (default)
    or "separable". Every choice gives the same output bits."""
    if route not in ROUTE_FLAGS or first_edt not in ("local", "separable"):
        raise QAIError(f"unknown route {route!r} / first_edt {first_edt!r}")
    return ROUTE_FLAGS[route] | (FLAG_EDT1_SEPARABLE if first_edt == "separable" else 0)


def _params(eta, idw_power, grad_threshold, sign_rule, b2_rule, output_c=False, route="auto",
            first_edt="local"):
    return default_params(eta=eta, idw_power=idw_power, grad_threshold=grad_threshold,
                          sign_rule=sign_rule, b2_rule=b2_rule,
                          flags=(FLAG_OUTPUT_C if output_c else 0) | route_flags(route, first_edt))


def mitigate(q: torch.Tensor, eb: float, eta: float = 0.9, idw_power: float = 1.0,
             grad_threshold: int = 2, sign_rule: int = SIGN_SUM, b2_rule: int = B2_SAME_Q,
             out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
             debug: bool = False, stream=None, output_c: bool = False, route: str = "auto",
             first_edt: str = "local"):
    """Algorithm 4 on a contiguous CUDA int32 tensor ``q`` (rank 1-3).

    Returns D'' as a float32 tensor of ``q``'s shape (the compensation C alone
    with ``output_c``), or ``(D'', maps)`` when ``debug`` with ``maps`` = dict
    of the per-step outputs (device tensors). ``route`` and ``first_edt``
    select how the EDTs are computed (see :func:`route_flags`; testing only).
    """
    lib = load()
    if not (q.is_cuda and q.dtype == torch.int32 and q.is_contiguous()):
        raise QAIError("q must be a contiguous CUDA int32 tensor")
    shape = tuple(q.shape)
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=q.device)
    dbg = None
    maps = None
    if debug:
        maps = {k: torch.empty(shape, dtype=t, device=q.device) for k, t in
                (("b1", torch.uint8), ("sb", torch.int8), ("dist1", torch.int32),
                 ("idx1", torch.int32), ("s", torch.int8), ("b2", torch.uint8),
                 ("dist2", torch.int32))}
        dbg = DebugOut(**{k: v.data_ptr() for k, v in maps.items()})
    _check_out(out, shape, q.device)
    if workspace is None:
        workspace = alloc_workspace(workspace_size(shape, with_index=debug), q.device)
    p = _params(eta, idw_power, grad_threshold, sign_rule, b2_rule, output_c, route, first_edt)
    with torch.cuda.device(q.device):
        rc = lib.qai_mitigate(q.data_ptr(), out.data_ptr(), len(shape), _dims(shape), float(eb),
                              ctypes.byref(p), workspace.data_ptr(), workspace.numel(), _stream(stream),
                              ctypes.byref(dbg) if dbg is not None else None)
    _check(rc)
    return (out, maps) if debug else out


def _check_out(out, shape, device):
    """``out`` must be a contiguous float32 tensor of ``shape`` on ``device``."""
    if not (out.dtype == torch.float32 and out.is_contiguous() and tuple(out.shape) == tuple(shape)
            and out.device == device):
        raise QAIError(f"out must be a contiguous float32 tensor of shape {tuple(shape)} on {device}")


def route_counts(workspace: torch.Tensor, shape, stream=None) -> dict:
    """How the last plain :func:`mitigate` on ``workspace`` (rank 2 or 3)
    computed the EDTs: ``queries`` (points with S != 0 off B1, where
    Dist2 matters), ``list_searched`` (those the shell search left to the
    search over all B2 sites), ``b2_sites`` (sites listed for it), ``dense``
    (the dense second EDT ran), ``signed_b1`` (B1 points with S != 0, -1
    when too many to list) and ``separable_first_edt`` (the bounded search of
    the first EDT fell short and the separable passes ran). Synchronises the
    stream."""
    c = (ctypes.c_int32 * 6)()
    _check(load().qai_route_counts(workspace.data_ptr(), len(shape), _dims(shape), c, _stream(stream)))
    return {"queries": c[0], "list_searched": c[1], "b2_sites": c[2], "dense": bool(c[3]),
            "signed_b1": c[4], "separable_first_edt": bool(c[5])}


def mitigate_host(q_host: torch.Tensor, eb: float, out_host: torch.Tensor | None = None,
                  workspace: torch.Tensor | None = None, stream=None, **kw):
    """Algorithm 4 from host memory: the library copies q in and D'' out on
    the stream. Pinned tensors keep the copies asynchronous; synchronise the
    stream before reading the result."""
    lib = load()
    if q_host.is_cuda or q_host.dtype != torch.int32 or not q_host.is_contiguous():
        raise QAIError("q_host must be a contiguous host int32 tensor")
    shape = tuple(q_host.shape)
    if out_host is None:
        out_host = torch.empty(shape, dtype=torch.float32, pin_memory=q_host.is_pinned())
    if workspace is None:
        workspace = alloc_workspace(workspace_size_host(shape))
    p = _params(kw.get("eta", 0.9), kw.get("idw_power", 1.0), kw.get("grad_threshold", 2),
                kw.get("sign_rule", SIGN_SUM), kw.get("b2_rule", B2_SAME_Q))
    rc = lib.qai_mitigate_host(q_host.data_ptr(), out_host.data_ptr(), len(shape), _dims(shape),
                               float(eb), ctypes.byref(p), workspace.data_ptr(), workspace.numel(),
                               _stream(stream))
    _check(rc)
    return out_host


def saved_size(shape) -> int:
    n = ctypes.c_size_t()
    _check(load().qai_saved_size(len(shape), _dims(shape), ctypes.byref(n)))
    return int(n.value)


def workspace_size_backward(shape, recompute: bool) -> int:
    n = ctypes.c_size_t()
    _check(load().qai_workspace_size_backward(len(shape), _dims(shape), 1 if recompute else 0,
                                              ctypes.byref(n)))
    return int(n.value)


def mitigate_save(q: torch.Tensor, eb: float, eta: float = 0.9, idw_power: float = 1.0,
                  grad_threshold: int = 2, sign_rule: int = SIGN_SUM, b2_rule: int = B2_SAME_Q,
                  output_c: bool = False, saved: torch.Tensor | None = None,
                  workspace: torch.Tensor | None = None, stream=None, out: torch.Tensor | None = None):
    """Forward that also keeps Dist1, Dist2 and S for the stored-mode adjoint.
    Returns ``(out, saved)``."""
    lib = load()
    shape = tuple(q.shape)
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=q.device)
    if saved is None:
        saved = alloc_workspace(saved_size(shape), q.device)
    if workspace is None:
        workspace = alloc_workspace(workspace_size(shape), q.device)
    p = _params(eta, idw_power, grad_threshold, sign_rule, b2_rule, output_c)
    _check(lib.qai_mitigate_save(q.data_ptr(), out.data_ptr(), len(shape), _dims(shape), float(eb),
                                 ctypes.byref(p), saved.data_ptr(), workspace.data_ptr(),
                                 workspace.numel(), _stream(stream)))
    return out, saved


def mitigate_backward(q: torch.Tensor, eb: float, grad_out: torch.Tensor, saved=None,
                      eta: float = 0.9, idw_power: float = 1.0, grad_threshold: int = 2,
                      sign_rule: int = SIGN_SUM, b2_rule: int = B2_SAME_Q,
                      want_grad_dprime: bool = True, workspace: torch.Tensor | None = None,
                      stream=None):
    """Adjoint of step E: returns ``(dL/dD' or None, tensor([dL/deta, dL/dp]))``
    (float64, on the device). ``saved`` from :func:`mitigate_save` selects the
    stored mode; ``None`` recomputes Dist1, Dist2 and S from ``q``."""
    lib = load()
    shape = tuple(q.shape)
    g = grad_out.contiguous().to(torch.float32)
    gd = torch.empty(shape, dtype=torch.float32, device=q.device) if want_grad_dprime else None
    gp = torch.empty(2, dtype=torch.float64, device=q.device)
    if workspace is None:
        workspace = alloc_workspace(workspace_size_backward(shape, saved is None), q.device)
    p = _params(eta, idw_power, grad_threshold, sign_rule, b2_rule)
    _check(lib.qai_mitigate_backward(
        q.data_ptr(), g.data_ptr(), gd.data_ptr() if gd is not None else None, gp.data_ptr(),
        len(shape), _dims(shape), float(eb), ctypes.byref(p),
        saved.data_ptr() if saved is not None else None,
        workspace.data_ptr(), workspace.numel(), _stream(stream)))
    return gd, gp


def dequantize(q: torch.Tensor, eb: float, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """D' = 2 q eps (Eq. 1) in float32, computed by the library's kernel."""
    if not (q.is_cuda and q.dtype == torch.int32 and q.is_contiguous()):
        raise QAIError("q must be a contiguous CUDA int32 tensor")
    if out is None:
        out = torch.empty(q.shape, dtype=torch.float32, device=q.device)
    _check_out(out, q.shape, q.device)
    _check(load().qai_dequantize(q.data_ptr(), out.data_ptr(), q.numel(), float(eb), _stream(stream)))
    return out


def mitigate_add(q: torch.Tensor, dprime: torch.Tensor, eb: float, eta: float = 0.9, idw_power: float = 1.0,
                 saved: torch.Tensor | None = None, workspace: torch.Tensor | None = None, stream=None,
                 out: torch.Tensor | None = None):
    """D'' = D' + C with the dequantized field ``dprime`` given (float32, q's
    shape): C from ``q`` by Algorithm 4 and the add, both in the library.
    ``saved`` (from :func:`saved_size`) also receives the stored-mode state."""
    lib = load()
    shape = tuple(q.shape)
    if not (dprime.is_cuda and dprime.dtype == torch.float32 and dprime.is_contiguous()
            and tuple(dprime.shape) == shape and dprime.device == q.device):
        raise QAIError("dprime must be a contiguous float32 CUDA tensor of q's shape")
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=q.device)
    _check_out(out, shape, q.device)
    if workspace is None:
        workspace = alloc_workspace(workspace_size(shape), q.device)
    p = _params(eta, idw_power, 2, SIGN_SUM, B2_SAME_Q)
    _check(lib.qai_mitigate_add(q.data_ptr(), dprime.data_ptr(), out.data_ptr(), len(shape), _dims(shape),
                                float(eb), ctypes.byref(p), saved.data_ptr() if saved is not None else None,
                                workspace.data_ptr(), workspace.numel(), _stream(stream)))
    return out


class QAIFunction(torch.autograd.Function):
    """D'' = D' + C(q; eta, p), differentiable in D', eta and p with the EDT
    assignment held fixed (the adjoint of step E, run by the CUDA library).

    ``QAIFunction.apply(dprime, eta, p, q, eb, stored)``: ``dprime`` float32
    field on the device, ``eta`` and ``p`` 0-dim float64 tensors, ``q`` the
    int32 indices, ``stored`` True keeps Dist1/Dist2/S from the forward,
    False recomputes them in the backward (no memory held between the two).
    The forward's D'' (C and the add) comes from the library.
    """

    @staticmethod
    def forward(ctx, dprime, eta, p, q, eb, stored=True):
        e, pw = float(eta), float(p)
        saved = alloc_workspace(saved_size(tuple(q.shape)), q.device) if stored else None
        out = mitigate_add(q, dprime.contiguous().to(torch.float32), eb, eta=e, idw_power=pw, saved=saved)
        ctx.save_for_backward(q)
        ctx.saved_state, ctx.eb, ctx.e, ctx.pw = saved, eb, e, pw
        return out

    @staticmethod
    def backward(ctx, grad):
        (q,) = ctx.saved_tensors
        _, gp = mitigate_backward(q, ctx.eb, grad, saved=ctx.saved_state, eta=ctx.e,
                                  idw_power=ctx.pw, want_grad_dprime=False)
        return grad, gp[0], gp[1], None, None, None


def tune(q: torch.Tensor, eb: float, x: torch.Tensor, eta: float = 0.9, p: float = 1.0,
         steps: int = 20, lr: float = 0.05, stored: bool = True):
    """Gradient descent on (eta, p) minimising mean((D'' - x)^2) against the
    original field ``x``; returns the list of (eta, p, loss) per step."""
    dprime = dequantize(q, eb)
    e = torch.tensor(eta, dtype=torch.float64, device=q.device, requires_grad=True)
    pw = torch.tensor(p, dtype=torch.float64, device=q.device, requires_grad=True)
    xs = x.to(torch.float32)
    hist = []
    for _ in range(steps):
        out = QAIFunction.apply(dprime, e, pw, q, eb, stored)
        loss = torch.mean((out.double() - xs.double()) ** 2)
        e.grad = pw.grad = None
        loss.backward()
        hist.append((float(e.detach()), float(pw.detach()), float(loss.detach())))
        with torch.no_grad():
            # normalised steps: the loss scale is eps^2, so divide by it
            e -= lr * e.grad / (eb * eb)
            pw -= lr * pw.grad / (eb * eb)
            pw.clamp_(min=0.05)
    return hist


class Batch:
    """A batch of fields for :func:`mitigate_batched`: the marshalled pointer,
    rank, extent and bound arrays, the outputs and the workspace, built once
    and reused across calls (so the library's cached CUDA graph is replayed)."""

    def __init__(self, qs, ebs, outs=None, workspace=None):
        self.qs = list(qs)
        n = len(self.qs)
        if n < 1 or len(ebs) != n:
            raise QAIError("need one eb per field")
        for q in self.qs:
            if not (q.is_cuda and q.dtype == torch.int32 and q.is_contiguous() and 1 <= q.dim() <= 3):
                raise QAIError("every field must be a contiguous CUDA int32 tensor of rank 1-3")
        self.outs = list(outs) if outs is not None else [
            torch.empty(q.shape, dtype=torch.float32, device=q.device) for q in self.qs]
        self.n = n
        self.q_ptrs = (ctypes.c_void_p * n)(*[q.data_ptr() for q in self.qs])
        self.out_ptrs = (ctypes.c_void_p * n)(*[o.data_ptr() for o in self.outs])
        self.ranks = (ctypes.c_int32 * n)(*[q.dim() for q in self.qs])
        dims = []
        for q in self.qs:
            d = list(q.shape) + [1] * (3 - q.dim())
            dims += d
        self.dims = (ctypes.c_int64 * (3 * n))(*dims)
        self.ebs = (ctypes.c_double * n)(*[float(e) for e in ebs])
        nb = ctypes.c_size_t()
        _check(load().qai_workspace_size_batched(n, self.ranks, self.dims, ctypes.byref(nb)))
        self.workspace = workspace if workspace is not None else alloc_workspace(nb.value, self.qs[0].device)

    def _args(self):
        return (self.n, self.q_ptrs, self.out_ptrs, self.ranks, self.dims, self.ebs)


def mitigate_batched(batch: Batch, stream=None, **kw):
    """Algorithm 4 on every field of ``batch`` in one call (persistent grouped
    launches over all fields, replayed from a cached CUDA graph). Returns
    ``batch.outs``."""
    p = _params(kw.get("eta", 0.9), kw.get("idw_power", 1.0), kw.get("grad_threshold", 2),
                kw.get("sign_rule", SIGN_SUM), kw.get("b2_rule", B2_SAME_Q))
    _check(load().qai_mitigate_batched(*batch._args(), ctypes.byref(p), batch.workspace.data_ptr(),
                                       batch.workspace.numel(), _stream(stream)))
    return batch.outs


def autotune_batched(batch: Batch, stream=None, **kw):
    """Time the candidates on ``batch`` and keep the fastest: for the grouped
    launches of the rank-2 and rank-3 fields the queue order, the points per
    work item and the column tiles; for rank 1 (and the per-field form) the
    stream count and field order. Returns {rank: {choice: value}}."""
    p = _params(kw.get("eta", 0.9), kw.get("idw_power", 1.0), kw.get("grad_threshold", 2),
                kw.get("sign_rule", SIGN_SUM), kw.get("b2_rule", B2_SAME_Q))
    ch = (BatchChoice * 3)()
    _check(load().qai_autotune_batched(*batch._args(), ctypes.byref(p), batch.workspace.data_ptr(),
                                       batch.workspace.numel(), _stream(stream), ch))
    return {c.rank: {"grouped": bool(c.grouped), "order": "largest first" if c.order else "as given",
                     "streams": c.streams, "ms": c.ms, "tile_w": c.tile_w, "rows_per_band": c.rows_per_band,
                     "points_per_block": c.points_per_block, "launches": c.launches}
            for c in ch if c.rank}


STATIC_MAX_POINTS = 2097152


def workspace_size_quality(shape, window: int = 7, stride: int = 2) -> int:
    n = ctypes.c_size_t()
    _check(load().qai_workspace_size_quality(len(shape), _dims(shape), int(window), int(stride),
                                             ctypes.byref(n)))
    return int(n.value)


def quality(x: torch.Tensor, y: torch.Tensor, window: int = 7, stride: int = 2, ssim_map: bool = False,
            workspace: torch.Tensor | None = None, stream=None):
    """PSNR (Eq. 4) and SSIM (Eq. 3 over sliding windows) of ``y`` against the
    original ``x`` on the GPU. Returns a dict (x_min, x_max, mse, psnr, ssim,
    windows), plus the per-window SSIM tensor under "map" when ``ssim_map``.
    Synchronises the stream to read the six numbers back."""
    lib = load()
    for t in (x, y):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise QAIError("x and y must be contiguous float32 CUDA tensors")
    if x.shape != y.shape:
        raise QAIError("x and y must have the same shape")
    shape = tuple(d for d in x.shape if d != 1) or (1,)   # the C ABI squeezes the same way
    if workspace is None:
        workspace = alloc_workspace(workspace_size_quality(shape, window, stride), x.device)
    res = torch.zeros(6, dtype=torch.float64, device=x.device)
    mp = None
    if ssim_map:
        counts = []
        for d in shape:
            m = min(window, d)
            counts.append((d - m) // stride + 1)
        mp = torch.empty(counts, dtype=torch.float32, device=x.device)
    st = _stream(stream)
    _check(lib.qai_quality(x.data_ptr(), y.data_ptr(), len(shape), _dims(shape), int(window), int(stride),
                           res.data_ptr(), mp.data_ptr() if mp is not None else None, workspace.data_ptr(),
                           workspace.numel(), st))
    vals = res.cpu()
    out = {"x_min": float(vals[0]), "x_max": float(vals[1]), "mse": float(vals[2]), "psnr": float(vals[3]),
           "ssim": float(vals[4]), "windows": int(vals[5:6].view(torch.int64)[0])}
    if mp is not None:
        out["map"] = mp
    return out


def mitigate_static(q: torch.Tensor, eb: float, out: torch.Tensor | None = None, stream=None, **kw):
    """Algorithm 4 without any device allocation by the library: for callers
    that cannot allocate device memory. Uses the scratch array compiled into
    libqai (fields up to STATIC_MAX_POINTS points); the first call on a device
    loads that array there, so make it before any region that must not
    allocate. Calls that overlap on the GPU race on that array, so keep them
    on one stream."""
    lib = load()
    if not (q.is_cuda and q.dtype == torch.int32 and q.is_contiguous()):
        raise QAIError("q must be a contiguous CUDA int32 tensor")
    shape = tuple(q.shape)
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=q.device)
    _check_out(out, shape, q.device)
    p = _params(kw.get("eta", 0.9), kw.get("idw_power", 1.0), kw.get("grad_threshold", 2),
                kw.get("sign_rule", SIGN_SUM), kw.get("b2_rule", B2_SAME_Q))
    with torch.cuda.device(q.device):
        _check(lib.qai_mitigate_static(q.data_ptr(), out.data_ptr(), len(shape), _dims(shape),
                                       float(eb), ctypes.byref(p), _stream(stream)))
    return out


def profile_enable(on: bool = True):
    _check(load().qai_profile_enable(1 if on else 0))


def profile_select(name: str | None = None):
    """Time only the kernels called ``name`` (None: all of them)."""
    _check(load().qai_profile_select(name.encode() if name else None))


def profile_read():
    """Per-kernel {name: (launches, total_ms, algo_bytes)} since the last read."""
    buf = (KernelStat * 64)()
    n = load().qai_profile_read(buf, 64)
    return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms, buf[i].algo_bytes)
            for i in range(n)}


def launch_count() -> int:
    return int(load().qai_launch_count())
