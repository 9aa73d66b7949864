"""FP64 CPU oracle of quantization-aware interpolation (ctypes wrapper).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The CUDA product path (``paper_2602_20097_gb300``) never imports it and
shares no code with it; the C source ``qai_oracle.c`` states the algorithm and
every reading of the paper that it takes (rules R1-R8).

Functions (numpy in, numpy out):

* :func:`mitigate` -- Algorithm 4 end to end, with every intermediate of
  steps A-E (``b1, sb, dist1, idx1, s, b2, dist2, comp``) and ``out`` = D''.
* :func:`edt` -- exact squared EDT with the nearest-site linear index
  (Algorithm 1 along x, then y, then z).
* :func:`boundary_and_sign` -- Algorithm 2 alone.
* :func:`grad_params` -- adjoint of step E with respect to eta and the IDW
  exponent p, the EDT assignment held fixed (no counterpart in the paper).
* :func:`boundary_of_s` -- GetBoundary(S) of Algorithm 3 for a given S.
* :func:`compensate` -- step E alone on given distances and S.
* :func:`mitigate_approx` -- Section VII-B's approximate parallelization:
  ghost planes for step A and for GetBoundary(S), both EDTs inside each slab.
* :func:`mitigate_independent` -- Section VII-B's embarrassingly parallel
  strategy: Algorithm 4 on each slab alone.
* :func:`slab_bounds` -- the slab partition both sharded strategies use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qai_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libqai_oracle.so")
_lock = threading.Lock()
_lib = None

SIGN_SUM, SIGN_FIRST = 0, 1
B2_SAME_Q, B2_LITERAL = 0, 1
INF32 = np.iinfo(np.int32).max


class _Params(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_double), ("idw_power", ctypes.c_double),
                ("grad_threshold", ctypes.c_int32), ("sign_rule", ctypes.c_int32),
                ("b2_rule", ctypes.c_int32), ("flags", ctypes.c_uint32)]


def build(force: bool = False) -> str:
    """Compile ``libqai_oracle.so`` with gcc (OpenMP over independent lines)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(_LIBDIR, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        # QAI_ORACLE_LIB lets the mutation tests load a deliberately broken copy.
        lib = ctypes.CDLL(os.environ.get("QAI_ORACLE_LIB") or build())
        P = ctypes.c_void_p
        lib.qai_oracle_mitigate.argtypes = [P, ctypes.c_int, P, ctypes.c_double,
                                            ctypes.POINTER(_Params)] + [P] * 9
        lib.qai_oracle_mitigate.restype = ctypes.c_int
        lib.qai_oracle_edt.argtypes = [P, ctypes.c_int, P, P, P]
        lib.qai_oracle_edt.restype = ctypes.c_int
        lib.qai_oracle_boundary_and_sign.argtypes = [P, ctypes.c_int, P,
                                                     ctypes.POINTER(_Params), P, P]
        lib.qai_oracle_boundary_and_sign.restype = None
        lib.qai_oracle_threads.restype = ctypes.c_int
        lib.qai_oracle_set_threads.argtypes = [ctypes.c_int]
        lib.qai_oracle_set_threads.restype = None
        lib.qai_oracle_grad_params.argtypes = [P, ctypes.c_int, P, ctypes.c_double,
                                               ctypes.POINTER(_Params), P, P]
        lib.qai_oracle_boundary_of_s.argtypes = [P, P, ctypes.c_int, P, ctypes.POINTER(_Params), P]
        lib.qai_oracle_boundary_of_s.restype = ctypes.c_int
        lib.qai_oracle_compensate.argtypes = [P, P, P, P, ctypes.c_int64, ctypes.c_double,
                                              ctypes.POINTER(_Params), P]
        lib.qai_oracle_compensate.restype = ctypes.c_int
        lib.qai_oracle_mitigate_approx.argtypes = [P, ctypes.c_int, P, ctypes.c_double,
                                                   ctypes.POINTER(_Params), ctypes.c_int] + [P] * 6
        lib.qai_oracle_mitigate_approx.restype = ctypes.c_int
        lib.qai_oracle_grad_params.restype = ctypes.c_int
        _lib = lib
    return _lib


def threads() -> int:
    """OpenMP threads the oracle uses (``OMP_NUM_THREADS`` or all cores)."""
    return int(_load().qai_oracle_threads())


def set_threads(n: int) -> None:
    """Use ``n`` OpenMP threads from now on (timing only; results do not
    depend on it)."""
    _load().qai_oracle_set_threads(int(n))


def _params(eta, idw_power, grad_threshold, sign_rule, b2_rule):
    return _Params(float(eta), float(idw_power), int(grad_threshold),
                   int(sign_rule), int(b2_rule), 0)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _dims(shape):
    return np.ascontiguousarray(shape, dtype=np.int64)


def mitigate(q, eb, eta=0.9, idw_power=1.0, grad_threshold=2,
             sign_rule=SIGN_SUM, b2_rule=B2_SAME_Q, debug=True):
    """Algorithm 4 on an int32 index field ``q`` (1-3 dims, C order).

    Returns a dict with ``out`` (D'', float64) and, when ``debug``, the
    intermediates ``b1, sb, dist1, idx1, s, b2, dist2, comp`` (same shape).
    Distances are squared, INF = INT32_MAX; ``idx1`` is a linear index, -1 if
    the field has no boundary point.
    """
    q = np.ascontiguousarray(q, dtype=np.int32)
    if q.ndim < 1 or q.ndim > 3:
        raise ValueError("rank must be 1..3")
    shp = q.shape
    res = {"out": np.empty(shp, np.float64)}
    if debug:
        res.update(b1=np.empty(shp, np.uint8), sb=np.empty(shp, np.int8),
                   dist1=np.empty(shp, np.int32), idx1=np.empty(shp, np.int32),
                   s=np.empty(shp, np.int8), b2=np.empty(shp, np.uint8),
                   dist2=np.empty(shp, np.int32), comp=np.empty(shp, np.float64))
    p = _params(eta, idw_power, grad_threshold, sign_rule, b2_rule)
    g = res.get
    rc = _load().qai_oracle_mitigate(
        _ptr(q), q.ndim, _ptr(_dims(shp)), float(eb), ctypes.byref(p), _ptr(res["out"]),
        _ptr(g("b1")), _ptr(g("sb")), _ptr(g("dist1")), _ptr(g("idx1")), _ptr(g("s")),
        _ptr(g("b2")), _ptr(g("dist2")), _ptr(g("comp")))
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments (rc={rc})")
    return res


def grad_params(q, eb, grad_out, eta=0.9, idw_power=1.0, grad_threshold=2,
                sign_rule=SIGN_SUM, b2_rule=B2_SAME_Q):
    """Adjoint of step E with the EDT assignment fixed: (dL/deta, dL/dp) for
    dL/dD'' = grad_out (FP64). dL/dD' is grad_out itself."""
    q = np.ascontiguousarray(q, dtype=np.int32)
    g = np.ascontiguousarray(grad_out, dtype=np.float64)
    if g.shape != q.shape:
        raise ValueError("grad_out must have q's shape")
    out = np.zeros(2, np.float64)
    p = _params(eta, idw_power, grad_threshold, sign_rule, b2_rule)
    rc = _load().qai_oracle_grad_params(_ptr(q), q.ndim, _ptr(_dims(q.shape)), float(eb),
                                        ctypes.byref(p), _ptr(g), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments (rc={rc})")
    return float(out[0]), float(out[1])


def edt(sites):
    """Exact squared EDT of a boolean site map, with nearest-site linear index."""
    s = np.ascontiguousarray(sites, dtype=np.uint8)
    dist = np.empty(s.shape, np.int32)
    idx = np.empty(s.shape, np.int32)
    rc = _load().qai_oracle_edt(_ptr(s), s.ndim, _ptr(_dims(s.shape)), _ptr(dist), _ptr(idx))
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments (rc={rc})")
    return dist, idx


def boundary_and_sign(q, grad_threshold=2, sign_rule=SIGN_SUM):
    """Algorithm 2 alone: (B1 uint8, S_B int8)."""
    q = np.ascontiguousarray(q, dtype=np.int32)
    b = np.empty(q.shape, np.uint8)
    s = np.empty(q.shape, np.int8)
    p = _params(0.9, 1.0, grad_threshold, sign_rule, 0)
    _load().qai_oracle_boundary_and_sign(_ptr(q), q.ndim, _ptr(_dims(q.shape)),
                                         ctypes.byref(p), _ptr(b), _ptr(s))
    return b, s


def boundary_of_s(q, s, grad_threshold=2, b2_rule=B2_SAME_Q):
    """GetBoundary(S) (second half of Algorithm 3) on interior points: uint8 B2."""
    q = np.ascontiguousarray(q, dtype=np.int32)
    s = np.ascontiguousarray(s, dtype=np.int8)
    if s.shape != q.shape:
        raise ValueError("s must have q's shape")
    b2 = np.empty(q.shape, np.uint8)
    p = _params(0.9, 1.0, grad_threshold, SIGN_SUM, b2_rule)
    rc = _load().qai_oracle_boundary_of_s(_ptr(q), _ptr(s), q.ndim, _ptr(_dims(q.shape)),
                                          ctypes.byref(p), _ptr(b2))
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments (rc={rc})")
    return b2


def compensate(q, dist1, dist2, s, eb, eta=0.9, idw_power=1.0):
    """Step E alone: D'' = 2 q eps + S w eta eps (float64), distances squared
    with INT32_MAX for INF."""
    q = np.ascontiguousarray(q, dtype=np.int32)
    d1 = np.ascontiguousarray(dist1, dtype=np.int32)
    d2 = np.ascontiguousarray(dist2, dtype=np.int32)
    s = np.ascontiguousarray(s, dtype=np.int8)
    if not (q.shape == d1.shape == d2.shape == s.shape):
        raise ValueError("q, dist1, dist2 and s must share a shape")
    out = np.empty(q.shape, np.float64)
    p = _params(eta, idw_power, 2, SIGN_SUM, B2_SAME_Q)
    rc = _load().qai_oracle_compensate(_ptr(q), _ptr(d1), _ptr(d2), _ptr(s), ctypes.c_int64(q.size),
                                       float(eb), ctypes.byref(p), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments (rc={rc})")
    return out


def slab_bounds(n0, nparts):
    """Planes [b, e) of each of the nparts slabs of an axis of extent n0."""
    return [(k * n0 // nparts, (k + 1) * n0 // nparts) for k in range(nparts)]


def _squeezed(shape):
    kept = tuple(n for n in shape if n > 1)
    return kept or (1,)


def mitigate_approx(q, eb, nparts, eta=0.9, idw_power=1.0, grad_threshold=2,
                    sign_rule=SIGN_SUM, b2_rule=B2_SAME_Q):
    """Section VII-B's approximate parallelization over ``nparts`` slabs of the
    slowest axis (after squeezing extent-1 axes; rank 2 or 3). Returns
    ``out, dist1, idx1 (whole-field index), s, b2, dist2``."""
    q = np.ascontiguousarray(q, dtype=np.int32)
    shp = q.shape
    res = {"out": np.empty(shp, np.float64), "dist1": np.empty(shp, np.int32),
           "idx1": np.empty(shp, np.int32), "s": np.empty(shp, np.int8),
           "b2": np.empty(shp, np.uint8), "dist2": np.empty(shp, np.int32)}
    p = _params(eta, idw_power, grad_threshold, sign_rule, b2_rule)
    rc = _load().qai_oracle_mitigate_approx(
        _ptr(q), q.ndim, _ptr(_dims(shp)), float(eb), ctypes.byref(p), int(nparts), _ptr(res["out"]),
        _ptr(res["dist1"]), _ptr(res["idx1"]), _ptr(res["s"]), _ptr(res["b2"]), _ptr(res["dist2"]))
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments (rc={rc})")
    return res


def mitigate_independent(q, eb, nparts, **kw):
    """Section VII-B's embarrassingly parallel strategy: Algorithm 4 on each of
    the ``nparts`` slabs of the slowest axis alone. Returns D'' (float64)."""
    q = np.ascontiguousarray(q, dtype=np.int32)
    sq = q.reshape(_squeezed(q.shape))
    out = np.empty(sq.shape, np.float64)
    for b, e in slab_bounds(sq.shape[0], nparts):
        out[b:e] = mitigate(sq[b:e], eb, debug=False, **kw)["out"]
    return out.reshape(q.shape)
