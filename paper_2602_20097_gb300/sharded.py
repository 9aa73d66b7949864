"""Sharded forms of the method over several processes (Section VII-B).

A rank-2 or rank-3 field (every extent >= 2) is cut along axis 0 (z of a 3-D
field, y of a 2-D one) into one slab per process: slab k holds the planes
``[floor(k n0 / P), floor((k + 1) n0 / P))`` (:func:`slab_bounds`). A process
holds its slab of q and gets back its slab of D''. The three strategies of the
paper:

``exact`` (sequentially compliant)
    D'' equals the one-process result bit for bit. Each process runs step A
    and the EDT passes along the other axes on its slab extended by one ghost
    plane per side; an all-to-all re-cuts the data into bands (every line along
    axis 0 through a range of axis-1 indices) for the last EDT pass; S comes
    back to the slabs for GetBoundary(S); the second EDT repeats the pattern,
    with step E fused into its last pass on the bands; D'' comes back. Four
    all-to-alls and one ghost exchange, no chain of processes waiting on each
    other (the paper's exact form passes the EDT along the column process by
    process).
``approximate`` (local communication)
    Ghost planes of q before step A and of S before GetBoundary(S); both EDTs
    stay inside the slab, so a point whose nearest boundary lies in another
    slab gets a different Dist1, S or Dist2 than the whole-field method.
``independent`` (embarrassingly parallel)
    Algorithm 4 on each slab alone, no communication.

The exchanges go through a :class:`Comm` (``torch.distributed``
all_to_all_single: NCCL between GPUs, gloo between hosts); every piece of
device work is a C-ABI call (``qai_shard_rows``, ``qai_shard_lines``,
``qai_shard_copy``, ``qai_mitigate``) made by :class:`CudaStages`. Nothing
here computes a step of the method.
"""
from __future__ import annotations

import ctypes
import threading
from typing import Optional, Sequence

import torch
import torch.distributed as dist

from . import qai

STRATEGIES = ("exact", "approximate", "independent")


def slab_bounds(n0: int, nparts: int):
    """Planes ``[b, e)`` of each of the ``nparts`` slabs of an axis of extent ``n0``."""
    return [(k * n0 // nparts, (k + 1) * n0 // nparts) for k in range(nparts)]


# ---- exchanges ----------------------------------------------------------------

class Comm:
    """An all-to-all of byte buffers among ``size`` processes: ``send`` is the
    concatenation of the blocks for ranks 0..size-1 (``send_counts`` bytes
    each); returns the concatenation of the blocks from ranks 0..size-1
    (``recv_counts`` bytes each)."""

    rank: int
    size: int

    def alltoall(self, send: torch.Tensor, send_counts: Sequence[int], recv_counts: Sequence[int]) -> torch.Tensor:
        raise NotImplementedError


class TorchComm(Comm):
    """``torch.distributed.all_to_all_single`` on a process group (NCCL for
    CUDA tensors, gloo for host tensors)."""

    def __init__(self, group=None):
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def alltoall(self, send, send_counts, recv_counts):
        out = torch.empty(int(sum(recv_counts)), dtype=torch.uint8, device=send.device)
        dist.all_to_all_single(out, send, list(map(int, recv_counts)), list(map(int, send_counts)),
                               group=self.group)
        return out


class HostCopyComm(TorchComm):
    """:class:`TorchComm` on a host backend (gloo) for device buffers: every
    all-to-all goes through host copies."""

    def alltoall(self, send, send_counts, recv_counts):
        return super().alltoall(send.cpu(), send_counts, recv_counts).to(send.device)


class LoopbackHub:
    """In-process stand-in for a process group: ``size`` host threads, one
    per emulated process, exchange through shared slots (test harness for one
    device; the threads' launches share one stream, so no kernel waits on
    another)."""

    def __init__(self, size: int, timeout: float = 300.0):
        self.size = size
        self.slots = [None] * size
        self.barrier = threading.Barrier(size, timeout=timeout)

    def comm(self, rank: int) -> Comm:
        return _LoopbackComm(self, rank)


class _LoopbackComm(Comm):
    def __init__(self, hub: LoopbackHub, rank: int):
        self.hub, self.rank, self.size = hub, rank, hub.size

    def alltoall(self, send, send_counts, recv_counts):
        hub = self.hub
        offs = [0]
        for c in send_counts:
            offs.append(offs[-1] + int(c))
        hub.slots[self.rank] = (send, offs)
        hub.barrier.wait()
        parts = []
        for src in range(self.size):
            buf, so = hub.slots[src]
            parts.append(buf[so[self.rank]:so[self.rank + 1]])
        for p, n in zip(parts, recv_counts):
            if p.numel() != int(n):
                raise RuntimeError("all-to-all sizes disagree between ranks")
        out = torch.cat(parts) if parts else torch.empty(0, dtype=torch.uint8, device=send.device)
        hub.barrier.wait()
        return out


# ---- device work ----------------------------------------------------------------

def _ptr(t: Optional[torch.Tensor], byte_offset: int = 0):
    return ctypes.c_void_p(t.data_ptr() + byte_offset) if t is not None else None


class CudaStages:
    """Each process's device work, through the C ABI (no arithmetic of the
    method in Python)."""

    out_dtype = torch.float32

    def __init__(self, params: "qai.Params"):
        self.params = params
        self.lib = qai.load()

    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def word_dtype(self, rank: int):
        return torch.int32 if rank == 3 else torch.int16

    def empty(self, shape, dtype, like):
        return torch.empty(tuple(shape), dtype=dtype, device=like.device)

    def rows(self, phase, q_ext, s_ext, eqm_ext, ext):
        """Row work on an extended slab; returns (eqm, words)."""
        rank = len(ext)
        ws = ctypes.c_size_t()
        wb = ctypes.c_int()
        qai._check(self.lib.qai_shard_sizes(rank, qai._dims(ext), ctypes.byref(ws), ctypes.byref(wb)))
        if eqm_ext is None:
            eqm_ext = self.empty(ext, torch.uint8, q_ext)
        words = self.empty(ext, self.word_dtype(rank), q_ext)
        scratch = torch.empty(max(int(ws.value), 1), dtype=torch.uint8, device=q_ext.device)
        qai._check(self.lib.qai_shard_rows(phase, rank, qai._dims(ext), _ptr(q_ext), _ptr(s_ext), _ptr(eqm_ext),
                                           _ptr(words), _ptr(scratch), ws.value, ctypes.byref(self.params),
                                           self._stream()))
        return eqm_ext, words

    def lines(self, phase, words, band, dims, eb, q=None, dist1=None, s=None, count=None):
        """Phase 1: (dist1, s, count) of the band; phase 2: D'' of the band."""
        rank = len(band)
        if phase == 1:
            dist1 = self.empty(band, torch.int32, words)
            s = self.empty(band, torch.int8, words)
            count = self.empty((band[1:]), torch.int16, words)
            out = None
        else:
            out = self.empty(band, torch.float32, words)
        qai._check(self.lib.qai_shard_lines(phase, rank, qai._dims(band), qai._dims(dims), _ptr(words), _ptr(q),
                                            _ptr(dist1), _ptr(s), _ptr(count), _ptr(out), float(eb),
                                            ctypes.byref(self.params), self._stream()))
        return (dist1, s, count) if phase == 1 else out

    def copy(self, dst, dst_off, dst_pitch, src, src_off, src_pitch, width, height):
        """``height`` runs of ``width`` bytes between flat uint8 tensors."""
        if width <= 0 or height <= 0:
            return
        qai._check(self.lib.qai_shard_copy(_ptr(dst, dst_off), int(dst_pitch), _ptr(src, src_off), int(src_pitch),
                                           int(width), int(height), self._stream()))

    def whole(self, q, eb):
        """Algorithm 4 on a slab alone (the independent strategy)."""
        out = torch.empty(q.shape, dtype=torch.float32, device=q.device)
        qai._check(self.lib.qai_mitigate(_ptr(q), _ptr(out), q.dim(), qai._dims(tuple(q.shape)), float(eb),
                                         ctypes.byref(self.params), None, 0, self._stream(), None))
        return out


# ---- one process's part ------------------------------------------------------------

def _bytes(t: torch.Tensor) -> torch.Tensor:
    if not t.is_contiguous():
        raise ValueError("exchange buffers must be contiguous")
    return t.view(-1).view(torch.uint8)


class _Plan:
    """Slab and band partition of a field for ``P`` processes (rank r)."""

    def __init__(self, dims, P, r, ghosts=True):
        self.dims = tuple(int(d) for d in dims)
        self.rank = len(self.dims)
        self.n0, self.n1 = self.dims[0], self.dims[1]
        self.inner = self.dims[2] if self.rank == 3 else 1
        self.P, self.r = P, r
        self.slabs = slab_bounds(self.n0, P)
        self.bands = slab_bounds(self.n1, P)
        g = 1 if ghosts else 0
        self.lo = [g if b > 0 else 0 for b, _ in self.slabs]
        self.hi = [g if e < self.n0 else 0 for _, e in self.slabs]

    def own(self, k):
        b, e = self.slabs[k]
        return e - b

    def ext_planes(self, k):
        return self.own(k) + self.lo[k] + self.hi[k]

    def ext_shape(self, k):
        return (self.ext_planes(k),) + self.dims[1:]

    def band_width(self, k):
        c0, c1 = self.bands[k]
        return c1 - c0

    def band_shape(self, k):
        return (self.n0, self.band_width(k)) + self.dims[2:]


def _ghost_exchange(stages, comm, plan, x_ext):
    """Fills the ghost planes of ``x_ext`` (an extended slab) from the
    neighbours' own edge planes."""
    r, P = plan.r, plan.P
    pb = plan.n1 * plan.inner * x_ext.element_size()
    flat = _bytes(x_ext)
    lo, own = plan.lo[r], plan.own(r)
    sc = [0] * P
    rc = [0] * P
    parts = []
    if r > 0:
        sc[r - 1] = pb
        parts.append(flat[lo * pb:(lo + 1) * pb])
    if r + 1 < P:
        sc[r + 1] = pb
        parts.append(flat[(lo + own - 1) * pb:(lo + own) * pb])
    if plan.lo[r]:
        rc[r - 1] = pb
    if plan.hi[r]:
        rc[r + 1] = pb
    send = torch.cat(parts) if parts else flat[:0]
    recv = comm.alltoall(send, sc, rc)
    at = 0
    if plan.lo[r]:
        stages.copy(flat, 0, pb, recv, at, pb, pb, 1)
        at += pb
    if plan.hi[r]:
        stages.copy(flat, (lo + own) * pb, pb, recv, at, pb, pb, 1)
    return x_ext


def _with_ghosts(stages, comm, plan, x_own):
    """The extended slab of ``x_own`` (own planes), ghosts from the neighbours."""
    r = plan.r
    ext = stages.empty(plan.ext_shape(r), x_own.dtype, x_own)
    pb = plan.n1 * plan.inner * x_own.element_size()
    stages.copy(_bytes(ext), plan.lo[r] * pb, pb, _bytes(x_own), 0, pb, pb, plan.own(r))
    return _ghost_exchange(stages, comm, plan, ext)


def _to_bands(stages, comm, plan, x, first_plane):
    """All-to-all from slabs to bands: ``x`` holds this process's slab starting
    at plane ``first_plane`` of its array; returns this process's band
    (n0 x width x inner) in x's dtype."""
    r, P = plan.r, plan.P
    isz = x.element_size()
    row = plan.inner * isz
    src = _bytes(x)
    own = plan.own(r)
    src0 = first_plane * plan.n1 * row
    send = torch.empty(own * plan.n1 * row, dtype=torch.uint8, device=x.device)
    sc, at = [], 0
    for j in range(P):
        c0, _ = plan.bands[j]
        w = plan.band_width(j) * row
        stages.copy(send, at, w, src, src0 + c0 * row, plan.n1 * row, w, own)
        sc.append(own * w)
        at += own * w
    rc = [plan.own(k) * plan.band_width(r) * row for k in range(P)]
    recv = comm.alltoall(send, sc, rc)
    return recv.view(x.dtype).view(plan.band_shape(r))


def _from_bands(stages, comm, plan, xb, ghosts):
    """All-to-all from bands back to slabs: returns this process's slab of
    ``xb``'s field, extended by its ghost planes when ``ghosts``."""
    r, P = plan.r, plan.P
    isz = xb.element_size()
    row = plan.inner * isz
    src = _bytes(xb)
    wr = plan.band_width(r) * row

    def planes(k):
        b, e = plan.slabs[k]
        return (b - plan.lo[k], e + plan.hi[k]) if ghosts else (b, e)

    sc = [(planes(j)[1] - planes(j)[0]) * wr for j in range(P)]
    send = torch.empty(sum(sc), dtype=torch.uint8, device=xb.device)
    at = 0
    for j in range(P):
        pb, pe = planes(j)
        stages.copy(send, at, wr, src, pb * wr, wr, wr, pe - pb)
        at += sc[j]
    mb, me = planes(r)
    n = me - mb
    rc = [n * plan.band_width(k) * row for k in range(P)]
    recv = comm.alltoall(send, sc, rc)
    shape = (n,) + plan.dims[1:]
    out = stages.empty(shape, xb.dtype, xb)
    dst = _bytes(out)
    at = 0
    for k in range(P):
        c0, _ = plan.bands[k]
        w = plan.band_width(k) * row
        stages.copy(dst, c0 * row, plan.n1 * row, recv, at, w, w, n)
        at += rc[k]
    return out


def run_rank(stages, comm: Comm, q_own: torch.Tensor, dims, eb: float, strategy: str = "exact"):
    """This process's part of a sharded call: ``q_own`` is its slab of q
    (planes of :func:`slab_bounds` for rank ``comm.rank``); returns its slab of
    D''. Every process of ``comm`` must call it with the same dims, eb and
    strategy."""
    if strategy not in STRATEGIES:
        raise ValueError(f"strategy must be one of {STRATEGIES}")
    dims = tuple(int(d) for d in dims)
    if len(dims) not in (2, 3) or min(dims) < 2:
        raise ValueError("sharded calls take rank-2 or rank-3 fields with every extent >= 2")
    P, r = comm.size, comm.rank
    if not 1 <= P <= dims[0]:
        raise ValueError(f"{P} processes need at least {P} planes along axis 0")
    plan = _Plan(dims, P, r, ghosts=strategy != "independent")
    if tuple(q_own.shape) != (plan.own(r),) + dims[1:]:
        raise ValueError(f"rank {r} holds planes {plan.slabs[r]}: q_own must have shape "
                         f"{(plan.own(r),) + dims[1:]}")
    q_own = q_own.contiguous()
    if strategy == "independent":
        return stages.whole(q_own, eb)

    lo, own = plan.lo[r], plan.own(r)
    ext = plan.ext_shape(r)
    q_ext = _with_ghosts(stages, comm, plan, q_own)
    eqm, w1 = stages.rows(1, q_ext, None, None, ext)
    if strategy == "approximate":
        # both EDTs inside the extended slab: its ghost planes hold no site
        # (they are the extended slab's own edge planes)
        d1, s_ext, cnt = stages.lines(1, w1, ext, dims, eb)
        _ghost_exchange(stages, comm, plan, s_ext)        # the neighbours' S
        _, w2 = stages.rows(2, q_ext, s_ext, eqm, ext)
        out = stages.lines(2, w2, ext, dims, eb, q=q_ext, dist1=d1, s=s_ext, count=cnt)
        return out[lo:lo + own]

    band = plan.band_shape(r)
    empty_band = plan.band_width(r) == 0
    w1_b = _to_bands(stages, comm, plan, w1, lo)
    q_b = _to_bands(stages, comm, plan, q_own, 0)
    if empty_band:
        d1_b = stages.empty(band, torch.int32, q_own)
        s_b = stages.empty(band, torch.int8, q_own)
        cnt_b = None
    else:
        d1_b, s_b, cnt_b = stages.lines(1, w1_b, band, dims, eb)
    s_ext = _from_bands(stages, comm, plan, s_b, ghosts=True)
    _, w2 = stages.rows(2, q_ext, s_ext, eqm, ext)
    w2_b = _to_bands(stages, comm, plan, w2, lo)
    if empty_band:
        out_b = stages.empty(band, stages.out_dtype, q_own)
    else:
        out_b = stages.lines(2, w2_b, band, dims, eb, q=q_b, dist1=d1_b, s=s_b, count=cnt_b)
    return _from_bands(stages, comm, plan, out_b, ghosts=False)


def mitigate(q_own: torch.Tensor, dims, eb: float, strategy: str = "exact", comm: Optional[Comm] = None,
             eta: float = 0.9, idw_power: float = 1.0, grad_threshold: int = 2, sign_rule: int = qai.SIGN_SUM,
             b2_rule: int = qai.B2_SAME_Q) -> torch.Tensor:
    """Sharded Algorithm 4 (Section VII-B) on CUDA tensors: this process's slab
    of q in, its slab of D'' (float32) out. ``comm`` defaults to the default
    process group (NCCL). See the module docstring for the strategies."""
    if not q_own.is_cuda or q_own.dtype != torch.int32:
        raise qai.QAIError("q_own must be a CUDA int32 tensor")
    if comm is None:
        comm = TorchComm()
    p = qai.Params(float(eta), float(idw_power), int(grad_threshold), int(sign_rule), int(b2_rule), 0)
    with torch.cuda.device(q_own.device):
        return run_rank(CudaStages(p), comm, q_own, dims, eb, strategy)
