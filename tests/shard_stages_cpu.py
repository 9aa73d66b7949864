"""Host stand-ins for the sharded path's device work (test helper).

:class:`CpuStages` has the interface of ``sharded.CudaStages`` and does each
piece of work with the oracle: step A and GetBoundary(S) by the oracle's
Algorithms 2 and 3, the passes along the axes other than axis 0 by the
oracle's EDT on each plane (row), the last pass by an exhaustive minimum over
each line along axis 0 (smallest plane index on ties), step E by the oracle's
compensation. With them, the sharded orchestration (slabs, ghost planes,
bands, all-to-alls) runs on host tensors over gloo and must reproduce the
oracle's whole-field (exact) or per-slab (approximate) results bit for bit.

A word carries the squared distance d and the sign code c of the nearest site
as 4 d + c, c = S_B + 1 (0 where no site exists, d = INT32_MAX).
"""
import numpy as np
import torch

import oracle

INF32 = np.iinfo(np.int32).max


class CpuStages:
    out_dtype = torch.float64

    def __init__(self, eta=0.9, idw_power=1.0, grad_threshold=2, sign_rule=0, b2_rule=0):
        self.eta, self.idw_power = eta, idw_power
        self.grad_threshold, self.sign_rule, self.b2_rule = grad_threshold, sign_rule, b2_rule

    def empty(self, shape, dtype, like):
        return torch.empty(tuple(shape), dtype=dtype)

    def rows(self, phase, q_ext, s_ext, eqm_ext, ext):
        q = q_ext.numpy()
        if phase == 1:
            sites, sign = oracle.boundary_and_sign(q, self.grad_threshold, self.sign_rule)
        else:
            sites = oracle.boundary_of_s(q, s_ext.numpy(), self.grad_threshold, self.b2_rule)
            sign = np.zeros(q.shape, np.int8)
        words = np.empty(q.shape, np.int64)
        for z in range(q.shape[0]):
            d, idx = oracle.edt(sites[z])
            code = np.where(idx >= 0, sign[z].ravel()[np.clip(idx, 0, None)].reshape(idx.shape) + 1, 0)
            words[z] = d.astype(np.int64) * 4 + code
        return torch.zeros(1), torch.from_numpy(words)

    def lines(self, phase, words, band, dims, eb, q=None, dist1=None, s=None, count=None):
        L = band[0]
        w = words.numpy().reshape(L, -1)
        g, code = w >> 2, w & 3
        big = np.int64(1) << 62
        g = np.where(g >= INF32, big, g)
        z = np.arange(L, dtype=np.int64)
        tot = g[None, :, :] + ((z[:, None] - z[None, :]) ** 2)[:, :, None]
        arg = np.argmin(tot, axis=1)                        # first minimum: smallest plane
        dist = np.take_along_axis(tot, arg[:, None, :], 1)[:, 0, :]
        none = dist >= big
        dist = np.where(none, INF32, dist).astype(np.int32).reshape(band)
        if phase == 1:
            c = np.take_along_axis(code, arg, 0)
            sgn = np.where(none, 0, c - 1).astype(np.int8).reshape(band)
            return torch.from_numpy(dist), torch.from_numpy(sgn), torch.zeros(1)
        out = oracle.compensate(q.numpy(), dist1.numpy(), dist, s.numpy(), eb, self.eta, self.idw_power)
        return torch.from_numpy(out)

    def copy(self, dst, dst_off, dst_pitch, src, src_off, src_pitch, width, height):
        if width <= 0 or height <= 0:
            return
        d = dst.as_strided((height, width), (dst_pitch, 1), dst.storage_offset() + dst_off)
        s = src.as_strided((height, width), (src_pitch, 1), src.storage_offset() + src_off)
        d.copy_(s)

    def whole(self, q, eb):
        return torch.from_numpy(oracle.mitigate(q.numpy(), eb, eta=self.eta, idw_power=self.idw_power,
                                                grad_threshold=self.grad_threshold, sign_rule=self.sign_rule,
                                                b2_rule=self.b2_rule, debug=False)["out"])
