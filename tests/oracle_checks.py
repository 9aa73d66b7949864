"""Independent numpy re-statements used to pin the oracle (test helpers).

Each function states one step of the method directly from its definition in
the paper, written separately from ``oracle/qai_oracle.c`` (no shared code):

* :func:`brute_edt` -- Eq. 2 by exhaustive search, O(N * B): squared distance
  to the nearest site and, among the nearest, the smallest linear index (R5).
* :func:`boundary_and_sign` -- Algorithm 2 with numpy slicing.
* :func:`propagate_and_b2` -- Algorithm 3 (S = S_B[I1]) and GetBoundary(S).
* :func:`compensate` -- step E, C = w * S * eta * eps, by the R7 case split.
"""
import numpy as np

INF32 = np.iinfo(np.int32).max


def squeeze_shape(shape):
    kept = tuple(n for n in shape if n > 1)
    return kept if kept else (1,)


def brute_edt(sites):
    sites = np.asarray(sites, bool)
    shp = sites.shape
    pts = np.indices(shp).reshape(len(shp), -1).T.astype(np.int64)
    site_lin = np.flatnonzero(sites.ravel())          # increasing linear index
    if site_lin.size == 0:
        return np.full(shp, INF32, np.int32), np.full(shp, -1, np.int32)
    sp = pts[site_lin]
    d2 = ((pts[:, None, :] - sp[None, :, :]) ** 2).sum(-1)
    arg = np.argmin(d2, axis=1)                       # first minimum = smallest index
    dist = d2[np.arange(len(pts)), arg]
    return dist.reshape(shp).astype(np.int32), site_lin[arg].reshape(shp).astype(np.int32)


def _interior_mask(shp):
    m = np.ones(shp, bool)
    for a, n in enumerate(shp):
        idx = np.arange(n)
        ok = (idx >= 1) & (idx <= n - 2)
        view = [1] * len(shp)
        view[a] = n
        m &= ok.reshape(view)
    return m


def _shift(a, axis, k):
    """b[i] = a[i + k] along ``axis`` (wrapped; only read at interior points)."""
    return np.roll(a, -k, axis=axis)


def boundary_and_sign(q, grad_threshold=2, sign_rule=0):
    q0 = np.asarray(q, np.int64)
    shp = q0.shape
    q = q0.reshape(squeeze_shape(shp))
    inner = _interior_mask(q.shape)
    differs = np.zeros(q.shape, bool)
    total = np.zeros(q.shape, np.int64)
    first = np.zeros(q.shape, np.int64)
    fast = np.zeros(q.shape, bool)
    for a in range(q.ndim):
        lo, hi = _shift(q, a, -1), _shift(q, a, +1)
        for nb in (lo, hi):
            d = nb != q
            first = np.where((first == 0) & d, np.sign(nb - q), first)
            differs |= d
            total += nb - q
        fast |= np.abs(hi - lo) >= grad_threshold
    b1 = inner & differs
    sign = first if sign_rule == 1 else np.sign(total)
    sb = np.where(b1 & ~fast, sign, 0)
    return b1.astype(np.uint8).reshape(shp), sb.astype(np.int8).reshape(shp)


def propagate_and_b2(q, b1, sb, idx1, b2_rule=0):
    shp = np.shape(q)
    q = np.asarray(q, np.int64).reshape(squeeze_shape(shp))
    b1 = np.asarray(b1).reshape(q.shape)
    sb = np.asarray(sb, np.int64).reshape(q.shape)
    idx1 = np.asarray(idx1, np.int64).reshape(q.shape)
    flat = sb.ravel()
    prop = np.where(idx1 >= 0, flat[np.clip(idx1, 0, None)], 0)
    s = np.where(b1 == 1, sb, prop)
    b2 = np.zeros(q.shape, bool)
    for a in range(q.ndim):
        for k in (-1, 1):
            qn, sn = _shift(q, a, k), _shift(s, a, k)
            cand = sn != s
            if b2_rule == 0:
                cand &= qn == q
            b2 |= cand
    b2 &= _interior_mask(q.shape)
    return s.astype(np.int8).reshape(shp), b2.astype(np.uint8).reshape(shp)


def compensate(q, dist1, dist2, s, eb, eta=0.9, idw_power=1.0):
    d1 = np.asarray(dist1, np.float64)
    d2 = np.asarray(dist2, np.float64)
    k1, k2 = np.sqrt(d1), np.sqrt(d2)
    with np.errstate(divide="ignore", invalid="ignore"):
        w = k2 ** idw_power / (k1 ** idw_power + k2 ** idw_power)
    w = np.where(np.asarray(dist2) == INF32, 1.0, w)
    w = np.where(np.asarray(dist2) == 0, 0.0, w)
    w = np.where(np.asarray(dist1) == 0, 1.0, w)
    w = np.where(np.asarray(dist1) == INF32, 0.0, w)
    c = np.asarray(s, np.float64) * w * eta * eb
    return 2.0 * np.asarray(q, np.float64) * eb + c, c


def random_index_field(rng, shape, kind):
    """Small int32 index fields with the structures the method meets."""
    if kind == "smooth":
        grids = np.meshgrid(*[np.linspace(0, 1, n) for n in shape], indexing="ij")
        x = sum(rng.uniform(1, 4) * np.sin(rng.uniform(1, 6) * g + rng.uniform(0, 6)) for g in grids)
        return np.floor(x * rng.uniform(1, 3) + 0.5).astype(np.int32)
    if kind == "noisy":
        return rng.integers(-2, 3, size=shape).astype(np.int32)
    if kind == "sparse":
        q = np.zeros(shape, np.int32)
        q[rng.random(shape) < 0.03] = 1
        return q
    if kind == "constant":
        return np.full(shape, 7, np.int32)
    if kind == "checker":
        return (np.indices(shape).sum(0) % 2).astype(np.int32)
    if kind == "step":
        ax = len(shape) - 1
        idx = np.indices(shape)[ax]
        return (idx >= shape[ax] // 2).astype(np.int32)
    if kind == "extreme":
        q = rng.integers(-2, 3, size=shape).astype(np.int64) * (2 ** 30 - 1)
        return np.clip(q, -(2 ** 31) + 1, 2 ** 31 - 1).astype(np.int32)
    raise ValueError(kind)
