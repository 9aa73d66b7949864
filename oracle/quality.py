"""FP64 quality metrics of Sec. III-B: SSIM (Eq. 3) over sliding windows and
PSNR (Eq. 4), in plain numpy.

TEST INFRASTRUCTURE. Only ``tests/`` and ``bench.py``'s CPU legs may import
this module; the CUDA product path never does.

Readings of the paper (the same in the kernels):

* Q1 -- the constants c1 = 1e-4 and c2 = 9e-4 of Eq. 3 assume data in [0, 1],
  so both fields are normalised by the ORIGINAL field's range before SSIM:
  v' = (v - min D1) / (max D1 - min D1); a constant original (range 0) is not
  scaled (divisor 1).
* Q2 -- "sample variances" and "sample covariance": centred sums over the
  window's n points divided by n - 1 (the textbook sample estimators); n = 1
  gives zero variances.
* Q3 -- the sliding window: on each axis of extent d (extent-1 axes dropped,
  as in Algorithm 2's squeeze), the window spans m = min(window, d) points
  and starts at 0, stride, 2 stride, ... while it fits (start + m <= d); the
  dataset's SSIM is the plain mean over all window placements.
* Q4 -- Eq. 4 with MSE the mean of (D1 - D2)^2 over all points; identical
  fields (MSE = 0) give +inf.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.lib.stride_tricks import sliding_window_view

C1 = 1e-4
C2 = 9e-4


def _squeeze(a):
    a = np.asarray(a, np.float64)
    shape = tuple(d for d in a.shape if d != 1) or (1,)
    return a.reshape(shape)


def normalise(x, y):
    """Q1: both fields scaled by the range of the original ``x``."""
    x, y = _squeeze(x), _squeeze(y)
    lo, hi = float(x.min()), float(x.max())
    r = hi - lo if hi > lo else 1.0
    return (x - lo) / r, (y - lo) / r


def window_extent(shape, window):
    """Q3: window length on each axis."""
    return tuple(min(window, d) for d in shape)


def window_counts(shape, window=7, stride=2):
    m = window_extent(shape, window)
    return tuple((d - k) // stride + 1 for d, k in zip(shape, m))


def ssim_of_window(a, b):
    """Eq. 3 on the points of one window (any shape), FP64, two-pass."""
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    n = a.size
    mu_a, mu_b = a.mean(), b.mean()
    da, db = a - mu_a, b - mu_b
    den = max(n - 1, 1)                                    # Q2
    var_a, var_b, cov = (da @ da) / den, (db @ db) / den, (da @ db) / den
    return ((2 * mu_a * mu_b + C1) * (2 * cov + C2)) / ((mu_a ** 2 + mu_b ** 2 + C1) * (var_a + var_b + C2))


def ssim_map(x, y, window=7, stride=2):
    """Eq. 3 at every window placement of Q3 (array over window starts)."""
    xn, yn = normalise(x, y)
    m = window_extent(xn.shape, window)
    sl = tuple(slice(None, None, stride) for _ in m)
    wa = sliding_window_view(xn, m)[sl]
    wb = sliding_window_view(yn, m)[sl]
    axes = tuple(range(xn.ndim, 2 * xn.ndim))
    n = int(np.prod(m))
    mu_a = wa.mean(axis=axes)
    mu_b = wb.mean(axis=axes)
    expand = (Ellipsis,) + (None,) * xn.ndim
    da = wa - mu_a[expand]
    db = wb - mu_b[expand]
    den = max(n - 1, 1)
    var_a = (da * da).sum(axis=axes) / den
    var_b = (db * db).sum(axis=axes) / den
    cov = (da * db).sum(axis=axes) / den
    return ((2 * mu_a * mu_b + C1) * (2 * cov + C2)) / ((mu_a ** 2 + mu_b ** 2 + C1) * (var_a + var_b + C2))


def ssim_at(x, y, starts, window=7, stride=2):
    """Eq. 3 at the given window indices only (for fields too large to map)."""
    xn, yn = normalise(x, y)
    m = window_extent(xn.shape, window)
    out = []
    for w in starts:
        sl = tuple(slice(i * stride, i * stride + k) for i, k in zip(w, m))
        out.append(ssim_of_window(xn[sl], yn[sl]))
    return np.array(out)


def ssim(x, y, window=7, stride=2):
    """The dataset's SSIM: mean of Eq. 3 over all windows (Q3)."""
    return float(np.mean(ssim_map(x, y, window, stride)))


def mse(x, y):
    x, y = _squeeze(x), _squeeze(y)
    return float(np.mean((x - y) ** 2))


def psnr(x, y):
    """Eq. 4: 20 log10(range(D1) / sqrt(MSE)); +inf for identical fields (Q4)."""
    x = _squeeze(x)
    e = mse(x, y)
    if e == 0.0:
        return math.inf
    r = float(x.max() - x.min())
    return 20.0 * math.log10(r / math.sqrt(e)) if r > 0 else -math.inf
