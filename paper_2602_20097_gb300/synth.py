"""Seeded synthetic fields and the pre-quantizer that turns them into inputs.

This module holds no step of the mitigation method: it makes the inputs that
both the CUDA path and the CPU oracle consume. Fields stand in for the paper's
datasets (Table I), which are not available here:

* :func:`sinusoids` -- sum of 8 seeded 3-D plane waves plus N(0, 0.01^2) noise.
* :func:`grf` -- Gaussian random field with isotropic power spectrum
  P(k) ~ k^-slope, normalised to [0, 1] (slope 11/3 for turbulence-like NYX /
  JHTDB stand-ins, 3 for smooth climate / weather stand-ins).
* :func:`grf_front` -- 0.5 * GRF(k^-3) + 0.5 * a tanh front of width 5 cells
  across a seeded random plane through the centre, renormalised to [0, 1].
* :func:`batch_specs` -- shapes, spectra and error bounds of the 96-field mixed
  batch.
* :func:`quantize` -- Eq. 1 pre-quantization q = round(x / 2 eb), rounding half
  up, in FP64; ``eb`` is absolute.

Everything is seeded; large fields are synthesised with ``torch.fft`` on the
device the caller names, so the same call gives the same field on that device.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def _rng(seed):
    return np.random.default_rng(seed)


def sinusoids(shape=(64, 64, 64), seed=1, noise_std=0.01, n_waves=8):
    """Sum of ``n_waves`` plane waves with integer frequencies 1-4 per axis,
    amplitudes U(0.5, 1), phases U(0, 2 pi), plus Gaussian noise (float32)."""
    rng = _rng(seed)
    nd = len(shape)
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) / n for n in shape], indexing="ij")
    x = np.zeros(shape, np.float64)
    for _ in range(n_waves):
        f = rng.integers(1, 5, size=nd)
        amp = rng.uniform(0.5, 1.0)
        phase = rng.uniform(0.0, 2.0 * math.pi)
        arg = sum(float(f[a]) * grids[a] for a in range(nd))
        x += amp * np.sin(2.0 * math.pi * arg + phase)
    x += rng.normal(0.0, noise_std, size=shape)
    return x.astype(np.float32)


def _normalise01(t):
    lo, hi = t.min(), t.max()
    return (t - lo) / (hi - lo)


def grf(shape, slope=11.0 / 3.0, seed=2, device="cpu"):
    """Gaussian random field, P(k) ~ |k|^-slope, DC removed, in [0, 1].

    White N(0,1) noise from a seeded torch generator on ``device`` is filtered
    in Fourier space by |k|^(-slope/2). Returns a float32 torch tensor.
    """
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    white = torch.randn(tuple(shape), generator=gen, device=device, dtype=torch.float32)
    spec = torch.fft.rfftn(white)
    del white
    k2 = None
    for a, n in enumerate(shape):
        if a == len(shape) - 1:
            f = torch.fft.rfftfreq(n, device=device)
        else:
            f = torch.fft.fftfreq(n, device=device)
        view = [1] * len(shape)
        view[a] = -1
        f2 = (f * f).reshape(view)
        k2 = f2 if k2 is None else k2 + f2
    amp = torch.where(k2 > 0, k2.clamp_min(1e-30) ** (-slope / 4.0), torch.zeros_like(k2))
    spec *= amp
    del amp, k2
    field = torch.fft.irfftn(spec, s=tuple(shape))
    del spec
    return _normalise01(field).to(torch.float32)


def grf_front(shape, seed=3, device="cpu", width=5.0):
    """Smooth k^-3 GRF plus a seeded tanh front (sharp gradients), in [0, 1]."""
    base = grf(shape, slope=3.0, seed=seed, device=device)
    rng = _rng(seed + 7919)
    nrm = rng.normal(size=len(shape))
    nrm /= np.linalg.norm(nrm)
    s = torch.zeros(tuple(shape), device=device, dtype=torch.float32)
    for a, n in enumerate(shape):
        view = [1] * len(shape)
        view[a] = -1
        c = (torch.arange(n, device=device, dtype=torch.float32) - (n - 1) / 2.0) * float(nrm[a])
        s = s + c.reshape(view)
    front = 0.5 * (1.0 + torch.tanh(s / width))
    return _normalise01(0.5 * base + 0.5 * front).to(torch.float32)


def batch_specs(n=96, seed=4242):
    """The mixed batch: even i are 2-D (ny ~ logU[256,1800], nx ~ logU[256,3600]),
    odd i are 3-D (nz ~ logU[64,256], ny, nx ~ logU[64,384]); spectrum k^-3
    when i % 4 < 2 else k^-11/3; relative eb = 10^U(-4,-2); seed 1000 + i."""
    rng = _rng(seed)

    def logu(lo, hi):
        return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))

    specs = []
    for i in range(n):
        if i % 2 == 0:
            shape = (logu(256, 1800), logu(256, 3600))
        else:
            shape = (logu(64, 256), logu(64, 384), logu(64, 384))
        slope = 3.0 if i % 4 < 2 else 11.0 / 3.0
        rel_eb = 10.0 ** rng.uniform(-4.0, -2.0)
        specs.append({"shape": shape, "slope": slope, "rel_eb": rel_eb, "seed": 1000 + i})
    return specs


def quantize(x, eb):
    """Eq. 1 pre-quantization: q = floor(x / (2 eb) + 1/2) in FP64, as int32.

    Accepts a numpy array or a torch tensor (returned on the same device).
    ``|x - 2 q eb| <= eb`` holds for every point.
    """
    if isinstance(x, torch.Tensor):
        return torch.floor(x.to(torch.float64) / (2.0 * eb) + 0.5).to(torch.int32)
    return np.floor(np.asarray(x, np.float64) / (2.0 * eb) + 0.5).astype(np.int32)


def value_range(x):
    """max(x) - min(x) as a Python float (numpy or torch)."""
    if isinstance(x, torch.Tensor):
        return float(x.max().item() - x.min().item())
    return float(np.max(x) - np.min(x))
