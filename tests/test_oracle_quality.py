"""Pins of the FP64 quality oracle (Sec. III-B: Eq. 3 SSIM, Eq. 4 PSNR):
hand-derived values (tests/golden/Q1_ssim_step.json), SSIM(x, x) = 1, the
closed form on constant fields, window placement, and planted mistakes that
each fail one of these."""
import json
import math
import os
import types

import numpy as np
import pytest

from oracle import quality

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "Q1_ssim_step.json")))


def _check_golden(q):
    x, y = np.array(GOLD["x"], float), np.array(GOLD["y"], float)
    assert np.allclose(q.ssim_map(x, y), GOLD["ssim_windows"], rtol=0, atol=1e-14)
    assert abs(q.ssim(x, y) - GOLD["ssim"]) < 1e-14
    assert abs(q.ssim(x, y, stride=1) - GOLD["ssim_stride1"]) < 1e-14
    assert abs(q.ssim(x, 2 * y) - GOLD["ssim_x_2y"]) < 1e-14
    x3 = np.broadcast_to(x, (7, 7, 9)).copy()
    y3 = np.broadcast_to(y, (7, 7, 9)).copy()
    assert np.allclose(q.ssim_map(x3, y3).ravel(), GOLD["ssim_3d_windows"], rtol=0, atol=1e-14)
    assert abs(q.ssim(x3, y3) - GOLD["ssim_3d"]) < 1e-14
    assert abs(q.mse(x, y) - GOLD["mse"]) < 1e-15
    assert abs(q.psnr(x, y) - GOLD["psnr"]) < 1e-12
    # an affine map of both fields changes nothing (normalisation by range(x))
    assert abs(q.ssim(3 * x + 5, 3 * y + 5) - GOLD["ssim"]) < 1e-13
    assert abs(q.psnr(3 * x + 5, 3 * y + 5) - GOLD["psnr"]) < 1e-12


def test_golden_values():
    _check_golden(quality)


@pytest.mark.parametrize("shape", [(50,), (20, 31), (9, 12, 15), (1, 30, 1, 40)])
def test_identical_fields_give_one(shape):
    x = np.random.default_rng(1).standard_normal(shape)
    assert np.allclose(quality.ssim_map(x, x), 1.0, rtol=0, atol=1e-12)
    assert quality.psnr(x, x) == math.inf


def test_constant_fields_closed_form():
    # a constant original is shifted to 0 and not scaled; Eq. 3 reduces to
    # (2ab + c1) / (a^2 + b^2 + c1) with a = 0, b = 0.7 - 0.3
    x, y = np.full((10, 10), 0.3), np.full((10, 10), 0.7)
    b = 0.7 - 0.3
    want = quality.C1 / (b * b + quality.C1)
    assert np.allclose(quality.ssim_map(x, y), want, rtol=0, atol=1e-15)
    assert quality.psnr(x, y) == -math.inf


def test_window_placement():
    assert quality.window_counts((5, 40, 9)) == (1, 17, 2)
    assert quality.window_counts((7,)) == (1,)
    assert quality.window_counts((3, 3)) == (1, 1)
    x = np.random.default_rng(2).random((11, 16, 13))
    y = x + 0.01 * np.random.default_rng(3).standard_normal(x.shape)
    full = quality.ssim_map(x, y)
    assert full.shape == quality.window_counts(x.shape)
    picks = [(0, 0, 0), (2, 4, 3), (1, 2, 1)]
    assert np.allclose(quality.ssim_at(x, y, picks), [full[p] for p in picks], rtol=0, atol=1e-14)


MUTATIONS = {
    "divisor n": ("den = max(n - 1, 1)", "den = max(n, 1)"),
    "stride ignored": ("sl = tuple(slice(None, None, stride) for _ in m)", "sl = tuple(slice(None) for _ in m)"),
    "c1 and c2 swapped": ("C1 = 1e-4\nC2 = 9e-4", "C1 = 9e-4\nC2 = 1e-4"),
    "range of y": ("lo, hi = float(x.min()), float(x.max())", "lo, hi = float(y.min()), float(y.max())"),
    "no min shift": ("return (x - lo) / r, (y - lo) / r", "return x / r, y / r"),
    "covariance not doubled": ("* (2 * cov + C2))", "* (cov + C2))"),
    "window too long": ("return tuple(min(window, d) for d in shape)", "return tuple(min(window + 1, d) for d in shape)"),
    "psnr uses 10 log10": ("20.0 * math.log10(r / math.sqrt(e))", "10.0 * math.log10(r / math.sqrt(e))"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistakes_fail_a_pin(name):
    src = open(quality.__file__).read()
    old, new = MUTATIONS[name]
    assert src.count(old) >= 1, name
    mod = types.ModuleType("quality_mutant")
    exec(compile(src.replace(old, new), "quality_mutant", "exec"), mod.__dict__)
    with pytest.raises((AssertionError, ValueError)):
        _check_golden(mod)
