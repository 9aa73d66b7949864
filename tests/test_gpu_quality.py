"""GPU quality metrics (Sec. III-B: Eq. 3 SSIM over sliding windows, Eq. 4
PSNR) against the FP64 oracle (oracle/quality.py, pinned in
test_oracle_quality.py).

Tolerances: every window statistic is a sum of at most ~30 fp32 roundings of
non-negative or centred terms (no E[x^2] - E[x]^2 cancellation), so each of
the two factors of Eq. 3 carries a relative error of a few 1e-6 at most and a
window's SSIM (|SSIM| <= 1) is within 1e-5; the mean over windows inherits
the same bound. MSE is an fp32 compensated sum (relative 1e-6), and PSNR =
20 log10(range / sqrt(MSE)) moves by 4.35e-6 dB per 1e-6 of MSE."""
import json
import os

import numpy as np
import pytest
import torch

from oracle import quality as oq
from paper_2602_20097_gb300 import qai, synth

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "Q1_ssim_step.json")))
TOL_W = 1e-5


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_golden_values_on_the_gpu():
    x, y = np.array(GOLD["x"]), np.array(GOLD["y"])
    r = qai.quality(_cuda(x), _cuda(y), ssim_map=True)
    assert r["windows"] == 2 and (r["x_min"], r["x_max"]) == (0.0, 1.0)
    assert np.allclose(r["map"].cpu().numpy(), GOLD["ssim_windows"], rtol=0, atol=TOL_W)
    assert abs(r["ssim"] - GOLD["ssim"]) <= TOL_W
    assert abs(r["mse"] - GOLD["mse"]) <= 1e-6 * GOLD["mse"]
    assert abs(r["psnr"] - GOLD["psnr"]) <= 1e-5
    assert abs(qai.quality(_cuda(x), _cuda(y), stride=1)["ssim"] - GOLD["ssim_stride1"]) <= TOL_W
    assert abs(qai.quality(_cuda(x), _cuda(2 * y))["ssim"] - GOLD["ssim_x_2y"]) <= TOL_W
    x3, y3 = np.broadcast_to(x, (7, 7, 9)), np.broadcast_to(y, (7, 7, 9))
    r3 = qai.quality(_cuda(x3), _cuda(y3), ssim_map=True)
    assert np.allclose(r3["map"].cpu().numpy().ravel(), GOLD["ssim_3d_windows"], rtol=0, atol=TOL_W)
    assert abs(r3["ssim"] - GOLD["ssim_3d"]) <= TOL_W


def _pair(shape, seed):
    """A field and its mitigated reconstruction (eb 1e-2 of the range)."""
    sq = tuple(d for d in shape if d > 1) or (1,)
    if len(sq) >= 2:
        x = synth.grf(sq, slope=11.0 / 3.0, seed=seed, device="cuda").float()
    else:
        x = torch.from_numpy(synth.sinusoids(sq, seed=seed)).float().cuda()
    eb = 1e-2 * synth.value_range(x)
    q = synth.quantize(x, eb)
    return x.reshape(shape).contiguous(), qai.mitigate(q, eb).reshape(shape).contiguous()


def _compare(x, y, window, stride):
    r = qai.quality(x, y, window=window, stride=stride, ssim_map=True)
    xn, yn = x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64)
    ref_map = oq.ssim_map(xn, yn, window, stride)
    got_map = r["map"].cpu().numpy().astype(np.float64).reshape(ref_map.shape)
    assert np.max(np.abs(got_map - ref_map)) <= TOL_W
    assert r["windows"] == ref_map.size
    assert abs(r["ssim"] - float(np.mean(ref_map))) <= TOL_W
    assert r["x_min"] == float(xn.min()) and r["x_max"] == float(xn.max())
    mse = oq.mse(xn, yn)
    assert abs(r["mse"] - mse) <= 1e-6 * mse + 1e-30
    if mse > 0:
        assert abs(r["psnr"] - oq.psnr(xn, yn)) <= 1e-5
    return r


SHAPES = [(5000,), (7,), (3,), (64, 100), (37, 1025), (180, 361), (16, 16, 16), (9, 130, 47),
          (33, 17, 65), (40, 64, 96), (6, 7, 8), (1, 50, 1, 60)]


@pytest.mark.parametrize("shape", SHAPES, ids=str)
def test_matches_oracle(shape):
    x, y = _pair(shape, seed=sum(shape))
    _compare(x, y, 7, 2)


@pytest.mark.parametrize("window,stride", [(7, 1), (11, 4), (3, 3), (1, 1), (2, 2), (11, 1)])
def test_window_and_stride_variants(window, stride):
    x, y = _pair((21, 45, 70), seed=window * 10 + stride)
    _compare(x, y, window, stride)


def test_noisy_and_offset_fields():
    g = torch.Generator(device="cpu").manual_seed(5)
    x = (torch.rand((30, 40, 50), generator=g, dtype=torch.float64) * 7 + 1000).float().cuda()
    y = (x.double() + 0.3 * torch.randn((30, 40, 50), generator=g, dtype=torch.float64).cuda()).float()
    _compare(x.contiguous(), y.contiguous(), 7, 2)
    r = qai.quality(x, x.clone())
    assert r["ssim"] == pytest.approx(1.0, abs=TOL_W) and r["psnr"] == float("inf")


def test_full_size_sampled_windows_and_determinism():
    shape = (512, 512, 512)
    x = synth.grf(shape, slope=11.0 / 3.0, seed=2, device="cuda").float()
    eb = 1e-3 * synth.value_range(x)
    q = synth.quantize(x, eb)
    y = qai.mitigate(q, eb)
    r1 = qai.quality(x, y, ssim_map=True)
    r2 = qai.quality(x, y)
    assert r1["ssim"] == r2["ssim"] and r1["mse"] == r2["mse"]
    nw = oq.window_counts(shape)
    assert r1["windows"] == nw[0] * nw[1] * nw[2]
    rng = np.random.default_rng(0)
    picks = [tuple(int(rng.integers(0, n)) for n in nw) for _ in range(300)]
    picks += [(0, 0, 0), tuple(n - 1 for n in nw), (nw[0] - 1, 0, nw[2] - 1)]
    # the windows touch only their own points: compare on the crops around them
    m = r1["map"]
    xr, yr = x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64)
    lo, hi = xr.min(), xr.max()
    for p in picks:
        sl = tuple(slice(2 * i, 2 * i + 7) for i in p)
        want = oq.ssim_of_window((xr[sl] - lo) / (hi - lo), (yr[sl] - lo) / (hi - lo))
        assert abs(float(m[p]) - want) <= TOL_W, p
    mse = float(np.mean((xr - yr) ** 2))
    assert abs(r1["mse"] - mse) <= 1e-6 * mse
    # the mean over every window, with the map's own values summed in FP64
    assert abs(r1["ssim"] - float(m.double().mean())) <= 1e-9


def test_argument_errors():
    x = torch.zeros((8, 8), device="cuda")
    for kw in ({"window": 0}, {"window": 12}, {"stride": 0}, {"stride": 5}):
        with pytest.raises(qai.QAIError):
            qai.quality(x, x, **kw)
    with pytest.raises(qai.QAIError):
        qai.quality(x, torch.zeros((8, 9), device="cuda"))
