"""Pins for the oracle's network primitives (CPU only).

Each check compares the oracle against something other than itself: a six-loop brute force on tiny
tensors, PyTorch's float64 library routines, closed-form identities, or explicit permutation formulas.
"""
import itertools
import math

import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle


def brute_conv(x, w, b, s):
    """Direct six-loop convolution with zero padding k//2 (pure Python, tiny sizes only)."""
    H, W, Cin = x.shape
    Cout, k, _, _ = w.shape
    p = k // 2
    Ho, Wo = (H + 2 * p - k) // s + 1, (W + 2 * p - k) // s + 1
    out = np.zeros((Ho, Wo, Cout))
    for oh, ow, co in itertools.product(range(Ho), range(Wo), range(Cout)):
        acc = float(b[co])
        for ky, kx, ci in itertools.product(range(k), range(k), range(Cin)):
            ih, iw = oh * s + ky - p, ow * s + kx - p
            if 0 <= ih < H and 0 <= iw < W:
                acc += float(w[co, ky, kx, ci]) * x[ih, iw, ci]
        out[oh, ow, co] = acc
    return out


@pytest.mark.parametrize("k,s,H,W", [(3, 1, 5, 7), (3, 2, 5, 7), (3, 2, 6, 8), (1, 1, 5, 7), (3, 1, 1, 1),
                                     (3, 2, 1, 2)])
def test_conv_brute_force(k, s, H, W):
    rng = np.random.default_rng(k * 100 + s * 10 + H)
    x = rng.normal(size=(H, W, 3))
    w = rng.normal(size=(4, k, k, 3)).astype(np.float32)
    b = rng.normal(size=4).astype(np.float32)
    got = oracle.conv2d(x, w, b, s)
    ref = brute_conv(x, w, b, s)
    assert got.shape == ref.shape
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("k,s", [(3, 1), (3, 2), (1, 1)])
def test_conv_vs_torch_float64(k, s):
    rng = np.random.default_rng(7)
    x = rng.normal(size=(13, 17, 24))
    w = rng.normal(size=(40, k, k, 24)).astype(np.float32)
    b = rng.normal(size=40).astype(np.float32)
    got = oracle.conv2d(x, w, b, s)
    xt = torch.from_numpy(x).permute(2, 0, 1)[None]
    wt = torch.from_numpy(w.astype(np.float64)).permute(0, 3, 1, 2)
    ref = F.conv2d(xt, wt, torch.from_numpy(b.astype(np.float64)), stride=s, padding=k // 2)
    np.testing.assert_allclose(got, ref[0].permute(1, 2, 0).numpy(), rtol=0, atol=1e-11)


def test_pixel_shuffle_matches_torch_and_formula():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(3, 5, 4 * 6))
    got = oracle.pixel_shuffle(x)
    ref = F.pixel_shuffle(torch.from_numpy(x).permute(2, 0, 1)[None], 2)[0].permute(1, 2, 0).numpy()
    np.testing.assert_array_equal(got, ref)
    # explicit index formula: out[2h+dy][2w+dx][c] = in[h][w][4c + 2dy + dx]
    for h, w_, c, dy, dx in [(0, 0, 0, 0, 1), (2, 4, 5, 1, 0), (1, 3, 2, 1, 1)]:
        assert got[2 * h + dy, 2 * w_ + dx, c] == x[h, w_, 4 * c + 2 * dy + dx]


def test_gelu_closed_form_and_identities():
    for v in [-6.0, -1.3, -1e-3, 0.0, 0.5, 1.0, 2.7, 8.0]:
        assert abs(oracle.gelu(v) - 0.5 * v * (1 + math.erf(v / math.sqrt(2)))) < 1e-15
        # x Phi(x) - (-x) Phi(-x) = x (Phi(x) + Phi(-x)) = x
        assert abs(oracle.gelu(v) - oracle.gelu(-v) - v) < 1e-14
    assert oracle.gelu(0.0) == 0.0
    assert abs(oracle.gelu(10.0) - 10.0) < 1e-15
    assert abs(float(F.gelu(torch.tensor(1.7, dtype=torch.float64))) - oracle.gelu(1.7)) < 1e-15


def test_scale_bins_log_spaced():
    s = np.array([oracle.scale(k) for k in range(64)])
    assert abs(s[0] - 0.11) < 1e-15 and abs(s[63] - 64.0) < 1e-12
    ratios = s[1:] / s[:-1]
    np.testing.assert_allclose(ratios, (64 / 0.11) ** (1 / 63), rtol=1e-12)
    # thresholds are the geometric midpoints of neighbouring bins
    for k in (1, 20, 63):
        assert abs(math.exp(oracle.log_threshold(k)) - math.sqrt(s[k - 1] * s[k])) < 1e-12 * s[k]


def test_qstep():
    assert oracle.qstep(32) == 1.0
    assert oracle.qstep(40) == 2.0
    assert oracle.qstep(24) == 0.5
    thr32, thr40 = oracle.thresholds(32), oracle.thresholds(40)
    np.testing.assert_allclose(thr40.astype(np.float64) - thr32.astype(np.float64), math.log(2.0), atol=1e-6)


def test_scale_index_straddles_thresholds():
    thr = oracle.thresholds(32)
    vals, want = [], []
    for k in range(1, 64):
        t = np.float64(thr[k - 1])
        lo = float(np.nextafter(np.float32(t), np.float32(-np.inf)))
        hi = float(np.nextafter(np.float32(t), np.float32(np.inf)))
        vals += [lo, float(t), hi]
        want += [k - 1, k - 1, k]           # equal to the threshold stays in the lower bin
    idx = oracle.scale_index(np.array(vals), 32)
    np.testing.assert_array_equal(idx, want)
    assert oracle.scale_index(np.array([-50.0, 50.0]), 32).tolist() == [0, 63]


def test_quantize_rounding_half_even_and_clamp():
    y = np.array([0.5, 1.5, 2.5, -0.5, -1.5, 300.0, -300.0, 0.49999, 254.5, 255.5])
    mu = np.zeros_like(y)
    ls = np.zeros_like(y)
    r, _ = oracle.quantize_y(y, mu, ls, 32)
    assert r.tolist() == [0, 2, 2, 0, -2, 255, -255, 0, 254, 255]
    # q = 2 at qp = 40: r = rint((y - mu) / 2)
    r2, _ = oracle.quantize_y(np.array([3.0, 5.0, -3.0]), np.array([0.0, 1.0, 0.0]), np.zeros(3), 40)
    assert r2.tolist() == [2, 2, -2]


def test_quantize_z_rms_index():
    s = [oracle.scale(k) for k in range(64)]
    # channel c holds integer values whose RMS sits inside bin k: nearest log bin must be k
    n = 16
    z = np.zeros((4, 4, 5))
    z[..., 1] = 3.0                               # RMS 3
    z[..., 2] = np.where(np.arange(16).reshape(4, 4) % 2 == 0, 1.0, 0.0)   # RMS sqrt(1/2)
    z[..., 3] = 400.0                             # clamps to 255 -> RMS 255 > 64: top bin
    z[..., 4] = -0.4                              # rounds to 0 -> bin 0
    zhat, iz = oracle.quantize_z(z)
    assert zhat[..., 3].max() == 255
    nearest = lambda v: int(np.argmin([abs(math.log(v) - math.log(t)) for t in s]))
    assert iz[0] == 0 and iz[4] == 0
    assert iz[1] == nearest(3.0)
    assert iz[2] == nearest(math.sqrt(0.5))
    assert iz[3] == 63
    del n


def test_replicate_padding_in_analysis():
    """Analysis of a 60x60 chunk equals analysis of the same chunk replicate-padded to 64x64 by hand."""
    import synthetic
    fr = synthetic.moving_texture(3, 2, 60, 60, max_step=3, period=64)
    padded = np.pad(fr, ((0, 0), (0, 4), (0, 4), (0, 0)), mode="edge")
    w = synthetic.draw_weights(0, 2, 5)
    np.testing.assert_array_equal(oracle.analysis(0, fr, w), oracle.analysis(0, padded, w))
