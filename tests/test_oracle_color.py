"""Pins of the oracle's colour interface (Appendix: YUV444 model interface; BT.709 for RGB; YUV420 chroma).

* BT.709: the luma weights sum to one and the chroma scale factors are 2 (1 - K_B) and 2 (1 - K_R), so
  white / grey map to chroma 0.5, pure blue to U = 1 and pure red to V = 1 exactly; the luma of the
  primaries is the standard's K_R, K_G, K_B; round trip RGB -> YUV -> RGB is the identity.
* YUV420: input replicates each chroma sample over its 2x2 block; output averages the block's pixels
  inside the frame; down(up(c)) = c for every size, including odd ones.
* YUV444 planar: a permutation of the interleaved channels.
"""
import numpy as np
import pytest

import oracle

KR, KG, KB = 0.2126, 0.7152, 0.0722


def _rgb(pixels):
    return np.array(pixels, np.uint8).reshape(1, 1, len(pixels), 3)


def test_bt709_primaries_and_neutrals():
    f = _rgb([(255, 255, 255), (128, 128, 128), (255, 0, 0), (0, 255, 0), (0, 0, 255), (0, 0, 0)])
    x = oracle.color_in(oracle.RGB_BT709, f, 1, 1, 6)[0, 0]
    assert abs(KR + KG + KB - 1.0) < 1e-15
    np.testing.assert_allclose(x[0], [1.0, 0.5, 0.5], atol=1e-12)
    np.testing.assert_allclose(x[1], [128 / 255, 0.5, 0.5], atol=1e-12)
    np.testing.assert_allclose(x[2, 0], KR, atol=1e-12)
    np.testing.assert_allclose(x[3, 0], KG, atol=1e-12)
    np.testing.assert_allclose(x[4, 0], KB, atol=1e-12)
    np.testing.assert_allclose(x[2, 2], 1.0, atol=1e-12)  # V of pure red
    np.testing.assert_allclose(x[4, 1], 1.0, atol=1e-12)  # U of pure blue
    np.testing.assert_allclose(x[5], [0.0, 0.5, 0.5], atol=1e-12)
    # the extremes of the chroma range: U in [0, 1], V in [0, 1] over all RGB corners
    corners = _rgb([(r, g, b) for r in (0, 255) for g in (0, 255) for b in (0, 255)])
    xc = oracle.color_in(oracle.RGB_BT709, corners, 1, 1, 8)[0, 0]
    assert xc[:, 1:].min() >= -1e-12 and xc[:, 1:].max() <= 1 + 1e-12


def test_bt709_round_trip():
    rng = np.random.default_rng(0)
    f = rng.integers(0, 256, (2, 5, 7, 3), dtype=np.uint8)
    x = oracle.color_in(oracle.RGB_BT709, f, 2, 5, 7)
    back = oracle.color_out(oracle.RGB_BT709, x, 2, 5, 7).reshape(2, 5, 7, 3)
    np.testing.assert_allclose(back, f / 255.0, atol=1e-12)
    # RGB format 0 is the identity
    np.testing.assert_array_equal(oracle.color_in(oracle.RGB, f, 2, 5, 7), f / 255.0)


@pytest.mark.parametrize("H,W", [(4, 6), (5, 7), (1, 1), (3, 2)])
def test_yuv420_replicate_and_average(H, W):
    rng = np.random.default_rng(H * 10 + W)
    Hc, Wc = (H + 1) // 2, (W + 1) // 2
    fb = oracle.frame_bytes(oracle.YUV420P, H, W)
    assert fb == H * W + 2 * Hc * Wc
    f = rng.integers(0, 256, 2 * fb, dtype=np.uint8)
    x = oracle.color_in(oracle.YUV420P, f, 2, H, W)
    for n in range(2):
        fr = f[n * fb:(n + 1) * fb]
        np.testing.assert_array_equal(x[n, :, :, 0], fr[:H * W].reshape(H, W) / 255.0)
        u = fr[H * W:H * W + Hc * Wc].reshape(Hc, Wc) / 255.0
        v = fr[H * W + Hc * Wc:].reshape(Hc, Wc) / 255.0
        for h in range(H):
            for w in range(W):
                assert x[n, h, w, 1] == u[h // 2, w // 2] and x[n, h, w, 2] == v[h // 2, w // 2]
    # replicated chroma averages back to itself, odd edges included
    back = oracle.color_out(oracle.YUV420P, x, 2, H, W)
    np.testing.assert_allclose(back, f / 255.0, atol=1e-15)
    # the mean over the block: a block with values 0, 1, 0, 1 gives 0.5
    if H >= 2 and W >= 2:
        x2 = np.zeros((1, H, W, 3))
        x2[0, 0, 1, 1] = x2[0, 1, 1, 1] = 1.0
        out = oracle.color_out(oracle.YUV420P, x2, 1, H, W)
        assert out[H * W] == 0.5


def test_yuv444_planar_is_a_permutation():
    rng = np.random.default_rng(1)
    H, W = 3, 4
    f = rng.integers(0, 256, 2 * 3 * H * W, dtype=np.uint8)
    x = oracle.color_in(oracle.YUV444P, f, 2, H, W)
    planes = f.reshape(2, 3, H, W)
    np.testing.assert_array_equal(x, np.moveaxis(planes, 1, 3) / 255.0)
    np.testing.assert_array_equal(oracle.color_out(oracle.YUV444P, x, 2, H, W), f / 255.0)


def test_bt709_output_clamps():
    # Y = 0, U = 0, V = 1: R = 0.7874 (in range), G and B below zero before clamping
    out = oracle.color_out(oracle.RGB_BT709, np.array([[[[0.0, 0.0, 1.0]]]]), 1, 1, 1)
    np.testing.assert_allclose(out, [1.0 - KR, 0.0, 0.0], atol=1e-12)
    # Y = 1, U = 1, V = 1: R and B above one before clamping
    out = oracle.color_out(oracle.RGB_BT709, np.array([[[[1.0, 1.0, 1.0]]]]), 1, 1, 1)
    assert out[0] == 1.0 and out[2] == 1.0 and 0.0 < out[1] < 1.0


def test_analysis_x_equals_analysis_for_rgb():
    import synthetic
    frames = synthetic.chunk_frames("tiny", seed=2)[:2]
    blob = synthetic.draw_weights(0, 2, seed=0)
    y1 = oracle.analysis(0, frames, blob)
    y2 = oracle.analysis_x(0, frames / 255.0, blob)
    np.testing.assert_array_equal(y1, y2)
