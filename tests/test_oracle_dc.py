"""Pins of the oracle's DC-block model (Appendix: every module built from depth-wise convolution blocks;
HT-S counts 6 / 7 / 11 and 3 per frame decoder).

* depth-wise convolution: brute force on a tiny tensor and PyTorch's grouped conv2d;
* every stage (patch embedding + chunk encoder, prior term, chunk decoder + context generation, frame
  decoders) against a float64 PyTorch model assembled from library layers with the same weights;
* the model's size: multiply-accumulates per 1080p frame (N = 8) within 5 % of the paper's 211 G (the
  widths are chosen for this; Table 3a), counted from the layer table;
* the chunk chain: the encoder's next context equals the decoder's, the first chunk is C = 0, the
  container is version 3.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
import synthetic
from synthetic.weights import dc_layer_table, split_dc_weights
from tests.test_oracle_pipeline import _conv, _n, _t


def test_dw_conv_brute_force_and_torch():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(5, 7, 6))
    w = rng.normal(size=(6, 3, 3, 1)).astype(np.float32)
    b = rng.normal(size=6).astype(np.float32)
    out = oracle.dw_conv(x, w, b)
    ref = np.zeros_like(x)
    for h in range(5):
        for ww in range(7):
            for c in range(6):
                acc = float(b[c])
                for ky in range(3):
                    for kx in range(3):
                        ih, iw = h + ky - 1, ww + kx - 1
                        if 0 <= ih < 5 and 0 <= iw < 7:
                            acc += float(w[c, ky, kx, 0]) * x[ih, iw, c]
                ref[h, ww, c] = acc
    np.testing.assert_allclose(out, ref, atol=1e-12)
    t = F.conv2d(_t(x), torch.from_numpy(w.astype(np.float64)).permute(0, 3, 1, 2), torch.from_numpy(b.astype(np.float64)),
                 padding=1, groups=6)
    np.testing.assert_allclose(out, _n(t), atol=1e-12)


def _block(x, W, p):
    a = _conv(x, W[f"{p}.a"])
    w, b = W[f"{p}.dw"]
    dw = F.conv2d(a, torch.from_numpy(w.astype(np.float64)).permute(0, 3, 1, 2), torch.from_numpy(b.astype(np.float64)),
                  padding=1, groups=w.shape[0])
    y = x + _conv(F.gelu(dw), W[f"{p}.b"])
    return y + _conv(F.gelu(_conv(y, W[f"{p}.c"])), W[f"{p}.d"])


def test_dc_stages_match_torch_model():
    N, H, Wd = 2, 32, 48
    blob = synthetic.draw_dc_weights(N, seed=1)
    assert blob.size == oracle.dc_weight_count(N)
    W = split_dc_weights(blob, N)
    frames = synthetic.moving_texture(3, N, H, Wd, max_step=3, period=64)
    x = frames / 255.0
    H8, W8 = 2 * (-(-H // 16)), 2 * (-(-Wd // 16))
    c_in = np.random.default_rng(2).normal(0, 1.0, (H8, W8, 128))
    # patch embedding: channel (3n + c) 64 + 8 dy + dx = PyTorch's pixel_unshuffle of the stacked frames
    stacked = np.transpose(x, (1, 2, 0, 3)).reshape(H, Wd, 3 * N)
    s2d = F.pixel_unshuffle(_t(stacked), 8)
    h = _conv(s2d, W["PE"]) + _conv(_t(c_in), W["EC"])
    for b in range(6):
        h = _block(h, W, f"E{b}")
    y_t = _n(_conv(h, W["ED"], 2))
    y = oracle.dc_analysis(N, x, blob, c_in)
    np.testing.assert_allclose(y, y_t, atol=1e-9 * max(1.0, np.abs(y_t).max()))
    np.testing.assert_allclose(oracle.dc_prior_term(N, c_in, H8, W8, blob), _n(_conv(_t(c_in), W["PC"], 2)), atol=1e-12)
    yhat = np.rint(y)
    Ft = F.gelu(F.pixel_shuffle(_conv(_t(yhat), W["DU"]), 2)) + _conv(_t(c_in), W["FC"])
    for b in range(7):
        Ft = _block(Ft, W, f"D{b}")
    g = Ft
    for b in range(11):
        g = _block(g, W, f"G{b}")
    Fo, c_out = oracle.dc_trunk(N, yhat, blob, c_in)
    np.testing.assert_allclose(Fo, _n(Ft), atol=1e-9 * max(1.0, np.abs(_n(Ft)).max()))
    np.testing.assert_allclose(c_out, _n(_conv(g, W["GO"])), atol=1e-9 * max(1.0, np.abs(c_out).max()))
    rec = oracle.dc_frames(N, Fo, H, Wd, blob)
    for f in range(N):
        hf = _conv(_t(Fo), W[f"FP.{f}"])
        for b in range(3):
            hf = _block(hf, W, f"F{f}.{b}")
        o = F.pixel_shuffle(_conv(hf, W[f"FO.{f}"]), 8)
        np.testing.assert_allclose(rec[f], np.clip(0.5 + _n(o)[:H, :Wd], 0, 1), atol=1e-9)


def test_dc_model_size_matches_the_paper():
    """Table 3a: DCVC-UF (HT-S) 211 G MACs per frame.  Counted from the layer table at 1080p, N = 8."""
    N, Hp, Wp = 8, 1088, 1920
    pos = {1: (Hp // 8) * (Wp // 8)}
    macs = 0
    for name, co, k, ci in dc_layer_table(N):
        if name in ("ED", "H1", "H2", "S1", "S2", "S3", "PC", "DU"):
            continue
        n = pos[1]
        macs += n * co * k * k * ci
    # layers at the latent and hyper-latent sizes
    Hy, Wy = Hp // 16, Wp // 16
    Hz, Wz = -(-Hy // 4), -(-Wy // 4)
    d = {nm: (co, k, ci) for nm, co, k, ci in dc_layer_table(N)}
    macs += Hy * Wy * np.prod(d["ED"]) * d["ED"][1] + Hy * Wy * np.prod(d["DU"]) * d["DU"][1]
    macs += Hy * Wy * np.prod(d["PC"]) * d["PC"][1] + Hy * Wy * np.prod(d["S3"]) * d["S3"][1]
    macs += (Hy // 2) * (Wy // 2) * np.prod(d["H1"]) * 3 + Hz * Wz * np.prod(d["H2"]) * 3
    macs += Hz * Wz * np.prod(d["S1"]) * 3 + 2 * Hz * 2 * Wz * np.prod(d["S2"]) * 3
    per_frame = macs / N
    assert abs(per_frame / 211e9 - 1) < 0.05, per_frame / 1e9


def test_dc_chunk_chain():
    N, H, W = 8, 64, 64
    blob = synthetic.draw_dc_weights(N, seed=0)
    c_e = c_d = None
    for i in range(3):
        fr = synthetic.moving_texture(30 + i, N, H, W, max_step=3, period=64)
        bits, c_e2, dbg = oracle.encode_chunk_t(2, fr, 32, 64, blob, None, c_e, debug=True)
        assert bits[4] == 3
        rec, yhat, c_d2 = oracle.decode_chunk_t(2, N, bits, H, W, blob, None, c_d)
        np.testing.assert_array_equal(c_e2, c_d2)
        np.testing.assert_array_equal(yhat, dbg["yhat"])
        F_, _ = oracle.dc_trunk(N, yhat, blob, c_d, want_c_out=False)
        np.testing.assert_array_equal(rec, oracle.dc_frames(N, F_, H, W, blob))
        assert np.sqrt(np.mean(c_e2 ** 2)) < 10.0  # the random-weight recursion stays bounded
        c_e, c_d = c_e2, c_d2
    b0, _ = oracle.encode_chunk_t(2, synthetic.moving_texture(30, N, H, W, max_step=3, period=64), 32, 64, blob, None,
                                  np.zeros((8, 8, 128)))
    b0n, _ = oracle.encode_chunk_t(2, synthetic.moving_texture(30, N, H, W, max_step=3, period=64), 32, 64, blob, None,
                                   None)
    assert b0 == b0n
