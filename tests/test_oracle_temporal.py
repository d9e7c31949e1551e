"""Pins of the oracle's temporal chunk context (Sec. 3.1, Fig. 3): the chunk feature F_i, the next
context C_{i+1}, and the conditioning of the encoder, the prior and the frame decoders on C_i.

* every temporal piece against a float64 PyTorch model assembled from library layers (conv2d,
  pixel_shuffle, gelu) with the same weights, for a random C_i;
* all-zero temporal weights reduce the codec exactly to the plain one (same sections, same frames);
* the encoder's C_{i+1} equals the decoder's bit for bit over a chunk sequence, and the decode of chunk i
  depends on C_i; the first chunk (no context) equals C = 0;
* container versions 3 / 4 require the temporal blob, 1 / 2 refuse it.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
import synthetic
from synthetic.weights import split_temporal_weights, split_weights
from tests._util import parse_container
from tests.test_oracle_pipeline import _conv, _n, _t, torch_decoder

ARCH, N = 0, 2


def _case(seed=0, H=64, W=64):
    frames = synthetic.moving_texture(20 + seed, N, H, W, max_step=3, period=64)
    blob = synthetic.draw_weights(ARCH, N, seed=3)
    tw = synthetic.draw_temporal_weights(ARCH, N, seed=seed)
    return frames, blob, tw


def test_temporal_layers_match_torch_model():
    H, W = 64, 48
    frames, blob, tw = _case(1, H, W)
    Wt = split_weights(blob, ARCH, N)
    Tt = split_temporal_weights(tw, ARCH, N)
    H8, W8, Cc = oracle.context_dims(ARCH, H, W)
    c_in = np.random.default_rng(5).normal(0, 0.5, (H8, W8, Cc))
    ec, pc = oracle.context_terms(ARCH, N, c_in, H8, W8, tw)
    np.testing.assert_allclose(ec, _n(_conv(_t(c_in), Tt["EC"])), atol=1e-12)
    np.testing.assert_allclose(pc, _n(_conv(_t(c_in), Tt["PC"], 2)), atol=1e-12)
    # encoder: A3 output + EC(C) before the interaction block
    bits, c_out, dbg = oracle.encode_chunk_t(ARCH, frames, 32, 16, blob, tw, c_in, debug=True)
    hp, wp = -(-H // 16) * 16, -(-W // 16) * 16
    x = np.pad(frames, ((0, 0), (0, hp - H), (0, wp - W), (0, 0)), mode="edge") / 255.0
    h = _t(np.transpose(x, (1, 2, 0, 3)).reshape(hp, wp, 3 * N))
    for name in ("A1", "A2", "A3"):
        h = F.gelu(_conv(h, Wt[name], 2))
    h = h + _t(ec)
    h = h + _conv(F.gelu(_conv(h, Wt["Xa"])), Wt["Xb"])
    np.testing.assert_allclose(dbg["y"], _n(_conv(h, Wt["A4"], 2)), atol=1e-10)
    # prior: S2 features + PC(C) before S3
    Hy, Wy = dbg["y"].shape[:2]
    s = _t(dbg["zhat"].astype(np.float64))
    for name in ("S1", "S2"):
        s = F.gelu(F.pixel_shuffle(_conv(s, Wt[name]), 2))
    s = s[:, :, :Hy, :Wy] + _t(pc)
    np.testing.assert_allclose(dbg["s"], _n(s), atol=1e-10)
    p = _n(_conv(s, Wt["S3"]))
    np.testing.assert_allclose(dbg["logsig"], p[..., 128:], atol=1e-10)
    # chunk feature and next context from the encoder's y^
    yhat = dbg["yhat"]
    Ft = F.gelu(F.pixel_shuffle(_conv(_t(yhat), Tt["FD"]), 2)) + _conv(_t(c_in), Tt["FC"])
    Fo = oracle.chunk_feature(ARCH, N, yhat, tw, c_in)
    np.testing.assert_allclose(Fo, _n(Ft), atol=1e-10)
    np.testing.assert_allclose(c_out, _n(F.gelu(_conv(Ft, Tt["CG"]))), atol=1e-10)
    np.testing.assert_allclose(oracle.context_next(ARCH, N, Fo, tw), c_out, atol=0)
    # frame decoders: D0 output + DF_f(F)
    rec = oracle.synthesis_f(ARCH, N, yhat, Fo, H, W, blob, tw)
    for f in range(N):
        hd = F.gelu(F.pixel_shuffle(_conv(_t(yhat), Wt[f"D0.{f}"]), 2)) + _conv(_t(Fo), Tt[f"DF.{f}"])
        hd = hd + _conv(F.gelu(_conv(hd, Wt[f"R1a.{f}"])), Wt[f"R1b.{f}"])
        hd = F.gelu(F.pixel_shuffle(_conv(hd, Wt[f"U1.{f}"]), 2))
        hd = hd + _conv(F.gelu(_conv(hd, Wt[f"R2a.{f}"])), Wt[f"R2b.{f}"])
        hd = F.gelu(F.pixel_shuffle(_conv(hd, Wt[f"U2.{f}"]), 2))
        o = F.pixel_shuffle(_conv(hd, Wt[f"U3.{f}"]), 2)
        np.testing.assert_allclose(rec[f], np.clip(0.5 + _n(o)[:H, :W], 0, 1), atol=1e-9)
        # without the feature the decoder is the plain one (the torch model of the plain path agrees)
    np.testing.assert_allclose(oracle.synthesis(ARCH, N, yhat, H, W, blob)[0], torch_decoder(yhat, 0, H, W, Wt),
                               atol=1e-9)


def test_zero_temporal_weights_reduce_to_plain_codec():
    frames, blob, tw = _case(2)
    tw0 = np.zeros_like(tw)
    H8, W8, Cc = oracle.context_dims(ARCH, 64, 64)
    c_in = np.random.default_rng(1).normal(0, 1, (H8, W8, Cc))
    bits_t, c_out = oracle.encode_chunk_t(ARCH, frames, 32, 16, blob, tw0, c_in)
    bits_p = oracle.encode_chunk(ARCH, frames, 32, 16, blob)
    assert bits_t[4] == 3 and bits_p[4] == 1
    assert bits_t[5:] == bits_p[5:]
    assert np.all(c_out == 0.0)  # GELU(0)
    fr_t, yh_t, _ = oracle.decode_chunk_t(ARCH, N, bits_t, 64, 64, blob, tw0, c_in)
    fr_p, yh_p = oracle.decode_chunk(ARCH, N, bits_p, 64, 64, blob)
    np.testing.assert_array_equal(fr_t, fr_p)
    np.testing.assert_array_equal(yh_t, yh_p)


def test_context_sequence_encoder_tracks_decoder():
    blob = synthetic.draw_weights(ARCH, N, seed=3)
    tw = synthetic.draw_temporal_weights(ARCH, N, seed=4)
    chunks = [synthetic.moving_texture(40 + i, N, 64, 64, max_step=3, period=64) for i in range(3)]
    c_enc = c_dec = None
    outs = []
    for i, fr in enumerate(chunks):
        bits, c_enc_next = oracle.encode_chunk_t(ARCH, fr, 32, 16, blob, tw, c_enc)
        rec, yh, c_dec_next = oracle.decode_chunk_t(ARCH, N, bits, 64, 64, blob, tw, c_dec)
        np.testing.assert_array_equal(c_enc_next, c_dec_next)
        outs.append((bits, rec))
        c_enc, c_dec = c_enc_next, c_dec_next
    # the first chunk's missing context is C = 0
    H8, W8, Cc = oracle.context_dims(ARCH, 64, 64)
    bits0z, c1z = oracle.encode_chunk_t(ARCH, chunks[0], 32, 16, blob, tw, np.zeros((H8, W8, Cc)))
    assert bits0z == outs[0][0]
    # decoding chunk 1 against another context: the prior's scales change, so the entropy decoder
    # either detects a corrupt lane or yields other frames (the context is used)
    try:
        rec_wrong, _, _ = oracle.decode_chunk_t(ARCH, N, outs[1][0], 64, 64, blob, tw, None)
        assert np.abs(rec_wrong - outs[1][1]).max() > 1e-3
    except RuntimeError as e:
        assert "code 3" in str(e)


def test_temporal_versions():
    frames, blob, tw = _case(3)
    mw = synthetic.draw_mean_weights(ARCH, seed=0)
    bits3, _ = oracle.encode_chunk_t(ARCH, frames, 32, 16, blob, tw, None)
    bits4, c4 = oracle.encode_chunk_t(ARCH, frames, 32, 16, blob, tw, None, mean_weights=mw)
    assert bits3[4] == 3 and bits4[4] == 4
    with pytest.raises(RuntimeError):
        oracle.decode_chunk(ARCH, N, bits3, 64, 64, blob)
    with pytest.raises(RuntimeError):
        oracle.decode_chunk_t(ARCH, N, bits4, 64, 64, blob, tw, None)  # needs the mean network too
    _, _, c4d = oracle.decode_chunk_t(ARCH, N, bits4, 64, 64, blob, tw, None, mean_weights=mw)
    np.testing.assert_array_equal(c4, c4d)
    with pytest.raises(RuntimeError):
        oracle.decode_chunk_t(ARCH, N, oracle.encode_chunk(ARCH, frames, 32, 16, blob), 64, 64, blob, tw, None)
    c = parse_container(bits3, 64)
    assert c["total"] == len(bits3)
