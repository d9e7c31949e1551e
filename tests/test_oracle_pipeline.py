"""Pins for the oracle's whole-chunk path (CPU only).

The network stages are checked against a float64 PyTorch model assembled from library layers
(conv2d, pixel_shuffle, gelu) with the same weights; the container is checked field by field; the
decoder must reproduce y^ = r^ q + mu exactly from the encoder's own intermediates.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
import synthetic
from synthetic.weights import split_weights, ARCHS


def _t(x):            # HWC numpy -> 1CHW torch
    return torch.from_numpy(np.ascontiguousarray(x, np.float64)).permute(2, 0, 1)[None]


def _n(t):            # 1CHW torch -> HWC numpy
    return t[0].permute(1, 2, 0).numpy()


def _conv(x, wb, s=1):
    w, b = wb
    wt = torch.from_numpy(w.astype(np.float64)).permute(0, 3, 1, 2)
    return F.conv2d(x, wt, torch.from_numpy(b.astype(np.float64)), stride=s, padding=w.shape[1] // 2)


def torch_encoder(frames, W, arch):
    N, H, Wd, _ = frames.shape
    hp, wp = -(-H // 16) * 16, -(-Wd // 16) * 16
    x = np.pad(frames, ((0, 0), (0, hp - H), (0, wp - Wd), (0, 0)), mode="edge") / 255.0
    x = np.transpose(x, (1, 2, 0, 3)).reshape(hp, wp, 3 * N)        # frame n -> channels 3n..3n+2
    h = _t(x)
    for name in ("A1", "A2", "A3"):
        h = F.gelu(_conv(h, W[name], 2))
    h = h + _conv(F.gelu(_conv(h, W["Xa"])), W["Xb"])
    y = _conv(h, W["A4"], 2)
    z = _conv(F.gelu(_conv(y, W["H1"], 2)), W["H2"], 2)
    return _n(y), _n(z)


def torch_hyper_synthesis(zhat, Hy, Wy, W, arch):
    s = _t(zhat.astype(np.float64))
    for name in ("S1", "S2"):
        s = F.gelu(F.pixel_shuffle(_conv(s, W[name]), 2))
    s = s[:, :, :Hy, :Wy]
    p = _n(_conv(s, W["S3"]))
    cy = ARCHS[arch]["cy"]
    return p[..., :cy], p[..., cy:]


def torch_decoder(yhat, f, H, Wd, W):
    h = F.gelu(F.pixel_shuffle(_conv(_t(yhat), W[f"D0.{f}"]), 2))
    h = h + _conv(F.gelu(_conv(h, W[f"R1a.{f}"])), W[f"R1b.{f}"])
    h = F.gelu(F.pixel_shuffle(_conv(h, W[f"U1.{f}"]), 2))
    h = h + _conv(F.gelu(_conv(h, W[f"R2a.{f}"])), W[f"R2b.{f}"])
    h = F.gelu(F.pixel_shuffle(_conv(h, W[f"U2.{f}"]), 2))
    o = F.pixel_shuffle(_conv(h, W[f"U3.{f}"]), 2)
    return np.clip(0.5 + _n(o)[:H, :Wd], 0.0, 1.0)


@pytest.mark.parametrize("arch,N,H,W", [(0, 2, 64, 64), (0, 2, 50, 70), (1, 1, 48, 80)])
def test_network_stages_match_torch_model(arch, N, H, W):
    frames = synthetic.moving_texture(11, N, H, W, max_step=3, period=64)
    blob = synthetic.draw_weights(arch, N, seed=2)
    Wt = split_weights(blob, arch, N)
    y = oracle.analysis(arch, frames, blob)
    z = oracle.hyper_analysis(arch, N, y, blob)
    y_t, z_t = torch_encoder(frames, Wt, arch)
    np.testing.assert_allclose(y, y_t, rtol=0, atol=1e-10)
    np.testing.assert_allclose(z, z_t, rtol=0, atol=1e-10)
    zhat, iz = oracle.quantize_z(z)
    mu, ls = oracle.hyper_synthesis(arch, N, zhat, y.shape[0], y.shape[1], blob)
    mu_t, ls_t = torch_hyper_synthesis(zhat, y.shape[0], y.shape[1], Wt, arch)
    np.testing.assert_allclose(mu, mu_t, rtol=0, atol=1e-10)
    np.testing.assert_allclose(ls, ls_t, rtol=0, atol=1e-10)
    rhat, idx = oracle.quantize_y(y, mu, ls, 32)
    yhat = rhat + mu
    rec = oracle.synthesis(arch, N, yhat, H, W, blob)
    for f in range(N):
        np.testing.assert_allclose(rec[f], torch_decoder(yhat, f, H, W, Wt), rtol=0, atol=1e-9)


@pytest.mark.parametrize("qp", [32, 27, 40])
def test_chunk_roundtrip_and_container(qp):
    frames = synthetic.chunk_frames("tiny", seed=1)[:2]
    blob = synthetic.draw_weights(0, 2, seed=0)
    K = 32
    bits, dbg = oracle.encode_chunk(0, frames, qp, K, blob, debug=True)
    # container fields
    assert bits[:4] == b"UFVC" and bits[4] == 1 and bits[5] == 0 and bits[6] == 2 and bits[7] == qp
    assert int.from_bytes(bits[8:10], "little") == 64 and int.from_bytes(bits[10:12], "little") == 64
    assert int.from_bytes(bits[12:16], "little") == K
    assert int.from_bytes(bits[16:20], "little") == min(K, dbg["zhat"].size)
    assert bytes(bits[20:20 + 64]) == dbg["iz"].tobytes()
    assert len(bits) % 4 == 0
    # the decoder recovers y^ = r^ q + mu exactly (its own hyper-synthesis from the decoded z^)
    frames_out, yhat = oracle.decode_chunk(0, 2, bits, 64, 64, blob)
    q = oracle.qstep(qp)
    np.testing.assert_array_equal(yhat, dbg["rhat"] * q + dbg["mu"])
    np.testing.assert_array_equal(frames_out, oracle.synthesis(0, 2, yhat, 64, 64, blob))
    # the scale indices follow log sigma; quantisation error is bounded by q/2 unless clipped
    err = np.abs(dbg["y"] - yhat)
    assert (err[np.abs(dbg["rhat"]) < 255] <= q / 2 + 1e-12).all()


def test_decoder_rejects_bad_container():
    frames = synthetic.chunk_frames("tiny", seed=1)[:2]
    blob = synthetic.draw_weights(0, 2, seed=0)
    bits = oracle.encode_chunk(0, frames, 32, 32, blob)
    with pytest.raises(RuntimeError):
        oracle.decode_chunk(0, 2, b"XXXX" + bits[4:], 64, 64, blob)
    with pytest.raises(RuntimeError):
        oracle.decode_chunk(0, 2, bits[:-4], 64, 64, blob)
    with pytest.raises(RuntimeError):                     # wrong shape for this stream
        oracle.decode_chunk(0, 2, bits, 64, 48, blob)
