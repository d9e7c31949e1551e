"""GPU parity of the colour interface (Appendix: YUV444 model interface, BT.709 for RGB, YUV420 chroma).

Bars:
  * FP32 latent from each format's frames within 1e-4 * max(1, |oracle|) of the oracle's analysis of its
    own colour conversion (the conversion is FP32 on the GPU, FP64 in the oracle);
  * decoded values in each format within 2e-6 of the oracle's conversion of the GPU's own YUV444
    reconstruction (float vs double arithmetic of one 3x3 matrix or one 2x2 mean), and that
    reconstruction within 1e-3 of the oracle's synthesis of the same y^;
  * bytes = rint(255 v) of the float output of the same decode, exactly;
  * exact equalities in every precision: a YUV444-planar chunk and a YUV420 chunk whose chroma,
    replicated, equals an interleaved chunk give bit-identical bit-streams to that interleaved chunk,
    and the planar output bytes are the interleaved output bytes rearranged.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests._util import psnr

pytestmark = pytest.mark.gpu


def U():
    from paper_2606_04410_b300 import ufvc
    return ufvc


def _layouts(rgb):
    """The same byte values as interleaved, YUV444 planar and (chroma subsampled) YUV420 chunks, plus the
    interleaved chunk that the YUV420 one stands for (chroma repeated over its 2x2 blocks)."""
    N, H, W, _ = rgb.shape
    planar = np.ascontiguousarray(np.moveaxis(rgb, 3, 1))
    u, v = rgb[:, ::2, ::2, 1], rgb[:, ::2, ::2, 2]
    i420 = np.concatenate([rgb[..., 0].reshape(N, -1), u.reshape(N, -1), v.reshape(N, -1)], axis=1)
    rep = rgb.copy()
    rep[..., 1] = np.repeat(np.repeat(u, 2, axis=1), 2, axis=2)[:, :H, :W]
    rep[..., 2] = np.repeat(np.repeat(v, 2, axis=1), 2, axis=2)[:, :H, :W]
    return planar, np.ascontiguousarray(i420), rep


def _as_input(u, fmt, rgb):
    planar, i420, _ = _layouts(rgb)
    return {u.COLOR_RGB: rgb, u.COLOR_RGB_BT709: rgb, u.COLOR_YUV444P: planar, u.COLOR_YUV420P: i420}[fmt]


@pytest.mark.parametrize("fmt", [1, 2, 3])
@pytest.mark.parametrize("arch,N,H,W,K", [(0, 2, 64, 64, 32), (0, 2, 61, 45, 16)])
def test_color_fp32_parity(fmt, arch, N, H, W, K):
    u = U()
    rgb = synthetic.moving_texture(300 + H, N, H, W, max_step=3, period=64)
    blob = synthetic.draw_weights(arch, N, seed=11)
    frames = _as_input(u, fmt, rgb)
    codec = u.Codec(arch, N, K, blob, "fp32", color=fmt)
    dev = torch.device("cuda:0")
    fr = torch.from_numpy(frames).to(dev)
    qp = 32
    st = {k: v.cpu().numpy() for k, v in codec.encode_stages(fr, qp, width=W, height=H).items()}
    x_o = oracle.color_in(fmt, frames, N, H, W)
    y_o = oracle.analysis_x(arch, x_o, blob)
    err = np.abs(st["y"] - y_o)
    assert (err <= 1e-4 * np.maximum(1.0, np.abs(y_o))).all(), err.max()
    bits, nb = codec.encode_chunk(fr, qp, width=W, height=H)
    assert codec.sync_status() == 0
    n = int(nb.item())
    out_f = codec.decode_chunk(bits, n, W, H, f32=True).cpu().numpy().ravel()
    out_b = codec.decode_chunk(bits, n, W, H).cpu().numpy().ravel()
    assert codec.sync_status() == 0
    # the same stream decoded to YUV444 planar floats = the network's reconstruction x^
    c444 = u.Codec(arch, N, K, blob, "fp32", color=u.COLOR_YUV444P)
    xh = np.moveaxis(c444.decode_chunk(bits, n, W, H, f32=True).cpu().numpy(), 1, 3)
    assert c444.sync_status() == 0
    yhat = st["rhat"].astype(np.float64) * oracle.qstep(qp) + st["mu"]
    rec_o = oracle.synthesis(arch, N, yhat, H, W, blob)
    assert np.abs(xh - rec_o).max() <= 1e-3
    ref = oracle.color_out(fmt, xh.astype(np.float64), N, H, W)
    assert out_f.size == N * u.frame_bytes(fmt, W, H) == ref.size
    assert np.abs(out_f - ref).max() <= 2e-6, np.abs(out_f - ref).max()
    np.testing.assert_array_equal(out_b, np.rint(np.float32(255.0) * out_f.astype(np.float32)).astype(np.uint8))
    # host-buffer calls give the same bytes
    hb = codec.encode_chunk_host(frames, qp, width=W, height=H)
    assert hb == bits[:n].cpu().numpy().tobytes()
    np.testing.assert_array_equal(np.asarray(codec.decode_chunk_host(hb, W, H)).ravel(), out_b)
    print("color fp32", (fmt, arch, N, H, W), "y err", float(err.max()), "psnr in format",
          psnr(out_f, frames.ravel() / 255.0))


@pytest.mark.parametrize("prec,arch,N,H,W,K", [("fp32", 0, 2, 63, 47, 32), ("bf16", 1, 2, 200, 328, 256),
                                               ("bf16", 1, 8, 128, 160, 4096), ("fp8", 1, 2, 128, 192, 256)])
def test_planar_and_420_equal_interleaved(prec, arch, N, H, W, K):
    u = U()
    rgb = synthetic.moving_texture(400 + H, N, H, W, max_step=16, refresh=0.1)
    blob = synthetic.draw_weights(arch, N, seed=5)
    planar, i420, rep = _layouts(rgb)
    dev = torch.device("cuda:0")
    codecs = {f: u.Codec(arch, N, K, blob, prec, color=f) for f in (u.COLOR_RGB, u.COLOR_YUV444P, u.COLOR_YUV420P)}
    if prec == "fp8":
        for f, c in codecs.items():  # same activation scales for all three: calibrate on the same chunk
            c.calibrate_fp8(torch.from_numpy(_as_input(u, f, rep)).to(dev), 32, width=W, height=H)
    streams = {}
    for f, src in ((u.COLOR_RGB, rgb), (u.COLOR_YUV444P, planar), (u.COLOR_RGB, rep), (u.COLOR_YUV420P, i420)):
        bits, nb = codecs[f].encode_chunk(torch.from_numpy(src).to(dev), 32, width=W, height=H)
        assert codecs[f].sync_status() == 0
        streams.setdefault(f, []).append(bits[:int(nb.item())].cpu().numpy().tobytes())
    assert streams[u.COLOR_RGB][0] == streams[u.COLOR_YUV444P][0]
    assert streams[u.COLOR_RGB][1] == streams[u.COLOR_YUV420P][0]
    # decode: planar output = interleaved output rearranged, byte for byte
    raw = streams[u.COLOR_RGB][0]
    bt = torch.from_numpy(np.frombuffer(raw, np.uint8).copy()).to(dev)
    o_rgb = codecs[u.COLOR_RGB].decode_chunk(bt, len(raw), W, H).cpu().numpy()
    o_pl = codecs[u.COLOR_YUV444P].decode_chunk(bt, len(raw), W, H).cpu().numpy()
    o_420 = codecs[u.COLOR_YUV420P].decode_chunk(bt, len(raw), W, H).cpu().numpy()
    assert all(c.sync_status() == 0 for c in codecs.values())
    np.testing.assert_array_equal(o_pl, np.moveaxis(o_rgb, 3, 1))
    np.testing.assert_array_equal(o_420[:, :H * W], o_rgb[..., 0].reshape(N, -1))
    # chroma of the YUV420 output: within one step of rint(255 * block mean) of the interleaved bytes
    # (those bytes are rounded once already)
    Hc, Wc = (H + 1) // 2, (W + 1) // 2
    cu = o_420[:, H * W:H * W + Hc * Wc].reshape(N, Hc, Wc).astype(np.float64)
    pad = np.pad(o_rgb[..., 1].astype(np.float64), ((0, 0), (0, 2 * Hc - H), (0, 2 * Wc - W)), mode="edge")
    m = pad.reshape(N, Hc, 2, Wc, 2).mean(axis=(2, 4))
    assert np.abs(cu - m).max() <= 1.0


@pytest.mark.parametrize("fmt", [1, 3])
def test_bf16_color_chunk_against_fp32(fmt):
    u = U()
    N, H, W, K = 2, 200, 328, 256
    rgb = synthetic.moving_texture(500, N, H, W, max_step=16, refresh=0.1)
    frames = _as_input(u, fmt, rgb)
    blob = synthetic.draw_weights(1, N, seed=7)
    dev = torch.device("cuda:0")
    fr = torch.from_numpy(frames).to(dev)
    res = {}
    for prec in ("bf16", "fp32"):
        c = u.Codec(1, N, K, blob, prec, color=fmt)
        bits, nb = c.encode_chunk(fr, 32, width=W, height=H)
        n = int(nb.item())
        out = c.decode_chunk(bits, n, W, H, f32=True).cpu().numpy().ravel()
        assert c.sync_status() == 0
        res[prec] = (n, psnr(out, frames.ravel() / 255.0))
    dps = res["bf16"][1] - res["fp32"][1]
    dbr = (res["bf16"][0] - res["fp32"][0]) / res["fp32"][0]
    print("bf16 vs fp32 in format", fmt, res, "dpsnr", dps, "dbitrate", dbr)
    assert abs(dps) < 0.05
    assert abs(dbr) < 0.01


def test_set_color_format_rejects_unknown():
    u = U()
    c = u.Codec(0, 2, 32, synthetic.draw_weights(0, 2, seed=0), "fp32")
    assert u.lib.ufvc_set_color_format(c.h, 4) == u.UFVC_ERR_ARG
    assert u.frame_bytes(4, 8, 8) == 0 and u.frame_bytes(3, 5, 3) == 15 + 2 * 3 * 2
