"""GPU parity of the DC-block model (arch 2: HT-S block counts, Appendix) against the FP64 oracle, through the
C ABI.  Chunks are coded as a stream: the model always carries its temporal context.

Bars:
  * FP32, staged on the GPU's own context and intermediates: y, mu, log sigma within 1e-4 * max(1, |v|);
    the next context within 1e-4 * max(1, |v|); frames within 1e-3 of the oracle's frame decoders given
    the GPU's y^ (the trunk is over 90 layers deep; FP32 rounding stays far below these bars);
  * BF16: the next context within 0.05 RMS(ref) of the oracle's on the GPU's y^ and context; PSNR within
    0.1 dB and stream size within 3 % of the FP32 DC path over the stream;
  * both: the encoder's next context equals the decoder's bit for bit; bit-stream sections byte-equal to
    the oracle's rANS of the GPU's symbols; a YUV444-planar chunk codes exactly like the interleaved one.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests._util import parse_container, psnr

pytestmark = pytest.mark.gpu

N = 8


def U():
    from paper_2606_04410_b300 import ufvc
    return ufvc


def _close(g, o, what, tol=1e-4):
    g = np.asarray(g, np.float64)
    err = np.abs(g - o)
    bound = tol * np.maximum(1.0, np.abs(o))
    assert (err <= bound).all(), f"{what}: max err {err.max():.3g} (|ref| max {np.abs(o).max():.3g})"
    return float(err.max())


def _chunks(n, H, W, seed):
    return [synthetic.moving_texture(seed + i, N, H, W, max_step=3, period=64) for i in range(n)]


def test_dc_fp32_chain_vs_oracle():
    u = U()
    H, W, K = 64, 64, 64
    blob = synthetic.draw_dc_weights(N, seed=0)
    codec = u.Codec(2, N, K, blob, "fp32")
    ce = [codec.new_context(W, H), codec.new_context(W, H)]
    cd = [codec.new_context(W, H), codec.new_context(W, H)]
    assert ce[0].shape[2] == 128
    report = {}
    for i, frames in enumerate(_chunks(3, H, W, 90)):
        cin_e, cin_d = (None, None) if i == 0 else (ce[i % 2], cd[i % 2])
        fr = torch.from_numpy(frames).cuda()
        st = {k: v.cpu().numpy() for k, v in codec.encode_stages(fr, 32, ctx_in=cin_e).items()}
        bits, nb = codec.encode_chunk_tc(fr, cin_e, ce[(i + 1) % 2], 32)
        n = int(nb.item())
        rec = codec.decode_chunk_tc(bits, n, W, H, cin_d, cd[(i + 1) % 2], f32=True).cpu().numpy()
        assert codec.sync_status() == 0
        assert torch.equal(ce[(i + 1) % 2], cd[(i + 1) % 2])
        raw = bits[:n].cpu().numpy().tobytes()
        assert raw[4] == 3 and raw[5] == 2
        c_in = None if i == 0 else cin_e.double().cpu().numpy()
        report[f"y{i}"] = _close(st["y"], oracle.dc_analysis(N, frames / 255.0, blob, c_in), "y")
        Hy, Wy = st["y"].shape[:2]
        pc = oracle.dc_prior_term(N, c_in, 2 * Hy, 2 * Wy, blob)
        mu_o, ls_o, _ = oracle.hyper_synthesis_add(2, N, st["zhat"], Hy, Wy, blob, pc)
        report[f"mu{i}"] = _close(st["mu"], mu_o, "mu")
        _close(st["logsig"], ls_o, "logsig")
        c = parse_container(raw, codec.Cz)
        assert oracle.rans_encode(st["rhat"].ravel(), st["idx"].ravel(), K) == c["ysec"]
        yhat = st["rhat"].astype(np.float64) + st["mu"]
        F_, c_next = oracle.dc_trunk(N, yhat, blob, c_in)
        report[f"ctx{i}"] = _close(ce[(i + 1) % 2].cpu().numpy(), c_next, "context")
        rec_o = oracle.dc_frames(N, F_, H, W, blob)
        report[f"rec{i}"] = float(np.abs(rec - rec_o).max())
        assert report[f"rec{i}"] <= 1e-3
    print("dc fp32", report)


def test_dc_bf16_chain():
    u = U()
    H, W, K = 64, 96, 256
    blob = synthetic.draw_dc_weights(N, seed=1)
    res = {}
    for prec in ("bf16", "fp32"):
        codec = u.Codec(2, N, K, blob, prec)
        ce = [codec.new_context(W, H), codec.new_context(W, H)]
        cd = [codec.new_context(W, H), codec.new_context(W, H)]
        sizes, ps, errs = [], [], []
        for i, frames in enumerate(_chunks(3, H, W, 95)):
            cin_e, cin_d = (None, None) if i == 0 else (ce[i % 2], cd[i % 2])
            fr = torch.from_numpy(frames).cuda()
            st = {k: v.cpu().numpy() for k, v in codec.encode_stages(fr, 32, ctx_in=cin_e).items()} \
                if prec == "bf16" else None
            bits, nb = codec.encode_chunk_tc(fr, cin_e, ce[(i + 1) % 2], 32)
            rec = codec.decode_chunk_tc(bits, bits.numel(), W, H, cin_d, cd[(i + 1) % 2], f32=True,
                                        d_nbytes=nb).cpu().numpy()
            assert codec.sync_status() == 0
            n = int(nb.item())
            assert torch.equal(ce[(i + 1) % 2], cd[(i + 1) % 2])
            if st is not None:
                c = parse_container(bits[:n].cpu().numpy().tobytes(), codec.Cz)
                assert oracle.rans_encode(st["rhat"].ravel(), st["idx"].ravel(), K) == c["ysec"]
                c_in = None if i == 0 else cin_e.float().cpu().numpy().astype(np.float64)
                _, ref = oracle.dc_trunk(N, st["rhat"] + st["mu"].astype(np.float64), blob, c_in)
                got = ce[(i + 1) % 2].float().cpu().numpy()
                rms = np.sqrt(np.mean((got - ref) ** 2)) / np.sqrt(np.mean(ref ** 2))
                assert rms <= 0.05, rms
                errs.append(float(rms))
            sizes.append(n)
            ps.append(psnr(rec, frames / 255.0))
        res[prec] = (sizes, ps, errs)
    dps = np.mean(res["bf16"][1]) - np.mean(res["fp32"][1])
    dbr = (sum(res["bf16"][0]) - sum(res["fp32"][0])) / sum(res["fp32"][0])
    print("dc bf16 vs fp32", res, "dpsnr", dps, "dbitrate", dbr)
    assert abs(dps) < 0.1
    assert abs(dbr) < 0.03


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_dc_planar_equals_interleaved(prec):
    u = U()
    H, W = 64, 64
    blob = synthetic.draw_dc_weights(N, seed=2)
    rgb = _chunks(1, H, W, 99)[0]
    planar = np.ascontiguousarray(np.moveaxis(rgb, 3, 1))
    a = u.Codec(2, N, 64, blob, prec)
    b = u.Codec(2, N, 64, blob, prec, color=u.COLOR_YUV444P)
    ba, na = a.encode_chunk(torch.from_numpy(rgb).cuda(), 32)
    bb, nb = b.encode_chunk(torch.from_numpy(planar).cuda(), 32)
    assert a.sync_status() == 0 and b.sync_status() == 0
    ra, rb = ba[:int(na.item())].cpu().numpy().tobytes(), bb[:int(nb.item())].cpu().numpy().tobytes()
    assert ra == rb
    oa = a.decode_chunk(ba, int(na.item()), W, H)
    ob = b.decode_chunk(bb, int(nb.item()), W, H)
    assert a.sync_status() == 0 and b.sync_status() == 0
    assert torch.equal(ob.cpu(), oa.cpu().permute(0, 3, 1, 2))


def test_dc_refuses_fp8_and_extra_temporal():
    u = U()
    blob = synthetic.draw_dc_weights(1, seed=0)
    with pytest.raises(u.UfvcError):
        u.Codec(2, 1, 64, blob, "fp8")
    c = u.Codec(2, 1, 64, blob, "bf16")
    tw = np.zeros(u.temporal_weight_count(1, 1), np.float32)
    assert u.lib.ufvc_set_temporal_context(c.h, u._ptr(tw), tw.size) == u.UFVC_ERR_ARG
