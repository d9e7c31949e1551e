"""GPU parity of the temporal chunk context (Sec. 3.1, Fig. 3) against the FP64 oracle, through the C ABI.

A stream of chunks is coded with the context carried between them (encoder and decoder each keep their
own).  Bars:
  * the encoder's C_{i+1} equals the decoder's bit for bit (both precisions);
  * FP32, staged on the GPU's own C_i and intermediates: y, mu, log sigma within 1e-4 * max(1, |v|),
    C_{i+1} within 1e-4 * max(1, |v|), frames within 1e-3 of the oracle's decoders given the GPU's y^;
  * BF16: C_{i+1} within 0.03 max|ref| elementwise and 0.01 RMS(ref) of the oracle's on the GPU's y^ and
    C_i; PSNR within 0.05 dB and stream size within 2 % of the FP32 temporal path;
  * both: bit-stream sections byte-equal to the oracle's rANS of the GPU's symbols; all-zero temporal
    weights give the plain codec's sections and frames exactly; version mismatches reported.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests._util import parse_container, psnr

pytestmark = pytest.mark.gpu

TOL_REL = 1e-4


def U():
    from paper_2606_04410_b300 import ufvc
    return ufvc


def _chunks(n, N, H, W, seed=0):
    if H <= 64:
        return [synthetic.moving_texture(seed + 60 + i, N, H, W, max_step=3, period=64) for i in range(n)]
    return [synthetic.moving_texture(seed + 60 + i, N, H, W, max_step=16, refresh=0.1) for i in range(n)]


def _close(g, o, what):
    g = np.asarray(g, np.float64)
    err = np.abs(g - o)
    bound = TOL_REL * np.maximum(1.0, np.abs(o))
    assert (err <= bound).all(), f"{what}: max err {err.max():.3g}"
    return float(err.max())


@pytest.mark.parametrize("arch,N,H,W,K", [(0, 2, 64, 64, 32), (1, 2, 96, 160, 256)])
def test_temporal_sequence_fp32(arch, N, H, W, K):
    u = U()
    blob = synthetic.draw_weights(arch, N, seed=7)
    tw = synthetic.draw_temporal_weights(arch, N, seed=1)
    codec = u.Codec(arch, N, K, blob, "fp32", temporal_weights=tw)
    dev = torch.device("cuda:0")
    q = oracle.qstep(32)
    ce = [codec.new_context(W, H), codec.new_context(W, H)]
    cd = [codec.new_context(W, H), codec.new_context(W, H)]
    assert ce[0].numel() * 4 == codec.context_bytes(W, H)
    report = {}
    for i, frames in enumerate(_chunks(3, N, H, W)):
        cin_e = None if i == 0 else ce[i % 2]
        cin_d = None if i == 0 else cd[i % 2]
        fr = torch.from_numpy(frames).to(dev)
        st = {k: v.cpu().numpy() for k, v in codec.encode_stages(fr, 32, ctx_in=cin_e).items()}
        bits, nb = codec.encode_chunk_tc(fr, cin_e, ce[(i + 1) % 2], 32)
        n = int(nb.item())
        rec = codec.decode_chunk_tc(bits, n, W, H, cin_d, cd[(i + 1) % 2], f32=True).cpu().numpy()
        assert codec.sync_status() == 0
        assert torch.equal(ce[(i + 1) % 2], cd[(i + 1) % 2]), "encoder must track the decoder's context"
        raw = bits[:n].cpu().numpy().tobytes()
        assert raw[4] == 3
        c_in = None if i == 0 else cin_e.double().cpu().numpy()
        H8, W8, _ = oracle.context_dims(arch, H, W)
        # encoder conditioning: y from the oracle with the GPU's context
        _, _, dbg = oracle.encode_chunk_t(arch, frames, 32, K, blob, tw, c_in, debug=True)
        report[f"y{i}"] = _close(st["y"], dbg["y"], "y")
        # prior conditioning, staged on the GPU's z^
        _, pc = oracle.context_terms(arch, N, c_in, H8, W8, tw)
        Hy, Wy = st["y"].shape[:2]
        mu_o, ls_o, _ = oracle.hyper_synthesis_add(arch, N, st["zhat"], Hy, Wy, blob, pc)
        report[f"mu{i}"] = _close(st["mu"], mu_o, "mu")
        _close(st["logsig"], ls_o, "logsig")
        # the single coding step
        c = parse_container(raw, codec.Cz)
        assert oracle.rans_encode(st["rhat"].ravel(), st["idx"].ravel(), K) == c["ysec"]
        # chunk feature, next context and frame decoders on the GPU's y^
        yhat = st["rhat"].astype(np.float64) * q + st["mu"]
        Fo = oracle.chunk_feature(arch, N, yhat, tw, c_in)
        report[f"ctx{i}"] = _close(ce[(i + 1) % 2].cpu().numpy(), oracle.context_next(arch, N, Fo, tw), "context")
        rec_o = oracle.synthesis_f(arch, N, yhat, Fo, H, W, blob, tw)
        report[f"rec{i}"] = float(np.abs(rec - rec_o).max())
        assert report[f"rec{i}"] <= 1e-3
    print("temporal fp32", (arch, N, H, W), report)


def _bf_ctx_check(arch, N, yhat, c_in, tw, c_gpu):
    Fo = oracle.chunk_feature(arch, N, yhat, tw, c_in)
    ref = oracle.context_next(arch, N, Fo, tw)
    err = np.abs(c_gpu - ref)
    assert err.max() <= 0.03 * np.abs(ref).max(), (err.max(), np.abs(ref).max())
    assert np.sqrt(np.mean(err ** 2)) <= 0.01 * np.sqrt(np.mean(ref ** 2)) + 1e-6
    return float(err.max())


@pytest.mark.parametrize("N,H,W,K", [(2, 200, 328, 256), (8, 128, 160, 4096)])
def test_temporal_sequence_bf16(N, H, W, K):
    u = U()
    blob = synthetic.draw_weights(1, N, seed=7)
    tw = synthetic.draw_temporal_weights(1, N, seed=2)
    dev = torch.device("cuda:0")
    res = {}
    for prec in ("bf16", "fp32"):
        codec = u.Codec(1, N, K, blob, prec, temporal_weights=tw)
        ce = [codec.new_context(W, H), codec.new_context(W, H)]
        cd = [codec.new_context(W, H), codec.new_context(W, H)]
        sizes, psnrs, errs = [], [], []
        for i, frames in enumerate(_chunks(3, N, H, W, seed=5)):
            cin_e = None if i == 0 else ce[i % 2]
            cin_d = None if i == 0 else cd[i % 2]
            fr = torch.from_numpy(frames).to(dev)
            st = {k: v.cpu().numpy() for k, v in codec.encode_stages(fr, 32, ctx_in=cin_e).items()} \
                if prec == "bf16" else None
            bits, nb = codec.encode_chunk_tc(fr, cin_e, ce[(i + 1) % 2], 32)
            # the size read on the device (the stream size changes from chunk to chunk)
            rec = codec.decode_chunk_tc(bits, bits.numel(), W, H, cin_d, cd[(i + 1) % 2], f32=True,
                                        d_nbytes=nb).cpu().numpy()
            assert codec.sync_status() == 0
            n = int(nb.item())
            assert torch.equal(ce[(i + 1) % 2], cd[(i + 1) % 2])
            if st is not None:
                raw = bits[:n].cpu().numpy().tobytes()
                c = parse_container(raw, codec.Cz)
                assert oracle.rans_encode(st["rhat"].ravel(), st["idx"].ravel(), K) == c["ysec"]
                yhat = st["rhat"].astype(np.float64) + st["mu"]
                c_in = None if i == 0 else cin_e.float().cpu().numpy().astype(np.float64)
                errs.append(_bf_ctx_check(1, N, yhat, c_in, tw, ce[(i + 1) % 2].float().cpu().numpy()))
            sizes.append(n)
            psnrs.append(psnr(rec, frames / 255.0))
        res[prec] = (sizes, psnrs, errs)
    dps = np.mean(res["bf16"][1]) - np.mean(res["fp32"][1])
    dbr = (sum(res["bf16"][0]) - sum(res["fp32"][0])) / sum(res["fp32"][0])
    print("temporal bf16 vs fp32", (N, H, W), res, "dpsnr", dps, "dbitrate", dbr)
    assert abs(dps) < 0.05
    assert abs(dbr) < 0.02


@pytest.mark.parametrize("prec,arch,N,H,W,K", [("fp32", 0, 2, 64, 64, 32), ("bf16", 1, 2, 128, 192, 256)])
def test_zero_temporal_weights_equal_plain(prec, arch, N, H, W, K):
    u = U()
    blob = synthetic.draw_weights(arch, N, seed=3)
    tw0 = np.zeros(u.temporal_weight_count(arch, N), np.float32)
    t = u.Codec(arch, N, K, blob, prec, temporal_weights=tw0)
    p = u.Codec(arch, N, K, blob, prec)
    frames = _chunks(1, N, H, W, seed=9)[0]
    fr = torch.from_numpy(frames).cuda()
    c_in = t.new_context(W, H).normal_()
    c_out = t.new_context(W, H)
    bt, nt = t.encode_chunk_tc(fr, c_in, c_out, 32)
    bp, npl = p.encode_chunk(fr, 32)
    assert t.sync_status() == 0 and p.sync_status() == 0
    rt, rp = bt[:int(nt.item())].cpu().numpy().tobytes(), bp[:int(npl.item())].cpu().numpy().tobytes()
    assert rt[4] == 3 and rp[4] == 1 and rt[5:] == rp[5:]
    ot = t.decode_chunk_tc(bt, int(nt.item()), W, H, c_in, c_out)
    op = p.decode_chunk(bp, int(npl.item()), W, H)
    assert t.sync_status() == 0
    assert torch.equal(ot, op)
    assert torch.count_nonzero(c_out) == 0  # GELU(0)
    # version mismatches are reported, not decoded
    p.decode_chunk(bt, int(nt.item()), W, H)
    assert p.sync_status() == u.UFVC_ERR_UNSUPPORTED
    t.decode_chunk(bp, int(npl.item()), W, H)
    assert t.sync_status() == u.UFVC_ERR_UNSUPPORTED


def test_temporal_argument_checks():
    u = U()
    blob = synthetic.draw_weights(1, 2, seed=0)
    tw = synthetic.draw_temporal_weights(1, 2, seed=0)
    c8 = u.Codec(1, 2, 64, blob, "fp8")
    assert u.lib.ufvc_set_temporal_context(c8.h, u._ptr(tw), tw.size) == u.UFVC_ERR_UNSUPPORTED
    p = u.Codec(1, 2, 64, blob, "bf16")
    fr = torch.zeros((2, 64, 64, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(u.UfvcError):
        p.encode_chunk_tc(fr, None, None, 32)  # no temporal context set
    t = u.Codec(1, 2, 64, blob, "bf16", temporal_weights=tw)
    c = t.new_context(64, 64)
    with pytest.raises(u.UfvcError):
        t.encode_chunk_tc(fr, c, c, 32)  # in and out must differ
    raw = torch.zeros(c.numel() * 2 + 16, dtype=torch.uint8, device="cuda")
    bits = torch.empty(t.max_bitstream_bytes(64, 64), dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = u.lib.ufvc_encode_chunk_tc(t.h, u._ptr(fr), 2, 64, 64, 32, u._ptr(bits), bits.numel(), u._ptr(nb),
                                    u.C.c_void_p(raw.data_ptr() + 2), None, u._stream(None))
    assert rc == u.UFVC_ERR_ARG  # misaligned context
