"""GPU parity of the progressive means (Sec. 3.4, Fig. 4a/4c) against the FP64 oracle, through the C ABI.

Bars (written out in each check):
  * FP32 contexts: each step's means within 1e-4 * max(1, |oracle|) of the oracle's mean step evaluated
    on the GPU's own reconstruction of the earlier partitions (staged, so one legitimate rounding
    crossing does not cascade); r^ equal to the oracle's rounding except inside the half-integer band
    tau = 1e-4 * max(1, |v|) (counted);
  * BF16 contexts (bf16 operands and hidden layer, FP32 accumulation): staged means within
    0.03 * max|oracle| elementwise and 0.01 * RMS(oracle) in RMS;
  * in both: y^ = r^ q + mu exactly, the decoder form repeats the encoder's means and y^ bit for bit,
    bit-stream sections byte-equal to the oracle's rANS of the GPU's symbols, and a decoded chunk
    bit-identical to synthesising the encoder's r^ q + mu.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests._util import near_half_integer, parse_container, psnr

pytestmark = pytest.mark.gpu

TOL_REL = 1e-4
TAU = 1e-4


def U():
    from paper_2606_04410_b300 import ufvc
    return ufvc


def _stage_inputs(arch, Hy, Wy, seed):
    rng = np.random.default_rng(seed)
    cy, cz = {0: (128, 64), 1: (256, 128)}[arch]
    y = rng.normal(0, 2.0, (Hy, Wy, cy)).astype(np.float32)
    mu0 = rng.normal(0, 0.5, (Hy, Wy, cy)).astype(np.float32)
    s = np.maximum(rng.normal(0, 0.7, (Hy, Wy, cz)), -0.17).astype(np.float32)
    return y, mu0, s


def _check_staged(arch, y, mu0, s, qp, r, mu, yhat, mw, bf16, report):
    """Partition by partition, against the oracle's mean step on the GPU's earlier partitions."""
    Hy, Wy, cy = mu0.shape
    part = oracle.partition_map(Hy, Wy, cy)
    q = oracle.qstep(qp)
    # y^ = r^ q + mu in FP32, exactly as the kernels round it
    np.testing.assert_array_equal(yhat, (r.astype(np.float32) * np.float32(q)).astype(np.float32) + mu)
    np.testing.assert_array_equal(mu[part == 0], mu0[part == 0])
    yh64 = yhat.astype(np.float64)
    mism = 0
    for k in (1, 2, 3):
        ref = oracle.mean_step(arch, k, yh64, s.astype(np.float64), mw)
        sel = part == k
        g, o = mu[sel].astype(np.float64), ref[sel]
        err = np.abs(g - o)
        if bf16:
            assert err.max() <= 0.03 * np.abs(o).max(), (k, err.max(), np.abs(o).max())
            assert np.sqrt(np.mean(err ** 2)) <= 0.01 * np.sqrt(np.mean(o ** 2))
        else:
            bound = TOL_REL * np.maximum(1.0, np.abs(o))
            assert (err <= bound).all(), (k, err.max())
        report[f"mu{k}_max_err"] = float(err.max())
        if y is not None:
            # r^ against the oracle's rounding of (y - mu^k) / q; the GPU's own mean decides in BF16
            v = (y[sel].astype(np.float64) - (g if bf16 else o)) / q
            exp = np.clip(np.rint(v), -255, 255)
            diff = r[sel].astype(np.int64) != exp
            band = near_half_integer(v, TAU * np.maximum(1.0, np.abs(v)))
            assert not (diff & ~band).any(), (k, int((diff & ~band).sum()))
            mism += int(diff.sum())
    if y is not None:
        v0 = (y[part == 0].astype(np.float64) - mu0[part == 0]) / q
        exp0 = np.clip(np.rint(v0), -255, 255)
        d0 = r[part == 0].astype(np.int64) != exp0
        assert not (d0 & ~near_half_integer(v0, TAU * np.maximum(1.0, np.abs(v0)))).any()
        report["rhat_boundary_mismatches"] = mism + int(d0.sum())


@pytest.mark.parametrize("arch,prec,Hy,Wy,qp", [(0, "fp32", 4, 4, 32), (0, "fp32", 7, 5, 40), (1, "fp32", 9, 13, 32),
                                                (1, "bf16", 17, 30, 32), (1, "bf16", 8, 120, 27), (1, "fp8", 5, 7, 32)])
def test_progressive_stage_vs_oracle(arch, prec, Hy, Wy, qp):
    u = U()
    N = 2
    blob = synthetic.draw_weights(arch, N, seed=3)
    mw = synthetic.draw_mean_weights(arch, seed=5)
    codec = u.Codec(arch, N, 64, blob, prec, mean_weights=mw)
    if prec == "fp8":  # the stage call needs no calibration: the mean network stays on bf16 operands
        pass
    y, mu0, s = _stage_inputs(arch, Hy, Wy, seed=Hy * 100 + Wy)
    dev = torch.device("cuda:0")
    yt, mt, st = (torch.from_numpy(a).to(dev) for a in (y, mu0, s))
    r, mu, yhat = (t.cpu().numpy() for t in codec.progressive_means(mt, st, qp, y=yt))
    report = {}
    _check_staged(arch, y, mu0, s, qp, r, mu, yhat, mw, prec != "fp32", report)
    # decoder form: the same r^ gives the same means and reconstruction, bit for bit
    r2, mu2, yhat2 = (t.cpu().numpy() for t in codec.progressive_means(mt, st, qp, rhat=torch.from_numpy(r).to(dev)))
    np.testing.assert_array_equal(r2, r)
    np.testing.assert_array_equal(mu2, mu)
    np.testing.assert_array_equal(yhat2, yhat)
    print("progressive stage report", (arch, prec, Hy, Wy, qp), report)


def _encode(codec, fr, qp):
    bits, nb = codec.encode_chunk(fr, qp)
    assert codec.sync_status() == 0
    n = int(nb.item())
    return bits, n, bits[:n].cpu().numpy().tobytes()


@pytest.mark.parametrize("arch,N,H,W,qp,K,prec", [(0, 2, 64, 64, 32, 32, "fp32"), (1, 2, 200, 328, 32, 256, "fp32"),
                                                  (1, 2, 200, 328, 32, 256, "bf16"), (1, 8, 128, 160, 32, 4096, "bf16")])
def test_progressive_chunk(arch, N, H, W, qp, K, prec):
    u = U()
    frames = synthetic.moving_texture(200 + H, N, H, W, max_step=3 if H <= 64 else 16, period=64) if H <= 64 else \
        synthetic.moving_texture(200 + H, N, H, W, max_step=16, refresh=0.1)
    blob = synthetic.draw_weights(arch, N, seed=7)
    mw = synthetic.draw_mean_weights(arch, seed=0)
    pm = u.Codec(arch, N, K, blob, prec, mean_weights=mw)
    plain = u.Codec(arch, N, K, blob, prec)
    dev = torch.device("cuda:0")
    fr = torch.from_numpy(frames).to(dev)
    st = {k: v.cpu().numpy() for k, v in pm.encode_stages(fr, qp).items()}
    bits_t, n, raw = _encode(pm, fr, qp)
    assert raw[4] == 2
    c = parse_container(raw, pm.Cz)
    assert c["total"] == n
    # the single coding step over the whole latent: sections = oracle rANS of the GPU's symbols
    assert oracle.rans_encode(st["rhat"].ravel(), st["idx"].ravel(), K) == c["ysec"]
    zidx = np.tile(st["iz"], st["zhat"].size // st["iz"].size)
    assert oracle.rans_encode(st["zhat"].ravel(), zidx, c["Kz"]) == c["zsec"]
    # scales and partition-0 means are the single pass's (FP32, from the GPU's z^)
    Hy, Wy = st["mu"].shape[:2]
    mu0_o, ls_o, s_o = oracle.hyper_synthesis(arch, N, st["zhat"], Hy, Wy, blob, want_s=True)
    part = oracle.partition_map(Hy, Wy, st["mu"].shape[2])
    err0 = np.abs(st["mu"][part == 0] - mu0_o[part == 0])
    assert (err0 <= TOL_REL * np.maximum(1.0, np.abs(mu0_o[part == 0]))).all()
    # staged means of partitions 1..3 (GPU y^ of the earlier partitions, oracle s from the GPU's z^)
    q = oracle.qstep(qp)
    yhat = (st["rhat"].astype(np.float32) * np.float32(q)).astype(np.float32) + st["mu"]
    report = {}
    _check_staged(arch, None, st["mu"], s_o.astype(np.float32), qp, st["rhat"], st["mu"], yhat, mw, prec != "fp32",
                  report)
    # r^ of partitions 1..3 follow the GPU's own means
    y = st["y"]
    exp = np.clip(np.rint((y.astype(np.float64) - st["mu"]) / q), -255, 255)
    band = near_half_integer((y.astype(np.float64) - st["mu"]) / q, TAU)
    assert not ((st["rhat"] != exp) & ~band).any()
    # decode: lossless, and the decoder repeats the encoder's means (bit-identical frames)
    rec = pm.decode_chunk(bits_t, n, W, H, f32=True)
    assert pm.sync_status() == 0
    rec2 = pm.synthesize(torch.from_numpy(yhat).to(dev), W, H)
    torch.cuda.synchronize()
    assert torch.equal(rec, rec2), "decoder must reproduce the encoder's progressive means exactly"
    if prec == "fp32":
        rec_o = oracle.synthesis(arch, N, yhat.astype(np.float64), H, W, blob)
        report["recon_max_err"] = float(np.abs(rec.cpu().numpy() - rec_o).max())
        assert report["recon_max_err"] <= 1e-3
    # single-pass stream of the same chunk: same scales, so same z^ section; compare rate and quality
    bits1_t, n1, raw1 = _encode(plain, fr, qp)
    assert raw1[4] == 1 and c["zsec"] == parse_container(raw1, pm.Cz)["zsec"]
    rec1 = plain.decode_chunk(bits1_t, n1, W, H, f32=True)
    # a mean-network context decodes version-1 streams as the single pass does
    rec1b = pm.decode_chunk(bits1_t, n1, W, H, f32=True)
    assert pm.sync_status() == 0 and plain.sync_status() == 0
    assert torch.equal(rec1, rec1b)
    # a context without the mean network refuses version 2 (status word, no fault)
    plain.decode_chunk(bits_t, n, W, H, f32=True)
    assert plain.sync_status() == u.UFVC_ERR_UNSUPPORTED
    report.update(bytes_pm=n, bytes_single=n1, dbitrate=(n - n1) / n1,
                  psnr_pm=psnr(rec.cpu().numpy(), frames / 255.0), psnr_single=psnr(rec1.cpu().numpy(), frames / 255.0))
    print("progressive chunk report", (arch, N, H, W, prec), report)


def test_set_progressive_means_rejects_bad_counts():
    u = U()
    blob = synthetic.draw_weights(0, 2, seed=0)
    codec = u.Codec(0, 2, 32, blob, "fp32")
    bad = np.zeros(u.mean_weight_count(0) - 1, np.float32)
    rc = u.lib.ufvc_set_progressive_means(codec.h, u._ptr(bad), bad.size)
    assert rc == u.UFVC_ERR_ARG
    mw = synthetic.draw_mean_weights(0, seed=0)
    assert u.lib.ufvc_set_progressive_means(codec.h, u._ptr(mw), mw.size) == 0
    assert u.lib.ufvc_set_progressive_means(codec.h, u._ptr(mw), mw.size) == u.UFVC_ERR_ARG
