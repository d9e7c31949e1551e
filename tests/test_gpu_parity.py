"""GPU parity of the FP32 chunk path against the FP64 oracle, through the C ABI.

Tolerances (FP32 kernels vs FP64 oracle):
  * y, z, mu, log sigma: |gpu - oracle| <= 1e-4 * max(1, |oracle|)  (FP32 rounding through <= 6 layers
    of fan-in <= 2304 stays orders of magnitude below this);
  * rounding decisions (z^, r^, scale indices): must be equal except where the oracle's FP64 value lies
    within tau = 1e-4 * max(1, |v|) of the rounding boundary (half-integer or threshold); such
    mismatches are counted and reported;
  * reconstruction: max |gpu - oracle| <= 1e-3 on [0, 1] pixels;
  * bit-streams: byte-exact (integer work).
Staging: each stage is compared given the GPU's own inputs to that stage (GPU z^ -> oracle
hyper-synthesis, GPU r^ and indices -> oracle rANS, GPU y^ -> oracle synthesis) so that one
legitimate boundary crossing does not cascade.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests._util import near_half_integer, near_threshold, parse_container, psnr

pytestmark = pytest.mark.gpu

TOL_REL = 1e-4
TAU = 1e-4
TOL_RECON = 1e-3


def U():
    from paper_2606_04410_b300 import ufvc
    return ufvc


def _close(gpu, ref, what):
    ref = np.asarray(ref, np.float64)
    err = np.abs(np.asarray(gpu, np.float64) - ref)
    bound = TOL_REL * np.maximum(1.0, np.abs(ref))
    assert (err <= bound).all(), f"{what}: max err {err.max():.3g}, worst ratio {(err / bound).max():.3g}"
    return float(err.max())


def _check_rounding(gpu_int, v_oracle, what, report):
    """Integers equal except inside the half-integer band of the oracle's pre-rounding value."""
    v = np.asarray(v_oracle, np.float64)
    ref = np.clip(np.rint(v), -255, 255)
    diff = np.asarray(gpu_int, np.int64) != ref
    band = near_half_integer(v, TAU * np.maximum(1.0, np.abs(v)))
    assert not (diff & ~band).any(), f"{what}: {int((diff & ~band).sum())} mismatches outside the band"
    assert (np.abs(np.asarray(gpu_int, np.int64) - ref)[diff] <= 1).all()
    report[what + "_boundary_mismatches"] = int(diff.sum())


def _check_index(gpu_idx, logsig_oracle, thr, what, report):
    ls = np.asarray(logsig_oracle, np.float64)
    ref = (thr.astype(np.float64)[None, :] < ls.reshape(-1, 1)).sum(1).reshape(ls.shape)
    diff = np.asarray(gpu_idx, np.int64) != ref
    band = near_threshold(ls, thr, TAU * 4)
    assert not (diff & ~band).any(), f"{what}: {int((diff & ~band).sum())} index mismatches outside the band"
    report[what + "_boundary_mismatches"] = int(diff.sum())


CASES = [  # (arch, N, H, W, qp, K)
    (0, 2, 64, 64, 32, 32),
    (0, 2, 64, 64, 27, 32),
    (1, 2, 200, 328, 32, 256),
    (1, 8, 128, 160, 40, 4096),
]


@pytest.mark.parametrize("arch,N,H,W,qp,K", CASES)
def test_chunk_parity(arch, N, H, W, qp, K):
    u = U()
    frames = synthetic.moving_texture(100 + H, N, H, W, max_step=3, period=64) if H <= 64 else \
        synthetic.moving_texture(100 + H, N, H, W, max_step=16, refresh=0.1)
    blob = synthetic.draw_weights(arch, N, seed=7)
    codec = u.Codec(arch, N, K, blob, "fp32")
    dev = torch.device("cuda:0")
    fr = torch.from_numpy(frames).to(dev)
    st = {k: v.cpu().numpy() for k, v in codec.encode_stages(fr, qp).items()}
    bits_t, nb_t = codec.encode_chunk(fr, qp)
    assert codec.sync_status() == 0
    nbytes = int(nb_t.item())
    bits = bits_t[:nbytes].cpu().numpy().tobytes()
    report = {}
    q = oracle.qstep(qp)

    # --- analysis and hyper-analysis (GPU frames -> oracle FP64)
    y_o = oracle.analysis(arch, frames, blob)
    report["y_max_err"] = _close(st["y"], y_o, "y")
    z_o = oracle.hyper_analysis(arch, N, y_o, blob)
    _check_rounding(st["zhat"], z_o, "zhat", report)
    # per-channel z^ index: exact given the GPU's z^
    _, iz_from_gpu_zhat = oracle.quantize_z(st["zhat"].astype(np.float64))
    np.testing.assert_array_equal(st["iz"], iz_from_gpu_zhat)

    # --- hyper-synthesis, staged on the GPU's z^
    mu_o, ls_o = oracle.hyper_synthesis(arch, N, st["zhat"], y_o.shape[0], y_o.shape[1], blob)
    report["mu_max_err"] = _close(st["mu"], mu_o, "mu")
    report["logsig_max_err"] = _close(st["logsig"], ls_o, "logsig")
    _check_index(st["idx"], ls_o, oracle.thresholds(qp), "idx", report)
    # r^ staged on the GPU's mu: the oracle value (y_oracle - mu_gpu) / q
    _check_rounding(st["rhat"], (y_o - st["mu"].astype(np.float64)) / q, "rhat", report)

    # --- bit-stream: header fields, and both sections byte-equal to the oracle's rANS given the
    #     GPU's symbols and indices; the oracle decodes them back exactly
    c = parse_container(bits, codec.Cz)
    assert c["total"] == nbytes and bits[:4] == b"UFVC"
    assert (c["N"], c["qp"], c["W"], c["H"], c["K"]) == (N, qp, W, H, K)
    np.testing.assert_array_equal(c["iz"], st["iz"])
    nz, ny = st["zhat"].size, st["rhat"].size
    zidx = np.tile(st["iz"], nz // st["iz"].size)
    assert oracle.rans_encode(st["zhat"].ravel(), zidx, c["Kz"]) == c["zsec"]
    assert oracle.rans_encode(st["rhat"].ravel(), st["idx"].ravel(), K) == c["ysec"]
    rdec, _ = oracle.rans_decode(c["ysec"], st["idx"].ravel(), ny, K)
    np.testing.assert_array_equal(rdec, st["rhat"].ravel())

    # --- decode on the GPU: lossless round trip and bit-identical to synthesising r^ q + mu
    rec = codec.decode_chunk(bits_t, nbytes, W, H, f32=True)
    assert codec.sync_status() == 0
    rhat_t = torch.from_numpy(st["rhat"]).to(dev).float()
    yhat_t = (rhat_t * q) + torch.from_numpy(st["mu"]).to(dev)
    rec2 = codec.synthesize(yhat_t, W, H)
    torch.cuda.synchronize()
    assert torch.equal(rec, rec2), "decoder's own hyper-synthesis must reproduce the encoder's mu exactly"

    # --- frame-specific decoders vs oracle on the same y^
    rec_o = oracle.synthesis(arch, N, yhat_t.double().cpu().numpy(), H, W, blob)
    err = np.abs(rec.cpu().numpy() - rec_o)
    report["recon_max_err"] = float(err.max())
    assert err.max() <= TOL_RECON
    # uint8 output = rint(255 x^) of the float output, within 1 LSB of the oracle's
    rec_u8 = codec.decode_chunk(bits_t, nbytes, W, H)
    assert codec.sync_status() == 0
    d = np.abs(rec_u8.cpu().numpy().astype(np.int64) - np.rint(rec_o * 255).astype(np.int64))
    assert d.max() <= 1
    report["psnr_db"] = psnr(rec.cpu().numpy(), frames / 255.0)
    report["bpp"] = 8 * nbytes / (N * H * W)
    print("parity report", (arch, N, H, W, qp, K), report)


def test_oracle_bitstream_decodes_on_gpu():
    """Oracle-encoded stream -> GPU decoder (when both sides' scale indices agree, which they do
    unless an index sits on a threshold; the check below asserts that first)."""
    u = U()
    frames = synthetic.chunk_frames("tiny", seed=3)[:2]
    blob = synthetic.draw_weights(0, 2, seed=1)
    bits_o, dbg = oracle.encode_chunk(0, frames, 32, 32, blob, debug=True)
    codec = u.Codec(0, 2, 32, blob, "fp32")
    zt = torch.from_numpy(dbg["zhat"]).cuda()
    mu_g, ls_g = codec.hyper_synthesis(zt, 4, 4)
    idx_g = (oracle.thresholds(32).astype(np.float64)[None, :] <
             ls_g.cpu().numpy().astype(np.float64).reshape(-1, 1)).sum(1)
    assert (idx_g == dbg["idx"].ravel()).all()
    bt = torch.from_numpy(np.frombuffer(bits_o, np.uint8).copy()).cuda()
    rec = codec.decode_chunk(bt, len(bits_o), 64, 64, f32=True)
    assert codec.sync_status() == 0
    rec_o, _ = oracle.decode_chunk(0, 2, bits_o, 64, 64, blob)
    assert np.abs(rec.cpu().numpy() - rec_o).max() <= TOL_RECON


@pytest.mark.parametrize("n,K", [(8_294_400, 4096), (1_000_003, 1024), (1_000_003, 16384), (777, 1), (100, 4096),
                                 (0, 64)])
def test_rans_sections_bit_exact(n, K):
    """Entropy-coding stress (round(mu + Laplace(0, b)) symbols, b log-uniform): GPU section bytes equal
    the oracle's, GPU decode is lossless, and the oracle's stream decodes on the GPU."""
    u = U()
    r, b = synthetic.laplace_symbols(n, seed=n % 97)
    thr = oracle.thresholds(32).astype(np.float64)
    idx = (thr[None, :] < np.log(b)[:, None]).sum(1).astype(np.uint8) if n else np.zeros(0, np.uint8)
    codec = u.Codec(0, 1, 32, synthetic.draw_weights(0, 1), "fp32")
    st, it = torch.from_numpy(r).cuda(), torch.from_numpy(idx).cuda()
    out, nb = codec.rans_encode(st, it, K)
    assert codec.sync_status() == 0
    gpu_sec = out[:int(nb.item())].cpu().numpy().tobytes()
    ref = oracle.rans_encode(r, idx, K)
    assert gpu_sec == ref
    dec = codec.rans_decode(out, int(nb.item()), it, n, K)
    assert codec.sync_status() == 0
    np.testing.assert_array_equal(dec.cpu().numpy(), r)
    ref_t = torch.from_numpy(np.frombuffer(ref, np.uint8).copy()).cuda()
    dec2 = codec.rans_decode(ref_t, len(ref), it, n, K)
    assert codec.sync_status() == 0
    np.testing.assert_array_equal(dec2.cpu().numpy(), r)


def test_corrupt_and_capacity_are_reported_not_faulted():
    u = U()
    frames = synthetic.chunk_frames("tiny", seed=2)[:2]
    blob = synthetic.draw_weights(0, 2, seed=0)
    codec = u.Codec(0, 2, 32, blob, "fp32")
    fr = torch.from_numpy(frames).cuda()
    bits, nb = codec.encode_chunk(fr, 32)
    assert codec.sync_status() == 0
    n = int(nb.item())
    # capacity too small: status CAPACITY and nothing written past the capacity (canary)
    cap = n // 2
    buf = torch.full((n + 64,), 0xA5, dtype=torch.uint8, device="cuda")
    nb2 = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = u.lib.ufvc_encode_chunk(codec.h, u._ptr(fr), 2, 64, 64, 32, u._ptr(buf), cap, u._ptr(nb2), u._stream(None))
    assert rc == 0
    assert codec.sync_status() == u.UFVC_ERR_CAPACITY
    assert (buf[cap:].cpu().numpy() == 0xA5).all()
    # corrupt magic -> CORRUPT; wrong shape -> ARG; truncated -> CORRUPT; flipped lane word -> CORRUPT
    for mutate, want in [(lambda b: b.__setitem__(0, ord("X")), u.UFVC_ERR_CORRUPT),
                         (lambda b: None, "trunc"),
                         (lambda b: b.__setitem__(n - 5, b[n - 5] ^ 0x10), u.UFVC_ERR_CORRUPT)]:
        b = bits[:n].clone()
        mutate(b)
        size = n - 8 if want == "trunc" else n
        codec.decode_chunk(b, size, 64, 64)
        assert codec.sync_status() == u.UFVC_ERR_CORRUPT
    rc = u.lib.ufvc_decode_chunk(codec.h, u._ptr(bits), n, u._ptr(torch.empty((2, 48, 64, 3), dtype=torch.uint8,
                                                                                device="cuda")),
                                 2, 64, 48, u._stream(None))
    assert rc == 0 and codec.sync_status() == u.UFVC_ERR_ARG
    # after all that the context still works
    rec = codec.decode_chunk(bits, n, 64, 64)
    assert codec.sync_status() == 0


def test_host_buffer_api_round_trip():
    u = U()
    frames = synthetic.chunk_frames("tiny", seed=4)[:2]
    blob = synthetic.draw_weights(0, 2, seed=0)
    codec = u.Codec(0, 2, 32, blob, "fp32")
    bits = codec.encode_chunk_host(frames, 32)
    fr = torch.from_numpy(frames).cuda()
    b2, nb = codec.encode_chunk(fr, 32)
    assert bits == b2[:int(nb.item())].cpu().numpy().tobytes()
    out = codec.decode_chunk_host(bits, 64, 64)
    ref = codec.decode_chunk(b2, int(nb.item()), 64, 64).cpu().numpy()
    np.testing.assert_array_equal(out, ref)


@pytest.mark.slow
def test_full_1080p_sampled_windows():
    """The 1080p 8-frame chunk at full size, in the launch configuration the benchmark times:
    entropy parameters over the whole latent, both sections byte-exact, and the analysis /
    synthesis on latent windows whose interior lies beyond the receptive field of the window edge."""
    u = U()
    arch, N, H, W, K, qp = 1, 8, 1080, 1920, 4096, 32
    frames = synthetic.chunk_frames("1080p", seed=0)
    blob = synthetic.draw_weights(arch, N, seed=0)
    codec = u.Codec(arch, N, K, blob, "fp32")
    fr = torch.from_numpy(frames).cuda()
    st = {k: v.cpu().numpy() for k, v in codec.encode_stages(fr, qp).items()}
    bits_t, nb_t = codec.encode_chunk(fr, qp)
    assert codec.sync_status() == 0
    bits = bits_t[:int(nb_t.item())].cpu().numpy().tobytes()
    report = {}
    # whole-latent entropy parameters from the GPU's z^
    mu_o, ls_o = oracle.hyper_synthesis(arch, N, st["zhat"], 68, 120, blob)
    report["mu_max_err"] = _close(st["mu"], mu_o, "mu")
    report["logsig_max_err"] = _close(st["logsig"], ls_o, "logsig")
    _check_index(st["idx"], ls_o, oracle.thresholds(qp), "idx", report)
    c = parse_container(bits, codec.Cz)
    assert oracle.rans_encode(st["rhat"].ravel(), st["idx"].ravel(), K) == c["ysec"]
    zidx = np.tile(st["iz"], st["zhat"].size // st["iz"].size)
    assert oracle.rans_encode(st["zhat"].ravel(), zidx, c["Kz"]) == c["zsec"]
    # analysis window: input rows/cols [256, 768) x [512, 1024) -> latent [16, 48) x [32, 64); the
    # interior [24, 40) x [40, 56) is exact (receptive-field radius < 48 input pixels = 3 latent px)
    y_win = oracle.analysis(arch, frames[:, 256:768, 512:1024], blob)
    _close(st["y"][24:40, 40:56], y_win[8:24, 8:24], "y window")
    # synthesis window: latent [20, 36) x [50, 66) -> output rows [320, 576) x cols [800, 1056);
    # interior latent [24, 32) x [54, 62) -> pixels [384, 512) x [864, 992)
    rec = codec.decode_chunk(bits_t, len(bits), W, H, f32=True).cpu().numpy()
    assert codec.sync_status() == 0
    yhat = st["rhat"].astype(np.float64) + st["mu"].astype(np.float32).astype(np.float64)
    win = oracle.synthesis(arch, N, yhat[20:36, 50:66], 256, 256, blob)
    err = np.abs(rec[:, 384:512, 864:992] - win[:, 64:192, 64:192])
    report["recon_window_max_err"] = float(err.max())
    assert err.max() <= TOL_RECON
    print("1080p report", report, "bytes", len(bits))
