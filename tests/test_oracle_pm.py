"""Pins of the oracle's progressive means (Sec. 3.4, Fig. 4a/4c): the four-partition split, the mean
steps of partitions 1..3 and the version-2 container that carries them.

What pins what:
* partition map: exact balance and Latin-square properties, brute-force counted (a wrong parity term or
  group index breaks one of them);
* mean step: PyTorch float64 conv2d / GELU model of the stated network on the same masked input,
  causality (no dependence on partitions >= k, real dependence on partitions < k), and the
  zero-kernel special case where mu^k is the bias exactly;
* progressive encode / decode: the zero-weight case reduces to the plain quantiser, each partition's
  r^ agrees with mean_step of the partitions before it, the decoder rebuilds the encoder's y^ exactly,
  and the container round trip.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
import synthetic
from synthetic.weights import split_mean_weights

ARCH = 0
CY, CZ = 128, 64


def test_partition_map_balance_and_latin_square():
    for Hy, Wy in ((4, 4), (6, 10), (5, 7)):
        pm = oracle.partition_map(Hy, Wy, CY)
        assert pm.max() == 3 and pm.min() == 0
        grp = CY // 4
        # inside every 2x2 block, every channel sees four different partitions
        for h in range(0, Hy - 1, 2):
            for w in range(0, Wy - 1, 2):
                blk = pm[h:h + 2, w:w + 2, :].reshape(4, CY)
                for c in range(CY):
                    assert sorted(blk[:, c]) == [0, 1, 2, 3]
                # at one position, the four channel groups sit in four different partitions
                for dy in (0, 1):
                    for dx in (0, 1):
                        groups = [pm[h + dy, w + dx, g * grp] for g in range(4)]
                        assert sorted(groups) == [0, 1, 2, 3]
                        # a channel group is one partition at one position
                        for g in range(4):
                            assert len(set(pm[h + dy, w + dx, g * grp:(g + 1) * grp])) == 1
        if Hy % 2 == 0 and Wy % 2 == 0:
            counts = np.bincount(pm.ravel(), minlength=4)
            assert (counts == Hy * Wy * CY // 4).all()
    # partition 0 at the origin holds channel group 0 (the step the single pass codes)
    assert oracle.partition(0, 0, 0, CY) == 0
    assert oracle.partition(0, 1, 0, CY) != oracle.partition(1, 0, 0, CY)


def _inputs(seed=0, Hy=4, Wy=6):
    rng = np.random.default_rng(seed)
    yhat = rng.normal(0, 1.0, (Hy, Wy, CY))
    s = np.maximum(rng.normal(0, 0.7, (Hy, Wy, CZ)), -0.17)
    return yhat, s


def _torch_mean_step(k, yhat, s, blob):
    """The stated network in PyTorch float64: [yhat on partitions < k, s] -> 3x3 -> GELU -> 1x1."""
    Hy, Wy, _ = yhat.shape
    part = oracle.partition_map(Hy, Wy, CY)
    x = np.concatenate([np.where(part < k, yhat, 0.0), s], axis=2)
    lw = split_mean_weights(blob, ARCH)
    wa, ba = lw[f"P{k}a"]
    wb, bb = lw[f"P{k}b"]
    t = torch.from_numpy(x).permute(2, 0, 1)[None]
    h = F.conv2d(t, torch.from_numpy(wa.astype(np.float64)).permute(0, 3, 1, 2), torch.from_numpy(ba.astype(np.float64)), padding=1)
    h = F.gelu(h)
    o = F.conv2d(h, torch.from_numpy(wb.astype(np.float64)).permute(0, 3, 1, 2), torch.from_numpy(bb.astype(np.float64)))
    return o[0].permute(1, 2, 0).numpy()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_mean_step_matches_torch_model(k):
    blob = synthetic.draw_mean_weights(ARCH, seed=1)
    assert blob.size == oracle.mean_weight_count(ARCH)
    yhat, s = _inputs(k)
    mu = oracle.mean_step(ARCH, k, yhat, s, blob)
    ref = _torch_mean_step(k, yhat, s, blob)
    assert np.abs(mu - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("k", [1, 2, 3])
def test_mean_step_is_causal(k):
    blob = synthetic.draw_mean_weights(ARCH, seed=2)
    yhat, s = _inputs(10 + k)
    part = oracle.partition_map(*yhat.shape[:2], CY)
    mu = oracle.mean_step(ARCH, k, yhat, s, blob)
    # partitions k..3 are not yet decoded: changing them must not move mu^k
    noisy = np.where(part >= k, yhat + 5.0, yhat)
    assert np.array_equal(oracle.mean_step(ARCH, k, noisy, s, blob), mu)
    # partitions before k are: one changed element of partition k-1 moves mu^k around it
    h, w = 1, 2
    c = int(np.nonzero(part[h, w] == k - 1)[0][0])
    bumped = yhat.copy()
    bumped[h, w, c] += 1.0
    d = np.abs(oracle.mean_step(ARCH, k, bumped, s, blob) - mu).max(axis=2)
    assert d[h, w] > 0
    assert d[h + 2:, :].max() == 0 and d[:, w + 2:].max() == 0  # 3x3 then 1x1: one pixel of reach


def test_mean_step_zero_kernels_give_bias():
    blob = synthetic.draw_mean_weights(ARCH, seed=3).copy()
    lw = split_mean_weights(blob, ARCH)
    for k in (1, 2, 3):
        lw[f"P{k}b"][0][...] = 0.0  # views into the blob
    yhat, s = _inputs(4)
    for k in (1, 2, 3):
        mu = oracle.mean_step(ARCH, k, yhat, s, blob)
        assert np.array_equal(mu, np.broadcast_to(lw[f"P{k}b"][1].astype(np.float64), mu.shape))


def _latent_case(seed=5, Hy=4, Wy=4):
    rng = np.random.default_rng(seed)
    y = rng.normal(0, 2.0, (Hy, Wy, CY))
    mu0 = rng.normal(0, 0.5, (Hy, Wy, CY))
    s = np.maximum(rng.normal(0, 0.7, (Hy, Wy, CZ)), -0.17)
    return y, mu0, s


@pytest.mark.parametrize("qp", [32, 40])
def test_progressive_zero_network_is_plain_quantiser(qp):
    y, mu0, s = _latent_case()
    blob = np.zeros(oracle.mean_weight_count(ARCH), np.float32)
    rh, yhat, mu_used = oracle.progressive_means(ARCH, y, np.zeros(y.shape, np.int16), mu0, s, qp, blob)
    part = oracle.partition_map(*y.shape[:2], CY)
    q = 2.0 ** ((qp - 32) / 8)
    expect_mu = np.where(part == 0, mu0, 0.0)
    assert np.array_equal(mu_used, expect_mu)
    expect_r = np.clip(np.rint((y - expect_mu) / q), -255, 255)
    assert np.array_equal(rh, expect_r.astype(np.int16))
    assert np.array_equal(yhat, rh * q + expect_mu)


def test_progressive_steps_follow_mean_step_and_decoder_repeats_them():
    y, mu0, s = _latent_case(6)
    blob = synthetic.draw_mean_weights(ARCH, seed=4)
    qp = 32
    rh, yhat, mu_used = oracle.progressive_means(ARCH, y, np.zeros(y.shape, np.int16), mu0, s, qp, blob)
    part = oracle.partition_map(*y.shape[:2], CY)
    assert np.array_equal(mu_used[part == 0], mu0[part == 0])
    for k in (1, 2, 3):
        muk = oracle.mean_step(ARCH, k, yhat, s, blob)  # yhat is final; mean_step reads only partitions < k
        sel = part == k
        assert np.array_equal(mu_used[sel], muk[sel])
        assert np.array_equal(rh[sel], np.clip(np.rint(y[sel] - muk[sel]), -255, 255).astype(np.int16))
    # the progressive means are not the single-pass ones
    assert np.abs(mu_used - mu0)[part > 0].min() > 0
    # decoder: same r^, no y -> the same means and reconstruction, bit for bit
    rd, yd, md = oracle.progressive_means(ARCH, None, rh, mu0, s, qp, blob)
    assert np.array_equal(rd, rh) and np.array_equal(yd, yhat) and np.array_equal(md, mu_used)


def test_chunk_round_trip_version_2():
    frames = synthetic.chunk_frames("tiny", seed=1)[:2]
    blob = synthetic.draw_weights(0, 2, seed=0)
    mw = synthetic.draw_mean_weights(0, seed=0)
    bits, dbg = oracle.encode_chunk(0, frames, 32, 32, blob, debug=True, mean_weights=mw)
    assert bits[4] == 2
    bits1, dbg1 = oracle.encode_chunk(0, frames, 32, 32, blob, debug=True)
    assert bits1[4] == 1
    # same y, z^, scales; the means of partitions 1..3 differ
    assert np.array_equal(dbg["y"], dbg1["y"]) and np.array_equal(dbg["zhat"], dbg1["zhat"])
    assert np.array_equal(dbg["idx"], dbg1["idx"])
    part = oracle.partition_map(4, 4, CY)
    assert np.array_equal(dbg["mu"][part == 0], dbg1["mu"][part == 0])
    assert not np.array_equal(dbg["mu"], dbg1["mu"])
    # the prior s is the one the hyper-synthesis gives
    _, _, s = oracle.hyper_synthesis(0, 2, dbg["zhat"], 4, 4, blob, want_s=True)
    assert np.array_equal(s, dbg["s"])
    # latent section = the oracle rANS of the coded r^ with the single-pass indices
    assert bits.endswith(oracle.rans_encode(dbg["rhat"].ravel(), dbg["idx"].ravel(), 32))
    fr, yhat = oracle.decode_chunk(0, 2, bits, 64, 64, blob, mean_weights=mw)
    assert np.array_equal(yhat, dbg["yhat"])
    assert np.array_equal(yhat, dbg["rhat"] * 1.0 + dbg["mu"])
    assert np.array_equal(fr, oracle.synthesis(0, 2, yhat, 64, 64, blob))
    # version 2 needs the mean network; version 1 ignores it
    with pytest.raises(RuntimeError):
        oracle.decode_chunk(0, 2, bits, 64, 64, blob)
    _, y1 = oracle.decode_chunk(0, 2, bits1, 64, 64, blob, want_frames=False, mean_weights=mw)
    assert np.array_equal(y1, dbg1["rhat"] * 1.0 + dbg1["mu"])
