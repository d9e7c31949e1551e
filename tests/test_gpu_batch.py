"""Batched chunk calls (serving): several chunks of one size coded with shared entropy-coding launches.

ufvc_encode_chunks / ufvc_decode_chunks run each chunk's own analysis, hyperprior and synthesis launches
and code the rANS sections of all chunks in one launch per stage.  The result must not depend on the
batching: every bit-stream and every decoded frame equals, byte for byte, what the single-chunk calls give
for the same chunk (integer and byte outputs: bit-exact).
"""
import numpy as np
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu


def U():
    from paper_2606_04410_b300 import ufvc
    return ufvc


CASES = [  # (arch, N, H, W, lanes, precision, batch)
    (0, 2, 64, 64, 32, "fp32", 3),
    (1, 8, 128, 160, 256, "bf16", 3),
    (1, 2, 200, 328, 4096, "bf16", 4),
    (1, 8, 72, 160, 512, "fp8", 2),
]


@pytest.mark.parametrize("arch,N,H,W,K,prec,B", CASES)
def test_batched_calls_equal_single_chunk_calls(arch, N, H, W, K, prec, B):
    u = U()
    blob = synthetic.draw_weights(arch, N, seed=4)
    codec = u.Codec(arch, N, K, blob, prec)
    chunks = [torch.from_numpy(synthetic.moving_texture(31 + b, N, H, W, max_step=8, refresh=0.1)).cuda()
              for b in range(B)]
    if prec == "fp8":
        codec.calibrate_fp8(chunks[0], 32)
    qps = [32, 28, 36, 32][:B]
    cap = codec.max_bitstream_bytes(W, H)
    # single-chunk calls
    ref_bits, ref_frames = [], []
    for b in range(B):
        bits, nb = codec.encode_chunk(chunks[b], qps[b])
        n = int(nb.item())
        ref_bits.append(bits[:n].clone())
        ref_frames.append(codec.decode_chunk(bits, n, W, H).clone())
    assert codec.sync_status() == 0
    # one batched encode, one batched decode (stream sizes read on the device)
    bits = [torch.zeros(cap, dtype=torch.uint8, device="cuda") for _ in range(B)]
    nbs = [torch.zeros(1, dtype=torch.int64, device="cuda") for _ in range(B)]
    codec.encode_chunks(chunks, qps, bits, nbs, width=W, height=H)
    outs = [torch.empty_like(ref_frames[b]) for b in range(B)]
    codec.decode_chunks(bits, nbs, W, H, outs)
    assert codec.sync_status() == 0
    for b in range(B):
        n = int(nbs[b].item())
        assert n == ref_bits[b].numel(), (b, n, ref_bits[b].numel())
        assert torch.equal(bits[b][:n], ref_bits[b]), f"chunk {b}: bit-stream differs"
        assert torch.equal(outs[b], ref_frames[b]), f"chunk {b}: frames differ"
    # a second batch in the same context (the batch positions' buffers are reused) in another order
    order = list(reversed(range(B)))
    bits2 = [torch.zeros(cap, dtype=torch.uint8, device="cuda") for _ in range(B)]
    codec.encode_chunks([chunks[b] for b in order], [qps[b] for b in order], bits2, nbs, width=W, height=H)
    assert codec.sync_status() == 0
    for i, b in enumerate(order):
        n = int(nbs[i].item())
        assert torch.equal(bits2[i][:n], ref_bits[b])


def test_batched_progressive_means():
    u = U()
    N, H, W = 2, 64, 96
    blob = synthetic.draw_weights(1, N, seed=6)
    codec = u.Codec(1, N, 128, blob, "bf16", mean_weights=synthetic.draw_mean_weights(1, seed=1))
    chunks = [torch.from_numpy(synthetic.moving_texture(50 + b, N, H, W, max_step=4)).cuda() for b in range(2)]
    cap = codec.max_bitstream_bytes(W, H)
    refs = []
    for c in chunks:
        b_, nb = codec.encode_chunk(c, 32)
        n = int(nb.item())
        refs.append((b_[:n].clone(), codec.decode_chunk(b_, n, W, H).clone()))
    bits = [torch.zeros(cap, dtype=torch.uint8, device="cuda") for _ in range(2)]
    nbs = [torch.zeros(1, dtype=torch.int64, device="cuda") for _ in range(2)]
    codec.encode_chunks(chunks, [32, 32], bits, nbs, width=W, height=H)
    outs = [torch.empty_like(refs[0][1]) for _ in range(2)]
    codec.decode_chunks(bits, nbs, W, H, outs)
    assert codec.sync_status() == 0
    for b in range(2):
        n = int(nbs[b].item())
        assert torch.equal(bits[b][:n], refs[b][0]) and torch.equal(outs[b], refs[b][1])


def test_batch_refusals():
    u = U()
    N = 2
    blob = synthetic.draw_weights(1, N, seed=2)
    codec = u.Codec(1, N, 64, blob, "bf16", temporal_weights=synthetic.draw_temporal_weights(1, N, seed=0))
    fr = torch.zeros((N, 64, 64, 3), dtype=torch.uint8, device="cuda")
    cap = codec.max_bitstream_bytes(64, 64)
    bits = [torch.zeros(cap, dtype=torch.uint8, device="cuda") for _ in range(2)]
    nbs = [torch.zeros(1, dtype=torch.int64, device="cuda") for _ in range(2)]
    with pytest.raises(u.UfvcError) as e:  # every stream carries its own temporal context
        codec.encode_chunks([fr, fr], [32, 32], bits, nbs)
    assert e.value.code == u.UFVC_ERR_UNSUPPORTED
    plain = u.Codec(1, N, 64, blob, "bf16")
    with pytest.raises(u.UfvcError) as e:
        plain.encode_chunks([fr] * 9, [32] * 9, [bits[0]] * 9, [nbs[0]] * 9)
    assert e.value.code == u.UFVC_ERR_ARG
