"""Pipelined host-buffer round trips (ufvc_pipe_*) against the synchronous host-buffer calls.

Every ticket's bit-stream (its first nbytes bytes) and decoded frames must equal, byte for byte, what
ufvc_encode_chunk_host / ufvc_decode_chunk_host give for the same chunk on a plain context; tickets of
different chunks in flight together must not mix; the contract's refusals (capacity below the bound, a
slot whose previous ticket was not waited for, a ticket waited for twice) are reported, not run.
"""
import numpy as np
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu


def U():
    from paper_2606_04410_b300 import ufvc
    return ufvc


def _sync_round_trip(u, codec, frames, W, H):
    bits = codec.encode_chunk_host(frames, 32, width=W, height=H)
    out = codec.decode_chunk_host(bits, W, H)
    assert codec.sync_status() == 0
    return bits, np.asarray(out).reshape(-1)


@pytest.mark.parametrize("N,H,W,K,depth,prec", [(8, 128, 160, 4096, 2, "bf16"), (2, 72, 120, 256, 3, "bf16"),
                                                  (8, 72, 160, 512, 2, "fp8"),
                                                  # five slots: each decode follows the second next encode
                                                  (2, 72, 120, 256, 5, "bf16")])
def test_pipe_equals_sync_calls(N, H, W, K, depth, prec):
    u = U()
    blob = synthetic.draw_weights(1, N, seed=3)
    codec = u.Codec(1, N, K, blob, prec)
    ref = u.Codec(1, N, K, blob, prec)
    chunks = [synthetic.moving_texture(50 + i, N, H, W, max_step=16, refresh=0.1) for i in range(max(5, depth + 3))]
    if prec == "fp8":  # the pipe's slots take the context's calibration as it stands when it is created
        cal = torch.from_numpy(chunks[0]).cuda()
        codec.calibrate_fp8(cal, 32)
        ref.calibrate_fp8(cal, 32)
    pipe = u.Pipe(codec, depth)
    cap = codec.max_bitstream_bytes(W, H)
    h_in = [torch.from_numpy(c).pin_memory() for c in chunks]
    h_bits = [torch.empty(cap, dtype=torch.uint8).pin_memory() for _ in range(depth)]
    h_out = [torch.empty((N, H, W, 3), dtype=torch.uint8).pin_memory() for _ in range(depth)]
    tickets, results = [], {}
    for i in range(len(chunks)):
        if i >= depth:  # free the slot: wait for the ticket submitted depth steps earlier
            t = tickets[i - depth]
            results[t] = (pipe.wait(t), h_bits[t % depth].numpy().copy(), h_out[t % depth].numpy().copy())
        tickets.append(pipe.submit(h_in[i], W, H, h_bits[i % depth], h_out[i % depth]))
    for t in tickets[-depth:]:
        results[t] = (pipe.wait(t), h_bits[t % depth].numpy().copy(), h_out[t % depth].numpy().copy())
    assert tickets == list(range(len(chunks)))
    for i, t in enumerate(tickets):
        nb, bits, out = results[t]
        rbits, rout = _sync_round_trip(u, ref, chunks[i], W, H)
        assert nb == len(rbits)
        assert bits[:nb].tobytes() == rbits, f"chunk {i}: bit-stream differs"
        np.testing.assert_array_equal(out.reshape(-1), rout)
    pipe.close()


def test_pipe_refusals():
    u = U()
    N, H, W = 2, 64, 64
    codec = u.Codec(1, N, 64, synthetic.draw_weights(1, N, seed=0), "bf16")
    pipe = u.Pipe(codec, 1)
    frames = torch.from_numpy(synthetic.moving_texture(1, N, H, W, max_step=3, period=64)).pin_memory()
    cap = codec.max_bitstream_bytes(W, H)
    small = torch.empty(cap - 1, dtype=torch.uint8).pin_memory()
    with pytest.raises(u.UfvcError) as e:
        pipe.submit(frames, W, H, small)
    assert e.value.code == u.UFVC_ERR_CAPACITY
    bits = torch.empty(cap, dtype=torch.uint8).pin_memory()
    t0 = pipe.submit(frames, W, H, bits)  # encode only (no frames back)
    with pytest.raises(u.UfvcError):
        pipe.submit(frames, W, H, bits)  # the only slot still holds ticket t0
    nb = pipe.wait(t0)
    assert 0 < nb <= cap
    with pytest.raises(u.UfvcError):
        pipe.wait(t0)  # waited for already
    rbits = codec.encode_chunk_host(frames, 32, width=W, height=H)
    assert bits[:nb].numpy().tobytes() == rbits
    pipe.close()
