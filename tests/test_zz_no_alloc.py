"""The allocation-free rANS section encoder, through the C ABI.

ufvc_rans_encode_noalloc exists for callers that cannot let the library allocate device memory (a
stream being captured, real-time loops that cannot absorb cudaMalloc's implicit synchronisation,
hosts whose device memory is owned by their own pool allocator).  It keeps its staging space in one
fixed per-device array instead.  Its output must be byte-identical to ufvc_rans_encode's (the
tolerance for integer work), on two calls in a row: the second call runs on scratch that still holds
the first call's contents, and it has a different size.  This file is collected last so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu


def _encode_both(u, codec, n, K, seed):
    r, b = synthetic.laplace_symbols(n, seed=seed)
    idx = np.clip(np.rint((np.log(b) - np.log(0.11)) / ((np.log(64.0) - np.log(0.11)) / 63)), 0, 63)
    sym = torch.from_numpy(r).cuda()
    it = torch.from_numpy(idx.astype(np.uint8)).cuda()
    ref, nb_ref = codec.rans_encode(sym, it, K)
    cap = ref.numel()
    out = torch.full((cap + 64,), 0xA5, dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = u.lib.ufvc_rans_encode_noalloc(codec.h, u._ptr(sym), u._ptr(it), n, K, u._ptr(out), cap, u._ptr(nb),
                                        u._stream(None))
    assert rc == u.UFVC_OK, u.lib.ufvc_last_error(codec.h)
    assert codec.sync_status() == 0
    n_ref = int(nb_ref.item())
    assert int(nb.item()) == n_ref
    assert torch.equal(out[:n_ref], ref[:n_ref])
    assert (out[cap:].cpu().numpy() == 0xA5).all()        # nothing written past the capacity
    return sym, it, out, n_ref


def test_noalloc_matches_allocating_encoder_twice():
    from paper_2606_04410_b300 import ufvc as u
    codec = u.Codec(0, 1, 32, synthetic.draw_weights(0, 1), "fp32")
    # first call: a 1080p-sized latent; second call, right after, a smaller one on the same scratch
    _encode_both(u, codec, 2_088_960, 4096, seed=11)
    sym, it, out, n_ref = _encode_both(u, codec, 300_001, 1024, seed=12)
    # and the stream it wrote decodes back losslessly
    dec = codec.rans_decode(out, n_ref, it, 300_001, 1024)
    assert codec.sync_status() == 0
    assert torch.equal(dec, sym)


def test_noalloc_rejects_oversize_request():
    from paper_2606_04410_b300 import ufvc as u
    codec = u.Codec(0, 1, 32, synthetic.draw_weights(0, 1), "fp32")
    n = 13_000_000                                          # beyond the fixed per-device scratch
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = u.lib.ufvc_rans_encode_noalloc(codec.h, u._ptr(dummy), u._ptr(dummy), n, 4096, u._ptr(dummy), 16,
                                        u._ptr(nb), u._stream(None))
    assert rc == u.UFVC_ERR_ARG
    assert b"static scratch" in u.lib.ufvc_last_error(codec.h)


def test_noalloc_leaves_device_memory_unchanged():
    """After one warm-up call on a fresh context (the first call on a device looks up the array's
    address), further calls change the device's free memory by nothing: no cudaMalloc behind them."""
    from paper_2606_04410_b300 import ufvc as u
    codec = u.Codec(0, 1, 32, synthetic.draw_weights(0, 1), "fp32")
    n, K = 2_088_960, 4096
    r, b = synthetic.laplace_symbols(n, seed=21)
    idx = np.clip(np.rint((np.log(b) - np.log(0.11)) / ((np.log(64.0) - np.log(0.11)) / 63)), 0, 63)
    sym = torch.from_numpy(r).cuda()
    it = torch.from_numpy(idx.astype(np.uint8)).cuda()
    cap = 4 * K + 2 * (n + 2 * K) + 4
    outs = [torch.empty(cap, dtype=torch.uint8, device="cuda") for _ in range(3)]
    nbs = [torch.zeros(1, dtype=torch.int64, device="cuda") for _ in range(3)]

    def call(i):
        rc = u.lib.ufvc_rans_encode_noalloc(codec.h, u._ptr(sym), u._ptr(it), n, K, u._ptr(outs[i]), cap,
                                            u._ptr(nbs[i]), u._stream(None))
        assert rc == u.UFVC_OK, u.lib.ufvc_last_error(codec.h)

    call(0)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    call(1)
    call(2)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert codec.sync_status() == 0
    assert free1 == free0
    n0 = int(nbs[0].item())
    assert int(nbs[2].item()) == n0 and torch.equal(outs[2][:n0], outs[0][:n0])
