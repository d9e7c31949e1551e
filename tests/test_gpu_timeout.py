"""The entropy kernels' bounded wait, made to run out on purpose (no fault, no hang).

Every rANS encode and decode launch copies the coding tables into shared memory and waits for the copy
for a bounded time.  ufvc_set_table_wait_limit shortens that bound to a clock, which no copy can meet:
the kernels must then record UFVC_ERR_TIMEOUT, return without coding or writing the stream, and leave
the context usable (the encoder's layout control block included) -- the next calls with the default
bound give the same bytes and symbols as before.
"""
import numpy as np
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu


def test_table_wait_runs_out_and_context_recovers():
    from paper_2606_04410_b300 import ufvc as u
    codec = u.Codec(0, 1, 32, synthetic.draw_weights(0, 1), "fp32")
    n, K = 300_000, 512
    r, b = synthetic.laplace_symbols(n, seed=5)
    idx = np.clip(np.rint((np.log(b) - np.log(0.11)) / ((np.log(64.0) - np.log(0.11)) / 63)), 0, 63)
    sym = torch.from_numpy(r).cuda()
    it = torch.from_numpy(idx.astype(np.uint8)).cuda()
    ref, nb_ref = codec.rans_encode(sym, it, K)
    assert codec.sync_status() == u.UFVC_OK
    n_ref = int(nb_ref.item())

    codec.set_table_wait_limit(1)
    bad, nb_bad = codec.rans_encode(sym, it, K)
    assert codec.sync_status() == u.UFVC_ERR_TIMEOUT
    assert int(nb_bad.item()) == 0              # nothing laid out (the size was never written)
    codec.rans_decode(ref, n_ref, it, n, K)
    assert codec.sync_status() == u.UFVC_ERR_TIMEOUT

    codec.set_table_wait_limit(0)
    again, nb_again = codec.rans_encode(sym, it, K)
    dec = codec.rans_decode(ref, n_ref, it, n, K)
    assert codec.sync_status() == u.UFVC_OK
    assert int(nb_again.item()) == n_ref and torch.equal(again[:n_ref], ref[:n_ref])
    assert torch.equal(dec, sym)


def test_table_wait_limit_rejects_negative():
    from paper_2606_04410_b300 import ufvc as u
    codec = u.Codec(0, 1, 32, synthetic.draw_weights(0, 1), "fp32")
    with pytest.raises(u.UfvcError) as e:
        codec.set_table_wait_limit(-1)
    assert e.value.code == u.UFVC_ERR_ARG
