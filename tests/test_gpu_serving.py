"""GPU tests of the continuous-batching server (ufvc_server_*): every request's bit-stream and decoded
frames are identical to the single-context calls on the same chunk whether it runs alone, in a batch of
same-shape requests, or in a mix of streams of different sizes on several slots (same kernels, no
cross-request arithmetic); graphs are captured and replayed; a stream's requests keep their order; the
HBM cap bounds the slots (idle slots of other sizes are released) and the stream buffers; a decode with
nothing encoded is refused."""
import numpy as np
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu

N, K, QP = 8, 256, 32
SIZES = [(256, 144), (320, 192), (160, 96)]


def U():
    from paper_2606_04410_b300 import ufvc
    return ufvc


def _frames(seed, W, H):
    return torch.from_numpy(synthetic.moving_texture(seed, N, H, W, max_step=8, refresh=0.1)).cuda()


def _reference(blob, fr, W, H, qp=QP):
    """Single-context encode + decode of one chunk: (bit-stream bytes, decoded frames)."""
    u = U()
    c = u.Codec(1, N, K, blob, "bf16")
    bits, nb = c.encode_chunk(fr, qp)
    n = int(nb.item())
    out = c.decode_chunk(bits, n, W, H)
    assert c.sync_status() == 0
    ref = (bits[:n].cpu().numpy().tobytes(), out.cpu().clone())
    c.close()
    return ref


def test_server_alone_and_mix_match_single_context():
    u = U()
    blob = synthetic.draw_weights(1, N, seed=1)
    specs = [(i, *SIZES[i % len(SIZES)]) for i in range(6)]
    frames = {i: _frames(40 + i, W, H) for i, W, H in specs}
    refs = {i: _reference(blob, frames[i], W, H) for i, W, H in specs}

    # alone: one stream, one request at a time
    srv = u.Server(1, N, K, blob, "bf16", max_slots=1)
    i, W, H = specs[0]
    sid = srv.open_stream(W, H, QP)
    bufs = srv.streams[sid]
    bufs["frames_in"].copy_(frames[i])
    torch.cuda.synchronize()
    for _ in range(3):  # direct run, capture, replay
        r = srv.wait(srv.submit(sid, u.UFVC_OP_ENCODE), 120000.0)
        assert r["status"] == 0
        assert bufs["bits"][:r["nbytes"]].cpu().numpy().tobytes() == refs[i][0]
        r = srv.wait(srv.submit(sid, u.UFVC_OP_DECODE), 120000.0)
        assert r["status"] == 0
        assert torch.equal(bufs["frames_out"].cpu(), refs[i][1])
    assert srv.stats()["graphs"] >= 2
    srv.close()

    # mix: six streams of three sizes, requests of all streams queued at once, several rounds
    srv = u.Server(1, N, K, blob, "bf16", max_slots=4)
    sids = {}
    for i, W, H in specs:
        sids[i] = srv.open_stream(W, H, QP)
        srv.streams[sids[i]]["frames_in"].copy_(frames[i])
    torch.cuda.synchronize()
    for rnd in range(3):
        reqs = [(i, op) for i, _, _ in specs for op in (u.UFVC_OP_ENCODE, u.UFVC_OP_DECODE)]
        if rnd == 0:  # one by one: the scheduler may start some before the rest are queued
            tickets = [(i, op, srv.submit(sids[i], op)) for i, op in reqs]
        else:  # all at once: each size's two encodes (then decodes) run as one batch
            ts = srv.submit_many([(sids[i], op) for i, op in reqs])
            tickets = [(i, op, t) for (i, op), t in zip(reqs, ts)]
        results = [(i, op, srv.wait(t, 120000.0)) for i, op, t in tickets]
        for i, op, r in results:
            assert r["status"] == 0, (rnd, i, op, r)
            b = srv.streams[sids[i]]
            if op == u.UFVC_OP_ENCODE:
                assert r["nbytes"] == len(refs[i][0])
        # a stream's decode ran after its encode of the same round
        for i, _, _ in specs:
            enc = [r for j, op, r in results if j == i and op == u.UFVC_OP_ENCODE][0]
            dec = [r for j, op, r in results if j == i and op == u.UFVC_OP_DECODE][0]
            assert dec["start_ms"] >= enc["done_ms"]
        if rnd:
            assert all(r["batch"] == 2 for _, _, r in results), [r["batch"] for _, _, r in results]
            # the three sizes' encode batches ran on three slots at the same time
            enc = {r["slot"]: r for _, op, r in results if op == u.UFVC_OP_ENCODE}
            assert len(enc) == 3
            assert max(r["start_ms"] for r in enc.values()) < min(r["done_ms"] for r in enc.values())
        for i, _, _ in specs:
            b = srv.streams[sids[i]]
            assert b["bits"][:int(b["nbytes"].item())].cpu().numpy().tobytes() == refs[i][0]
            assert torch.equal(b["frames_out"].cpu(), refs[i][1])
    st = srv.stats()
    assert st["completed"] == 3 * 2 * len(specs) and st["queued"] == 0
    assert 1 <= st["slots"] <= 4 and st["graphs"] >= 2
    assert st["batches"] >= 2 * 6 and st["batched"] >= 2 * 12
    srv.close()


def test_server_batches_same_shape_requests():
    """Four streams of one size queued at once run as one encode batch and one decode batch on one slot
    (the slot's batch size is 4 at this size); each stream's bit-stream and frames equal the
    single-context calls'.  A fifth stream of the size waits for the next batch; streams at another rate
    are not batched with them."""
    u = U()
    blob = synthetic.draw_weights(1, N, seed=5)
    W, H = SIZES[2]
    qps = [QP, QP, QP, QP, QP, QP + 4]
    frames = [_frames(90 + i, W, H) for i in range(len(qps))]
    refs = [_reference(blob, frames[i], W, H, qps[i]) for i in range(len(qps))]
    srv = u.Server(1, N, K, blob, "bf16", max_slots=1)
    sids = [srv.open_stream(W, H, q) for q in qps]
    for sid, fr in zip(sids, frames):
        srv.streams[sid]["frames_in"].copy_(fr)
    torch.cuda.synchronize()
    for rnd in range(3):  # direct runs, captures, replays
        reqs = [(sid, op) for op in (u.UFVC_OP_ENCODE, u.UFVC_OP_DECODE) for sid in sids]
        res = [srv.wait(t, 120000.0) for t in srv.submit_many(reqs)]
        assert all(r["status"] == 0 for r in res)
        enc, dec = res[:len(sids)], res[len(sids):]
        assert [r["batch"] for r in enc[:4]] == [4] * 4 and len({r["start_ms"] for r in enc[:4]}) == 1
        assert enc[4]["batch"] == 1 and enc[5]["batch"] == 1  # the fifth stream and the other rate
        assert [r["batch"] for r in dec[:4]] == [4] * 4
        for i, sid in enumerate(sids):
            b = srv.streams[sid]
            assert b["bits"][:int(b["nbytes"].item())].cpu().numpy().tobytes() == refs[i][0], (rnd, i)
            assert torch.equal(b["frames_out"].cpu(), refs[i][1]), (rnd, i)
    st = srv.stats()
    assert st["slots"] == 1 and st["batches"] >= 6 and st["graphs"] >= 2
    srv.close()


def test_fp8_server_matches_single_context():
    """An FP8 server calibrated on a chunk codes like a single FP8 context calibrated on the same chunk
    (the slots share the server's scales): byte-identical bit-streams and frames; uncalibrated, its
    requests are refused."""
    u = U()
    blob = synthetic.draw_weights(1, N, seed=6)
    W, H = SIZES[2]
    frames = [_frames(130 + i, W, H) for i in range(3)]
    c = u.Codec(1, N, K, blob, "fp8")
    c.calibrate_fp8(frames[0], QP)
    refs = []
    for fr in frames:
        bits, nb = c.encode_chunk(fr, QP)
        n = int(nb.item())
        refs.append((bits[:n].cpu().numpy().tobytes(), c.decode_chunk(bits, n, W, H).cpu().clone()))
    assert c.sync_status() == 0
    raw = u.Server(1, N, K, blob, "fp8", max_slots=1)
    sid = raw.open_stream(W, H, QP)
    raw.streams[sid]["frames_in"].copy_(frames[0])
    torch.cuda.synchronize()
    assert raw.wait(raw.submit(sid, u.UFVC_OP_ENCODE), 120000.0)["status"] == u.UFVC_ERR_ARG
    raw.close()
    srv = u.Server(1, N, K, blob, "fp8", max_slots=2)
    srv.calibrate_fp8(frames[0], QP)
    sids = [srv.open_stream(W, H, QP) for _ in frames]
    for sid, fr in zip(sids, frames):
        srv.streams[sid]["frames_in"].copy_(fr)
    torch.cuda.synchronize()
    reqs = [(sid, op) for op in (u.UFVC_OP_ENCODE, u.UFVC_OP_DECODE) for sid in sids]
    assert all(srv.wait(t, 120000.0)["status"] == 0 for t in srv.submit_many(reqs))
    for sid, ref in zip(sids, refs):
        b = srv.streams[sid]
        assert b["bits"][:int(b["nbytes"].item())].cpu().numpy().tobytes() == ref[0]
        assert torch.equal(b["frames_out"].cpu(), ref[1])
    srv.close()


def test_server_hbm_cap_releases_idle_slots_and_bounds_streams():
    u = U()
    blob = synthetic.draw_weights(1, N, seed=2)
    (Wa, Ha), (Wb, Hb) = SIZES[0], SIZES[1]
    fa, fb = _frames(7, Wa, Ha), _frames(8, Wb, Hb)
    ra, rb = _reference(blob, fa, Wa, Ha), _reference(blob, fb, Wb, Hb)
    # a cap that holds the two streams and ONE slot of either size
    probe = u.Server(1, N, K, blob, "bf16", max_slots=2)
    s0 = probe.open_stream(Wa, Ha, QP)
    s1 = probe.open_stream(Wb, Hb, QP)
    probe.streams[s0]["frames_in"].copy_(fa)
    probe.streams[s1]["frames_in"].copy_(fb)
    torch.cuda.synchronize()
    probe.wait(probe.submit(s0, u.UFVC_OP_ENCODE), 120000.0)
    used_a = probe.stats()["hbm_used"]
    probe.wait(probe.submit(s1, u.UFVC_OP_ENCODE), 120000.0)
    used_ab = probe.stats()["hbm_used"]
    probe.close()
    assert used_ab > used_a
    cap = used_a + (used_ab - used_a) // 2 + (used_ab - used_a) // 4  # room for one of the two slots only
    srv = u.Server(1, N, K, blob, "bf16", hbm_cap_bytes=cap, max_slots=4)
    a = srv.open_stream(Wa, Ha, QP)
    b = srv.open_stream(Wb, Hb, QP)
    srv.streams[a]["frames_in"].copy_(fa)
    srv.streams[b]["frames_in"].copy_(fb)
    torch.cuda.synchronize()
    tickets = []
    for _ in range(2):
        for sid in (a, b):
            tickets.append(srv.submit(sid, u.UFVC_OP_ENCODE))
            tickets.append(srv.submit(sid, u.UFVC_OP_DECODE))
    for t in tickets:
        assert srv.wait(t, 120000.0)["status"] == 0
    st = srv.stats()
    assert st["hbm_used"] <= cap and st["slots"] == 1
    for sid, ref in ((a, ra), (b, rb)):
        buf = srv.streams[sid]
        assert buf["bits"][:int(buf["nbytes"].item())].cpu().numpy().tobytes() == ref[0]
        assert torch.equal(buf["frames_out"].cpu(), ref[1])
    # stream buffers beyond the cap are refused
    with pytest.raises(u.UfvcError) as e:
        srv.open_stream(3840, 2160, QP)
    assert e.value.code == u.UFVC_ERR_OOM
    srv.close()


def test_server_refuses_decode_before_encode_and_bad_calls():
    u = U()
    blob = synthetic.draw_weights(1, N, seed=3)
    srv = u.Server(1, N, K, blob, "bf16", max_slots=1)
    sid = srv.open_stream(160, 96, QP)
    r = srv.wait(srv.submit(sid, u.UFVC_OP_DECODE), 120000.0)
    assert r["status"] == u.UFVC_ERR_ARG
    with pytest.raises(u.UfvcError):
        srv.submit(sid + 5, u.UFVC_OP_ENCODE)
    with pytest.raises(u.UfvcError):
        srv.submit(sid, 7)
    with pytest.raises(u.UfvcError):
        srv.open_stream(8, 8, QP)
    srv.close()


def test_server_streams_carry_temporal_context():
    """Each stream's chunks form one context chain on the server (its encoder's and decoder's context kept
    on the device between requests, on whatever slots they run): bit-streams and frames equal a single
    context coding the same chunks in order, with progressive means as well (version-4 streams)."""
    u = U()
    blob = synthetic.draw_weights(1, N, seed=4)
    tw = synthetic.draw_temporal_weights(1, N, seed=3)
    mw = synthetic.draw_mean_weights(1, seed=3)
    specs = [(0, *SIZES[0]), (1, *SIZES[2]), (2, *SIZES[0])]
    rounds = 3
    chunks = {i: [_frames(70 + 10 * i + r, W, H) for r in range(rounds)] for i, W, H in specs}
    refs = {}
    for i, W, H in specs:  # single-context reference chains
        c = u.Codec(1, N, K, blob, "bf16", temporal_weights=tw, mean_weights=mw)
        ce = [c.new_context(W, H), c.new_context(W, H)]
        cd = [c.new_context(W, H), c.new_context(W, H)]
        out = []
        for r in range(rounds):
            bits, nb = c.encode_chunk_tc(chunks[i][r], ce[r % 2] if r else None, ce[(r + 1) % 2], QP)
            n = int(nb.item())
            fr = c.decode_chunk_tc(bits, n, W, H, cd[r % 2] if r else None, cd[(r + 1) % 2])
            assert c.sync_status() == 0
            out.append((bits[:n].cpu().numpy().tobytes(), fr.cpu().clone()))
        refs[i] = out
        c.close()
    srv = u.Server(1, N, K, blob, "bf16", max_slots=2, temporal_weights=tw, mean_weights=mw)
    sids = {i: srv.open_stream(W, H, QP) for i, W, H in specs}
    # the optional networks are set before the first stream only
    assert u.lib.ufvc_server_set_progressive_means(srv.h, u._ptr(mw), mw.size) == u.UFVC_ERR_ARG
    for r in range(rounds):
        for i, _, _ in specs:
            srv.streams[sids[i]]["frames_in"].copy_(chunks[i][r])
        torch.cuda.synchronize()
        tickets = []
        for i, _, _ in specs:
            tickets.append((i, srv.submit(sids[i], u.UFVC_OP_ENCODE)))
            tickets.append((i, srv.submit(sids[i], u.UFVC_OP_DECODE)))
        for i, t in tickets:
            assert srv.wait(t, 120000.0)["status"] == 0
        for i, _, _ in specs:
            b = srv.streams[sids[i]]
            raw = b["bits"][:int(b["nbytes"].item())].cpu().numpy().tobytes()
            assert raw[4] == 4
            assert raw == refs[i][r][0], (i, r)
            assert torch.equal(b["frames_out"].cpu(), refs[i][r][1]), (i, r)
    assert srv.stats()["graphs"] >= 2
    # a chunk encoded over an undecoded one: its decode is refused (the decoder's chain lost a chunk)
    sid = sids[0]
    t = srv.submit_many([(sid, u.UFVC_OP_ENCODE), (sid, u.UFVC_OP_ENCODE), (sid, u.UFVC_OP_DECODE)])
    res = [srv.wait(x, 120000.0) for x in t]
    assert [r["status"] for r in res] == [0, 0, u.UFVC_ERR_ARG]
    srv.close()


def test_server_dc_model_streams_carry_context():
    """A server on the DC-block model (whose temporal context is built in) keeps every stream's context
    chain on the device: bit-streams and frames equal a single context coding the same chunks in order."""
    u = U()
    n = 2
    blob = synthetic.draw_dc_weights(n, seed=5)
    sizes = [(64, 64), (96, 64)]
    rounds = 3
    chunks = {i: [torch.from_numpy(synthetic.moving_texture(120 + 10 * i + r, n, H, W, max_step=3, period=64)).cuda()
                  for r in range(rounds)] for i, (W, H) in enumerate(sizes)}
    refs = {}
    for i, (W, H) in enumerate(sizes):
        c = u.Codec(2, n, 64, blob, "bf16")
        ce = [c.new_context(W, H), c.new_context(W, H)]
        cd = [c.new_context(W, H), c.new_context(W, H)]
        out = []
        for r in range(rounds):
            bits, nb = c.encode_chunk_tc(chunks[i][r], ce[r % 2] if r else None, ce[(r + 1) % 2], QP)
            m = int(nb.item())
            fr = c.decode_chunk_tc(bits, m, W, H, cd[r % 2] if r else None, cd[(r + 1) % 2])
            assert c.sync_status() == 0
            out.append((bits[:m].cpu().numpy().tobytes(), fr.cpu().clone()))
        refs[i] = out
        c.close()
    srv = u.Server(2, n, 64, blob, "bf16", max_slots=2)
    sids = {i: srv.open_stream(W, H, QP) for i, (W, H) in enumerate(sizes)}
    for r in range(rounds):
        for i in sids:
            srv.streams[sids[i]]["frames_in"].copy_(chunks[i][r])
        torch.cuda.synchronize()
        tickets = [(i, srv.submit(sids[i], op)) for i in sids for op in (u.UFVC_OP_ENCODE, u.UFVC_OP_DECODE)]
        for i, t in tickets:
            assert srv.wait(t, 120000.0)["status"] == 0
        for i in sids:
            b = srv.streams[sids[i]]
            raw = b["bits"][:int(b["nbytes"].item())].cpu().numpy().tobytes()
            assert raw[4] == 3 and raw[5] == 2
            assert raw == refs[i][r][0], (i, r)
            assert torch.equal(b["frames_out"].cpu(), refs[i][r][1]), (i, r)
    srv.close()
