"""Full-size (1080p, 8 frames, 4096 lanes: the configuration the benchmark times) checks of the optional
paths, through properties that hold at any size (the FP64 oracle of a whole 1080p chunk would take
minutes; the element-wise parity of these paths is tested at small sizes in the other files):

* progressive means: the decoder repeats the encoder's means (decoded frames bit-identical to
  synthesising the encoder's r^ q + mu) and the latent section is the oracle's rANS of the GPU's symbols;
* temporal context and the DC-block model: over a stream of three chunks the encoder's context equals
  the decoder's bit for bit and every chunk's latent section is the oracle's rANS of the GPU's symbols;
* colour interface: YUV444-planar and YUV420 chunks code exactly like the interleaved chunk of the same
  channel values.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests._util import parse_container

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N, W, H, K, QP = 8, 1920, 1080, 4096, 32


def U():
    from paper_2606_04410_b300 import ufvc
    return ufvc


@pytest.fixture(scope="module")
def chunks():
    return [synthetic.chunk_frames("1080p", seed=s) for s in range(3)]


def _section_matches(codec, bits, n, st):
    c = parse_container(bits[:n].cpu().numpy().tobytes(), codec.Cz)
    assert oracle.rans_encode(st["rhat"].ravel(), st["idx"].ravel(), K) == c["ysec"]


def test_progressive_means_1080p(chunks):
    u = U()
    blob = synthetic.draw_weights(1, N, seed=0)
    c = u.Codec(1, N, K, blob, "bf16", mean_weights=synthetic.draw_mean_weights(1, seed=0))
    fr = torch.from_numpy(chunks[0]).cuda()
    st = {k: v.cpu().numpy() for k, v in c.encode_stages(fr, QP).items()}
    bits, nb = c.encode_chunk(fr, QP)
    n = int(nb.item())
    rec = c.decode_chunk(bits, n, W, H, f32=True)
    assert c.sync_status() == 0
    _section_matches(c, bits, n, st)
    yhat = torch.from_numpy(st["rhat"]).cuda().float() + torch.from_numpy(st["mu"]).cuda()
    assert torch.equal(rec, c.synthesize(yhat, W, H))


@pytest.mark.parametrize("arch", [1, 2], ids=["temporal", "dc_model"])
def test_context_chain_1080p(chunks, arch):
    u = U()
    if arch == 1:
        c = u.Codec(1, N, K, synthetic.draw_weights(1, N, seed=0), "bf16",
                    temporal_weights=synthetic.draw_temporal_weights(1, N, seed=0))
    else:
        c = u.Codec(2, N, K, synthetic.draw_dc_weights(N, seed=0), "bf16")
    ce = [c.new_context(W, H), c.new_context(W, H)]
    cd = [c.new_context(W, H), c.new_context(W, H)]
    for i, frames in enumerate(chunks):
        fr = torch.from_numpy(frames).cuda()
        cin_e, cin_d = (None, None) if i == 0 else (ce[i % 2], cd[i % 2])
        st = {k: v.cpu().numpy() for k, v in c.encode_stages(fr, QP, ctx_in=cin_e).items()}
        bits, nb = c.encode_chunk_tc(fr, cin_e, ce[(i + 1) % 2], QP)
        c.decode_chunk_tc(bits, bits.numel(), W, H, cin_d, cd[(i + 1) % 2], d_nbytes=nb)
        assert c.sync_status() == 0
        assert torch.equal(ce[(i + 1) % 2], cd[(i + 1) % 2]), (arch, i)
        assert torch.isfinite(ce[(i + 1) % 2].float()).all()
        _section_matches(c, bits, int(nb.item()), st)


def test_color_layouts_1080p(chunks):
    u = U()
    blob = synthetic.draw_weights(1, N, seed=0)
    rgb = chunks[1]
    planar = np.ascontiguousarray(np.moveaxis(rgb, 3, 1))
    uu, vv = rgb[:, ::2, ::2, 1], rgb[:, ::2, ::2, 2]
    i420 = np.ascontiguousarray(np.concatenate([rgb[..., 0].reshape(N, -1), uu.reshape(N, -1), vv.reshape(N, -1)], 1))
    rep = rgb.copy()
    rep[..., 1] = np.repeat(np.repeat(uu, 2, axis=1), 2, axis=2)[:, :H, :W]
    rep[..., 2] = np.repeat(np.repeat(vv, 2, axis=1), 2, axis=2)[:, :H, :W]
    out = {}
    for fmt, src in ((u.COLOR_RGB, rgb), (u.COLOR_YUV444P, planar), (u.COLOR_RGB, rep), (u.COLOR_YUV420P, i420)):
        c = u.Codec(1, N, K, blob, "bf16", color=fmt)
        bits, nb = c.encode_chunk(torch.from_numpy(src).cuda(), QP, width=W, height=H)
        assert c.sync_status() == 0
        out.setdefault(fmt, []).append(bits[:int(nb.item())].cpu().numpy().tobytes())
        c.close()
    assert out[u.COLOR_RGB][0] == out[u.COLOR_YUV444P][0]
    assert out[u.COLOR_RGB][1] == out[u.COLOR_YUV420P][0]
