"""GPU tests of the first analysis layer read straight from the frame bytes (BF16), element by element.

The chunk encoder's first layer (the patch embedding of the stacked chunk, Sec. 3.1: frame n's three
channels become input channels 3n .. 3n+2, replicate-padded to a multiple of 16, then a 3x3 stride-2
convolution + GELU) runs in one of two tcgen05 kernels that read the uint8 frames themselves: the
TMA-window kernel (interleaved RGB with rows of a multiple of 16 bytes) and the register-staged kernel
(every format and width).  Both read their operand in place from shared memory through hand-built
no-swizzle matrix descriptors, so a wrong stride in a descriptor would pair input channels with the
wrong weights.  Each output element is compared here with a float64 PyTorch convolution of the same
bf16 operands -- the input bytes as v / 256 (exact in bf16) and the weights as bf16(w * 256 / 255), the
factor that keeps x = v / 255 -- through ``ufvc_first_layer``:

    |gpu - ref| <= 8e-3 |ref| + 2e-3 max|ref|

(products of bf16 values are exact in FP32 and the sums are FP32; the output is rounded to bf16, 2^-9
relative, and the GELU on the tensor-core path is a fitted form within 2.6e-5 of the erf form).
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import synthetic
from synthetic.weights import split_weights

pytestmark = pytest.mark.gpu


def U():
    from paper_2606_04410_b300 import ufvc
    return ufvc


def channel_bytes(frames: np.ndarray, fmt: int, N: int, H: int, W: int) -> np.ndarray:
    """The network's input channels as bytes [H][W][3N]: frame n's three channels at 3n .. 3n+2, in the
    caller's layout (RGB interleaved, YUV444 planar, or YUV420 planar with each chroma sample repeated
    over its 2 x 2 block)."""
    u = U()
    out = np.zeros((H, W, 3 * N), np.uint8)
    flat = frames.reshape(N, -1)
    for n in range(N):
        if fmt == u.COLOR_RGB:
            out[..., 3 * n:3 * n + 3] = flat[n].reshape(H, W, 3)
        elif fmt == u.COLOR_YUV444P:
            out[..., 3 * n:3 * n + 3] = flat[n].reshape(3, H, W).transpose(1, 2, 0)
        else:
            Hc, Wc = (H + 1) // 2, (W + 1) // 2
            y = flat[n][:H * W].reshape(H, W)
            cu = flat[n][H * W:H * W + Hc * Wc].reshape(Hc, Wc)
            cv = flat[n][H * W + Hc * Wc:].reshape(Hc, Wc)
            out[..., 3 * n] = y
            out[..., 3 * n + 1] = cu.repeat(2, 0).repeat(2, 1)[:H, :W]
            out[..., 3 * n + 2] = cv.repeat(2, 0).repeat(2, 1)[:H, :W]
    return out


def reference_rows(ch: np.ndarray, w: np.ndarray, b: np.ndarray, rows: range) -> torch.Tensor:
    """float64 GELU(conv3x3 stride 2, zero pad 1) of the replicate-padded input, output rows `rows` only.
    ch: bytes [H][W][3N]; w: [64][3][3][3N] float32; b: [64]."""
    H, W, _ = ch.shape
    Hp, Wp = -(-H // 16) * 16, -(-W // 16) * 16
    xp = np.pad(ch, ((0, Hp - H), (0, Wp - W), (0, 0)), mode="edge")  # replicate padding (bytes)
    r0, r1 = rows.start, rows.stop
    lo, hi = 2 * r0 - 1, 2 * r1  # input rows read by output rows r0 .. r1-1 (zero outside 0 .. Hp-1)
    x = xp[max(lo, 0):min(hi, Hp)].astype(np.float64) / 256.0
    xt = F.pad(torch.from_numpy(x).permute(2, 0, 1)[None], (1, 1, max(0, -lo), max(0, hi - Hp)))
    scale = np.float32(1.0) / np.float32(255.0 / 256.0)
    wb = torch.from_numpy(np.float32(scale) * w.astype(np.float32)).to(torch.bfloat16).to(torch.float64)
    y = F.conv2d(xt, wb.permute(0, 3, 1, 2), torch.from_numpy(b.astype(np.float64)), stride=2)
    return F.gelu(y)[0].permute(1, 2, 0)


def check_rows(got: torch.Tensor, ref: torch.Tensor, what: str):
    err = (got - ref).abs()
    scale = float(ref.abs().max())
    bound = 8e-3 * ref.abs() + 2e-3 * scale
    bad = int((err > bound).sum())
    assert bad == 0, f"{what}: {bad} elements out of bound, max err {float(err.max()):.4g}, scale {scale:.3g}"


def frames_for(fmt: int, N: int, H: int, W: int, seed: int) -> np.ndarray:
    u = U()
    rgb = synthetic.moving_texture(seed, N, H, W, max_step=8, refresh=0.1)
    if fmt == u.COLOR_RGB:
        return rgb
    if fmt == u.COLOR_YUV444P:  # any bytes will do: the layer sees the planes as its channels
        return np.ascontiguousarray(rgb.transpose(0, 3, 1, 2))
    Hc, Wc = (H + 1) // 2, (W + 1) // 2
    y = rgb[..., 0].reshape(N, -1)
    cu = rgb[:, ::2, ::2, 1][:, :Hc, :Wc].reshape(N, -1)
    cv = rgb[:, ::2, ::2, 2][:, :Hc, :Wc].reshape(N, -1)
    return np.ascontiguousarray(np.concatenate([y, cu, cv], 1))


CASES = [  # (N, H, W, colour format name, kernels to run)
    (2, 72, 200, "RGB", (1,)),          # 3W % 16 = 8: register-staged kernel only, ragged 13-column tiles
    (2, 40, 64, "RGB", (1, 2)),         # N = 2 (8 channel slots), TMA windows
    (8, 50, 176, "RGB", (1, 2)),        # N = 8 (24 channels), ragged height (50 -> 64, replicated rows)
    (4, 36, 100, "RGB", (1,)),          # N = 4, ragged width (100 -> 112, replicated columns), 3W % 16 = 12
    (6, 46, 90, "YUV420P", (1,)),       # N = 6, odd chroma planes (23 x 45), chroma repeated
    (8, 40, 96, "YUV444P", (1,)),       # planar frames
]


@pytest.mark.parametrize("N,H,W,fmt_name,kernels", CASES)
def test_first_layer_vs_float64(N, H, W, fmt_name, kernels):
    u = U()
    fmt = getattr(u, "COLOR_" + fmt_name)
    blob = synthetic.draw_weights(1, N, seed=11, bias_std=0.1)
    codec = u.Codec(1, N, 64, blob, "bf16", color=fmt)
    frames = frames_for(fmt, N, H, W, seed=H + W)
    fr = torch.from_numpy(frames).cuda()
    w, b = split_weights(blob, 1, N)["A1"]
    ch = channel_bytes(frames, fmt, N, H, W)
    Ho = -(-H // 16) * 8
    ref = reference_rows(ch, w, b, range(0, Ho))
    outs = []
    for k in kernels:
        got = codec.first_layer(fr, W, H, kernel=k)
        assert codec.sync_status() == 0
        check_rows(got.double().cpu(), ref, f"kernel {k}")
        outs.append(got)
    auto = codec.first_layer(fr, W, H, kernel=0)
    assert codec.sync_status() == 0
    for o in outs:  # both kernels issue the same MMAs on the same operands
        assert torch.equal(o, auto)


def test_first_layer_1080p_row_bands():
    """The 1080p chunk of the benchmark (8 frames, 1920 x 1080 padded to 1088): both kernels, output
    rows at the top edge, in the middle and at the bottom (where rows 1080..1087 are the last frame row
    repeated), every column and channel."""
    u = U()
    N, H, W = 8, 1080, 1920
    blob = synthetic.draw_weights(1, N, seed=0)
    codec = u.Codec(1, N, 4096, blob, "bf16")
    frames = synthetic.chunk_frames("1080p", seed=0)
    fr = torch.from_numpy(frames).cuda()
    w, b = split_weights(blob, 1, N)["A1"]
    ch = channel_bytes(frames, u.COLOR_RGB, N, H, W)
    got = {k: codec.first_layer(fr, W, H, kernel=k) for k in (1, 2)}
    assert codec.sync_status() == 0
    assert torch.equal(got[1], got[2])
    for r0, r1 in ((0, 10), (267, 277), (532, 544)):
        ref = reference_rows(ch, w, b, range(r0, r1))
        check_rows(got[2][r0:r1].double().cpu(), ref, f"rows {r0}..{r1}")


def test_first_layer_refusals():
    u = U()
    blob = synthetic.draw_weights(1, 2, seed=1)
    codec = u.Codec(1, 2, 64, blob, "bf16")
    fr = torch.zeros((2, 40, 200, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(u.UfvcError) as e:   # 600-byte rows: not whole 16-byte TMA rows
        codec.first_layer(fr, 200, 40, kernel=2)
    assert e.value.code == u.UFVC_ERR_ARG
    f32 = u.Codec(1, 2, 64, blob, "fp32")
    with pytest.raises(u.UfvcError) as e:   # the FP32 path packs the frames first
        f32.first_layer(fr, 200, 40)
    assert e.value.code == u.UFVC_ERR_UNSUPPORTED
