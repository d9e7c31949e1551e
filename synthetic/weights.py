"""Random-init weights for the plain chunk codec, as one flat float32 blob.

Blob layout (what ``ufvc_create`` and the oracle both read): the layers below in order; for each layer
its kernel as float32 [Cout][k][k][Cin] (NHWC-friendly, input channel fastest), then its bias
float32 [Cout].  Kernels are drawn N(0, 2/fan_in) with fan_in = k*k*Cin; biases N(0, bias_std^2).

Layer list for chunk length N (widths per architecture in ``ARCHS``; e0..e2 = analysis widths,
Cy = latent channels, Cz = hyper-latent channels, Cd1/Cd2 = decoder widths):

    A1 (e0, 3, 3N)   A2 (e1, 3, e0)   A3 (e2, 3, e1)   Xa (e2, 3, e2)   Xb (e2, 1, e2)   A4 (Cy, 3, e2)
    H1 (Cz, 3, Cy)   H2 (Cz, 3, Cz)
    S1 (4Cz, 3, Cz)  S2 (4Cz, 3, Cz)  S3 (2Cy, 1, Cz)
    then for each frame position f = 0..N-1:
    D0 (4Cd1, 3, Cy) R1a (Cd1, 3, Cd1) R1b (Cd1, 3, Cd1) U1 (4Cd2, 3, Cd1)
    R2a (Cd2, 3, Cd2) R2b (Cd2, 3, Cd2) U2 (4Cd2, 3, Cd2) U3 (12, 3, Cd2)
"""
from __future__ import annotations

import numpy as np

# arch 0: the tiny 64x64 workload; arch 1: the 1080p-family workload (720p, 480p and 4K use it too).
ARCHS = {
    0: dict(enc=(64, 96, 128), cy=128, cz=64, cd1=128, cd2=64),
    1: dict(enc=(64, 128, 192), cy=256, cz=128, cd1=128, cd2=64),
}


def layer_table(arch: int, n_frames: int) -> list[tuple[str, int, int, int]]:
    """[(name, Cout, k, Cin)] in blob order."""
    a = ARCHS[arch]
    e0, e1, e2 = a["enc"]
    cy, cz, cd1, cd2 = a["cy"], a["cz"], a["cd1"], a["cd2"]
    t = [("A1", e0, 3, 3 * n_frames), ("A2", e1, 3, e0), ("A3", e2, 3, e1),
         ("Xa", e2, 3, e2), ("Xb", e2, 1, e2), ("A4", cy, 3, e2),
         ("H1", cz, 3, cy), ("H2", cz, 3, cz),
         ("S1", 4 * cz, 3, cz), ("S2", 4 * cz, 3, cz), ("S3", 2 * cy, 1, cz)]
    for f in range(n_frames):
        t += [(f"D0.{f}", 4 * cd1, 3, cy), (f"R1a.{f}", cd1, 3, cd1), (f"R1b.{f}", cd1, 3, cd1),
              (f"U1.{f}", 4 * cd2, 3, cd1), (f"R2a.{f}", cd2, 3, cd2), (f"R2b.{f}", cd2, 3, cd2),
              (f"U2.{f}", 4 * cd2, 3, cd2), (f"U3.{f}", 12, 3, cd2)]
    return t


def weight_count(arch: int, n_frames: int) -> int:
    return sum(co * k * k * ci + co for _, co, k, ci in layer_table(arch, n_frames))


def draw_weights(arch: int, n_frames: int, seed: int = 0, bias_std: float = 0.01) -> np.ndarray:
    """Flat float32 blob (see module docstring)."""
    rng = np.random.default_rng(seed)
    parts = []
    for _, co, k, ci in layer_table(arch, n_frames):
        fan_in = k * k * ci
        parts.append(rng.normal(0.0, np.sqrt(2.0 / fan_in), size=co * k * k * ci).astype(np.float32))
        parts.append(rng.normal(0.0, bias_std, size=co).astype(np.float32))
    return np.ascontiguousarray(np.concatenate(parts))


def split_weights(blob: np.ndarray, arch: int, n_frames: int) -> dict[str, tuple[np.ndarray, np.ndarray]]:
    """name -> (kernel [Cout][k][k][Cin], bias [Cout]) views into the blob (for tests)."""
    out, off = {}, 0
    for name, co, k, ci in layer_table(arch, n_frames):
        n = co * k * k * ci
        out[name] = (blob[off:off + n].reshape(co, k, k, ci), blob[off + n:off + n + co])
        off += n + co
    assert off == blob.size
    return out


def mean_layer_table(arch: int) -> list[tuple[str, int, int, int]]:
    """[(name, Cout, k, Cin)] of the progressive-mean blob."""
    a = ARCHS[arch]
    cy, cz = a["cy"], a["cz"]
    t = []
    for k in (1, 2, 3):
        t += [(f"P{k}a", cz, 3, cy + cz), (f"P{k}b", cy, 1, cz)]
    return t


def draw_mean_weights(arch: int, seed: int = 0, bias_std: float = 0.01) -> np.ndarray:
    """Flat float32 blob of the progressive-mean layers, N(0, 2/fan_in) kernels (own random stream)."""
    rng = np.random.default_rng([seed, 4])
    parts = []
    for _, co, k, ci in mean_layer_table(arch):
        fan_in = k * k * ci
        parts.append(rng.normal(0.0, np.sqrt(2.0 / fan_in), size=co * k * k * ci).astype(np.float32))
        parts.append(rng.normal(0.0, bias_std, size=co).astype(np.float32))
    return np.ascontiguousarray(np.concatenate(parts))


def split_mean_weights(blob: np.ndarray, arch: int) -> dict[str, tuple[np.ndarray, np.ndarray]]:
    out, off = {}, 0
    for name, co, k, ci in mean_layer_table(arch):
        n = co * k * k * ci
        out[name] = (blob[off:off + n].reshape(co, k, k, ci), blob[off + n:off + n + co])
        off += n + co
    assert off == blob.size
    return out


def temporal_layer_table(arch: int, n_frames: int) -> list[tuple[str, int, int, int]]:
    """[(name, Cout, k, Cin)] of the temporal-context blob (Cf = Cc = 64)."""
    a = ARCHS[arch]
    cf = cc = 64
    t = [("EC", a["enc"][2], 1, cc), ("FD", 4 * cf, 3, a["cy"]), ("FC", cf, 1, cc), ("CG", cc, 3, cf),
         ("PC", a["cz"], 3, cc)]
    t += [(f"DF.{f}", a["cd1"], 1, cf) for f in range(n_frames)]
    return t


LOOP_GAIN = 0.1  # std factor of EC and FC, the two layers that feed a chunk's context into the next one


def draw_temporal_weights(arch: int, n_frames: int, seed: int = 0, bias_std: float = 0.01,
                          loop_gain: float = LOOP_GAIN) -> np.ndarray:
    """Flat float32 blob of the temporal-context layers, N(0, 2/fan_in) kernels (own random stream).  EC and
    FC, through which C_i reaches C_{i+1} (C_i -> EC -> y -> y^ -> F, and C_i -> FC -> F, then CG), are drawn
    with loop_gain times the standard deviation, so that the untrained recursion contracts instead of
    growing from chunk to chunk (at loop_gain = 1 the context grows about tenfold every few chunks)."""
    rng = np.random.default_rng([seed, 7])
    parts = []
    for name, co, k, ci in temporal_layer_table(arch, n_frames):
        fan_in = k * k * ci
        g = loop_gain if name in ("EC", "FC") else 1.0
        parts.append(rng.normal(0.0, g * np.sqrt(2.0 / fan_in), size=co * k * k * ci).astype(np.float32))
        parts.append(rng.normal(0.0, bias_std, size=co).astype(np.float32))
    return np.ascontiguousarray(np.concatenate(parts))


def split_temporal_weights(blob: np.ndarray, arch: int, n_frames: int) -> dict[str, tuple[np.ndarray, np.ndarray]]:
    out, off = {}, 0
    for name, co, k, ci in temporal_layer_table(arch, n_frames):
        n = co * k * k * ci
        out[name] = (blob[off:off + n].reshape(co, k, k, ci), blob[off + n:off + n + co])
        off += n + co
    assert off == blob.size
    return out


# DC-block model (arch 2): chunk width 512, frame-decoder width 256, context 128, latent 256, hyper-latent 128
DC = dict(c=512, cf=256, cc=128, cy=256, cz=128)


def dc_layer_table(n_frames: int) -> list[tuple[str, int, int, int]]:
    """[(name, Cout, k, Cin)] of the DC-block model's blob; a depth-wise layer ("*.dw") has Cin = 1."""
    c, cf, cc, cy, cz = DC["c"], DC["cf"], DC["cc"], DC["cy"], DC["cz"]

    def block(prefix, w):
        return [(f"{prefix}.a", w, 1, w), (f"{prefix}.dw", w, 3, 1), (f"{prefix}.b", w, 1, w),
                (f"{prefix}.c", 2 * w, 1, w), (f"{prefix}.d", w, 1, 2 * w)]
    t = [("PE", c, 1, 3 * n_frames * 64), ("EC", c, 1, cc)]
    for b in range(6):
        t += block(f"E{b}", c)
    t += [("ED", cy, 3, c), ("H1", cz, 3, cy), ("H2", cz, 3, cz), ("S1", 4 * cz, 3, cz), ("S2", 4 * cz, 3, cz),
          ("S3", 2 * cy, 1, cz), ("PC", cz, 3, cc), ("DU", 4 * c, 1, cy), ("FC", c, 1, cc)]
    for b in range(7):
        t += block(f"D{b}", c)
    for b in range(11):
        t += block(f"G{b}", c)
    t += [("GO", cc, 1, c)]
    for f in range(n_frames):
        t += [(f"FP.{f}", cf, 1, c)]
        for b in range(3):
            t += block(f"F{f}.{b}", cf)
        t += [(f"FO.{f}", 192, 1, cf)]
    return t


def draw_dc_weights(n_frames: int, seed: int = 0, bias_std: float = 0.01, branch_gain: float = 0.2,
                    loop_gain: float = 0.1) -> np.ndarray:
    """Flat float32 blob of the DC-block model, N(0, 2/fan_in) kernels, except: the last layer of each residual
    branch (".b", ".d") at branch_gain times that standard deviation, so that 24 chunk-level and 3 frame-level
    blocks of residual additions keep the activations' scale; and EC, FC (the context's way into the next
    chunk) and GO (the context generator's output) at loop_gain, so that the untrained context recursion
    contracts (with GO at full gain the context's scale grows about 1.3x per chunk)."""
    rng = np.random.default_rng([seed, 11])
    parts = []
    for name, co, k, ci in dc_layer_table(n_frames):
        g = loop_gain if name in ("EC", "FC", "GO") else branch_gain if name.endswith((".b", ".d")) else 1.0
        fan_in = k * k * ci
        parts.append(rng.normal(0.0, g * np.sqrt(2.0 / fan_in), size=co * k * k * ci).astype(np.float32))
        parts.append(rng.normal(0.0, bias_std, size=co).astype(np.float32))
    return np.ascontiguousarray(np.concatenate(parts))


def split_dc_weights(blob: np.ndarray, n_frames: int) -> dict[str, tuple[np.ndarray, np.ndarray]]:
    out, off = {}, 0
    for name, co, k, ci in dc_layer_table(n_frames):
        n = co * k * k * ci
        out[name] = (blob[off:off + n].reshape(co, k, k, ci), blob[off + n:off + n + co])
        off += n + co
    assert off == blob.size
    return out
