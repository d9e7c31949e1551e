"""Moving-texture video chunks (seeded, synthetic).

Each RGB channel is a smooth random field, the sum of 8 random 2-D sinusoids

    F(x, y) = sum_j a_j * sin(2*pi*(u_j*x + v_j*y)/P + phi_j),
    a_j ~ U(0.5, 1),  u_j, v_j ~ U(-4, 4) cycles per period P,  phi_j ~ U(0, 2*pi),

mapped to 127.5 + 127.5 * F / sum_j a_j.  Frame n samples the field at (x + sx_n, y + sy_n), where the
integer shift (sx_n, sy_n) is a cumulative sum of per-frame steps drawn from U{-max_step..max_step}^2
(frame 0 is unshifted).  Optionally a fraction of the block x block tiles of every frame after the first
is replaced by a fresh field (new content entering the scene).  Integer noise U{-noise..noise} is added
and the result clipped to [0, 255].

The tiny workload uses P = 64, max_step = 3, no refresh; the 1080p workload uses P = width (frequencies
scaled to the frame width), max_step = 16 and 10 % refreshed 64x64 blocks.
"""
from __future__ import annotations

import numpy as np


def _field(rng: np.random.Generator, xs: np.ndarray, ys: np.ndarray, period: float) -> np.ndarray:
    """Evaluate one channel's field on the grid ys x xs (float64, range [-sum a, sum a])."""
    a = rng.uniform(0.5, 1.0, 8)
    u = rng.uniform(-4.0, 4.0, 8)
    v = rng.uniform(-4.0, 4.0, 8)
    phi = rng.uniform(0.0, 2.0 * np.pi, 8)
    out = np.zeros((ys.size, xs.size), np.float64)
    for j in range(8):
        # sin(A + B) = sin A cos B + cos A sin B keeps the evaluation separable (outer products).
        ax = 2.0 * np.pi * u[j] * xs / period + phi[j]
        by = 2.0 * np.pi * v[j] * ys / period
        out += a[j] * (np.outer(np.cos(by), np.sin(ax)) + np.outer(np.sin(by), np.cos(ax)))
    return out / a.sum()


def moving_texture(seed: int, n_frames: int, height: int, width: int, max_step: int,
                   period: float | None = None, refresh: float = 0.0, block: int = 64,
                   noise: int = 4) -> np.ndarray:
    """Return uint8 frames [n_frames][height][width][3] (RGB, C-contiguous)."""
    rng = np.random.default_rng(seed)
    period = float(width if period is None else period)
    steps = rng.integers(-max_step, max_step + 1, size=(n_frames, 2))
    steps[0] = 0
    shifts = np.cumsum(steps, axis=0)
    # Draw the per-channel field parameters once; evaluate per frame at shifted coordinates.
    chan_seeds = rng.integers(0, 2**63 - 1, size=3)
    frames = np.empty((n_frames, height, width, 3), np.uint8)
    nby, nbx = -(-height // block), -(-width // block)
    for n in range(n_frames):
        sx, sy = shifts[n]
        xs = np.arange(width, dtype=np.float64) + sx
        ys = np.arange(height, dtype=np.float64) + sy
        img = np.empty((height, width, 3), np.float64)
        for c in range(3):
            img[:, :, c] = _field(np.random.default_rng(int(chan_seeds[c])), xs, ys, period)
        if refresh > 0.0 and n > 0:
            nblk = int(round(refresh * nby * nbx))
            picks = rng.choice(nby * nbx, size=nblk, replace=False)
            for b in picks:
                by, bx = divmod(int(b), nbx)
                y0, x0 = by * block, bx * block
                y1, x1 = min(y0 + block, height), min(x0 + block, width)
                bxs = np.arange(x0, x1, dtype=np.float64)
                bys = np.arange(y0, y1, dtype=np.float64)
                for c in range(3):
                    img[y0:y1, x0:x1, c] = _field(rng, bxs, bys, period)
        pix = 127.5 + 127.5 * img
        pix = np.rint(pix) + rng.integers(-noise, noise + 1, size=pix.shape)
        frames[n] = np.clip(pix, 0, 255).astype(np.uint8)
    return frames


def chunk_frames(name: str, seed: int = 0) -> np.ndarray:
    """The named synthetic workloads: 'tiny' (4 frames 64x64), '1080p' (8 frames 1920x1080),
    '720p' / '480p' / '4k' (8 frames; serving-mix resolutions)."""
    if name == "tiny":
        return moving_texture(seed, 4, 64, 64, max_step=3, period=64)
    sizes = {"1080p": (1080, 1920), "720p": (720, 1280), "480p": (480, 854), "4k": (2160, 3840)}
    h, w = sizes[name]
    return moving_texture(seed, 8, h, w, max_step=16, refresh=0.10)
