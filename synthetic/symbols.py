"""Entropy-coding stress symbols: quantised latents drawn as r = clip(round(mu + Laplace(0, b)), -255, 255)
with mu ~ N(0, 1) and b log-uniform on [0.11, 64], independently per element.

Returns the symbols and the per-element b; mapping b to a scale index is the codec's job (each side does
it with its own threshold table), not this module's.
"""
from __future__ import annotations

import numpy as np


def laplace_symbols(n: int, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    rng = np.random.default_rng(seed)
    mu = rng.normal(0.0, 1.0, n)
    b = np.exp(rng.uniform(np.log(0.11), np.log(64.0), n))
    r = np.clip(np.rint(mu + rng.laplace(0.0, b)), -255, 255).astype(np.int16)
    return r, b
