"""Test-side helpers: container parsing and rounding-boundary bands (no codec arithmetic)."""
import numpy as np


def parse_container(bits: bytes, cz: int) -> dict:
    """Split a bit-stream into header fields and its two sections (byte ranges)."""
    b = np.frombuffer(bits, np.uint8)
    hdr = (20 + cz + 3) // 4 * 4
    K = int.from_bytes(bits[12:16], "little")
    Kz = int.from_bytes(bits[16:20], "little")
    cz_counts = np.frombuffer(bits[hdr:hdr + 4 * Kz], np.uint32)
    zlen = (4 * Kz + 2 * int(cz_counts.sum()) + 3) // 4 * 4
    y0 = hdr + zlen
    y_counts = np.frombuffer(bits[y0:y0 + 4 * K], np.uint32)
    ylen = (4 * K + 2 * int(y_counts.sum()) + 3) // 4 * 4
    return dict(arch=b[5], N=b[6], qp=b[7], W=int.from_bytes(bits[8:10], "little"),
                H=int.from_bytes(bits[10:12], "little"), K=K, Kz=Kz, iz=b[20:20 + cz].copy(), hdr=hdr,
                zsec=bits[hdr:hdr + zlen], ysec=bits[y0:y0 + ylen], total=y0 + ylen)


def near_half_integer(v: np.ndarray, tau: np.ndarray) -> np.ndarray:
    """True where v lies within tau of k + 1/2 (where rounding may legitimately go either way)."""
    return np.abs(np.abs(v - np.floor(v)) - 0.5) < tau


def near_threshold(v: np.ndarray, thr: np.ndarray, tau: float) -> np.ndarray:
    """True where v lies within tau of any threshold."""
    d = np.min(np.abs(v.reshape(-1, 1) - thr.reshape(1, -1).astype(np.float64)), axis=1)
    return (d < tau).reshape(v.shape)


def psnr(a: np.ndarray, b: np.ndarray) -> float:
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10 * np.log10(1.0 / mse)
