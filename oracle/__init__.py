"""FP64 CPU oracle of the chunk-coding path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import this
package.  It wraps ``ufvc_oracle.c`` (plain C, FP64, OpenMP) through ctypes and shares no code with the
CUDA library.  See the C file's header for the paper passages and readings each function follows.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` (brute force on tiny tensors,
closed forms, library cross-checks, exact bit counts).  The rate-distortion behaviour of the
random-weight codec is "parity unpinned" (random weights have no published R-D to compare with).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ufvc_oracle.c")
_LIB = os.path.join(_HERE, "libufvc_oracle.so")

NBINS, NSYM, RMAX = 64, 511, 255


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, -O2, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_gelu.restype = C.c_double
        _lib.orc_gelu.argtypes = [C.c_double]
        _lib.orc_scale.restype = C.c_double
        _lib.orc_scale.argtypes = [C.c_int]
        _lib.orc_log_threshold.restype = C.c_double
        _lib.orc_log_threshold.argtypes = [C.c_int]
        _lib.orc_qstep.restype = C.c_double
        _lib.orc_qstep.argtypes = [C.c_int]
        _lib.orc_weight_count.restype = C.c_size_t
        _lib.orc_weight_count.argtypes = [C.c_int, C.c_int]
        _lib.orc_mean_weight_count.restype = C.c_size_t
        _lib.orc_mean_weight_count.argtypes = [C.c_int]
        _lib.orc_partition.restype = C.c_int
        _lib.orc_partition.argtypes = [C.c_int] * 4
        _lib.orc_rans_encode.restype = C.c_size_t
    return _lib


def _p(a: np.ndarray) -> C.c_void_p:
    assert a.flags["C_CONTIGUOUS"]
    return C.c_void_p(a.ctypes.data)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


# ---------------------------------------------------------------- primitives
def conv2d(x: np.ndarray, w: np.ndarray, b: np.ndarray, stride: int) -> np.ndarray:
    """x [H][W][Cin] float64, w [Cout][k][k][Cin] float32, b [Cout] float32 -> [Ho][Wo][Cout]."""
    x = np.ascontiguousarray(x, np.float64)
    w = np.ascontiguousarray(w, np.float32)
    b = np.ascontiguousarray(b, np.float32)
    H, W, Cin = x.shape
    Cout, k, _, _ = w.shape
    p = k // 2
    Ho, Wo = (H + 2 * p - k) // stride + 1, (W + 2 * p - k) // stride + 1
    out = np.empty((Ho, Wo, Cout), np.float64)
    lib().orc_conv2d(_p(x), H, W, Cin, _p(w), _p(b), Cout, k, stride, _p(out))
    return out


def gelu(x: float) -> float:
    return lib().orc_gelu(float(x))


def pixel_shuffle(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float64)
    H, W, C4 = x.shape
    out = np.empty((2 * H, 2 * W, C4 // 4), np.float64)
    lib().orc_pixel_shuffle(_p(x), H, W, C4 // 4, _p(out))
    return out


def scale(k: int) -> float:
    return lib().orc_scale(k)


def log_threshold(k: int) -> float:
    return lib().orc_log_threshold(k)


def qstep(qp: int) -> float:
    return lib().orc_qstep(qp)


def thresholds(qp: int) -> np.ndarray:
    thr = np.empty(NBINS - 1, np.float32)
    lib().orc_thresholds(qp, _p(thr))
    return thr


def build_tables() -> tuple[np.ndarray, np.ndarray]:
    """(freq [64][511] uint32, cum [64][512] uint32)."""
    freq = np.empty((NBINS, NSYM), np.uint32)
    cum = np.empty((NBINS, NSYM + 1), np.uint32)
    lib().orc_build_tables(_p(freq), _p(cum))
    return freq, cum


def weight_count(arch: int, n_frames: int) -> int:
    return int(lib().orc_weight_count(arch, n_frames))


def latent_dims(arch: int, H: int, W: int) -> dict:
    v = [C.c_int() for _ in range(6)]
    _check(lib().orc_latent_dims(arch, H, W, *[C.byref(t) for t in v]), "latent_dims")
    return dict(zip(["Hy", "Wy", "Hz", "Wz", "Cy", "Cz"], [t.value for t in v]))


# ---------------------------------------------------------------- rANS
def rans_encode(sym: np.ndarray, tab: np.ndarray, K: int, freq: np.ndarray | None = None,
                cum: np.ndarray | None = None, offset: int = RMAX) -> bytes:
    if freq is None:
        freq, cum = build_tables()
    sym = np.ascontiguousarray(sym, np.int16)
    tab = np.ascontiguousarray(tab, np.uint8)
    freq = np.ascontiguousarray(freq, np.uint32)
    cum = np.ascontiguousarray(cum, np.uint32)
    nsym = freq.shape[1]
    n = sym.size
    cap = 4 * K + 2 * (n + 2 * K) + 4
    out = np.empty(cap, np.uint8)
    size = lib().orc_rans_encode(_p(sym), _p(tab), C.c_size_t(n), K, _p(freq), _p(cum), nsym, offset,
                                 _p(out), C.c_size_t(cap))
    if size == 0:
        raise RuntimeError("oracle rans_encode: capacity")
    return out[:size].tobytes()


def rans_decode(buf: bytes, tab: np.ndarray, n: int, K: int, freq: np.ndarray | None = None,
                cum: np.ndarray | None = None, offset: int = RMAX) -> tuple[np.ndarray, int]:
    if freq is None:
        freq, cum = build_tables()
    tab = np.ascontiguousarray(tab, np.uint8)
    freq = np.ascontiguousarray(freq, np.uint32)
    cum = np.ascontiguousarray(cum, np.uint32)
    a = np.frombuffer(buf, np.uint8).copy() if len(buf) else np.zeros(1, np.uint8)
    sym = np.empty(max(n, 1), np.int16)
    used = C.c_size_t()
    rc = lib().orc_rans_decode(_p(a), C.c_size_t(len(buf)), _p(tab), C.c_size_t(n), K, _p(freq), _p(cum),
                               freq.shape[1], offset, _p(sym), C.byref(used))
    _check(rc, "rans_decode")
    return sym[:n], used.value


# ---------------------------------------------------------------- colour interface
RGB, RGB_BT709, YUV444P, YUV420P = 0, 1, 2, 3


def frame_bytes(fmt: int, H: int, W: int) -> int:
    lib().orc_frame_bytes.restype = C.c_size_t
    return int(lib().orc_frame_bytes(fmt, H, W))


def color_in(fmt: int, frames: np.ndarray, N: int, H: int, W: int) -> np.ndarray:
    """Caller's frames (N * frame_bytes uint8) -> the network's channels [N][H][W][3] in [0, 1]."""
    f = np.ascontiguousarray(frames, np.uint8).ravel()
    assert f.size == N * frame_bytes(fmt, H, W)
    x = np.empty((N, H, W, 3), np.float64)
    _check(lib().orc_color_in(fmt, _p(f), N, H, W, _p(x)), "color_in")
    return x


def color_out(fmt: int, x: np.ndarray, N: int, H: int, W: int) -> np.ndarray:
    """Reconstruction [N][H][W][3] in [0, 1] -> the format's layout as values in [0, 1] (N * frame_bytes)."""
    x = np.ascontiguousarray(x, np.float64)
    out = np.empty(N * frame_bytes(fmt, H, W), np.float64)
    _check(lib().orc_color_out(fmt, _p(x), N, H, W, _p(out)), "color_out")
    return out


# ---------------------------------------------------------------- network stages
def analysis_x(arch: int, x: np.ndarray, weights: np.ndarray) -> np.ndarray:
    """Latent from the network's input channels x [N][H][W][3] in [0, 1]."""
    x = np.ascontiguousarray(x, np.float64)
    N, H, W, _ = x.shape
    d = latent_dims(arch, H, W)
    y = np.empty((d["Hy"], d["Wy"], d["Cy"]), np.float64)
    _check(lib().orc_analysis_x(arch, N, _p(x), H, W, _p(weights), _p(y)), "analysis_x")
    return y


def analysis(arch: int, frames: np.ndarray, weights: np.ndarray) -> np.ndarray:
    frames = np.ascontiguousarray(frames, np.uint8)
    N, H, W, _ = frames.shape
    d = latent_dims(arch, H, W)
    y = np.empty((d["Hy"], d["Wy"], d["Cy"]), np.float64)
    _check(lib().orc_analysis(arch, N, _p(frames), H, W, _p(weights), _p(y)), "analysis")
    return y


def hyper_analysis(arch: int, N: int, y: np.ndarray, weights: np.ndarray) -> np.ndarray:
    y = np.ascontiguousarray(y, np.float64)
    Hy, Wy, _ = y.shape
    cz = {0: 64, 1: 128, 2: 128}[arch]
    z = np.empty(((Hy + 3) // 4, (Wy + 3) // 4, cz), np.float64)
    _check(lib().orc_hyper_analysis(arch, N, _p(y), Hy, Wy, _p(weights), _p(z)), "hyper_analysis")
    return z


def quantize_z(z: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    z = np.ascontiguousarray(z, np.float64)
    Hz, Wz, Cz = z.shape
    zhat = np.empty(z.shape, np.int16)
    iz = np.empty(Cz, np.uint8)
    _check(lib().orc_quantize_z(_p(z), Hz * Wz, Cz, _p(zhat), _p(iz)), "quantize_z")
    return zhat, iz


def hyper_synthesis(arch: int, N: int, zhat: np.ndarray, Hy: int, Wy: int, weights: np.ndarray,
                    want_s: bool = False):
    """-> (mu, log sigma), or with want_s (mu, log sigma, s): s = the S2 feature map [Hy][Wy][Cz], the
    prior of the progressive mean steps."""
    zhat = np.ascontiguousarray(zhat, np.int16)
    Hz, Wz, _ = zhat.shape
    cy, cz = {0: (128, 64), 1: (256, 128), 2: (256, 128)}[arch]
    mu = np.empty((Hy, Wy, cy), np.float64)
    ls = np.empty((Hy, Wy, cy), np.float64)
    sp = np.empty((Hy, Wy, cz), np.float64)
    _check(lib().orc_hyper_synthesis_s(arch, N, _p(zhat), Hz, Wz, Hy, Wy, _p(weights), _p(mu), _p(ls), _p(sp)),
           "hyper_synthesis")
    return (mu, ls, sp) if want_s else (mu, ls)


# ---------------------------------------------------------------- progressive means (Sec. 3.4)
def mean_weight_count(arch: int) -> int:
    return int(lib().orc_mean_weight_count(arch))


def partition(h: int, w: int, c: int, cy: int) -> int:
    return int(lib().orc_partition(h, w, c, cy))


def partition_map(Hy: int, Wy: int, cy: int) -> np.ndarray:
    """[Hy][Wy][Cy] uint8: the partition (0..3) of each latent element."""
    out = np.empty((Hy, Wy, cy), np.uint8)
    lib().orc_partition_map(Hy, Wy, cy, _p(out))
    return out


def mean_step(arch: int, k: int, yhat: np.ndarray, s: np.ndarray, mean_weights: np.ndarray) -> np.ndarray:
    """mu^k (k = 1..3) from yhat restricted to partitions < k and the prior s."""
    yhat = np.ascontiguousarray(yhat, np.float64)
    s = np.ascontiguousarray(s, np.float64)
    mw = np.ascontiguousarray(mean_weights, np.float32)
    Hy, Wy, cy = yhat.shape
    mu = np.empty((Hy, Wy, cy), np.float64)
    _check(lib().orc_mean_step(arch, k, _p(yhat), _p(s), Hy, Wy, _p(mw), _p(mu)), "mean_step")
    return mu


def progressive_means(arch: int, y: np.ndarray | None, rhat: np.ndarray, mu0: np.ndarray, s: np.ndarray, qp: int,
                      mean_weights: np.ndarray):
    """The four partition steps.  Encoder (y given): -> (rhat, yhat, mu_used) with rhat recomputed on
    partitions 1..3; decoder (y None): rhat is the decoded one."""
    mu0 = np.ascontiguousarray(mu0, np.float64)
    s = np.ascontiguousarray(s, np.float64)
    mw = np.ascontiguousarray(mean_weights, np.float32)
    rh = np.array(rhat, dtype=np.int16, order="C", copy=True)
    Hy, Wy, _ = mu0.shape
    yhat = np.empty(mu0.shape, np.float64)
    mu_used = np.empty(mu0.shape, np.float64)
    yy = None if y is None else np.ascontiguousarray(y, np.float64)
    _check(lib().orc_progressive_means(arch, _p(yy) if yy is not None else None, _p(rh), _p(mu0), _p(s), Hy, Wy,
                                       qp, _p(mw), _p(yhat), _p(mu_used)), "progressive_means")
    return rh, yhat, mu_used


def quantize_y(y: np.ndarray, mu: np.ndarray, logsig: np.ndarray, qp: int):
    y, mu, logsig = (np.ascontiguousarray(a, np.float64) for a in (y, mu, logsig))
    rhat = np.empty(y.shape, np.int16)
    idx = np.empty(y.shape, np.uint8)
    _check(lib().orc_quantize_y(_p(y), _p(mu), _p(logsig), C.c_size_t(y.size), qp, _p(rhat), _p(idx)),
           "quantize_y")
    return rhat, idx


def scale_index(logsig: np.ndarray, qp: int) -> np.ndarray:
    logsig = np.ascontiguousarray(logsig, np.float64)
    idx = np.empty(logsig.shape, np.uint8)
    _check(lib().orc_scale_index(_p(logsig), C.c_size_t(logsig.size), qp, _p(idx)), "scale_index")
    return idx


def synthesis(arch: int, N: int, yhat: np.ndarray, H: int, W: int, weights: np.ndarray) -> np.ndarray:
    yhat = np.ascontiguousarray(yhat, np.float64)
    Hy, Wy, _ = yhat.shape
    out = np.empty((N, H, W, 3), np.float64)
    _check(lib().orc_synthesis(arch, N, _p(yhat), Hy, Wy, H, W, _p(weights), _p(out)), "synthesis")
    return out


class _Debug(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("y", "z", "zhat", "iz", "mu", "logsig", "rhat", "idx", "s", "yhat")]


def encode_chunk(arch: int, frames: np.ndarray, qp: int, K: int, weights: np.ndarray, debug: bool = False,
                 mean_weights: np.ndarray | None = None):
    """-> bit-stream bytes (and, with debug, a dict of every intermediate).  With mean_weights the
    stream is version 2 (progressive means on partitions 1..3; debug "mu" is the mean each element was
    coded with)."""
    frames = np.ascontiguousarray(frames, np.uint8)
    N, H, W, _ = frames.shape
    d = latent_dims(arch, H, W)
    ny = d["Hy"] * d["Wy"] * d["Cy"]
    nz = d["Hz"] * d["Wz"] * d["Cz"]
    cap = 64 + d["Cz"] + 4 * (K + min(K, nz)) + 2 * (ny + nz + 4 * K) + 16
    out = np.empty(cap, np.uint8)
    nbytes = C.c_size_t()
    dbg = None
    arrs = {}
    if debug:
        arrs = dict(y=np.empty((d["Hy"], d["Wy"], d["Cy"])), z=np.empty((d["Hz"], d["Wz"], d["Cz"])),
                    zhat=np.empty((d["Hz"], d["Wz"], d["Cz"]), np.int16), iz=np.empty(d["Cz"], np.uint8),
                    mu=np.empty((d["Hy"], d["Wy"], d["Cy"])), logsig=np.empty((d["Hy"], d["Wy"], d["Cy"])),
                    rhat=np.empty((d["Hy"], d["Wy"], d["Cy"]), np.int16),
                    idx=np.empty((d["Hy"], d["Wy"], d["Cy"]), np.uint8),
                    s=np.empty((d["Hy"], d["Wy"], d["Cz"])), yhat=np.empty((d["Hy"], d["Wy"], d["Cy"])))
        dbg = _Debug(**{k: v.ctypes.data for k, v in arrs.items()})
    mw = None if mean_weights is None else np.ascontiguousarray(mean_weights, np.float32)
    rc = lib().orc_encode_chunk(arch, N, _p(frames), H, W, qp, K, _p(weights), _p(mw) if mw is not None else None,
                                _p(out), C.c_size_t(cap),
                                C.byref(nbytes), C.byref(dbg) if dbg is not None else None)
    _check(rc, "encode_chunk")
    bits = out[:nbytes.value].tobytes()
    return (bits, arrs) if debug else bits


def decode_chunk(arch: int, N: int, bits: bytes, H: int, W: int, weights: np.ndarray,
                 want_frames: bool = True, mean_weights: np.ndarray | None = None):
    """-> (frames [N][H][W][3] float64 in [0,1] or None, yhat [Hy][Wy][Cy])."""
    d = latent_dims(arch, H, W)
    a = np.frombuffer(bits, np.uint8).copy()
    yhat = np.empty((d["Hy"], d["Wy"], d["Cy"]), np.float64)
    frames = np.empty((N, H, W, 3), np.float64) if want_frames else None
    mw = None if mean_weights is None else np.ascontiguousarray(mean_weights, np.float32)
    rc = lib().orc_decode_chunk(arch, N, _p(a), C.c_size_t(len(bits)), H, W, _p(weights),
                                _p(mw) if mw is not None else None,
                                _p(frames) if want_frames else None, _p(yhat))
    _check(rc, "decode_chunk")
    return frames, yhat


# ---------------------------------------------------------------- temporal chunk context
class _Opts(C.Structure):
    _fields_ = [("pm", C.c_void_p), ("tw", C.c_void_p), ("c_in", C.c_void_p), ("c_out", C.c_void_p)]


def temporal_weight_count(arch: int, N: int) -> int:
    lib().orc_temporal_weight_count.restype = C.c_size_t
    return int(lib().orc_temporal_weight_count(arch, N))


def context_dims(arch: int, H: int, W: int) -> tuple[int, int, int]:
    v = [C.c_int() for _ in range(3)]
    _check(lib().orc_context_dims(arch, H, W, *[C.byref(t) for t in v]), "context_dims")
    return tuple(t.value for t in v)


def chunk_feature(arch: int, N: int, yhat: np.ndarray, tw: np.ndarray, c_in: np.ndarray | None) -> np.ndarray:
    """F_i = GELU(PS(FD(y^))) + FC(C_i)  [2Hy][2Wy][64]; c_in None = the first chunk (C = 0)."""
    yhat = np.ascontiguousarray(yhat, np.float64)
    tw = np.ascontiguousarray(tw, np.float32)
    Hy, Wy, _ = yhat.shape
    ci = None if c_in is None else np.ascontiguousarray(c_in, np.float64)
    F = np.empty((2 * Hy, 2 * Wy, 64), np.float64)
    _check(lib().orc_chunk_feature(arch, N, _p(yhat), Hy, Wy, _p(tw), _p(ci) if ci is not None else None, _p(F)),
           "chunk_feature")
    return F


def context_next(arch: int, N: int, F: np.ndarray, tw: np.ndarray) -> np.ndarray:
    F = np.ascontiguousarray(F, np.float64)
    tw = np.ascontiguousarray(tw, np.float32)
    H8, W8, _ = F.shape
    c = np.empty((H8, W8, 64), np.float64)
    _check(lib().orc_context_next(arch, N, _p(F), H8, W8, _p(tw), _p(c)), "context_next")
    return c


def context_terms(arch: int, N: int, c_in: np.ndarray | None, H8: int, W8: int, tw: np.ndarray):
    """(EC(C_i) [H8][W8][e2], PC(C_i) [H8/2][W8/2][Cz])."""
    tw = np.ascontiguousarray(tw, np.float32)
    e2, cz = {0: (128, 64), 1: (192, 128)}[arch]
    ec = np.empty((H8, W8, e2), np.float64)
    pc = np.empty((H8 // 2, W8 // 2, cz), np.float64)
    ci = None if c_in is None else np.ascontiguousarray(c_in, np.float64)
    _check(lib().orc_context_terms(arch, N, _p(ci) if ci is not None else None, H8, W8, _p(tw), _p(ec), _p(pc)),
           "context_terms")
    return ec, pc


def hyper_synthesis_add(arch: int, N: int, zhat: np.ndarray, Hy: int, Wy: int, weights: np.ndarray,
                        add_s: np.ndarray):
    """Hyper-synthesis with add_s [Hy][Wy][Cz] added to the features before S3 -> (mu, log sigma, s)."""
    zhat = np.ascontiguousarray(zhat, np.int16)
    Hz, Wz, _ = zhat.shape
    cy, cz = {0: (128, 64), 1: (256, 128), 2: (256, 128)}[arch]
    mu = np.empty((Hy, Wy, cy), np.float64)
    ls = np.empty((Hy, Wy, cy), np.float64)
    sp = np.empty((Hy, Wy, cz), np.float64)
    add = np.ascontiguousarray(add_s, np.float64)
    _check(lib().orc_hyper_synthesis_add(arch, N, _p(zhat), Hz, Wz, Hy, Wy, _p(weights), _p(add), _p(mu), _p(ls),
                                         _p(sp)), "hyper_synthesis_add")
    return mu, ls, sp


def synthesis_f(arch: int, N: int, yhat: np.ndarray, F: np.ndarray, H: int, W: int, weights: np.ndarray,
                tw: np.ndarray) -> np.ndarray:
    yhat = np.ascontiguousarray(yhat, np.float64)
    F = np.ascontiguousarray(F, np.float64)
    tw = np.ascontiguousarray(tw, np.float32)
    Hy, Wy, _ = yhat.shape
    out = np.empty((N, H, W, 3), np.float64)
    _check(lib().orc_synthesis_f(arch, N, _p(yhat), Hy, Wy, H, W, _p(weights), _p(F), _p(tw), _p(out)),
           "synthesis_f")
    return out


def encode_chunk_t(arch: int, frames: np.ndarray, qp: int, K: int, weights: np.ndarray, tw: np.ndarray,
                   c_in: np.ndarray | None, mean_weights: np.ndarray | None = None, debug: bool = False):
    """Temporal-context encode: -> (bits, C_{i+1}) or, with debug, (bits, C_{i+1}, intermediates)."""
    frames = np.ascontiguousarray(frames, np.uint8)
    N, H, W, _ = frames.shape
    d = latent_dims(arch, H, W)
    H8, W8, Cc = context_dims(arch, H, W)
    ny = d["Hy"] * d["Wy"] * d["Cy"]
    nz = d["Hz"] * d["Wz"] * d["Cz"]
    cap = 64 + d["Cz"] + 4 * (K + min(K, nz)) + 2 * (ny + nz + 4 * K) + 16
    out = np.empty(cap, np.uint8)
    nbytes = C.c_size_t()
    tw = None if tw is None else np.ascontiguousarray(tw, np.float32)  # None for the DC-block model (arch 2)
    mw = None if mean_weights is None else np.ascontiguousarray(mean_weights, np.float32)
    ci = None if c_in is None else np.ascontiguousarray(c_in, np.float64)
    c_out = np.empty((H8, W8, Cc), np.float64)
    o = _Opts(mw.ctypes.data if mw is not None else None, tw.ctypes.data if tw is not None else None,
              ci.ctypes.data if ci is not None else None, c_out.ctypes.data)
    arrs, dbg = {}, None
    if debug:
        arrs = dict(y=np.empty((d["Hy"], d["Wy"], d["Cy"])), z=np.empty((d["Hz"], d["Wz"], d["Cz"])),
                    zhat=np.empty((d["Hz"], d["Wz"], d["Cz"]), np.int16), iz=np.empty(d["Cz"], np.uint8),
                    mu=np.empty((d["Hy"], d["Wy"], d["Cy"])), logsig=np.empty((d["Hy"], d["Wy"], d["Cy"])),
                    rhat=np.empty((d["Hy"], d["Wy"], d["Cy"]), np.int16),
                    idx=np.empty((d["Hy"], d["Wy"], d["Cy"]), np.uint8),
                    s=np.empty((d["Hy"], d["Wy"], d["Cz"])), yhat=np.empty((d["Hy"], d["Wy"], d["Cy"])))
        dbg = _Debug(**{k: v.ctypes.data for k, v in arrs.items()})
    rc = lib().orc_encode_chunk_opts(arch, N, _p(frames), H, W, qp, K, _p(weights), C.byref(o), _p(out),
                                     C.c_size_t(cap), C.byref(nbytes), C.byref(dbg) if dbg is not None else None)
    _check(rc, "encode_chunk_opts")
    bits = out[:nbytes.value].tobytes()
    return (bits, c_out, arrs) if debug else (bits, c_out)


def decode_chunk_t(arch: int, N: int, bits: bytes, H: int, W: int, weights: np.ndarray, tw: np.ndarray,
                   c_in: np.ndarray | None, mean_weights: np.ndarray | None = None):
    """Temporal-context decode: -> (frames [N][H][W][3] in [0, 1], y^, C_{i+1})."""
    d = latent_dims(arch, H, W)
    H8, W8, Cc = context_dims(arch, H, W)
    a = np.frombuffer(bits, np.uint8).copy()
    yhat = np.empty((d["Hy"], d["Wy"], d["Cy"]), np.float64)
    frames = np.empty((N, H, W, 3), np.float64)
    tw = None if tw is None else np.ascontiguousarray(tw, np.float32)
    mw = None if mean_weights is None else np.ascontiguousarray(mean_weights, np.float32)
    ci = None if c_in is None else np.ascontiguousarray(c_in, np.float64)
    c_out = np.empty((H8, W8, Cc), np.float64)
    o = _Opts(mw.ctypes.data if mw is not None else None, tw.ctypes.data if tw is not None else None,
              ci.ctypes.data if ci is not None else None, c_out.ctypes.data)
    rc = lib().orc_decode_chunk_opts(arch, N, _p(a), C.c_size_t(len(bits)), H, W, _p(weights), C.byref(o),
                                     _p(frames), _p(yhat))
    _check(rc, "decode_chunk_opts")
    return frames, yhat, c_out


# ---------------------------------------------------------------- DC-block model (arch 2)
DC_C, DC_CF, DC_CC = 512, 256, 128


def dc_weight_count(N: int) -> int:
    lib().orc_dc_weight_count.restype = C.c_size_t
    return int(lib().orc_dc_weight_count(N))


def dw_conv(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Depth-wise 3x3, zero padding 1: x [H][W][C], w [C][3][3][1], b [C]."""
    x = np.ascontiguousarray(x, np.float64)
    H, W, Cc = x.shape
    out = np.empty_like(x)
    lib().orc_dw_conv(_p(x), H, W, Cc, _p(np.ascontiguousarray(w, np.float32)), _p(np.ascontiguousarray(b, np.float32)),
                      _p(out))
    return out


def dc_analysis(N: int, x: np.ndarray, weights: np.ndarray, c_in: np.ndarray | None) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float64)
    _, H, W, _ = x.shape
    d = latent_dims(2, H, W)
    y = np.empty((d["Hy"], d["Wy"], d["Cy"]), np.float64)
    ci = None if c_in is None else np.ascontiguousarray(c_in, np.float64)
    _check(lib().orc_dc_analysis(N, _p(x), H, W, _p(weights), _p(ci) if ci is not None else None, _p(y)), "dc_analysis")
    return y


def dc_prior_term(N: int, c_in: np.ndarray | None, H8: int, W8: int, weights: np.ndarray) -> np.ndarray:
    pc = np.empty((H8 // 2, W8 // 2, 128), np.float64)
    ci = None if c_in is None else np.ascontiguousarray(c_in, np.float64)
    _check(lib().orc_dc_prior_term(N, _p(ci) if ci is not None else None, H8, W8, _p(weights), _p(pc)), "dc_prior_term")
    return pc


def dc_trunk(N: int, yhat: np.ndarray, weights: np.ndarray, c_in: np.ndarray | None, want_c_out: bool = True):
    """Chunk decoder (-> F [2Hy][2Wy][512]) and context generation (-> C_{i+1} [2Hy][2Wy][128])."""
    yhat = np.ascontiguousarray(yhat, np.float64)
    Hy, Wy, _ = yhat.shape
    F = np.empty((2 * Hy, 2 * Wy, DC_C), np.float64)
    c_out = np.empty((2 * Hy, 2 * Wy, DC_CC), np.float64) if want_c_out else None
    ci = None if c_in is None else np.ascontiguousarray(c_in, np.float64)
    _check(lib().orc_dc_trunk(N, _p(yhat), Hy, Wy, _p(weights), _p(ci) if ci is not None else None, _p(F),
                              _p(c_out) if c_out is not None else None), "dc_trunk")
    return F, c_out


def dc_frames(N: int, F: np.ndarray, H: int, W: int, weights: np.ndarray) -> np.ndarray:
    F = np.ascontiguousarray(F, np.float64)
    H8, W8, _ = F.shape
    out = np.empty((N, H, W, 3), np.float64)
    _check(lib().orc_dc_frames(N, _p(F), H8, W8, H, W, _p(weights), _p(out)), "dc_frames")
    return out


def num_threads() -> int:
    return int(lib().orc_num_threads())
