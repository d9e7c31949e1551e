"""Thin ctypes binding of libufvc.so (include/ufvc.h).  Argument marshalling only: every step of the
chunk path runs in the library's CUDA kernels.  Device buffers are torch CUDA tensors; the stream is
torch's current stream unless one is given.  There is no CPU fallback: if the library cannot be
loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

_LIB_PATH = _build.LIB
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libufvc.so not built ({_LIB_PATH}); run `python -m paper_2606_04410_b300.build`")
lib = C.CDLL(_LIB_PATH)

UFVC_OK, UFVC_ERR_ARG, UFVC_ERR_CAPACITY, UFVC_ERR_CORRUPT, UFVC_ERR_OOM, UFVC_ERR_CUDA, UFVC_ERR_TIMEOUT, \
    UFVC_ERR_UNSUPPORTED, UFVC_PENDING = range(9)
STATUS_NAMES = ["OK", "ERR_ARG", "ERR_CAPACITY", "ERR_CORRUPT", "ERR_OOM", "ERR_CUDA", "ERR_TIMEOUT",
                "ERR_UNSUPPORTED", "PENDING"]
PRECISIONS = {"fp32": 0, "bf16": 1, "fp8": 2}

# Every symbol the header declares (checked by the CPU test suite).
EXPORTS = [
    "ufvc_weight_count", "ufvc_create", "ufvc_destroy", "ufvc_layer_shape", "ufvc_latent_dims",
    "ufvc_max_bitstream_bytes", "ufvc_encode_chunk", "ufvc_decode_chunk", "ufvc_decode_chunk_f32",
    "ufvc_encode_chunk_host", "ufvc_decode_chunk_host", "ufvc_sync_status", "ufvc_encode_stages",
    "ufvc_hyper_synthesis", "ufvc_quantize", "ufvc_synthesize", "ufvc_rans_encode", "ufvc_rans_decode",
    "ufvc_get_tables", "ufvc_set_profiling", "ufvc_get_profile", "ufvc_last_error", "ufvc_conv_layer",
    "ufvc_rans_encode_noalloc", "ufvc_decode_chunk_dev", "ufvc_server_create", "ufvc_server_destroy",
    "ufvc_server_open_stream", "ufvc_server_stream_buffers", "ufvc_server_submit", "ufvc_server_submit_many", "ufvc_server_poll",
    "ufvc_server_wait", "ufvc_server_stats_get", "ufvc_server_last_error", "ufvc_calibrate_fp8",
    "ufvc_get_fp8_scales", "ufvc_mean_weight_count", "ufvc_set_progressive_means", "ufvc_progressive_means",
    "ufvc_frame_bytes", "ufvc_set_color_format", "ufvc_temporal_weight_count", "ufvc_set_temporal_context",
    "ufvc_context_bytes", "ufvc_encode_chunk_tc", "ufvc_decode_chunk_tc", "ufvc_encode_stages_tc",
    "ufvc_server_set_temporal_context", "ufvc_server_calibrate_fp8", "ufvc_server_set_progressive_means", "ufvc_pipe_create",
    "ufvc_pipe_submit", "ufvc_pipe_wait", "ufvc_pipe_destroy", "ufvc_first_layer",
    "ufvc_set_table_wait_limit", "ufvc_set_conv_pairs", "ufvc_encode_chunks", "ufvc_decode_chunks",
]
COLOR_RGB, COLOR_RGB_BT709, COLOR_YUV444P, COLOR_YUV420P = range(4)
UFVC_OP_ENCODE, UFVC_OP_DECODE = 0, 1


class ufvc_config(C.Structure):
    _fields_ = [("arch", C.c_int), ("chunk_len", C.c_int), ("lanes", C.c_int), ("precision", C.c_int),
                ("device", C.c_int)]


class ufvc_result(C.Structure):
    _fields_ = [("status", C.c_int), ("op", C.c_int), ("stream_id", C.c_int), ("slot", C.c_int),
                ("submit_ms", C.c_double), ("start_ms", C.c_double), ("done_ms", C.c_double),
                ("nbytes", C.c_uint64), ("batch", C.c_int)]


class ufvc_server_stats(C.Structure):
    _fields_ = [("slots", C.c_int), ("busy_slots", C.c_int), ("queued", C.c_int), ("graphs", C.c_int),
                ("completed", C.c_uint64), ("hbm_used", C.c_size_t), ("hbm_cap", C.c_size_t),
                ("batches", C.c_uint64), ("batched", C.c_uint64)]


_vp, _sz, _i = C.c_void_p, C.c_size_t, C.c_int
_sigs = {
    "ufvc_weight_count": (_sz, [_i, _i]),
    "ufvc_create": (_i, [C.POINTER(ufvc_config), _vp, _sz, C.POINTER(_vp)]),
    "ufvc_destroy": (None, [_vp]),
    "ufvc_layer_shape": (_i, [_i, _i, _i, _vp, _vp, _vp]),
    "ufvc_latent_dims": (_i, [_i, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp]),
    "ufvc_max_bitstream_bytes": (_sz, [_vp, _i, _i]),
    "ufvc_encode_chunk": (_i, [_vp, _vp, _i, _i, _i, _i, _vp, _sz, _vp, _vp]),
    "ufvc_decode_chunk": (_i, [_vp, _vp, _sz, _vp, _i, _i, _i, _vp]),
    "ufvc_decode_chunk_f32": (_i, [_vp, _vp, _sz, _vp, _i, _i, _i, _vp]),
    "ufvc_encode_chunk_host": (_i, [_vp, _vp, _i, _i, _i, _i, _vp, _sz, C.POINTER(_sz), _vp]),
    "ufvc_decode_chunk_host": (_i, [_vp, _vp, _sz, _vp, _i, _i, _i, _vp]),
    "ufvc_sync_status": (_i, [_vp, _vp]),
    "ufvc_encode_stages": (_i, [_vp, _vp, _i, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "ufvc_hyper_synthesis": (_i, [_vp, _vp, _i, _i, _i, _i, _vp, _vp, _vp]),
    "ufvc_quantize": (_i, [_vp, _vp, _vp, _vp, _sz, _i, _vp, _vp, _vp]),
    "ufvc_synthesize": (_i, [_vp, _vp, _i, _i, _vp, _vp]),
    "ufvc_rans_encode": (_i, [_vp, _vp, _vp, _sz, _i, _vp, _sz, _vp, _vp]),
    "ufvc_rans_encode_noalloc": (_i, [_vp, _vp, _vp, _sz, _i, _vp, _sz, _vp, _vp]),
    "ufvc_rans_decode": (_i, [_vp, _vp, _sz, _vp, _sz, _i, _vp, _vp]),
    "ufvc_get_tables": (_i, [_vp, _vp, _vp, _i, _vp]),
    "ufvc_set_profiling": (_i, [_vp, _i]),
    "ufvc_get_profile": (_i, [_vp, _vp, _vp, _vp, _i, C.POINTER(_i)]),
    "ufvc_last_error": (C.c_char_p, [_vp]),
    "ufvc_conv_layer": (_i, [_vp, _i, _vp, _i, _i, _i, _i, _i, _vp, _i, _i, _vp]),
    "ufvc_first_layer": (_i, [_vp, _vp, _i, _i, _i, _vp, _vp]),
    "ufvc_set_table_wait_limit": (_i, [_vp, C.c_longlong]),
    "ufvc_set_conv_pairs": (_i, [_vp, _i]),
    "ufvc_encode_chunks": (_i, [_vp, _i, _vp, _i, _i, _i, _vp, _vp, _sz, _vp, _vp]),
    "ufvc_decode_chunks": (_i, [_vp, _i, _vp, _sz, _vp, _vp, _i, _i, _i, _vp]),
    "ufvc_decode_chunk_dev": (_i, [_vp, _vp, _sz, _vp, _vp, _i, _i, _i, _vp]),
    "ufvc_server_create": (_i, [C.POINTER(ufvc_config), _vp, _sz, _sz, _i, C.POINTER(_vp)]),
    "ufvc_server_destroy": (None, [_vp]),
    "ufvc_server_open_stream": (_i, [_vp, _i, _i, _i, C.POINTER(_i)]),
    "ufvc_server_stream_buffers": (_i, [_vp, _i, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_sz),
                                        C.POINTER(_vp)]),
    "ufvc_server_submit": (_i, [_vp, _i, _i, C.POINTER(C.c_uint64)]),
    "ufvc_server_submit_many": (_i, [_vp, _i, _vp, _vp, _vp]),
    "ufvc_server_poll": (_i, [_vp, C.c_uint64, C.POINTER(ufvc_result)]),
    "ufvc_server_wait": (_i, [_vp, C.c_uint64, C.c_double, C.POINTER(ufvc_result)]),
    "ufvc_server_stats_get": (_i, [_vp, C.POINTER(ufvc_server_stats)]),
    "ufvc_server_last_error": (C.c_char_p, [_vp]),
    "ufvc_calibrate_fp8": (_i, [_vp, _vp, _i, _i, _i, _i, _vp]),
    "ufvc_get_fp8_scales": (_i, [_vp, _vp, _i]),
    "ufvc_mean_weight_count": (_sz, [_i]),
    "ufvc_frame_bytes": (_sz, [_i, _i, _i]),
    "ufvc_set_color_format": (_i, [_vp, _i]),
    "ufvc_temporal_weight_count": (_sz, [_i, _i]),
    "ufvc_set_temporal_context": (_i, [_vp, _vp, _sz]),
    "ufvc_server_set_temporal_context": (_i, [_vp, _vp, _sz]),
    "ufvc_server_calibrate_fp8": (_i, [_vp, _vp, _i, _i, _i, _i]),
    "ufvc_server_set_progressive_means": (_i, [_vp, _vp, _sz]),
    "ufvc_pipe_create": (_i, [_vp, _i, C.POINTER(_vp)]),
    "ufvc_pipe_submit": (_i, [_vp, _vp, _i, _i, _i, _i, _vp, _sz, _vp, C.POINTER(C.c_longlong)]),
    "ufvc_pipe_wait": (_i, [_vp, C.c_longlong, C.POINTER(_sz)]),
    "ufvc_pipe_destroy": (None, [_vp]),
    "ufvc_context_bytes": (_sz, [_vp, _i, _i]),
    "ufvc_encode_chunk_tc": (_i, [_vp, _vp, _i, _i, _i, _i, _vp, _sz, _vp, _vp, _vp, _vp]),
    "ufvc_decode_chunk_tc": (_i, [_vp, _vp, _sz, _vp, _vp, _i, _i, _i, _i, _vp, _vp, _vp]),
    "ufvc_encode_stages_tc": (_i, [_vp, _vp, _i, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "ufvc_set_progressive_means": (_i, [_vp, _vp, _sz]),
    "ufvc_progressive_means": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _i, _i, _vp, _vp, _vp, _vp]),
}
for _name, (_res, _args) in _sigs.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class UfvcError(RuntimeError):
    def __init__(self, code: int, msg: str = ""):
        super().__init__(f"{STATUS_NAMES[code] if 0 <= code < len(STATUS_NAMES) else code}: {msg}")
        self.code = code


def _ptr(t) -> C.c_void_p | None:
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        assert t.is_contiguous()
        return C.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return C.c_void_p(t.ctypes.data)
    raise TypeError(type(t))


def _stream(stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def weight_count(arch: int, chunk_len: int) -> int:
    return int(lib.ufvc_weight_count(arch, chunk_len))


def frame_bytes(color: int, width: int, height: int) -> int:
    return int(lib.ufvc_frame_bytes(color, width, height))


def temporal_weight_count(arch: int, chunk_len: int) -> int:
    return int(lib.ufvc_temporal_weight_count(arch, chunk_len))


def mean_weight_count(arch: int) -> int:
    return int(lib.ufvc_mean_weight_count(arch))


def latent_dims(arch: int, width: int, height: int) -> dict:
    v = [C.c_int() for _ in range(6)]
    rc = lib.ufvc_latent_dims(arch, width, height, *[C.byref(x) for x in v])
    if rc:
        raise UfvcError(rc, "latent_dims")
    return dict(zip(["Hy", "Wy", "Hz", "Wz", "Cy", "Cz"], [x.value for x in v]))


class Codec:
    """One ufvc_ctx.  Methods mirror the C entry points (ufvc_<name>)."""

    def __init__(self, arch: int, chunk_len: int, lanes: int, weights: np.ndarray, precision: str = "fp32",
                 device: int = 0, mean_weights: np.ndarray | None = None, color: int = COLOR_RGB,
                 temporal_weights: np.ndarray | None = None):
        self.arch, self.N, self.K, self.precision = arch, chunk_len, lanes, precision
        self.device = device
        cfg = ufvc_config(arch, chunk_len, lanes, PRECISIONS[precision], device)
        w = np.ascontiguousarray(weights, np.float32)
        h = C.c_void_p()
        rc = lib.ufvc_create(C.byref(cfg), _ptr(w), w.size, C.byref(h))
        if rc:
            raise UfvcError(rc, "ufvc_create")
        self.h = h
        dims = latent_dims(arch, 16, 16)
        self.Cy, self.Cz = dims["Cy"], dims["Cz"]
        if mean_weights is not None:
            mw = np.ascontiguousarray(mean_weights, np.float32)
            self._check(lib.ufvc_set_progressive_means(self.h, _ptr(mw), mw.size), "set_progressive_means")
        self.color = COLOR_RGB
        if color != COLOR_RGB:
            self.set_color_format(color)
        if temporal_weights is not None:
            tw = np.ascontiguousarray(temporal_weights, np.float32)
            self._check(lib.ufvc_set_temporal_context(self.h, _ptr(tw), tw.size), "set_temporal_context")
            self._temporal = True

    # ---- temporal chunk context
    def context_bytes(self, width: int, height: int) -> int:
        return int(lib.ufvc_context_bytes(self.h, width, height))

    def new_context(self, width: int, height: int, device=None) -> torch.Tensor:
        """A context buffer [2 ceil(H/16)][2 ceil(W/16)][Cc] (Cc = 64, 128 for the DC-block model; bf16, or
        float32 in FP32 contexts)."""
        dt = torch.float32 if self.precision == "fp32" else torch.bfloat16
        h8, w8 = 2 * (-(-height // 16)), 2 * (-(-width // 16))
        cc = self.context_bytes(width, height) // (h8 * w8 * (4 if self.precision == "fp32" else 2))
        return torch.empty((h8, w8, cc), dtype=dt, device=device or torch.device(f"cuda:{self.device}"))

    def encode_chunk_tc(self, frames: torch.Tensor, ctx_in, ctx_out, qp: int = 32, bits=None, nbytes=None,
                        stream=None, width=None, height=None):
        N = frames.shape[0]
        W, H = self.frame_dims(frames, width, height)
        if bits is None:
            bits = torch.empty(self.max_bitstream_bytes(W, H), dtype=torch.uint8, device=frames.device)
        if nbytes is None:
            nbytes = torch.zeros(1, dtype=torch.int64, device=frames.device)
        self._check(lib.ufvc_encode_chunk_tc(self.h, _ptr(frames), N, W, H, qp, _ptr(bits), bits.numel(), _ptr(nbytes),
                                             _ptr(ctx_in), _ptr(ctx_out), _stream(stream)), "encode_chunk_tc")
        return bits, nbytes

    def decode_chunk_tc(self, bits: torch.Tensor, nbytes: int, width: int, height: int, ctx_in, ctx_out, out=None,
                        f32: bool = False, stream=None, d_nbytes: torch.Tensor | None = None) -> torch.Tensor:
        """Decode against the stream's context; with d_nbytes (device int64) the size is read on the device
        and nbytes is the readable capacity."""
        if out is None:
            shape = (self.N, height, width, 3) if self.color in (COLOR_RGB, COLOR_RGB_BT709) else \
                (self.N, 3, height, width) if self.color == COLOR_YUV444P else (self.N, frame_bytes(self.color, width, height))
            out = torch.empty(shape, dtype=torch.float32 if f32 else torch.uint8, device=bits.device)
        self._check(lib.ufvc_decode_chunk_tc(self.h, _ptr(bits), int(nbytes), _ptr(d_nbytes), _ptr(out), int(f32),
                                             self.N, width,
                                             height, _ptr(ctx_in), _ptr(ctx_out), _stream(stream)), "decode_chunk_tc")
        return out

    def set_color_format(self, color: int):
        self._check(lib.ufvc_set_color_format(self.h, color), "set_color_format")
        self.color = color

    def frame_dims(self, frames, width=None, height=None) -> tuple[int, int]:
        """(W, H) of a chunk tensor: [N][H][W][3] for RGB formats, [N][3][H][W] for YUV444 planar; YUV420
        chunks ([N][frame bytes]) need width and height."""
        if width is not None:
            return width, height
        if self.color in (COLOR_RGB, COLOR_RGB_BT709):
            return frames.shape[2], frames.shape[1]
        if self.color == COLOR_YUV444P:
            return frames.shape[3], frames.shape[2]
        raise ValueError("YUV420 chunks need width and height")

    def close(self):
        if getattr(self, "h", None):
            lib.ufvc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int, what: str):
        if rc:
            raise UfvcError(rc, f"{what}: {lib.ufvc_last_error(self.h).decode()}")

    # ---- FP8 calibration
    def calibrate_fp8(self, frames: torch.Tensor, qp: int = 32, stream=None, width=None, height=None):
        N = frames.shape[0]
        W, H = self.frame_dims(frames, width, height)
        self._check(lib.ufvc_calibrate_fp8(self.h, _ptr(frames), N, W, H, qp, _stream(stream)), "calibrate_fp8")

    def fp8_scales(self) -> np.ndarray:
        out = np.zeros(15, np.float32)
        self._check(lib.ufvc_get_fp8_scales(self.h, _ptr(out), 15), "get_fp8_scales")
        return out

    # ---- chunk calls
    def max_bitstream_bytes(self, width: int, height: int) -> int:
        return int(lib.ufvc_max_bitstream_bytes(self.h, width, height))

    def encode_chunk(self, frames: torch.Tensor, qp: int = 32, bits: torch.Tensor | None = None,
                     nbytes: torch.Tensor | None = None, stream=None, width=None, height=None):
        """frames: cuda uint8 chunk in the context's colour format -> (bits cuda uint8 [capacity], nbytes
        cuda int64 [1])."""
        N = frames.shape[0]
        W, H = self.frame_dims(frames, width, height)
        if bits is None:
            bits = torch.empty(self.max_bitstream_bytes(W, H), dtype=torch.uint8, device=frames.device)
        if nbytes is None:
            nbytes = torch.zeros(1, dtype=torch.int64, device=frames.device)
        self._check(lib.ufvc_encode_chunk(self.h, _ptr(frames), N, W, H, qp, _ptr(bits), bits.numel(), _ptr(nbytes),
                                          _stream(stream)), "encode_chunk")
        return bits, nbytes

    def decode_chunk(self, bits: torch.Tensor, nbytes: int, width: int, height: int, out: torch.Tensor | None = None,
                     f32: bool = False, stream=None) -> torch.Tensor:
        if out is None:
            shape = (self.N, height, width, 3) if self.color in (COLOR_RGB, COLOR_RGB_BT709) else \
                (self.N, 3, height, width) if self.color == COLOR_YUV444P else (self.N, frame_bytes(self.color, width, height))
            out = torch.empty(shape, dtype=torch.float32 if f32 else torch.uint8, device=bits.device)
        fn = lib.ufvc_decode_chunk_f32 if f32 else lib.ufvc_decode_chunk
        self._check(fn(self.h, _ptr(bits), int(nbytes), _ptr(out), self.N, width, height, _stream(stream)),
                    "decode_chunk")
        return out

    def encode_chunk_host(self, frames: np.ndarray | torch.Tensor, qp: int = 32, stream=None, width=None,
                          height=None) -> bytes:
        N = frames.shape[0]
        W, H = self.frame_dims(frames, width, height)
        cap = self.max_bitstream_bytes(W, H)
        out = torch.empty(cap, dtype=torch.uint8).pin_memory() if torch.cuda.is_available() else np.empty(cap, np.uint8)
        nb = C.c_size_t()
        rc = lib.ufvc_encode_chunk_host(self.h, _ptr(frames), N, W, H, qp, _ptr(out), cap, C.byref(nb),
                                        _stream(stream))
        self._check(rc, "encode_chunk_host")
        return bytes(out[:nb.value].numpy() if isinstance(out, torch.Tensor) else out[:nb.value])

    def decode_chunk_host(self, bits, width: int, height: int, out=None, stream=None):
        if out is None:
            out = np.empty(self.N * frame_bytes(self.color, width, height), np.uint8)
            if self.color in (COLOR_RGB, COLOR_RGB_BT709):
                out = out.reshape(self.N, height, width, 3)
        src = bits if isinstance(bits, (np.ndarray, torch.Tensor)) else np.frombuffer(bits, np.uint8).copy()
        n = src.numel() if isinstance(src, torch.Tensor) else src.size
        self._check(lib.ufvc_decode_chunk_host(self.h, _ptr(src), n, _ptr(out), self.N, width, height,
                                               _stream(stream)), "decode_chunk_host")
        return out

    def sync_status(self, stream=None) -> int:
        return int(lib.ufvc_sync_status(self.h, _stream(stream)))

    # ---- stages
    def encode_stages(self, frames: torch.Tensor, qp: int = 32, stream=None, width=None, height=None,
                      ctx_in=None) -> dict:
        W, H = self.frame_dims(frames, width, height)
        d = latent_dims(self.arch, W, H)
        dev = frames.device
        yshape = (d["Hy"], d["Wy"], d["Cy"])
        out = dict(y=torch.empty(yshape, device=dev), zhat=torch.empty((d["Hz"], d["Wz"], d["Cz"]), dtype=torch.int16,
                                                                        device=dev),
                   iz=torch.empty(d["Cz"], dtype=torch.uint8, device=dev), mu=torch.empty(yshape, device=dev),
                   logsig=torch.empty(yshape, device=dev), rhat=torch.empty(yshape, dtype=torch.int16, device=dev),
                   idx=torch.empty(yshape, dtype=torch.uint8, device=dev))
        keys = ("y", "zhat", "iz", "mu", "logsig", "rhat", "idx")
        if ctx_in is not None or getattr(self, "_temporal", False):
            self._check(lib.ufvc_encode_stages_tc(self.h, _ptr(frames), W, H, qp, _ptr(ctx_in),
                                                  *[_ptr(out[k]) for k in keys], _stream(stream)), "encode_stages_tc")
        else:
            self._check(lib.ufvc_encode_stages(self.h, _ptr(frames), W, H, qp, *[_ptr(out[k]) for k in keys],
                                               _stream(stream)), "encode_stages")
        return out

    def hyper_synthesis(self, zhat: torch.Tensor, Hy: int, Wy: int, stream=None):
        Hz, Wz, _ = zhat.shape
        mu = torch.empty((Hy, Wy, self.Cy), device=zhat.device)
        ls = torch.empty((Hy, Wy, self.Cy), device=zhat.device)
        self._check(lib.ufvc_hyper_synthesis(self.h, _ptr(zhat), Hz, Wz, Hy, Wy, _ptr(mu), _ptr(ls), _stream(stream)),
                    "hyper_synthesis")
        return mu, ls

    def progressive_means(self, mu0: torch.Tensor, s: torch.Tensor, qp: int = 32, y: torch.Tensor | None = None,
                          rhat: torch.Tensor | None = None, stream=None):
        """The four-partition mean steps: encoder form (y given) or decoder form (rhat given) ->
        (rhat, mu the mean each element is coded with, yhat = rhat q + mu)."""
        Hy, Wy, _ = mu0.shape
        r = torch.empty(mu0.shape, dtype=torch.int16, device=mu0.device)
        mu = torch.empty_like(mu0)
        yhat = torch.empty_like(mu0)
        self._check(lib.ufvc_progressive_means(self.h, _ptr(y), _ptr(rhat), _ptr(mu0), _ptr(s), Hy, Wy, qp, _ptr(r),
                                               _ptr(mu), _ptr(yhat), _stream(stream)), "progressive_means")
        return r, mu, yhat

    def quantize(self, y, mu, logsig, qp: int = 32, stream=None):
        rhat = torch.empty(y.shape, dtype=torch.int16, device=y.device)
        idx = torch.empty(y.shape, dtype=torch.uint8, device=y.device)
        self._check(lib.ufvc_quantize(self.h, _ptr(y), _ptr(mu), _ptr(logsig), y.numel(), qp, _ptr(rhat), _ptr(idx),
                                      _stream(stream)), "quantize")
        return rhat, idx

    def synthesize(self, yhat: torch.Tensor, width: int, height: int, stream=None) -> torch.Tensor:
        out = torch.empty((self.N, height, width, 3), device=yhat.device)
        self._check(lib.ufvc_synthesize(self.h, _ptr(yhat), width, height, _ptr(out), _stream(stream)), "synthesize")
        return out

    def rans_encode(self, sym: torch.Tensor, idx: torch.Tensor, lanes: int, capacity: int | None = None,
                    stream=None):
        n = sym.numel()
        if capacity is None:
            capacity = 4 * lanes + 2 * (n + 2 * lanes) + 4
        out = torch.empty(capacity, dtype=torch.uint8, device=sym.device)
        nb = torch.zeros(1, dtype=torch.int64, device=sym.device)
        self._check(lib.ufvc_rans_encode(self.h, _ptr(sym), _ptr(idx), n, lanes, _ptr(out), capacity, _ptr(nb),
                                         _stream(stream)), "rans_encode")
        return out, nb

    def rans_decode(self, data: torch.Tensor, nbytes: int, idx: torch.Tensor, n: int, lanes: int, stream=None):
        sym = torch.empty(max(n, 1), dtype=torch.int16, device=data.device)
        self._check(lib.ufvc_rans_decode(self.h, _ptr(data), int(nbytes), _ptr(idx), n, lanes, _ptr(sym),
                                         _stream(stream)), "rans_decode")
        return sym[:n]

    def conv_layer(self, layer: int, x: torch.Tensor, stride: int, act: int, mode: int, out: torch.Tensor,
                   stream=None) -> torch.Tensor:
        H, W, _ = x.shape
        oh, ow = out.shape[0], out.shape[1]
        self._check(lib.ufvc_conv_layer(self.h, layer, _ptr(x), H, W, stride, act, mode, _ptr(out), oh, ow,
                                        _stream(stream)), "conv_layer")
        return out

    def first_layer(self, frames: torch.Tensor, width: int, height: int, kernel: int = 0, stream=None) -> torch.Tensor:
        """A1 from the frame bytes: bf16 [ceil16(H)/2][ceil16(W)/2][64] (kernel 0 auto, 1 register, 2 TMA)."""
        out = torch.empty(((height + 15) // 16 * 8, (width + 15) // 16 * 8, 64), dtype=torch.bfloat16,
                          device=frames.device)
        self._check(lib.ufvc_first_layer(self.h, _ptr(frames), width, height, kernel, _ptr(out), _stream(stream)),
                    "first_layer")
        return out

    def encode_chunks(self, frames: list, qps: list, bits: list, nbytes: list, width: int | None = None,
                      height: int | None = None, stream=None):
        """Batched encode: frames[b] (device tensors of one size) into bits[b], sizes into nbytes[b]."""
        B = len(frames)
        H = height if height is not None else frames[0].shape[1]
        W = width if width is not None else frames[0].shape[2]
        P = C.c_void_p * B
        self._check(lib.ufvc_encode_chunks(self.h, B, P(*[_ptr(f) for f in frames]), self.N, W, H,
                                           (C.c_int * B)(*qps), P(*[_ptr(b) for b in bits]), bits[0].numel(),
                                           P(*[_ptr(n) for n in nbytes]), _stream(stream)), "encode_chunks")

    def decode_chunks(self, bits: list, nbytes: list, width: int, height: int, outs: list, stream=None):
        """Batched decode: bits[b] (sizes on the device in nbytes[b]) into uint8 frames outs[b]."""
        B = len(bits)
        P = C.c_void_p * B
        self._check(lib.ufvc_decode_chunks(self.h, B, P(*[_ptr(b) for b in bits]), bits[0].numel(),
                                           P(*[_ptr(n) for n in nbytes]), P(*[_ptr(o) for o in outs]), self.N, width,
                                           height, _stream(stream)), "decode_chunks")

    def set_conv_pairs(self, enable: bool):
        """Decoder pixel-shuffle layers on SM pairs (True, the default) or one SM per tile."""
        self._check(lib.ufvc_set_conv_pairs(self.h, int(bool(enable))), "set_conv_pairs")

    def set_table_wait_limit(self, cycles: int):
        self._check(lib.ufvc_set_table_wait_limit(self.h, int(cycles)), "set_table_wait_limit")

    def get_tables(self, qp: int = 32):
        freq = np.empty((64, 511), np.uint32)
        cum = np.empty((64, 512), np.uint32)
        thr = np.empty(63, np.float32)
        self._check(lib.ufvc_get_tables(self.h, _ptr(freq), _ptr(cum), qp, _ptr(thr)), "get_tables")
        return freq, cum, thr

    def set_profiling(self, enable: bool):
        self._check(lib.ufvc_set_profiling(self.h, int(enable)), "set_profiling")

    def get_profile(self, max_entries: int = 64) -> list[tuple[str, float, int]]:
        names = C.create_string_buffer(32 * max_entries)
        ms = np.zeros(max_entries, np.float32)
        launches = np.zeros(max_entries, np.int32)
        cnt = C.c_int()
        self._check(lib.ufvc_get_profile(self.h, names, _ptr(ms), _ptr(launches), max_entries, C.byref(cnt)),
                    "get_profile")
        raw = names.raw
        return [(raw[32 * i:32 * i + 32].split(b"\0")[0].decode(), float(ms[i]), int(launches[i]))
                for i in range(cnt.value)]


class Pipe:
    """Pipelined host-buffer round trips (ufvc_pipe_*): `depth` slots sharing codec's weights; submit()
    enqueues frames -> encode -> bit-stream to host -> back -> decode -> frames to host and returns a
    ticket; wait(ticket) returns the stream size.  Host buffers (page-locked for asynchronous copies) must
    stay alive until their ticket has been waited for."""

    def __init__(self, codec: "Codec", depth: int = 2):
        h = C.c_void_p()
        rc = lib.ufvc_pipe_create(codec.h, depth, C.byref(h))
        if rc:
            raise UfvcError(rc, "ufvc_pipe_create")
        self.h, self.codec, self.depth = h, codec, depth

    def submit(self, h_frames, width: int, height: int, h_bits, h_out=None, qp: int = 32) -> int:
        t = C.c_longlong()
        n = h_frames.shape[0]
        cap = h_bits.numel() if isinstance(h_bits, torch.Tensor) else h_bits.size
        rc = lib.ufvc_pipe_submit(self.h, _ptr(h_frames), n, width, height, qp, _ptr(h_bits), cap, _ptr(h_out),
                                  C.byref(t))
        if rc:
            raise UfvcError(rc, "ufvc_pipe_submit")
        return t.value

    def wait(self, ticket: int) -> int:
        nb = C.c_size_t()
        rc = lib.ufvc_pipe_wait(self.h, ticket, C.byref(nb))
        if rc:
            raise UfvcError(rc, "ufvc_pipe_wait")
        return nb.value

    def close(self):
        if getattr(self, "h", None):
            lib.ufvc_pipe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching chunk server (include/ufvc.h, "Serving").  Streams own device-resident input,
    bit-stream and output buffers, exposed here as torch tensors that alias the library's memory."""

    def __init__(self, arch: int, chunk_len: int, lanes: int, weights: np.ndarray, precision: str = "bf16",
                 hbm_cap_bytes: int = 0, max_slots: int = 8, device: int = 0,
                 temporal_weights: np.ndarray | None = None, mean_weights: np.ndarray | None = None):
        self.N = chunk_len
        self.device = device
        w = np.ascontiguousarray(weights, dtype=np.float32)
        cfg = ufvc_config(arch, chunk_len, lanes, PRECISIONS[precision], device)
        h = C.c_void_p()
        rc = lib.ufvc_server_create(C.byref(cfg), _ptr(w), w.size, hbm_cap_bytes, max_slots, C.byref(h))
        if rc:
            raise UfvcError(rc, "server_create")
        self.h = h
        self.streams: dict[int, dict] = {}
        if temporal_weights is not None:
            tw = np.ascontiguousarray(temporal_weights, np.float32)
            self._check(lib.ufvc_server_set_temporal_context(self.h, _ptr(tw), tw.size), "server_set_temporal_context")
        if mean_weights is not None:
            mw = np.ascontiguousarray(mean_weights, np.float32)
            self._check(lib.ufvc_server_set_progressive_means(self.h, _ptr(mw), mw.size), "server_set_progressive_means")

    def calibrate_fp8(self, frames: torch.Tensor, qp: int = 32, width: int | None = None, height: int | None = None):
        """FP8 servers: activation scales from the FP32 path on this chunk (before the first stream)."""
        H = height if height is not None else frames.shape[1]
        W = width if width is not None else frames.shape[2]
        self._check(lib.ufvc_server_calibrate_fp8(self.h, _ptr(frames), self.N, W, H, qp), "server_calibrate_fp8")

    def close(self):
        if self.h:
            lib.ufvc_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int, what: str):
        if rc:
            raise UfvcError(rc, f"{what}: {lib.ufvc_server_last_error(self.h).decode()}")

    def open_stream(self, width: int, height: int, qp: int = 32) -> int:
        sid = C.c_int()
        self._check(lib.ufvc_server_open_stream(self.h, width, height, qp, C.byref(sid)), "open_stream")
        fin, bits, nb, fout = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p()
        cap = C.c_size_t()
        self._check(lib.ufvc_server_stream_buffers(self.h, sid.value, C.byref(fin), C.byref(bits), C.byref(nb),
                                                   C.byref(cap), C.byref(fout)), "stream_buffers")
        shape = (self.N, height, width, 3)
        self.streams[sid.value] = dict(
            frames_in=_alias(fin.value, shape, torch.uint8, self.device),
            frames_out=_alias(fout.value, shape, torch.uint8, self.device),
            bits=_alias(bits.value, (cap.value,), torch.uint8, self.device),
            nbytes=_alias(nb.value, (1,), torch.int64, self.device), width=width, height=height, qp=qp)
        return sid.value

    def submit(self, stream_id: int, op: int) -> int:
        t = C.c_uint64()
        self._check(lib.ufvc_server_submit(self.h, stream_id, op, C.byref(t)), "submit")
        return t.value

    def submit_many(self, requests: list[tuple[int, int]]) -> list[int]:
        """Queue [(stream_id, op), ...] at once (all or none); returns their tickets."""
        n = len(requests)
        sids = (C.c_int * max(n, 1))(*[r[0] for r in requests])
        ops = (C.c_int * max(n, 1))(*[r[1] for r in requests])
        t = (C.c_uint64 * max(n, 1))()
        self._check(lib.ufvc_server_submit_many(self.h, n, sids, ops, t), "submit_many")
        return [int(t[i]) for i in range(n)]

    def poll(self, ticket: int) -> dict:
        r = ufvc_result()
        lib.ufvc_server_poll(self.h, ticket, C.byref(r))
        return {f: getattr(r, f) for f, _ in ufvc_result._fields_}

    def wait(self, ticket: int, timeout_ms: float = -1.0) -> dict:
        r = ufvc_result()
        lib.ufvc_server_wait(self.h, ticket, timeout_ms, C.byref(r))
        return {f: getattr(r, f) for f, _ in ufvc_result._fields_}

    def stats(self) -> dict:
        s = ufvc_server_stats()
        self._check(lib.ufvc_server_stats_get(self.h, C.byref(s)), "stats")
        return {f: getattr(s, f) for f, _ in ufvc_server_stats._fields_}


def _alias(ptr: int, shape: tuple, dtype: torch.dtype, device: int) -> torch.Tensor:
    """A torch tensor viewing library-owned device memory (no copy, no ownership: valid while the
    server lives)."""
    n = 1
    for d in shape:
        n *= d
    nbytes = n * torch.empty((), dtype=dtype).element_size()

    class _Arr:
        __cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False), "version": 3,
                                    "strides": None}
    return torch.as_tensor(_Arr(), device=f"cuda:{device}").view(dtype).view(shape)
