"""Benchmark: 1080p 8-frame chunk encode + decode through libufvc (one step = one chunk encoded and
decoded: pack, analysis + cross-frame interaction, hyper-analysis, z^, hyper-synthesis, quantise +
scale index, both rANS sections, bit-stream layout; header/lane parse, z^ decode, hyper-synthesis,
scale index, whole-latent decode + dequantise, 8 frame-specific decoders, uint8 frames).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp32] [--impl ours|reference]
                    [--width W --height H]

Prints ONE JSON line (rank 0).  The headline path is BF16 (tensor cores); the FP32 path is timed beside
it under the same methodology and reported with the PSNR and bitrate deltas.  Under torchrun every rank
codes its own chunks (weak scaling, no data-path collective); the timed region is bracketed by a
barrier and a synchronize, max over ranks.  --impl reference times the FP64 CPU oracle on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

W, H, N, K, QP = 1920, 1080, 8, 4096, 32
WORKLOAD = "1080p 8-frame chunk (1920x1080 padded to 1920x1088), arch 1 (analysis 64/128/192, Cy=256, Cz=128, " \
           "8 frame-specific decoders 128->64), K=4096 rANS lanes, qp=32"
METRIC = "1080p 8-frame-chunk enc/dec frames/s, BF16 vs FP32 (dPSNR<=0.05dB); p99 latency"


def peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f) | {"source": "measured"}
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2032.0,
                "source": "fallback"}


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, device: int):
        self.p = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{device}.csv")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(device), "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline() -> dict:
    """The FP64 oracle, as it stands, on a bounded sample: the same 8-frame chunk cropped to a window of
    the 1080p frames, encoded and decoded; frames/s scaled to the full 1080p area (the oracle's cost is
    proportional to the pixel count)."""
    import oracle
    import synthetic
    frames = synthetic.chunk_frames("1080p", seed=0)
    blob = synthetic.draw_weights(1, N, seed=0)
    oracle.build()
    h, w = 256, 384
    crop = np.ascontiguousarray(frames[:, :h, :w])
    t0 = time.perf_counter()
    bits = oracle.encode_chunk(1, crop, QP, K, blob)
    t1 = time.perf_counter()
    oracle.decode_chunk(1, N, bits, h, w, blob)
    t2 = time.perf_counter()
    scale = (1088 * 1920) / (h * w)
    t_chunk = (t2 - t0) * scale
    return {"value": N / t_chunk, "unit": "frames/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"one 8-frame chunk cropped to {w}x{h} (1/{scale:.1f} of the padded 1080p area), encode "
                      f"{t1 - t0:.2f}s + decode {t2 - t1:.2f}s, scaled by area to a full 1080p chunk",
            "enc_fps": N / ((t1 - t0) * scale), "dec_fps": N / ((t2 - t1) * scale)}


def run_reference(args) -> None:
    rank, world, _ = env_rank()
    if rank != 0:
        return
    vals = []
    for _ in range(args.warmup):
        cpu_baseline()
    cb = None
    for _ in range(args.steps):
        cb = cpu_baseline()
        vals.append(cb["value"])
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * N / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "fp64 oracle (CPU)"},
            "cpu_baseline": {k: cb[k] for k in ("kind", "cores", "sample")} | {"value": v, "unit": "frames/s"},
            "e2e": {"value": v, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def conv_flops(Hy: int, Wy: int) -> dict:
    """Algorithmic FLOPs (2 x MACs) of each decoder conv stage for an N-frame chunk with latent Hy x Wy."""
    p1, p2, p3 = 4 * Hy * Wy, 16 * Hy * Wy, 64 * Hy * Wy   # pixels at 1/8, 1/4, 1/2 resolution
    return {"dec.D0": N * Hy * Wy * 512 * 256 * 9 * 2, "dec.R1": 2 * N * p1 * 128 * 128 * 9 * 2,
            "dec.U1": N * p1 * 256 * 128 * 9 * 2, "dec.R2": 2 * N * p2 * 64 * 64 * 9 * 2,
            "dec.U2": N * p2 * 256 * 64 * 9 * 2, "dec.U3": N * p3 * 12 * 64 * 9 * 2}


def time_codec(codec, fr, frames_np, W_, H_, steps, warmup, profile, flush, dist=None, world=1):
    """Encode + decode one chunk per step; per-step CUDA events on the launching stream, L2 flushed
    between steps (outside the events).  Returns timings, stage profile, stream size and PSNR."""
    import torch
    dev = fr.device
    cap = codec.max_bitstream_bytes(W_, H_)
    bits = torch.empty(cap, dtype=torch.uint8, device=dev)
    nbytes = torch.zeros(1, dtype=torch.int64, device=dev)
    out = torch.empty((N, H_, W_, 3), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    nb = 0
    for _ in range(warmup):  # also establishes the stream size, which the decoder call takes from the host
        codec.encode_chunk(fr, QP, bits, nbytes)
        nb = int(nbytes.item())
        codec.decode_chunk(bits, nb, W_, H_, out)
    assert codec.sync_status() == 0
    rec = out.float().cpu().numpy() / 255.0
    psnr = float(10 * np.log10(1.0 / np.mean((rec - frames_np / 255.0) ** 2)))
    codec.set_profiling(profile)
    prof_acc: dict[str, list] = {}
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    if dist is not None and world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(steps):
        flush.fill_(i & 0xFF)
        evs[i][0].record(stream)
        codec.encode_chunk(fr, QP, bits, nbytes)
        evs[i][1].record(stream)
        codec.decode_chunk(bits, nb, W_, H_, out)
        evs[i][2].record(stream)
        if profile:
            for name, ms, nl in codec.get_profile():
                prof_acc.setdefault(name, []).append((ms, nl))
    torch.cuda.synchronize()
    if dist is not None and world > 1:
        dist.barrier()
    codec.set_profiling(False)
    assert codec.sync_status() == 0
    t_enc = [evs[i][0].elapsed_time(evs[i][1]) for i in range(steps)]
    t_dec = [evs[i][1].elapsed_time(evs[i][2]) for i in range(steps)]
    return dict(t_enc=t_enc, t_dec=t_dec, prof=prof_acc, nbytes=nb, psnr=psnr, cap=cap)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--precision", default=os.environ.get("UFVC_BENCH_PRECISION", "bf16"))
    ap.add_argument("--width", type=int, default=W)
    ap.add_argument("--height", type=int, default=H)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32-path", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    args.warmup = max(args.warmup, 3)

    import torch
    import torch.distributed as dist

    import synthetic
    from paper_2606_04410_b300 import ufvc as U

    rank, world, local = env_rank()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    W_, H_ = args.width, args.height
    if (W_, H_) == (W, H):
        frames_np = synthetic.chunk_frames("1080p", seed=rank)
    else:
        frames_np = synthetic.moving_texture(rank, N, H_, W_, max_step=16, refresh=0.10)
    blob = synthetic.draw_weights(1, N, seed=0)
    fr = torch.from_numpy(frames_np).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 126 MB L2

    codec = U.Codec(1, N, K, blob, args.precision, device=local)
    sampler = ClockSampler(local)
    r = time_codec(codec, fr, frames_np, W_, H_, args.steps, args.warmup, True, flush, dist, world)
    clocks = sampler.stop()
    t_step = [a + b for a, b in zip(r["t_enc"], r["t_dec"])]
    total_ms = sum(t_step)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = N * args.steps * world / (total_ms / 1000.0)

    # ---- dominant kernel roofline (per-stage events recorded inside the same timed steps)
    prof_acc = r["prof"]
    stage_ms = {k: statistics.mean(m for m, _ in v) for k, v in prof_acc.items()}
    stage_total_ms = {k: sum(m for m, _ in v) / args.steps for k, v in prof_acc.items()}
    launches_per_step = sum(sum(n for _, n in v) for v in prof_acc.values()) / args.steps
    hy, wy = -(-H_ // 16), -(-W_ // 16)
    flops = conv_flops(hy, wy)
    conv_stages = {k: v for k, v in stage_ms.items() if k in flops}
    top = max(conv_stages, key=conv_stages.get)
    pk = peaks()
    if args.precision == "fp32":
        peak = 148 * 128 * 2 * pk.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
        bound, peak_src = "alu", f"derived: 148 SMs x 128 FP32 FMA/clk x 2 x {pk.get('sm_max_mhz', 2032.0):.0f} MHz"
    else:
        peak = pk["bf16_tflops_sustained"] if args.precision == "bf16" else 2 * pk["bf16_tflops_sustained"]
        bound = "tensor"
        peak_src = f"{pk['source']} bf16 sustained" + (" x2 (fp8 nominal ratio)" if args.precision == "fp8" else "")
    achieved = flops[top] / (conv_stages[top] / 1000.0) / 1e12
    dec_conv_ms = sum(v for k, v in stage_total_ms.items() if k in flops)
    roofline = {"bound": bound, "kernel": f"conv_tc {top}" if bound == "tensor" else f"conv_simt {top}",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": peak_src,
                "decoder_convs": {"tflops": sum(flops.values()) / (dec_conv_ms / 1000.0) / 1e12,
                                  "frac": sum(flops.values()) / (dec_conv_ms / 1000.0) / 1e12 / peak},
                "stage_ms_per_step": {k: round(v, 4) for k, v in
                                      sorted(stage_total_ms.items(), key=lambda kv: -kv[1])}}

    # ---- the FP32 path under the same methodology (the baseline the BF16 path must beat)
    fp32 = None
    if args.precision != "fp32" and not args.no_fp32_path:
        c32 = U.Codec(1, N, K, blob, "fp32", device=local)
        s32 = max(3, args.steps // 4)
        r32 = time_codec(c32, fr, frames_np, W_, H_, s32, 3, False, flush)
        v32 = N * s32 / (sum(a + b for a, b in zip(r32["t_enc"], r32["t_dec"])) / 1000.0)
        fp32 = {"value": v32, "enc_fps": N / (statistics.mean(r32["t_enc"]) / 1000.0),
                "dec_fps": N / (statistics.mean(r32["t_dec"]) / 1000.0), "psnr_db": r32["psnr"],
                "bytes_per_chunk": r32["nbytes"], "steps": s32}
        c32.close()

    # ---- end-to-end through the host-buffer C calls (pinned host memory, copies inside the region)
    cap = r["cap"]
    h_frames = torch.from_numpy(frames_np).pin_memory()
    h_bits = torch.empty(cap, dtype=torch.uint8).pin_memory()
    h_out = torch.empty((N, H_, W_, 3), dtype=torch.uint8).pin_memory()
    import ctypes as C
    nbh = C.c_size_t()
    e2e_ms = []
    for i in range(max(3, args.steps // 2) + 2):
        t0 = time.perf_counter()
        rc = U.lib.ufvc_encode_chunk_host(codec.h, U._ptr(h_frames), N, W_, H_, QP, U._ptr(h_bits), cap,
                                          C.byref(nbh), U._stream(None))
        assert rc == 0
        rc = U.lib.ufvc_decode_chunk_host(codec.h, U._ptr(h_bits), nbh.value, U._ptr(h_out), N, W_, H_,
                                          U._stream(None))
        assert rc == 0
        if i >= 2:
            e2e_ms.append((time.perf_counter() - t0) * 1000.0)
    e2e = {"value": N * world / (statistics.mean(e2e_ms) / 1000.0), "unit": "frames/s",
           "h2d_bytes_per_step": int(h_frames.numel() + nbh.value),
           "d2h_bytes_per_step": int(nbh.value + h_out.numel() + 8)}

    if rank == 0:
        workload = WORKLOAD if (W_, H_) == (W, H) else \
            WORKLOAD.replace("1080p 8-frame chunk (1920x1080 padded to 1920x1088)", f"{W_}x{H_} 8-frame chunk")
        line = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp32": "f32", "bf16": "bf16", "fp8": "e4m3"}[args.precision], "data": "synthetic",
                "config": {"workload": workload, "precision": args.precision, "chunk_frames": N, "width": W_,
                           "height": H_, "lanes": K, "qp": QP, "l2": "flushed between steps (256 MB write)",
                           "parallelism": f"{world} independent streams (one chunk per rank per step)"},
                "enc_fps": N / (statistics.mean(r["t_enc"]) / 1000.0),
                "dec_fps": N / (statistics.mean(r["t_dec"]) / 1000.0),
                "latency_ms": {"p50": float(np.percentile(t_step, 50)), "p99": float(np.percentile(t_step, 99)),
                               "enc_p99": float(np.percentile(r["t_enc"], 99)),
                               "dec_p99": float(np.percentile(r["t_dec"], 99))},
                "psnr_db": r["psnr"], "bytes_per_chunk": r["nbytes"], "bpp": 8 * r["nbytes"] / (N * W_ * H_),
                "roofline": roofline, "e2e": e2e, "gpu_launches": int(round(launches_per_step * args.steps)),
                "clocks": clocks}
        if fp32 is not None:
            line["fp32_path"] = fp32
            line["speedup_vs_fp32"] = value / fp32["value"]
            line["dpsnr_db_vs_fp32"] = r["psnr"] - fp32["psnr_db"]
            line["dbitrate_vs_fp32"] = (r["nbytes"] - fp32["bytes_per_chunk"]) / fp32["bytes_per_chunk"]
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
