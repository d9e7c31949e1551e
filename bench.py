"""Benchmark: 1080p 8-frame chunk encode + decode through libufvc (one step = one chunk encoded and
decoded: frame bytes -> first analysis layer (read by its own kernel in BF16), analysis + cross-frame
interaction, hyper-analysis, z^, hyper-synthesis, quantise +
scale index, both rANS sections, bit-stream layout; header/lane parse, z^ decode, hyper-synthesis,
scale index, whole-latent decode + dequantise, 8 frame-specific decoders, uint8 frames).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp32] [--impl ours|reference]
                    [--width W --height H] [--no-cpu-baseline] [--no-fp32-path] [--no-entropy-sweep]
                    [--no-serving] [--no-fp8] [--no-pm] [--no-color] [--no-temporal] [--no-dc]
                    [--serving-windows R:S,...] [--serving-windows-fp32 R:S,...]

Prints ONE JSON line (rank 0).  The headline path is BF16 (tensor cores); the FP32 path is timed beside
it under the same methodology and reported with the PSNR and bitrate deltas.  Extra keys: the decoder
conv stages against their own bounds (tensor or HBM), the entropy-coding stress at 4K (8.29 M symbols,
lane counts 1024..65536), and the serving mix (64 streams of four sizes, Poisson arrivals, through the
continuous-batching server) for BF16 and FP32.  Under torchrun every rank codes its own chunks and
serves its share of the streams (weak scaling, no data-path collective); the timed region is bracketed
by a barrier and a synchronize, max over ranks.  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
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
        self.path = os.path.join(tempfile.gettempdir(), f"ufvc_bench_clocks_{os.getpid()}_{device}.csv")
        try:
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


CROP_H, CROP_W = 256, 384
CROP_WORKLOAD = f"{CROP_W}x{CROP_H} crop (top-left) of the 1080p 8-frame chunk, arch 1, K=4096 rANS lanes, qp=32"


def oracle_crop_step() -> tuple[float, float]:
    """One encode + decode of the crop by the FP64 oracle; returns (encode s, decode s)."""
    import oracle
    import synthetic
    frames = synthetic.chunk_frames("1080p", seed=0)
    blob = synthetic.draw_weights(1, N, seed=0)
    crop = np.ascontiguousarray(frames[:, :CROP_H, :CROP_W])
    t0 = time.perf_counter()
    bits = oracle.encode_chunk(1, crop, QP, K, blob)
    t1 = time.perf_counter()
    oracle.decode_chunk(1, N, bits, CROP_H, CROP_W, blob)
    return t1 - t0, time.perf_counter() - t1


def cpu_baseline() -> dict:
    """The FP64 oracle, as it stands, on the host cores: one whole 1080p 8-frame chunk encoded and
    decoded with every OpenMP thread (measured, not scaled), plus the crop on one thread (scaled by area
    to the full chunk, labelled as such) in a child process so the thread count can be set."""
    import oracle
    import synthetic
    oracle.build()
    frames = synthetic.chunk_frames("1080p", seed=0)
    blob = synthetic.draw_weights(1, N, seed=0)
    t0 = time.perf_counter()
    bits = oracle.encode_chunk(1, frames, QP, K, blob)
    t1 = time.perf_counter()
    oracle.decode_chunk(1, N, bits, H, W, blob)
    t2 = time.perf_counter()
    out = {"value": N / (t2 - t0), "unit": "frames/s", "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"one whole 1080p 8-frame chunk (1920x1080), encode {t1 - t0:.1f} s + decode {t2 - t1:.1f} s, "
                     f"{oracle.num_threads()} OpenMP threads, measured",
           "enc_fps": N / (t1 - t0), "dec_fps": N / (t2 - t1)}
    env = dict(os.environ, OMP_NUM_THREADS="1")
    code = "import bench, json; print(json.dumps(bench.oracle_crop_step()))"
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=600)
        te, td = json.loads(r.stdout.strip().splitlines()[-1])
        area = (1088 * 1920) / (CROP_H * CROP_W)
        out["single_core"] = {"value": N / ((te + td) * area), "unit": "frames/s", "cores": 1,
                              "sample": f"{CROP_WORKLOAD}: encode {te:.2f} s + decode {td:.2f} s on one thread, "
                                        f"scaled by the area ratio {area:.1f} to a full chunk"}
    except (subprocess.SubprocessError, ValueError, IndexError, OSError) as e:
        out["single_core"] = {"unavailable": str(e)[:200]}
    return out


def run_reference(args) -> None:
    """The reference arm: the FP64 oracle on the host cores, each step one encode + decode of the crop
    (about 2 s on 16 threads, so K + W steps stay within minutes).  ms_per_step is the measured time of
    a crop step; value converts it to full-chunk frames/s by the area ratio (the oracle's cost is
    proportional to the pixel count: direct convolutions per output pixel, one rANS step per symbol)."""
    rank, world, _ = env_rank()
    if rank != 0:
        return
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        oracle_crop_step()
    steps = [sum(oracle_crop_step()) for _ in range(args.steps)]
    t = statistics.mean(steps)
    area = (1088 * 1920) / (CROP_H * CROP_W)
    v = N / (t * area)
    sample = f"{CROP_WORKLOAD}, encode + decode per step, {oracle.num_threads()} OpenMP threads"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": sample, "precision": "fp64 oracle (CPU)",
                       "value_basis": f"full 1080p chunk frames/s = 8 / (crop step time x area ratio {area:.1f})"},
            "cpu_baseline": {"kind": "oracle", "cores": oracle.num_threads(), "sample": sample, "value": v,
                             "unit": "frames/s"},
            "e2e": {"value": v, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def dc_flops(Hy: int, Wy: int) -> dict:
    """Tensor-core FLOPs (2 x MACs) of one encode and one decode of the DC-block model (arch 2, N frames) at
    latent size Hy x Wy, from its layer table: the encoder runs patch embedding, encoder blocks, ED, H1, H2,
    PC and, to track the context, the chunk decoder and the context generation; the decoder runs PC, the
    chunk decoder, the frame decoders and the context generation.  (S1..S3 are the FP32 path.)"""
    from synthetic.weights import dc_layer_table
    P8, P16 = 4 * Hy * Wy, Hy * Wy
    Hz, Wz = -(-Hy // 4), -(-Wy // 4)
    pos = {"ED": P16, "PC": P16, "DU": P16, "H1": (-(-Hy // 2)) * (-(-Wy // 2)), "H2": Hz * Wz}
    enc = dec = 0
    for name, co, k, ci in dc_layer_table(N):
        if name in ("S1", "S2", "S3"):
            continue
        f = 2 * pos.get(name, P8) * co * k * k * ci
        head = name.split(".")[0]
        if name in ("PE", "EC", "ED", "H1", "H2") or (head.startswith("E") and head[1:].isdigit()):
            enc += f
        elif name.startswith(("FP", "FO")) or (head.startswith("F") and head[1:].isdigit()):
            dec += f
        elif name == "FC" or name in ("DU", "PC", "GO") or head[0] in "DG":
            enc += f
            dec += f
    return {"enc": enc, "dec": dec}


def conv_flops(Hy: int, Wy: int) -> dict:
    """Algorithmic FLOPs (2 x MACs) of each decoder conv stage for an N-frame chunk with latent Hy x Wy."""
    p1, p2, p3 = 4 * Hy * Wy, 16 * Hy * Wy, 64 * Hy * Wy   # pixels at 1/8, 1/4, 1/2 resolution
    return {"dec.D0": N * Hy * Wy * 512 * 256 * 9 * 2, "dec.R1": 2 * N * p1 * 128 * 128 * 9 * 2,
            "dec.U1": N * p1 * 256 * 128 * 9 * 2, "dec.R2": 2 * N * p2 * 64 * 64 * 9 * 2,
            "dec.U2": N * p2 * 256 * 64 * 9 * 2, "dec.U3": N * p3 * 12 * 64 * 9 * 2}


def conv_bytes(Hy: int, Wy: int, H_: int, W_: int) -> dict:
    """Algorithmic HBM bytes of each decoder conv stage (bf16 activations read once and written once,
    residuals read once, the final frames as uint8; weights are negligible)."""
    a0 = Hy * Wy * 256 * 2                      # y^ (bf16), shared by the N decoders
    a1, a2, a3 = N * 4 * Hy * Wy * 128 * 2, N * 16 * Hy * Wy * 64 * 2, N * 64 * Hy * Wy * 64 * 2
    return {"dec.D0": a0 + a1, "dec.R1": 2 * a1 + 3 * a1, "dec.U1": a1 + a2, "dec.R2": 2 * a2 + 3 * a2,
            "dec.U2": a2 + a3, "dec.U3": a3 + N * H_ * W_ * 3}


def compute_peaks(pk: dict, precision: str) -> dict:
    """Peaks each stage is measured against: tensor (burst bf16, x2 for E4M3 by the nominal ratio), TF32
    tensor (burst bf16 x 0.5, the nominal ratio), FP32 ALU (148 SMs x 128 FMA/clk x 2 at the maximum SM
    clock, derived) and HBM (measured copy)."""
    mhz = pk.get("sm_max_mhz", 2032.0)
    src = pk["source"]
    tens = pk["bf16_tflops"] * (2 if precision == "fp8" else 1)
    return {"tensor": {"peak": tens, "unit": "TFLOP/s",
                       "source": f"{src} bf16 burst" + (" x2 (fp8 nominal ratio)" if precision == "fp8" else "")},
            "tf32": {"peak": pk["bf16_tflops"] * 0.5, "unit": "TFLOP/s",
                     "source": f"{src} bf16 burst x0.5 (tf32 nominal ratio)"},
            "alu": {"peak": 148 * 128 * 2 * mhz * 1e6 / 1e12, "unit": "TFLOP/s",
                    "source": f"derived: 148 SMs x 128 FP32 FMA/clk x 2 x {mhz:.0f} MHz"},
            "hbm": {"peak": pk["hbm_gbs"], "unit": "GB/s", "source": f"{src} HBM copy"}}


def stage_work(hy: int, wy: int, H_: int, W_: int, nbytes: int, lanes: int, precision: str) -> dict:
    """Algorithmic work of one occurrence of every profiled stage of the plain model's step (arch 1, N
    frames, latent hy x wy): {stage: {"flops": F, "flop_kind": "tensor"|"tf32"|"alu", "bytes": B, "lane_steps": S}}.
    Bytes count every tensor a stage reads or writes once (activations bf16 on the tensor-core path, f32
    on the FP32 path; y, mu, log sigma f32; r^ int16; indices u8; bit-stream words), FLOPs = 2 x MACs;
    lane_steps = the longest lane's symbol count for the rANS stages."""
    from synthetic.weights import layer_table
    tab = {name: (co, k, ci) for name, co, k, ci in layer_table(1, N)}
    Hp, Wp = -(-H_ // 16) * 16, -(-W_ // 16) * 16
    h1, w1 = Hp // 2, Wp // 2
    h2, w2, h3, w3 = h1 // 2, w1 // 2, h1 // 4, w1 // 4
    hh, wh = -(-hy // 2), -(-wy // 2)
    hz, wz = -(-hh // 2), -(-wh // 2)

    def fl(name, h, w):
        co, k, ci = tab[name]
        return 2 * h * w * co * k * k * ci

    a = 4 if precision == "fp32" else (1 if precision == "fp8" else 2)
    kind = "alu" if precision == "fp32" else "tensor"
    n, nz = hy * wy * 256, hz * wz * 128
    e0, e1, e2 = 64, 128, 192
    out = {
        "A1": {"flops": fl("A1", h1, w1), "flop_kind": kind, "bytes": N * H_ * W_ * 3 + h1 * w1 * e0 * a},
        "analysis": {"flops": fl("A2", h2, w2) + fl("A3", h3, w3) + fl("Xa", h3, w3) + fl("Xb", h3, w3)
                     + fl("A4", hy, wy), "flop_kind": kind,
                     "bytes": (h1 * w1 * e0 + h2 * w2 * e1 * 2 + h3 * w3 * e2 * 7) * a + n * 4},
        "hyper_analysis": {"flops": fl("H1", hh, wh) + fl("H2", hz, wz), "flop_kind": kind,
                           "bytes": n * 4 + n * a * 2 + hh * wh * 128 * a * 2 + nz * 4 + nz * 2},
        # S1..S3 with the entropy parameters formed in S3's pass (encoder: y in; mu, log sigma, r^, idx out;
        # decoder: mu, idx out), the mean of the two; TF32 tensor cores in every precision (the GEMM
        # executes three products per multiply-add: the FLOPs here are the algorithmic ones)
        "hyper_synthesis": {"flops": fl("S1", hz, wz) + fl("S2", 2 * hz, 2 * wz) + fl("S3", hy, wy),
                            "flop_kind": "tf32",
                            "bytes": nz * 2 + 4 * hz * wz * 128 * 4 * 2 + 16 * hz * wz * 128 * 4 * 2
                                     + n * (4 + 4 + 4 + 2 + 1 + 4 + 1) // 2},
        "quantize": {"bytes": n * (4 + 4 + 4 + 2 + 1)},
        # both sections coded, laid out and the header written: symbols + indices in, the stream out
        "rans_encode": {"bytes": (n + nz) * 3 + nbytes, "lane_steps": -(-n // lanes)},
        # header + lane counts checked, z^ decoded
        "rans_decode_z": {"bytes": nz * 2 + 4 * min(lanes, nz) + 4096, "lane_steps": -(-nz // min(lanes, nz))},
        "scale_index": {"bytes": n * (4 + 1)},
        # stream + indices + mu in, y^ = r^ q + mu out (activation type)
        "rans_decode_y": {"bytes": nbytes + n * (1 + 4 + (4 if precision == "fp32" else a)),
                          "lane_steps": -(-n // lanes)},
        "dequant": {"bytes": n * (2 + 4 + (4 if precision == "fp32" else a))},
    }
    cb = conv_bytes(hy, wy, H_, W_)
    for k, f in conv_flops(hy, wy).items():
        out[k] = {"flops": f, "flop_kind": kind, "bytes": cb[k] * (2 if precision == "fp32" else 1)}
    return out


def stage_roofline(stage_ms: dict, work: dict, pk: dict) -> dict:
    """Each stage against its own bound: the compute peak of its kind or HBM, whichever its work takes
    longer at.  ms = mean time of one occurrence (the hyper-synthesis runs once in each direction)."""
    out = {}
    for k, ms in stage_ms.items():
        w = work.get(k)
        if w is None:
            continue
        t = ms / 1000.0
        tc = w.get("flops", 0) / (pk[w.get("flop_kind", "tensor")]["peak"] * 1e12)
        tm = w["bytes"] / (pk["hbm"]["peak"] * 1e9)
        if tc >= tm:
            kind = w["flop_kind"]
            ach = w["flops"] / t / 1e12
            e = {"bound": kind, "achieved": ach, "peak": pk[kind]["peak"], "unit": "TFLOP/s",
                 "frac": ach / pk[kind]["peak"], "algorithmic": w["flops"], "peak_source": pk[kind]["source"]}
        else:
            ach = w["bytes"] / t / 1e9
            e = {"bound": "hbm", "achieved": ach, "peak": pk["hbm"]["peak"], "unit": "GB/s",
                 "frac": ach / pk["hbm"]["peak"], "algorithmic": w["bytes"], "peak_source": pk["hbm"]["source"]}
        e["ms"] = ms
        e["floor_ms"] = 1000.0 * max(tc, tm)
        if "lane_steps" in w:
            e["lane_chain_ns_per_step"] = 1e6 * ms / w["lane_steps"]
        out[k] = {kk: (round(vv, 5) if isinstance(vv, float) else vv) for kk, vv in e.items()}
    return out


def entropy_sweep(U, dev, lanes=(1024, 4096, 16384, 65536), n=240 * 135 * 256, reps=5) -> dict:
    """Entropy-coding stress at 4K: n = 8 294 400 symbols round(mu + Laplace(0, b)), b log-uniform on
    [0.11, 64], scale index = the bin of b under the library's own thresholds; rANS encode and decode of
    the whole latent as one section per lane count, CUDA-event timed, lossless round trip checked."""
    import torch
    import synthetic
    blob = synthetic.draw_weights(0, 1, seed=0)
    codec = U.Codec(0, 1, 32, blob, "fp32", device=dev.index or 0)
    freq, _, thr = codec.get_tables(32)
    r, b = synthetic.laplace_symbols(n, seed=3)
    idx = (thr.astype(np.float64)[None, :] < np.log(b)[:, None]).sum(1).astype(np.uint8)
    ideal_bits = float(-np.log2(freq[idx, r.astype(np.int64) + 255] / 65536.0).sum())
    vals, cnts = np.unique(r, return_counts=True)
    pr = cnts / n
    st, it = torch.from_numpy(r).to(dev), torch.from_numpy(idx).to(dev)
    out = {"symbols": n, "ideal_bits_per_symbol": ideal_bits / n,
           "empirical_entropy_bits_per_symbol": float(-(pr * np.log2(pr)).sum()), "lanes": {}}
    hbm = peaks()["hbm_gbs"]
    for K_ in lanes:
        enc_ms, dec_ms = [], []
        for i in range(reps + 2):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            sec, nb = codec.rans_encode(st, it, K_)
            e1.record()
            nbytes = int(nb.item())
            e1b = torch.cuda.Event(enable_timing=True)
            e1b.record()
            dec = codec.rans_decode(sec, nbytes, it, n, K_)
            e2.record()
            torch.cuda.synchronize()
            if i >= 2:
                enc_ms.append(e0.elapsed_time(e1))
                dec_ms.append(e1b.elapsed_time(e2))
        assert codec.sync_status() == 0 and torch.equal(dec, st), f"rANS round trip failed at K={K_}"
        te, td = statistics.median(enc_ms), statistics.median(dec_ms)
        be, bd = 3 * n + nbytes, nbytes + n + 2 * n
        out["lanes"][str(K_)] = {
            "bytes": nbytes, "bits_per_symbol": 8 * nbytes / n, "overhead_vs_ideal": 8 * nbytes / ideal_bits - 1,
            "enc_ms": te, "dec_ms": td, "enc_gbs": be / te / 1e6, "dec_gbs": bd / td / 1e6,
            "enc_hbm_frac": be / te / 1e6 / hbm, "dec_hbm_frac": bd / td / 1e6 / hbm,
            "enc_ns_per_lane_symbol": te * 1e6 / (n / K_), "dec_ns_per_lane_symbol": td * 1e6 / (n / K_),
            "round_trip": "lossless"}
    codec.close()
    return out


# DRAM bytes per 1080p launch from one ncu capture of the SAME kernel build (dram__bytes_read.sum +
# dram__bytes_write.sum on the 960x544 chunk, scaled by the 4x pixel count).  An entry must be removed
# when its kernel changes.
NCU_TRAFFIC_1080P = {"dec.U2": 4 * (35.841536e6 + 74.318080e6), "dec.U3": 4 * (138.866688e6 + 6.584832e6)}

SERVING_MIX = [((854, 480), 0.40), ((1280, 720), 0.30), ((1920, 1080), 0.25), ((3840, 2160), 0.05)]


def serving_bench(U, dev, frames_1080p, blob, precision: str, windows: list, n_streams: int = 64, temporal=None,
                  seed: int = 0, drain_s: float = 120.0, dist=None, rank: int = 0, world: int = 1) -> dict:
    """Serving mix: n_streams streams of the SERVING_MIX resolutions (assigned by seed), each with Poisson
    chunk arrivals (one 8-frame chunk per Exp(mean 8/30 s) at 30 fps, divided by the window's rate
    multiplier), each stream's requests alternating encode and decode across all windows (a decode codes
    the stream's latest device-resident bit-stream, so every chunk is decoded, in order), submitted in real time to the continuous-batching server (HBM cap
    150 GB).  `windows` = [(rate multiplier, seconds), ...] run back to back on the same warm server,
    each drained before the next.  Per window: latency = submit -> completion on the server's clock;
    frames/s = frames of the completed requests / (last completion - first submit); the share of
    requests that ran in same-shape batches.  Content: the 1080p synthetic chunk, cropped for the
    smaller sizes and tiled 2 x 2 for 4K.  Under torchrun every rank serves the streams s with
    s mod world == rank (same global trace); frames and the span are aggregated over ranks (sum,
    slowest), latencies gathered."""
    import torch
    from paper_2606_04410_b300 import shard
    rng = np.random.default_rng(seed)
    sizes = [sz for sz, _ in SERVING_MIX]
    which = rng.choice(len(sizes), size=n_streams, p=[p for _, p in SERVING_MIX])
    src = torch.from_numpy(frames_1080p).to(dev)
    content = {}
    for W_, H_ in sizes:
        if W_ <= 1920:
            content[(W_, H_)] = src[:, :H_, :W_].contiguous()
        else:
            content[(W_, H_)] = src.repeat(1, 2, 2, 1)[:, :H_, :W_].contiguous()
    srv = U.Server(1, N, K, blob, precision, hbm_cap_bytes=150 << 30, max_slots=8, device=dev.index or 0,
                   temporal_weights=temporal)
    owned = shard.shard(list(range(n_streams)), rank, world)
    sids = {}
    for j in owned:
        W_, H_ = sizes[which[j]]
        sid = srv.open_stream(W_, H_, QP)
        srv.streams[sid]["frames_in"].copy_(content[(W_, H_)])
        sids[j] = sid
    torch.cuda.synchronize()
    # warm-up (slots, plans, workspaces, graph capture): every stream alone once, then all streams queued
    # at once twice (the batch sizes the windows meet: direct run, then capture), then drain
    warm = []
    for sid in sids.values():
        warm.append(srv.submit(sid, U.UFVC_OP_ENCODE))
        warm.append(srv.submit(sid, U.UFVC_OP_DECODE))
    for _ in range(2):
        warm += srv.submit_many([(sid, op) for op in (U.UFVC_OP_ENCODE, U.UFVC_OP_DECODE) for sid in sids.values()])
    for t in warm:
        assert srv.wait(t, 600000.0)["status"] == 0
    out = {"streams": n_streams, "mix": {f"{w}x{h}": int((which == i).sum()) for i, (w, h) in enumerate(sizes)},
           "ranks": world, "hbm_cap_gb": 150, "rates": {}}
    next_op = [U.UFVC_OP_ENCODE] * n_streams  # a stream's requests alternate across windows too
    for rate, window_s in windows:
        events = []
        for j in range(n_streams):  # the global trace (same on every rank), then this rank's share
            t = rng.exponential(8 / 30 / rate)
            while t < window_s:
                if j in sids:
                    events.append((t, sids[j], next_op[j]))
                next_op[j] = U.UFVC_OP_DECODE if next_op[j] == U.UFVC_OP_ENCODE else U.UFVC_OP_ENCODE
                t += rng.exponential(8 / 30 / rate)
        events.sort()
        st0 = srv.stats()
        if dist is not None and world > 1:
            dist.barrier()
        tickets = []
        t0 = time.perf_counter()
        for t, sid, op in events:
            d = t0 + t - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tickets.append((sid, op, srv.submit(sid, op)))
        deadline = time.perf_counter() + drain_s
        res = [(sid, op, srv.wait(tk, max(1.0, (deadline - time.perf_counter()) * 1000.0)))
               for sid, op, tk in tickets]
        done = [(sid, op, r) for sid, op, r in res if r["status"] == 0]
        pending = sum(1 for _, _, r in res if r["status"] == U.UFVC_PENDING)
        for _, _, tk in tickets:  # drain whatever the deadline left before the next window
            srv.wait(tk, 600000.0)
        st = srv.stats()
        lats = [(op, r["done_ms"] - r["submit_ms"]) for _, op, r in done]
        span_ms = (max(r["done_ms"] for _, _, r in done) - min(r["submit_ms"] for _, _, r in res)) if done else 1.0
        n_req, n_pend, n_batched = len(events), pending, st["batched"] - st0["batched"]
        if dist is not None and world > 1:
            gathered = [None] * world
            dist.all_gather_object(gathered, (lats, n_req, n_pend, n_batched))
            lats = [x for g in gathered for x in g[0]]
            n_req, n_pend = sum(g[1] for g in gathered), sum(g[2] for g in gathered)
            n_batched = sum(g[3] for g in gathered)
        n_done, span_ms = shard.aggregate(len(done), span_ms, dist if world > 1 else None, dev)
        lat = np.array([v for _, v in lats] or [0.0])
        lat_e = np.array([v for op, v in lats if op == U.UFVC_OP_ENCODE] or [0.0])
        lat_d = np.array([v for op, v in lats if op == U.UFVC_OP_DECODE] or [0.0])
        pc = lambda a, q: round(float(np.percentile(a, q)), 3)
        out["rates"][f"x{rate:g}"] = {
            "window_s": window_s, "offered_frames_per_s": round(N * n_req / window_s, 1), "requests": n_req,
            "completed": int(n_done), "pending_after_drain": n_pend,
            "frames_per_s": round(N * n_done / (span_ms / 1000.0), 1),
            "batched_share": round(n_batched / max(1, n_done), 3),
            "latency_ms": {"p50": pc(lat, 50), "p99": pc(lat, 99), "enc_p50": pc(lat_e, 50),
                           "enc_p99": pc(lat_e, 99), "dec_p50": pc(lat_d, 50), "dec_p99": pc(lat_d, 99)}}
    st = srv.stats()
    out.update({"slots": st["slots"], "graphs": st["graphs"], "batches": st["batches"],
                "hbm_used_gb": round(st["hbm_used"] / 2**30, 2)})
    srv.close()
    return out


def parse_windows(spec: str) -> list:
    """'1:60,2:8' -> [(1.0, 60.0), (2.0, 8.0)] (rate multiplier : seconds)."""
    return [(float(a), float(b)) for a, b in (w.split(":") for w in spec.split(",") if w)]


def time_codec(codec, fr, frames_np, W_, H_, steps, warmup, profile, flush, dist=None, world=1, temporal=False):
    """Encode + decode one chunk per step; per-step CUDA events on the launching stream, L2 flushed
    between steps (outside the events).  Returns timings, stage profile, stream size and PSNR.  With
    temporal, consecutive steps form one stream: each step's chunk is coded against the context the
    previous step produced (encoder and decoder each double-buffer their own)."""
    import torch
    dev = fr.device
    cap = codec.max_bitstream_bytes(W_, H_)
    bits = torch.empty(cap, dtype=torch.uint8, device=dev)
    nbytes = torch.zeros(1, dtype=torch.int64, device=dev)
    from paper_2606_04410_b300 import ufvc as U
    out = torch.empty(N * U.frame_bytes(codec.color, W_, H_), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    nb = 0
    ce = [codec.new_context(W_, H_), codec.new_context(W_, H_)] if temporal else None
    cd = [codec.new_context(W_, H_), codec.new_context(W_, H_)] if temporal else None
    k = [0]

    def enc():
        if temporal:
            codec.encode_chunk_tc(fr, ce[k[0] % 2] if k[0] else None, ce[(k[0] + 1) % 2], QP, bits, nbytes,
                                  width=W_, height=H_)
        else:
            codec.encode_chunk(fr, QP, bits, nbytes, width=W_, height=H_)

    def dec():
        if temporal:
            # the stream size changes from chunk to chunk: the decoder reads it on the device
            codec.decode_chunk_tc(bits, bits.numel(), W_, H_, cd[k[0] % 2] if k[0] else None, cd[(k[0] + 1) % 2], out,
                                  d_nbytes=nbytes)
            k[0] += 1
        else:
            codec.decode_chunk(bits, nb, W_, H_, out)

    for _ in range(warmup):  # also establishes the stream size, which the decoder call takes from the host
        enc()
        nb = int(nbytes.item())
        dec()
    assert codec.sync_status() == 0
    rec = out.float().cpu().numpy() / 255.0
    psnr = float(10 * np.log10(1.0 / np.mean((rec - frames_np.ravel() / 255.0) ** 2)))
    # timed steps: no host synchronisation between steps (the library's stage events accumulate and are
    # read once at the end), so the host enqueues ahead of the device as a serving loop does; the step
    # events bracket exactly one encode and one decode
    codec.set_profiling(profile)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    if dist is not None and world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(steps):
        flush.fill_(i & 0xFF)
        evs[i][0].record(stream)
        enc()
        evs[i][1].record(stream)
        dec()
        evs[i][2].record(stream)
    torch.cuda.synchronize()
    if dist is not None and world > 1:
        dist.barrier()
    prof_acc: dict[str, list] = {}
    if profile:
        for name, ms, nl in codec.get_profile(max_entries=64 * steps):
            prof_acc.setdefault(name, []).append((ms, nl))
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
    ap.add_argument("--no-entropy-sweep", action="store_true")
    ap.add_argument("--no-fp8", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-pm", action="store_true", help="skip the progressive-means variant")
    ap.add_argument("--no-color", action="store_true", help="skip the colour-format variants")
    ap.add_argument("--no-temporal", action="store_true", help="skip the temporal-context variant")
    ap.add_argument("--no-dc", action="store_true", help="skip the DC-block model (HT-S counts)")
    ap.add_argument("--serving-windows", default="1:60,2:8,4:8,8:5",
                    help="BF16 serving windows, rate multiplier:seconds, comma-separated")
    ap.add_argument("--serving-windows-fp32", default="0.25:8,1:4")
    ap.add_argument("--serving-windows-temporal", default="1:8,4:5")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    args.warmup = max(args.warmup, 3)

    import torch
    import torch.distributed as dist

    import synthetic
    from paper_2606_04410_b300 import shard
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
    if args.precision == "fp8":  # activation scales from the FP32 path on this chunk (seed 0 on rank 0)
        codec.calibrate_fp8(fr, QP)
    sampler = ClockSampler(local)
    r = time_codec(codec, fr, frames_np, W_, H_, args.steps, args.warmup, True, flush, dist, world)
    clocks = sampler.stop()
    t_step = [a + b for a, b in zip(r["t_enc"], r["t_dec"])]
    frames_all, total_ms = shard.aggregate(N * args.steps, sum(t_step), dist if world > 1 else None, dev)
    value = frames_all / (total_ms / 1000.0)

    # ---- roofline of every stage (per-stage events recorded inside the same timed steps) and of the
    #      dominant kernel.  The step runs 2 ms at the maximum SM clock (sampled below), so the tensor
    #      peak is the burst figure; the sustained one (a seconds-long GEMM loop at a power-capped clock) is
    #      reported beside it.
    prof_acc = r["prof"]
    stage_total_ms = {k: sum(m for m, _ in v) / args.steps for k, v in prof_acc.items()}
    # one occurrence of a stage = its share of a step (the hyper-synthesis runs in both directions; the
    # tail of the decoder may run frame by frame, as several entries of one stage)
    occ = {"hyper_synthesis": 2}
    stage_ms = {k: v / occ.get(k, 1) for k, v in stage_total_ms.items()}
    launches_per_step = sum(sum(n for _, n in v) for v in prof_acc.values()) / args.steps
    hy, wy = -(-H_ // 16), -(-W_ // 16)
    flops = conv_flops(hy, wy)
    conv_stages = {k: v for k, v in stage_ms.items() if k in flops}
    top = max(conv_stages, key=conv_stages.get)
    pk = peaks()
    peaks_used = compute_peaks(pk, args.precision)
    stages = stage_roofline(stage_ms, stage_work(hy, wy, H_, W_, r["nbytes"], K, args.precision), peaks_used)
    kern = {"dec.U3": "conv_tc_final_kernel<1>", "dec.R2": "conv_tc_halo_kernel<64,2,1>"}
    tr = stages[top]
    dec_conv_ms = sum(v for k, v in stage_total_ms.items() if k in flops)
    cpeak = peaks_used["tensor" if args.precision != "fp32" else "alu"]
    roofline = {"bound": tr["bound"], "kernel": (kern.get(top, "conv_tc_kernel") if args.precision != "fp32"
                                                 else "conv_simt") + f" ({top})",
                "achieved": tr["achieved"], "peak": tr["peak"], "unit": tr["unit"], "frac": tr["frac"],
                "traffic": NCU_TRAFFIC_1080P.get(top) if (W_, H_) == (W, H) and args.precision == "bf16" else None,
                "traffic_unit": "bytes per launch", "peak_source": tr["peak_source"],
                "per_launch": {"algorithmic": tr["algorithmic"], "ms": tr["ms"]},
                "stage_roofline": stages,
                "decoder_convs": {"tflops": sum(flops.values()) / (dec_conv_ms / 1000.0) / 1e12,
                                  "frac": sum(flops.values()) / (dec_conv_ms / 1000.0) / 1e12 / cpeak["peak"]},
                "stage_ms_per_step": {k: round(v, 4) for k, v in
                                      sorted(stage_total_ms.items(), key=lambda kv: -kv[1])}}
    if args.precision != "fp32":
        sus = pk["bf16_tflops_sustained"] * (2 if args.precision == "fp8" else 1)
        roofline["frac_of_sustained"] = tr["achieved"] / sus if tr["unit"] == "TFLOP/s" else None
        roofline["sustained_peak"] = sus

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

    # ---- the FP8 E4M3 variant under the same methodology (calibrated on this chunk)
    fp8 = None
    if args.precision == "bf16" and not args.no_fp8:
        c8 = U.Codec(1, N, K, blob, "fp8", device=local)
        c8.calibrate_fp8(fr, QP)
        s8 = max(3, args.steps // 2)
        r8 = time_codec(c8, fr, frames_np, W_, H_, s8, 3, True, flush)
        v8 = N * s8 / (sum(a + b for a, b in zip(r8["t_enc"], r8["t_dec"])) / 1000.0)
        fp8 = {"value": v8, "enc_fps": N / (statistics.mean(r8["t_enc"]) / 1000.0),
               "dec_fps": N / (statistics.mean(r8["t_dec"]) / 1000.0), "psnr_db": r8["psnr"],
               "bytes_per_chunk": r8["nbytes"], "steps": s8,
               "stage_ms_per_step": {k: round(sum(m for m, _ in v) / s8, 4) for k, v in
                                     sorted(r8["prof"].items(), key=lambda kv: -sum(m for m, _ in kv[1]))}}
        c8.close()

    # ---- the four-partition progressive means (BF16, same methodology): the paper's full entropy model,
    #      scales still from one pass so the stream is still coded in one step
    pm = None
    if args.precision == "bf16" and not args.no_pm:
        cpm = U.Codec(1, N, K, blob, "bf16", device=local, mean_weights=synthetic.draw_mean_weights(1, seed=0))
        spm = max(3, args.steps // 2)
        rp = time_codec(cpm, fr, frames_np, W_, H_, spm, 3, True, flush)
        vp = N * spm / (sum(a + b for a, b in zip(rp["t_enc"], rp["t_dec"])) / 1000.0)
        stage_pm = {k: round(sum(m for m, _ in v) / spm, 4) for k, v in
                    sorted(rp["prof"].items(), key=lambda kv: -sum(m for m, _ in kv[1]))}
        pm = {"value": vp, "enc_fps": N / (statistics.mean(rp["t_enc"]) / 1000.0),
              "dec_fps": N / (statistics.mean(rp["t_dec"]) / 1000.0), "psnr_db": rp["psnr"],
              "bytes_per_chunk": rp["nbytes"], "steps": spm,
              "dbitrate_vs_single_pass": (rp["nbytes"] - r["nbytes"]) / r["nbytes"],
              "dpsnr_db_vs_single_pass": rp["psnr"] - r["psnr"],
              "progressive_means_ms_per_step": stage_pm.get("progressive_means"),
              "stage_ms_per_step": stage_pm}
        cpm.close()

    # ---- the temporal chunk context (BF16): every step's chunk coded against the previous step's context
    tcx = None
    if args.precision == "bf16" and not args.no_temporal:
        ct = U.Codec(1, N, K, blob, "bf16", device=local, temporal_weights=synthetic.draw_temporal_weights(1, N, seed=0))
        stc = max(3, args.steps // 2)
        rt = time_codec(ct, fr, frames_np, W_, H_, stc, 3, True, flush, temporal=True)
        vt = N * stc / (sum(a + b for a, b in zip(rt["t_enc"], rt["t_dec"])) / 1000.0)
        st_t = {k: round(sum(m for m, _ in v) / stc, 4) for k, v in
                sorted(rt["prof"].items(), key=lambda kv: -sum(m for m, _ in kv[1]))}
        tcx = {"value": vt, "enc_fps": N / (statistics.mean(rt["t_enc"]) / 1000.0),
               "dec_fps": N / (statistics.mean(rt["t_dec"]) / 1000.0), "psnr_db": rt["psnr"],
               "bytes_per_chunk": rt["nbytes"], "steps": stc, "chunk_context_ms_per_step": st_t.get("chunk_context"),
               "stage_ms_per_step": st_t}
        ct.close()

    # ---- the DC-block model at the paper's HT-S block counts (arch 2), BF16, context carried between steps
    dcx = None
    if args.precision == "bf16" and not args.no_dc:
        cdc = U.Codec(2, N, K, synthetic.draw_dc_weights(N, seed=0), "bf16", device=local)
        sdc = max(3, args.steps // 2)
        rd = time_codec(cdc, fr, frames_np, W_, H_, sdc, 3, True, flush, temporal=True)
        t_enc, t_dec = statistics.mean(rd["t_enc"]), statistics.mean(rd["t_dec"])
        fl = dc_flops(-(-H_ // 16), -(-W_ // 16))
        st_d = {k: round(sum(m for m, _ in v) / sdc, 4) for k, v in
                sorted(rd["prof"].items(), key=lambda kv: -sum(m for m, _ in kv[1]))}
        pk_dc, pk_dc_sus = peaks()["bf16_tflops"], peaks()["bf16_tflops_sustained"]
        tf = (fl["enc"] + fl["dec"]) / ((t_enc + t_dec) / 1000.0) / 1e12
        dcx = {"value": N * sdc / (sum(a + b for a, b in zip(rd["t_enc"], rd["t_dec"])) / 1000.0),
               "enc_fps": N / (t_enc / 1000.0), "dec_fps": N / (t_dec / 1000.0), "psnr_db": rd["psnr"],
               "bytes_per_chunk": rd["nbytes"], "steps": sdc, "macs_per_frame_g": 205.3,
               "tensor_tflop_per_step": (fl["enc"] + fl["dec"]) / 1e12, "tensor_tflops": tf,
               "tensor_frac_of_burst": tf / pk_dc, "tensor_frac_of_sustained": tf / pk_dc_sus,
               "stage_ms_per_step": st_d}
        cdc.close()
        if not args.no_fp32_path:  # the FP32 DC model on the same chunk sequence (3 context steps), one timed step
            c32 = U.Codec(2, N, K, synthetic.draw_dc_weights(N, seed=0), "fp32", device=local)
            r32 = time_codec(c32, fr, frames_np, W_, H_, 1, 3, False, flush, temporal=True)
            c32.close()
            dcx["fp32_fps"] = N / ((r32["t_enc"][0] + r32["t_dec"][0]) / 1000.0)
            dcx["dpsnr_db_vs_fp32"] = rd["psnr"] - r32["psnr"]
            dcx["dbitrate_vs_fp32"] = (rd["nbytes"] - r32["nbytes"]) / r32["nbytes"]

    # ---- colour interface (YUV444 model interface): BT.709 RGB and YUV420 chunks of the same content
    color = None
    if args.precision == "bf16" and not args.no_color and (W_, H_) == (W, H):
        color = {}
        for name, fmt in (("rgb_bt709", U.COLOR_RGB_BT709), ("yuv420p", U.COLOR_YUV420P)):
            cc = U.Codec(1, N, K, blob, "bf16", device=local, color=fmt)
            if fmt == U.COLOR_YUV420P:  # the chunk's channels as Y, U, V with U, V subsampled 2x2
                u_, v_ = frames_np[:, ::2, ::2, 1], frames_np[:, ::2, ::2, 2]
                src = np.concatenate([frames_np[..., 0].reshape(N, -1), u_.reshape(N, -1), v_.reshape(N, -1)], 1)
            else:
                src = frames_np
            src = np.ascontiguousarray(src)
            fr_c = torch.from_numpy(src).to(dev)
            sc = max(3, args.steps // 4)
            rc_ = time_codec(cc, fr_c, src, W_, H_, sc, 3, True, flush)
            vc = N * sc / (sum(a + b for a, b in zip(rc_["t_enc"], rc_["t_dec"])) / 1000.0)
            st_c = {k: round(sum(m for m, _ in v) / sc, 4) for k, v in rc_["prof"].items()}
            color[name] = {"value": vc, "frame_bytes": U.frame_bytes(fmt, W_, H_), "psnr_db": rc_["psnr"],
                           "bytes_per_chunk": rc_["nbytes"], "pack_ms": st_c.get("pack"),
                           "color_out_ms": st_c.get("color_out"), "dec_u3_ms": st_c.get("dec.U3"), "steps": sc}
            cc.close()

    # ---- end-to-end through the host-buffer C calls (pinned host memory, copies inside the region)
    cap = r["cap"]
    h_frames = torch.from_numpy(frames_np).pin_memory()
    h_bits = torch.empty(cap, dtype=torch.uint8).pin_memory()
    h_out = torch.empty((N, H_, W_, 3), dtype=torch.uint8).pin_memory()
    import ctypes as C
    nbh = C.c_size_t()
    e2e_ms = []
    for i in range(max(3, args.steps // 2) + 2):  # serial: one synchronous encode + decode call per step
        t0 = time.perf_counter()
        rc = U.lib.ufvc_encode_chunk_host(codec.h, U._ptr(h_frames), N, W_, H_, QP, U._ptr(h_bits), cap,
                                          C.byref(nbh), U._stream(None))
        assert rc == 0
        rc = U.lib.ufvc_decode_chunk_host(codec.h, U._ptr(h_bits), nbh.value, U._ptr(h_out), N, W_, H_,
                                          U._stream(None))
        assert rc == 0
        if i >= 2:
            e2e_ms.append((time.perf_counter() - t0) * 1000.0)
    serial = {"value": N * world / (statistics.mean(e2e_ms) / 1000.0), "unit": "frames/s",
              "method": "ufvc_encode_chunk_host + ufvc_decode_chunk_host, one step at a time",
              "h2d_bytes_per_step": int(h_frames.numel() + nbh.value),
              "d2h_bytes_per_step": int(nbh.value + h_out.numel() + 8)}
    # pipelined (ufvc_pipe_*, five slots, with which the pipe enqueues a ticket's decode two encodes after
    # its own: 1.76 ms per 1080p step in steady state against 1.86 with four slots and 1.91 with three,
    # where the decode follows the next encode): every step still copies its frames in, its bit-stream
    # buffer out and back, and its decoded frames out; one slot's copies overlap the other slots' kernels.
    # The timed region runs from the first submit to the last wait (pipeline fill and drain included, over
    # 48 steps or more, about 0.1 s at 1080p, so that they weigh as in a stream of chunks rather than a
    # handful).
    depth, n_pipe = 5, max(48, args.steps)
    pipe = U.Pipe(codec, depth)
    pb = [torch.empty(cap, dtype=torch.uint8).pin_memory() for _ in range(depth)]
    po = [torch.empty((N, H_, W_, 3), dtype=torch.uint8).pin_memory() for _ in range(depth)]
    for rep in range(2):  # the first pass allocates the slots' plans and is not kept
        if dist is not None and world > 1:
            dist.barrier()
        tk = []
        t0 = time.perf_counter()
        for i in range(n_pipe):
            if i >= depth:
                pipe.wait(tk[i - depth])
            tk.append(pipe.submit(h_frames, W_, H_, pb[i % depth], po[i % depth], QP))
        for t in tk[-depth:]:
            nb_pipe = pipe.wait(t)
        pipe_ms = (time.perf_counter() - t0) * 1000.0
    pipe.close()
    frames_e2e, pipe_ms_max = shard.aggregate(N * n_pipe, pipe_ms, dist if world > 1 else None, dev)
    e2e = {"value": frames_e2e / (pipe_ms_max / 1000.0), "unit": "frames/s",
           "method": f"ufvc_pipe_submit / ufvc_pipe_wait, {depth} slots, {n_pipe} steps",
           "h2d_bytes_per_step": int(h_frames.numel() + cap), "d2h_bytes_per_step": int(cap + 8 + h_out.numel()),
           "bytes_per_chunk": int(nb_pipe), "serial": serial}

    # serving mix (every rank serves its share of the streams)
    serving = None
    if not args.no_serving and (W_, H_) == (W, H):
        dd = dist if world > 1 else None
        wins = parse_windows(args.serving_windows_fp32 if args.precision == "fp32" else args.serving_windows)
        serving = {args.precision: serving_bench(U, dev, frames_np, blob, args.precision, wins,
                                                 dist=dd, rank=rank, world=world)}
        if args.precision != "fp32" and not args.no_fp32_path:
            serving["fp32"] = serving_bench(U, dev, frames_np, blob, "fp32", parse_windows(args.serving_windows_fp32),
                                            dist=dd, rank=rank, world=world)
        if args.precision == "bf16" and not args.no_temporal:  # every stream carries its context chain
            serving["bf16_temporal"] = serving_bench(U, dev, frames_np, blob, "bf16",
                                                     parse_windows(args.serving_windows_temporal), dist=dd,
                                                     rank=rank, world=world,
                                                     temporal=synthetic.draw_temporal_weights(1, N, seed=0))

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
        if fp8 is not None:
            if fp32 is not None:
                fp8["dpsnr_db_vs_fp32"] = fp8["psnr_db"] - fp32["psnr_db"]
                fp8["dbitrate_vs_fp32"] = (fp8["bytes_per_chunk"] - fp32["bytes_per_chunk"]) / fp32["bytes_per_chunk"]
                fp8["speedup_vs_fp32"] = fp8["value"] / fp32["value"]
            line["fp8_path"] = fp8
        if color is not None:
            line["color_formats"] = color
        if tcx is not None:
            line["temporal_context_path"] = tcx
        if dcx is not None:
            line["dc_model_path"] = dcx
        if pm is not None:
            if fp32 is not None:
                pm["dbitrate_vs_fp32"] = (pm["bytes_per_chunk"] - fp32["bytes_per_chunk"]) / fp32["bytes_per_chunk"]
                pm["dpsnr_db_vs_fp32"] = pm["psnr_db"] - fp32["psnr_db"]
            line["progressive_means_path"] = pm
        if not args.no_entropy_sweep:
            line["entropy_sweep"] = entropy_sweep(U, dev)
        if serving is not None:
            line["serving"] = serving
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
