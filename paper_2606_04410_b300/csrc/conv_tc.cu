// BF16 implicit-GEMM convolution on the 5th-generation tensor cores (tcgen05 + TMEM), fed by TMA.
//
// GEMM view of one conv group: M = output pixels, N = output channels, K = taps x input channels.
// A CTA tile is 128 output pixels (a TH x TW block of one output image, TW * TH = 128) by BN output
// channels.  For tap (ky, kx) and a 64-channel chunk, the A tile is the TH x TW block of input pixels
// shifted by the tap, fetched by one TMA tiled load whose out-of-range rows are zero-filled (the
// convolution's zero padding).  Stride-2 layers view the NHWC input as (C, 2, W/2, 2, H/2) so that a
// tap again maps to one TMA box.  The B tile is BN rows (output channels) x 64 K of the K-major
// weight matrix [group][Cout][k*k*Cin].  Both land 128-byte swizzled in shared memory and feed
// tcgen05.mma (M=128, N=BN, K=16 per instruction) accumulating in TMEM.
//
// Persistent, warp-specialised CTA (one per SM): warp 0 issues TMA loads into a STAGES-deep ring;
// warp 1 owns TMEM and issues the MMAs; sixteen epilogue warps drain a double-buffered TMEM
// accumulator (tcgen05.ld), add bias, apply GELU / residual / pixel shuffle / crop / final frame
// mapping and store, while the MMAs of the next tile run.  Every mbarrier wait is bounded: on a
// timeout the kernel records UFVC_ERR_TIMEOUT, all roles stop, in-flight copies and MMAs are waited
// for (bounded), TMEM is freed and the kernel returns.
#include "ufvc_internal.h"
#include "tc_ptx.h"

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>
#include <cstdio>

namespace ufvc {

constexpr long long kSpinLimit = 4000000000LL;  // ~2 s at 2 GHz
constexpr int kEpiWarps = 16;  // four per TMEM lane quarter
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kBiasMax = 4096;                       // biases staged in shared memory (16 KB)
constexpr int kSmemExtra = 1024 + 512 + 16 + 4 * kBiasMax;  // alignment slack, barriers, bias table

// Epilogue groups of the streaming kernel: EG groups of 16 / EG epilogue warps drain EG different tiles
// at once (each tile's 128 accumulator rows by the group's 4 / EG warps per TMEM lane quarter), so the
// per-tile latency of narrow tiles (staging barrier, TMA store) overlaps; 2 EG TMEM accumulators.
__host__ __device__ constexpr int epi_groups(int BN) { return BN >= 192 ? 1 : BN == 128 ? 2 : 4; }



struct TcArgs {
    int Ho, Wo, TW, TH, tiles_w, tiles_h, n_tiles, groups, total_tiles;
    int ksteps, cin_chunks, k, pad, stride, a_grouped;
    const float* bias;
    int b_gs;
    int Cout;
    int mode, act, out_f32;
    void* out;
    long long out_gs;
    int out_h, out_w, out_c;
    const __nv_bfloat16* res;
    long long res_gs;
    int ps_major;  // pixel shuffle with sub-pixel-major accumulator columns (column = sub * out_c + channel)
    int c_rank;    // staged epilogue: 4 = NHWC store map (C, W, H, G); 5 = pixel-shuffle map (C', dx, W, dy, G*H)
    // FP8 E4M3 operands: accumulator column co is scaled by cscale[g * b_gs + co] (input tensor scale x the
    // output channel's weight scale); out_inv != 0: the output is E4M3 code = value * out_inv; res8: an
    // E4M3 residual of scale res_s
    const float* cscale;
    float out_inv;
    const uint8_t* res8;
    float res_s;
    int* err;
    // NHWC outputs: 1 when every pixel's channel run starts 16-byte aligned and Cout is a multiple of 32,
    // so the epilogue may store NV consecutive channels as 16-byte vectors; else channel by channel
    int vec_out;
    unsigned long long kmask;  // K steps that run (bit ks); the others have all-zero weights
    // split K (layers with few tiles): work unit u = tile u / ksplit, K range u % ksplit; each range's raw
    // sums go to ws [ksplit][groups][Ho][Wo][ws_c] (float) and conv_tc_split_reduce_kernel finishes the layer
    int ksplit;
    float* ws;
    int ws_c;
};

// All groups' biases (groups x Cout floats) copied once into shared memory when they fit; the epilogue
// then reads them from there instead of global memory.
__device__ __forceinline__ const float* stage_bias(const TcArgs& p, float* sbias) {
    const int total = p.groups * p.b_gs;
    if (total > kBiasMax) return p.bias;
    for (int i = threadIdx.x; i < total; i += blockDim.x) sbias[i] = __ldg(p.bias + i);
    return sbias;  // visible after the block barrier that follows the set-up
}

// CL: acquire at cluster scope (a barrier the other CTA of a pair arrives on)
template <bool CL = false>
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err,
                                         bool honour_abort = true) {
    auto test = [&] { return CL ? ptx::mbar_try_wait_cluster(bar, parity) : ptx::mbar_try_wait(bar, parity); };
    if (test()) return true;
    const long long t0 = clock64();
    while (true) {
        if (test()) return true;
        if (honour_abort && *abort_flag) return false;
        if (clock64() - t0 > kSpinLimit) {
            *abort_flag = 1;
            atomicCAS(err, 0, (int)UFVC_ERR_TIMEOUT);
            return false;
        }
    }
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) { ptx::tmem_ld32(taddr, v); }

// Operand scales (FP8), bias and activation, in place, for NV (16 or 32) consecutive accumulator
// columns of one output pixel.
template <int NV>
__device__ __forceinline__ void bias_act_cols(const TcArgs& p, const float* bias_all, int g, int co0, float* v) {
    if (p.cscale) {  // FP8: undo the operand scales first
        const float* cs = p.cscale + (size_t)g * p.b_gs + co0;
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] *= (co0 + i < p.Cout) ? __ldg(cs + i) : 0.0f;
    }
    const float* bias = bias_all + (size_t)g * p.b_gs + co0;
    if (co0 + NV <= p.Cout) {  // warp-uniform 16-byte loads (every lane reads the same columns)
#pragma unroll
        for (int i = 0; i < NV / 4; ++i) {
            const float4 b = reinterpret_cast<const float4*>(bias)[i];  // shared or global: plain loads
            v[4 * i] += b.x; v[4 * i + 1] += b.y; v[4 * i + 2] += b.z; v[4 * i + 3] += b.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] += (co0 + i < p.Cout) ? bias[i] : 0.0f;
    }
    if (p.act) {
#pragma unroll
        for (int i = 0; i < NV; i += 2) gelu_tc2(v[i], v[i + 1]);
    }
}

// bias_act_cols, then (NHWC outputs with a residual) the residual read from global memory.
template <int NV>
__device__ __forceinline__ void finish_cols(const TcArgs& p, const float* bias_all, int g, int oh, int ow, int co0,
                                            float* v) {
    bias_act_cols<NV>(p, bias_all, g, co0, v);
    if (p.mode == OUT_NHWC && p.res8 && co0 < p.Cout) {
        const uint4* r = reinterpret_cast<const uint4*>(p.res8 + (size_t)g * p.res_gs +
                                                        ((size_t)oh * p.out_w + ow) * p.out_c + co0);
#pragma unroll
        for (int i = 0; i < NV / 16; ++i) {
            uint4 u = r[i];
            const __nv_fp8x2_storage_t* h = reinterpret_cast<const __nv_fp8x2_storage_t*>(&u);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float2 f = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2(h[j], __NV_E4M3)));
                v[16 * i + 2 * j] += f.x * p.res_s;
                v[16 * i + 2 * j + 1] += f.y * p.res_s;
            }
        }
    }
    if (p.mode == OUT_NHWC && !p.out_f32 && p.res && co0 < p.Cout) {
        const uint4* r = reinterpret_cast<const uint4*>(p.res + (size_t)g * p.res_gs +
                                                        ((size_t)oh * p.out_w + ow) * p.out_c + co0);
#pragma unroll
        for (int i = 0; i < NV / 8; ++i) {
            uint4 u = r[i];
            const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&u);
#pragma unroll
            for (int j = 0; j < 8; ++j) v[8 * i + j] += __bfloat162float(h[j]);
        }
    }
}

// Epilogue of NV (16 or 32) consecutive accumulator columns of one output pixel, stored by this thread.
template <int NV>
__device__ __forceinline__ void store_cols(const TcArgs& p, const float* bias_all, int g, int oh, int ow, int co0,
                                           float* v) {
    finish_cols<NV>(p, bias_all, g, oh, ow, co0, v);
    if (p.mode == OUT_NHWC && !p.vec_out) {
        // channel by channel (e.g. 12 outputs: a pixel's run is neither 16-byte aligned nor NV long)
        const size_t o = (size_t)g * p.out_gs + ((size_t)oh * p.out_w + ow) * p.out_c;
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const int c = co0 + i;
            if (c >= p.Cout) break;
            if (p.out_inv != 0.0f)
                reinterpret_cast<uint8_t*>(p.out)[o + c] =
                    (uint8_t)__nv_cvt_float_to_fp8(v[i] * p.out_inv, __NV_SATFINITE, __NV_E4M3);
            else if (p.out_f32)
                reinterpret_cast<float*>(p.out)[o + c] = v[i];
            else
                reinterpret_cast<__nv_bfloat16*>(p.out)[o + c] = __float2bfloat16_rn(v[i]);
        }
        return;
    }
    if (p.out_inv != 0.0f && (p.mode == OUT_NHWC || (p.mode == OUT_PS && p.ps_major))) {
        // E4M3 output: NV consecutive channels of one pixel
        size_t o;
        if (p.mode == OUT_NHWC) {
            if (co0 >= p.Cout) return;
            o = (size_t)g * p.out_gs + ((size_t)oh * p.out_w + ow) * p.out_c + co0;
        } else {
            const int sub = co0 / p.out_c, cb = co0 - sub * p.out_c;
            const int y = 2 * oh + (sub >> 1), x = 2 * ow + (sub & 1);
            if (sub > 3 || y >= p.out_h || x >= p.out_w) return;
            o = (size_t)g * p.out_gs + ((size_t)y * p.out_w + x) * p.out_c + cb;
        }
        uint32_t w[NV / 4];
#pragma unroll
        for (int i = 0; i < NV / 4; ++i) {
            const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(v[4 * i] * p.out_inv, v[4 * i + 1] * p.out_inv),
                                                         __NV_SATFINITE, __NV_E4M3);
            const uint32_t hi = __nv_cvt_float2_to_fp8x2(
                make_float2(v[4 * i + 2] * p.out_inv, v[4 * i + 3] * p.out_inv), __NV_SATFINITE, __NV_E4M3);
            w[i] = lo | (hi << 16);
        }
        uint4* d = reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(p.out) + o);
#pragma unroll
        for (int i = 0; i < NV / 16; ++i) d[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
        return;
    }
    if (p.mode == OUT_NHWC) {
        if (co0 >= p.Cout) return;
        const size_t o = (size_t)g * p.out_gs + ((size_t)oh * p.out_w + ow) * p.out_c + co0;
        if (p.out_f32) {
            float4* d = reinterpret_cast<float4*>(reinterpret_cast<float*>(p.out) + o);
#pragma unroll
            for (int i = 0; i < NV / 4; ++i) d[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            return;
        }
        uint4* d = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(p.out) + o);
#pragma unroll
        for (int i = 0; i < NV / 8; ++i)
            d[i] = make_uint4(pack_bf16(v[8 * i], v[8 * i + 1]), pack_bf16(v[8 * i + 2], v[8 * i + 3]),
                              pack_bf16(v[8 * i + 4], v[8 * i + 5]), pack_bf16(v[8 * i + 6], v[8 * i + 7]));
        return;
    }
    if (p.ps_major) {
        // sub-pixel-major columns: the NV columns are NV consecutive channels of one output pixel
        const int sub = co0 / p.out_c, cb = co0 - sub * p.out_c;
        const int y = 2 * oh + (sub >> 1), x = 2 * ow + (sub & 1);
        if (sub > 3 || y >= p.out_h || x >= p.out_w) return;
        uint4* d = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(p.out) + (size_t)g * p.out_gs +
                                            ((size_t)y * p.out_w + x) * p.out_c + cb);
#pragma unroll
        for (int i = 0; i < NV / 8; ++i)
            d[i] = make_uint4(pack_bf16(v[8 * i], v[8 * i + 1]), pack_bf16(v[8 * i + 2], v[8 * i + 3]),
                              pack_bf16(v[8 * i + 4], v[8 * i + 5]), pack_bf16(v[8 * i + 6], v[8 * i + 7]));
        return;
    }
    // pixel shuffle x2: column co -> channel co/4 at sub-pixel (dy, dx) = ((co>>1)&1, co&1)
    const int cb = co0 >> 2;
    constexpr int NC = NV / 4;  // output channels covered
#pragma unroll
    for (int sub = 0; sub < 4; ++sub) {
        const int y = 2 * oh + (sub >> 1), x = 2 * ow + (sub & 1);
        if (y >= p.out_h || x >= p.out_w) continue;
        const size_t o = (size_t)g * p.out_gs + ((size_t)y * p.out_w + x) * p.out_c + cb;
        if (p.mode == OUT_PS) {
            if (cb >= p.out_c) continue;
            uint32_t w[NC / 2];
#pragma unroll
            for (int j = 0; j < NC / 2; ++j) w[j] = pack_bf16(v[4 * (2 * j) + sub], v[4 * (2 * j + 1) + sub]);
            if constexpr (NC == 8) {
                *reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(p.out) + o) = make_uint4(w[0], w[1], w[2], w[3]);
            } else {
                *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(p.out) + o) = make_uint2(w[0], w[1]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < NC; ++j) {
                if (cb + j >= p.out_c) break;
                const float f = fminf(fmaxf(0.5f + v[4 * j + sub], 0.0f), 1.0f);
                if (p.mode == OUT_PS_FINAL_F32)
                    reinterpret_cast<float*>(p.out)[o + j] = f;
                else
                    reinterpret_cast<uint8_t*>(p.out)[o + j] = (uint8_t)rintf(f * 255.0f);
            }
        }
    }
}

// STAGED: the epilogue writes the bf16 output tile into a 128-byte-swizzled staging tile in shared memory
// (64-column slabs of 128 rows x 128 B, the layout a TMA box of 64 channels x TW x TH has) and one thread
// per slab group stores it with TMA tiled stores, which clip at the tensor edges.  Otherwise every
// epilogue thread stores its own pixel's columns.
// OP selects the operand rows of a pipeline stage: OP_BF16 = 64 bf16 channels in 128-byte rows with the
// 128-byte swizzle; OP_E4M3 = 64 E4M3 channels (kind::f8f6f4, K = 32 per MMA) in 64-byte rows with the
// 64-byte swizzle, accumulators rescaled in the epilogue; OP_BF16_32 = 32 bf16 channels in 64-byte rows
// (the first layer, whose 3N <= 30 input channels would fill only part of a 64-channel stage).
enum { OP_BF16 = 0, OP_E4M3 = 1, OP_BF16_32 = 2 };

// KM: some K steps are skipped (TcArgs::kmask); otherwise every step runs and the loops carry no test.
// MT = 2: a tile is two 128-pixel sub-tiles stacked vertically (2 TH x TW pixels, one TMA box of 256 rows),
// which share each stage's weight tile: two MMAs per K slice into two accumulators, 25 % fewer operand
// bytes landing in shared memory per MMA; one epilogue group drains and stores the sub-tiles in turn.
// PAIR: the kernel runs as clusters of two CTAs on two SMs that share one MMA of M = 256
// (tcgen05.mma.cta_group::2, issued by the even CTA): a tile is two stacked 128-pixel sub-tiles, one per
// CTA; each CTA loads its own sub-tile's input rows and HALF of the stage's weight rows (BN / 2), and
// each holds its sub-tile's 128 x BN accumulator in its own TMEM, so a third fewer operand bytes land in
// each SM's shared memory per MMA at BN = 256.  Both CTAs' loads complete on the even CTA's stage
// barrier (its producer expects the bytes of both); the MMA commits arrive on both CTAs' barriers; the
// odd CTA's epilogue frees an accumulator by arriving on the even CTA's barrier.
// O8 (with STAGED): the output is E4M3 codes (value x out_inv), staged as 64-byte rows per 64-channel slab
// without swizzle; otherwise a staged output is bf16 (also for E4M3 operands, e.g. the layer feeding the
// bf16 final layer).
template <int BN, int STAGES, bool STAGED, int OP = OP_BF16, bool KM = false, int MT = 1, bool PAIR = false,
          bool O8 = false>
__global__ void __launch_bounds__(kThreads, 1)
    conv_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmC, const TcArgs p) {
    constexpr bool F8 = OP == OP_E4M3;
    static_assert(!O8 || (STAGED && F8), "E4M3 staging: staged E4M3 layers");
    constexpr int SLAB = 128 * (O8 ? 64 : 128);  // bytes of one 64-channel staging slab
    constexpr int ROWB = OP == OP_BF16 ? 128 : 64;  // bytes of one K row of a stage
    constexpr int CH = OP == OP_BF16_32 ? 32 : 64;  // input channels per stage
    static_assert(MT == 1 || (MT == 2 && (OP == OP_BF16 || OP == OP_E4M3)), "two sub-tiles: 64-channel rows");
    static_assert(!PAIR || ((OP == OP_BF16 || OP == OP_E4M3) && !KM && BN % 32 == 0), "CTA pairs: 64-channel rows");
    constexpr int A_BYTES = 128 * MT * ROWB;
    constexpr int B_BYTES = (PAIR ? BN / 2 : BN) * ROWB;  // this CTA's weight rows of a stage
    // 128-pixel sub-tiles of a tile; a pair's CTA r holds sub-tiles r MT .. r MT + MT - 1, and the pair's
    // MMA h joins sub-tile h of both CTAs (M = 256)
    constexpr int SUBS = PAIR ? 2 * MT : MT;
    constexpr int EG = MT == 2 ? 1 : epi_groups(BN);  // epilogue groups (tiles drained concurrently)
    constexpr int WPQ = 4 / EG;         // warps per TMEM lane quarter in a group
    constexpr int NACC = 2 * EG;        // TMEM accumulators
    constexpr int C_BYTES = STAGED ? (BN / 64) * SLAB * EG : 0;
    constexpr int ACOLS = MT * BN;      // TMEM columns of one tile's accumulator(s)
    constexpr uint32_t TMEM_COLS = (NACC * ACOLS <= 32) ? 32 : (NACC * ACOLS <= 64) ? 64 : (NACC * ACOLS <= 128) ? 128
                                   : (NACC * ACOLS <= 256) ? 256 : 512;
    static_assert(NACC * ACOLS <= 512, "TMEM columns");
    // each of the WPQ warps of a lane quarter in a group drains PER of the BN columns
    constexpr int PER = BN / WPQ < 16 ? 16 : BN / WPQ;
    constexpr int CHUNK = PER % 32 == 0 ? 32 : 16;  // accumulator columns per tcgen05.ld round
    // slab groups of the staged epilogue: GQ column parts of a group that share 64-column slabs
    constexpr int GQ = (PER % 64 == 0) ? 1 : (64 % PER == 0 ? 64 / PER : WPQ);
    constexpr int SG = WPQ / GQ;  // slab groups per epilogue group
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + STAGES * A_BYTES;
    uint8_t* sC = sB + STAGES * B_BYTES;  // staging tile (STAGED), 1024-byte aligned
    uint64_t* full = reinterpret_cast<uint64_t*>(sC + C_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;
    uint64_t* tempty = tfull + NACC;
    uint64_t* drain = tempty + NACC;
    uint64_t* cwritten = drain + 1;   // per slab group: all its threads wrote the staging tile
    uint64_t* cfree = cwritten + 4;   // per slab group: its previous TMA stores have read the staging tile
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(cfree + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* sbias = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(tmem_slot + 2) + 15) & ~uintptr_t(15));
    const float* bias_all = stage_bias(p, sbias);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t crank = PAIR ? ptx::cluster_rank() : 0;  // this CTA's place in its pair
    const int cid = PAIR ? blockIdx.x >> 1 : blockIdx.x, ncl = PAIR ? gridDim.x >> 1 : gridDim.x;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < NACC; ++a) {
            ptx::mbar_init(&tfull[a], 1);
            // pairs: one arrival per epilogue warp of the group, in both CTAs (on the even CTA's barrier)
            ptx::mbar_init(&tempty[a], PAIR ? 2 * 4 * WPQ : 128 * WPQ);
        }
        ptx::mbar_init(drain, 1);
        for (int gq = 0; gq < 4; ++gq) {
            ptx::mbar_init(&cwritten[gq], 128 * GQ);
            ptx::mbar_init(&cfree[gq], 1);
        }
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 1) {
        if constexpr (PAIR) ptx::tmem_alloc_pair(tmem_slot, TMEM_COLS);
        else ptx::tmem_alloc(tmem_slot, TMEM_COLS);
    }
    if (warp == 0 && lane == 0) {
        ptx::prefetch_tmap(&tmA);
        ptx::prefetch_tmap(&tmB);
        if (STAGED) ptx::prefetch_tmap(&tmC);
    }
    ptx::tc_fence_before();
    if constexpr (PAIR) ptx::cluster_sync();  // both CTAs' barriers exist before either signals the other's
    else __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    // the set-up above (barriers, TMEM, biases, descriptor prefetch) may overlap the previous kernel's
    // tail; its outputs are read, and this kernel's written, only after it has completed
    pdl_trigger();
    pdl_wait();
    const int tiles_m = p.tiles_w * p.tiles_h;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            int it = 0;
            uint32_t last_par[STAGES];
            bool used[STAGES];
#pragma unroll
            for (int s = 0; s < STAGES; ++s) { used[s] = false; last_par[s] = 0; }
            bool ok = true;
            for (int u = cid; u < p.total_tiles && ok; u += ncl) {
                const int t = u / p.ksplit, kr = u - t * p.ksplit;
                const int nt = t % p.n_tiles, r = t / p.n_tiles, mt = r % tiles_m, g = r / tiles_m;
                const int h0 = (mt / p.tiles_w) * p.TH * SUBS + (int)crank * MT * p.TH, w0 = (mt % p.tiles_w) * p.TW;
                const int ag = p.a_grouped ? g : 0;
                const int ke = (kr + 1) * p.ksteps / p.ksplit;
                for (int ks = kr * p.ksteps / p.ksplit; ks < ke; ++ks) {
                    if (KM && !((p.kmask >> ks) & 1ull)) continue;  // all-zero weights: no stage
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1;
                    ++it;
                    if (!wait_bar(&empty[s], ph ^ 1, abort_flag, p.err)) { ok = false; break; }
                    const int tap = ks / p.cin_chunks, c0 = (ks - tap * p.cin_chunks) * CH;
                    const int ky = tap / p.k, kx = tap - ky * p.k;
                    if constexpr (PAIR) {
                        // both CTAs' copies complete on the even CTA's barrier, which expects all of them
                        const uint32_t fb = ptx::mapa(ptx::smem_u32(&full[s]), 0);
                        if (crank == 0) ptx::mbar_arrive_expect_tx(&full[s], 2 * (A_BYTES + B_BYTES));
                        if (p.stride == 1) {
                            ptx::tma_load_4d_pair(sA + s * A_BYTES, &tmA, fb, c0, w0 + kx - p.pad, h0 + ky - p.pad, ag);
                        } else {
                            const int tx = kx - p.pad, ty = ky - p.pad;
                            const int wp = tx & 1, hp = ty & 1;
                            ptx::tma_load_5d_pair(sA + s * A_BYTES, &tmA, fb, c0, wp, w0 + ((tx - wp) >> 1), hp,
                                                  h0 + ((ty - hp) >> 1));
                        }
                        ptx::tma_load_3d_pair(sB + s * B_BYTES, &tmB, fb, ks * CH, nt * BN + (int)crank * (BN / 2), g);
                    } else {
                        ptx::mbar_arrive_expect_tx(&full[s], A_BYTES + B_BYTES);
                        if (p.stride == 1) {
                            ptx::tma_load_4d(sA + s * A_BYTES, &tmA, &full[s], c0, w0 + kx - p.pad, h0 + ky - p.pad, ag);
                        } else {
                            const int tx = kx - p.pad, ty = ky - p.pad;
                            const int wp = tx & 1, hp = ty & 1;
                            ptx::tma_load_5d(sA + s * A_BYTES, &tmA, &full[s], c0, wp, w0 + ((tx - wp) >> 1), hp,
                                             h0 + ((ty - hp) >> 1));
                        }
                        ptx::tma_load_3d(sB + s * B_BYTES, &tmB, &full[s], ks * CH, nt * BN, g);
                    }
                    used[s] = true;
                    last_par[s] = ph;
                }
            }
            // make sure no copy is still writing shared memory when the CTA exits (pairs: the even CTA's
            // barriers count the odd CTA's copies too, and the odd CTA stays until the closing cluster
            // barrier, which the even CTA reaches after these waits)
            if (!PAIR || crank == 0) {
#pragma unroll
                for (int s = 0; s < STAGES; ++s)
                    if (used[s]) wait_bar(&full[s], last_par[s], abort_flag, p.err, false);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer (pairs: the even CTA's)
        if (PAIR && crank != 0) {
            // the odd CTA issues nothing; its accumulators are complete when the even CTA's last commit lands
            if (lane == 0) wait_bar(drain, 0, abort_flag, p.err, false);
        } else if (lane == 0) {
            constexpr uint32_t idesc = F8 ? (PAIR ? ptx::idesc_e4m3_m256(BN) : ptx::idesc_e4m3(BN))
                                          : PAIR ? ptx::idesc_bf16_m256(BN) : ptx::idesc_bf16(BN);
            int it = 0, tl = 0;
            bool ok = true;
            for (int u = cid; u < p.total_tiles && ok; u += ncl, ++tl) {
                const int kr = u % p.ksplit;
                const int acc = tl % NACC, use = tl / NACC;
                if (!wait_bar<PAIR>(&tempty[acc], (use & 1) ^ 1, abort_flag, p.err)) break;
                ptx::tc_fence_after();
                const uint32_t d = tmem_base + acc * ACOLS;
                bool first = true;  // the tile's first executed step overwrites the accumulator
                const int ke = (kr + 1) * p.ksteps / p.ksplit;
                for (int ks = kr * p.ksteps / p.ksplit; ks < ke; ++ks) {
                    if (KM && !((p.kmask >> ks) & 1ull)) continue;
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1;
                    ++it;
                    if (!wait_bar(&full[s], ph, abort_flag, p.err)) { ok = false; break; }
                    ptx::tc_fence_after();
                    const uint32_t a0 = ptx::smem_u32(sA + s * A_BYTES), b0 = ptx::smem_u32(sB + s * B_BYTES);
                    if constexpr (F8 && PAIR) {
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk)  // M = 256 over the pair, 2 x K=32 E4M3 per 64-byte row
#pragma unroll
                            for (int h = 0; h < MT; ++h)
                                ptx::mma_f8_pair(d + h * BN, ptx::sdesc_sw64(a0 + h * 8192 + kk * 32),
                                                 ptx::sdesc_sw64(b0 + kk * 32), idesc, !first || kk != 0);
                    } else if constexpr (F8) {
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk)  // 2 x K=32 E4M3 per 64-byte row
#pragma unroll
                            for (int h = 0; h < MT; ++h)  // sub-tile h: rows 128 h .. of the A box
                                ptx::mma_f8(d + h * BN, ptx::sdesc_sw64(a0 + h * 8192 + kk * 32),
                                            ptx::sdesc_sw64(b0 + kk * 32), idesc, !first || kk != 0);
                    } else if constexpr (OP == OP_BF16_32) {
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk)  // 2 x K=16 BF16 per 64-byte row
                            ptx::mma_f16(d, ptx::sdesc_sw64(a0 + kk * 32), ptx::sdesc_sw64(b0 + kk * 32), idesc,
                                         !first || kk != 0);
                    } else if constexpr (PAIR) {
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)  // M = 256: rows 0..127 from this CTA, 128..255 from the odd one
#pragma unroll
                            for (int h = 0; h < MT; ++h)  // sub-tile h of both CTAs
                                ptx::mma_f16_pair(d + h * BN, ptx::sdesc_sw128(a0 + h * 16384 + kk * 32),
                                                  ptx::sdesc_sw128(b0 + kk * 32), idesc, !first || kk != 0);
                    } else {
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)  // 4 x K=16 BF16 per 128-byte row
#pragma unroll
                            for (int h = 0; h < MT; ++h)  // sub-tile h: rows 128 h .. of the A box
                                ptx::mma_f16(d + h * BN, ptx::sdesc_sw128(a0 + h * 16384 + kk * 32),
                                             ptx::sdesc_sw128(b0 + kk * 32), idesc, !first || kk != 0);
                    }
                    if constexpr (PAIR) ptx::mma_commit_pair(&empty[s], 3);  // both CTAs' stage s is free
                    else ptx::mma_commit(&empty[s]);
                    first = false;
                }
                if (ok) {
                    if constexpr (PAIR) ptx::mma_commit_pair(&tfull[acc], 3);
                    else ptx::mma_commit(&tfull[acc]);
                }
            }
            // all issued MMAs complete before TMEM is released
            if constexpr (PAIR) ptx::mma_commit_pair(drain, 3);
            else ptx::mma_commit(drain);
            wait_bar(drain, 0, abort_flag, p.err, false);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue warps
        const int q = warp & 3;                   // TMEM lane quarter this warp may access
        const int colq = (warp - 2) >> 2;         // 0..3: four warps (one per lane quarter) each
        const int egrp = colq / WPQ, cpart = colq % WPQ;  // epilogue group, column part within it
        const int row = q * 32 + lane;
        const int grp = egrp * SG + cpart / GQ;   // slab group (staged epilogue)
        const int lead = 2 + 4 * (egrp * WPQ + (cpart / GQ) * GQ);  // first warp of the slab group
        const bool elected = STAGED && warp == lead && lane == 0;
        uint8_t* sCg = sC + egrp * (BN / 64) * SLAB;             // this group's staging slabs
        int tl = egrp, k = 0;  // k counts sub-tiles (the staging barriers' phases)
        bool run = true;
        for (int u = cid + egrp * ncl; run && u < p.total_tiles; u += EG * ncl, tl += EG) {
            const int t = u / p.ksplit, kr = u - t * p.ksplit;
            const int acc = tl % NACC, use = tl / NACC;
            if (!__all_sync(0xffffffffu, wait_bar(&tfull[acc], use & 1, abort_flag, p.err))) break;
            ptx::tc_fence_after();
            const int nt = t % p.n_tiles, r = t / p.n_tiles, mt = r % tiles_m, g = r / tiles_m;
            const int w0 = (mt % p.tiles_w) * p.TW;
#pragma unroll 1
            for (int hs = 0; hs < MT; ++hs, ++k) {
                const int h0 = (mt / p.tiles_w) * p.TH * SUBS + ((PAIR ? (int)crank * MT : 0) + hs) * p.TH;
                const int oh = h0 + row / p.TW, ow = w0 + row % p.TW;
                const bool valid = oh < p.Ho && ow < p.Wo;
                const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + acc * ACOLS + hs * BN;
                const int c_begin = cpart * PER;
                bool ok = true;
#pragma unroll 1
                for (int c = c_begin; c < c_begin + PER && c < BN; c += CHUNK) {
                    float v[CHUNK];
                    if constexpr (CHUNK == 32) tmem_ld32(taddr + c, v); else ptx::tmem_ld16(taddr + c, v);
                    if constexpr (STAGED) {
                        if (valid) finish_cols<CHUNK>(p, bias_all, g, oh, ow, nt * BN + c, v);
                        if (c == c_begin && k > 0) {
                            // the group's previous TMA stores must have read its staging slabs
                            if (elected) {
                                ptx::bulk_wait_read0();
                                ptx::mbar_arrive(&cfree[grp]);
                            }
                            ok = __all_sync(0xffffffffu, wait_bar(&cfree[grp], (k - 1) & 1, abort_flag, p.err));
                            if (!ok) break;  // warp-uniform: the next tcgen05.ld needs the whole warp
                        }
                        if constexpr (O8) {
                            // row `row` of slab c/64: 64 E4M3 codes in order, 16 bytes at a time
                            const uint32_t base = ptx::smem_u32(sCg) + (c >> 6) * SLAB + row * 64 + (c & 63);
#pragma unroll
                            for (int i = 0; i < CHUNK / 16; ++i) {
                                uint32_t wq[4];
#pragma unroll
                                for (int k4 = 0; k4 < 4; ++k4) {
                                    const float* f = v + 16 * i + 4 * k4;
                                    const uint32_t lo = __nv_cvt_float2_to_fp8x2(
                                        make_float2(f[0] * p.out_inv, f[1] * p.out_inv), __NV_SATFINITE, __NV_E4M3);
                                    const uint32_t hi = __nv_cvt_float2_to_fp8x2(
                                        make_float2(f[2] * p.out_inv, f[3] * p.out_inv), __NV_SATFINITE, __NV_E4M3);
                                    wq[k4] = lo | (hi << 16);
                                }
                                ptx::st_shared_v4(base + 16 * i, wq[0], wq[1], wq[2], wq[3]);
                            }
                        } else {
                            // row `row` of slab c/64, 16-byte chunks XOR-swizzled by row & 7 (the TMA 128-byte swizzle)
                            const uint32_t base = ptx::smem_u32(sCg) + (c >> 6) * SLAB + row * 128;
#pragma unroll
                            for (int i = 0; i < CHUNK / 8; ++i) {
                                const int j = ((c & 63) >> 3) + i;
                                ptx::st_shared_v4(base + ((j ^ (row & 7)) << 4), pack_bf16(v[8 * i], v[8 * i + 1]),
                                                  pack_bf16(v[8 * i + 2], v[8 * i + 3]),
                                                  pack_bf16(v[8 * i + 4], v[8 * i + 5]),
                                                  pack_bf16(v[8 * i + 6], v[8 * i + 7]));
                            }
                        }
                    } else {
                        if (valid) {
                            if (p.ksplit > 1) {  // this K range's raw sums
                                float4* dst = reinterpret_cast<float4*>(
                                    p.ws + (((size_t)kr * p.groups + g) * p.Ho * p.Wo + (size_t)oh * p.Wo + ow) * p.ws_c +
                                    nt * BN + c);
#pragma unroll
                                for (int i = 0; i < CHUNK / 4; ++i)
                                    dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                            } else {
                                store_cols<CHUNK>(p, bias_all, g, oh, ow, nt * BN + c, v);
                            }
                        }
                    }
                }
                if (hs == MT - 1) {  // every sub-tile's columns are in registers or staged: free the accumulator
                    ptx::tc_fence_before();
                    if constexpr (PAIR) {  // one arrival per warp, on the even CTA's barrier
                        __syncwarp();
                        if (lane == 0) ptx::mbar_arrive_remote(ptx::mapa(ptx::smem_u32(&tempty[acc]), 0));
                    } else {
                        ptx::mbar_arrive(&tempty[acc]);
                    }
                }
                if (!ok) { run = false; break; }
                if constexpr (STAGED) {
                    ptx::fence_proxy_async();  // this thread's staging writes -> visible to the TMA (async proxy)
                    ptx::mbar_arrive(&cwritten[grp]);
                    if (warp == lead) {  // the elected thread's warp (warp-uniform)
                        bool w_ok = true;
                        if (lane == 0) w_ok = wait_bar(&cwritten[grp], k & 1, abort_flag, p.err);
                        if (!__shfl_sync(0xffffffffu, (int)w_ok, 0)) { run = false; break; }
                    }
                    if (elected && h0 < p.Ho) {  // a sub-tile wholly below the output stores nothing
                        const int lo = (cpart / GQ) * GQ * PER;
                        const int hi = lo + GQ * PER < BN ? lo + GQ * PER : BN;
                        for (int sl = lo >> 6; sl < (hi + 63) >> 6; ++sl) {
                            const int col0 = nt * BN + sl * 64;
                            const uint8_t* src = sCg + sl * SLAB;
                            if (p.c_rank == 4) {
                                ptx::tma_store_4d(&tmC, src, col0, w0, h0, g);
                            } else {
                                const int sub = col0 / p.out_c, c0 = col0 - sub * p.out_c;
                                ptx::tma_store_5d(&tmC, src, c0, sub & 1, w0, sub >> 1, g * p.Ho + h0);
                            }
                        }
                    }
                    if (elected) ptx::bulk_commit();
                }
            }
        }
        if (elected) ptx::bulk_wait0();  // stores complete before the CTA (and its shared memory) ends
    }
    ptx::tc_fence_before();
    // pairs: neither CTA leaves (freeing the shared memory and barriers the other signals) before both
    // are done
    if constexpr (PAIR) ptx::cluster_sync();
    else __syncthreads();
    if (warp == 1) {
        ptx::tc_fence_after();
        if constexpr (PAIR) ptx::tmem_dealloc_pair(tmem_base, TMEM_COLS);
        else ptx::tmem_dealloc(tmem_base, TMEM_COLS);
    }
}


// ------------------------------------------------------------------------------------------------
// Stride-1 3x3 layers with 64 input channels and <= 64 outputs (R2, U3 of the decoders): the weights stay
// resident in shared memory (9 taps x BN columns, BN <= 64), and a tile is a strip of 128 output
// pixels of one row, so its A operand for all nine taps comes from the three input rows above, on and
// below it (130 pixels each, one TMA box per row, zero-filled outside the image): tap (ky, kx) is the
// 128-row window starting kx rows into row ky.  The 128-byte swizzle is a function of the shared-memory
// address (as TMA writes it), so such a window is described by its start address alone (base offset 0),
// exactly like the 32-byte K-slice advance.  Input traffic per tile drops from 9 tiles to 3 rows
// and weight traffic to one load per CTA and (group, N tile).  Tiles are handed out in contiguous
// ranges so a CTA changes weights at most a few times; a change waits until the MMAs that read the old
// weights have completed.
// ------------------------------------------------------------------------------------------------
constexpr int kHaloRowBytes = 17 * 1024;  // 130 rows x 128 B, rounded up to the 1024-B swizzle repeat
__host__ __device__ constexpr int halo_groups(int BN) { return BN == 16 ? 4 : 2; }
constexpr int kHaloBoxBytes = 130 * 128;
// E4M3 operands (F8): 130 rows x 64 B with the 64-byte swizzle, rounded up to its 512-B repeat
constexpr int kHaloRowBytes8 = 17 * 512;
constexpr int kHaloBoxBytes8 = 130 * 64;

// Epilogue of the resident-weight kernel.  The 16 epilogue warps form halo_groups(BN) groups that drain
// different tiles at once, each from its own pair of TMEM accumulators: BN = 64 -> two groups of eight
// warps (two column halves of 32 x four TMEM lane quarters), BN = 16 -> four groups of four warps.
// OUTK: 0 = every thread stores its own pixel; 1 = bf16 NHWC (BN = 64) through a swizzled staging
// tile per group and a TMA store; 2 = E4M3 NHWC codes (BN = 64) through a plain staging tile (128 pixel
// rows of 64 bytes) per group and a TMA store.  (The final frame layer has its own kernel,
// conv_tc_final_kernel.)
// F8: E4M3 operands (kind::f8f6f4, K = 32 per MMA) in 64-byte rows with the 64-byte swizzle; a tap's
// window is again its start address kx rows into the input row; the epilogue rescales each accumulator
// column by the input scale times the output channel's weight scale (finish_cols).
template <int BN, int STAGES, int OUTK, bool F8 = false>
__global__ void __launch_bounds__(kThreads, 1)
    conv_tc_halo_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        const __grid_constant__ CUtensorMap tmC, const TcArgs p) {
    constexpr int RB = F8 ? 64 : 128;  // bytes of one pixel's 64 input channels
    constexpr int ROWB = F8 ? kHaloRowBytes8 : kHaloRowBytes;
    constexpr int A_BYTES = 3 * ROWB;
    constexpr int B_BYTES = 9 * BN * RB;
    constexpr int EG = halo_groups(BN);      // tiles drained concurrently (epilogue groups)
    constexpr int WPG = 16 / EG;             // warps per group: WPG / 4 column parts x 4 lane quarters
    constexpr int CPW = BN / (WPG / 4);      // accumulator columns per warp (16 or 32)
    constexpr int NACC = 2 * EG;             // TMEM accumulators
    constexpr uint32_t TMEM_COLS = NACC * BN <= 128 ? 128 : 256;
    constexpr int C_BYTES = OUTK == 1 ? EG * 128 * BN * 2 : OUTK == 2 ? EG * 128 * BN : 0;  // per group
    static_assert(BN == 16 || BN == 64, "resident-weight kernel: N tile of 16 or 64");
    static_assert(OUTK == 0 || BN == 64, "staged stores: N = 64");
    static_assert(OUTK != 2 || F8, "E4M3 staging: FP8 layers");
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sB = smem;
    uint8_t* sA = smem + B_BYTES;
    uint8_t* sC = sA + STAGES * A_BYTES;  // staging (OUTK != 0), 1024-byte aligned
    uint64_t* full = reinterpret_cast<uint64_t*>(sC + C_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;
    uint64_t* tempty = tfull + NACC;
    uint64_t* bfull = tempty + NACC;
    uint64_t* bfree = bfull + 1;
    uint64_t* drain = bfree + 1;
    uint64_t* cwritten = drain + 1;
    uint64_t* cfree = cwritten + 4;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(cfree + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* sbias = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(tmem_slot + 2) + 15) & ~uintptr_t(15));
    const float* bias_all = stage_bias(p, sbias);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < NACC; ++a) {
            ptx::mbar_init(&tfull[a], 1);
            ptx::mbar_init(&tempty[a], 32 * WPG);
        }
        ptx::mbar_init(bfull, 1);
        ptx::mbar_init(bfree, 1);
        ptx::mbar_init(drain, 1);
        for (int gq = 0; gq < 4; ++gq) {
            ptx::mbar_init(&cwritten[gq], 32 * WPG);
            ptx::mbar_init(&cfree[gq], 1);
        }
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 1) ptx::tmem_alloc(tmem_slot, TMEM_COLS);
    if (warp == 0 && lane == 0) {
        ptx::prefetch_tmap(&tmA);
        ptx::prefetch_tmap(&tmB);
        if (OUTK) ptx::prefetch_tmap(&tmC);
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    // the set-up above (barriers, TMEM, biases, descriptor prefetch) may overlap the previous kernel's
    // tail; its outputs are read, and this kernel's written, only after it has completed
    pdl_trigger();
    pdl_wait();
    // tile t = ((g * n_tiles + nt) * Ho + oh) * tiles_w + strip; this CTA owns [t_begin, t_end)
    const int t_begin = (int)((long long)p.total_tiles * blockIdx.x / gridDim.x);
    const int t_end = (int)((long long)p.total_tiles * (blockIdx.x + 1) / gridDim.x);

    if (warp == 0) {
        if (lane == 0) {
            int it = 0, cur_key = -1, nb = 0;
            uint32_t bfree_par = 0, last_par[STAGES];
            bool used[STAGES];
#pragma unroll
            for (int s = 0; s < STAGES; ++s) { used[s] = false; last_par[s] = 0; }
            for (int t = t_begin; t < t_end; ++t, ++it) {
                const int strip = t % p.tiles_w, r = t / p.tiles_w, oh = r % p.Ho, key = r / p.Ho;
                const int nt = key % p.n_tiles, g = key / p.n_tiles;
                if (key != cur_key) {
                    if (cur_key >= 0) {  // the MMAs that read the previous weights must be complete
                        if (!wait_bar(bfree, bfree_par, abort_flag, p.err)) break;
                        bfree_par ^= 1;
                    }
                    ptx::mbar_arrive_expect_tx(bfull, B_BYTES);
                    for (int tap = 0; tap < 9; ++tap) ptx::tma_load_3d(sB + tap * BN * RB, &tmB, bfull, tap * 64, nt * BN, g);
                    cur_key = key;
                    ++nb;
                }
                const int s = it % STAGES;
                const uint32_t ph = (it / STAGES) & 1;
                if (!wait_bar(&empty[s], ph ^ 1, abort_flag, p.err)) break;
                ptx::mbar_arrive_expect_tx(&full[s], 3 * (F8 ? kHaloBoxBytes8 : kHaloBoxBytes));
                const int ag = p.a_grouped ? g : 0, w0 = strip * 128;
                for (int ky = 0; ky < 3; ++ky)
                    ptx::tma_load_4d(sA + s * A_BYTES + ky * ROWB, &tmA, &full[s], 0, w0 - 1, oh + ky - 1, ag);
                used[s] = true;
                last_par[s] = ph;
            }
            // make sure no copy is still writing shared memory when the CTA exits
#pragma unroll
            for (int s = 0; s < STAGES; ++s)
                if (used[s]) wait_bar(&full[s], last_par[s], abort_flag, p.err, false);
            if (nb) wait_bar(bfull, (nb - 1) & 1, abort_flag, p.err, false);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = F8 ? ptx::idesc_e4m3(BN) : ptx::idesc_bf16(BN);
            int it = 0, tl = 0, cur_key = -1;
            uint32_t bfull_par = 0;
            for (int t = t_begin; t < t_end; ++t, ++it, ++tl) {
                const int key = t / p.tiles_w / p.Ho;
                if (key != cur_key) {
                    if (cur_key >= 0) ptx::mma_commit(bfree);  // old weights free once these MMAs finish
                    if (!wait_bar(bfull, bfull_par, abort_flag, p.err)) break;
                    bfull_par ^= 1;
                    ptx::tc_fence_after();
                    cur_key = key;
                }
                const int acc = tl % NACC, use = tl / NACC;
                if (!wait_bar(&tempty[acc], (use & 1) ^ 1, abort_flag, p.err)) break;
                const int s = it % STAGES;
                const uint32_t ph = (it / STAGES) & 1;
                if (!wait_bar(&full[s], ph, abort_flag, p.err)) break;
                ptx::tc_fence_after();
                const uint32_t d = tmem_base + acc * BN;
                const uint32_t a0 = ptx::smem_u32(sA + s * A_BYTES), b0 = ptx::smem_u32(sB);
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const int ky = tap / 3, kx = tap % 3;
                    if constexpr (F8) {
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk)  // 2 x K=32 E4M3 per 64-byte row
                            ptx::mma_f8(d, ptx::sdesc_sw64(a0 + ky * ROWB + kx * 64 + kk * 32),
                                        ptx::sdesc_sw64(b0 + tap * BN * 64 + kk * 32), idesc, (tap | kk) != 0);
                    } else {
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            ptx::mma_f16(d, ptx::sdesc_sw128(a0 + ky * ROWB + kx * 128 + kk * 32),
                                         ptx::sdesc_sw128(b0 + tap * BN * 128 + kk * 32), idesc, (tap | kk) != 0);
                    }
                }
                ptx::mma_commit(&empty[s]);
                ptx::mma_commit(&tfull[acc]);
            }
            ptx::mma_commit(drain);
            wait_bar(drain, 0, abort_flag, p.err, false);
        }
        __syncwarp();
    } else {
        // epilogue: warp 2 + 4 c + q reads TMEM lane quarter q; c = grp * (WPG / 4) + part
        const int q = warp & 3, colq = (warp - 2) >> 2, row = q * 32 + lane;
        const int grp = colq / (WPG / 4), part = colq % (WPG / 4);
        const bool lead_warp = warp == 2 + grp * WPG;
        const bool elected = OUTK != 0 && lead_warp && lane == 0;
        uint8_t* sCg = sC + grp * (128 * BN * (OUTK == 2 ? 1 : 2));
        int tl = grp, k = 0;
        for (int t = t_begin + grp; t < t_end; t += EG, tl += EG, ++k) {
            const int acc = tl % NACC, use = tl / NACC;
            if (!__all_sync(0xffffffffu, wait_bar(&tfull[acc], use & 1, abort_flag, p.err))) break;
            ptx::tc_fence_after();
            const int strip = t % p.tiles_w, r = t / p.tiles_w, oh = r % p.Ho, key = r / p.Ho;
            const int nt = key % p.n_tiles, g = key / p.n_tiles;
            const int ow = strip * 128 + row;
            const bool valid = ow < p.Wo;
            const int co0 = nt * BN + part * CPW;
            float v[CPW];
            const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + acc * BN + part * CPW;
            if constexpr (CPW == 32) ptx::tmem_ld32(taddr, v); else ptx::tmem_ld16(taddr, v);
            ptx::tc_fence_before();
            ptx::mbar_arrive(&tempty[acc]);  // the accumulator is in registers: TMEM free for the next tile
            if constexpr (OUTK == 0) {
                if (valid) store_cols<CPW>(p, bias_all, g, oh, ow, co0, v);
            } else {
                if (valid) finish_cols<CPW>(p, bias_all, g, oh, ow, co0, v);
                if (k > 0) {  // the group's previous TMA store must have read its staging tile
                    if (elected) {
                        ptx::bulk_wait_read0();
                        ptx::mbar_arrive(&cfree[grp]);
                    }
                    if (!__all_sync(0xffffffffu, wait_bar(&cfree[grp], (k - 1) & 1, abort_flag, p.err))) break;
                }
                if constexpr (OUTK == 2) {
                    // E4M3 codes, 64-byte pixel rows in order (no swizzle), 16 bytes at a time
                    const uint32_t base = ptx::smem_u32(sCg) + row * 64 + part * CPW;
#pragma unroll
                    for (int i = 0; i < CPW / 16; ++i) {
                        uint32_t wq[4];
#pragma unroll
                        for (int k4 = 0; k4 < 4; ++k4) {
                            const float* f = v + 16 * i + 4 * k4;
                            const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(f[0] * p.out_inv, f[1] * p.out_inv),
                                                                         __NV_SATFINITE, __NV_E4M3);
                            const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(f[2] * p.out_inv, f[3] * p.out_inv),
                                                                         __NV_SATFINITE, __NV_E4M3);
                            wq[k4] = lo | (hi << 16);
                        }
                        ptx::st_shared_v4(base + 16 * i, wq[0], wq[1], wq[2], wq[3]);
                    }
                } else {
                    const uint32_t base = ptx::smem_u32(sCg) + row * 128;
#pragma unroll
                    for (int i = 0; i < CPW / 8; ++i) {
                        const int j = part * (CPW / 8) + i;
                        ptx::st_shared_v4(base + ((j ^ (row & 7)) << 4), pack_bf16(v[8 * i], v[8 * i + 1]),
                                          pack_bf16(v[8 * i + 2], v[8 * i + 3]), pack_bf16(v[8 * i + 4], v[8 * i + 5]),
                                          pack_bf16(v[8 * i + 6], v[8 * i + 7]));
                    }
                }
                ptx::fence_proxy_async();
                ptx::mbar_arrive(&cwritten[grp]);
                if (lead_warp) {
                    bool w_ok = true;
                    if (lane == 0) w_ok = wait_bar(&cwritten[grp], k & 1, abort_flag, p.err);
                    if (!__shfl_sync(0xffffffffu, (int)w_ok, 0)) break;
                }
                if (elected) {
                    ptx::tma_store_4d(&tmC, sCg, nt * BN, strip * 128, oh, g);
                    ptx::bulk_commit();
                }
            }
        }
        if (elected) ptx::bulk_wait0();
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem_base, TMEM_COLS);
    }
}

// ------------------------------------------------------------------------------------------------
// Stride-1 3x3 layers with 64 bf16 inputs and 64 bf16 NHWC outputs (the decoders' R2) with the three
// horizontal taps in the MMA's N dimension.  With A = input pixels and B = one tap's 64 x 64 weights
// (the resident-weight kernel above) each MMA is M = 128, N = 64: 6 KB of operands read from shared
// memory per 262 KFLOP, so the tensor cores wait on shared memory.  Here B for kernel row ky is the
// 192 x 64 matrix of the three taps (kx, c) stacked, so one MMA of N = 192 per (ky, 16 channels)
// computes, for every input pixel x of the strip,
//     D[x][(kx, c)] = sum_ky sum_ci w[c][ky][kx][ci] in[oh + ky - 1][x][ci]
// (12 MMAs per tile instead of 36, 10 KB of operands per 786 KFLOP), and the epilogue applies the
// horizontal shift: out[oh][x][c] = D[x - 1][(0, c)] + D[x][(1, c)] + D[x + 1][(2, c)].  Accumulator
// rows are pixels, i.e. TMEM lanes, so the neighbours are warp shuffles: warp quarter q holds input
// pixels x0 + 30 q - 1 .. x0 + 30 q + 30 (one 32-pixel TMA box per quarter and input row, halos
// overlapping) and its lanes 1..30 produce output pixels x0 + 30 q .. x0 + 30 q + 29, so a tile is a
// strip of 120 output pixels of one row.  The resident weights keep the tap-major layout of the kernel
// above (tap = 3 ky + kx, 64 rows each), so the three taps of one ky are 192 consecutive rows.
// Two epilogue groups of eight warps (two column halves x four lane quarters) drain alternate tiles
// from two accumulators of 192 columns; outputs go through a swizzled staging tile per group and a
// TMA store of 120 pixels x 64 channels, which clips at the image edge.  A residual (p.res) arrives
// by TMA in the staging tile itself (the layout the output is stored from): the group's elected thread
// loads the residual of the group's next tile as soon as the previous store has read the tile, so the
// epilogue threads add it from shared memory instead of waiting on global loads.
// ------------------------------------------------------------------------------------------------
// F8: E4M3 operands (kind::f8f6f4, K = 32 per MMA) in 64-byte rows with the 64-byte swizzle, E4M3
// outputs (value x out_inv) staged as plain 64-byte rows, and an E4M3 residual of scale res_s; the
// accumulator columns are rescaled per output channel (input scale x weight scale) after the three
// horizontal taps are summed, which share the channel's scale.
constexpr int kKxnStrip = 120;       // output pixels per tile
template <int STAGES, bool F8 = false>
__global__ void __launch_bounds__(kThreads, 1)
    conv_tc_kxn_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                       const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmR,
                       const TcArgs p) {
    constexpr int RB = F8 ? 64 : 128;         // bytes of one pixel's 64 channels
    constexpr int BOXB = 32 * RB;             // one 32-pixel box
    constexpr int ROWB = 4 * BOXB;            // one input row of a tile: four boxes
    constexpr int A_BYTES = 3 * ROWB;
    constexpr int B_BYTES = 9 * 64 * RB;
    constexpr int CSLOT = F8 ? 8192 : 16384;  // one staging tile of 120 pixel rows
    constexpr int C_BYTES = 2 * CSLOT;
    constexpr uint32_t TMEM_COLS = 512;  // accumulators at columns 0 and 256, 192 columns each
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sB = smem;
    uint8_t* sA = smem + B_BYTES;
    uint8_t* sC = sA + STAGES * A_BYTES;
    uint64_t* full = reinterpret_cast<uint64_t*>(sC + C_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* bfull = tempty + 2;
    uint64_t* bfree = bfull + 1;
    uint64_t* drain = bfree + 1;
    uint64_t* cwritten = drain + 1;
    uint64_t* cfree = cwritten + 2;
    uint64_t* rfull = cfree + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(rfull + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* sbias = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(tmem_slot + 2) + 15) & ~uintptr_t(15));
    const float* bias_all = stage_bias(p, sbias);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            ptx::mbar_init(&tfull[a], 1);
            ptx::mbar_init(&tempty[a], 32 * 8);
            ptx::mbar_init(&cwritten[a], 32 * 8);
            ptx::mbar_init(&cfree[a], 1);
            ptx::mbar_init(&rfull[a], 1);
        }
        ptx::mbar_init(bfull, 1);
        ptx::mbar_init(bfree, 1);
        ptx::mbar_init(drain, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 1) ptx::tmem_alloc(tmem_slot, TMEM_COLS);
    if (warp == 0 && lane == 0) {
        ptx::prefetch_tmap(&tmA);
        ptx::prefetch_tmap(&tmB);
        ptx::prefetch_tmap(&tmC);
        if (p.res) ptx::prefetch_tmap(&tmR);
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    pdl_trigger();
    pdl_wait();
    // tile t = (g * Ho + oh) * tiles_w + strip; this CTA owns [t_begin, t_end)
    const int t_begin = (int)((long long)p.total_tiles * blockIdx.x / gridDim.x);
    const int t_end = (int)((long long)p.total_tiles * (blockIdx.x + 1) / gridDim.x);

    if (warp == 0) {
        if (lane == 0) {
            int it = 0, cur_g = -1, nb = 0;
            uint32_t bfree_par = 0, last_par[STAGES];
            bool used[STAGES];
#pragma unroll
            for (int s = 0; s < STAGES; ++s) { used[s] = false; last_par[s] = 0; }
            for (int t = t_begin; t < t_end; ++t, ++it) {
                const int strip = t % p.tiles_w, r = t / p.tiles_w, oh = r % p.Ho, g = r / p.Ho;
                if (g != cur_g) {
                    if (cur_g >= 0) {  // the MMAs that read the previous group's weights must be complete
                        if (!wait_bar(bfree, bfree_par, abort_flag, p.err)) break;
                        bfree_par ^= 1;
                    }
                    ptx::mbar_arrive_expect_tx(bfull, B_BYTES);
                    for (int tap = 0; tap < 9; ++tap) ptx::tma_load_3d(sB + tap * 64 * RB, &tmB, bfull, tap * 64, 0, g);
                    cur_g = g;
                    ++nb;
                }
                const int s = it % STAGES;
                const uint32_t ph = (it / STAGES) & 1;
                if (!wait_bar(&empty[s], ph ^ 1, abort_flag, p.err)) break;
                ptx::mbar_arrive_expect_tx(&full[s], A_BYTES);
                const int ag = p.a_grouped ? g : 0, x0 = strip * kKxnStrip;
                for (int ky = 0; ky < 3; ++ky)
                    for (int q = 0; q < 4; ++q)
                        ptx::tma_load_4d(sA + s * A_BYTES + ky * ROWB + q * BOXB, &tmA, &full[s], 0,
                                         x0 + 30 * q - 1, oh + ky - 1, ag);
                used[s] = true;
                last_par[s] = ph;
            }
#pragma unroll
            for (int s = 0; s < STAGES; ++s)
                if (used[s]) wait_bar(&full[s], last_par[s], abort_flag, p.err, false);
            if (nb) wait_bar(bfull, (nb - 1) & 1, abort_flag, p.err, false);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = F8 ? ptx::idesc_e4m3(192) : ptx::idesc_bf16(192);
            int it = 0, cur_g = -1;
            uint32_t bfull_par = 0;
            for (int t = t_begin; t < t_end; ++t, ++it) {
                const int g = t / p.tiles_w / p.Ho;
                if (g != cur_g) {
                    if (cur_g >= 0) ptx::mma_commit(bfree);  // old weights free once these MMAs finish
                    if (!wait_bar(bfull, bfull_par, abort_flag, p.err)) break;
                    bfull_par ^= 1;
                    ptx::tc_fence_after();
                    cur_g = g;
                }
                const int acc = it & 1, use = it >> 1;
                if (!wait_bar(&tempty[acc], (use & 1) ^ 1, abort_flag, p.err)) break;
                const int s = it % STAGES;
                const uint32_t ph = (it / STAGES) & 1;
                if (!wait_bar(&full[s], ph, abort_flag, p.err)) break;
                ptx::tc_fence_after();
                const uint32_t d = tmem_base + acc * 256;
                const uint32_t a0 = ptx::smem_u32(sA + s * A_BYTES), b0 = ptx::smem_u32(sB);
#pragma unroll
                for (int ky = 0; ky < 3; ++ky) {
                    if constexpr (F8) {
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk)
                            ptx::mma_f8(d, ptx::sdesc_sw64(a0 + ky * ROWB + kk * 32),
                                        ptx::sdesc_sw64(b0 + ky * 192 * 64 + kk * 32), idesc, (ky | kk) != 0);
                    } else {
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            ptx::mma_f16(d, ptx::sdesc_sw128(a0 + ky * ROWB + kk * 32),
                                         ptx::sdesc_sw128(b0 + ky * 192 * 128 + kk * 32), idesc, (ky | kk) != 0);
                    }
                }
                ptx::mma_commit(&empty[s]);
                ptx::mma_commit(&tfull[acc]);
            }
            ptx::mma_commit(drain);
            wait_bar(drain, 0, abort_flag, p.err, false);
        }
        __syncwarp();
    } else {
        // epilogue: warp 2 + 4 c + q reads TMEM lane quarter q; c = 2 grp + part (channels 32 part ..)
        const int q = warp & 3, colq = (warp - 2) >> 2, grp = colq >> 1, part = colq & 1;
        const bool lead_warp = warp == 2 + grp * 8;
        const bool elected = lead_warp && lane == 0;
        const bool inner = lane >= 1 && lane <= 30;  // lanes that produce an output pixel
        const int srow = 30 * q + lane - 1;           // its row of the 120-pixel strip
        const bool res = F8 ? p.res8 != nullptr : p.res != nullptr;
        uint8_t* sCg = sC + grp * CSLOT;
        // the residual of tile t into the staging tile (elected thread)
        auto load_res = [&](int t) {
            const int strip = t % p.tiles_w, r = t / p.tiles_w, oh = r % p.Ho, g = r / p.Ho;
            ptx::mbar_arrive_expect_tx(&rfull[grp], kKxnStrip * RB);
            ptx::tma_load_4d(sCg, &tmR, &rfull[grp], 0, strip * kKxnStrip, oh, g);
        };
        int n_res = 0;  // residual loads issued
        if (res && elected && t_begin + grp < t_end) { load_res(t_begin + grp); ++n_res; }
        int k = 0;
        for (int t = t_begin + grp, tl = grp; t < t_end; t += 2, tl += 2, ++k) {
            const int use = tl >> 1;
            if (!__all_sync(0xffffffffu, wait_bar(&tfull[grp], use & 1, abort_flag, p.err))) break;
            ptx::tc_fence_after();
            const int strip = t % p.tiles_w, r = t / p.tiles_w, oh = r % p.Ho, g = r / p.Ho;
            const int co0 = part * 32;
            const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + grp * 256 + co0;
            float v[32], u[32];
            ptx::tmem_ld32(taddr + 64, v);  // kx = 1: this pixel
            ptx::tmem_ld32(taddr, u);       // kx = 0: the pixel to the left contributes
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] += __shfl_up_sync(0xffffffffu, u[i], 1);
            ptx::tmem_ld32(taddr + 128, u);  // kx = 2: the pixel to the right contributes
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] += __shfl_down_sync(0xffffffffu, u[i], 1);
            ptx::tc_fence_before();
            ptx::mbar_arrive(&tempty[grp]);  // the accumulator is in registers: TMEM free for the next tile
            bias_act_cols<32>(p, bias_all, g, co0, v);
            // this pixel's row of the staging tile: bf16 128-byte rows with the 128-byte swizzle, or E4M3
            // 64-byte rows in order (this thread's 32 channels: bytes 32 part ..)
            const uint32_t base = ptx::smem_u32(sCg) + srow * RB;
            if (res) {  // the residual tile has landed in the staging tile
                if (!__all_sync(0xffffffffu, wait_bar(&rfull[grp], k & 1, abort_flag, p.err))) break;
                if (inner) {
                    if constexpr (F8) {
#pragma unroll
                        for (int i = 0; i < 2; ++i) {
                            const uint4 w = ptx::ld_shared_v4(base + part * 32 + 16 * i);
                            const __nv_fp8x2_storage_t* h = reinterpret_cast<const __nv_fp8x2_storage_t*>(&w);
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                const float2 f = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2(h[e], __NV_E4M3)));
                                v[16 * i + 2 * e] += f.x * p.res_s;
                                v[16 * i + 2 * e + 1] += f.y * p.res_s;
                            }
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const uint4 w = ptx::ld_shared_v4(base + (((part * 4 + i) ^ (srow & 7)) << 4));
                            const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&w);
#pragma unroll
                            for (int e = 0; e < 8; ++e) v[8 * i + e] += __bfloat162float(h[e]);
                        }
                    }
                }
            } else if (k > 0) {  // the group's previous TMA store must have read its staging tile
                if (elected) {
                    ptx::bulk_wait_read0();
                    ptx::mbar_arrive(&cfree[grp]);
                }
                if (!__all_sync(0xffffffffu, wait_bar(&cfree[grp], (k - 1) & 1, abort_flag, p.err))) break;
            }
            if (inner) {
                if constexpr (F8) {
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        uint32_t wq[4];
#pragma unroll
                        for (int k4 = 0; k4 < 4; ++k4) {
                            const float* f = v + 16 * i + 4 * k4;
                            const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(f[0] * p.out_inv, f[1] * p.out_inv),
                                                                         __NV_SATFINITE, __NV_E4M3);
                            const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(f[2] * p.out_inv, f[3] * p.out_inv),
                                                                         __NV_SATFINITE, __NV_E4M3);
                            wq[k4] = lo | (hi << 16);
                        }
                        ptx::st_shared_v4(base + part * 32 + 16 * i, wq[0], wq[1], wq[2], wq[3]);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int j = part * 4 + i;
                        ptx::st_shared_v4(base + ((j ^ (srow & 7)) << 4), pack_bf16(v[8 * i], v[8 * i + 1]),
                                          pack_bf16(v[8 * i + 2], v[8 * i + 3]), pack_bf16(v[8 * i + 4], v[8 * i + 5]),
                                          pack_bf16(v[8 * i + 6], v[8 * i + 7]));
                    }
                }
            }
            ptx::fence_proxy_async();
            ptx::mbar_arrive(&cwritten[grp]);
            if (lead_warp) {
                bool w_ok = true;
                if (lane == 0) w_ok = wait_bar(&cwritten[grp], k & 1, abort_flag, p.err);
                if (!__shfl_sync(0xffffffffu, (int)w_ok, 0)) break;
            }
            if (elected) {  // (a tile lying wholly past a cropped output stores nothing)
                if (strip * kKxnStrip < min(p.out_w, p.Wo) && oh < p.out_h)
                    ptx::tma_store_4d(&tmC, sCg, 0, strip * kKxnStrip, oh, g);
                ptx::bulk_commit();
                if (res && t + 2 < t_end) {  // the next residual once the store has read the tile
                    ptx::bulk_wait_read0();
                    load_res(t + 2);
                    ++n_res;
                }
            }
        }
        if (elected && n_res > k)  // a residual load that no tile consumed (stopped early): let it land
            wait_bar(&rfull[grp], (n_res - 1) & 1, abort_flag, p.err, false);
        if (elected) ptx::bulk_wait0();
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem_base, TMEM_COLS);
    }
}

// ------------------------------------------------------------------------------------------------
// Final decoder layer (3x3, 64 -> 12 channels, pixel shuffle, x^ = clamp(0.5 + o, 0, 1)) in scatter
// form.  With only 12 outputs, the gather form would stream every input pixel nine times through the
// tensor cores (one K=64 slice per tap) for an N of 16.  Instead each input pixel is multiplied ONCE by
// the 64 x 108 matrix of all (tap, channel) weights:
//     P[r][x][(ky, kx, c)] = sum_ci in[r][x][ci] w[c][ky][kx][ci]          (M = pixels, N = 108, K = 64)
//     o[y][x][c] = b[c] + sum_{ky, kx} P[y + ky - 1][x + kx - 1][(ky, kx, c)]  (zero outside the image)
// Tiles are input rows of a 120-pixel strip, taken in row order, so each input row is loaded once per
// strip.  Warp q of the 128 accumulator rows holds input pixels x0 + 30 q - 1 .. x0 + 30 q + 30 (one TMA
// box of 32 pixels each; the one-pixel halos overlap) and produces the outputs of its lanes 1..30, so
// the kx neighbours are warp shuffles.  Four TMEM buffers (128 columns each) hold the P rows of the
// three input rows an output row needs while the next one is computed.  Accumulator column of
// (ky, kx, c): 32 (c / 3) + 9 ky + 3 kx + c % 3, so epilogue column group k (warps 2+4k..5+4k) owns
// output channels 3k..3k+2 and reads one aligned 32-column block per P row.
// OUTK: 0 = every thread stores its outputs; 1 = uint8 frame rows through a staging block and TMA
// stores (three 240-byte boxes per output row pair of a strip); 2 = the same for float frames.
// ------------------------------------------------------------------------------------------------
constexpr int kFinStrip = 120;  // output pixels per strip

template <int OUTK>
__global__ void __launch_bounds__(kThreads, 1)
    conv_tc_final_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                         const __grid_constant__ CUtensorMap tmC, const TcArgs p) {
    constexpr int STAGES = 8, A_BYTES = 128 * 128, B_BYTES = 128 * 128, NACC = 4;
    constexpr uint32_t TMEM_COLS = 512;
    // staging: RG output rows (each three boxes of 240 elements) gathered before one barrier and their
    // TMA stores, so the epilogue warps meet once per RG rows (a barrier every row took half of the
    // layer's epilogue time; 4, 8, 16, 32 rows: 0.171, 0.163, 0.158, 0.157 ms per 1080p step)
    constexpr int RG = OUTK == 1 ? 16 : 8;
    constexpr int CSLOT = OUTK == 1 ? 1536 : OUTK == 2 ? 6144 : 0, C_BYTES = RG * CSLOT;
    // staging box stride in elements: every box starts 128-byte aligned (a TMA requirement on the
    // shared-memory address): 512 B for uint8, 480 floats = 1920 B for float
    constexpr int BOXE = OUTK == 1 ? 512 : 480;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sB = smem;
    uint8_t* sA = sB + B_BYTES;
    uint8_t* sC = sA + STAGES * A_BYTES;
    uint64_t* full = reinterpret_cast<uint64_t*>(sC + C_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;
    uint64_t* tempty = tfull + NACC;
    uint64_t* bfull = tempty + NACC;
    uint64_t* bfree = bfull + 1;
    uint64_t* drain = bfree + 1;
    uint64_t* cwritten = drain + 1;
    uint64_t* cfree = cwritten + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(cfree + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* sbias = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(tmem_slot + 2) + 15) & ~uintptr_t(15));
    const float* bias_all = stage_bias(p, sbias);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < NACC; ++a) {
            ptx::mbar_init(&tfull[a], 1);
            ptx::mbar_init(&tempty[a], 32 * kEpiWarps);
        }
        ptx::mbar_init(bfull, 1);
        ptx::mbar_init(bfree, 1);
        ptx::mbar_init(drain, 1);
        ptx::mbar_init(cwritten, 32 * kEpiWarps);
        ptx::mbar_init(cfree, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 1) ptx::tmem_alloc(tmem_slot, TMEM_COLS);
    if (warp == 0 && lane == 0) {
        ptx::prefetch_tmap(&tmA);
        ptx::prefetch_tmap(&tmB);
        if (OUTK) ptx::prefetch_tmap(&tmC);
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    // the set-up above (barriers, TMEM, biases, descriptor prefetch) may overlap the previous kernel's
    // tail; its outputs are read, and this kernel's written, only after it has completed
    pdl_trigger();
    pdl_wait();
    // work item t = (g * tiles_w + strip) * Ho + y (one output row of one strip); this CTA owns
    // [t_begin, t_end), cut into runs of one (g, strip)
    const int t_begin = (int)((long long)p.total_tiles * blockIdx.x / gridDim.x);
    const int t_end = (int)((long long)p.total_tiles * (blockIdx.x + 1) / gridDim.x);
    const int Ho = p.Ho;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer: one input row per P row
        if (lane == 0) {
            int it = 0, cur_g = -1, nb = 0;
            uint32_t bfree_par = 0, last_par[STAGES];
            bool used[STAGES];
#pragma unroll
            for (int s = 0; s < STAGES; ++s) { used[s] = false; last_par[s] = 0; }
            bool ok = true;
            for (int t = t_begin; t < t_end && ok;) {
                const int ya = t % Ho, r = t / Ho, strip = r % p.tiles_w, g = r / p.tiles_w;
                const int te = min(t_end, (r + 1) * Ho), yb = ya + (te - t) - 1;
                if (g != cur_g) {
                    if (cur_g >= 0) {  // the MMAs that read the previous weights must be complete
                        if (!wait_bar(bfree, bfree_par, abort_flag, p.err)) break;
                        bfree_par ^= 1;
                    }
                    ptx::mbar_arrive_expect_tx(bfull, B_BYTES);
                    ptx::tma_load_3d(sB, &tmB, bfull, 0, 0, g);
                    cur_g = g;
                    ++nb;
                }
                const int r0 = max(ya - 1, 0), r1 = min(yb + 1, Ho - 1), ag = p.a_grouped ? g : 0;
                for (int row = r0; row <= r1; ++row, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1;
                    if (!wait_bar(&empty[s], ph ^ 1, abort_flag, p.err)) { ok = false; break; }
                    ptx::mbar_arrive_expect_tx(&full[s], A_BYTES);
                    for (int q = 0; q < 4; ++q)
                        ptx::tma_load_4d(sA + s * A_BYTES + q * 4096, &tmA, &full[s], 0,
                                         strip * kFinStrip + 30 * q - 1, row, ag);
                    used[s] = true;
                    last_par[s] = ph;
                }
                t = te;
            }
#pragma unroll
            for (int s = 0; s < STAGES; ++s)
                if (used[s]) wait_bar(&full[s], last_par[s], abort_flag, p.err, false);
            if (nb) wait_bar(bfull, (nb - 1) & 1, abort_flag, p.err, false);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer: P row = 4 MMAs (K = 64)
        if (lane == 0) {
            constexpr uint32_t idesc = ptx::idesc_bf16(128);
            int it = 0, pr = 0, cur_g = -1;
            uint32_t bfull_par = 0;
            bool ok = true;
            for (int t = t_begin; t < t_end && ok;) {
                const int ya = t % Ho, r = t / Ho, g = r / p.tiles_w;
                const int te = min(t_end, (r + 1) * Ho), yb = ya + (te - t) - 1;
                if (g != cur_g) {
                    if (cur_g >= 0) ptx::mma_commit(bfree);
                    if (!wait_bar(bfull, bfull_par, abort_flag, p.err)) break;
                    bfull_par ^= 1;
                    ptx::tc_fence_after();
                    cur_g = g;
                }
                const int r0 = max(ya - 1, 0), r1 = min(yb + 1, Ho - 1);
                for (int row = r0; row <= r1; ++row, ++it, ++pr) {
                    const int acc = pr % NACC, use = pr / NACC;
                    if (!wait_bar(&tempty[acc], (use & 1) ^ 1, abort_flag, p.err)) { ok = false; break; }
                    const int s = it % STAGES;
                    if (!wait_bar(&full[s], (it / STAGES) & 1, abort_flag, p.err)) { ok = false; break; }
                    ptx::tc_fence_after();
                    const uint32_t a0 = ptx::smem_u32(sA + s * A_BYTES), b0 = ptx::smem_u32(sB);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        ptx::mma_f16(tmem_base + acc * 128, ptx::sdesc_sw128(a0 + kk * 32),
                                     ptx::sdesc_sw128(b0 + kk * 32), idesc, kk != 0);
                    ptx::mma_commit(&empty[s]);
                    ptx::mma_commit(&tfull[acc]);
                }
                t = te;
            }
            ptx::mma_commit(drain);
            wait_bar(drain, 0, abort_flag, p.err, false);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue: one output row at a time
        // Each P row is read from TMEM once, right when it is complete, and its TMEM buffer released at
        // once: P row j holds the ky = 0 taps of output row j + 1, ky = 1 of row j and ky = 2 of row j - 1,
        // so three running tap sums (SA: output j - 1, SB: j, SC: j + 1) take its 27 values, and output
        // j - 1 is finished after row j (taps added in row order, ky = 0, 1, 2).
        const int q = warp & 3, k = (warp - 2) >> 2;
        const bool elected = OUTK != 0 && warp == 2 && lane == 0;
        const uint32_t lane_base = tmem_base + ((uint32_t)(q * 32) << 16) + 32 * k;
        int pr = 0, waited = 0, o = 0, pc = 0, y0 = 0;  // o: rows in the open group, pc: groups stored
        bool ok = true;
        for (int t = t_begin; t < t_end && ok;) {
            const int ya = t % Ho, r = t / Ho, strip = r % p.tiles_w, g = r / p.tiles_w;
            const int te = min(t_end, (r + 1) * Ho), yb = ya + (te - t) - 1;
            const int r0 = max(ya - 1, 0), r1 = min(yb + 1, Ho - 1);
            const float* bias = bias_all + (size_t)g * p.b_gs + 3 * k;
            const float b0 = bias[0], b1 = bias[1], b2 = bias[2];
            const int xo = strip * kFinStrip + 30 * q + lane - 1;
            const bool xvalid = lane >= 1 && lane <= 30 && xo < p.Wo;
            // this thread's three staging elements (the same for every row): element xb of the strip's
            // 720-element output row pair lies in box xb / 240
            int se[3];
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                const int c = 3 * k + cc, dy = (c >> 1) & 1;
                const int xb = (2 * (30 * q + lane - 1) + (c & 1)) * 3 + (c >> 2);
                se[cc] = (xb / 240) * BOXE + dy * 240 + xb % 240;
            }
            // output row y from its nine tap sums S (kx-major within each channel's 9)
            auto emit = [&](int y, const float* S, bool last) -> bool {
                float outv[3];
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    const float left = __shfl_up_sync(0xffffffffu, S[cc], 1);        // kx = 0 of pixel x - 1
                    const float right = __shfl_down_sync(0xffffffffu, S[6 + cc], 1);  // kx = 2 of pixel x + 1
                    const float bb = cc == 0 ? b0 : cc == 1 ? b1 : b2;
                    outv[cc] = fminf(fmaxf(0.5f + (bb + left + S[3 + cc] + right), 0.0f), 1.0f);
                }
                if constexpr (OUTK == 0) {
                    if (xvalid) {
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc) {
                            const int c = 3 * k + cc, ch = c >> 2, oy = 2 * y + ((c >> 1) & 1), ox = 2 * xo + (c & 1);
                            if (oy >= p.out_h || ox >= p.out_w) continue;
                            const size_t off = (size_t)g * p.out_gs + ((size_t)oy * p.out_w + ox) * 3 + ch;
                            if (p.mode == OUT_PS_FINAL_F32) reinterpret_cast<float*>(p.out)[off] = outv[cc];
                            else reinterpret_cast<uint8_t*>(p.out)[off] = (uint8_t)rintf(outv[cc] * 255.0f);
                        }
                    }
                } else {
                    if (o == 0) {  // a new group: the previous group's TMA stores must have read the staging
                        if (pc > 0) {
                            if (elected) {
                                ptx::bulk_wait_read0();
                                ptx::mbar_arrive(cfree);
                            }
                            if (!__all_sync(0xffffffffu, wait_bar(cfree, (pc - 1) & 1, abort_flag, p.err))) return false;
                        }
                        y0 = y;  // (a group's rows are consecutive rows of one run)
                    }
                    uint8_t* slot = sC + o * CSLOT;
                    if (xvalid) {
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc) {
                            if constexpr (OUTK == 1) slot[se[cc]] = (uint8_t)rintf(outv[cc] * 255.0f);
                            else reinterpret_cast<float*>(slot)[se[cc]] = outv[cc];
                        }
                    }
                    ++o;
                    if (o == RG || last) {  // the group is complete: one barrier, then its rows' stores
                        ptx::fence_proxy_async();
                        ptx::mbar_arrive(cwritten);
                        if (warp == 2) {
                            bool w_ok = true;
                            if (lane == 0) w_ok = wait_bar(cwritten, pc & 1, abort_flag, p.err);
                            if (!__shfl_sync(0xffffffffu, (int)w_ok, 0)) return false;
                        }
                        if (elected) {
                            for (int h = 0; h < o; ++h)
#pragma unroll
                                for (int b = 0; b < 3; ++b)
                                    ptx::tma_store_3d(&tmC, sC + h * CSLOT + b * BOXE * (OUTK == 1 ? 1 : 4),
                                                      strip * 2 * kFinStrip * 3 + b * 240, 2 * (y0 + h), g);
                            ptx::bulk_commit();
                        }
                        ++pc;
                        o = 0;
                    }
                }
                return true;
            };
            float SA[9], SB[9], SC[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) { SA[i] = 0.f; SB[i] = 0.f; }
            for (int j = r0; j <= r1; ++j) {
                while (waited <= pr + (j - r0)) {  // P row j is in TMEM
                    if (!__all_sync(0xffffffffu, wait_bar(&tfull[waited % NACC], (waited / NACC) & 1, abort_flag,
                                                          p.err))) { ok = false; break; }
                    ++waited;
                }
                if (!ok) break;
                ptx::tc_fence_after();
                float v[32];
                tmem_ld32(lane_base + ((pr + j - r0) % NACC) * 128, v);
                ptx::tc_fence_before();
                ptx::mbar_arrive(&tempty[(pr + j - r0) % NACC]);  // the row is in registers
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    SA[i] += v[18 + i];
                    SB[i] += v[9 + i];
                    SC[i] = v[i];
                }
                if (j - 1 >= ya && !emit(j - 1, SA, j - 1 == yb)) { ok = false; break; }
#pragma unroll
                for (int i = 0; i < 9; ++i) { SA[i] = SB[i]; SB[i] = SC[i]; }
            }
            if (!ok) break;
            if (r1 == yb && !emit(yb, SA, true)) { ok = false; break; }  // the image's last row has no row below
            pr += r1 - r0 + 1;
            t = te;
        }
        if (elected) ptx::bulk_wait0();
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem_base, TMEM_COLS);
    }
}

// ------------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------------
// The driver's tensor-map encoder, resolved through the runtime so that the library itself does not
// link libcuda (it must load on machines without a GPU driver).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

static bool encode_map(CUtensorMap* m, const void* base, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
                       const cuuint32_t* box, CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                       CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B) {
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    CUresult r = enc(m, dt, rank, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool encode_f32_map_sw128(void* map, const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
                          const uint32_t* box) {
    cuuint64_t d[5], st[4];
    cuuint32_t b[5];
    if (rank < 1 || rank > 5) return false;
    for (int i = 0; i < rank; ++i) { d[i] = dims[i]; b[i] = box[i]; }
    for (int i = 0; i + 1 < rank; ++i) st[i] = strides[i];
    return encode_map(static_cast<CUtensorMap*>(map), base, rank, d, st, b, CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                      CU_TENSOR_MAP_SWIZZLE_128B);
}

// Frames [N][H][row_bytes] uint8 as a 3D tensor map (bytes, rows, frames) with box (box_x, box_y, N), no
// swizzle; map points at a 64-byte aligned CUtensorMap.
bool encode_frames_map(void* map, const void* frames, int N, int H, int row_bytes, int box_x, int box_y) {
    const cuuint64_t dims[3] = {(cuuint64_t)row_bytes, (cuuint64_t)H, (cuuint64_t)N};
    const cuuint64_t strides[2] = {(cuuint64_t)row_bytes, (cuuint64_t)H * row_bytes};
    const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, (cuuint32_t)N};
    return encode_map(static_cast<CUtensorMap*>(map), frames, 3, dims, strides, box, CU_TENSOR_MAP_DATA_TYPE_UINT8,
                      CU_TENSOR_MAP_SWIZZLE_NONE);
}

// Output tile TW x TH = 128 pixels with the least padding; with th_divides, TH must divide Ho.
// rm: sub-tiles stacked vertically in a tile (two sub-tiles, SM pairs), so a tile covers rm * TH rows
static void pick_tile(int Ho, int Wo, int* TW, int* TH, bool th_divides = false, int rm = 1) {
    long long best = -1;
    for (int tw = 128; tw >= 8; tw >>= 1) {
        const int th = 128 / tw;
        if (th_divides && Ho % th != 0) continue;
        const long long cost = (long long)((Wo + tw - 1) / tw) * tw * ((Ho + th * rm - 1) / (th * rm)) * th * rm;
        if (best < 0 || cost < best) { best = cost; *TW = tw; *TH = th; }
    }
}

template <int BN, int STAGES, bool STAGED, int OP = OP_BF16, bool KM = false, int MT = 1, bool PAIR = false,
          bool O8 = false>
static cudaError_t launch_bn(const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& c, const TcArgs& args,
                             cudaStream_t s) {
    constexpr int ROWB = OP == OP_BF16 ? 128 : 64;
    constexpr int EG = MT == 2 ? 1 : epi_groups(BN);
    constexpr int kSmem = STAGES * (128 * MT * ROWB + (PAIR ? BN / 2 : BN) * ROWB) +
                          (STAGED ? (BN / 64) * 128 * (O8 ? 64 : 128) * EG : 0) + kSmemExtra;
    static_assert(kSmem <= 227 * 1024, "shared memory per CTA");
    const int smem = kSmem;
    const void* fn = (const void*)conv_tc_kernel<BN, STAGES, STAGED, OP, KM, MT, PAIR, O8>;
    cudaError_t e = smem_optin(fn, smem);
    if (e != cudaSuccess) return e;
    if constexpr (PAIR) {
        // one cluster of two CTAs per pair of SMs that can hold them at once, each cluster a tile at a time
        const int pairs = max_pairs(fn, smem, kThreads);
        if (pairs < 1) return cudaErrorInvalidConfiguration;
        const int grid = 2 * (args.total_tiles < pairs ? args.total_tiles : pairs);
        return launch_pdl_pair(conv_tc_kernel<BN, STAGES, STAGED, OP, KM, MT, PAIR, O8>, dim3(grid), dim3(kThreads),
                               smem, s, a, b, c, args);
    }
    const int sms = sm_count();
    const int grid = args.total_tiles < sms ? args.total_tiles : sms;
    return launch_pdl(conv_tc_kernel<BN, STAGES, STAGED, OP, KM, MT, PAIR, O8>, dim3(grid), dim3(kThreads), smem, s, a,
                      b, c, args);
}

// d.in: bf16 NHWC [groups or 1][H][W][Cin] (Cin a multiple of 64); d.w: bf16 [groups][cout_pad][k*k*Cin];
// returns a CUDA error or cudaSuccess; UFVC argument problems return cudaErrorInvalidValue.
template <int BN, int STAGES, int OUTK, bool F8 = false>
static cudaError_t launch_halo(const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& c, const TcArgs& args,
                               cudaStream_t s) {
    constexpr int C_BYTES = OUTK == 1 ? halo_groups(BN) * 128 * BN * 2 : OUTK == 2 ? halo_groups(BN) * 128 * BN : 0;
    constexpr int kSmem = 9 * BN * (F8 ? 64 : 128) + STAGES * 3 * (F8 ? kHaloRowBytes8 : kHaloRowBytes) + C_BYTES +
                          kSmemExtra;
    static_assert(kSmem <= 227 * 1024, "shared memory per CTA");
    const int smem = kSmem;
    cudaError_t e = smem_optin((const void*)conv_tc_halo_kernel<BN, STAGES, OUTK, F8>, smem);
    if (e != cudaSuccess) return e;
    const int sms = sm_count();
    const int grid = args.total_tiles < sms ? args.total_tiles : sms;
    return launch_pdl(conv_tc_halo_kernel<BN, STAGES, OUTK, F8>, dim3(grid), dim3(kThreads), smem, s, a, b, c, args);
}

template <int STAGES, bool F8 = false>
static cudaError_t launch_kxn(const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& c, const CUtensorMap& r,
                              const TcArgs& args, cudaStream_t s) {
    constexpr int RB = F8 ? 64 : 128;
    constexpr int kSmem = 9 * 64 * RB + STAGES * 3 * 4 * 32 * RB + 2 * (F8 ? 8192 : 16384) + kSmemExtra;
    static_assert(kSmem <= 227 * 1024, "shared memory per CTA");
    cudaError_t e = smem_optin((const void*)conv_tc_kxn_kernel<STAGES, F8>, kSmem);
    if (e != cudaSuccess) return e;
    const int sms = sm_count();
    const int grid = args.total_tiles < sms ? args.total_tiles : sms;
    return launch_pdl(conv_tc_kxn_kernel<STAGES, F8>, dim3(grid), dim3(kThreads), kSmem, s, a, b, c, r, args);
}

template <int OUTK>
static cudaError_t launch_final(const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& c, const TcArgs& args,
                                cudaStream_t s) {
    constexpr int kSmem = 128 * 128 + 8 * 128 * 128 + (OUTK == 1 ? 16 * 1536 : OUTK == 2 ? 8 * 6144 : 0) + kSmemExtra;
    static_assert(kSmem <= 227 * 1024, "shared memory per CTA");
    cudaError_t e = smem_optin((const void*)conv_tc_final_kernel<OUTK>, kSmem);
    if (e != cudaSuccess) return e;
    const int sms = sm_count();
    const int grid = args.total_tiles < sms ? args.total_tiles : sms;
    return launch_pdl(conv_tc_final_kernel<OUTK>, dim3(grid), dim3(kThreads), kSmem, s, a, b, c, args);
}

// The final decoder layer in scatter form (d.wsc: bf16 [groups][128][64], row 32 (c / 3) + 9 ky + 3 kx
// + c % 3 = tap (ky, kx) of output channel c, other rows zero).
static cudaError_t launch_conv_final(const ConvDesc& d, cudaStream_t s) {
    const int Ho = d.H, Wo = d.W;
    TcArgs a{};
    a.ksplit = 1;
    a.Ho = Ho; a.Wo = Wo;
    a.TW = kFinStrip; a.TH = 1;
    a.tiles_w = (Wo + kFinStrip - 1) / kFinStrip;
    a.tiles_h = Ho;
    a.n_tiles = 1;
    a.groups = d.groups;
    a.total_tiles = a.tiles_w * Ho * d.groups;
    a.k = 3; a.pad = 1; a.stride = 1; a.a_grouped = d.in_gs != 0;
    a.bias = d.b; a.b_gs = (int)d.b_gs; a.Cout = d.Cout;
    a.mode = d.mode; a.act = 0;
    a.out = d.out; a.out_gs = d.out_gs; a.out_h = d.out_h; a.out_w = d.out_w; a.out_c = 3;
    a.err = d.err;
    const cuuint64_t esz = 2;
    CUtensorMap ma, mb, mc;
    {
        const int G = a.a_grouped ? d.groups : 1;
        cuuint64_t dims[4] = {64, (cuuint64_t)Wo, (cuuint64_t)Ho, (cuuint64_t)G};
        cuuint64_t str[3] = {64 * esz, (cuuint64_t)Wo * 64 * esz,
                             a.a_grouped ? (cuuint64_t)d.in_gs * esz : (cuuint64_t)Ho * Wo * 64 * esz};
        cuuint32_t box[4] = {64, 32, 1, 1};
        if (!encode_map(&ma, d.in, 4, dims, str, box)) return cudaErrorInvalidValue;
    }
    {
        cuuint64_t dims[3] = {64, 128, (cuuint64_t)d.groups};
        cuuint64_t str[2] = {64 * esz, 128 * 64 * esz};
        cuuint32_t box[3] = {64, 128, 1};
        if (!encode_map(&mb, d.wsc, 3, dims, str, box)) return cudaErrorInvalidValue;
    }
    const bool f32 = d.mode == OUT_PS_FINAL_F32;
    const size_t es = f32 ? 4 : 1;
    const bool contiguous = d.groups == 1 || d.out_gs == (long long)d.out_h * d.out_w * 3;
    const bool staged = contiguous && (d.out_w * 3 * es) % 16 == 0;
    mc = mb;
    if (staged) {
        cuuint64_t dims[3] = {(cuuint64_t)d.out_w * 3, (cuuint64_t)d.out_h, (cuuint64_t)d.groups};
        cuuint64_t str[2] = {(cuuint64_t)d.out_w * 3 * es, (cuuint64_t)d.out_h * d.out_w * 3 * es};
        cuuint32_t box[3] = {240, 2, 1};
        if (!encode_map(&mc, d.out, 3, dims, str, box,
                        f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT8,
                        CU_TENSOR_MAP_SWIZZLE_NONE))
            return cudaErrorInvalidValue;
        return f32 ? launch_final<2>(ma, mb, mc, a, s) : launch_final<1>(ma, mb, mc, a, s);
    }
    return launch_final<0>(ma, mb, mc, a, s);
}

// Split K for bf16 NHWC layers with few 128-pixel tiles (the hyper-analysis H1, H2 on a 1080p latent: 16
// and 4 tiles, each running 36 or 18 K steps one after another on a single SM): as many K ranges as fill
// about one CTA per SM, each of at least four 64-channel steps.  1 = no split.
int conv_tc_ksplit(const ConvDesc& d) {
    if (d.w8 || d.kmask || d.mode != OUT_NHWC || d.res) return 1;
    if (d.Cin % 64 != 0 || (d.stride != 1 && d.stride != 2) || d.k % 2 == 0 || d.Cout % 4 != 0) return 1;
    if (d.stride == 1 && d.k == 3 && d.Cin == 64 && d.cout_pad <= 64) return 1;  // the resident-weight kernels
    const int out_c = d.out_c_stride ? d.out_c_stride : d.Cout;
    if (out_c % 4 != 0 || d.out_gs % 4 != 0 || (reinterpret_cast<uintptr_t>(d.out) & 15) != 0) return 1;
    const int pad = d.k / 2;
    const long long Ho = (d.H + 2 * pad - d.k) / d.stride + 1, Wo = (d.W + 2 * pad - d.k) / d.stride + 1;
    const int sms = sm_count();
    int BN = d.cout_pad >= 256 ? 256 : d.cout_pad;
    long long tiles = (Ho * Wo + 127) / 128 * (d.cout_pad / BN) * d.groups;
    if (BN == 256 && tiles < sms) tiles *= 2;  // (N tiles of 128, as launch_conv_tc picks them)
    const int ksteps = d.k * d.k * (d.Cin / 64);
    if (tiles * 4 > sms || ksteps < 8) return 1;
    long long ks = sms / tiles;
    if (ks > ksteps / 4) ks = ksteps / 4;
    return ks >= 2 ? (int)ks : 1;
}

size_t conv_tc_workspace(const ConvDesc& d) {
    const int ks = conv_tc_ksplit(d);
    if (ks < 2) return 0;
    const int pad = d.k / 2;
    const size_t Ho = (d.H + 2 * pad - d.k) / d.stride + 1, Wo = (d.W + 2 * pad - d.k) / d.stride + 1;
    return (size_t)ks * d.groups * Ho * Wo * d.cout_pad;
}

// The split layers' finish: out = act(bias + (((range 0) + range 1) + ...)), four channels per thread
__global__ void conv_tc_split_reduce_kernel(const TcArgs p) {
    pdl_trigger();
    pdl_wait();
    const int C4 = p.Cout >> 2;
    const long long per_g = (long long)p.Ho * p.Wo * C4, total = per_g * p.groups;
    const size_t slice = (size_t)p.groups * p.Ho * p.Wo * p.ws_c;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(i / per_g);
        const long long rem = i - (long long)g * per_g;
        const int m = (int)(rem / C4), c = (int)(rem - (long long)m * C4) * 4;
        const int oh = m / p.Wo, ow = m - oh * p.Wo;
        if (oh >= p.out_h || ow >= p.out_w) continue;
        const float* src = p.ws + ((size_t)g * p.Ho * p.Wo + m) * p.ws_c + c;
        float4 v = *reinterpret_cast<const float4*>(src);
        for (int kr = 1; kr < p.ksplit; ++kr) {
            const float4 u = *reinterpret_cast<const float4*>(src + kr * slice);
            v.x += u.x; v.y += u.y; v.z += u.z; v.w += u.w;
        }
        const float* b = p.bias + (size_t)g * p.b_gs + c;
        v.x += b[0]; v.y += b[1]; v.z += b[2]; v.w += b[3];
        if (p.act) { gelu_tc2(v.x, v.y); gelu_tc2(v.z, v.w); }
        const size_t o = (size_t)g * p.out_gs + ((size_t)oh * p.out_w + ow) * p.out_c + c;
        if (p.out_f32) *reinterpret_cast<float4*>(static_cast<float*>(p.out) + o) = v;
        else *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(p.out) + o) = make_uint2(pack_bf16(v.x, v.y), pack_bf16(v.z, v.w));
    }
}

cudaError_t launch_conv_tc(const ConvDesc& d, cudaStream_t s, int* nl) {
    int nl_ = 0;
    if (!nl) nl = &nl_;
    if (d.wsc && (d.mode == OUT_PS_FINAL_U8 || d.mode == OUT_PS_FINAL_F32) && d.k == 3 && d.stride == 1 &&
        d.Cin == 64 && d.Cout == 12)
        return launch_conv_final(d, s);
    const bool c32 = d.Cin == 32 && d.w8 == nullptr;  // one 32-channel stage per tap (bf16)
    if ((d.Cin % 64 != 0 && !c32) || (d.stride != 1 && d.stride != 2) || (d.stride == 2 && ((d.H | d.W) & 1)))
        return cudaErrorInvalidValue;
    const int pad = d.k / 2;
    // even k (the 2x2 form of a stride-2 layer on space-to-depth input): taps at offsets -k/2 .. k/2 - 1,
    // the output has the input's size
    const int Ho = (d.H + 2 * pad - d.k) / d.stride + 1 - (d.k % 2 == 0 ? 1 : 0);
    const int Wo = (d.W + 2 * pad - d.k) / d.stride + 1 - (d.k % 2 == 0 ? 1 : 0);
    if (d.k % 2 == 0 && d.stride != 1) return cudaErrorInvalidValue;
    int BN = d.cout_pad >= 256 ? 256 : d.cout_pad;
    if (d.cout_pad % BN != 0 || !(BN == 16 || BN == 64 || BN == 128 || BN == 192 || BN == 256))
        return cudaErrorInvalidValue;
    // stride-1 3x3 layers with 64 input channels and at most 64 output channels: resident weights,
    // three input rows per 128-pixel strip (wider layers keep one N tile on the streaming kernel, which
    // re-reads the input less than several N tiles would)
    const bool f8 = d.w8 != nullptr;  // E4M3 operands
    // E4M3 layers of this shape (the decoders' R2) take the resident-weight kernel with E4M3 NHWC outputs
    // staged for TMA stores; other E4M3 layers the streaming kernel with the per-thread epilogue
    const int out_c0 = (d.mode == OUT_NHWC && d.out_c_stride) ? d.out_c_stride : d.Cout;
    const bool halo8 = f8 && d.stride == 1 && d.k == 3 && d.Cin == 64 && d.cout_pad == 64 && d.mode == OUT_NHWC &&
                       !d.out_f32 && d.out_inv != 0.f && out_c0 % 16 == 0 && d.out_gs % 16 == 0;
    const bool halo = (!f8 && !c32 && d.stride == 1 && d.k == 3 && d.Cin == 64 && (d.cout_pad == 16 || d.cout_pad == 64)) ||
                      halo8;
    if (halo) BN = d.cout_pad;
    // NHWC layers with fewer 128-pixel tiles than SMs at N = 256 (the encoder's A4 on a 1080p latent: 64
    // tiles) take N tiles of 128, so that twice as many SMs share the work
    if (BN == 256 && d.mode == OUT_NHWC && ((long long)Ho * Wo + 127) / 128 * (d.cout_pad / 256) * d.groups < sm_count())
        BN = 128;
    // bf16 64 -> 64 layers with staged NHWC outputs: the three horizontal taps in N (conv_tc_kxn_kernel)
    // (E4M3: the layers the resident-weight E4M3 kernel takes, with 64 outputs)
    const bool kxn = halo && d.Cout == 64 && d.cout_pad == 64 && d.mode == OUT_NHWC && !d.out_f32 &&
                     (f8 ? halo8 : out_c0 % 8 == 0 && d.out_gs % 8 == 0);
    // staged epilogue (bf16 output through shared memory and TMA stores): NHWC, or a sub-pixel-major
    // pixel shuffle written whole (no crop) with 64-channel runs; grouped pixel-shuffle outputs are
    // stored through one map whose row dimension spans all groups, so tiles must not cross a group's
    // last row (TH divides Ho)
    const int Cq = d.Cout / 4;
    // (E4M3 operands: E4M3 outputs are staged as codes, the pixel-shuffle layer feeding the final layer as
    // bf16; both with 16-byte aligned rows)
    const bool o8 = f8 && d.out_inv != 0.f;
    const bool ps_stage = !halo && !c32 && BN >= 64 && d.mode == OUT_PS && d.ps_major && Cq % 64 == 0 &&
                          d.out_h == 2 * Ho && d.out_w == 2 * Wo &&
                          (d.groups == 1 || d.out_gs == 4LL * Ho * Wo * Cq);
    const int out_c = (d.mode == OUT_NHWC && d.out_c_stride) ? d.out_c_stride : d.Cout;
    // (split-K layers write raw range sums instead, finished by conv_tc_split_reduce_kernel)
    int ksplit = conv_tc_ksplit(d);
    if (ksplit > 1 && (!d.tc_ws || d.tc_ws_cap < conv_tc_workspace(d))) ksplit = 1;
    const bool nhwc_stage = ksplit == 1 && !halo && BN >= 64 && d.mode == OUT_NHWC && !d.out_f32 &&
                            (f8 ? o8 && out_c % 16 == 0 && d.out_gs % 16 == 0 : out_c % 8 == 0 && d.out_gs % 8 == 0);
    const bool staged = ps_stage || nhwc_stage;
    TcArgs a{};
    a.ksplit = 1;
    if (halo) { a.TW = kxn ? kKxnStrip : 128; a.TH = 1; } else pick_tile(Ho, Wo, &a.TW, &a.TH, ps_stage && d.groups > 1);
    // two stacked 128-pixel sub-tiles per tile (sharing each stage's weights): the 128-output layers with
    // NHWC bf16 outputs that keep at least two such tiles per SM (decoder R1, encoder A2 at video sizes;
    // small layers such as H1 or the mean network would leave SMs idle)
    const long long pairs = (long long)((Wo + a.TW - 1) / a.TW) * ((Ho + 2 * a.TH - 1) / (2 * a.TH)) *
                            (d.cout_pad / 128) * d.groups;
    // (E4M3 operands too, with E4M3 outputs: the FP8 decoders' R1)
    const int MT = ((!f8 || o8) && !c32 && !halo && nhwc_stage && BN == 128 && d.kmask == 0 && pairs >= 2 * 148) ? 2 : 1;
    // CTA pairs (one M = 256 MMA over two SMs, each loading half of the weights): the staged BN = 256
    // layers (the decoders' pixel-shuffle layers D0, U1, U2)
    // (and the two-sub-tile 128-output layers with at least four waves of pair tiles: each SM then lands its
    // two 128-pixel A tiles and half of the weight rows per stage, 40 KB instead of 48 KB)
    // (E4M3 operands: only the layer with bf16 outputs, U2; with E4M3 outputs D0 and U1 ran 2-6 % slower on
    // pairs than on single SMs)
    const bool pair = d.pairs && !c32 && !halo && staged && d.kmask == 0 &&
                      ((BN == 256 && !o8) || (!f8 && BN == 128 && MT == 2 && pairs >= 4 * 148));
    const int SUB = pair ? 2 * MT : MT;  // 128-pixel sub-tiles per tile
    if (SUB > 1) pick_tile(Ho, Wo, &a.TW, &a.TH, ps_stage && d.groups > 1, SUB);  // the stack's rows fit Ho
    a.Ho = Ho; a.Wo = Wo;
    a.tiles_w = (Wo + a.TW - 1) / a.TW;
    a.tiles_h = (Ho + a.TH * SUB - 1) / (a.TH * SUB);
    a.n_tiles = d.cout_pad / BN;
    a.groups = d.groups;
    a.total_tiles = a.tiles_w * a.tiles_h * a.n_tiles * d.groups;
    if (ksplit > 1) {  // work units: (tile, K range)
        a.ksplit = ksplit;
        a.ws = d.tc_ws;
        a.ws_c = d.cout_pad;
        a.total_tiles *= ksplit;
    }
    a.cin_chunks = c32 ? 1 : d.Cin / 64;
    a.ksteps = d.k * d.k * a.cin_chunks;
    if (d.kmask && a.ksteps > 64) return cudaErrorInvalidValue;  // the skip mask has one bit per K step
    // steps skipped by kmask have all-zero weights, so a kernel that runs every step computes the same
    // result: only the staged BF16 N = 64 kernel (the space-to-depth first layer) reads the mask
    a.kmask = d.kmask ? d.kmask : ~0ull;
    a.k = d.k; a.pad = pad; a.stride = d.stride; a.a_grouped = d.in_gs != 0;
    a.bias = d.btc ? d.btc : d.b; a.b_gs = (int)d.b_gs; a.Cout = d.Cout;
    a.ps_major = d.mode == OUT_PS && d.ps_major;
    a.mode = d.mode; a.act = d.act; a.out_f32 = d.out_f32;
    a.out = d.out; a.out_gs = d.out_gs; a.out_h = d.out_h; a.out_w = d.out_w;
    a.out_c = (d.mode == OUT_NHWC) ? d.Cout : d.Cout / 4;
    if (d.mode == OUT_NHWC && d.out_c_stride) a.out_c = d.out_c_stride;
    a.vec_out = d.Cout % 32 == 0 && a.out_c % 16 == 0 && d.out_gs % 16 == 0 &&
                (reinterpret_cast<uintptr_t>(d.out) & 15) == 0;
    if (d.res && d.mode == OUT_NHWC && !(a.vec_out && d.res_gs % 16 == 0 && (reinterpret_cast<uintptr_t>(d.res) & 15) == 0))
        return cudaErrorInvalidValue;  // residuals are read 16 bytes at a time
    a.res = reinterpret_cast<const __nv_bfloat16*>(d.res); a.res_gs = d.res_gs;
    a.err = d.err;
    a.c_rank = ps_stage ? 5 : 4;
    if (f8) {
        a.res = nullptr;
        a.res8 = reinterpret_cast<const uint8_t*>(d.res);
        a.res_s = d.res_s;
        a.cscale = d.cscale;
        a.out_inv = d.out_inv;
    }

    CUtensorMap ma, mb;
    const cuuint64_t esz = f8 ? 1 : 2;
    const CUtensorMapDataType dt = f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const CUtensorMapSwizzle swz = (f8 || c32) ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
    const cuuint32_t boxc = c32 ? 32 : 64;  // channels of a stage
    bool ok;
    if (d.stride == 1) {
        const int G = a.a_grouped ? d.groups : 1;
        cuuint64_t dims[4] = {(cuuint64_t)d.Cin, (cuuint64_t)d.W, (cuuint64_t)d.H, (cuuint64_t)G};
        cuuint64_t str[3] = {d.Cin * esz, (cuuint64_t)d.W * d.Cin * esz, (cuuint64_t)d.H * d.W * d.Cin * esz};
        if (a.a_grouped) str[2] = (cuuint64_t)d.in_gs * esz;
        cuuint32_t box[4] = {boxc, (cuuint32_t)a.TW, (cuuint32_t)(a.TH * MT), 1};
        if (halo) { box[1] = kxn ? 32 : 130; box[2] = 1; }
        ok = encode_map(&ma, d.in, 4, dims, str, box, dt, swz);
    } else {
        cuuint64_t dims[5] = {(cuuint64_t)d.Cin, 2, (cuuint64_t)d.W / 2, 2, (cuuint64_t)d.H / 2};
        cuuint64_t str[4] = {d.Cin * esz, 2 * d.Cin * esz, (cuuint64_t)d.W * d.Cin * esz,
                             2ull * d.W * d.Cin * esz};
        cuuint32_t box[5] = {boxc, 1, (cuuint32_t)a.TW, 1, (cuuint32_t)(a.TH * MT)};
        ok = encode_map(&ma, d.in, 5, dims, str, box, dt, swz);
    }
    if (!ok) return cudaErrorInvalidValue;
    {
        const cuuint64_t K = (cuuint64_t)d.k * d.k * d.Cin;
        cuuint64_t dims[3] = {K, (cuuint64_t)d.cout_pad, (cuuint64_t)d.groups};
        cuuint64_t str[2] = {K * esz, K * d.cout_pad * esz};
        cuuint32_t box[3] = {boxc, (cuuint32_t)(pair ? BN / 2 : BN), 1};  // a pair's CTA loads half the rows
        if (!encode_map(&mb, f8 ? d.w8 : d.wtc, 3, dims, str, box, dt, swz)) return cudaErrorInvalidValue;
    }
    CUtensorMap mc = mb;  // unused by the unstaged kernels
    if (halo8) {
        // E4M3 codes [G][out_h][out_w][out_c], positions beyond Ho x Wo dropped; 64-byte boxes, no swizzle
        const int Hd = d.out_h < Ho ? d.out_h : Ho, Wd = d.out_w < Wo ? d.out_w : Wo;
        cuuint64_t dims[4] = {(cuuint64_t)out_c, (cuuint64_t)Wd, (cuuint64_t)Hd, (cuuint64_t)d.groups};
        cuuint64_t str[3] = {(cuuint64_t)out_c, (cuuint64_t)d.out_w * out_c,
                             d.groups > 1 ? (cuuint64_t)d.out_gs : (cuuint64_t)d.out_h * d.out_w * out_c};
        cuuint32_t box[4] = {64, (cuuint32_t)(kxn ? kKxnStrip : 128), 1, 1};
        if (!encode_map(&mc, d.out, 4, dims, str, box, CU_TENSOR_MAP_DATA_TYPE_UINT8, CU_TENSOR_MAP_SWIZZLE_NONE))
            return cudaErrorInvalidValue;
        if (!kxn) return launch_halo<64, 4, 2, true>(ma, mb, mc, a, s);
        CUtensorMap mr = mc;  // the E4M3 residual, loaded into the staging tile
        if (a.res8) {
            cuuint64_t rstr[3] = {str[0], str[1], d.groups > 1 ? (cuuint64_t)d.res_gs : str[2]};
            if (!encode_map(&mr, d.res, 4, dims, rstr, box, CU_TENSOR_MAP_DATA_TYPE_UINT8, CU_TENSOR_MAP_SWIZZLE_NONE))
                return cudaErrorInvalidValue;
        }
        return launch_kxn<6, true>(ma, mb, mc, mr, a, s);
    }
    if (f8 && staged) {
        // staged outputs of E4M3 layers: codes (64-byte boxes, no swizzle) or bf16 (128-byte swizzle)
        const cuuint64_t oe = o8 ? 1 : 2;
        const CUtensorMapDataType odt = o8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
        const CUtensorMapSwizzle osw = o8 ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_128B;
        bool okc;
        if (ps_stage) {
            cuuint64_t dims[5] = {(cuuint64_t)Cq, 2, (cuuint64_t)Wo, 2, (cuuint64_t)Ho * d.groups};
            cuuint64_t str[4] = {Cq * oe, 2 * Cq * oe, 2ull * Wo * Cq * oe, 4ull * Wo * Cq * oe};
            cuuint32_t box[5] = {64, 1, (cuuint32_t)a.TW, 1, (cuuint32_t)a.TH};
            okc = encode_map(&mc, d.out, 5, dims, str, box, odt, osw);
        } else {
            const int Hd = d.out_h < Ho ? d.out_h : Ho, Wd = d.out_w < Wo ? d.out_w : Wo;
            cuuint64_t dims[4] = {(cuuint64_t)out_c, (cuuint64_t)Wd, (cuuint64_t)Hd, (cuuint64_t)d.groups};
            cuuint64_t str[3] = {out_c * oe, (cuuint64_t)d.out_w * out_c * oe,
                                 d.groups > 1 ? (cuuint64_t)d.out_gs * oe : (cuuint64_t)d.out_h * d.out_w * out_c * oe};
            cuuint32_t box[4] = {64, (cuuint32_t)a.TW, (cuuint32_t)a.TH, 1};
            okc = encode_map(&mc, d.out, 4, dims, str, box, odt, osw);
        }
        if (!okc) return cudaErrorInvalidValue;
        if (!o8)
            return BN != 256 ? cudaErrorInvalidValue
                   : pair    ? launch_bn<256, 8, true, OP_E4M3, false, 1, true>(ma, mb, mc, a, s)
                             : launch_bn<256, 5, true, OP_E4M3>(ma, mb, mc, a, s);
        switch (BN) {
            case 64: return launch_bn<64, 8, true, OP_E4M3, false, 1, false, true>(ma, mb, mc, a, s);
            case 128:
                return MT == 2 ? launch_bn<128, 8, true, OP_E4M3, false, 2, false, true>(ma, mb, mc, a, s)
                               : launch_bn<128, 8, true, OP_E4M3, false, 1, false, true>(ma, mb, mc, a, s);
            case 192: return launch_bn<192, 7, true, OP_E4M3, false, 1, false, true>(ma, mb, mc, a, s);
            default: return launch_bn<256, 6, true, OP_E4M3, false, 1, false, true>(ma, mb, mc, a, s);
        }
    }
    if (f8) {
        if (d.mode != OUT_NHWC && !(d.mode == OUT_PS && d.ps_major)) return cudaErrorInvalidValue;
        switch (BN) {
            case 16: return launch_bn<16, 8, false, OP_E4M3>(ma, mb, mc, a, s);
            case 64: return launch_bn<64, 8, false, OP_E4M3>(ma, mb, mc, a, s);
            case 128: return launch_bn<128, 8, false, OP_E4M3>(ma, mb, mc, a, s);
            case 192: return launch_bn<192, 8, false, OP_E4M3>(ma, mb, mc, a, s);
            default: return launch_bn<256, 7, false, OP_E4M3>(ma, mb, mc, a, s);
        }
    }
    if (halo) {
        // staged stores: bf16 NHWC (64 channels per strip pixel), or the final u8 frame whose rows are a
        // multiple of 16 bytes (three 256-byte boxes per output row pair of a strip)
        const bool st_nhwc = BN == 64 && d.mode == OUT_NHWC && !d.out_f32 && out_c % 8 == 0 && d.out_gs % 8 == 0;
        if (st_nhwc) {
            const int Hd = d.out_h < Ho ? d.out_h : Ho, Wd = d.out_w < Wo ? d.out_w : Wo;
            cuuint64_t dims[4] = {(cuuint64_t)out_c, (cuuint64_t)Wd, (cuuint64_t)Hd, (cuuint64_t)d.groups};
            cuuint64_t str[3] = {out_c * esz, (cuuint64_t)d.out_w * out_c * esz,
                                 d.groups > 1 ? (cuuint64_t)d.out_gs * esz : (cuuint64_t)d.out_h * d.out_w * out_c * esz};
            cuuint32_t box[4] = {64, (cuuint32_t)(kxn ? kKxnStrip : 128), 1, 1};
            if (!encode_map(&mc, d.out, 4, dims, str, box)) return cudaErrorInvalidValue;
            if (!kxn) return launch_halo<64, 2, 1>(ma, mb, mc, a, s);
            CUtensorMap mr = mc;  // the residual, loaded into the staging tile: the output's layout and box
            if (a.res) {
                cuuint64_t rstr[3] = {str[0], str[1], d.groups > 1 ? (cuuint64_t)d.res_gs * esz : str[2]};
                if (!encode_map(&mr, d.res, 4, dims, rstr, box)) return cudaErrorInvalidValue;
            }
            return launch_kxn<2>(ma, mb, mc, mr, a, s);
        }
        return BN == 16 ? launch_halo<16, 3, 0>(ma, mb, mc, a, s) : launch_halo<64, 2, 0>(ma, mb, mc, a, s);
    }
    if (staged) {
        bool okc;
        if (ps_stage) {
            // [G][2Ho][2Wo][Cq] viewed as (Cq, dx, Wo, dy, G*Ho)
            cuuint64_t dims[5] = {(cuuint64_t)Cq, 2, (cuuint64_t)Wo, 2, (cuuint64_t)Ho * d.groups};
            cuuint64_t str[4] = {Cq * esz, 2 * Cq * esz, 2ull * Wo * Cq * esz, 4ull * Wo * Cq * esz};
            cuuint32_t box[5] = {64, 1, (cuuint32_t)a.TW, 1, (cuuint32_t)a.TH};
            okc = encode_map(&mc, d.out, 5, dims, str, box);
        } else {
            // [G][out_h][out_w][out_c], positions beyond Ho x Wo dropped
            const int Hd = d.out_h < Ho ? d.out_h : Ho, Wd = d.out_w < Wo ? d.out_w : Wo;
            cuuint64_t dims[4] = {(cuuint64_t)out_c, (cuuint64_t)Wd, (cuuint64_t)Hd, (cuuint64_t)d.groups};
            cuuint64_t str[3] = {out_c * esz, (cuuint64_t)d.out_w * out_c * esz,
                                 d.groups > 1 ? (cuuint64_t)d.out_gs * esz : (cuuint64_t)d.out_h * d.out_w * out_c * esz};
            cuuint32_t box[4] = {64, (cuuint32_t)a.TW, (cuuint32_t)a.TH, 1};
            okc = encode_map(&mc, d.out, 4, dims, str, box);
        }
        if (!okc) return cudaErrorInvalidValue;
        if (c32) return BN == 64 ? launch_bn<64, 12, true, OP_BF16_32>(ma, mb, mc, a, s) : cudaErrorInvalidValue;
        switch (BN) {
            case 64: return a.kmask != ~0ull ? launch_bn<64, 6, true, OP_BF16, true>(ma, mb, mc, a, s)
                                             : launch_bn<64, 6, true>(ma, mb, mc, a, s);
            case 128: return MT == 2 ? (pair ? launch_bn<128, 4, true, OP_BF16, false, 2, true>(ma, mb, mc, a, s)
                                             : launch_bn<128, 3, true, OP_BF16, false, 2>(ma, mb, mc, a, s))
                                     : launch_bn<128, 4, true>(ma, mb, mc, a, s);
            case 192: return launch_bn<192, 4, true>(ma, mb, mc, a, s);
            default: return pair ? launch_bn<256, 4, true, OP_BF16, false, 1, true>(ma, mb, mc, a, s)
                                 : launch_bn<256, 3, true>(ma, mb, mc, a, s);
        }
    }
    if (c32) return BN == 64 ? launch_bn<64, 12, false, OP_BF16_32>(ma, mb, mc, a, s) : cudaErrorInvalidValue;
    cudaError_t e;
    switch (BN) {
        case 16: e = launch_bn<16, 8, false>(ma, mb, mc, a, s); break;
        case 64: e = launch_bn<64, 8, false>(ma, mb, mc, a, s); break;
        case 128: e = launch_bn<128, 6, false>(ma, mb, mc, a, s); break;
        case 192: e = launch_bn<192, 5, false>(ma, mb, mc, a, s); break;
        default: e = launch_bn<256, 4, false>(ma, mb, mc, a, s); break;
    }
    if (e != cudaSuccess || ksplit == 1) return e;
    const long long n4 = (long long)d.groups * Ho * Wo * (d.Cout / 4);
    const unsigned blocks = (unsigned)((n4 + 255) / 256 < 4096 ? (n4 + 255) / 256 : 4096);
    ++*nl;
    return launch_pdl(conv_tc_split_reduce_kernel, dim3(blocks), dim3(256), (size_t)0, s, a);
}

}  // namespace ufvc
