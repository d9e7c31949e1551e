// Hyper-synthesis layers (S1, S2, S3) on the 5th-generation tensor cores at FP32-level accuracy.
//
// A float x is split into two TF32 parts: hi(x) = x rounded to the nearest TF32 value (10 fraction bits;
// the 13 low bits of the FP32 fraction rounded away, halves away from zero) and lo(x) = hi(x - hi(x))
// (x - hi(x) is exact in FP32), so that |x - hi(x) - lo(x)| <= 2^-22 |x|.  A product a w is taken as
// hi(a) hi(w) + hi(a) lo(w) + lo(a) hi(w); the terms left out are of order 2^-22 |a w| and, rounded to
// nearest rather than truncated, of either sign, so they do not add up along K.
// The three products run as one GEMM over a tripled K: for tap t and input channel c, K index
// (t, part, c) pairs the input plane (hi, hi, lo)[part] with the weight plane (hi, lo, hi)[part].
// tcgen05.mma kind::tf32 reads each operand from its 32-bit container; the parts carry no bits below
// the TF32 mantissa, so nothing is rounded on the way in, and the product of two parts (11 x 11
// significant bits) is exact before it enters the FP32 accumulator.
//
// One CTA per (128-pixel tile, 256 output channels, K range): warp 0 loads the input plane tile (one
// TMA box of 32 channels x TW x TH pixels, zero-filled outside the image: the convolution's padding)
// and the weight tile (256 rows x 32 K) into a 4-stage ring, warp 1 issues four MMAs (M = 128,
// N = 256, K = 8) per stage into a TMEM accumulator, and four epilogue warps write the range's raw sums
// to the split-K workspace [K range][Ho * Wo][Cout].  conv_simt_reduce_kernel and
// conv_simt_reduce_entropy_kernel then add the ranges in range order and apply the bias, GELU, pixel
// shuffle, crop, mu / log sigma split and entropy parameters, as for the SIMT layers.  Tiles and K
// ranges depend only on the layer shape, so encoder and decoder compute identical bits.
// Every mbarrier wait is bounded: on a timeout the kernel records UFVC_ERR_TIMEOUT, all roles stop,
// in-flight copies and MMAs are waited for (bounded), TMEM is freed and the kernel returns.
#include "ufvc_internal.h"
#include "tc_ptx.h"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cstring>

namespace ufvc {

namespace {

constexpr long long kTfSpin = 4000000000LL;  // ~2 s at 2 GHz
constexpr int kTfBN = 256, kTfStages = 4, kTfThreads = 192;
constexpr int kTfABytes = 128 * 128, kTfBBytes = kTfBN * 128;
constexpr size_t kTfSmem = 1024 + (size_t)kTfStages * (kTfABytes + kTfBBytes) + 128;

struct TfArgs {
    int Ho, Wo, TW, tiles_w;
    int k, pad, C;      // kernel size, padding, input channels (a multiple of 32)
    int nck, cchunks;   // K steps (taps x 3 parts x C / 32), 32-channel chunks of C
    int KS, Cout;
    float* ws;
    int* err;
};

__device__ __forceinline__ bool tf_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err,
                                        bool honour_abort = true) {
    if (ptx::mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (ptx::mbar_try_wait(bar, parity)) return true;
        if (honour_abort && *abort_flag) return false;
        if (clock64() - t0 > kTfSpin) {
            *abort_flag = 1;
            atomicCAS(err, 0, (int)UFVC_ERR_TIMEOUT);
            return false;
        }
    }
}

// x rounded to the nearest TF32 value (finite x; a carry out of the fraction steps the exponent, as it should)
__device__ __forceinline__ float tf_hi(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__global__ void __launch_bounds__(kTfThreads, 1)
    conv_tf32x3_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                       const TfArgs p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + kTfStages * kTfABytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + kTfStages * kTfBBytes);
    uint64_t* empty = full + kTfStages;
    uint64_t* done = empty + kTfStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kTfStages; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 1);
        }
        ptx::mbar_init(done, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 1) ptx::tmem_alloc(tmem_slot, kTfBN);
    if (warp == 0 && lane == 0) {
        ptx::prefetch_tmap(&tmA);
        ptx::prefetch_tmap(&tmB);
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    // the set-up above may overlap the previous kernel's tail; its outputs are read only after it completed
    pdl_trigger();
    pdl_wait();
    const int TH = 128 / p.TW;
    const int mt = blockIdx.x, nt = blockIdx.y, kr = blockIdx.z;
    const int h0 = (mt / p.tiles_w) * TH, w0 = (mt % p.tiles_w) * p.TW;
    const int k0 = (int)((long long)kr * p.nck / p.KS), k1 = (int)((long long)(kr + 1) * p.nck / p.KS);
    const int per_tap = 3 * p.cchunks;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t last_par[kTfStages];
            bool used[kTfStages];
#pragma unroll
            for (int s = 0; s < kTfStages; ++s) { used[s] = false; last_par[s] = 0; }
            int it = 0;
            for (int ks = k0; ks < k1; ++ks, ++it) {
                const int s = it % kTfStages;
                const uint32_t ph = (it / kTfStages) & 1;
                if (!tf_wait(&empty[s], ph ^ 1, abort_flag, p.err)) break;
                const int tap = ks / per_tap, rem = ks - tap * per_tap, part = rem / p.cchunks;
                const int ca = (part == 2 ? p.C : 0) + (rem - part * p.cchunks) * 32;  // plane hi, hi, lo
                const int ky = tap / p.k, kx = tap - ky * p.k;
                ptx::mbar_arrive_expect_tx(&full[s], kTfABytes + kTfBBytes);
                ptx::tma_load_3d(sA + s * kTfABytes, &tmA, &full[s], ca, w0 + kx - p.pad, h0 + ky - p.pad);
                ptx::tma_load_3d(sB + s * kTfBBytes, &tmB, &full[s], ks * 32, nt * kTfBN, 0);
                used[s] = true;
                last_par[s] = ph;
            }
            // no copy may still be writing shared memory when the CTA exits
#pragma unroll
            for (int s = 0; s < kTfStages; ++s)
                if (used[s]) tf_wait(&full[s], last_par[s], abort_flag, p.err, false);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = ptx::idesc_tf32(kTfBN);
            int it = 0;
            for (int ks = k0; ks < k1; ++ks, ++it) {
                const int s = it % kTfStages;
                const uint32_t ph = (it / kTfStages) & 1;
                if (!tf_wait(&full[s], ph, abort_flag, p.err)) break;
                ptx::tc_fence_after();
                const uint32_t a0 = ptx::smem_u32(sA + s * kTfABytes), b0 = ptx::smem_u32(sB + s * kTfBBytes);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)  // 4 x K = 8 TF32 per 128-byte row
                    ptx::mma_tf32(tmem_base, ptx::sdesc_sw128(a0 + kk * 32), ptx::sdesc_sw128(b0 + kk * 32), idesc,
                                  ks != k0 || kk != 0);
                ptx::mma_commit(&empty[s]);
            }
            ptx::mma_commit(done);  // arrives once every MMA issued above has completed
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue: warps 2..5
        const int q = warp & 3;  // the TMEM lane quarter this warp may access
        const int row = q * 32 + lane;
        const int oh = h0 + row / p.TW, ow = w0 + row % p.TW;
        const bool valid = oh < p.Ho && ow < p.Wo;
        const bool ok = __all_sync(0xffffffffu, tf_wait(done, 0, abort_flag, p.err));
        ptx::tc_fence_after();
        if (__all_sync(0xffffffffu, ok && !*abort_flag)) {
            const size_t M = (size_t)p.Ho * p.Wo;
            float* dst = p.ws + ((size_t)kr * M + (size_t)(valid ? oh * p.Wo + ow : 0)) * p.Cout + nt * kTfBN;
#pragma unroll 1
            for (int c = 0; c < kTfBN; c += 32) {
                float v[32];
                ptx::tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) + c, v);
                if (valid) {
                    float4* d4 = reinterpret_cast<float4*>(dst + c);
#pragma unroll
                    for (int i = 0; i < 8; ++i) d4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                }
            }
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem_base, kTfBN);
    }
}

// The input's TF32 planes: out[p][0..C) = hi(x[p][c]), out[p][C..2C) = lo(x[p][c]).  Four channels per
// thread (C % 4 == 0).
__global__ void tf32_planes_kernel(const float* __restrict__ x, long long n4, int C4, float* __restrict__ out) {
    pdl_trigger();
    pdl_wait();
    const float4* x4 = reinterpret_cast<const float4*>(x);
    float4* o4 = reinterpret_cast<float4*>(out);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
        const long long px = i / C4;
        const int c = (int)(i - px * C4);
        const float4 v = x4[i];
        const float4 h = make_float4(tf_hi(v.x), tf_hi(v.y), tf_hi(v.z), tf_hi(v.w));
        const float4 l = make_float4(tf_hi(v.x - h.x), tf_hi(v.y - h.y), tf_hi(v.z - h.z), tf_hi(v.w - h.w));
        o4[px * 2 * C4 + c] = h;
        o4[px * 2 * C4 + C4 + c] = l;
    }
}

// Output tile TW x (128 / TW) with the least padded area.
int tf_pick_tw(int Ho, int Wo) {
    long long best = -1;
    int tw_best = 128;
    for (int tw = 128; tw >= 8; tw >>= 1) {
        const int th = 128 / tw;
        const long long cost = (long long)((Wo + tw - 1) / tw) * tw * ((Ho + th - 1) / th) * th;
        if (best < 0 || cost < best) { best = cost; tw_best = tw; }
    }
    return tw_best;
}

struct TfPlan {
    int TW, tiles_w, tiles_h, n_tiles, nck, KS;
};

TfPlan tf_plan(const ConvDesc& d) {
    TfPlan t;
    t.TW = tf_pick_tw(d.H, d.W);
    t.tiles_w = (d.W + t.TW - 1) / t.TW;
    t.tiles_h = (d.H + 128 / t.TW - 1) / (128 / t.TW);
    t.n_tiles = d.Cout / kTfBN;
    t.nck = d.k * d.k * 3 * (d.Cin / 32);
    // K ranges: about one wave of CTAs (one per SM), at least four K steps per range
    const long long ctas = (long long)t.tiles_w * t.tiles_h * t.n_tiles;
    long long ks = 148 / ctas;
    if (ks > t.nck / 4) ks = t.nck / 4;
    t.KS = (int)(ks < 1 ? 1 : ks);
    return t;
}

size_t planes_floats(const ConvDesc& d) { return ((size_t)d.H * d.W * 2 * d.Cin + 63) & ~(size_t)63; }

}  // namespace

bool conv_tf32x3_ok(const ConvDesc& d) {
    return d.wtf && d.groups == 1 && d.stride == 1 && (d.k == 1 || d.k == 3) && d.Cin % 32 == 0 && d.Cin > 0 &&
           d.Cout % kTfBN == 0 && d.Cout > 0 && d.in_gs == 0;
}

size_t conv_tf32x3_workspace(const ConvDesc& d) {
    const TfPlan t = tf_plan(d);
    return planes_floats(d) + (size_t)t.KS * d.H * d.W * d.Cout;
}

cudaError_t launch_tf32x3_gemm(const ConvDesc& d, cudaStream_t st, int* KS, const float** sums) {
    if (!conv_tf32x3_ok(d) || !d.ws || d.ws_cap < conv_tf32x3_workspace(d) ||
        (reinterpret_cast<uintptr_t>(d.in) & 15) || (reinterpret_cast<uintptr_t>(d.ws) & 255))
        return cudaErrorInvalidValue;
    const TfPlan t = tf_plan(d);
    float* planes = d.ws;
    float* ws = d.ws + planes_floats(d);
    // the input's hi / lo planes
    const long long n4 = (long long)d.H * d.W * d.Cin / 4;
    const unsigned blocks = (unsigned)((n4 + 255) / 256 < 4096 ? (n4 + 255) / 256 : 4096);
    cudaError_t e = launch_pdl(tf32_planes_kernel, dim3(blocks), dim3(256), (size_t)0, st,
                               static_cast<const float*>(d.in), n4, d.Cin / 4, planes);
    if (e != cudaSuccess) return e;
    // A: planes as (2C, W, H) float, box (32, TW, 128 / TW); B: weights as (K', Cout, 1), box (32, 256, 1)
    alignas(64) CUtensorMap ma, mb;
    const uint64_t da[3] = {(uint64_t)2 * d.Cin, (uint64_t)d.W, (uint64_t)d.H};
    const uint64_t sa[2] = {(uint64_t)2 * d.Cin * 4, (uint64_t)d.W * 2 * d.Cin * 4};
    const uint32_t ba[3] = {32, (uint32_t)t.TW, (uint32_t)(128 / t.TW)};
    const uint64_t K3 = (uint64_t)d.k * d.k * 3 * d.Cin;
    const uint64_t db[3] = {K3, (uint64_t)d.Cout, 1};
    const uint64_t sb[2] = {K3 * 4, K3 * 4 * d.Cout};
    const uint32_t bb[3] = {32, (uint32_t)kTfBN, 1};
    if (!encode_f32_map_sw128(&ma, planes, 3, da, sa, ba) || !encode_f32_map_sw128(&mb, d.wtf, 3, db, sb, bb))
        return cudaErrorInvalidValue;
    e = smem_optin(reinterpret_cast<const void*>(conv_tf32x3_kernel), (int)kTfSmem);
    if (e != cudaSuccess) return e;
    TfArgs a;
    a.Ho = d.H; a.Wo = d.W; a.TW = t.TW; a.tiles_w = t.tiles_w;
    a.k = d.k; a.pad = d.k / 2; a.C = d.Cin;
    a.nck = t.nck; a.cchunks = d.Cin / 32;
    a.KS = t.KS; a.Cout = d.Cout;
    a.ws = ws;
    a.err = d.err;
    e = launch_pdl(conv_tf32x3_kernel, dim3((unsigned)(t.tiles_w * t.tiles_h), (unsigned)t.n_tiles, (unsigned)t.KS),
                   dim3(kTfThreads), kTfSmem, st, ma, mb, a);
    *KS = t.KS;
    *sums = ws;
    return e;
}

}  // namespace ufvc
