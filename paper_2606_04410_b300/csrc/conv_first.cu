// The first analysis layer read straight from the chunk's frame bytes (BF16 tensor cores).
//
// A1 is a 3x3 stride-2 convolution of the 3N stacked input channels (frames stacked along channels,
// Sec. 3.1) to 64 outputs with GELU.  Run as a layer over a packed bf16 input tensor it needs a pack pass
// that writes 2.7x the frame bytes (32 bf16 channels per pixel) and an A1 pass that reads them back; here
// one kernel reads the caller's uint8 frames once and feeds the tensor cores from shared memory.
//
// GEMM view of a tile: M = 128 output pixels (16 rows x 8 columns), N = 64 output channels, K = 9 taps x
// CTP channels (channel 3 n + colour of frame n; CTP = 3N rounded up to 16, the rest zero).  The tile's
// input window (33 x 17 pixels of every frame; replicate padding inside the padded frame size, zeros where
// the convolution's own padding lies) is written to shared memory as bf16 (a byte v as v / 256, exact in
// bf16; the weights carry 256 / 255) in the layout [window row][column parity][8-channel group]
// [column / 2][8 channels].  For tap (ky, kx) and 16 channels, output pixel (oy, ox) reads window pixel
// (2 oy + ky, 2 ox + kx), i.e. column ox + kx / 2 of parity kx & 1 of row 2 oy + ky: eight consecutive ox
// are eight consecutive 16-byte rows and consecutive oy are two window rows apart, which is the canonical
// K-major operand layout without swizzle (core matrices of 8 rows x 16 bytes; SBO = two window rows
// between 8-row groups, LBO = one 8-channel group between the two core matrices of K = 16).  So one
// tcgen05.mma (M = 128, N = 64, K = 16) per tap and 16 channels reads the window in place, without an
// im2col copy; the weights [KC][64 rows][128 B] (K = tap CTP + channel, 128-byte swizzle) stay in shared
// memory, already swizzled in global memory.  Accumulators in TMEM (two), drained with tcgen05.ld; bias,
// GELU, bf16 NHWC stores.
//
// Two kernels build the window: conv_first_tma_kernel (interleaved RGB with 16-byte rows: the window
// bytes come by TMA, warp-specialised) and conv_first_kernel (every format: the window bytes are loaded
// into registers one tile ahead).  Both issue the same MMAs on the same operands, so a chunk gives the
// same bits through either.  Every wait is bounded: on a timeout the kernel records UFVC_ERR_TIMEOUT and
// stops.
#include "ufvc_internal.h"
#include "tc_ptx.h"

#include <cuda.h>
#include <cuda_fp8.h>

namespace ufvc {

constexpr int kT4H = 16, kT4W = 8;                      // output tile
constexpr int kW4H = 2 * kT4H + 1, kW4W = 2 * kT4W + 1;  // its 33 x 17 window
constexpr int kW4Px = kW4H * kW4W;
constexpr long long kFirstSpin = 4000000000LL;          // ~2 s at 2 GHz

__host__ __device__ constexpr int first_kc(int k_per_tap) { return (9 * k_per_tap + 63) / 64; }
__host__ __device__ constexpr int first_ctp(int ct) { return (ct + 15) / 16 * 16; }
// converted window: per row 2 parities x CTP/8 groups x 9 columns x 16 bytes
__host__ __device__ constexpr int first_w4_group() { return 9 * 16; }
__host__ __device__ constexpr int first_w4_par(int ctp) { return ctp / 8 * first_w4_group(); }
__host__ __device__ constexpr int first_w4_row(int ctp) { return 2 * first_w4_par(ctp); }
__host__ __device__ constexpr size_t first_w4_bytes(int ctp) { return (size_t)kW4H * first_w4_row(ctp); }

// Explicit shared-memory accesses: the kernels' shared pointers pass through an integer (for 1024-byte
// alignment), after which plain C++ loads through them would be generic loads
__device__ __forceinline__ uint32_t lds_u8(uint32_t addr) {
    uint32_t v;
    asm("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ float4 lds_f4(uint32_t addr) {
    float4 v;
    asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return v;
}
__device__ __forceinline__ int lds_volatile(uint32_t addr) {
    int v;
    asm volatile("ld.volatile.shared.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

// bf16 bits of v / 256 for two bytes: 32768 + v / 256 is exact in FP32 (unit in the last place 2^-8)
__device__ __forceinline__ uint32_t bytes_bf16x2(uint32_t a, uint32_t b) {
    const float fa = __uint_as_float(0x47000000u | a) - 32768.0f, fb = __uint_as_float(0x47000000u | b) - 32768.0f;
    __nv_bfloat162 h = __floats2bfloat162_rn(fa, fb);
    return *reinterpret_cast<uint32_t*>(&h);
}

// Shared-memory matrix descriptor, K-major without swizzle: core matrices of 8 rows x 16 bytes, lbo bytes
// between the two core matrices of K = 16, sbo bytes between 8-row groups; version 1 (sm_100 family).
__device__ __forceinline__ uint64_t sdesc_none(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version; swizzle mode 0 (none)
    return d;
}

__device__ __forceinline__ bool first_wait(uint64_t* bar, uint32_t par, volatile int* stop, int* err,
                                           bool honour_stop = true) {
    if (ptx::mbar_try_wait(bar, par)) return true;
    const long long t0 = clock64();
    while (true) {
        if (ptx::mbar_try_wait(bar, par)) return true;
        if (honour_stop && lds_volatile(ptx::smem_u32((const void*)stop))) return false;
        if (clock64() - t0 > kFirstSpin) {
            *stop = 1;
            atomicCAS(err, 0, (int)UFVC_ERR_TIMEOUT);
            return false;
        }
    }
}

// The tile's MMAs: window xw (layout above) x weights sB_u into accumulator d (thread of the issuing warp)
template <int CTP>
__device__ __forceinline__ void first_mma(uint32_t d, uint32_t xw, uint32_t sB_u) {
    constexpr int GS = first_w4_group(), PS = first_w4_par(CTP), RS = first_w4_row(CTP);
    constexpr uint32_t idesc = ptx::idesc_bf16(64);
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
        const int ky = tap / 3, kx = tap % 3;
#pragma unroll
        for (int s = 0; s < CTP / 16; ++s) {
            const int kb = tap * CTP + 16 * s;  // K offset in the weights
            const uint32_t a = xw + ky * RS + (kx & 1) * PS + 2 * s * GS + (kx >> 1) * 16;
            ptx::mma_f16(d, sdesc_none(a, GS, 2 * RS), ptx::sdesc_sw128(sB_u + (kb >> 6) * 8192 + ((kb & 63) >> 4) * 32),
                         idesc, (tap | s) != 0);
        }
    }
}

// NV consecutive output channels (NV a multiple of 16) as E4M3 codes of value x inv, 16 bytes at a time
template <int NV>
__device__ __forceinline__ void store_e4m3(const float* v, float inv, uint8_t* dst) {
#pragma unroll
    for (int i = 0; i < NV / 16; ++i) {
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float* f = v + 16 * i + 4 * k;
            const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(f[0] * inv, f[1] * inv), __NV_SATFINITE, __NV_E4M3);
            const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(f[2] * inv, f[3] * inv), __NV_SATFINITE, __NV_E4M3);
            w[k] = lo | (hi << 16);
        }
        reinterpret_cast<uint4*>(dst)[i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Epilogue of 32 accumulator columns (half) of output pixel (oh, ow): bias, GELU, NHWC store as bf16, or
// as E4M3 codes of value x out_inv when out_inv != 0 (an FP8 context's A1)
__device__ __forceinline__ void first_store(float* v, uint32_t bias_u, void* out, float out_inv, int oh, int ow,
                                            int Wo, int half) {
#pragma unroll
    for (int c = 0; c < 32; c += 4) {
        const float4 bb = lds_f4(bias_u + half * 128 + 4 * c);
        v[c] += bb.x; v[c + 1] += bb.y; v[c + 2] += bb.z; v[c + 3] += bb.w;
        gelu_tc2(v[c], v[c + 1]);
        gelu_tc2(v[c + 2], v[c + 3]);
    }
    if (out_inv != 0.f) {
        store_e4m3<32>(v, out_inv, static_cast<uint8_t*>(out) + ((size_t)oh * Wo + ow) * 64 + half * 32);
        return;
    }
    uint4* d = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(out) + ((size_t)oh * Wo + ow) * 64 + half * 32);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        uint32_t u[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            __nv_bfloat162 h = __floats2bfloat162_rn(v[8 * i + 2 * e], v[8 * i + 2 * e + 1]);
            u[e] = *reinterpret_cast<uint32_t*>(&h);
        }
        d[i] = make_uint4(u[0], u[1], u[2], u[3]);
    }
}

// ------------------------------------------------------------------------------------------------
// Register-staged kernel (every colour format).  Per tile k: the window bytes of tile k (loaded into
// registers during tile k - 1) are converted into window buffer k % 2; one thread issues the tile's MMAs
// into accumulator k % 2; the loads of tile k + 1 are issued; then tile k - 1 is drained while the MMAs
// run.  One CTA of 16 warps per SM.
// ------------------------------------------------------------------------------------------------
constexpr int kRegThreads = 512;

// byte of channel (frame n, colour) at frame pixel (sh, sw) in colour format FMT (0: RGB interleaved;
// 2: YUV444 planar; 3: YUV420 planar, each chroma sample serving its 2x2 block)
template <int FMT>
__device__ __forceinline__ uint32_t chan_byte(const uint8_t* __restrict__ fr, int n, int colour, int sh, int sw,
                                              int H, int W) {
    if (FMT == 0) return __ldg(fr + ((size_t)n * H * W + (size_t)sh * W + sw) * 3 + colour);
    if (FMT == 2) return __ldg(fr + ((size_t)(3 * n + colour) * H + sh) * W + sw);
    const int Wc = (W + 1) >> 1, Hc = (H + 1) >> 1;
    const size_t pl = (size_t)H * W, cpl = (size_t)Hc * Wc;
    // one load at a selected offset (no branch, so the loads of a tile stay in flight together)
    const size_t o = colour == 0 ? (size_t)sh * W + sw : pl + (colour - 1) * cpl + (size_t)(sh >> 1) * Wc + (sw >> 1);
    return __ldg(fr + (size_t)n * (pl + 2 * cpl) + o);
}

template <int FMT, int CT>
__global__ void __launch_bounds__(kRegThreads, 1)
    conv_first_kernel(const uint8_t* __restrict__ frames, int N, int H, int W, int Ho, int Wo,
                      const uint4* __restrict__ wimg, const float* __restrict__ bias, void* __restrict__ out,
                      float out_inv, int* err) {
    constexpr int CTP = first_ctp(CT);
    constexpr int KCB = first_kc(CTP);
    constexpr int PR = CT / 8;  // 8-channel groups holding real channels
    constexpr int GS = first_w4_group(), PS = first_w4_par(CTP), RS = first_w4_row(CTP);
    constexpr int XB = (int)first_w4_bytes(CTP);
    constexpr int CI = (kW4Px * PR + kRegThreads - 1) / kRegThreads;  // window items per thread
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sB = smem;             // KCB x [64 rows][128 B]
    uint8_t* sx = sB + KCB * 8192;  // 2 x converted window
    float* sbias = reinterpret_cast<float*>(sx + 2 * XB);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sbias + 64);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 2);
    volatile int* stop = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {
        uint4* dB = reinterpret_cast<uint4*>(sB);
        for (int i = tid; i < KCB * 512; i += kRegThreads) dB[i] = __ldg(wimg + i);
        if (tid < 64) sbias[tid] = __ldg(bias + tid);
        uint4* dx = reinterpret_cast<uint4*>(sx);  // groups past the real channels stay zero
        for (int i = tid; i < 2 * XB / 16; i += kRegThreads) dx[i] = make_uint4(0u, 0u, 0u, 0u);
        if (tid == 0) {
            ptx::mbar_init(&bar[0], 1);
            ptx::mbar_init(&bar[1], 1);
            *stop = 0;
            ptx::fence_mbar_init();
        }
        if (warp == 0) ptx::tmem_alloc(tmem_slot, 128);
    }
    ptx::fence_proxy_async();
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    pdl_trigger();
    pdl_wait();  // frames may come from, and the output be read by, the neighbouring kernels

    const int tiles_w = (Wo + kT4W - 1) / kT4W;
    const int tiles = tiles_w * ((Ho + kT4H - 1) / kT4H);
    const int nch = 3 * N;
    const uint32_t sB_u = ptx::smem_u32(sB), sx_u = ptx::smem_u32(sx), bias_u = ptx::smem_u32(sbias);
    const uint32_t stop_u = ptx::smem_u32((const void*)stop);
    uint32_t item[CI];  // (group, window row, window column) of items tid + 512 j, group-major
#pragma unroll
    for (int j = 0; j < CI; ++j) {
        const int i = tid + kRegThreads * j;
        const int g = i / kW4Px, px = i - g * kW4Px, ly = px / kW4W, lx = px - ly * kW4W;
        item[j] = i < kW4Px * PR ? (uint32_t)(g << 16 | ly << 8 | lx) : 0xFFFFFFFFu;
    }
    uint32_t rb[CI][8];

    // the window bytes of tile t into registers (window pixel (ly, lx) = frame pixel (2 h0 - 1 + ly,
    // 2 w0 - 1 + lx); replicate the last row / column, zeros left of and above the frame)
    auto load = [&](int t) {
        const int h0 = (t / tiles_w) * kT4H, w0 = (t % tiles_w) * kT4W;
#pragma unroll
        for (int j = 0; j < CI; ++j) {
            const uint32_t it = item[j];
            const int g = (int)(it >> 16), ly = (int)((it >> 8) & 0xFF), lx = (int)(it & 0xFF);
            const int ih = 2 * h0 - 1 + ly, iw = 2 * w0 - 1 + lx;
            const bool in = it != 0xFFFFFFFFu && ih >= 0 && iw >= 0;
            const int sh = ih < H ? ih : H - 1, sw = iw < W ? iw : W - 1;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int c = 8 * g + e;
                rb[j][e] = in && c < nch ? chan_byte<FMT>(frames, c / 3, c % 3, sh, sw, H, W) : 0u;
            }
        }
    };
    // registers -> window buffer xw
    auto store = [&](uint32_t xw) {
#pragma unroll
        for (int j = 0; j < CI; ++j) {
            const uint32_t it = item[j];
            if (it != 0xFFFFFFFFu) {
                const int g = (int)(it >> 16), ly = (int)((it >> 8) & 0xFF), lx = (int)(it & 0xFF);
                ptx::st_shared_v4(xw + ly * RS + (lx & 1) * PS + g * GS + (lx >> 1) * 16,
                                  bytes_bf16x2(rb[j][0], rb[j][1]), bytes_bf16x2(rb[j][2], rb[j][3]),
                                  bytes_bf16x2(rb[j][4], rb[j][5]), bytes_bf16x2(rb[j][6], rb[j][7]));
            }
        }
    };
    // wait for the MMAs of tile k (thread 0), then drain accumulator k % 2
    auto drain = [&](int k, int t) -> bool {
        const int b = k & 1;
        if (tid == 0) first_wait(&bar[b], (k >> 1) & 1, stop, err);
        __syncthreads();
        if (lds_volatile(stop_u)) return false;
        ptx::tc_fence_after();
        const int q = warp & 3, cq = warp >> 2, row = q * 32 + lane;  // 16 columns per warp
        float v[16];
        ptx::tmem_ld16(tmem_base + b * 64 + ((uint32_t)(q * 32) << 16) + cq * 16, v);
        const int h0 = (t / tiles_w) * kT4H, w0 = (t % tiles_w) * kT4W;
        const int oh = h0 + (row >> 3), ow = w0 + (row & 7);
        if (oh < Ho && ow < Wo) {
#pragma unroll
            for (int c = 0; c < 16; c += 4) {
                const float4 bb = lds_f4(bias_u + cq * 64 + 4 * c);
                v[c] += bb.x; v[c + 1] += bb.y; v[c + 2] += bb.z; v[c + 3] += bb.w;
                gelu_tc2(v[c], v[c + 1]);
                gelu_tc2(v[c + 2], v[c + 3]);
            }
            if (out_inv != 0.f) {
                store_e4m3<16>(v, out_inv, static_cast<uint8_t*>(out) + ((size_t)oh * Wo + ow) * 64 + cq * 16);
            } else {
                uint4* d = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(out) + ((size_t)oh * Wo + ow) * 64 +
                                                    cq * 16);
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    uint32_t u[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        __nv_bfloat162 h = __floats2bfloat162_rn(v[8 * i + 2 * e], v[8 * i + 2 * e + 1]);
                        u[e] = *reinterpret_cast<uint32_t*>(&h);
                    }
                    d[i] = make_uint4(u[0], u[1], u[2], u[3]);
                }
            }
        }
        ptx::tc_fence_before();
        __syncthreads();  // accumulator b is free again
        return true;
    };

    int t = blockIdx.x, tprev = -1, k = 0;
    if (t < tiles) load(t);
    for (; t < tiles; t += gridDim.x, ++k) {
        const int b = k & 1;
        store(sx_u + b * XB);  // window b was last read by the MMAs of tile k - 2, drained before
        ptx::fence_proxy_async();
        ptx::tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            ptx::tc_fence_after();
            first_mma<CTP>(tmem_base + b * 64, sx_u + b * XB, sB_u);
            ptx::mma_commit(&bar[b]);
        }
        if (t + (int)gridDim.x < tiles) load(t + gridDim.x);
        if (k > 0 && !drain(k - 1, tprev)) break;
        tprev = t;
    }
    if (k > 0 && tprev >= 0) drain(k - 1, tprev);
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem_base, 128);
    }
}

// ------------------------------------------------------------------------------------------------
// Warp-specialised variant for interleaved RGB frames whose rows are whole 16-byte units (3 W % 16 = 0).
// The output tile is 16 rows x 8 columns, and the operand is read by the MMAs straight from the converted
// window, without an im2col copy:
//   * the window (33 x 17 pixels of every frame) comes by TMA: frames are viewed as a 3D byte tensor
//     (3 W, H, N) and a tile's window (bytes 3 (2 w0 - 1) .. +50 of rows 2 h0 - 1 .. +32) is one box of
//     64 x 33 x N bytes starting at byte 6 w0 - 16 (a multiple of 16; the window starts 13 bytes in).
//     Coordinates left of and above the frame read zeros (the convolution's padding); rows below the frame
//     are read as its last row;
//   * converter warps write it as bf16 in the layout [window row][column parity][8-channel group]
//     [column / 2][8 channels] (channel 3 n + colour, CTP = 3N rounded up to 16 channels per pixel);
//   * for tap (ky, kx) and 16 channels, output pixel (oy, ox) reads window pixel (2 oy + ky, 2 ox + kx),
//     i.e. column ox + kx / 2 of parity kx & 1 of row 2 oy + ky: eight consecutive ox are eight consecutive
//     16-byte rows and consecutive oy are two window rows apart, which is the canonical K-major layout
//     without swizzle (core matrices of 8 rows x 16 bytes; SBO = two window rows between 8-row groups,
//     LBO = one 8-channel group between the two core matrices of K = 16).  So one tcgen05.mma per tap and
//     16 channels reads the window in place (9 CTP / 16 MMAs per tile).
// Roles: warps 0-7 convert, warp 8 issues the MMAs, warp 9 the TMA loads, warps 10-17 drain the
// accumulators.  Raw windows (kRawBufs deep, enough bytes in flight per SM to cover the DRAM latency),
// converted windows (two) and TMEM accumulators (two) pass between the roles through mbarriers, every
// wait bounded.
// ------------------------------------------------------------------------------------------------
constexpr int kRawBX = 64;                                   // box bytes per window row (13 + 51 used)
constexpr int kConvWarps = 8, kMmaWarp = 8, kTmaWarp = 9, kEpiWarp0 = 10;
constexpr int kTmaThreads = 18 * 32;
constexpr int kRawBufs = 6;

__host__ __device__ constexpr size_t first_raw_bytes(int n) { return ((size_t)n * kW4H * kRawBX + 127) & ~size_t(127); }
__host__ __device__ constexpr size_t first_tma_smem(int ct, int n) {
    return 1024 + (size_t)first_kc(first_ctp(ct)) * 8192 + 2 * first_w4_bytes(first_ctp(ct)) +
           kRawBufs * first_raw_bytes(n) + 256 + 256;
}
__host__ __device__ constexpr size_t first_reg_smem(int ct) {
    return 1024 + (size_t)first_kc(first_ctp(ct)) * 8192 + 2 * first_w4_bytes(first_ctp(ct)) + 256 + 64;
}

// barrier 1 over the converter warps; returns the OR of pred over them
__device__ __forceinline__ int conv_sync_or(int pred) {
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.s32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, 256, p;\n\t"
        "selp.s32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r) : "r"(pred) : "memory");
    return r;
}
__device__ __forceinline__ void conv_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// 8 channels 8 P .. 8 P + 7 of the window pixel whose bytes start at rw + base (frame f at f x 33 x 64)
template <int P>
__device__ __forceinline__ uint4 window_group(uint32_t rw, uint32_t base, int nch) {
    uint32_t b[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int c = 8 * P + e;
        b[e] = c < nch ? lds_u8(rw + base + (c / 3) * (kW4H * kRawBX) + c % 3) : 0u;
    }
    return make_uint4(bytes_bf16x2(b[0], b[1]), bytes_bf16x2(b[2], b[3]), bytes_bf16x2(b[4], b[5]),
                      bytes_bf16x2(b[6], b[7]));
}

template <int CT>
__global__ void __launch_bounds__(kTmaThreads, 1)
    conv_first_tma_kernel(const __grid_constant__ CUtensorMap tmF, int N, int H, int Ho, int Wo,
                          const uint4* __restrict__ wimg, const float* __restrict__ bias,
                          void* __restrict__ out, float out_inv, int* err) {
    constexpr int CTP = first_ctp(CT);
    constexpr int KCB = first_kc(CTP);             // 64-element K chunks of the weights (K = 9 CTP)
    constexpr int PR = CT / 8;                     // 8-channel groups holding real channels
    constexpr int GS = first_w4_group(), PS = first_w4_par(CTP), RS = first_w4_row(CTP);
    constexpr int XB = (int)first_w4_bytes(CTP);
    constexpr int CI = (kW4Px * PR + 255) / 256;   // window items per converter thread
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t RAWB = (uint32_t)first_raw_bytes(N);
    uint8_t* sB = smem;                           // KCB x [64 rows][128 B]
    uint8_t* sx = sB + KCB * 8192;                // 2 x converted window
    uint8_t* sraw = sx + 2 * XB;                  // kRawBufs x [N][33][64] window bytes
    float* sbias = reinterpret_cast<float*>(sraw + kRawBufs * RAWB);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sbias + 64);
    uint64_t *raw_full = bars, *raw_empty = bars + kRawBufs, *x_full = bars + 2 * kRawBufs;
    uint64_t *x_empty = x_full + 2, *acc_full = x_full + 4, *acc_empty = x_full + 6, *drain = x_full + 8;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* stop = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {
        uint4* dB = reinterpret_cast<uint4*>(sB);
        for (int i = tid; i < KCB * 512; i += kTmaThreads) dB[i] = __ldg(wimg + i);
        if (tid < 64) sbias[tid] = __ldg(bias + tid);
        uint4* dx = reinterpret_cast<uint4*>(sx);  // groups past the real channels stay zero
        for (int i = tid; i < 2 * XB / 16; i += kTmaThreads) dx[i] = make_uint4(0u, 0u, 0u, 0u);
        if (tid == 0) {
            for (int i = 0; i < kRawBufs; ++i) {
                ptx::mbar_init(&raw_full[i], 1);
                ptx::mbar_init(&raw_empty[i], 1);
            }
            for (int i = 0; i < 2; ++i) {
                ptx::mbar_init(&x_full[i], 1);
                ptx::mbar_init(&x_empty[i], 1);
                ptx::mbar_init(&acc_full[i], 1);
                ptx::mbar_init(&acc_empty[i], 256);
            }
            ptx::mbar_init(drain, 1);
            *stop = 0;
            ptx::fence_mbar_init();
        }
        if (warp == 0) ptx::tmem_alloc(tmem_slot, 128);
        if (warp == kTmaWarp && lane == 0) ptx::prefetch_tmap(&tmF);
    }
    ptx::fence_proxy_async();
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    pdl_trigger();
    pdl_wait();

    const int tiles_w = (Wo + kT4W - 1) / kT4W;
    const int tiles = tiles_w * ((Ho + kT4H - 1) / kT4H);

    if (warp < kConvWarps) {
        // ------------------------------------------------------------ raw window -> bf16 window
        const int nch = 3 * N;
        const uint32_t sx_u = ptx::smem_u32(sx), stop_u = ptx::smem_u32((const void*)stop);
        uint32_t item[CI];  // (group, window row, window column) of items tid + 256 j, group-major
#pragma unroll
        for (int j = 0; j < CI; ++j) {
            const int i = tid + 256 * j;
            const int g = i / kW4Px, px = i - g * kW4Px, ly = px / kW4W, lx = px - ly * kW4W;
            item[j] = i < kW4Px * PR ? (uint32_t)(g << 16 | ly << 8 | lx) : 0xFFFFFFFFu;
        }
        int k = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++k) {
            const int r = k % kRawBufs, b = k & 1;
            const uint32_t rpar = (k / kRawBufs) & 1, par = (k >> 1) & 1;
            const int h0 = (t / tiles_w) * kT4H;
            const int lymax = H - 1 - (2 * h0 - 1);  // window rows past it repeat the frame's last row
            if (tid == 0) {
                first_wait(&raw_full[r], rpar, stop, err);
                first_wait(&x_empty[b], par ^ 1, stop, err);  // the MMAs of tile k - 2 have read window b
            }
            if (conv_sync_or(lds_volatile(stop_u))) break;
            const uint32_t rw = ptx::smem_u32(sraw) + r * RAWB, xw = sx_u + b * XB;
#pragma unroll
            for (int j = 0; j < CI; ++j) {
                const uint32_t it = item[j];
                if (it != 0xFFFFFFFFu) {
                    const int g = (int)(it >> 16), ly = (int)((it >> 8) & 0xFF), lx = (int)(it & 0xFF);
                    const int lys = ly < lymax ? ly : (lymax > 0 ? lymax : 0);
                    const uint32_t base = (uint32_t)(lys * kRawBX + 13 + 3 * lx);
                    uint4 v;
                    if (g == 0) v = window_group<0>(rw, base, nch);
                    else if (g == 1) v = window_group<1>(rw, base, nch);
                    else v = window_group<2>(rw, base, nch);
                    ptx::st_shared_v4(xw + ly * RS + (lx & 1) * PS + g * GS + (lx >> 1) * 16, v.x, v.y, v.z, v.w);
                }
            }
            ptx::fence_proxy_async();  // window b -> visible to the tensor cores
            conv_sync();
            if (tid == 0) {
                ptx::mbar_arrive(&raw_empty[r]);
                ptx::mbar_arrive(&x_full[b]);
            }
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t sB_u = ptx::smem_u32(sB), sx_u = ptx::smem_u32(sx);
            int k = 0;
            for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++k) {
                const int b = k & 1;
                const uint32_t par = (k >> 1) & 1;
                if (!first_wait(&x_full[b], par, stop, err)) break;
                if (!first_wait(&acc_empty[b], par ^ 1, stop, err)) break;
                ptx::tc_fence_after();
                first_mma<CTP>(tmem_base + b * 64, sx_u + b * XB, sB_u);
                ptx::mma_commit(&x_empty[b]);
                ptx::mma_commit(&acc_full[b]);
            }
            ptx::mma_commit(drain);  // every issued MMA completes before TMEM is released
            first_wait(drain, 0, stop, err, false);
        }
        __syncwarp();
    } else if (warp == kTmaWarp) {
        // ------------------------------------------------------------ TMA window loads
        if (lane == 0) {
            int k = 0;
            for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++k) {
                const int r = k % kRawBufs;
                const uint32_t rpar = (k / kRawBufs) & 1;
                if (!first_wait(&raw_empty[r], rpar ^ 1, stop, err)) break;
                const int h0 = (t / tiles_w) * kT4H, w0 = (t % tiles_w) * kT4W;
                ptx::mbar_arrive_expect_tx(&raw_full[r], (uint32_t)(N * kW4H * kRawBX));
                ptx::tma_load_3d(sraw + r * RAWB, &tmF, &raw_full[r], 6 * w0 - 16, 2 * h0 - 1, 0);
            }
            // no copy may still be writing shared memory when the CTA exits: the last load into each
            // buffer (loads k - kRawBufs .. k - 1) has completed
            for (int j = k - kRawBufs; j < k; ++j)
                if (j >= 0) first_wait(&raw_full[j % kRawBufs], (j / kRawBufs) & 1, stop, err, false);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3, half = (warp - kEpiWarp0) >> 2, row = q * 32 + lane;
        int k = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++k) {
            const int b = k & 1;
            const uint32_t par = (k >> 1) & 1;
            if (!__all_sync(0xffffffffu, first_wait(&acc_full[b], par, stop, err))) break;
            ptx::tc_fence_after();
            float v[32];
            ptx::tmem_ld32(tmem_base + b * 64 + ((uint32_t)(q * 32) << 16) + half * 32, v);
            ptx::tc_fence_before();
            ptx::mbar_arrive(&acc_empty[b]);
            const int h0 = (t / tiles_w) * kT4H, w0 = (t % tiles_w) * kT4W;
            const int oh = h0 + (row >> 3), ow = w0 + (row & 7);
            if (oh < Ho && ow < Wo) first_store(v, ptx::smem_u32(sbias), out, out_inv, oh, ow, Wo, half);
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem_base, 128);
    }
}

template <int CT>
static cudaError_t launch_first_tma_t(const uint8_t* frames, int N, int H, int W, int Ho, int Wo, const void* wimg,
                                      const float* bias, void* out, float out_inv, int* err, cudaStream_t s) {
    alignas(64) CUtensorMap map;
    if (!encode_frames_map(&map, frames, N, H, 3 * W, kRawBX, kW4H)) return cudaErrorInvalidValue;
    cudaError_t e = smem_optin((const void*)conv_first_tma_kernel<CT>, (int)first_tma_smem(CT, 8));
    if (e != cudaSuccess) return e;
    const int sms = sm_count();
    const int tiles = ((Wo + kT4W - 1) / kT4W) * ((Ho + kT4H - 1) / kT4H);
    const int grid = tiles < sms ? tiles : sms;
    return launch_pdl(conv_first_tma_kernel<CT>, dim3(grid), dim3(kTmaThreads), first_tma_smem(CT, N), s, map, N, H,
                      Ho, Wo, static_cast<const uint4*>(wimg), bias, out, out_inv, err);
}

template <int FMT, int CT>
static cudaError_t launch_first_t(const uint8_t* frames, int N, int H, int W, int Ho, int Wo, const void* wimg,
                                  const float* bias, void* out, float out_inv, int* err, cudaStream_t s) {
    const size_t smem = first_reg_smem(CT);
    cudaError_t e = smem_optin((const void*)conv_first_kernel<FMT, CT>, (int)smem);
    if (e != cudaSuccess) return e;
    const int sms = sm_count();
    const int tiles = ((Wo + kT4W - 1) / kT4W) * ((Ho + kT4H - 1) / kT4H);
    const int grid = tiles < sms ? tiles : sms;
    return launch_pdl(conv_first_kernel<FMT, CT>, dim3(grid), dim3(kRegThreads), smem, s, frames, N, H, W, Ho, Wo,
                      static_cast<const uint4*>(wimg), bias, out, out_inv, err);
}

int first_layer_ct(int n_frames) {
    return n_frames >= 2 && n_frames <= 8 && n_frames % 2 == 0 ? (3 * n_frames + 7) / 8 * 8 : 0;
}

int first_layer_pitch(int n_frames) { return first_ctp(first_layer_ct(n_frames)); }

size_t first_layer_weight_bytes(int pitch) { return (size_t)first_kc(pitch) * 8192; }

void first_layer_weights(const float* w, int n_frames, float scale, int pitch, uint16_t* img) {
    const int ci = 3 * n_frames;
    for (size_t i = 0; i < first_layer_weight_bytes(pitch) / 2; ++i) img[i] = 0;
    for (int co = 0; co < 64; ++co)
        for (int tap = 0; tap < 9; ++tap)
            for (int c = 0; c < ci; ++c) {
                const int k = tap * pitch + c, j = k >> 6, chunk = ((k & 63) >> 3) ^ (co & 7);
                const size_t e = (size_t)j * 4096 + (size_t)co * 64 + chunk * 8 + (k & 7);
                const __nv_bfloat16 h = __float2bfloat16(scale * w[((size_t)co * 9 + tap) * ci + c]);
                img[e] = *reinterpret_cast<const uint16_t*>(&h);
            }
}

bool first_layer_tma_ok(int fmt, int W, const void* frames) {
    return fmt == 0 && (3 * W) % 16 == 0 && (reinterpret_cast<uintptr_t>(frames) & 15) == 0;
}

cudaError_t launch_first_layer(const uint8_t* frames, int fmt, int N, int H, int W, int Ho, int Wo, const void* wimg,
                               const float* bias, void* out, float out_inv, int* err, cudaStream_t s, int sel) {
    const int ct = first_layer_ct(N);
    const bool tma = first_layer_tma_ok(fmt, W, frames);
    if (sel == 2 && !tma) return cudaErrorInvalidValue;
    if (tma && sel != 1) {
        switch (ct) {  // whole 16-byte rows: the window comes by TMA
            case 8: return launch_first_tma_t<8>(frames, N, H, W, Ho, Wo, wimg, bias, out, out_inv, err, s);
            case 16: return launch_first_tma_t<16>(frames, N, H, W, Ho, Wo, wimg, bias, out, out_inv, err, s);
            case 24: return launch_first_tma_t<24>(frames, N, H, W, Ho, Wo, wimg, bias, out, out_inv, err, s);
            default: return cudaErrorInvalidValue;
        }
    }
#define UFVC_FIRST(F)                                                                                          \
    switch (ct) {                                                                                              \
        case 8: return launch_first_t<F, 8>(frames, N, H, W, Ho, Wo, wimg, bias, out, out_inv, err, s);                 \
        case 16: return launch_first_t<F, 16>(frames, N, H, W, Ho, Wo, wimg, bias, out, out_inv, err, s);               \
        case 24: return launch_first_t<F, 24>(frames, N, H, W, Ho, Wo, wimg, bias, out, out_inv, err, s);               \
        default: return cudaErrorInvalidValue;                                                                 \
    }
    switch (fmt) {
        case 0: UFVC_FIRST(0)
        case 2: UFVC_FIRST(2)
        case 3: UFVC_FIRST(3)
        default: return cudaErrorInvalidValue;
    }
#undef UFVC_FIRST
}

}  // namespace ufvc
