// Elementwise and entropy-coding kernels.
//
//  * pack          : chunk frames uint8 [N][H][W][3] -> /255, replicate pad to x16, frames stacked into
//                    channels (frame n -> channels 3n..3n+2), zero channels up to the padded count
//                    (the patch-embedding input of Sec. 3.1).
//  * zquant        : z^ = clamp(rint(z), +-255) and the per-channel scale index of z^.
//  * quantize      : r^ = clamp(rint((y - mu) / q), +-255) and the scale index of log sigma (Sec. 3.4).
//  * rANS          : K interleaved lanes, the whole latent coded in one step (Sec. 3.4): element i goes
//                    to lane i mod K; 32-bit state in [2^16, 2^32), 16-bit probabilities, 16-bit words,
//                    at most one renormalisation word per symbol.
#include "ufvc_internal.h"

#include <cuda_fp8.h>

#include <algorithm>
#include "tc_ptx.h"

#include <cub/block/block_scan.cuh>

namespace ufvc {

__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, 0, code); }

// ------------------------------------------------------------------------------------------------
// pack
// ------------------------------------------------------------------------------------------------
// BT.709, full range, chroma centred at 0.5: Y = 0.2126 R + 0.7152 G + 0.0722 B, U = (B - Y) / 1.8556 + 0.5,
// V = (R - Y) / 1.5748 + 0.5, on RGB bytes / 255
__device__ __forceinline__ void bt709_from_bytes(const uint32_t* b, float* v) {
    const float r = b[0] / 255.0f, g = b[1] / 255.0f, bl = b[2] / 255.0f;
    const float y = fmaf(0.0722f, bl, fmaf(0.7152f, g, 0.2126f * r));
    v[0] = y;
    v[1] = fmaf(bl - y, 1.0f / 1.8556f, 0.5f);
    v[2] = fmaf(r - y, 1.0f / 1.5748f, 0.5f);
}

// frame n's three network channels of pixel (sh, sw), as floats in [0, 1]
template <int FMT>
__device__ __forceinline__ void px_values(const uint8_t* __restrict__ fr, int n, int sh, int sw, int H, int W, float* v) {
    uint32_t b[3];
    px_bytes<FMT>(fr, n, sh, sw, H, W, b);
    if (FMT == 1) bt709_from_bytes(b, v);
    else { v[0] = b[0] / 255.0f; v[1] = b[1] / 255.0f; v[2] = b[2] / 255.0f; }
}

template <int FMT>
__global__ void pack_kernel(const uint8_t* __restrict__ frames, int N, int H, int W, int Hp, int Wp, int Cp,
                            float* __restrict__ x) {
    pdl_trigger();
    pdl_wait();
    const size_t pix = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= (size_t)Hp * Wp) return;
    const int h = (int)(pix / Wp), w = (int)(pix % Wp);
    const int sh = h < H ? h : H - 1, sw = w < W ? w : W - 1;
    float* o = x + pix * Cp;
    float cur[3] = {0.f, 0.f, 0.f};
    int cur_n = -1;
    for (int c0 = 0; c0 < Cp; c0 += 4) {
        float v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = c0 + j, n = c / 3;
            if (n < N && n != cur_n) { px_values<FMT>(frames, n, sh, sw, H, W, cur); cur_n = n; }
            v[j] = (n < N) ? cur[c - 3 * n] : 0.0f;
        }
        *reinterpret_cast<float4*>(o + c0) = make_float4(v[0], v[1], v[2], v[3]);
    }
}

void launch_pack(const uint8_t* frames, int N, int H, int W, int Hp, int Wp, int Cp, float* x, cudaStream_t s,
                 int fmt) {
    const size_t npix = (size_t)Hp * Wp;
    const dim3 g((unsigned)((npix + 255) / 256));
    switch (fmt) {
        case 1: (void)launch_pdl(pack_kernel<1>, g, dim3(256), 0, s, frames, N, H, W, Hp, Wp, Cp, x); break;
        case 2: (void)launch_pdl(pack_kernel<2>, g, dim3(256), 0, s, frames, N, H, W, Hp, Wp, Cp, x); break;
        case 3: (void)launch_pdl(pack_kernel<3>, g, dim3(256), 0, s, frames, N, H, W, Hp, Wp, Cp, x); break;
        default: (void)launch_pdl(pack_kernel<0>, g, dim3(256), 0, s, frames, N, H, W, Hp, Wp, Cp, x); break;
    }
}

// bf16 bits of frame n's three channels times in_scale: bytes through the table (v / 255, or v / 256 for
// in_scale = 255 / 256), BT.709 in float
template <int FMT>
__device__ __forceinline__ void px_bf16(const uint8_t* __restrict__ fr, int n, int sh, int sw, int H, int W,
                                        const uint16_t* lut, float in_scale, uint32_t& b0, uint32_t& b1,
                                        uint32_t& b2) {
    uint32_t b[3];
    px_bytes<FMT>(fr, n, sh, sw, H, W, b);
    if (FMT == 1) {
        float v[3];
        bt709_from_bytes(b, v);
        b0 = __bfloat16_as_ushort(__float2bfloat16_rn(v[0] * in_scale));
        b1 = __bfloat16_as_ushort(__float2bfloat16_rn(v[1] * in_scale));
        b2 = __bfloat16_as_ushort(__float2bfloat16_rn(v[2] * in_scale));
    } else {
        b0 = lut[b[0]]; b1 = lut[b[1]]; b2 = lut[b[2]];
    }
}

__device__ __forceinline__ uint32_t pack_bf16_pair(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// bf16 variant for the tensor-core path (rows of CP = 32 or 64 channels, 3N <= CP of them real).  A block
// packs a segment of 128 pixels of one row, one thread per pixel: the thread reads its 3N bytes (a warp
// reads 96 consecutive bytes of each frame row), converts them, and writes its row into a shared-memory
// tile (16-byte chunk k of row p at chunk k ^ (p % chunks): no bank conflicts); the block then copies the
// tile to global memory with consecutive threads writing consecutive 16-byte chunks.
constexpr int kPackPix = 128;

template <int CP, int FMT>
__global__ void __launch_bounds__(kPackPix) pack_bf16_kernel(const uint8_t* __restrict__ frames, int N, int H,
                                                             int W, int Hp, int Wp, __nv_bfloat16* __restrict__ x) {
    pdl_trigger();
    pdl_wait();
    constexpr int KC = CP / 8;  // 16-byte chunks per pixel row
    __shared__ uint4 tile[kPackPix * KC];
    __shared__ uint16_t lut[256];  // bf16 bits of v / 255 (a division per entry, not per pixel)
    for (int v = threadIdx.x; v < 256; v += blockDim.x) lut[v] = __bfloat16_as_ushort(__float2bfloat16_rn(v / 255.0f));
    __syncthreads();
    const int p = threadIdx.x, w0 = blockIdx.x * kPackPix, w = w0 + p;
    const int sw = w < W ? w : W - 1;  // replicate the last column
    for (int h = blockIdx.y; h < Hp; h += gridDim.y) {
        const int sh = h < H ? h : H - 1;  // replicate the last row
        uint32_t pk[32];
#pragma unroll
        for (int n = 0; n < 16; ++n) {
            // channels 3n, 3n+1, 3n+2 -> bf16 halves 3n .. 3n+2 of the packed row
            uint32_t b0 = 0, b1 = 0, b2 = 0;
            if (n < N) px_bf16<FMT>(frames, n, sh, sw, H, W, lut, 1.0f, b0, b1, b2);
            // halves 3n, 3n+1, 3n+2 land in words (3n)/2 .. (3n+2)/2 (n even: w, w, w+1 low; n odd: w high, w+1)
            if ((n & 1) == 0) {
                pk[3 * n / 2] = b0 | (b1 << 16);
                pk[3 * n / 2 + 1] = b2;
            } else {
                pk[(3 * n - 1) / 2] |= b0 << 16;
                pk[(3 * n + 1) / 2] = b1 | (b2 << 16);
            }
        }
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const uint4 c = k < 6 ? make_uint4(pk[4 * k], pk[4 * k + 1], pk[4 * k + 2], pk[4 * k + 3])
                                  : make_uint4(0u, 0u, 0u, 0u);
            tile[p * KC + (k ^ (p & (KC - 1)))] = c;
        }
        __syncthreads();
        uint4* dst = reinterpret_cast<uint4*>(x + ((size_t)h * Wp + w0) * CP);
#pragma unroll
        for (int i = 0; i < KC; ++i) {
            const int idx = p + kPackPix * i, pr = idx / KC, k = idx % KC;
            if (w0 + pr < Wp) dst[idx] = tile[pr * KC + (k ^ (pr & (KC - 1)))];
        }
        __syncthreads();
    }
}

// Space-to-depth variant (3N <= 32) for the first layer's 2x2 form: pixel (h, w) becomes sub-pixel
// (h & 1, w & 1) of super-pixel (h / 2, w / 2), whose 128 channels are [2 (h & 1) + (w & 1)][32].  A block
// packs a 128-pixel segment of both rows of a super-row, so its 64 super-pixels (16 KB) are written as one
// contiguous run; shared-memory chunk c (16 bytes) of the segment is kept at c ^ ((c >> 4) & 7).  Values
// are x * kS2dInScale: a byte v becomes v / 256, exact in bf16 (the 2x2 weights carry the inverse factor).
template <int FMT>
__global__ void __launch_bounds__(kPackPix) pack_bf16_s2d_kernel(const uint8_t* __restrict__ frames, int N, int H,
                                                                 int W, int Hp, int Wp, __nv_bfloat16* __restrict__ x) {
    pdl_trigger();
    pdl_wait();
    __shared__ uint4 tile[kPackPix * 8];
    __shared__ uint16_t lut[256];
    for (int v = threadIdx.x; v < 256; v += blockDim.x) lut[v] = __bfloat16_as_ushort(__float2bfloat16_rn(v / 256.0f));
    __syncthreads();
    const int p = threadIdx.x, w0 = blockIdx.x * kPackPix, w = w0 + p;
    const int sw = w < W ? w : W - 1;  // replicate the last column
    const int Ws = Wp >> 1, npix = Wp - w0 < kPackPix ? Wp - w0 : kPackPix;
    for (int Y = blockIdx.y; Y < (Hp >> 1); Y += gridDim.y) {
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const int h = 2 * Y + dy, sh = h < H ? h : H - 1;  // replicate the last row
            uint32_t pk[24];
#pragma unroll
            for (int n = 0; n < 16; ++n) {
                uint32_t b0 = 0, b1 = 0, b2 = 0;
                if (n < N) px_bf16<FMT>(frames, n, sh, sw, H, W, lut, kS2dInScale, b0, b1, b2);
                if ((n & 1) == 0) {
                    pk[3 * n / 2] = b0 | (b1 << 16);
                    pk[3 * n / 2 + 1] = b2;
                } else {
                    pk[(3 * n - 1) / 2] |= b0 << 16;
                    pk[(3 * n + 1) / 2] = b1 | (b2 << 16);
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint4 c = make_uint4(pk[4 * k], pk[4 * k + 1], pk[4 * k + 2], pk[4 * k + 3]);
                const int ch = (p >> 1) * 16 + dy * 8 + (p & 1) * 4 + k;  // chunk within the segment
                tile[ch ^ ((ch >> 4) & 7)] = c;
            }
        }
        __syncthreads();
        uint4* dst = reinterpret_cast<uint4*>(x) + ((size_t)Y * Ws + (w0 >> 1)) * 16;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int ch = p + kPackPix * i;
            if ((ch >> 4) < (npix >> 1)) dst[ch] = tile[ch ^ ((ch >> 4) & 7)];  // super-pixel ch / 16
        }
        __syncthreads();
    }
}

template <int FMT>
static void launch_pack_bf16_fmt(const uint8_t* frames, int N, int H, int W, int Hp, int Wp, int Cp,
                                 __nv_bfloat16* x, cudaStream_t s, bool s2d) {
    const dim3 grid((unsigned)((Wp + kPackPix - 1) / kPackPix), (unsigned)(Hp < 65535 ? Hp : 65535));
    if (Cp == 32 && s2d)  // Hp, Wp even
        (void)launch_pdl(pack_bf16_s2d_kernel<FMT>, dim3(dim3(grid.x, (unsigned)((Hp >> 1) < 65535 ? (Hp >> 1) : 65535))), dim3(kPackPix), (size_t)(0), s, frames, N, H, W, Hp, Wp, x);
    else if (Cp == 32)  // 3N <= 32
        (void)launch_pdl(pack_bf16_kernel<32, FMT>, dim3(grid), dim3(kPackPix), (size_t)(0), s, frames, N, H, W, Hp, Wp, x);
    else
        (void)launch_pdl(pack_bf16_kernel<64, FMT>, dim3(grid), dim3(kPackPix), (size_t)(0), s, frames, N, H, W, Hp, Wp, x);
}

void launch_pack_bf16(const uint8_t* frames, int N, int H, int W, int Hp, int Wp, int Cp, __nv_bfloat16* x,
                      cudaStream_t s, bool s2d, int fmt) {
    switch (fmt) {
        case 1: launch_pack_bf16_fmt<1>(frames, N, H, W, Hp, Wp, Cp, x, s, s2d); break;
        case 2: launch_pack_bf16_fmt<2>(frames, N, H, W, Hp, Wp, Cp, x, s, s2d); break;
        case 3: launch_pack_bf16_fmt<3>(frames, N, H, W, Hp, Wp, Cp, x, s, s2d); break;
        default: launch_pack_bf16_fmt<0>(frames, N, H, W, Hp, Wp, Cp, x, s, s2d); break;
    }
}

// E4M3 variant: the same segment scheme with 64-byte pixel rows; x = v / 255 is stored as the E4M3 code
// of x * 448 (the per-tensor scale of [0, 1] data: 1 / 448).
template <int FMT>
__global__ void __launch_bounds__(kPackPix) pack_fp8_kernel(const uint8_t* __restrict__ frames, int N, int H,
                                                            int W, int Hp, int Wp, uint8_t* __restrict__ x) {
    pdl_trigger();
    pdl_wait();
    __shared__ uint4 tile[kPackPix * 4];
    __shared__ uint8_t lut[256];
    for (int v = threadIdx.x; v < 256; v += blockDim.x)
        lut[v] = (uint8_t)__nv_cvt_float_to_fp8((v / 255.0f) * 448.0f, __NV_SATFINITE, __NV_E4M3);
    __syncthreads();
    const int p = threadIdx.x, w0 = blockIdx.x * kPackPix, w = w0 + p;
    const int sw = w < W ? w : W - 1;
    for (int h = blockIdx.y; h < Hp; h += gridDim.y) {
        const int sh = h < H ? h : H - 1;
        uint32_t pk[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) pk[i] = 0u;
#pragma unroll
        for (int n = 0; n < 16; ++n) {
            if (n < N) {
                uint32_t bytes[3], code[3];
                px_bytes<FMT>(frames, n, sh, sw, H, W, bytes);
                if (FMT == 1) {
                    float v[3];
                    bt709_from_bytes(bytes, v);
#pragma unroll
                    for (int c = 0; c < 3; ++c) code[c] = (uint8_t)__nv_cvt_float_to_fp8(v[c] * 448.0f, __NV_SATFINITE, __NV_E4M3);
                } else {
#pragma unroll
                    for (int c = 0; c < 3; ++c) code[c] = lut[bytes[c]];
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int b = 3 * n + c;  // byte b of the row: word b / 4, byte b % 4
                    pk[b >> 2] |= code[c] << (8 * (b & 3));
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) tile[p * 4 + (k ^ (p & 3))] = make_uint4(pk[4 * k], pk[4 * k + 1], pk[4 * k + 2], pk[4 * k + 3]);
        __syncthreads();
        uint4* dst = reinterpret_cast<uint4*>(x + ((size_t)h * Wp + w0) * 64);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int idx = p + kPackPix * i, pr = idx >> 2, k = idx & 3;
            if (w0 + pr < Wp) dst[idx] = tile[pr * 4 + (k ^ (pr & 3))];
        }
        __syncthreads();
    }
}

void launch_pack_fp8(const uint8_t* frames, int N, int H, int W, int Hp, int Wp, uint8_t* x, cudaStream_t s, int fmt) {
    const dim3 grid((unsigned)((Wp + kPackPix - 1) / kPackPix), (unsigned)(Hp < 65535 ? Hp : 65535));
    switch (fmt) {
        case 1: (void)launch_pdl(pack_fp8_kernel<1>, grid, dim3(kPackPix), 0, s, frames, N, H, W, Hp, Wp, x); break;
        case 2: (void)launch_pdl(pack_fp8_kernel<2>, grid, dim3(kPackPix), 0, s, frames, N, H, W, Hp, Wp, x); break;
        case 3: (void)launch_pdl(pack_fp8_kernel<3>, grid, dim3(kPackPix), 0, s, frames, N, H, W, Hp, Wp, x); break;
        default: (void)launch_pdl(pack_fp8_kernel<0>, grid, dim3(kPackPix), 0, s, frames, N, H, W, Hp, Wp, x); break;
    }
}

// [H][W][C] float -> E4M3 codes of value * inv, rows of pitch Wd pixels (C a multiple of 4)
__global__ void f32_to_e4m3_rows_kernel(const float4* a, int H, int W, int C4, float inv, uint8_t* out, int Wd) {
    pdl_trigger();
    pdl_wait();
    const size_t n = (size_t)H * W * C4;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / ((size_t)W * C4), rem = i - row * W * C4;
        const float4 v = a[i];
        const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(v.x * inv, v.y * inv), __NV_SATFINITE, __NV_E4M3);
        const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(v.z * inv, v.w * inv), __NV_SATFINITE, __NV_E4M3);
        *reinterpret_cast<uint32_t*>(out + (row * Wd * C4 + rem) * 4) = lo | (hi << 16);
    }
}

void launch_f32_to_e4m3_rows(const float* a, int H, int W, int C, float inv, uint8_t* out, int Wd, cudaStream_t s) {
    const size_t n = (size_t)H * W * (C / 4);
    const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 4096);
    (void)launch_pdl(f32_to_e4m3_rows_kernel, dim3(blocks ? blocks : 1), dim3(256), (size_t)(0), s, reinterpret_cast<const float4*>(a), H, W, C / 4, inv,
                                                             out, Wd);
}

// *slot = max(*slot, max |x[i]|) (slot zeroed by the caller); non-negative floats order as their bits
__global__ void absmax_kernel(const float* __restrict__ x, size_t n, float* slot) {
    pdl_trigger();
    pdl_wait();
    float m = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(x[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(slot), __float_as_int(m));
}

void launch_absmax(const float* x, size_t n, float* slot, cudaStream_t s) {
    const size_t blocks = std::min<size_t>((n + 255) / 256, 2048);
    (void)launch_pdl(absmax_kernel, dim3((unsigned)(blocks ? blocks : 1)), dim3(256), (size_t)(0), s, x, n, slot);
}

// ------------------------------------------------------------------------------------------------
// z^ quantisation and per-channel index.  iz[c] = #{k : S_c > T_k}, S_c = sum z^^2 (exact integer),
// T_k = floor(npos * exp(2 t_k)) precomputed on the host in FP64: S_c > npos e^{2 t_k} <=>
// ln sqrt(S_c / npos) > t_k, i.e. the nearest log bin of the channel's RMS.
// ------------------------------------------------------------------------------------------------
__global__ void zquant_kernel(const float* __restrict__ z, int npos, int cz, const uint64_t* __restrict__ zthr,
                              int16_t* __restrict__ zhat, uint8_t* __restrict__ iz) {
    pdl_trigger();
    pdl_wait();
    const int c = blockIdx.x;
    unsigned long long S = 0;
    for (int p = threadIdx.x; p < npos; p += blockDim.x) {
        const float v = fminf(fmaxf(rintf(z[(size_t)p * cz + c]), -255.0f), 255.0f);
        const int q = (int)v;
        zhat[(size_t)p * cz + c] = (int16_t)q;
        S += (unsigned long long)(q * q);
    }
    __shared__ unsigned long long red[256];
    red[threadIdx.x] = S;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int k = 0;
        for (int j = 0; j < kBins - 1; ++j) k += red[0] > zthr[j];
        iz[c] = (uint8_t)k;
    }
}

void launch_zquant(const float* z, int npos, int cz, const uint64_t* zthr, int16_t* zhat, uint8_t* iz,
                   cudaStream_t s) {
    (void)launch_pdl(zquant_kernel, dim3(cz), dim3(256), (size_t)(0), s, z, npos, cz, zthr, zhat, iz);
}

// ------------------------------------------------------------------------------------------------
// quantize / scale index
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ int count_below(const float* thr, float v) {
    // #{k : thr[k] < v} for the 63 ascending thresholds (binary search)
    int lo = 0, hi = kBins - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (thr[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void quantize_kernel(const float* __restrict__ y, const float* __restrict__ mu,
                                const float* __restrict__ logsig, size_t n, const float* __restrict__ thr_all,
                                const float* __restrict__ qinv_all, const int* qp_dev, int qp_host,
                                int16_t* __restrict__ rhat, uint8_t* __restrict__ idx) {
    pdl_trigger();
    pdl_wait();
    __shared__ float thr[kBins - 1];
    const int qp = qp_dev ? *qp_dev : qp_host;
    if (threadIdx.x < kBins - 1) thr[threadIdx.x] = thr_all[qp * (kBins - 1) + threadIdx.x];
    __syncthreads();
    const float qinv = qinv_all[qp];
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        if (rhat) {
            // explicit round-to-nearest ops: no FMA contraction, same result on every launch
            const float r = rintf(__fmul_rn(__fsub_rn(y[i], mu[i]), qinv));
            rhat[i] = (int16_t)fminf(fmaxf(r, -255.0f), 255.0f);
        }
        idx[i] = (uint8_t)count_below(thr, logsig[i]);
    }
}

static unsigned grid_for(size_t n, int per_block) {
    size_t g = (n + per_block - 1) / per_block;
    if (g > 148 * 16) g = 148 * 16;
    return (unsigned)(g ? g : 1);
}

void launch_quantize(const float* y, const float* mu, const float* logsig, size_t n, const float* thr_all,
                     const float* qinv_all, const int* qp_dev, int qp_host, int16_t* rhat, uint8_t* idx,
                     cudaStream_t s) {
    (void)launch_pdl(quantize_kernel, dim3(grid_for(n, 256)), dim3(256), (size_t)(0), s, y, mu, logsig, n, thr_all, qinv_all, qp_dev, qp_host, rhat, idx);
}

void launch_scale_index(const float* logsig, size_t n, const float* thr_all, const int* qp_dev, uint8_t* idx,
                        cudaStream_t s) {
    (void)launch_pdl(quantize_kernel, dim3(grid_for(n, 256)), dim3(256), (size_t)(0), s, nullptr, nullptr, logsig, n, thr_all, thr_all, qp_dev, 0,
                                                    nullptr, idx);
}

__global__ void i16_to_f32_kernel(const int16_t* a, size_t n, float* out) {
    pdl_trigger();
    pdl_wait();
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (float)a[i];
}

void launch_i16_to_f32(const int16_t* a, size_t n, float* out, cudaStream_t s) {
    (void)launch_pdl(i16_to_f32_kernel, dim3(grid_for(n, 256)), dim3(256), (size_t)(0), s, a, n, out);
}

__global__ void f32_to_bf16_kernel(const float* a, size_t n, __nv_bfloat16* out) {
    pdl_trigger();
    pdl_wait();
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(a[i]);
}

void launch_f32_to_bf16(const float* a, size_t n, __nv_bfloat16* out, cudaStream_t s) {
    (void)launch_pdl(f32_to_bf16_kernel, dim3(grid_for(n, 256)), dim3(256), (size_t)(0), s, a, n, out);
}

// [H][W][C] float -> bf16 rows of pitch Wd pixels (C a multiple of 4); positions beyond W are left as they are
__global__ void f32_to_bf16_rows_kernel(const float4* a, int H, int W, int C4, __nv_bfloat16* out, int Wd) {
    pdl_trigger();
    pdl_wait();
    const size_t n = (size_t)H * W * C4;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / ((size_t)W * C4), rem = i - row * W * C4;
        const float4 v = a[i];
        __nv_bfloat162* d = reinterpret_cast<__nv_bfloat162*>(out + (row * Wd * C4 + rem) * 4);
        d[0] = __floats2bfloat162_rn(v.x, v.y);
        d[1] = __floats2bfloat162_rn(v.z, v.w);
    }
}

void launch_f32_to_bf16_rows(const float* a, int H, int W, int C, __nv_bfloat16* out, int Wd, cudaStream_t s) {
    const size_t n = (size_t)H * W * (C / 4);
    (void)launch_pdl(f32_to_bf16_rows_kernel, dim3(grid_for(n, 256)), dim3(256), (size_t)(0), s, reinterpret_cast<const float4*>(a), H, W, C / 4, out, Wd);
}

// ------------------------------------------------------------------------------------------------
// rANS encode: one thread per lane, lanes of up to two sections in one launch.  Each lane runs its
// elements backwards (last first) and writes its words backwards into its scratch row, so that the
// row's tail [cap_lane - words, cap_lane) is the lane stream in decoding order.
// ------------------------------------------------------------------------------------------------
struct RansSecPair { RansSection s[2]; int nsec; long long spin; };

// Lanes per block: small blocks spread the lanes over the SMs (each block holds its own copy of the
// tables), so that the lanes' dependent chains do not queue behind each other on one SM's shared
// memory: the 4096 lanes of a 1080p latent section run on 128 SMs (decode) or the 2 x 4096 of the two
// encoded sections on 128 SMs (encode).
constexpr int kRansThreadsEnc = 64;
constexpr int kRansThreadsDec = 32;

// Loads issued where they stand: the per-lane prefetches below must not be moved down next to their use.
__device__ __forceinline__ int ld_early_u8(const uint8_t* p) {
    unsigned short v;
    asm volatile("ld.global.nc.u8 %0, [%1];" : "=h"(v) : "l"(p));
    return (int)v;
}
__device__ __forceinline__ int ld_early_s16(const int16_t* p) {
    short v;
    asm volatile("ld.global.nc.s16 %0, [%1];" : "=h"(v) : "l"(p));
    return (int)v;
}
__device__ __forceinline__ uint32_t ld_early_u16(const uint16_t* p) {
    unsigned short v;
    asm volatile("ld.global.nc.u16 %0, [%1];" : "=h"(v) : "l"(p));
    return (uint32_t)v;
}
constexpr int kTabBytes = kBins * kNsym * 4;       // 130816, a multiple of 16
constexpr int kCoarseBytes = kBins * kCoarse * 2 + kBins * 4;  // 65792: bucket owners, then end-run lengths
constexpr int kPF = 16;                            // per-lane prefetch depth (symbols / table indices)
constexpr long long kLoadSpin = 4000000000LL;      // ~2 s bounded wait for the table copy

// The packed tables (and optionally the coarse decoding index) land in shared memory by TMA bulk copies
// issued by one thread; every thread waits on the copy's mbarrier for at most `spin` clocks (0: about
// 2 s).  Returns false (and records UFVC_ERR_TIMEOUT) if the copy did not complete in time; the issuing
// thread then waits once more, for at most about 2 s, for its copies in flight before the block exits.
__device__ __forceinline__ bool load_tables(uint32_t* tab, const uint32_t* __restrict__ tables, uint16_t* coarse,
                                            const uint16_t* __restrict__ coarse_g, uint64_t* bar, int* status,
                                            long long spin) {
    if (spin <= 0) spin = kLoadSpin;
    if (threadIdx.x == 0) {
        ptx::mbar_init(bar, 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ptx::mbar_arrive_expect_tx(bar, kTabBytes + (coarse ? kCoarseBytes : 0));
        for (int off = 0; off < kTabBytes; off += 32768) {
            const int n = kTabBytes - off < 32768 ? kTabBytes - off : 32768;
            ptx::bulk_load(reinterpret_cast<uint8_t*>(tab) + off, reinterpret_cast<const uint8_t*>(tables) + off, n, bar);
        }
        if (coarse)
            for (int off = 0; off < kCoarseBytes; off += 32768) {
                const int n = kCoarseBytes - off < 32768 ? kCoarseBytes - off : 32768;
                ptx::bulk_load(reinterpret_cast<uint8_t*>(coarse) + off,
                               reinterpret_cast<const uint8_t*>(coarse_g) + off, n, bar);
            }
    }
    const long long t0 = clock64();
    while (!ptx::mbar_try_wait(bar, 0)) {
        if (clock64() - t0 > spin) {
            set_status(status, UFVC_ERR_TIMEOUT);
            if (threadIdx.x == 0) {  // the issuing thread waits once more, bounded, for its copies in flight
                const long long t1 = clock64();
                while (!ptx::mbar_try_wait(bar, 0) && clock64() - t1 < kLoadSpin) {
                }
            }
            return false;  // (no block barrier here: threads may reach this point at different times)
        }
    }
    return true;
}

// rANS encode: one thread per lane, lanes of up to two sections in one launch.  Each lane runs its
// elements backwards (last first) and writes its words backwards into its scratch row, so that the
// row's tail [cap_lane - words, cap_lane) is the lane stream in decoding order.  The step has no branch:
// the renormalisation word is stored under a predicate, and out-of-range inputs are clamped and
// reported once per lane.
__global__ void __launch_bounds__(kRansThreadsEnc) rans_encode_kernel(const RansSecPair P,
                                                                   const uint32_t* __restrict__ tables) {
    extern __shared__ __align__(16) uint32_t tab[];  // [64][511] (freq << 16) | cum
    __shared__ uint64_t bar;
    int lane = blockIdx.x * blockDim.x + threadIdx.x;
    int si = 0;
    if (lane >= P.s[0].K) { lane -= P.s[0].K; si = 1; }
    const bool mine = si < P.nsec && lane < P.s[si].K;
    if (!load_tables(tab, tables, nullptr, nullptr, &bar, P.s[0].status, P.spin)) {
        // no words for this lane: a zero count, which the layout kernels refuse to copy
        if (mine) {
            pdl_wait();
            P.s[si].counts[lane] = 0;
        }
        return;
    }
    pdl_trigger();  // the tables above are constants: loaded while the previous kernel finishes
    pdl_wait();
    if (!mine) return;
    const RansSection& S = P.s[si];
    const size_t n = S.n;
    const int K = S.K, per = S.idx_period;
    const int cnt = (size_t)lane < n ? (int)((n - lane + K - 1) / K) : 0;
    uint16_t* row = S.scratch + (size_t)lane * S.cap_lane;
    int wp = S.cap_lane;
    uint32_t x = kRansL, bad = 0;
    const int16_t* sym = S.sym + lane;
    const uint8_t* idx = S.idx + lane;
    // The (table, symbol) pairs of the next kPF elements are fetched while the current kPF are coded,
    // so the serial state chain does not wait on memory.
    int tc[kPF], vc[kPF], tn[kPF], vn[kPF];
    auto fetch = [&](int mtop, int* td, int* vd) {
        if (per) {
#pragma unroll
            for (int u = 0; u < kPF; ++u) {
                const int m = mtop - u;
                td[u] = 0;
                vd[u] = 0;
                if (m >= 0) {
                    td[u] = ld_early_u8(S.idx + ((size_t)lane + (size_t)m * K) % (size_t)per);
                    vd[u] = ld_early_s16(sym + (size_t)m * K);
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < kPF; ++u) {
                const int m = mtop - u;
                td[u] = 0;
                vd[u] = 0;
                if (m >= 0) {
                    td[u] = ld_early_u8(idx + (size_t)m * K);
                    vd[u] = ld_early_s16(sym + (size_t)m * K);
                }
            }
        }
    };
    auto step = [&](int t, int v) {
        v += kRmax;
        const bool ok = (uint32_t)t < (uint32_t)kBins && (uint32_t)v < (uint32_t)kNsym;
        bad |= !ok;
        const uint32_t e = tab[ok ? t * kNsym + v : kRmax];
        const uint32_t f = e >> 16, c = e & 0xFFFFu;
        const bool o = x >= (f << 16);  // f << 16 < 2^32 as f <= 65026
        if (o) row[wp - 1] = (uint16_t)(x & 0xFFFFu);
        wp -= o ? 1 : 0;
        x = o ? x >> 16 : x;
        const uint32_t q = x / f;
        x = (q << 16) + (x - q * f) + c;
    };
    fetch(cnt - 1, tc, vc);
    int mtop = cnt - 1;
    for (; mtop >= kPF - 1; mtop -= kPF) {  // full blocks of kPF elements
        fetch(mtop - kPF, tn, vn);
#pragma unroll
        for (int u = 0; u < kPF; ++u) step(tc[u], vc[u]);
#pragma unroll
        for (int u = 0; u < kPF; ++u) { tc[u] = tn[u]; vc[u] = vn[u]; }
    }
#pragma unroll
    for (int u = 0; u < kPF; ++u)  // the remaining mtop + 1 < kPF elements
        if (u <= mtop) step(tc[u], vc[u]);
    if (bad) set_status(S.status, UFVC_ERR_ARG);
    row[--wp] = (uint16_t)(x & 0xFFFFu);
    row[--wp] = (uint16_t)(x >> 16);
    S.counts[lane] = (uint32_t)(S.cap_lane - wp);
}

void launch_rans_encode(const RansSection* secs, int nsec, const uint32_t* packed_tables, cudaStream_t s,
                        long long spin) {
    RansSecPair P{};
    P.nsec = nsec;
    P.spin = spin;
    int total = 0;
    for (int i = 0; i < nsec; ++i) { P.s[i] = secs[i]; total += secs[i].K; }
    (void)smem_optin((const void*)rans_encode_kernel, kTabBytes);
    (void)launch_pdl(rans_encode_kernel, dim3((total + kRansThreadsEnc - 1) / kRansThreadsEnc), dim3(kRansThreadsEnc), (size_t)(kTabBytes), s, P, packed_tables);
}

// ------------------------------------------------------------------------------------------------
// rANS finalize: single block scans the lane counts of each section, writes them and the section
// padding, and records each lane's destination byte offset; then a copy kernel moves the words.
// Nothing is written at or past `capacity`.
// ------------------------------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
using BlockScanU64 = cub::BlockScan<unsigned long long, kScanThreads>;

__global__ void __launch_bounds__(kScanThreads) rans_finalize_kernel(const RansSecPair P, uint8_t* out,
                                                                     size_t hdr_bytes, size_t capacity,
                                                                     uint64_t* nbytes, uint64_t* off_ws,
                                                                     int* status) {
    pdl_trigger();
    pdl_wait();
    __shared__ typename BlockScanU64::TempStorage tmp;
    __shared__ unsigned long long base_sh;
    if (threadIdx.x == 0) base_sh = hdr_bytes;
    __syncthreads();
    size_t ws_base = 0;
    for (int si = 0; si < P.nsec; ++si) {
        const RansSection& S = P.s[si];
        const int K = S.K;
        const int per = (K + kScanThreads - 1) / kScanThreads;
        const int j0 = threadIdx.x * per;
        // a lane holds 2 .. cap_lane words; any other count comes from a lane whose encoder stopped early
        // (its table copy timed out): it is laid out as empty and reported
        auto count = [&](int j) -> uint32_t {
            const uint32_t c = S.counts[j];
            return c >= 2 && c <= (uint32_t)S.cap_lane ? c : 0u;
        };
        unsigned long long local = 0;
        bool bad = false;
        for (int j = j0; j < j0 + per && j < K; ++j) {
            const uint32_t c = count(j);
            bad |= c == 0;
            local += c;
        }
        if (bad) set_status(status, UFVC_ERR_TIMEOUT);
        unsigned long long excl, total;
        BlockScanU64(tmp).ExclusiveSum(local, excl, total);
        const unsigned long long base = base_sh;
        const unsigned long long words_at = base + 4ull * K;
        for (int j = j0; j < j0 + per && j < K; ++j) {
            const uint32_t c = count(j);
            off_ws[ws_base + j] = words_at + 2ull * excl;
            excl += c;
            const size_t cp = base + 4ull * j;
            if (cp + 4 <= capacity) {
                out[cp] = c & 0xFF; out[cp + 1] = (c >> 8) & 0xFF; out[cp + 2] = (c >> 16) & 0xFF; out[cp + 3] = c >> 24;
            }
        }
        const unsigned long long end = words_at + 2ull * total;
        const unsigned long long end4 = (end + 3) & ~3ull;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (unsigned long long b = end; b < end4; ++b)
                if (b < capacity) out[b] = 0;
            base_sh = end4;
        }
        __syncthreads();
        ws_base += K;
    }
    if (threadIdx.x == 0) {
        *nbytes = base_sh;
        if (base_sh > capacity) set_status(status, UFVC_ERR_CAPACITY);
    }
}

__global__ void rans_copy_kernel(const RansSecPair P, uint8_t* out, size_t capacity, const uint64_t* off_ws) {
    pdl_trigger();
    pdl_wait();
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, l = threadIdx.x & 31;
    int lane = warp, si = 0;
    size_t ws = 0;
    if (lane >= P.s[0].K) { lane -= P.s[0].K; si = 1; ws = P.s[0].K; }
    if (si >= P.nsec || lane >= P.s[si].K) return;
    const RansSection& S = P.s[si];
    const uint32_t words = S.counts[lane];
    if (words < 2 || words > (uint32_t)S.cap_lane) return;  // reported by the finaliser
    const uint16_t* src = S.scratch + (size_t)lane * S.cap_lane + (S.cap_lane - words);
    const uint64_t dst = off_ws[ws + lane];
    if (dst + 2ull * words > capacity) return;  // status already records the capacity error
    uint16_t* d = reinterpret_cast<uint16_t*>(out + dst);
    for (uint32_t w = l; w < words; w += 32) d[w] = src[w];
}

void launch_rans_finalize(const RansSection* secs, int nsec, uint8_t* out, size_t hdr_bytes, size_t capacity,
                          uint64_t* nbytes, uint64_t* offsets_ws, int* status, cudaStream_t s) {
    RansSecPair P{};
    P.nsec = nsec;
    int total = 0;
    for (int i = 0; i < nsec; ++i) { P.s[i] = secs[i]; total += secs[i].K; }
    (void)launch_pdl(rans_finalize_kernel, dim3(1), dim3(kScanThreads), (size_t)(0), s, P, out, hdr_bytes, capacity, nbytes, offsets_ws, status);
    const int threads = 256;
    (void)launch_pdl(rans_copy_kernel, dim3((unsigned)(((size_t)total * 32 + threads - 1) / threads)), dim3(threads), (size_t)(0), s, P, out, capacity,
                                                                                               offsets_ws);
}

// ------------------------------------------------------------------------------------------------
// rANS decode.  parse: single block reads the K lane counts of a section, checks 2 <= words <= n_j + 2
// and that the section fits in the stream, and produces each lane's byte offset.  decode: one thread
// per lane; every read stays inside the lane's words; a lane that ends with a state != 2^16 or with
// unread / missing words marks the stream corrupt.
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kScanThreads) rans_parse_kernel(const RansDecodeJob J, size_t expect_end_host,
                                                                  const uint64_t* expect_end_dev, int* status) {
    pdl_trigger();
    pdl_wait();
    __shared__ typename BlockScanU64::TempStorage tmp;
    __shared__ int bad, prior;
    if (threadIdx.x == 0) { bad = 0; prior = *status; }
    __syncthreads();
    if (prior != 0) return;
    const size_t expect_end = expect_end_dev ? (size_t)*expect_end_dev : expect_end_host;
    const unsigned long long off = J.sec_off_dev ? *J.sec_off_dev : J.sec_off_host;
    const int K = J.K;
    const size_t n = J.n;
    if (off + 4ull * K > J.nbytes) {
        if (threadIdx.x == 0) set_status(status, UFVC_ERR_CORRUPT);
        return;
    }
    const int per = (K + kScanThreads - 1) / kScanThreads;
    const int j0 = threadIdx.x * per;
    unsigned long long local = 0;
    for (int j = j0; j < j0 + per && j < K; ++j) {
        const uint8_t* p = J.bits + off + 4ull * j;
        const uint32_t c = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
        const size_t cnt = (size_t)j < n ? (n - j + K - 1) / K : 0;
        if (c < 2 || c > cnt + 2) bad = 1;
        local += c;
    }
    unsigned long long excl, total;
    BlockScanU64(tmp).ExclusiveSum(local, excl, total);
    __syncthreads();
    const unsigned long long words_at = off + 4ull * K;
    const unsigned long long end4 = (words_at + 2ull * total + 3) & ~3ull;
    const bool fits = end4 <= J.nbytes && (expect_end == 0 || end4 == expect_end);
    if (bad || !fits) {
        if (threadIdx.x == 0) set_status(status, UFVC_ERR_CORRUPT);
        return;
    }
    for (int j = j0; j < j0 + per && j < K; ++j) {
        const uint8_t* p = J.bits + off + 4ull * j;
        const uint32_t c = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
        J.lane_off[j] = words_at + 2ull * excl;
        J.lane_words[j] = c;
        excl += c;
    }
    if (threadIdx.x == 0 && J.next_off) *J.next_off = end4;
}

void launch_rans_parse(const RansDecodeJob& j, int* status, cudaStream_t s) {
    (void)launch_pdl(rans_parse_kernel, dim3(1), dim3(kScanThreads), (size_t)(0), s, j, 0, nullptr, status);
}

void launch_rans_parse_expect(const RansDecodeJob& j, size_t expect_end, const uint64_t* expect_end_dev, int* status,
                              cudaStream_t s) {
    (void)launch_pdl(rans_parse_kernel, dim3(1), dim3(kScanThreads), (size_t)(0), s, j, expect_end, expect_end_dev, status);
}

// rANS decode.  Each thread runs LPT lanes (g, g + G, ... with G = ceil(K / LPT)), their steps interleaved
// so the serial state chains of different lanes overlap in one instruction stream.  PER: the table index
// of element i is idx[i mod idx_period] (the hyper-latent's per-channel tables) instead of idx[i].
// The common path of a step has no branch: the slot's bucket gives the candidate symbols, one predicated
// bisection step settles buckets of one or two candidates, and only wider buckets (table tails) enter a
// loop.  The renormalisation word is read every step at the lane's read position (a lane stream is read
// sequentially, so it stays in L1) and selected when the state drops below L.
template <int LPT, bool PER>
__global__ void __launch_bounds__(kRansThreadsDec) rans_decode_kernel(const RansDecodeJob J,
                                                                   const uint32_t* __restrict__ tables,
                                                                   const uint16_t* __restrict__ coarse_g, int* status,
                                                                   long long spin) {
    extern __shared__ __align__(16) uint32_t tab[];                      // [64][511] (freq << 16) | cum
    uint16_t* coarse = reinterpret_cast<uint16_t*>(tab + kBins * kNsym);  // [64][kCoarse], then [64] end runs
    const uint32_t* runs = reinterpret_cast<const uint32_t*>(coarse + kBins * kCoarse);  // A | B << 16
    __shared__ uint64_t bar;
    if (!load_tables(tab, tables, coarse, coarse_g, &bar, status, spin)) return;
    pdl_trigger();  // the tables above are constants: loaded while the previous kernel finishes
    pdl_wait();
    if (*(volatile int*)status != 0) return;
    const int K = J.K, G = (K + LPT - 1) / LPT;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const size_t n = J.n;
    int cnt[LPT], lane[LPT];
    bool live[LPT];
    uint32_t x[LPT], r[LPT], words[LPT];
    const uint16_t* wp[LPT];
    const uint8_t* ip[LPT];
    int16_t* sp[LPT];
    int cmin = 1 << 30;
#pragma unroll
    for (int j = 0; j < LPT; ++j) {
        lane[j] = g + j * G;
        live[j] = lane[j] < K;
        const int l = live[j] ? lane[j] : g;  // a thread's missing lane mirrors its first lane, with no symbols
        cnt[j] = live[j] && (size_t)l < n ? (int)((n - l + K - 1) / K) : 0;
        if (live[j]) cmin = cnt[j] < cmin ? cnt[j] : cmin;
        wp[j] = reinterpret_cast<const uint16_t*>(J.bits + J.lane_off[l]);
        words[j] = J.lane_words[l];  // >= 2 (checked by the parse)
        x[j] = ((uint32_t)wp[j][0] << 16) | wp[j][1];
        r[j] = 2;
        ip[j] = J.idx + l;
        sp[j] = J.sym + l;
    }
    // table indices of the next kPF symbols of every lane are fetched while the current kPF are decoded
    int tc[LPT][kPF], tn[LPT][kPF];
    auto fetch = [&](int m0, int (*td)[kPF]) {
#pragma unroll
        for (int j = 0; j < LPT; ++j)
#pragma unroll
            for (int u = 0; u < kPF; ++u) {
                const int m = m0 + u;
                td[j][u] = 0;
                if (m < cnt[j]) {
                    if (PER)
                        td[j][u] = ld_early_u8(J.idx + ((size_t)lane[j] + (size_t)m * K) % (size_t)J.idx_period);
                    else
                        td[j][u] = ld_early_u8(ip[j] + (size_t)m * K);
                }
            }
    };
    uint32_t bad = 0;
    // one symbol of every lane j with act[j]
    auto step = [&](const int* t_in, const bool* act) {
        int s[LPT], hi[LPT];
        uint32_t slot[LPT], w[LPT];
        const uint32_t* T[LPT];
#pragma unroll
        for (int j = 0; j < LPT; ++j) {
            int t = t_in[j];
            bad |= (uint32_t)t >= (uint32_t)kBins;
            t = (uint32_t)t < (uint32_t)kBins ? t : 0;
            T[j] = tab + t * kNsym;
            w[j] = __ldg(wp[j] + (r[j] < words[j] ? r[j] : words[j] - 1));
            slot[j] = x[j] & 0xFFFFu;
            const int b = (int)(slot[j] >> kCoarseShift);
            const uint16_t* C = coarse + t * kCoarse;
            const uint32_t ab = runs[t];
            const int A = (int)(ab & 0xFFFFu), B = (int)(ab >> 16), sl = (int)slot[j];
            // symbol s with cum(s) <= slot < cum(s+1): in the unit-frequency end runs it is the slot itself
            // (shifted on the right), elsewhere it lies in [owner of the bucket's first slot, owner of the
            // next bucket's first slot], clipped to the middle [A, 510 - B]
            const bool tail_l = sl < A, tail_r = sl >= (int)kProbM - B;
            const int lo = max((int)C[b], A), up = min(b + 1 < kCoarse ? (int)C[b + 1] : kNsym - 1, kNsym - 1 - B);
            s[j] = tail_l ? sl : tail_r ? sl - ((int)kProbM - kNsym) : lo;
            hi[j] = tail_l || tail_r ? s[j] : up;
        }
        // the first bisection step is predicated (mid = s when s == hi)
        bool more = false;
#pragma unroll
        for (int j = 0; j < LPT; ++j) {
            const int mid = (s[j] + hi[j] + 1) >> 1;
            const bool le = (T[j][mid] & 0xFFFFu) <= slot[j];
            const bool go = s[j] < hi[j];
            s[j] = go && le ? mid : s[j];
            hi[j] = go && !le ? mid - 1 : hi[j];
            more |= s[j] < hi[j];
        }
        if (more) {
#pragma unroll
            for (int j = 0; j < LPT; ++j) {
                while (s[j] < hi[j]) {
                    const int mid = (s[j] + hi[j] + 1) >> 1;
                    if ((T[j][mid] & 0xFFFFu) <= slot[j]) s[j] = mid; else hi[j] = mid - 1;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < LPT; ++j) {
            const uint32_t e = T[j][s[j]];
            const uint32_t xn = (e >> 16) * (x[j] >> 16) + slot[j] - (e & 0xFFFFu);
            const bool rn = xn < kRansL;
            if (act[j]) {
                x[j] = rn ? (xn << 16) | w[j] : xn;
                r[j] += rn ? 1u : 0u;
                *sp[j] = (int16_t)(s[j] - kRmax);
                sp[j] += K;
            }
        }
    };
    fetch(0, tc);
    int m0 = 0;
    for (; m0 + kPF <= cmin; m0 += kPF) {  // full blocks: every live lane has all kPF symbols
        fetch(m0 + kPF, tn);
#pragma unroll
        for (int u = 0; u < kPF; ++u) {
            int tu[LPT];
#pragma unroll
            for (int j = 0; j < LPT; ++j) tu[j] = tc[j][u];
            step(tu, live);
        }
#pragma unroll
        for (int j = 0; j < LPT; ++j)
#pragma unroll
            for (int u = 0; u < kPF; ++u) tc[j][u] = tn[j][u];
    }
    // the tail: live lanes' counts differ by at most one, so at most kPF symbols per lane remain
#pragma unroll
    for (int u = 0; u < kPF; ++u) {
        int tu[LPT];
        bool act[LPT], any = false;
#pragma unroll
        for (int j = 0; j < LPT; ++j) {
            tu[j] = tc[j][u];
            act[j] = m0 + u < cnt[j];
            any |= act[j];
        }
        if (!any) break;
        step(tu, act);
    }
    if (bad) set_status(status, UFVC_ERR_ARG);
#pragma unroll
    for (int j = 0; j < LPT; ++j)
        if (live[j] && (x[j] != kRansL || r[j] != words[j])) set_status(status, UFVC_ERR_CORRUPT);
}

#ifndef UFVC_RANS_DEC_LPT
#define UFVC_RANS_DEC_LPT 1
#endif
constexpr int kRansDecLPT = UFVC_RANS_DEC_LPT;  // lanes per decoding thread

void launch_rans_decode(const RansDecodeJob& j, const uint32_t* packed_tables, const uint16_t* coarse, int* status,
                        cudaStream_t s, long long spin) {
    const int smem = kTabBytes + kCoarseBytes;
    (void)smem_optin((const void*)rans_decode_kernel<kRansDecLPT, false>, smem);
    (void)smem_optin((const void*)rans_decode_kernel<1, true>, smem);
    if (j.idx_period) {
        (void)launch_pdl(rans_decode_kernel<1, true>, dim3((j.K + kRansThreadsDec - 1) / kRansThreadsDec), dim3(kRansThreadsDec), (size_t)(smem), s, j, packed_tables, coarse, status, spin);
    } else {
        const int G = (j.K + kRansDecLPT - 1) / kRansDecLPT;
        (void)launch_pdl(rans_decode_kernel<kRansDecLPT, false>, dim3((G + kRansThreadsDec - 1) / kRansThreadsDec), dim3(kRansThreadsDec), (size_t)(smem), s, j, packed_tables, coarse, status, spin);
    }
}

// y^ = r^ q + mu (explicitly rounded ops), to float and / or bf16; q from the parsed rate
__global__ void dequant_kernel(const int16_t* __restrict__ rhat, const float* __restrict__ mu, size_t n,
                               const float* __restrict__ qstep_all, const int* __restrict__ qp_dev,
                               float* __restrict__ yf, __nv_bfloat16* __restrict__ yb, uint8_t* __restrict__ y8,
                               float inv8, int qp_host) {
    pdl_trigger();
    pdl_wait();
    const float q = qstep_all[qp_dev ? *qp_dev : qp_host];
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float v = __fadd_rn(__fmul_rn((float)rhat[i], q), mu[i]);
        if (yf) yf[i] = v;
        if (yb) yb[i] = __float2bfloat16_rn(v);
        if (y8) y8[i] = (uint8_t)__nv_cvt_float_to_fp8(v * inv8, __NV_SATFINITE, __NV_E4M3);
    }
}

void launch_dequant(const int16_t* rhat, const float* mu, size_t n, const float* qstep_all, const int* qp_dev,
                    float* yf, __nv_bfloat16* yb, cudaStream_t s, uint8_t* y8, float inv8, int qp_host) {
    (void)launch_pdl(dequant_kernel, dim3(grid_for(n, 256)), dim3(256), (size_t)(0), s, rhat, mu, n, qstep_all, qp_dev, yf,
                     yb, y8, inv8, qp_host);
}

// ------------------------------------------------------------------------------------------------
// container header
// ------------------------------------------------------------------------------------------------
__global__ void write_header_kernel(uint8_t* out, int version, int arch, int N, int qp, int W, int H, int K, int Kz,
                                    const uint8_t* iz, int Cz, size_t capacity, int* status) {
    pdl_trigger();
    pdl_wait();
    const size_t hdr = (20 + (size_t)Cz + 3) & ~(size_t)3;
    if (hdr > capacity) {
        if (threadIdx.x == 0) set_status(status, UFVC_ERR_CAPACITY);
        return;
    }
    for (int i = threadIdx.x; i < (int)hdr; i += blockDim.x) {
        uint8_t v = 0;
        if (i < 4) v = "UFVC"[i];
        else if (i == 4) v = (uint8_t)version;
        else if (i == 5) v = (uint8_t)arch;
        else if (i == 6) v = (uint8_t)N;
        else if (i == 7) v = (uint8_t)qp;
        else if (i < 10) v = (uint8_t)(W >> (8 * (i - 8)));
        else if (i < 12) v = (uint8_t)(H >> (8 * (i - 10)));
        else if (i < 16) v = (uint8_t)((uint32_t)K >> (8 * (i - 12)));
        else if (i < 20) v = (uint8_t)((uint32_t)Kz >> (8 * (i - 16)));
        else if (i < 20 + Cz) v = iz[i - 20];
        out[i] = v;
    }
}

void launch_write_header(uint8_t* out, int version, int arch, int N, int qp, int W, int H, int K, int Kz,
                         const uint8_t* iz, int Cz, size_t capacity, int* status, cudaStream_t s) {
    (void)launch_pdl(write_header_kernel, dim3(1), dim3(256), (size_t)(0), s, out, version, arch, N, qp, W, H, K, Kz, iz,
                     Cz, capacity, status);
}

__global__ void parse_header_kernel(const uint8_t* b, size_t nbytes, int arch, int N, int W, int H, int K, int Kz,
                                    int Cz, int allow_pm, int temporal, int* qp_dev, int* ver_dev, uint8_t* iz,
                                    int* status) {
    pdl_trigger();
    pdl_wait();
    if (threadIdx.x != 0) return;
    const size_t hdr = (20 + (size_t)Cz + 3) & ~(size_t)3;
    *qp_dev = 32;
    *ver_dev = 1;
    for (int c = 0; c < Cz; ++c) iz[c] = 0;
    if (nbytes < hdr || b[0] != 'U' || b[1] != 'F' || b[2] != 'V' || b[3] != 'C' || b[4] < 1 || b[4] > 4) {
        set_status(status, UFVC_ERR_CORRUPT);
        return;
    }
    const int v_pm = b[4] == 2 || b[4] == 4, v_tc = b[4] >= 3;
    // progressive means without a mean network, or a temporal-context mismatch with the context
    if ((v_pm && !allow_pm) || v_tc != temporal) {
        set_status(status, UFVC_ERR_UNSUPPORTED);
        return;
    }
    const int w = b[8] | (b[9] << 8), h = b[10] | (b[11] << 8);
    const uint32_t k = b[12] | (b[13] << 8) | (b[14] << 16) | ((uint32_t)b[15] << 24);
    const uint32_t kz = b[16] | (b[17] << 8) | (b[18] << 16) | ((uint32_t)b[19] << 24);
    if (b[5] != arch || b[6] != N || w != W || h != H) { set_status(status, UFVC_ERR_ARG); return; }
    if (b[7] > 63 || k != (uint32_t)K || kz != (uint32_t)Kz) { set_status(status, UFVC_ERR_CORRUPT); return; }
    for (int c = 0; c < Cz; ++c) {
        if (b[20 + c] >= kBins) { set_status(status, UFVC_ERR_CORRUPT); return; }
        iz[c] = b[20 + c];
    }
    *qp_dev = b[7];
    *ver_dev = v_pm ? 2 : 1;
}

void launch_parse_header(const uint8_t* bits, size_t nbytes, int arch, int N, int W, int H, int K, int Kz, int Cz,
                         bool allow_pm, bool temporal, int* qp_dev, int* ver_dev, uint8_t* iz, int* status,
                         cudaStream_t s) {
    (void)launch_pdl(parse_header_kernel, dim3(1), dim3(32), (size_t)(0), s, bits, nbytes, arch, N, W, H, K, Kz, Cz,
                     (int)allow_pm, (int)temporal, qp_dev, ver_dev, iz, status);
}

}  // namespace ufvc
