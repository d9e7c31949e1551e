// Elementwise and entropy-coding kernels.
//
//  * pack          : chunk frames uint8 [N][H][W][3] -> /255, replicate pad to x16, frames stacked into
//                    channels (frame n -> channels 3n..3n+2), zero channels up to the padded count
//                    (the patch-embedding input of Sec. 3.1).
//  * zquant        : z^ = clamp(rint(z), +-255) and the per-channel scale index of z^.
//  * quantize      : r^ = clamp(rint((y - mu) / q), +-255) and the scale index of log sigma (Sec. 3.4).
//  * dequant       : y^ = r^ q + mu where the progressive means (or the encoder's context tracking) need
//                    it as a pass of its own (the rANS decoder writes it directly otherwise, rans.cu).
#include "ufvc_internal.h"

#include <cuda_fp8.h>

#include <algorithm>
#include "tc_ptx.h"


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

}  // namespace ufvc
