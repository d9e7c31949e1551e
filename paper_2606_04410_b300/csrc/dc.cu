// DC-block model (Appendix: every module built from depth-wise convolution blocks, HT-S block counts):
// the three elementwise / depth-wise kernels it needs besides the library's 1x1 and 3x3 convolutions.
//
//   pack_s2d8   frames -> patch-embedding input [H8][W8][3N 64]: channel (3n + c) 64 + 8 dy + dx holds
//               frame n's channel c at pixel (8 h8 + dy, 8 w8 + dx) (replicate padding to multiples of 16);
//   dw_conv     depth-wise 3x3 (zero padding 1) + bias + GELU, NHWC, grouped (each group its own filters),
//               float activations (exact erf GELU) or bf16 (the tensor-core epilogues' GELU), float weights
//               [g][9][C];
//   ps8_out     the frame decoders' last 1x1 output o [N][H8][W8][192] -> x^ = clamp(0.5 + o, 0, 1) at
//               pixel (8 h8 + dy, 8 w8 + dx), channel c = o[.][.][64 c + 8 dy + dx], cropped, as uint8
//               rint(255 x^) or float.
// All three are bandwidth-bound; each thread moves 8 channels (16 or 32 bytes) at a time.
#include "ufvc_internal.h"

#include <cuda_bf16.h>

namespace ufvc {

namespace {

template <typename T>
__device__ __forceinline__ void ld8(const T* p, float* v);
template <>
__device__ __forceinline__ void ld8<float>(const float* p, float* v) {
    const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
template <>
__device__ __forceinline__ void ld8<__nv_bfloat16>(const __nv_bfloat16* p, float* v) {
    const uint4 u = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        v[2 * j] = __uint_as_float(w[j] << 16);
        v[2 * j + 1] = __uint_as_float(w[j] & 0xFFFF0000u);
    }
}

template <typename T>
__device__ __forceinline__ void st8(T* p, const float* v);
template <>
__device__ __forceinline__ void st8<float>(float* p, const float* v) {
    reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
}
template <>
__device__ __forceinline__ void st8<__nv_bfloat16>(__nv_bfloat16* p, const float* v) {
    uint4 u;
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
        w[j] = *reinterpret_cast<uint32_t*>(&h);
    }
    u.x = w[0]; u.y = w[1]; u.z = w[2]; u.w = w[3];
    *reinterpret_cast<uint4*>(p) = u;
}

// the caller's frame formats (see the pack kernels of the plain model): frame n's three channels
template <int FMT>
__device__ __forceinline__ void px3(const uint8_t* __restrict__ fr, int n, int sh, int sw, int H, int W, float* v) {
    uint32_t b[3];
    if (FMT <= 1) {
        const uint8_t* p = fr + ((size_t)n * H * W + (size_t)sh * W + sw) * 3;
        b[0] = p[0]; b[1] = p[1]; b[2] = p[2];
    } else if (FMT == 2) {
        const size_t pl = (size_t)H * W;
        const uint8_t* p = fr + (size_t)n * 3 * pl + (size_t)sh * W + sw;
        b[0] = p[0]; b[1] = p[pl]; b[2] = p[2 * pl];
    } else {
        const int Wc = (W + 1) >> 1, Hc = (H + 1) >> 1;
        const size_t pl = (size_t)H * W, cpl = (size_t)Hc * Wc;
        const uint8_t* f = fr + (size_t)n * (pl + 2 * cpl);
        const size_t ci = (size_t)(sh >> 1) * Wc + (sw >> 1);
        b[0] = f[(size_t)sh * W + sw]; b[1] = f[pl + ci]; b[2] = f[pl + cpl + ci];
    }
    const float r = b[0] / 255.0f, g = b[1] / 255.0f, bl = b[2] / 255.0f;
    if (FMT == 1) {  // BT.709 (full range, chroma centred at 0.5)
        const float y = fmaf(0.0722f, bl, fmaf(0.7152f, g, 0.2126f * r));
        v[0] = y;
        v[1] = fmaf(bl - y, 1.0f / 1.8556f, 0.5f);
        v[2] = fmaf(r - y, 1.0f / 1.5748f, 0.5f);
    } else {
        v[0] = r; v[1] = g; v[2] = bl;
    }
}

// one thread per (super-row h8, frame n, sub-row dy, position w8), w8 fastest: a warp reads 32 consecutive
// 8-pixel runs of one frame row; each thread writes its three 8-channel runs.  bf16 runs hold x * kS2dInScale
// (a byte v becomes v / 256, exact in bf16; the patch embedding's bf16 weights carry the inverse factor).
template <int FMT, typename T>
__global__ void pack_s2d8_kernel(const uint8_t* __restrict__ frames, int N, int H, int W, int H8, int W8,
                                 T* __restrict__ x) {
    pdl_trigger();
    pdl_wait();
    const int C0 = 3 * N * 64;
    const unsigned total = (unsigned)H8 * W8 * N * 8;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const unsigned w8 = t % W8;
        unsigned r = t / W8;
        const int dy = (int)(r & 7);
        r >>= 3;
        const int n = (int)(r % N), h8 = (int)(r / N);
        const int h = 8 * h8 + dy, sh = h < H ? h : H - 1;
        float v[3][8];
#pragma unroll
        for (int dx = 0; dx < 8; ++dx) {
            const int w = 8 * (int)w8 + dx, sw = w < W ? w : W - 1;
            float p[3];
            px3<FMT>(frames, n, sh, sw, H, W, p);
            const float k = sizeof(T) == 2 ? kS2dInScale : 1.0f;
            v[0][dx] = p[0] * k; v[1][dx] = p[1] * k; v[2][dx] = p[2] * k;
        }
        T* o = x + ((size_t)h8 * W8 + w8) * C0 + (size_t)(3 * n) * 64 + 8 * dy;
#pragma unroll
        for (int c = 0; c < 3; ++c) st8<T>(o + c * 64, v[c]);
    }
}

__device__ __forceinline__ float gelu_erf(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

// one thread per (row, strip of kDwPix output pixels, run of 8 channels) of group blockIdx.y, channel run
// fastest: a warp reads 32 consecutive runs (512 bytes of bf16) per load; the strip's 3 x (kDwPix + 2) input
// runs are loaded once for its kDwPix outputs; the group's 9 x C filter taps and C biases are staged in
// shared memory once per block (C <= kDwMaxC)
constexpr int kDwPix = 4;
constexpr int kDwMaxC = 512;

template <typename T>
__global__ void __launch_bounds__(256, 2) dw_conv_kernel(const T* __restrict__ x, int H, int W, int C, long long gs,
                                                      const float* __restrict__ w, const float* __restrict__ b,
                                                      T* __restrict__ out) {
    __shared__ __align__(16) float sw[10 * kDwMaxC];  // 9 taps x C, then the biases
    const int g = blockIdx.y;
    for (int i = threadIdx.x; i < 9 * C; i += blockDim.x) sw[i] = w[(size_t)g * 9 * C + i];
    for (int i = threadIdx.x; i < C; i += blockDim.x) sw[9 * C + i] = b[(size_t)g * C + i];
    __syncthreads();
    pdl_trigger();
    pdl_wait();
    const int c8 = C >> 3, ws = (W + kDwPix - 1) / kDwPix;
    const unsigned total = (unsigned)H * ws * c8;
    const T* xg = x + g * gs;
    T* og = out + g * gs;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int cr = (int)(t % c8);
        const unsigned r = t / c8;
        const int s0 = (int)(r % ws) * kDwPix, h = (int)(r / ws);
        const int c0 = 8 * cr;
        float acc[kDwPix][8], bias[8];
        ld8<float>(sw + 9 * C + c0, bias);
#pragma unroll
        for (int q = 0; q < kDwPix; ++q)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[q][j] = bias[j];
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
            // the row's kDwPix + 2 input runs are all loaded before any arithmetic (clamped addresses, zeroed
            // outside the image), so their latencies overlap instead of forming load -> use chains
            const int ih = h + ky - 1;
            const bool rv = ih >= 0 && ih < H;
            const T* row = xg + (size_t)(ih < 0 ? 0 : (ih >= H ? H - 1 : ih)) * W * C + c0;
            uint4 raw[kDwPix + 2][sizeof(T) / 2];  // 8 channels: one 16-byte vector (bf16) or two (float)
            bool cv[kDwPix + 2];
#pragma unroll
            for (int u = 0; u < kDwPix + 2; ++u) {  // input column s0 - 1 + u
                const int iw = s0 - 1 + u;
                cv[u] = rv && iw >= 0 && iw < W;
                const uint4* src = reinterpret_cast<const uint4*>(row + (size_t)(iw < 0 ? 0 : (iw >= W ? W - 1 : iw)) * C);
#pragma unroll
                for (int e = 0; e < (int)(sizeof(T) / 2); ++e) raw[u][e] = src[e];
            }
            float k[3][8];  // this kernel row's three taps, read from shared memory once per row
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) ld8<float>(sw + (3 * ky + kx) * C + c0, k[kx]);
#pragma unroll
            for (int u = 0; u < kDwPix + 2; ++u) {
                float v[8];
                ld8<T>(reinterpret_cast<const T*>(raw[u]), v);
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = cv[u] ? v[j] : 0.0f;
#pragma unroll
                for (int q = 0; q < kDwPix; ++q) {  // output column s0 + q uses tap kx = u - q
                    const int kx = u - q;
                    if (kx < 0 || kx > 2) continue;
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[q][j] = fmaf(k[kx][j], v[j], acc[q][j]);
                }
            }
        }
        T* o = og + ((size_t)h * W + s0) * C + c0;
#pragma unroll
        for (int q = 0; q < kDwPix; ++q) {
            if (s0 + q >= W) break;
            // bf16 activations: the tensor-core epilogues' GELU (|error| < 2.6e-5, far below the bf16 rounding
            // of the result); float activations: the exact erf form
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[q][j] = sizeof(T) == 2 ? gelu_tc(acc[q][j]) : gelu_erf(acc[q][j]);
            st8<T>(o + (size_t)q * C, acc[q]);
        }
    }
}

// one thread per output pixel (n, y, x)
template <bool U8>
__global__ void ps8_out_kernel(const float* __restrict__ o, int N, int H8, int W8, int H, int W,
                               void* __restrict__ frames) {
    pdl_trigger();
    pdl_wait();
    const long long total = (long long)N * H * W;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(t % W);
        long long r = t / W;
        const int y = (int)(r % H);
        const int n = (int)(r / H);
        const float* src = o + (((size_t)n * H8 + (y >> 3)) * W8 + (x >> 3)) * 192 + 8 * (y & 7) + (x & 7);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float v = fminf(fmaxf(0.5f + src[64 * c], 0.0f), 1.0f);
            if (U8) static_cast<uint8_t*>(frames)[3 * t + c] = (uint8_t)rintf(255.0f * v);
            else static_cast<float*>(frames)[3 * t + c] = v;
        }
    }
}

unsigned grid_of(long long n) {
    long long g = (n + 255) / 256;
    if (g > 148 * 16) g = 148 * 16;
    return (unsigned)(g ? g : 1);
}

}  // namespace

void launch_pack_s2d8(const uint8_t* frames, int N, int H, int W, int H8, int W8, void* x, bool f32, int fmt,
                      cudaStream_t s) {
    const dim3 g(grid_of((long long)H8 * W8 * N * 8));
#define PACK8(F)                                                                                              \
    (f32 ? launch_pdl(pack_s2d8_kernel<F, float>, g, dim3(256), 0, s, frames, N, H, W, H8, W8, (float*)x)     \
         : launch_pdl(pack_s2d8_kernel<F, __nv_bfloat16>, g, dim3(256), 0, s, frames, N, H, W, H8, W8,          \
                      (__nv_bfloat16*)x))
    switch (fmt) {
        case 1: (void)PACK8(1); break;
        case 2: (void)PACK8(2); break;
        case 3: (void)PACK8(3); break;
        default: (void)PACK8(0); break;
    }
#undef PACK8
}

// C <= kDwMaxC, a multiple of 8; blocks spread over the groups (gridDim.y = G) so each stages one group's taps
void launch_dw_conv(const void* x, int G, int H, int W, int C, long long gs, const float* w, const float* b, void* out,
                    bool f32, cudaStream_t s) {
    if (C > kDwMaxC || (C & 7) || G < 1) return;
    long long per = (long long)H * ((W + kDwPix - 1) / kDwPix) * (C >> 3);
    unsigned gx = grid_of(per);
    const unsigned cap = (148u * 16u + G - 1) / G;  // about sixteen blocks per SM in all
    if (gx > cap) gx = cap ? cap : 1;
    const dim3 g(gx, (unsigned)G);
    if (f32)
        (void)launch_pdl(dw_conv_kernel<float>, g, dim3(256), 0, s, (const float*)x, H, W, C, gs, w, b, (float*)out);
    else
        (void)launch_pdl(dw_conv_kernel<__nv_bfloat16>, g, dim3(256), 0, s, (const __nv_bfloat16*)x, H, W, C, gs, w, b,
                         (__nv_bfloat16*)out);
}

void launch_ps8_out(const float* o, int N, int H8, int W8, int H, int W, void* frames, bool u8, cudaStream_t s) {
    const dim3 g(grid_of((long long)N * H * W));
    if (u8) (void)launch_pdl(ps8_out_kernel<true>, g, dim3(256), 0, s, o, N, H8, W8, H, W, frames);
    else (void)launch_pdl(ps8_out_kernel<false>, g, dim3(256), 0, s, o, N, H8, W8, H, W, frames);
}

}  // namespace ufvc
