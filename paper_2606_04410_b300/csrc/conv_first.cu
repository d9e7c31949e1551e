// The first analysis layer read straight from the chunk's frame bytes (BF16 tensor cores).
//
// A1 is a 3x3 stride-2 convolution of the 3N stacked input channels (frames stacked along channels,
// Sec. 3.1) to 64 outputs with GELU.  Run as a layer over a packed bf16 input tensor it needs a pack pass
// that writes 2.7x the frame bytes (32 bf16 channels per pixel) and an A1 pass that reads them back; here
// one kernel reads the caller's uint8 frames once and builds the tensor-core operand in shared memory.
//
// GEMM view: M = 128 output pixels (an 8 x 16 block), N = 64 output channels, K = 9 taps x CT channels
// (CT = 3N rounded up to 8, N even; K padded to KC 64-element chunks with zeros).  Per tile:
//   1. the bytes of the block's input window (17 x 33 pixels of every frame; replicate padding inside the
//      padded frame size, zeros where the convolution's own padding lies) are loaded into registers one
//      tile ahead, then written to shared memory as bf16 pixels of CT contiguous channels (channel
//      3 n + colour; a byte v as v / 256, exact in bf16; the weights carry 256 / 255);
//   2. the A operand [128 pixels][KC x 64] is copied from those pixels 16 bytes (8 channels of one tap) at
//      a time, K-major with the 128-byte swizzle, into one of two buffers;
//   3. one thread issues KC x 4 tcgen05.mma (M = 128, N = 64, K = 16) into one of two TMEM accumulators;
//   4. sixteen warps drain it (tcgen05.ld), add the bias, apply GELU and store bf16 NHWC.
// The MMAs of tile k + 1 are issued before tile k is drained, and the loads of tile k + 2 are in flight
// meanwhile.  The weights [KC][64 rows][128 B] stay in shared memory (already swizzled in global memory,
// copied once per CTA).  One CTA per SM.  The wait for the MMAs is bounded: on a timeout the kernel
// records UFVC_ERR_TIMEOUT and stops.
#include "ufvc_internal.h"
#include "tc_ptx.h"

namespace ufvc {

constexpr int kFirstThreads = 512;
constexpr int kFirstTH = 8, kFirstTW = 16;                        // output block of one tile
constexpr int kWinH = 2 * kFirstTH + 1, kWinW = 2 * kFirstTW + 1;  // its 17 x 33 input window
constexpr int kWinPx = kWinH * kWinW;
constexpr int kFirstItems = (kWinPx * 4 + kFirstThreads - 1) / kFirstThreads;  // (pixel, frame pair) per thread
constexpr long long kFirstSpin = 4000000000LL;                                 // ~2 s at 2 GHz

__host__ __device__ constexpr int first_kc(int ct) { return (9 * ct + 63) / 64; }
__host__ __device__ constexpr size_t first_win_bytes(int ct) { return ((size_t)kWinPx * ct * 2 + 15) & ~size_t(15); }
__host__ __device__ constexpr size_t first_smem(int ct) {
    return 1024 + (size_t)first_kc(ct) * (2 * 16384 + 8192) + first_win_bytes(ct) + 256 + 64;
}

__device__ __forceinline__ uint4 ld_shared_v4(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr));
    return v;
}

// bf16 bits of v / 256 for two bytes: 32768 + v / 256 is exact in FP32 (unit in the last place 2^-8)
__device__ __forceinline__ uint32_t bytes_bf16x2(uint32_t a, uint32_t b) {
    const float fa = __uint_as_float(0x47000000u | a) - 32768.0f, fb = __uint_as_float(0x47000000u | b) - 32768.0f;
    __nv_bfloat162 h = __floats2bfloat162_rn(fa, fb);
    return *reinterpret_cast<uint32_t*>(&h);
}

template <int FMT, int CT>
__global__ void __launch_bounds__(kFirstThreads, 1)
    conv_first_kernel(const uint8_t* __restrict__ frames, int N, int H, int W, int Ho, int Wo,
                      const uint4* __restrict__ wimg, const float* __restrict__ bias, __nv_bfloat16* __restrict__ out,
                      int* err) {
    constexpr int KC = first_kc(CT);
    constexpr int PARTS = CT / 8;  // 16-byte chunks per tap
    constexpr int ABUF = KC * 16384;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;               // 2 x KC x [128 rows][128 B]
    uint8_t* sB = sA + 2 * ABUF;      // KC x [64 rows][128 B]
    uint8_t* sx = sB + KC * 8192;     // window pixels [17 x 33][CT] bf16
    float* sbias = reinterpret_cast<float*>(sx + first_win_bytes(CT));
    uint64_t* bar = reinterpret_cast<uint64_t*>(sbias + 64);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 2);
    volatile int* stop = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // set-up (constant inputs only): weights, biases, zero K columns past 9 CT, zero window, barriers, TMEM
    {
        uint4* dB = reinterpret_cast<uint4*>(sB);
        for (int i = tid; i < KC * 512; i += kFirstThreads) dB[i] = __ldg(wimg + i);
        if (tid < 64) sbias[tid] = __ldg(bias + tid);
        constexpr int K0 = 9 * CT;  // a multiple of 8: whole 16-byte chunks
        for (int i = tid; i < 2 * 128 * (KC * 8 - K0 / 8); i += kFirstThreads) {
            const int buf = i & 1, row = (i >> 1) & 127, k0 = K0 + 8 * (i >> 8);
            ptx::st_shared_v4(ptx::smem_u32(sA) + buf * ABUF + (k0 >> 6) * 16384 + row * 128 +
                                  ((((k0 & 63) >> 3) ^ (row & 7)) << 4), 0u, 0u, 0u, 0u);
        }
        uint4* dx = reinterpret_cast<uint4*>(sx);
        for (int i = tid; i < (int)(first_win_bytes(CT) / 16); i += kFirstThreads) dx[i] = make_uint4(0u, 0u, 0u, 0u);
        if (tid == 0) {
            ptx::mbar_init(&bar[0], 1);
            ptx::mbar_init(&bar[1], 1);
            *stop = 0;
            ptx::fence_mbar_init();
        }
        if (warp == 0) ptx::tmem_alloc(tmem_slot, 128);
    }
    ptx::fence_proxy_async();  // the operand bytes written above -> visible to the tensor cores
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    pdl_trigger();
    pdl_wait();  // frames may come from, and the output be read by, the neighbouring kernels

    const int tiles_w = (Wo + kFirstTW - 1) / kFirstTW;
    const int tiles = tiles_w * ((Ho + kFirstTH - 1) / kFirstTH);
    const int items = kWinPx * (N >> 1);
    const uint32_t sA_u = ptx::smem_u32(sA), sB_u = ptx::smem_u32(sB), sx_u = ptx::smem_u32(sx);
    uint32_t rb[kFirstItems][6];
    // the thread's share of a tile is the same in every tile: window items i = tid + 512 j as
    // (frame pair, window row, window column), and the (source, destination) offsets of its A chunks
    uint32_t item[kFirstItems];
#pragma unroll
    for (int j = 0; j < kFirstItems; ++j) {
        const int i = tid + j * kFirstThreads;
        const int pr = i / kWinPx, px = i - pr * kWinPx, ly = px / kWinW, lx = px - ly * kWinW;
        item[j] = i < items ? (uint32_t)(pr << 16 | ly << 8 | lx) : 0xFFFFFFFFu;
    }
    constexpr int BI = (128 * 9 * PARTS + kFirstThreads - 1) / kFirstThreads;
    uint32_t chunk[BI];
#pragma unroll
    for (int j = 0; j < BI; ++j) {
        const int i = tid + j * kFirstThreads;
        const int row = i & 127, tp = i >> 7;
        const int tap = tp / PARTS, part = tp - tap * PARTS;
        const int ky = tap / 3, kx = tap - 3 * ky;
        const int px = (2 * (row >> 4) + ky) * kWinW + 2 * (row & 15) + kx;
        const int k0 = tap * CT + 8 * part;
        const uint32_t src = (uint32_t)(px * CT + 8 * part) * 2;
        const uint32_t dst = (uint32_t)((k0 >> 6) * 16384 + row * 128 + ((((k0 & 63) >> 3) ^ (row & 7)) << 4));
        chunk[j] = i < 128 * 9 * PARTS ? (src | dst << 16) : 0xFFFFFFFFu;  // src < 2^15, dst < 2^16
    }
    const size_t fstride = FMT == 0 ? (size_t)H * W * 3 : 0;

    // 1a. the window bytes of tile t into registers (window pixel (ly, lx) = frame pixel
    //     (2 h0 - 1 + ly, 2 w0 - 1 + lx); replicate the last row / column, zeros left of and above the frame)
    auto load = [&](int t) {
        const int h0 = (t / tiles_w) * kFirstTH, w0 = (t % tiles_w) * kFirstTW;
#pragma unroll
        for (int j = 0; j < kFirstItems; ++j) {
            const uint32_t it = item[j];
            const int pr = (int)(it >> 16), ly = (int)((it >> 8) & 0xFF), lx = (int)(it & 0xFF);
            const int ih = 2 * h0 - 1 + ly, iw = 2 * w0 - 1 + lx;
#pragma unroll
            for (int e = 0; e < 6; ++e) rb[j][e] = 0u;
            if (it != 0xFFFFFFFFu && ih >= 0 && iw >= 0) {
                const int sh = ih < H ? ih : H - 1, sw = iw < W ? iw : W - 1;
                if constexpr (FMT == 0) {
                    const uint8_t* p0 = frames + (size_t)(2 * pr) * fstride + (size_t)(sh * W + sw) * 3;
                    const uint8_t* p1 = p0 + fstride;
                    rb[j][0] = __ldg(p0); rb[j][1] = __ldg(p0 + 1); rb[j][2] = __ldg(p0 + 2);
                    rb[j][3] = __ldg(p1); rb[j][4] = __ldg(p1 + 1); rb[j][5] = __ldg(p1 + 2);
                } else {
                    px_bytes<FMT>(frames, 2 * pr, sh, sw, H, W, &rb[j][0]);
                    px_bytes<FMT>(frames, 2 * pr + 1, sh, sw, H, W, &rb[j][3]);
                }
            }
        }
    };
    // 1b. registers -> window pixels (channels 6 p .. 6 p + 5 of pixel (ly, lx))
    auto store = [&]() {
#pragma unroll
        for (int j = 0; j < kFirstItems; ++j) {
            const uint32_t it = item[j];
            if (it != 0xFFFFFFFFu) {
                const int pr = (int)(it >> 16), px = (int)((it >> 8) & 0xFF) * kWinW + (int)(it & 0xFF);
                const uint32_t a = sx_u + (px * CT + 6 * pr) * 2;
                asm volatile("st.shared.b32 [%0], %1;" ::"r"(a), "r"(bytes_bf16x2(rb[j][0], rb[j][1])) : "memory");
                asm volatile("st.shared.b32 [%0], %1;" ::"r"(a + 4), "r"(bytes_bf16x2(rb[j][2], rb[j][3])) : "memory");
                asm volatile("st.shared.b32 [%0], %1;" ::"r"(a + 8), "r"(bytes_bf16x2(rb[j][4], rb[j][5])) : "memory");
            }
        }
    };
    // 2. A rows of buffer buf: pixel row r, K elements tap CT + c (tap = 3 ky + kx), 16 bytes per chunk
    auto build = [&](int buf) {
        const uint32_t dA = sA_u + buf * ABUF;
#pragma unroll
        for (int j = 0; j < BI; ++j) {
            const uint32_t c = chunk[j];
            if (c != 0xFFFFFFFFu) {
                const uint4 v = ld_shared_v4(sx_u + (c & 0xFFFFu));
                ptx::st_shared_v4(dA + (c >> 16), v.x, v.y, v.z, v.w);
            }
        }
    };
    // 3. the MMAs of buffer buf into accumulator buf, completion on bar[buf] (thread 0)
    auto mma = [&](int buf) {
        ptx::tc_fence_after();
        constexpr uint32_t idesc = ptx::idesc_bf16(64);
#pragma unroll
        for (int j = 0; j < KC; ++j)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                ptx::mma_f16(tmem_base + buf * 64, ptx::sdesc_sw128(sA_u + buf * ABUF + j * 16384 + kk * 32),
                             ptx::sdesc_sw128(sB_u + j * 8192 + kk * 32), idesc, (j | kk) != 0);
        ptx::mma_commit(&bar[buf]);
    };

    int t = blockIdx.x;
    if (t < tiles) {
        load(t);
        store();
        __syncthreads();
        build(0);
        ptx::fence_proxy_async();
        ptx::tc_fence_before();
        __syncthreads();
        if (tid == 0) mma(0);
        if (t + (int)gridDim.x < tiles) load(t + gridDim.x);
    }
    for (int k = 0; t < tiles; ++k, t += gridDim.x) {
        const int b = k & 1, t1 = t + gridDim.x, t2 = t1 + gridDim.x;
        if (t1 < tiles) {  // tile k + 1: window, operand and MMAs
            store();
            __syncthreads();
            build(b ^ 1);
            ptx::fence_proxy_async();
            ptx::tc_fence_before();
            __syncthreads();
            if (tid == 0) mma(b ^ 1);
            if (t2 < tiles) load(t2);
        }
        if (tid == 0) {
            const uint32_t par = (k >> 1) & 1;
            bool done = ptx::mbar_try_wait(&bar[b], par);
            const long long c0 = clock64();
            while (!done) {
                done = ptx::mbar_try_wait(&bar[b], par);
                if (!done && clock64() - c0 > kFirstSpin) {
                    atomicCAS(err, 0, (int)UFVC_ERR_TIMEOUT);
                    *stop = 1;
                    break;
                }
            }
        }
        __syncthreads();
        if (*stop) break;
        ptx::tc_fence_after();
        // 4. epilogue of tile k: warp w drains TMEM lanes 32 (w % 4) .. +31, columns 16 (w / 4) .. +15
        {
            const int q = warp & 3, cq = warp >> 2, row = q * 32 + lane;
            float v[16];
            ptx::tmem_ld16(tmem_base + b * 64 + ((uint32_t)(q * 32) << 16) + cq * 16, v);
            const int h0 = (t / tiles_w) * kFirstTH, w0 = (t % tiles_w) * kFirstTW;
            const int oh = h0 + (row >> 4), ow = w0 + (row & 15);
            if (oh < Ho && ow < Wo) {
                const float4* bs = reinterpret_cast<const float4*>(sbias + cq * 16);
#pragma unroll
                for (int c = 0; c < 16; c += 4) {
                    const float4 bb = bs[c >> 2];
                    v[c] += bb.x; v[c + 1] += bb.y; v[c + 2] += bb.z; v[c + 3] += bb.w;
                    gelu_tc2(v[c], v[c + 1]);
                    gelu_tc2(v[c + 2], v[c + 3]);
                }
                uint4* d = reinterpret_cast<uint4*>(out + ((size_t)oh * Wo + ow) * 64 + cq * 16);
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
        __syncthreads();  // accumulator b and operand buffer b are free again
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem_base, 128);
    }
}

template <int FMT, int CT>
static cudaError_t launch_first_t(const uint8_t* frames, int N, int H, int W, int Ho, int Wo, const void* wimg,
                                  const float* bias, __nv_bfloat16* out, int* err, cudaStream_t s) {
    const size_t smem = first_smem(CT);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(conv_first_kernel<FMT, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = ((Wo + kFirstTW - 1) / kFirstTW) * ((Ho + kFirstTH - 1) / kFirstTH);
    const int grid = tiles < sms ? tiles : sms;
    return launch_pdl(conv_first_kernel<FMT, CT>, dim3(grid), dim3(kFirstThreads), smem, s, frames, N, H, W, Ho, Wo,
                      static_cast<const uint4*>(wimg), bias, out, err);
}

int first_layer_ct(int n_frames) {
    return n_frames >= 2 && n_frames <= 8 && n_frames % 2 == 0 ? (3 * n_frames + 7) / 8 * 8 : 0;
}

size_t first_layer_weight_bytes(int ct) { return (size_t)first_kc(ct) * 8192; }

void first_layer_weights(const float* w, int n_frames, float scale, uint16_t* img) {
    const int ct = first_layer_ct(n_frames), kc = first_kc(ct), ci = 3 * n_frames;
    for (size_t i = 0; i < first_layer_weight_bytes(ct) / 2; ++i) img[i] = 0;
    for (int co = 0; co < 64; ++co)
        for (int tap = 0; tap < 9; ++tap)
            for (int c = 0; c < ci; ++c) {
                const int k = tap * ct + c, j = k >> 6, chunk = ((k & 63) >> 3) ^ (co & 7);
                const size_t e = (size_t)j * 4096 + (size_t)co * 64 + chunk * 8 + (k & 7);
                const __nv_bfloat16 h = __float2bfloat16(scale * w[((size_t)co * 9 + tap) * ci + c]);
                img[e] = *reinterpret_cast<const uint16_t*>(&h);
            }
    (void)kc;
}

cudaError_t launch_first_layer(const uint8_t* frames, int fmt, int N, int H, int W, int Ho, int Wo, const void* wimg,
                               const float* bias, __nv_bfloat16* out, int* err, cudaStream_t s) {
    const int ct = first_layer_ct(N);
#define UFVC_FIRST(F)                                                                                          \
    switch (ct) {                                                                                              \
        case 8: return launch_first_t<F, 8>(frames, N, H, W, Ho, Wo, wimg, bias, out, err, s);                 \
        case 16: return launch_first_t<F, 16>(frames, N, H, W, Ho, Wo, wimg, bias, out, err, s);               \
        case 24: return launch_first_t<F, 24>(frames, N, H, W, Ho, Wo, wimg, bias, out, err, s);               \
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
