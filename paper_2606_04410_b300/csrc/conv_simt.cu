// FP32 implicit-GEMM convolution on CUDA cores (FFMA), NHWC.
//
// Used for the whole FP32 path and, in every precision, for the hyper-synthesis (the single-step
// parameter estimation of Sec. 3.4): encoder and decoder must derive bit-identical (mu, log sigma)
// from z^, so this kernel is deterministic: the arithmetic of an output element depends only on the
// layer's shapes, never on timing — products accumulate with explicit fmaf in a fixed order (taps
// row-major, then input channels ascending) and, where the K steps are split into KS contiguous
// ranges to fill the GPU, the range sums are added in range order by a second kernel.  No atomics.
//
// Kernels: 128 x BN tiles (BN = 64, or 16 for the narrow final layers) for large layers; 64 x 64
// tiles with 4 x 4 outputs per thread, optionally split along K, for the small hyper layers.  K is
// staged 16 input channels at a time through double-buffered shared memory.  Epilogue: bias, optional
// GELU, optional residual, optional pixel shuffle x2 / crop / split of the channels into two tensors,
// or the final frame mapping x^ = clamp(0.5 + o, 0, 1) (float or uint8).
#include "ufvc_internal.h"

namespace ufvc {

__device__ __forceinline__ float gelu_erf(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

// (c0, c1) = (a * b0 + c0, a * b1 + c1), each one IEEE fused multiply-add rounded to nearest (the packed
// FP32 instruction of sm_100+: the results of two fmaf calls in one issue slot)
__device__ __forceinline__ void fma2_bcast(float& c0, float& c1, float a, float b0, float b1) {
    asm("{\n\t.reg .b64 pa, pb, pc;\n\t"
        "mov.b64 pa, {%2, %2};\n\t"
        "mov.b64 pb, {%3, %4};\n\t"
        "mov.b64 pc, {%0, %1};\n\t"
        "fma.rn.f32x2 pc, pa, pb, pc;\n\t"
        "mov.b64 {%0, %1}, pc;\n\t}"
        : "+f"(c0), "+f"(c1)
        : "f"(a), "f"(b0), "f"(b1));
}

__device__ __forceinline__ void store_out(const ConvDesc& d, int g, int oh, int ow, int co, float v) {
    if (d.mode == OUT_NHWC) {
        if (oh >= d.out_h || ow >= d.out_w) return;
        const size_t pix = (size_t)oh * d.out_w + ow;
        if (d.split && co >= d.split) {
            const int c2 = d.Cout - d.split;
            d.out2[(size_t)g * d.out_gs + pix * c2 + (co - d.split)] = v;
            return;
        }
        const int C = d.split ? d.split : d.Cout;
        const size_t o = (size_t)g * d.out_gs + pix * C + co;
        if (d.res) v += ((const float*)d.res)[(size_t)g * d.res_gs + pix * C + co];
        ((float*)d.out)[o] = v;
        return;
    }
    const int c = co >> 2, y = 2 * oh + ((co >> 1) & 1), x = 2 * ow + (co & 1);
    if (y >= d.out_h || x >= d.out_w) return;
    const int C = d.Cout >> 2;
    const size_t o = (size_t)g * d.out_gs + ((size_t)y * d.out_w + x) * C + c;
    if (d.mode == OUT_PS) {
        if (d.res) v += ((const float*)d.res)[(size_t)g * d.res_gs + ((size_t)y * d.out_w + x) * C + c];
        ((float*)d.out)[o] = v;
    } else {
        v = fminf(fmaxf(0.5f + v, 0.0f), 1.0f);
        if (d.mode == OUT_PS_FINAL_F32)
            ((float*)d.out)[o] = v;
        else
            ((uint8_t*)d.out)[o] = (uint8_t)rintf(v * 255.0f);
    }
}

// Output channels co..co+3 (co % 4 == 0) of one pixel: one 16-byte access when d.vec4 (NHWC output,
// channel counts, split and group strides multiples of 4, 16-byte aligned tensors), else four scalar
// stores.
__device__ __forceinline__ void store_out4(const ConvDesc& d, int g, int oh, int ow, int co, float4 v) {
    if (d.vec4) {
        if (oh >= d.out_h || ow >= d.out_w) return;
        const size_t pix = (size_t)oh * d.out_w + ow;
        if (d.split && co >= d.split) {
            const int c2 = d.Cout - d.split;
            *reinterpret_cast<float4*>(d.out2 + (size_t)g * d.out_gs + pix * c2 + (co - d.split)) = v;
            return;
        }
        const int C = d.split ? d.split : d.Cout;
        const size_t o = (size_t)g * d.out_gs + pix * C + co;
        if (d.res) {
            const float4 r = *reinterpret_cast<const float4*>((const float*)d.res + (size_t)g * d.res_gs + pix * C + co);
            v.x += r.x; v.y += r.y; v.z += r.z; v.w += r.w;
        }
        *reinterpret_cast<float4*>((float*)d.out + o) = v;
        return;
    }
    store_out(d, g, oh, ow, co, v.x);
    store_out(d, g, oh, ow, co + 1, v.y);
    store_out(d, g, oh, ow, co + 2, v.z);
    store_out(d, g, oh, ow, co + 3, v.w);
}

template <int BM, int BN>
__global__ void __launch_bounds__(256) conv_simt_kernel(const ConvDesc d, int Ho, int Wo) {
    pdl_trigger();
    pdl_wait();
    constexpr int BK = 16;
    constexpr int TN = BN / 4;    // threads along N, 4 output channels each
    constexpr int TM = 256 / TN;  // threads along M
    constexpr int PM = BM / TM;   // pixels per thread: 8 (128 x 64), 2 (128 x 16 or 32 x 64)
    constexpr int RA = (BM * BK / 4 + 255) / 256;  // float4 A loads per thread
    static_assert(PM == 8 || PM == 2, "tile");
    static_assert(PM == 2 || BM == 128, "interleaved mapping needs BM = 128");
    __shared__ __align__(16) float As[2][BK][BM + 4];  // +4: fewer bank conflicts on the transposed store
    __shared__ __align__(16) float Bs[2][BK][BN];

    const int g = blockIdx.z;
    const float* in = (const float*)d.in + (size_t)g * d.in_gs;
    const float* w = d.w + (size_t)g * d.w_gs;
    const float* bias = d.b + (size_t)g * d.b_gs;
    const int M = Ho * Wo;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int tid = threadIdx.x;
    const int H = d.H, W = d.W, Cin = d.Cin, Cout = d.Cout, k = d.k, s = d.stride, p = d.k / 2;

    // A loads: RA float4 per thread (pixel q >> 2, channels 4 * (q & 3) .. +3 of the 16-channel chunk)
    int a_oh[RA], a_ow[RA];
    bool a_ok[RA];
#pragma unroll
    for (int r = 0; r < RA; ++r) {
        const int m = m0 + ((tid + r * 256) >> 2);
        a_ok[r] = ((tid + r * 256) >> 2) < BM && m < M;
        a_oh[r] = a_ok[r] ? m / Wo : 0;
        a_ow[r] = a_ok[r] ? m - a_oh[r] * Wo : 0;
    }
    const int a_cg = tid & 3;
    // B loads: BK * BN / 4 float4 (row = i / (BN/4), 4 output channels)
    const bool b_act = tid < BK * BN / 4;
    const int b_row = tid / (BN / 4), b_cg = tid % (BN / 4);
    const int b_co = n0 + b_cg * 4;

    const int nck = Cin / BK, nsteps = k * k * nck;
    float4 ra[RA], rb;

    auto load_regs = [&](int step) {
        const int tap = step / nck, c0 = (step - tap * nck) * BK;
        const int ky = tap / k, kx = tap - ky * k;
#pragma unroll
        for (int r = 0; r < RA; ++r) {
            const int ih = a_oh[r] * s + ky - p, iw = a_ow[r] * s + kx - p;
            if (a_ok[r] && ih >= 0 && ih < H && iw >= 0 && iw < W)
                ra[r] = *reinterpret_cast<const float4*>(in + ((size_t)ih * W + iw) * Cin + c0 + a_cg * 4);
            else
                ra[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (b_act) {
            if (b_co < Cout)
                rb = *reinterpret_cast<const float4*>(w + ((size_t)tap * Cin + c0 + b_row) * Cout + b_co);
            else
                rb = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto store_smem = [&](int buf) {
#pragma unroll
        for (int r = 0; r < RA; ++r) {
            const int pix = (tid + r * 256) >> 2;
            if (pix >= BM) continue;
            As[buf][a_cg * 4 + 0][pix] = ra[r].x;
            As[buf][a_cg * 4 + 1][pix] = ra[r].y;
            As[buf][a_cg * 4 + 2][pix] = ra[r].z;
            As[buf][a_cg * 4 + 3][pix] = ra[r].w;
        }
        if (b_act) *reinterpret_cast<float4*>(&Bs[buf][b_row][b_cg * 4]) = rb;
    };

    const int tn = tid % TN, tm = tid / TN;
    float acc[PM][4];
#pragma unroll
    for (int i = 0; i < PM; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    load_regs(0);
    store_smem(0);
    __syncthreads();
    for (int step = 0; step < nsteps; ++step) {
        const int buf = step & 1;
        if (step + 1 < nsteps) load_regs(step + 1);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 b = *reinterpret_cast<const float4*>(&Bs[buf][kk][tn * 4]);
            float a[PM];
            if constexpr (PM == 8) {
                const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][tm * 4]);
                const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + tm * 4]);
                a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
                a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
            } else {
                const float2 a0 = *reinterpret_cast<const float2*>(&As[buf][kk][tm * 2]);
                a[0] = a0.x; a[1] = a0.y;
            }
#pragma unroll
            for (int i = 0; i < PM; ++i) {
                acc[i][0] = fmaf(a[i], b.x, acc[i][0]);
                acc[i][1] = fmaf(a[i], b.y, acc[i][1]);
                acc[i][2] = fmaf(a[i], b.z, acc[i][2]);
                acc[i][3] = fmaf(a[i], b.w, acc[i][3]);
            }
        }
        if (step + 1 < nsteps) store_smem(buf ^ 1);
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < PM; ++i) {
        const int pix = (PM == 8) ? (i < 4 ? tm * 4 + i : 64 + tm * 4 + (i - 4)) : tm * 2 + i;
        const int m = m0 + pix;
        if (m >= M) continue;
        const int oh = m / Wo, ow = m - (m / Wo) * Wo;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int co = n0 + tn * 4 + j;
            if (co >= Cout) continue;
            float v = acc[i][j] + bias[co];
            if (d.act) v = gelu_erf(v);
            store_out(d, g, oh, ow, co, v);
        }
    }
}

// 64 x 64 tile, 256 threads, 4 x 4 outputs per thread (pixels tm*4.., channels tn*4..), K staged BK
// input channels per step; global loads run two steps ahead of the FMAs (two register sets) and the
// shared-memory tiles are double-buffered.  blockIdx.z = g * KS + ks: K steps [ks * nsteps / KS,
// (ks + 1) * nsteps / KS).  PARTIAL: write the range sums to ws[g][ks][m][co] (added by
// conv_simt_reduce_kernel); otherwise finish the outputs here (KS = 1).
template <bool PARTIAL, int BK>
__global__ void __launch_bounds__(256) conv_simt64_kernel(const ConvDesc d, int Ho, int Wo, int KS, float* ws) {
    pdl_trigger();
    pdl_wait();
    constexpr int BM = 64, BN = 64;
    constexpr int AV = BM * BK / 4 / 256;  // float4 A loads per thread
    constexpr int BV = BK * BN / 4 / 256;  // float4 B loads per thread
    constexpr int CG = BK / 4;             // float4 groups per pixel
    __shared__ __align__(16) float As[2][BK][BM + 4];
    __shared__ __align__(16) float Bs[2][BK][BN];

    const int g = blockIdx.z / KS, ks = blockIdx.z - g * KS;
    const float* in = (const float*)d.in + (size_t)g * d.in_gs;
    const float* w = d.w + (size_t)g * d.w_gs;
    const int M = Ho * Wo;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int tid = threadIdx.x;
    const int H = d.H, W = d.W, Cin = d.Cin, Cout = d.Cout, k = d.k, s = d.stride, p = d.k / 2;

    int a_oh[AV], a_ow[AV];
    bool a_ok[AV];
#pragma unroll
    for (int r = 0; r < AV; ++r) {
        const int m = m0 + (tid + r * 256) / CG;
        a_ok[r] = m < M;
        a_oh[r] = a_ok[r] ? m / Wo : 0;
        a_ow[r] = a_ok[r] ? m - a_oh[r] * Wo : 0;
    }
    const int nck = Cin / BK, nsteps = k * k * nck;
    const int s_begin = (int)((long long)ks * nsteps / KS), s_end = (int)((long long)(ks + 1) * nsteps / KS);
    float4 ra[2][AV], rb[2][BV];
    auto load_regs = [&](int step, float4* qa, float4* qb) {
        const int tap = step / nck, c0 = (step - tap * nck) * BK;
        const int ky = tap / k, kx = tap - ky * k;
#pragma unroll
        for (int r = 0; r < AV; ++r) {
            const int ih = a_oh[r] * s + ky - p, iw = a_ow[r] * s + kx - p;
            const int cg = (tid + r * 256) % CG;
            if (a_ok[r] && ih >= 0 && ih < H && iw >= 0 && iw < W)
                qa[r] = *reinterpret_cast<const float4*>(in + ((size_t)ih * W + iw) * Cin + c0 + cg * 4);
            else
                qa[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int r = 0; r < BV; ++r) {
            const int q = tid + r * 256, row = q >> 4, co = n0 + (q & 15) * 4;
            if (co < Cout)
                qb[r] = *reinterpret_cast<const float4*>(w + ((size_t)tap * Cin + c0 + row) * Cout + co);
            else
                qb[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto store_smem = [&](int buf, const float4* qa, const float4* qb) {
#pragma unroll
        for (int r = 0; r < AV; ++r) {
            const int q = tid + r * 256, pix = q / CG, cg = q % CG;
            As[buf][cg * 4 + 0][pix] = qa[r].x;
            As[buf][cg * 4 + 1][pix] = qa[r].y;
            As[buf][cg * 4 + 2][pix] = qa[r].z;
            As[buf][cg * 4 + 3][pix] = qa[r].w;
        }
#pragma unroll
        for (int r = 0; r < BV; ++r) {
            const int q = tid + r * 256;
            *reinterpret_cast<float4*>(&Bs[buf][q >> 4][(q & 15) * 4]) = qb[r];
        }
    };

    const int tn = tid & 15, tm = tid >> 4;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    auto fma_tile = [&](int buf) {
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a = *reinterpret_cast<const float4*>(&As[buf][kk][tm * 4]);
            const float4 b = *reinterpret_cast<const float4*>(&Bs[buf][kk][tn * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                acc[i][0] = fmaf(av[i], b.x, acc[i][0]);
                acc[i][1] = fmaf(av[i], b.y, acc[i][1]);
                acc[i][2] = fmaf(av[i], b.z, acc[i][2]);
                acc[i][3] = fmaf(av[i], b.w, acc[i][3]);
            }
        }
    };
    // step t = s_begin + i uses shared buffer i & 1 and register set i & 1; the body is written out
    // for both parities so that the register sets stay registers
    if (s_begin < s_end) load_regs(s_begin, ra[0], rb[0]);
    if (s_begin + 1 < s_end) load_regs(s_begin + 1, ra[1], rb[1]);
    if (s_begin < s_end) store_smem(0, ra[0], rb[0]);
    __syncthreads();
    for (int t = s_begin; t < s_end; t += 2) {
        if (t + 2 < s_end) load_regs(t + 2, ra[0], rb[0]);
        fma_tile(0);
        if (t + 1 < s_end) store_smem(1, ra[1], rb[1]);
        __syncthreads();
        if (t + 1 >= s_end) break;
        if (t + 3 < s_end) load_regs(t + 3, ra[1], rb[1]);
        fma_tile(1);
        if (t + 2 < s_end) store_smem(0, ra[0], rb[0]);
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + tm * 4 + i;
        if (m >= M) continue;
        const int co0 = n0 + tn * 4;
        if (PARTIAL) {
            float* dst = ws + (((size_t)g * KS + ks) * M + m) * Cout + co0;
            if (co0 + 3 < Cout) {
                *reinterpret_cast<float4*>(dst) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (co0 + j < Cout) dst[j] = acc[i][j];
            }
            continue;
        }
        const int oh = m / Wo, ow = m - oh * Wo;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int co = co0 + j;
            if (co >= Cout) continue;
            float v = acc[i][j] + d.b[(size_t)g * d.b_gs + co];
            if (d.act) v = gelu_erf(v);
            store_out(d, g, oh, ow, co, v);
        }
    }
}

// 64 x 128 tile, 128 threads, 8 x 8 outputs per thread: pixels tm*4 .. +3 and 32 + tm*4 .. +3, channels
// tn*4 .. +3 and 64 + tn*4 .. +3 (tm = tid / 16, tn = tid % 16), so each K step reads two float4 of A
// and two of B from shared memory for 64 FMAs (the 4 x 4 tiles are bound by shared-memory bandwidth).
// K staged 16 input channels per step, global loads two steps ahead, shared tiles double-buffered;
// split-K ranges and the PARTIAL workspace exactly as in conv_simt64_kernel.  Cout % 128 == 0.
template <bool PARTIAL>
__global__ void __launch_bounds__(128, 3) conv_simt88_kernel(const ConvDesc d, int Ho, int Wo, int KS, float* ws) {
    pdl_trigger();
    pdl_wait();
    constexpr int BM = 64, BN = 128, BK = 16;
    __shared__ __align__(16) float As[2][BK][BM + 4];
    __shared__ __align__(16) float Bs[2][BK][BN];

    const int g = blockIdx.z / KS, ks = blockIdx.z - g * KS;
    const float* in = (const float*)d.in + (size_t)g * d.in_gs;
    const float* w = d.w + (size_t)g * d.w_gs;
    const int M = Ho * Wo;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int tid = threadIdx.x;
    const int H = d.H, W = d.W, Cin = d.Cin, Cout = d.Cout, k = d.k, s = d.stride, p = d.k / 2;

    // A loads: 2 float4 per thread (pixel q >> 2, channels 4 (q & 3) .. +3), q = tid + 128 r
    int a_oh[2], a_ow[2];
    bool a_ok[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int m = m0 + ((tid + 128 * r) >> 2);
        a_ok[r] = m < M;
        a_oh[r] = a_ok[r] ? m / Wo : 0;
        a_ow[r] = a_ok[r] ? m - a_oh[r] * Wo : 0;
    }
    const int nck = Cin / BK, nsteps = k * k * nck;
    const int s_begin = (int)((long long)ks * nsteps / KS), s_end = (int)((long long)(ks + 1) * nsteps / KS);
    float4 ra[2][2], rb[2][4];
    // the next step to load, as (tap, ky, kx, channel chunk): steps are loaded in order
    int l_tap = s_begin / nck, l_ck = s_begin - l_tap * nck, l_ky = l_tap / k, l_kx = l_tap - l_ky * k;
    auto load_regs = [&](int, float4* qa, float4* qb) {
        const int tap = l_tap, c0 = l_ck * BK, ky = l_ky, kx = l_kx;
        if (++l_ck == nck) {
            l_ck = 0;
            ++l_tap;
            if (++l_kx == k) { l_kx = 0; ++l_ky; }
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int ih = a_oh[r] * s + ky - p, iw = a_ow[r] * s + kx - p;
            if (a_ok[r] && ih >= 0 && ih < H && iw >= 0 && iw < W)
                qa[r] = *reinterpret_cast<const float4*>(in + ((size_t)ih * W + iw) * Cin + c0 + ((tid + 128 * r) & 3) * 4);
            else
                qa[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {  // B: row q >> 5, channels n0 + 4 (q & 31) .. +3
            const int q = tid + 128 * r;
            qb[r] = *reinterpret_cast<const float4*>(w + ((size_t)tap * Cin + c0 + (q >> 5)) * Cout + n0 + (q & 31) * 4);
        }
    };
    auto store_smem = [&](int buf, const float4* qa, const float4* qb) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int q = tid + 128 * r, pix = q >> 2, cg = q & 3;
            As[buf][cg * 4 + 0][pix] = qa[r].x;
            As[buf][cg * 4 + 1][pix] = qa[r].y;
            As[buf][cg * 4 + 2][pix] = qa[r].z;
            As[buf][cg * 4 + 3][pix] = qa[r].w;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int q = tid + 128 * r;
            *reinterpret_cast<float4*>(&Bs[buf][q >> 5][(q & 31) * 4]) = qb[r];
        }
    };

    const int tn = tid & 15, tm = tid >> 4;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    auto fma_tile = [&](int buf) {
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][tm * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][32 + tm * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tn * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tn * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; j += 2) fma2_bcast(acc[i][j], acc[i][j + 1], av[i], bv[j], bv[j + 1]);
        }
    };
    if (s_begin < s_end) load_regs(s_begin, ra[0], rb[0]);
    if (s_begin + 1 < s_end) load_regs(s_begin + 1, ra[1], rb[1]);
    if (s_begin < s_end) store_smem(0, ra[0], rb[0]);
    __syncthreads();
    for (int t = s_begin; t < s_end; t += 2) {
        if (t + 2 < s_end) load_regs(t + 2, ra[0], rb[0]);
        fma_tile(0);
        if (t + 1 < s_end) store_smem(1, ra[1], rb[1]);
        __syncthreads();
        if (t + 1 >= s_end) break;
        if (t + 3 < s_end) load_regs(t + 3, ra[1], rb[1]);
        fma_tile(1);
        if (t + 2 < s_end) store_smem(0, ra[0], rb[0]);
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = m0 + (i < 4 ? tm * 4 + i : 32 + tm * 4 + i - 4);
        if (m >= M) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int co0 = n0 + h * 64 + tn * 4;
            if (PARTIAL) {
                *reinterpret_cast<float4*>(ws + (((size_t)g * KS + ks) * M + m) * Cout + co0) =
                    make_float4(acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2], acc[i][4 * h + 3]);
            } else {
                const int oh = m / Wo, ow = m - oh * Wo;
                const float* b = d.b + (size_t)g * d.b_gs + co0;
                float4 v = make_float4(acc[i][4 * h] + b[0], acc[i][4 * h + 1] + b[1], acc[i][4 * h + 2] + b[2],
                                       acc[i][4 * h + 3] + b[3]);
                if (d.act) { v.x = gelu_erf(v.x); v.y = gelu_erf(v.y); v.z = gelu_erf(v.z); v.w = gelu_erf(v.w); }
                store_out4(d, g, oh, ow, co0, v);
            }
        }
    }
}

// out = bias + (((range 0) + range 1) + ...), then the layer's activation and output mapping
__global__ void conv_simt_reduce_kernel(const ConvDesc d, int Ho, int Wo, int KS, const float* ws) {
    pdl_trigger();
    pdl_wait();
    // four channels per thread (Cout % 4 == 0 for the split layers); 32-bit element indices per group
    const int M = Ho * Wo, C4 = d.Cout >> 2;
    const int per_g4 = M * C4;
    const size_t per_g = (size_t)M * d.Cout;
    const long long total4 = (long long)per_g4 * d.groups;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total4; i += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(i / per_g4);
        const int r4 = (int)(i - (long long)g * per_g4);
        const int m = r4 / C4, co = (r4 - m * C4) * 4;
        const float* src = ws + (size_t)g * KS * per_g + (size_t)r4 * 4;
        float4 v = *reinterpret_cast<const float4*>(src);
        for (int ks = 1; ks < KS; ++ks) {
            const float4 u = *reinterpret_cast<const float4*>(src + (size_t)ks * per_g);
            v.x += u.x; v.y += u.y; v.z += u.z; v.w += u.w;
        }
        const float* b = d.b + (size_t)g * d.b_gs + co;
        v.x += b[0]; v.y += b[1]; v.z += b[2]; v.w += b[3];
        if (d.act) { v.x = gelu_erf(v.x); v.y = gelu_erf(v.y); v.z = gelu_erf(v.z); v.w = gelu_erf(v.w); }
        const int oh = m / Wo, ow = m - oh * Wo;
        store_out4(d, g, oh, ow, co, v);
    }
}

// The last hyper-synthesis layer's reduction with the entropy parameters formed in the same pass: each
// thread sums four mu columns and the four log sigma columns of the same channels (range sums in range
// order, then the bias, as conv_simt_reduce_kernel), writes mu (and log sigma with ent_keep_ls), the four
// scale indices and, with ent_y, the four quantised residuals -- the quantiser's arithmetic, term for term.
__global__ void conv_simt_reduce_entropy_kernel(const ConvDesc d, int M, int KS, const float* ws) {
    pdl_trigger();
    pdl_wait();
    __shared__ float thr[kBins - 1];
    const int qp = d.ent_qp_dev ? *d.ent_qp_dev : d.ent_qp;
    if (threadIdx.x < kBins - 1) thr[threadIdx.x] = d.ent_thr[qp * (kBins - 1) + threadIdx.x];
    __syncthreads();
    const float qinv = d.ent_qinv[qp];
    const int C = d.split, C4 = C >> 2;
    const size_t per = (size_t)M * d.Cout;
    const int total = M * C4;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int m = i / C4, c = (i - m * C4) * 4;
        const float* sm = ws + (size_t)m * d.Cout + c;
        const float* sl = sm + C;
        float4 mu = *reinterpret_cast<const float4*>(sm), ls = *reinterpret_cast<const float4*>(sl);
        for (int ks = 1; ks < KS; ++ks) {
            const float4 a = *reinterpret_cast<const float4*>(sm + ks * per);
            const float4 b = *reinterpret_cast<const float4*>(sl + ks * per);
            mu.x += a.x; mu.y += a.y; mu.z += a.z; mu.w += a.w;
            ls.x += b.x; ls.y += b.y; ls.z += b.z; ls.w += b.w;
        }
        mu.x += d.b[c]; mu.y += d.b[c + 1]; mu.z += d.b[c + 2]; mu.w += d.b[c + 3];
        ls.x += d.b[C + c]; ls.y += d.b[C + c + 1]; ls.z += d.b[C + c + 2]; ls.w += d.b[C + c + 3];
        const size_t o = (size_t)m * C + c;
        *reinterpret_cast<float4*>(static_cast<float*>(d.out) + o) = mu;
        if (d.ent_keep_ls) *reinterpret_cast<float4*>(d.out2 + o) = ls;
        const uint32_t id = (uint32_t)count_below(thr, ls.x) | ((uint32_t)count_below(thr, ls.y) << 8) |
                            ((uint32_t)count_below(thr, ls.z) << 16) | ((uint32_t)count_below(thr, ls.w) << 24);
        *reinterpret_cast<uint32_t*>(d.ent_idx + o) = id;
        if (d.ent_y) {
            const float4 y = *reinterpret_cast<const float4*>(d.ent_y + o);
            const float r0 = fminf(fmaxf(rintf(__fmul_rn(__fsub_rn(y.x, mu.x), qinv)), -255.0f), 255.0f);
            const float r1 = fminf(fmaxf(rintf(__fmul_rn(__fsub_rn(y.y, mu.y), qinv)), -255.0f), 255.0f);
            const float r2 = fminf(fmaxf(rintf(__fmul_rn(__fsub_rn(y.z, mu.z), qinv)), -255.0f), 255.0f);
            const float r3 = fminf(fmaxf(rintf(__fmul_rn(__fsub_rn(y.w, mu.w), qinv)), -255.0f), 255.0f);
            const uint32_t lo = (uint32_t)(uint16_t)(int16_t)r0 | ((uint32_t)(uint16_t)(int16_t)r1 << 16);
            const uint32_t hi = (uint32_t)(uint16_t)(int16_t)r2 | ((uint32_t)(uint16_t)(int16_t)r3 << 16);
            *reinterpret_cast<uint2*>(d.ent_rhat + o) = make_uint2(lo, hi);
        }
    }
}

// The launch rule, shared by the launcher and the workspace query.  Returns the tile kind
// (0: 128 x 16, 1: 128 x 64, 2: 64 x 64) and, for kind 2, the number of K ranges.
static int simt_plan(const ConvDesc& d, int* KS) {
    const int p = d.k / 2;
    const int Ho = (d.H + 2 * p - d.k) / d.stride + 1, Wo = (d.W + 2 * p - d.k) / d.stride + 1;
    const long long M = (long long)Ho * Wo;
    *KS = 1;
    if (d.Cout <= 16) return 0;
    const long long ctas128 = ((M + 127) / 128) * ((d.Cout + 63) / 64) * d.groups;
    if (ctas128 >= 4 * 148) return 1;
    const int nsteps16 = d.k * d.k * (d.Cin / 16);
    if (d.Cout % 128 == 0 && d.Cin % 16 == 0) {
        // small layers with 128-multiple widths (the hyper-synthesis): 64 x 128 tiles of 8 x 8 per
        // thread, K split into as many ranges as one wave of three CTAs per SM holds
        const long long ctas = ((M + 63) / 64) * (d.Cout / 128) * d.groups;
        long long ks = 3 * 148 / ctas;
        if (ks == 0 && nsteps16 >= 2) {
            // more than one wave (S3 at 1080p: 512 CTAs on 444 slots): halve K when the half-work CTAs pack
            // the waves tighter (3 waves of half the work against 2 of the whole)
            const long long slots = 3 * 148, w1 = (ctas + slots - 1) / slots, w2 = (2 * ctas + slots - 1) / slots;
            if (w2 < 2 * w1) ks = 2;
        }
        if (ks > 16) ks = 16;
        if (ks > nsteps16) ks = nsteps16;
        *KS = (int)(ks < 1 ? 1 : ks);
        return 3;
    }
    if (d.Cout % 4) return 2;  // (KS = 1: the split-K reduction handles four channels per thread)
    // other small layers: 64 x 64 tiles, K split until two CTAs per SM
    const long long ctas64 = ((M + 63) / 64) * ((d.Cout + 63) / 64) * d.groups;
    const int nsteps = d.k * d.k * (d.Cin / (d.Cin % 32 == 0 ? 32 : 16));
    long long ks = (2 * 148 + ctas64 - 1) / ctas64;
    if (ks > 9) ks = 9;
    if (ks > nsteps) ks = nsteps;
    *KS = (int)(ks < 1 ? 1 : ks);
    return 2;
}

size_t conv_simt_workspace(const ConvDesc& d) {
    if (conv_tf32x3_ok(d)) return conv_tf32x3_workspace(d);
    int KS;
    const int kind = simt_plan(d, &KS);
    if ((kind != 2 && kind != 3) || KS == 1) return 0;
    const int p = d.k / 2;
    const int Ho = (d.H + 2 * p - d.k) / d.stride + 1, Wo = (d.W + 2 * p - d.k) / d.stride + 1;
    return (size_t)KS * d.groups * Ho * Wo * d.Cout;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

static unsigned reduce_blocks(const ConvDesc& d, int M) {  // one thread per four output channels
    const size_t total4 = (size_t)d.groups * M * (d.Cout / 4);
    return (unsigned)((total4 + 255) / 256 < 4096 ? (total4 + 255) / 256 : 4096);
}

cudaError_t launch_conv_simt(const ConvDesc& d_in, cudaStream_t st, int* nl) {
    int nl_ = 0;
    if (!nl) nl = &nl_;
    ConvDesc d = d_in;
    d.vec4 = d.mode == OUT_NHWC && d.Cout % 4 == 0 && d.split % 4 == 0 && d.out_gs % 4 == 0 && aligned16(d.out) &&
             (!d.split || (aligned16(d.out2) && (d.Cout - d.split) % 4 == 0)) &&
             (!d.res || (aligned16(d.res) && d.res_gs % 4 == 0)) && aligned16(d.b) && d.b_gs % 4 == 0;
    const int p = d.k / 2;
    const int Ho = (d.H + 2 * p - d.k) / d.stride + 1, Wo = (d.W + 2 * p - d.k) / d.stride + 1;
    const int M = Ho * Wo;
    int KS;
    const int kind = simt_plan(d, &KS);
    // the entropy parameters of the last hyper-synthesis layer: in its split-K reduction when it has one
    // and the tensors allow four channels per thread, else by the quantiser after the layer
    const bool want_ent = d.ent_idx != nullptr;
    const bool tf = conv_tf32x3_ok(d);  // the TF32 three-product GEMM, then the range-sum reduction below
    const bool fuse_ent = want_ent && (tf || (kind == 3 && KS > 1)) && d.groups == 1 && d.mode == OUT_NHWC &&
                          d.act == 0 && !d.res && d.split > 0 && d.split % 4 == 0 && d.Cout == 2 * d.split &&
                          aligned16(d.out) && (!d.ent_keep_ls || aligned16(d.out2)) && aligned16(d.b) &&
                          (reinterpret_cast<uintptr_t>(d.ent_idx) & 3) == 0 &&
                          (!d.ent_y || (aligned16(d.ent_y) && (reinterpret_cast<uintptr_t>(d.ent_rhat) & 7) == 0));
    if (want_ent && !fuse_ent) {  // the layer as usual (mu and log sigma written), then the quantiser
        ConvDesc u = d_in;
        u.ent_idx = nullptr;
        u.ent_keep_ls = 1;
        cudaError_t e = launch_conv_simt(u, st, nl);
        if (e != cudaSuccess) return e;
        ++*nl;
        launch_quantize(d.ent_y, static_cast<const float*>(d.out), d.out2, (size_t)M * d.split, d.ent_thr, d.ent_qinv,
                        d.ent_qp_dev, d.ent_qp, d.ent_y ? d.ent_rhat : nullptr, d.ent_idx, st);
        return cudaGetLastError();
    }
    if (tf) {
        const float* sums = nullptr;
        cudaError_t e = launch_tf32x3_gemm(d, st, &KS, &sums);
        if (e != cudaSuccess) return e;
        *nl += 2;
        if (fuse_ent) {
            const int n4 = M * (d.split / 4);
            const unsigned blocks = (unsigned)((n4 + 255) / 256 < 4096 ? (n4 + 255) / 256 : 4096);
            ++*nl, (void)launch_pdl(conv_simt_reduce_entropy_kernel, dim3(blocks), dim3(256), (size_t)(0), st, d, M, KS,
                                    sums);
        } else {
            ++*nl, (void)launch_pdl(conv_simt_reduce_kernel, dim3(reduce_blocks(d, M)), dim3(256), (size_t)(0), st, d, Ho,
                                    Wo, KS, sums);
        }
        return cudaGetLastError();
    }
    if (kind == 0) {
        dim3 grid((M + 127) / 128, (d.Cout + 15) / 16, d.groups);
        ++*nl, (void)launch_pdl(conv_simt_kernel<128, 16>, dim3(grid), dim3(256), (size_t)(0), st, d, Ho, Wo);
    } else if (kind == 1) {
        dim3 grid((M + 127) / 128, (d.Cout + 63) / 64, d.groups);
        ++*nl, (void)launch_pdl(conv_simt_kernel<128, 64>, dim3(grid), dim3(256), (size_t)(0), st, d, Ho, Wo);
    } else if (kind == 3) {
        dim3 grid((M + 63) / 64, d.Cout / 128, d.groups * KS);
        if (KS > 1) {
            if (!d.ws || d.ws_cap < conv_simt_workspace(d)) return cudaErrorInvalidValue;
            ++*nl, (void)launch_pdl(conv_simt88_kernel<true>, dim3(grid), dim3(128), (size_t)(0), st, d, Ho, Wo, KS, d.ws);
            if (fuse_ent) {
                const int n4 = M * (d.split / 4);
                const unsigned blocks = (unsigned)((n4 + 255) / 256 < 4096 ? (n4 + 255) / 256 : 4096);
                ++*nl, (void)launch_pdl(conv_simt_reduce_entropy_kernel, dim3(blocks), dim3(256), (size_t)(0), st, d, M, KS,
                                 d.ws);
                return cudaGetLastError();
            }
            ++*nl, (void)launch_pdl(conv_simt_reduce_kernel, dim3(reduce_blocks(d, M)), dim3(256), (size_t)(0), st, d, Ho, Wo, KS, d.ws);
        } else {
            ++*nl, (void)launch_pdl(conv_simt88_kernel<false>, dim3(grid), dim3(128), (size_t)(0), st, d, Ho, Wo, 1, nullptr);
        }
    } else if (KS > 1) {
        if (!d.ws || d.ws_cap < conv_simt_workspace(d)) return cudaErrorInvalidValue;  // caller's workspace
        dim3 grid((M + 63) / 64, (d.Cout + 63) / 64, d.groups * KS);
        if (d.Cin % 32 == 0)
            ++*nl, (void)launch_pdl(conv_simt64_kernel<true, 32>, dim3(grid), dim3(256), (size_t)(0), st, d, Ho, Wo, KS, d.ws);
        else
            ++*nl, (void)launch_pdl(conv_simt64_kernel<true, 16>, dim3(grid), dim3(256), (size_t)(0), st, d, Ho, Wo, KS, d.ws);
        ++*nl, (void)launch_pdl(conv_simt_reduce_kernel, dim3(reduce_blocks(d, M)), dim3(256), (size_t)(0), st, d, Ho, Wo, KS, d.ws);
    } else {
        dim3 grid((M + 63) / 64, (d.Cout + 63) / 64, d.groups);
        if (d.Cin % 32 == 0)
            ++*nl, (void)launch_pdl(conv_simt64_kernel<false, 32>, dim3(grid), dim3(256), (size_t)(0), st, d, Ho, Wo, 1, nullptr);
        else
            ++*nl, (void)launch_pdl(conv_simt64_kernel<false, 16>, dim3(grid), dim3(256), (size_t)(0), st, d, Ho, Wo, 1, nullptr);
    }
    return cudaGetLastError();
}

}  // namespace ufvc
