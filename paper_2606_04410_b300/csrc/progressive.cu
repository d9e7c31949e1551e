// Progressive means over four latent partitions (Sec. 3.4, Fig. 4a and 4c).
//
// The single parameter pass (the hyper-synthesis) gives log sigma for every latent element and the
// means mu^0 of partition 0, so the scale indices, and with them the whole entropy-coding step, need
// nothing else.  The means of partitions 1, 2, 3 are estimated afterwards, one partition at a time,
// by a small network over the partitions already reconstructed and the hyper-synthesis features s:
//     in_k  = [ y^ on partitions < k (zero elsewhere) ; s ]          (Cy + Cz channels)
//     mu^k  = P_k,b( GELU( P_k,a(in_k) ) )                           (3x3 then 1x1)
// and on partition k:  encoder r^ = clamp(rint((y - mu^k) / q)),  both  y^ = r^ q + mu^k.
// The decoder runs the same steps after the single entropy-decoding step; it reproduces the encoder's
// means bit for bit because both run the same kernels on the same inputs.
//
// Partition (reading of the figure): channel group g = c / (Cy / 4), position t = 2 (h mod 2) +
// (w mod 2) in its 2x2 block, partition (t + g) mod 4.
//
// This file holds the two elementwise kernels of a step; the convolutions are the library's
// convolution kernels (tensor cores in BF16 / FP8 contexts, the FP32 SIMT kernel otherwise).
#include "ufvc_internal.h"

namespace ufvc {

namespace {

__device__ __forceinline__ int partition_of(int h, int w, int c, int cy) {
    return (2 * (h & 1) + (w & 1) + c / (cy >> 2)) & 3;
}

template <typename T>
__device__ __forceinline__ void store8(T* dst, const float* v);

template <>
__device__ __forceinline__ void store8<float>(float* dst, const float* v) {
    reinterpret_cast<float4*>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
}

template <>
__device__ __forceinline__ void store8<__nv_bfloat16>(__nv_bfloat16* dst, const float* v) {
    uint4 u;
    __nv_bfloat162 p0 = __floats2bfloat162_rn(v[0], v[1]), p1 = __floats2bfloat162_rn(v[2], v[3]);
    __nv_bfloat162 p2 = __floats2bfloat162_rn(v[4], v[5]), p3 = __floats2bfloat162_rn(v[6], v[7]);
    u.x = *reinterpret_cast<uint32_t*>(&p0);
    u.y = *reinterpret_cast<uint32_t*>(&p1);
    u.z = *reinterpret_cast<uint32_t*>(&p2);
    u.w = *reinterpret_cast<uint32_t*>(&p3);
    *reinterpret_cast<uint4*>(dst) = u;
}

__device__ __forceinline__ void load8(const float* src, float* v) {
    const float4 a = reinterpret_cast<const float4*>(src)[0], b = reinterpret_cast<const float4*>(src)[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

__device__ __forceinline__ void load8(const int16_t* src, float* v) {
    const uint4 u = *reinterpret_cast<const uint4*>(src);
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        v[2 * j] = (float)(int16_t)(w[j] & 0xFFFF);
        v[2 * j + 1] = (float)(int16_t)(w[j] >> 16);
    }
}

__device__ __forceinline__ void store8(int16_t* dst, const float* r) {
    uint4 u;
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
        w[j] = (uint32_t)(uint16_t)(int16_t)r[2 * j] | ((uint32_t)(uint16_t)(int16_t)r[2 * j + 1] << 16);
    u.x = w[0]; u.y = w[1]; u.z = w[2]; u.w = w[3];
    *reinterpret_cast<uint4*>(dst) = u;
}

// r^ = clamp(rint((y - m) / q), -255, 255) with explicitly rounded operations (the quantiser's formula)
__device__ __forceinline__ float quant(float y, float m, float qinv) {
    return fminf(fmaxf(rintf(__fmul_rn(__fsub_rn(y, m), qinv)), -255.0f), 255.0f);
}

// The step-0 input of the mean network: y^ on partition 0 (r^ q + mu^0; the encoder first quantises
// partition 0 with mu^0), zero on partitions 1..3, and the features s in channels [Cy, Cy + Cz).
// One thread per (pixel, run of 8 channels) of the Cy + Cz input channels.
template <typename T>
__global__ void pm_init_kernel(const float* __restrict__ y, int16_t* __restrict__ rhat, const float* __restrict__ mu0,
                               const float* __restrict__ s, int Hy, int Wy, int cy, int cz,
                               const float* __restrict__ qstep_all, const float* __restrict__ qinv_all,
                               const int* qp_dev, int qp_host, T* __restrict__ in) {
    pdl_trigger();
    pdl_wait();
    const int cin = cy + cz, g8 = cin >> 3;
    const int qp = qp_dev ? *qp_dev : qp_host;
    const float q = qstep_all[qp], qinv = qinv_all[qp];
    const long long total = (long long)Hy * Wy * g8;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int pix = (int)(t / g8), c0 = (int)(t - (long long)pix * g8) * 8;
        const int h = pix / Wy, w = pix - h * Wy;
        float v[8];
        if (c0 >= cy) {
            load8(s + (size_t)pix * cz + (c0 - cy), v);
        } else if (partition_of(h, w, c0, cy) == 0) {
            const size_t i = (size_t)pix * cy + c0;
            float m[8], r[8];
            load8(mu0 + i, m);
            if (y) {
                float yy[8];
                load8(y + i, yy);
#pragma unroll
                for (int j = 0; j < 8; ++j) r[j] = quant(yy[j], m[j], qinv);
                store8(rhat + i, r);
            } else {
                load8(rhat + i, r);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = __fadd_rn(__fmul_rn(r[j], q), m[j]);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = 0.f;
        }
        store8<T>(in + (size_t)pix * cin + c0, v);
    }
}

// Step k (1..3) on partition k: the mean mu^k replaces mu^0 in `mu`, the encoder (y != null)
// re-quantises r^ with it, and y^ = r^ q + mu^k enters the mean network's input for the next steps.
// A decoder whose stream was coded without progressive means (*ver_dev != 2) leaves everything as is.
template <typename T>
__global__ void pm_step_kernel(int k, const float* __restrict__ y, int16_t* __restrict__ rhat, float* __restrict__ mu,
                               const float* __restrict__ muk, int Hy, int Wy, int cy, int cz,
                               const float* __restrict__ qstep_all, const float* __restrict__ qinv_all,
                               const int* qp_dev, int qp_host, const int* ver_dev, T* __restrict__ in) {
    pdl_trigger();
    pdl_wait();
    if (ver_dev && *ver_dev != 2) return;
    const int cin = cy + cz, g8 = cy >> 3;
    const int qp = qp_dev ? *qp_dev : qp_host;
    const float q = qstep_all[qp], qinv = qinv_all[qp];
    const long long total = (long long)Hy * Wy * g8;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int pix = (int)(t / g8), c0 = (int)(t - (long long)pix * g8) * 8;
        const int h = pix / Wy, w = pix - h * Wy;
        if (partition_of(h, w, c0, cy) != k) continue;
        const size_t i = (size_t)pix * cy + c0;
        float m[8], r[8], v[8];
        load8(muk + i, m);
        if (y) {
            float yy[8];
            load8(y + i, yy);
#pragma unroll
            for (int j = 0; j < 8; ++j) r[j] = quant(yy[j], m[j], qinv);
            store8(rhat + i, r);
        } else {
            load8(rhat + i, r);
        }
        store8<float>(mu + i, m);
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = __fadd_rn(__fmul_rn(r[j], q), m[j]);
        store8<T>(in + (size_t)pix * cin + c0, v);
    }
}

unsigned pm_grid(long long n) {
    long long g = (n + 255) / 256;
    if (g > 148 * 8) g = 148 * 8;
    return (unsigned)(g ? g : 1);
}

}  // namespace

void launch_pm_init(const float* y, int16_t* rhat, const float* mu0, const float* s, int Hy, int Wy, int cy, int cz,
                    const float* qstep_all, const float* qinv_all, const int* qp_dev, int qp_host, void* in, bool f32,
                    cudaStream_t st) {
    const long long n = (long long)Hy * Wy * ((cy + cz) >> 3);
    if (f32)
        (void)launch_pdl(pm_init_kernel<float>, dim3(pm_grid(n)), dim3(256), 0, st, y, rhat, mu0, s, Hy, Wy, cy, cz,
                         qstep_all, qinv_all, qp_dev, qp_host, static_cast<float*>(in));
    else
        (void)launch_pdl(pm_init_kernel<__nv_bfloat16>, dim3(pm_grid(n)), dim3(256), 0, st, y, rhat, mu0, s, Hy, Wy,
                         cy, cz, qstep_all, qinv_all, qp_dev, qp_host, static_cast<__nv_bfloat16*>(in));
}

void launch_pm_step(int k, const float* y, int16_t* rhat, float* mu, const float* muk, int Hy, int Wy, int cy, int cz,
                    const float* qstep_all, const float* qinv_all, const int* qp_dev, int qp_host, const int* ver_dev,
                    void* in, bool f32, cudaStream_t st) {
    const long long n = (long long)Hy * Wy * (cy >> 3);
    if (f32)
        (void)launch_pdl(pm_step_kernel<float>, dim3(pm_grid(n)), dim3(256), 0, st, k, y, rhat, mu, muk, Hy, Wy, cy,
                         cz, qstep_all, qinv_all, qp_dev, qp_host, ver_dev, static_cast<float*>(in));
    else
        (void)launch_pdl(pm_step_kernel<__nv_bfloat16>, dim3(pm_grid(n)), dim3(256), 0, st, k, y, rhat, mu, muk, Hy,
                         Wy, cy, cz, qstep_all, qinv_all, qp_dev, qp_host, ver_dev, static_cast<__nv_bfloat16*>(in));
}

}  // namespace ufvc
