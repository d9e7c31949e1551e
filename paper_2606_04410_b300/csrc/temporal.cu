// Temporal chunk context (Sec. 3.1, Fig. 3): the one elementwise step the context path needs besides
// the library's convolutions.  The prior is conditioned by adding PC(C_i) (a float tensor the size of
// the hyper-synthesis features) to those features before their last layer; the encoder and the decoder
// run this same kernel on the same values, so they obtain the same scales.
#include "ufvc_internal.h"

namespace ufvc {

namespace {

__global__ void add_f32_kernel(float* __restrict__ a, const float* __restrict__ b, size_t n) {
    pdl_trigger();
    pdl_wait();
    const size_t n4 = n >> 2;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        float4 x = reinterpret_cast<float4*>(a)[i];
        const float4 y = reinterpret_cast<const float4*>(b)[i];
        x.x = __fadd_rn(x.x, y.x); x.y = __fadd_rn(x.y, y.y); x.z = __fadd_rn(x.z, y.z); x.w = __fadd_rn(x.w, y.w);
        reinterpret_cast<float4*>(a)[i] = x;
    }
    for (size_t i = (n4 << 2) + (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        a[i] = __fadd_rn(a[i], b[i]);
}

}  // namespace

// a and b are 16-byte aligned (device allocations)
void launch_add_f32(float* a, const float* b, size_t n, cudaStream_t s) {
    size_t g = (n / 4 + 255) / 256;
    if (g > 148 * 8) g = 148 * 8;
    (void)launch_pdl(add_f32_kernel, dim3((unsigned)(g ? g : 1)), dim3(256), 0, s, a, b, n);
}

}  // namespace ufvc
