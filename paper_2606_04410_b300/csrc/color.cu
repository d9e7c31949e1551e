// Colour interface, output side (the model's output is YUV444; the Appendix converts it back to the
// caller's format).  The final decoder layer writes x^ = clamp(0.5 + o, 0, 1) as float [N][H][W][3];
// this kernel maps it to the caller's layout:
//   1: RGB interleaved through BT.709 (R = Y + 1.5748 (V - 0.5), B = Y + 1.8556 (U - 0.5),
//      G = (Y - 0.2126 R - 0.0722 B) / 0.7152), clamped to [0, 1];
//   2: YUV444 planar [N][3][H][W];
//   3: YUV420 planar per frame: Y [H][W], then U and V [ceil(H/2)][ceil(W/2)], each chroma sample the
//      mean of its 2x2 block's pixels inside the frame.
// Values are written as float, or as uint8 rint(255 v) (round half to even).
#include "ufvc_internal.h"

namespace ufvc {

namespace {

template <bool F32>
__device__ __forceinline__ void put(void* out, size_t i, float v) {
    if (F32) static_cast<float*>(out)[i] = v;
    else static_cast<uint8_t*>(out)[i] = (uint8_t)rintf(255.0f * v);
}

// one thread per pixel (formats 1, 2)
template <int FMT, bool F32>
__global__ void color_out_px_kernel(const float* __restrict__ x, int N, int H, int W, void* __restrict__ out) {
    pdl_trigger();
    pdl_wait();
    const size_t pl = (size_t)H * W, total = (size_t)N * pl;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const float* v = x + 3 * t;
        const float y = v[0], u = v[1], w = v[2];
        if (FMT == 1) {
            const float r = fmaf(1.5748f, w - 0.5f, y), b = fmaf(1.8556f, u - 0.5f, y);
            const float g = (y - 0.2126f * r - 0.0722f * b) * (1.0f / 0.7152f);
            put<F32>(out, 3 * t, fminf(fmaxf(r, 0.f), 1.f));
            put<F32>(out, 3 * t + 1, fminf(fmaxf(g, 0.f), 1.f));
            put<F32>(out, 3 * t + 2, fminf(fmaxf(b, 0.f), 1.f));
        } else {
            const size_t n = t / pl, i = t - n * pl;
            put<F32>(out, (3 * n) * pl + i, y);
            put<F32>(out, (3 * n + 1) * pl + i, u);
            put<F32>(out, (3 * n + 2) * pl + i, w);
        }
    }
}

// one thread per 2x2 block (format 3): its (up to) four luma samples and one U, one V
template <bool F32>
__global__ void color_out_420_kernel(const float* __restrict__ x, int N, int H, int W, void* __restrict__ out) {
    pdl_trigger();
    pdl_wait();
    const int Hc = (H + 1) >> 1, Wc = (W + 1) >> 1;
    const size_t pl = (size_t)H * W, cpl = (size_t)Hc * Wc, fb = pl + 2 * cpl, total = (size_t)N * cpl;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const size_t n = t / cpl, ci = t - n * cpl;
        const int hc = (int)(ci / Wc), wc = (int)(ci - (size_t)hc * Wc);
        float su = 0.f, sv = 0.f;
        int cnt = 0;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const int h = 2 * hc + dy, w = 2 * wc + dx;
                if (h < H && w < W) {
                    const float* v = x + 3 * (n * pl + (size_t)h * W + w);
                    put<F32>(out, n * fb + (size_t)h * W + w, v[0]);
                    su += v[1];
                    sv += v[2];
                    ++cnt;
                }
            }
        const float inv = cnt == 4 ? 0.25f : (cnt == 2 ? 0.5f : 1.0f);
        put<F32>(out, n * fb + pl + ci, su * inv);
        put<F32>(out, n * fb + pl + cpl + ci, sv * inv);
    }
}

unsigned color_grid(size_t n) {
    size_t g = (n + 255) / 256;
    if (g > 148 * 16) g = 148 * 16;
    return (unsigned)(g ? g : 1);
}

}  // namespace

size_t frame_bytes(int fmt, int W, int H) {
    if (fmt == UFVC_COLOR_YUV420P) return (size_t)H * W + 2 * (size_t)((H + 1) / 2) * ((W + 1) / 2);
    return (size_t)3 * H * W;
}

void launch_color_out(int fmt, bool f32, const float* x, int N, int H, int W, void* out, cudaStream_t s) {
    const size_t npix = (size_t)N * H * W;
    const size_t nblk = (size_t)N * ((H + 1) / 2) * ((W + 1) / 2);
    if (fmt == UFVC_COLOR_YUV420P) {
        if (f32) (void)launch_pdl(color_out_420_kernel<true>, dim3(color_grid(nblk)), dim3(256), 0, s, x, N, H, W, out);
        else (void)launch_pdl(color_out_420_kernel<false>, dim3(color_grid(nblk)), dim3(256), 0, s, x, N, H, W, out);
    } else if (fmt == UFVC_COLOR_RGB_BT709) {
        if (f32) (void)launch_pdl(color_out_px_kernel<1, true>, dim3(color_grid(npix)), dim3(256), 0, s, x, N, H, W, out);
        else (void)launch_pdl(color_out_px_kernel<1, false>, dim3(color_grid(npix)), dim3(256), 0, s, x, N, H, W, out);
    } else {
        if (f32) (void)launch_pdl(color_out_px_kernel<2, true>, dim3(color_grid(npix)), dim3(256), 0, s, x, N, H, W, out);
        else (void)launch_pdl(color_out_px_kernel<2, false>, dim3(color_grid(npix)), dim3(256), 0, s, x, N, H, W, out);
    }
}

}  // namespace ufvc
