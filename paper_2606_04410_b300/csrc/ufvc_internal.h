// Internal declarations of libufvc (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>
#include <map>
#include <memory>

#include "../../include/ufvc.h"

namespace ufvc {

#ifdef __CUDACC__
// Programmatic dependent launch.  Kernels of the coding path are launched with programmatic stream
// serialization (launch_pdl): a kernel's CTAs may start while the previous kernel of the stream finishes,
// so its set-up overlaps that kernel's tail.  Every such kernel calls pdl_wait() before it reads anything
// an earlier kernel wrote or writes anything an earlier kernel reads (pdl_wait returns once the previous
// kernel has completed and its writes are visible), and pdl_trigger() to let the next kernel start.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// GELU x * Phi(x) with the normal CDF written as a logistic of an odd polynomial:
// Phi(x) ~= 1 / (1 + exp(-x P(min(x^2, 100)))), P(t) = 1.59501577 + 7.40112920e-2 t - 7.03033577e-4 t^2.
// P was fitted for this kernel by minimising max |x (Phi(x) - approximation)| over [-14, 14]: the GELU
// error is below 2.6e-5 everywhere (P > 0 on the clamped range, so the logistic saturates the right way
// for large |x|), against the 2^-9 relative rounding of the bf16 activation it feeds.  Cost: six FP32
// operations and two MUFU operations (ex2, rcp) with -log2(e) folded into the coefficients.
__device__ __forceinline__ float gelu_tc(float x) {
    const float t = fminf(x * x, 100.0f);
    float p = fmaf(t, 7.03033577e-4f * 1.44269504088896341f, -7.40112920e-2f * 1.44269504088896341f);
    p = fmaf(p, t, -1.59501577f * 1.44269504088896341f);
    float e, r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(p * x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.0f + e));
    return x * r;
}

// The same GELU for two values at once, the logistic taken as 0.5 + 0.5 tanh(z / 2) and z / 2 =
// x P(t) / 2 evaluated in packed half precision with one tanh.approx.f16x2 for both values; the final
// product x (0.5 + 0.5 tanh) is FP32.  Half precision adds about 1e-3 absolute to the logistic, so the
// GELU's relative error stays at or below the 2^-9 rounding of the bf16 activation it is stored as.
// (|x| > 255 squares to +inf in half precision and is clamped to t = 100; |x| beyond the half range
// gives tanh = +-1, the exact limits.)
__device__ __forceinline__ void gelu_tc2(float& a, float& b) {
    const __half2 x = __floats2half2_rn(a, b);
    const __half2 t = __hmin2(__hmul2(x, x), __float2half2_rn(100.0f));
    __half2 q = __hfma2(t, __float2half2_rn(-7.03033577e-4f * 0.5f), __float2half2_rn(7.40112920e-2f * 0.5f));
    q = __hfma2(q, t, __float2half2_rn(1.59501577f * 0.5f));
    const __half2 z = __hmul2(q, x);
    uint32_t ti;
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(ti) : "r"(*reinterpret_cast<const uint32_t*>(&z)));
    const float2 th = __half22float2(*reinterpret_cast<const __half2*>(&ti));
    a *= fmaf(0.5f, th.x, 0.5f);
    b *= fmaf(0.5f, th.y, 0.5f);
}

// Colour interface (the model's input is YUV444; callers give RGB or YUV): the three bytes of frame n's
// pixel (sh, sw) in the caller's format.  0, 1: RGB interleaved [N][H][W][3] (1 is converted with
// BT.709); 2: YUV444 planar [N][3][H][W]; 3: YUV420 planar per frame, Y [H][W] then U and V
// [ceil(H/2)][ceil(W/2)], each chroma sample serving its 2x2 block.
template <int FMT>
__device__ __forceinline__ void px_bytes(const uint8_t* __restrict__ fr, int n, int sh, int sw, int H, int W,
                                         uint32_t* b) {
    if (FMT <= 1) {
        const uint8_t* p = fr + ((size_t)n * H * W + (size_t)sh * W + sw) * 3;
        b[0] = __ldg(p); b[1] = __ldg(p + 1); b[2] = __ldg(p + 2);
    } else if (FMT == 2) {
        const size_t pl = (size_t)H * W;
        const uint8_t* p = fr + (size_t)n * 3 * pl + (size_t)sh * W + sw;
        b[0] = __ldg(p); b[1] = __ldg(p + pl); b[2] = __ldg(p + 2 * pl);
    } else {
        const int Wc = (W + 1) >> 1, Hc = (H + 1) >> 1;
        const size_t pl = (size_t)H * W, cpl = (size_t)Hc * Wc;
        const uint8_t* f = fr + (size_t)n * (pl + 2 * cpl);
        const size_t ci = (size_t)(sh >> 1) * Wc + (sw >> 1);
        b[0] = __ldg(f + (size_t)sh * W + sw); b[1] = __ldg(f + pl + ci); b[2] = __ldg(f + pl + cpl + ci);
    }
}

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) applies to the current device only.  smem_optin sets it
// for `func` on the current device the first time a size at least `bytes` is needed there (thread-safe;
// one record per kernel and device).  sm_count caches the SM count of the current device.
cudaError_t smem_optin(const void* func, int bytes);
int sm_count();
// clusters of two CTAs of `func` (smem bytes of dynamic shared memory, `threads` per CTA) that the current
// device holds at once (0 if none or unknown); cached per kernel and device, after smem_optin
int max_pairs(const void* func, int smem, int threads);

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// launch_pdl for clusters of two CTAs (a CTA pair sharing tcgen05.mma.cta_group::2); grid.x even
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl_pair(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                   Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = 2;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}
#endif

constexpr int kBins = 64;          // scale bins s_k, k = 0..63, log-spaced on [0.11, 64]
constexpr int kRmax = 255;         // |r^| <= 255
constexpr int kNsym = 511;         // symbols -255..255
constexpr uint32_t kProbM = 1u << 16;
constexpr uint32_t kRansL = 1u << 16;

#ifdef __CUDACC__
// #{k : thr[k] < v} for the 63 ascending scale-index thresholds (the scale index of log sigma v).  The
// thresholds are the log-domain midpoints of log-spaced bins, so they are nearly equally spaced: a
// linear guess from the first and last is within a step of the count, and the two loops move it to the
// exact count (for any guess, NaN and infinities included: the result is the comparisons', not the
// guess's).
__device__ __forceinline__ int count_below(const float* thr, float v) {
    const float t0 = thr[0], tl = thr[kBins - 2];
    const float gf = (v - t0) * (float)(kBins - 2) / (tl - t0) + 1.0f;
    int c = gf <= 0.0f ? 0 : gf >= (float)(kBins - 1) ? kBins - 1 : (int)gf;
    while (c > 0 && !(thr[c - 1] < v)) --c;
    while (c < kBins - 1 && thr[c] < v) ++c;
    return c;
}
#endif

// The BF16 space-to-depth input holds x * 255/256: a byte v is stored as v / 256, which bf16 represents
// exactly (eight significant bits), and the first layer's 2x2 weights are multiplied by 256/255, so the
// input planes add no rounding of their own to the analysis.
constexpr float kS2dInScale = 255.0f / 256.0f;

// ---------------------------------------------------------------------------------------------
// Host-side tables (FP64 construction, built once per context)
// ---------------------------------------------------------------------------------------------
struct HostTables {
    std::vector<uint32_t> freq;   // [64][511]
    std::vector<uint32_t> cum;    // [64][512]
    std::vector<uint32_t> packed; // [64][511]  (freq << 16) | cum   (both fit in 16 bits)
    std::vector<float> thr;       // [64 qp][63]  float(t_k + ln q(qp))
    std::vector<float> qstep;     // [64]  q(qp) as float
    std::vector<float> qinv;      // [64]  1/q(qp) as float
    std::vector<double> log_thr;  // [63]  t_k in FP64 (z^ RMS index)
    std::vector<uint8_t> dec;     // decoder table image (build_decode_tables)
};
void build_host_tables(HostTables& t);
double qstep_fp64(int qp);

// ---------------------------------------------------------------------------------------------
// Architecture
// ---------------------------------------------------------------------------------------------
struct Arch { int e0, e1, e2, cy, cz, cd1, cd2; };
bool get_arch(int arch, Arch* a);
bool layer_shape(int arch, int N, int l, int* cout, int* k, int* cin);
size_t weight_count(int arch, int N);
// progressive-mean blob: P1a P1b P2a P2b P3a P3b (a: 3x3, Cy + Cz -> Cz; b: 1x1, Cz -> Cy)
bool mean_layer_shape(int arch, int l, int* cout, int* k, int* cin);
size_t mean_weight_count(int arch);
constexpr int kMeanLayers = 6;
// DC-block model (arch 2): widths and the blob indices of its shared layers (encoder blocks from DC_E0,
// decoder blocks from DC_D0, context blocks from DC_G0, five layers each); frame layers from kDcShared,
// kDcPerFrame per frame position (FP, 3 blocks, FO)
constexpr int kDcC = 512, kDcCf = 256, kDcCc = 128, kDcCy = 256, kDcCz = 128;
enum DcLayer { DC_PE = 0, DC_EC = 1, DC_E0 = 2, DC_ED = 32, DC_H1 = 33, DC_H2, DC_S1, DC_S2, DC_S3, DC_PC, DC_DU,
               DC_FC, DC_D0 = 41, DC_G0 = 76, DC_GO = 131 };
constexpr int kDcShared = 132, kDcPerFrame = 17;
bool dc_layer_shape(int N, int l, int* cout, int* k, int* cin);
// DC-block kernels (dc.cu): patch-embedding pack, depth-wise 3x3 + GELU (weights [g][9][C] float), x8 output
void launch_pack_s2d8(const uint8_t* frames, int N, int H, int W, int H8, int W8, void* x, bool f32, int fmt,
                      cudaStream_t s);
void launch_dw_conv(const void* x, int G, int H, int W, int C, long long gs, const float* w, const float* b, void* out,
                    bool f32, cudaStream_t s);
void launch_ps8_out(const float* o, int N, int H8, int W8, int H, int W, void* frames, bool u8, cudaStream_t s);

// temporal chunk context: feature and context channels, and the shared layers (then DF per frame)
constexpr int kCf = 64, kCc = 64;
enum TemporalLayer { TL_EC = 0, TL_FD, TL_FC, TL_CG, TL_PC, TL_N };
bool temporal_layer_shape(int arch, int N, int l, int* cout, int* k, int* cin);
size_t temporal_weight_count(int arch, int N);

enum EncLayer { L_A1 = 0, L_A2, L_A3, L_XA, L_XB, L_A4, L_H1, L_H2, L_S1, L_S2, L_S3, L_NENC };
enum DecLayer { D_D0 = 0, D_R1A, D_R1B, D_U1, D_R2A, D_R2B, D_U2, D_U3, D_NDEC };

// ---------------------------------------------------------------------------------------------
// Convolution launch descriptor (shared by the FP32 SIMT and the tcgen05 kernels)
// ---------------------------------------------------------------------------------------------
enum OutMode { OUT_NHWC = 0, OUT_PS = 1, OUT_PS_FINAL_F32 = 2, OUT_PS_FINAL_U8 = 3 };

struct ConvDesc {
    const void* in = nullptr;   // NHWC [H][W][Cin] (float or bf16 by kernel)
    long long in_gs = 0;        // elements between groups (0: shared input)
    int H = 0, W = 0, Cin = 0;  // Cin: padded channel count of the stored tensor
    const float* w = nullptr;   // SIMT: [k*k][Cin][Cout] float
    long long w_gs = 0;
    const float* b = nullptr;   // [Cout]
    long long b_gs = 0;
    int Cout = 0, k = 3, stride = 1;
    int mode = OUT_NHWC;
    int act = 0;                // 1: GELU (exact erf form)
    void* out = nullptr;        // destination tensor
    long long out_gs = 0;
    int out_h = 0, out_w = 0;   // destination spatial dims (positions outside are dropped: crop)
    const void* res = nullptr;  // residual added after the activation (same layout as out)
    long long res_gs = 0;
    float* out2 = nullptr;      // channels >= split go to out2 (NHWC with Cout - split channels)
    int split = 0;
    int groups = 1;
    // tensor-core path
    const void* wtc = nullptr;  // bf16 [groups][cout_pad][k*k*Cin] (K-major)
    int cout_pad = 0;           // Cout rounded up to the N tile
    int out_f32 = 0;            // NHWC output stored as float (else bf16)
    int out_c_stride = 0;       // NHWC output channel count if different from Cout
    const float* btc = nullptr; // tensor-core bias in accumulator-column order (nullptr: same as b)
    int ps_major = 0;           // tensor-core weights in sub-pixel-major column order (pixel shuffle layers)
    const void* wsc = nullptr;  // final layer, scatter form: bf16 [groups][128][64] (row = tap x channel)
    // FP8 E4M3 (precision UFVC_FP8): weights [groups][cout_pad][k*k*Cin] E4M3; accumulator column co is
    // multiplied by cscale[g * b_gs + co]; out_inv != 0: E4M3 output (code = value * out_inv), else the
    // output is bf16 (or float with out_f32); res is then an E4M3 residual of scale res_s
    const void* w8 = nullptr;
    const float* cscale = nullptr;
    float out_inv = 0.f;
    float res_s = 0.f;
    float* ws = nullptr;        // SIMT split-K workspace (conv_simt_workspace(d) floats), or nullptr
    size_t ws_cap = 0;
    float* tc_ws = nullptr;     // tensor-core split-K workspace (conv_tc_workspace(d) floats), or nullptr
    size_t tc_ws_cap = 0;
    int* err = nullptr;         // device status word (bounded-wait timeouts)
    int vec4 = 0;               // SIMT: set by the launcher when NHWC outputs may be written 16 bytes at a time
    // tensor-core path: K steps (tap x 64-channel chunk, tap-major) whose weights are all zero and are
    // skipped (bit ks set = step ks runs; 0 = every step runs)
    unsigned long long kmask = 0;
    // tensor-core path: the staged BN = 256 layers may run on CTA pairs (tcgen05.mma.cta_group::2)
    int pairs = 1;
    // The last hyper-synthesis layer (columns [0, split) = mu, [split, Cout) = log sigma) with the entropy
    // parameters formed in its output pass: ent_idx = #{k : thr_qp[k] < log sigma} and, with ent_y,
    // ent_rhat = clamp(rint((y - mu) / q)), qp = *ent_qp_dev (or ent_qp).  mu goes to out; log sigma to
    // out2 only with ent_keep_ls.  Formed in the split-K reduction where there is one, else by the
    // quantiser after the layer (the same arithmetic either way).
    uint8_t* ent_idx = nullptr;
    const float* ent_y = nullptr;
    int16_t* ent_rhat = nullptr;
    const float* ent_thr = nullptr;   // [64 qp][63]
    const float* ent_qinv = nullptr;  // [64]
    const int* ent_qp_dev = nullptr;
    int ent_qp = 0;
    int ent_keep_ls = 1;
    // hyper-synthesis layers on the tensor cores (conv_tf32.cu): weights [Cout][k*k][3][Cin] float, the
    // TF32 parts (hi, lo, hi) of each weight; launched through launch_conv_simt, whose workspace then
    // holds the input's TF32 planes and the K-range sums
    const float* wtf = nullptr;
};

// api.cu internals used by the server: a context sharing another's weights, and a plan's device bytes
ufvc_ctx* ctx_clone_shared(const ufvc_ctx* base);
int ctx_color(const ufvc_ctx* ctx);   // the context's colour format (ufvc_color)
bool ctx_temporal(const ufvc_ctx* ctx);  // the context carries a temporal chunk context (C_i)
size_t ctx_plan_bytes(const ufvc_ctx* ctx, int W, int H);

// nl (optional): incremented by the number of kernels launched (the layer, its split-K reduction, the
// quantiser where the entropy parameters are not formed in the reduction)
cudaError_t launch_conv_simt(const ConvDesc& d, cudaStream_t s, int* nl = nullptr);
// floats of split-K workspace the SIMT launch of d uses (0: none)
size_t conv_simt_workspace(const ConvDesc& d);
cudaError_t launch_conv_tc(const ConvDesc& d, cudaStream_t s, int* nl = nullptr);  // nl: launches beyond the conv
// TF32 three-product GEMM of a hyper-synthesis layer (conv_tf32.cu): conv_tf32x3_ok(d) when d has wtf and
// a shape it takes (stride 1, k = 1 or 3, Cin % 32 == 0, Cout % 256 == 0, one group); the workspace holds
// the input's planes then the K-range sums; launch_tf32x3_gemm launches the planes and GEMM kernels and
// returns the number of K ranges and where their sums start
bool conv_tf32x3_ok(const ConvDesc& d);
size_t conv_tf32x3_workspace(const ConvDesc& d);
cudaError_t launch_tf32x3_gemm(const ConvDesc& d, cudaStream_t s, int* KS, const float** sums);
// A float32 tensor map with the 128-byte swizzle (conv_tc.cu); map points at a 64-byte aligned CUtensorMap
bool encode_f32_map_sw128(void* map, const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
                          const uint32_t* box);
int conv_tc_ksplit(const ConvDesc& d);         // K ranges of a split tensor-core layer (1: not split)
size_t conv_tc_workspace(const ConvDesc& d);   // floats of its range-sum workspace (0: none)
// fmt: the caller's colour format (ufvc_color); the network reads its three channels per frame
void launch_pack_bf16(const uint8_t* frames, int N, int H, int W, int Hp, int Wp, int Cp, __nv_bfloat16* x,
                      cudaStream_t s, bool s2d, int fmt);
// First analysis layer straight from the frame bytes (conv_first.cu), BF16, colour formats 0, 2, 3 and
// even N, 2 <= N <= 8 (first_layer_ct(N) = 0 otherwise).  first_layer_weights writes the swizzled bf16
// image (first_layer_weight_bytes(pitch) bytes) of the [64][3][3][3N] weights times scale with
// K = tap x pitch + channel, pitch = first_layer_pitch(N) (3N rounded up to 16).
// out = GELU(A1(frames)) bf16 NHWC [Ho][Wo][64].
int first_layer_ct(int n_frames);
int first_layer_pitch(int n_frames);
size_t first_layer_weight_bytes(int pitch);
void first_layer_weights(const float* w, int n_frames, float scale, int pitch, uint16_t* img);
bool encode_frames_map(void* map, const void* frames, int N, int H, int row_bytes, int box_x, int box_y);
// sel: 0 = the kernel the chunk path picks (TMA windows where first_layer_tma_ok), 1 = the register-staged
// kernel, 2 = the TMA kernel (cudaErrorInvalidValue where first_layer_tma_ok is false)
bool first_layer_tma_ok(int fmt, int W, const void* frames);
// out: bf16 NHWC [Ho][Wo][64], or E4M3 codes of value x out_inv when out_inv != 0
cudaError_t launch_first_layer(const uint8_t* frames, int fmt, int N, int H, int W, int Ho, int Wo, const void* wimg,
                               const float* bias, void* out, float out_inv, int* err, cudaStream_t s, int sel = 0);
// colour interface, output side (color.cu): x^ float [N][H][W][3] -> the caller's format (fmt 1..3), float
// or uint8; frame_bytes = bytes of one frame in format fmt
size_t frame_bytes(int fmt, int W, int H);
void launch_color_out(int fmt, bool f32, const float* x, int N, int H, int W, void* out, cudaStream_t s);

// ---------------------------------------------------------------------------------------------
// Elementwise / entropy kernels
// ---------------------------------------------------------------------------------------------
void launch_pack(const uint8_t* frames, int N, int H, int W, int Hp, int Wp, int Cp, float* x, cudaStream_t s,
                 int fmt);
void launch_zquant(const float* z, int npos, int cz, const uint64_t* zthr, int16_t* zhat, uint8_t* iz,
                   cudaStream_t s);
void launch_quantize(const float* y, const float* mu, const float* logsig, size_t n, const float* thr_all,
                     const float* qinv_all, const int* qp_dev, int qp_host, int16_t* rhat, uint8_t* idx,
                     cudaStream_t s);
void launch_scale_index(const float* logsig, size_t n, const float* thr_all, const int* qp_dev, uint8_t* idx,
                        cudaStream_t s);
void launch_i16_to_f32(const int16_t* a, size_t n, float* out, cudaStream_t s);
void launch_f32_to_bf16(const float* a, size_t n, __nv_bfloat16* out, cudaStream_t s);
void launch_f32_to_bf16_rows(const float* a, int H, int W, int C, __nv_bfloat16* out, int Wd, cudaStream_t s);
// FP8 E4M3 helpers: packed input rows of 64 bytes (scale 1/448), float -> E4M3 rows, |x| maximum
void launch_pack_fp8(const uint8_t* frames, int N, int H, int W, int Hp, int Wp, uint8_t* x, cudaStream_t s, int fmt);
void launch_f32_to_e4m3_rows(const float* a, int H, int W, int C, float inv, uint8_t* out, int Wd, cudaStream_t s);
void launch_absmax(const float* x, size_t n, float* slot, cudaStream_t s);

// rANS (rans.cu).  Encoding: one launch codes the sections of up to kRansMaxStreams streams (a chunk's
// stream: its z^ section, then its y^ section; or one bare section) and lays each stream out (lane counts,
// words, padding) after `base` header bytes, writing the header itself when hdr_len > 0.  The control
// block (tickets and published block totals) must be zero before the first launch; every launch leaves it
// zero.  Staging rows: [K][cap_lane] u16 per section, cap_lane >= n / K + 3.
constexpr int kRansMaxBlocks = 1024;
constexpr int kRansMaxStreams = 8;
constexpr int kRansMaxEncSec = 2 * kRansMaxStreams;
struct RansCtl {
    unsigned int ticket, done;
    uint64_t flag[kRansMaxBlocks];
};
struct RansEncSec {
    const int16_t* sym;       // symbols r^ in [-255, 255]
    const uint8_t* idx;       // table index per element, or per channel when idx_period > 0
    int idx_period;
    uint32_t n;
    int K;
    uint16_t* rows;
    int cap_lane;
    int stream;               // the stream (output) it belongs to; a stream's sections are consecutive
    int nblk, first, prev, last;  // set by the launcher
    int lpb;                  // set by the launcher: lanes per block (its first lpb threads)
};
struct RansEncStream {
    uint8_t* out;
    uint64_t capacity;
    uint64_t* nbytes;         // device: size of the stream written
    uint64_t base;            // first section's byte offset (the header length)
    int hdr_len;              // 0: no header
    uint8_t hdr20[20];        // the header's fixed fields, then cz scale indices from iz, then zeros
    const uint8_t* iz;
    int cz;
};
struct RansEncJob {
    RansEncSec s[kRansMaxEncSec];
    int nsec;
    RansEncStream st[kRansMaxStreams];
    int nstreams;
    int grid, lpb;            // set by the launcher: blocks, the largest section's lanes per block
    int stage_bytes;          // set by the launcher: the staged words' bytes in shared memory (16-aligned)
    RansCtl* ctl;
    int* status;
    long long spin;           // bound on the table-copy wait in clocks (0: about 2 s)
};
cudaError_t launch_rans_encode(RansEncJob& j, const uint32_t* packed_tables, cudaStream_t s);
size_t rans_ctl_bytes();

// Decoding sections of the same shape (K lanes, n elements, one per chunk) in one launch; the lane-count
// checks and offsets are inside the launch.  Output: r^ (int16) or, fused, y^ = r^ q + mu as bf16, float
// or E4M3 codes (q = qstep_all[*qp_dev], or qstep_all[qp_host]).  With hdr_cz > 0 every section's launch
// blocks first check its container header against the context (arch, N, W, H, Ky lanes of the latent
// section, K = Kz lanes here, the progressive-means and temporal flags) and the section's first block
// writes the rate and the version (2 for progressive means, else 1) to qp_out / ver_out.
enum { kDecSym = 0, kDecBf16 = 1, kDecF32 = 2, kDecE4M3 = 3 };
constexpr int kRansMaxDecSec = 8;
struct RansDecSec {
    const uint8_t* bits;
    uint64_t nbytes;                 // readable bytes from bits
    uint64_t sec_off;                // section offset, or read from sec_off_dev when that is not null
    const uint64_t* sec_off_dev;
    uint64_t expect_end;             // the section must end exactly here (0: anywhere up to nbytes) ...
    const uint64_t* expect_end_dev;  // ... or at the device value
    const uint8_t* idx;              // per element, or per channel (idx_period)
    uint64_t* next_off;              // device: the byte after the section (may be null)
    int16_t* sym;
    void* yout;
    const float* mu;
    const int* qp_dev;
    int* qp_out;
    int* ver_out;
};
struct RansDecJob {
    RansDecSec s[kRansMaxDecSec];
    int nsec;
    int idx_period;
    uint32_t n;
    int K;
    int out;
    const float* qstep_all;
    int qp_host;
    float inv8;
    int hdr_cz, arch, N, W, H, Ky, allow_pm, temporal;
    int* status;
    long long spin;
    int threads, bps;                // set by the launcher: threads per block, blocks per section
};
cudaError_t launch_rans_decode(RansDecJob& j, const uint8_t* dec_tables, cudaStream_t s);
// the decoder's table image (196864 bytes) from cum [64][512]
void build_decode_tables(const std::vector<uint32_t>& cum_all, std::vector<uint8_t>& out);

// y^ = r^ q + mu with q = qstep_all[*qp_dev] (qp_dev null: qstep_all[qp_host]); yf and / or yb may be null
void launch_dequant(const int16_t* rhat, const float* mu, size_t n, const float* qstep_all, const int* qp_dev,
                    float* yf, __nv_bfloat16* yb, cudaStream_t s, uint8_t* y8 = nullptr, float inv8 = 0.f,
                    int qp_host = 0);



// Progressive means (progressive.cu).  `in` is the mean network's input [Hy][Wy][Cy + Cz], float (f32)
// or bf16.  init: y^ of partition 0 (the encoder, y != null, first quantises partition 0 with mu0 into
// rhat) and the features s; step k: on partition k, mu <- muk, encoder r^ re-quantised, y^ into `in`
// (skipped when ver_dev is given and *ver_dev != 2).  qp from *qp_dev, else qp_host.
// temporal context (temporal.cu): a += b over n floats
void launch_add_f32(float* a, const float* b, size_t n, cudaStream_t s);

void launch_pm_init(const float* y, int16_t* rhat, const float* mu0, const float* s, int Hy, int Wy, int cy, int cz,
                    const float* qstep_all, const float* qinv_all, const int* qp_dev, int qp_host, void* in, bool f32,
                    cudaStream_t st);
void launch_pm_step(int k, const float* y, int16_t* rhat, float* mu, const float* muk, int Hy, int Wy, int cy, int cz,
                    const float* qstep_all, const float* qinv_all, const int* qp_dev, int qp_host, const int* ver_dev,
                    void* in, bool f32, cudaStream_t st);

}  // namespace ufvc

// context internals for other translation units (defined in api.cu)
namespace ufvc {
const uint32_t* ctx_packed_tables(const ufvc_ctx* c);
long long ctx_table_spin(const ufvc_ctx* c);
int* ctx_status_word(ufvc_ctx* c);
int ctx_device(const ufvc_ctx* c);
void ctx_set_error(ufvc_ctx* c, const char* msg);
}  // namespace ufvc
