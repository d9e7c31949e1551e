// C-ABI entry points of libufvc: context, per-shape plans, and the chunk encode / decode pipelines.
//
// Encode (Sec. 3.1, 3.4): pack -> analysis A1..A3, cross-frame interaction X, A4 -> y; hyper-analysis
// H1, H2 -> z; z^ and its per-channel index; hyper-synthesis S1..S3 -> (mu, log sigma) for every
// latent element in ONE pass; r^ and scale indices; both rANS sections in one launch; header and
// lane layout.  Decode: header + lane counts; z^ section; the same hyper-synthesis; indices; the whole
// latent in ONE decoding step fused with y^ = r^ q + mu; the N frame-specific decoders (Sec. 3.2) as
// grouped launches (group = frame position, each with its own weights).
#include "ufvc_internal.h"

#include <algorithm>
#include <cuda_fp8.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

using namespace ufvc;

namespace {

struct LayerW {
    int cout = 0, k = 0, cin = 0, cin_p = 0, groups = 1;
    float* w = nullptr;  // FP32 SIMT layout [k*k][cin_p][cout] per group, groups back to back
    float* b = nullptr;  // [cout] per group
    long long w_gs = 0, b_gs = 0;
    // tensor-core copy (BF16 precision): bf16 [groups][cout_pad][k*k][cin_tc], K-major
    __nv_bfloat16* wtc = nullptr;
    int cout_pad = 0, cin_tc = 0;
    // pixel-shuffle layers: tensor-core rows (accumulator columns) in sub-pixel-major order, row
    // s * cout/4 + c = output channel 4c + s, so that a run of columns is a run of channels of ONE
    // output pixel; btc holds the biases in the same order
    int ps_major = 0;
    float* btc = nullptr;
    // final layer (3x3, 64 -> 12, pixel shuffle, frame mapping) in scatter form: bf16 [groups][128][64],
    // row 32 (c / 3) + 9 ky + 3 kx + c % 3 = the 64 input-channel weights of output channel c at tap
    // (ky, kx); the other rows zero
    __nv_bfloat16* wsc = nullptr;
    // FP8 E4M3 copy (precision UFVC_FP8): E4M3 codes [groups][cout_pad][tap][cin_tc] in the row order of
    // wtc, weight = code * wscale[g][row] with wscale = absmax over the output channel's weights / 448;
    // after calibration cs8[g][row] = (input tensor scale) * wscale, out_inv = 1 / (output tensor scale)
    // (0: the output is bf16 or float), res_s = the residual tensor's scale
    uint8_t* w8 = nullptr;
    std::vector<float> wscale;
    float* cs8 = nullptr;
    float out_inv = 0.f, res_s = 0.f;
    unsigned long long kmask = 0;  // tensor-core K steps that run (0: all); see ConvDesc::kmask
    // hyper-synthesis layers of the plain model (every precision): [cout][k*k][3][cin] float, the TF32
    // parts (hi, lo, hi) of each weight for the three-product tensor-core GEMM (conv_tf32.cu)
    float* wtf = nullptr;
};

// Activation tensors of the FP8 path, each with one per-tensor scale (absmax / 448 on the FP32 path of a
// calibration chunk; the packed input in [0, 1] has 1 / 448).
enum Fp8Tensor { T_X = 0, T_A1, T_A2, T_A3, T_XT, T_A3R, T_Y, T_HB, T_YHAT, T_D0, T_R1A, T_R1B, T_U1, T_R2A,
                 T_R2B, T_NT };

// Split-K workspace of the SIMT convolution, grown on first use.  One per direction of a plan (an
// encode and a decode may run concurrently on different streams) and one for the stage entry points.
struct Workspace {
    float* p = nullptr;
    size_t cap = 0;
};

struct Plan {
    int W = 0, H = 0, Hp = 0, Wp = 0, C0p = 0;
    int h1 = 0, w1 = 0, h2 = 0, w2 = 0, h3 = 0, w3 = 0, Hy = 0, Wy = 0, hh = 0, wh = 0, Hz = 0, Wz = 0;
    size_t ny = 0, nz = 0, hdr = 0;
    int Kz = 0, cap_z = 0, cap_y = 0;
    // encoder buffers
    float *x = nullptr, *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *xt = nullptr, *y = nullptr, *hb = nullptr,
          *z = nullptr, *zf = nullptr, *s1 = nullptr, *s2 = nullptr, *mu = nullptr, *ls = nullptr;
    int16_t *zhat = nullptr, *rhat = nullptr;
    uint8_t *iz = nullptr, *idx = nullptr;
    uint16_t *scr_z = nullptr, *scr_y = nullptr;  // rANS staging rows of the two sections
    RansCtl* ctl = nullptr;                       // rANS layout control block (zero between launches)
    uint64_t* zthr = nullptr;
    // decoder buffers
    int16_t *dzhat = nullptr, *drhat = nullptr;
    uint8_t* didx = nullptr;
    int* qp_dev = nullptr;
    uint64_t* next_z = nullptr;  // the byte after the z^ section
    float *dzf = nullptr, *ds1 = nullptr, *ds2 = nullptr, *dmu = nullptr, *dls = nullptr, *yhat = nullptr;
    __nv_bfloat16* yhat_bf = nullptr;
    // BF16 hyper-analysis inputs, rows and columns rounded up to even sizes (zero) for the stride-2 view
    int Hye = 0, Wye = 0, hhe = 0, whe = 0;
    __nv_bfloat16 *y_bf = nullptr, *hb_bf = nullptr;
    // decoder activations: float in FP32 precision, bf16 (same buffers, half used) otherwise
    float *bufA = nullptr, *bufT = nullptr, *bufB = nullptr, *bufT2 = nullptr, *bufC = nullptr;
    int* ver_dev = nullptr;  // decoder: container version of the stream being decoded
    float* fstage = nullptr; // decoder, colour formats other than RGB: x^ float [N][H][W][3] before conversion
    // progressive means, per direction: the mean network's input [Hy][Wy][Cy + Cz] and hidden layer
    // [Hy][Wy][Cz] (float in FP32 precision, bf16 otherwise), and the step's means [Hy][Wy][Cy] (float)
    float *pm_in_e = nullptr, *pm_h_e = nullptr, *pm_mu_e = nullptr;
    float *pm_in_d = nullptr, *pm_h_d = nullptr, *pm_mu_d = nullptr;
    bool pm_enc_ready = false, pm_dec_ready = false;
    // temporal context: the all-zero context of a stream's first chunk [H8][W8][Cc], the chunk feature
    // [H8][W8][Cf] (activation type) and the prior's context term [Hy][Wy][Cz] (float) per direction, and
    // the encoder's own y^ (activation type) from which it tracks the decoder's context
    float *t_zero = nullptr, *t_F_e = nullptr, *t_pc_e = nullptr, *t_yh_e = nullptr, *t_F_d = nullptr,
          *t_pc_d = nullptr;
    bool t_enc_ready = false, t_dec_ready = false;
    // DC-block model activations (activation type; o float): encoder s2d input, trunk and block scratch;
    // decoder trunk, block scratch and the frame decoders' [N][H8][W8][.] tensors
    float *dc_x0 = nullptr, *dc_h = nullptr, *dc_t1e = nullptr, *dc_t2e = nullptr, *dc_t3e = nullptr;
    float *dc_F = nullptr, *dc_t1d = nullptr, *dc_t2d = nullptr, *dc_t3d = nullptr, *dc_hf = nullptr,
          *dc_f1 = nullptr, *dc_f2 = nullptr, *dc_f3 = nullptr, *dc_o = nullptr;
    bool enc_ready = false, dec_ready = false;
    std::vector<void*> allocs;
    Workspace ws_enc, ws_dec;
};

struct ProfEntry {
    char name[32];
    cudaEvent_t a = nullptr, b = nullptr;
    int launches = 0;
};

}  // namespace

struct ufvc_ctx {
    ufvc_config cfg{};
    Arch arch{};
    int N = 0;
    HostTables tabs;
    uint32_t* d_packed = nullptr;
    uint8_t* d_dec = nullptr;  // rANS decoding tables (build_decode_tables)
    float *d_thr = nullptr, *d_qstep = nullptr, *d_qinv = nullptr;
    int* d_status = nullptr;
    long long table_spin = 0;  // bound on the entropy kernels' table-copy wait (clocks; 0: about 2 s)
    int conv_pairs = 1;        // the staged BN = 256 tensor-core layers run on CTA pairs
    int conv_launches = 0;     // kernels launched by conv() (the profiler's launch counts)
    LayerW enc[L_NENC];
    LayerW dec[D_NDEC];
    // BF16 with 3N <= 32: A1 as a 2x2 stride-1 layer on the space-to-depth input (the 3x3 stride-2
    // taps regrouped by 2x2 super-pixel; weight rows [64][tap][sub-pixel][32]; bias shared with enc[L_A1])
    LayerW a1s2d;
    void* first_w = nullptr;  // A1's weight image for the kernels that read frame bytes (BF16 and FP8)
    // progressive means (ufvc_set_progressive_means): P1a P1b P2a P2b P3a P3b; pm_on selects version-2
    // streams (partitions 1..3 coded with the progressive means)
    LayerW pm[kMeanLayers];
    bool pm_on = false;
    int color = UFVC_COLOR_RGB;  // the caller's frame format (ufvc_color)
    // temporal chunk context (ufvc_set_temporal_context): EC FD FC CG PC and the per-frame DF (grouped);
    // cur_cin / cur_cout: the context buffers of the call in progress (null: first chunk / not wanted)
    LayerW tl[TL_N];
    LayerW tdf;
    bool tc_on = false;
    int cc = kCc;  // temporal context channels
    // DC-block model (arch 2): its shared layers by blob index (depth-wise layers: w = [9][C] float) and
    // the frame-decoder layers grouped over the frame positions; it always carries the temporal context
    bool dcm = false;
    std::vector<LayerW> dcl;
    LayerW dcf[kDcPerFrame];
    const void* cur_cin = nullptr;
    void* cur_cout = nullptr;
    std::map<long long, Plan*> plans;
    std::string err;
    // standalone rANS scratch
    uint16_t* r_scr = nullptr;  // ufvc_rans_encode: staging rows and layout control block
    RansCtl* r_ctl = nullptr;
    size_t r_scr_words = 0;
    // host-API staging
    uint8_t *st_frames = nullptr, *st_bits = nullptr;
    uint64_t* st_nbytes = nullptr;
    size_t st_frames_sz = 0, st_bits_sz = 0;
    // profiling
    bool prof_on = false;
    std::vector<ProfEntry> prof;
    size_t prof_n = 0;
    // SIMT split-K workspace for the stage entry points, and the one the running call uses
    Workspace ws_stage;
    Workspace* cur_ws = &ws_stage;
    // weights and tables borrowed from another context (ctx_clone_shared): not freed here
    bool borrowed = false;
    // FP8: per-tensor activation scales (calibrated), and the absmax probe of a calibration run
    bool fp8_ready = false;
    float act_scale[T_NT] = {};
    float* amax = nullptr;  // device [T_NT] while a calibration run records activation maxima
};

// ------------------------------------------------------------------------------------------------
// helpers
// ------------------------------------------------------------------------------------------------
#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                         \
            return e_ == cudaErrorMemoryAllocation ? UFVC_ERR_OOM : UFVC_ERR_CUDA;                 \
        }                                                                                          \
    } while (0)

static ufvc_status fail(ufvc_ctx* ctx, ufvc_status s, const char* msg) {
    if (ctx) ctx->err = msg;
    return s;
}

template <class T>
static ufvc_status dalloc(ufvc_ctx* ctx, Plan* p, T** ptr, size_t count) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, count ? count * sizeof(T) : 16);
    if (e != cudaSuccess) {
        ctx->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        return UFVC_ERR_OOM;
    }
    if (p) p->allocs.push_back(v);
    *ptr = (T*)v;
    return UFVC_OK;
}

static void prof_begin(ufvc_ctx* ctx, const char* name, cudaStream_t s) {
    if (!ctx->prof_on) return;
    if (ctx->prof_n == ctx->prof.size()) {
        ProfEntry e;
        cudaEventCreate(&e.a);
        cudaEventCreate(&e.b);
        ctx->prof.push_back(e);
    }
    ProfEntry& e = ctx->prof[ctx->prof_n];
    snprintf(e.name, sizeof(e.name), "%s", name);
    e.launches = 0;
    cudaEventRecord(e.a, s);
}

static void prof_end(ufvc_ctx* ctx, cudaStream_t s, int launches) {
    if (!ctx->prof_on) return;
    ProfEntry& e = ctx->prof[ctx->prof_n++];
    e.launches = launches;
    cudaEventRecord(e.b, s);
}

static int ceil_div(int a, int b) { return (a + b - 1) / b; }
static int conv_out(int x, int k, int s) { return (x + 2 * (k / 2) - k) / s + 1; }

// One convolution launch.  Layers with a tensor-core weight copy run on tcgen05 in BF16 precision
// (bf16 activations in and out, except out_f32); all others (and every layer in FP32 precision) run on
// the deterministic FP32 SIMT kernel.
// The entropy parameters formed with the last hyper-synthesis layer (ConvDesc::ent_*): scale indices, and
// with y the quantised residuals
struct EntParams {
    uint8_t* idx;
    const float* y;
    int16_t* rhat;
    const int* qp_dev;
    int qp;
    bool keep_ls;
};

static ufvc_status conv(ufvc_ctx* ctx, const LayerW& L, const void* in, int H, int W, int stride, int act, int mode,
                        void* out, int out_h, int out_w, cudaStream_t s, const void* res = nullptr,
                        float* out2 = nullptr, int split = 0, long long in_gs = 0, long long out_gs = 0,
                        long long res_gs = 0, int groups = 1, bool out_f32 = false, const EntParams* ent = nullptr);

static bool use_tc(const ufvc_ctx* ctx, const LayerW& L);

// ------------------------------------------------------------------------------------------------
// plans
// ------------------------------------------------------------------------------------------------
static void free_plan(Plan* p) {
    for (void* v : p->allocs) cudaFree(v);
    cudaFree(p->ws_enc.p);
    cudaFree(p->ws_dec.p);
    delete p;
}

static void init_plan_shape(const ufvc_ctx* ctx, Plan* p, int W, int H) {
    p->W = W; p->H = H;
    p->Hp = ceil_div(H, 16) * 16; p->Wp = ceil_div(W, 16) * 16;
    // packed input channels: 16-multiple for the SIMT kernel; for tcgen05 one 64-channel stage, or in BF16
    // one 32-channel stage when the 3N frame channels fit (N <= 10)
    p->C0p = ctx->cfg.precision == UFVC_FP32                              ? ceil_div(3 * ctx->N, 16) * 16
             : (ctx->cfg.precision == UFVC_BF16 && 3 * ctx->N <= 32) ? 32
                                                                     : ceil_div(3 * ctx->N, 64) * 64;
    p->h1 = conv_out(p->Hp, 3, 2); p->w1 = conv_out(p->Wp, 3, 2);
    p->h2 = conv_out(p->h1, 3, 2); p->w2 = conv_out(p->w1, 3, 2);
    p->h3 = conv_out(p->h2, 3, 2); p->w3 = conv_out(p->w2, 3, 2);
    p->Hy = conv_out(p->h3, 3, 2); p->Wy = conv_out(p->w3, 3, 2);
    p->hh = conv_out(p->Hy, 3, 2); p->wh = conv_out(p->Wy, 3, 2);
    p->Hz = conv_out(p->hh, 3, 2); p->Wz = conv_out(p->wh, 3, 2);
    p->Hye = p->Hy + (p->Hy & 1); p->Wye = p->Wy + (p->Wy & 1);
    p->hhe = p->hh + (p->hh & 1); p->whe = p->wh + (p->wh & 1);
    p->ny = (size_t)p->Hy * p->Wy * ctx->arch.cy;
    p->nz = (size_t)p->Hz * p->Wz * ctx->arch.cz;
    p->Kz = (size_t)ctx->cfg.lanes < p->nz ? ctx->cfg.lanes : (int)p->nz;
    p->cap_z = (int)(p->nz / p->Kz + 3);
    p->cap_y = (int)(p->ny / ctx->cfg.lanes + 3);
    p->hdr = (20 + (size_t)ctx->arch.cz + 3) & ~(size_t)3;
}

// The device buffers of a plan's encoder (enc) and decoder (dec) halves: allocated, or with dry_bytes only
// counted (256-byte granules).  Activations that the tensor cores read and write are bf16 in BF16
// precision (the float-typed buffers are then half used), float otherwise.
static ufvc_status plan_buffers(ufvc_ctx* ctx, Plan* p, bool enc, bool dec, size_t* dry_bytes) {
    const Arch& a = ctx->arch;
    const int N = ctx->N, K = ctx->cfg.lanes;
    const bool fp32 = ctx->cfg.precision == UFVC_FP32;
    const size_t act = fp32 ? 1 : 2;  // activation elements per float
    ufvc_status st = UFVC_OK;
#define AL(ptr, n)                                                                        \
    do {                                                                                  \
        const size_t n_ = (n);                                                            \
        if (dry_bytes) *dry_bytes += (n_ * sizeof(*(ptr)) + 255) & ~(size_t)255;          \
        else if ((st = dalloc(ctx, p, &(ptr), n_)) != UFVC_OK) return st;                 \
    } while (0)
    if (enc) {
        AL(p->x, ((size_t)p->Hp * p->Wp * p->C0p + act - 1) / act);
        AL(p->a1, ((size_t)p->h1 * p->w1 * a.e0 + act - 1) / act);
        AL(p->a2, ((size_t)p->h2 * p->w2 * a.e1 + act - 1) / act);
        AL(p->a3, ((size_t)p->h3 * p->w3 * a.e2 + act - 1) / act);
        AL(p->xt, ((size_t)p->h3 * p->w3 * a.e2 + act - 1) / act);
        AL(p->y, p->ny);
        if (fp32) {
            AL(p->hb, (size_t)p->hh * p->wh * a.cz);
        } else {
            AL(p->y_bf, (size_t)p->Hye * p->Wye * a.cy);
            AL(p->hb_bf, (size_t)p->hhe * p->whe * a.cz);
        }
        AL(p->z, p->nz);
        AL(p->zf, p->nz);
        AL(p->s1, (size_t)4 * p->Hz * p->Wz * a.cz);
        AL(p->s2, (size_t)p->Hy * p->Wy * a.cz);
        AL(p->mu, p->ny);
        AL(p->ls, p->ny);
        AL(p->zhat, p->nz);
        AL(p->rhat, p->ny);
        AL(p->iz, (size_t)a.cz);
        AL(p->idx, p->ny);
        AL(p->scr_z, (size_t)p->Kz * p->cap_z);
        AL(p->scr_y, (size_t)K * p->cap_y);
        AL(p->ctl, 1);
        if (!dry_bytes && cudaMemset(p->ctl, 0, sizeof(RansCtl)) != cudaSuccess) return UFVC_ERR_CUDA;
        AL(p->zthr, (size_t)kBins - 1);
        if (ctx->dcm) {
            const size_t P = (size_t)p->h3 * p->w3;
            AL(p->dc_x0, (P * 3 * N * 64 + act - 1) / act);
            AL(p->dc_h, (P * kDcC + act - 1) / act);
            AL(p->dc_t1e, (P * kDcC + act - 1) / act);
            AL(p->dc_t2e, (P * kDcC + act - 1) / act);
            AL(p->dc_t3e, (P * 2 * kDcC + act - 1) / act);
        }
    }
    if (dec) {
        AL(p->dzhat, p->nz);
        AL(p->didx, p->ny);
        AL(p->qp_dev, 1);
        AL(p->ver_dev, 1);
        AL(p->next_z, 1);
        AL(p->dzf, p->nz);
        AL(p->ds1, (size_t)4 * p->Hz * p->Wz * a.cz);
        AL(p->ds2, (size_t)p->Hy * p->Wy * a.cz);
        AL(p->dmu, p->ny);
        AL(p->dls, p->ny);
        if (fp32) AL(p->yhat, p->ny);
        else AL(p->yhat_bf, p->ny);
        AL(p->drhat, p->ny);
        const size_t n1 = (size_t)N * 4 * p->Hy * p->Wy * a.cd1;
        const size_t n2 = (size_t)N * 16 * p->Hy * p->Wy * a.cd2;
        const size_t n3 = (size_t)N * 64 * p->Hy * p->Wy * a.cd2;
        AL(p->bufA, (n1 + act - 1) / act);
        AL(p->bufT, (n1 + act - 1) / act);
        AL(p->bufB, (n2 + act - 1) / act);
        AL(p->bufT2, (n2 + act - 1) / act);
        AL(p->bufC, (n3 + act - 1) / act);
        if (ctx->dcm) {
            const size_t P = (size_t)p->h3 * p->w3;
            AL(p->dc_F, (P * kDcC + act - 1) / act);
            AL(p->dc_t1d, (P * kDcC + act - 1) / act);
            AL(p->dc_t2d, (P * kDcC + act - 1) / act);
            AL(p->dc_t3d, (P * 2 * kDcC + act - 1) / act);
            AL(p->dc_hf, (N * P * kDcCf + act - 1) / act);
            AL(p->dc_f1, (N * P * kDcCf + act - 1) / act);
            AL(p->dc_f2, (N * P * kDcCf + act - 1) / act);
            AL(p->dc_f3, (N * P * 2 * kDcCf + act - 1) / act);
            AL(p->dc_o, N * P * 192);
        }
    }
#undef AL
    return UFVC_OK;
}

// The progressive-means buffers of one direction of a plan (allocated, or counted into dry_bytes).
static ufvc_status pm_buffers(ufvc_ctx* ctx, Plan* p, bool enc, size_t* dry_bytes) {
    const Arch& a = ctx->arch;
    const size_t act = ctx->cfg.precision == UFVC_FP32 ? 1 : 2;
    const size_t npix = (size_t)p->Hy * p->Wy;
    ufvc_status st = UFVC_OK;
    float** bufs[3] = {enc ? &p->pm_in_e : &p->pm_in_d, enc ? &p->pm_h_e : &p->pm_h_d, enc ? &p->pm_mu_e : &p->pm_mu_d};
    const size_t n[3] = {(npix * (a.cy + a.cz) + act - 1) / act, (npix * a.cz + act - 1) / act, npix * a.cy};
    for (int i = 0; i < 3; ++i) {
        if (dry_bytes) *dry_bytes += (n[i] * sizeof(float) + 255) & ~(size_t)255;
        else if ((st = dalloc(ctx, p, bufs[i], n[i])) != UFVC_OK) return st;
    }
    return UFVC_OK;
}

// The temporal-context buffers of one direction of a plan (the zero context with the encoder half).
static ufvc_status tc_buffers(ufvc_ctx* ctx, Plan* p, bool enc, size_t* dry_bytes) {
    const size_t act = ctx->cfg.precision == UFVC_FP32 ? 1 : 2;
    const size_t n8 = (size_t)4 * p->Hy * p->Wy, ny = p->ny;
    ufvc_status st = UFVC_OK;
    struct { float** b; size_t n; } bufs[4] = {
        {enc ? &p->t_F_e : &p->t_F_d, (n8 * kCf + act - 1) / act},
        {enc ? &p->t_pc_e : &p->t_pc_d, (size_t)p->Hy * p->Wy * ctx->arch.cz},
        {enc ? &p->t_yh_e : nullptr, (ny + act - 1) / act},
        {enc ? &p->t_zero : nullptr, (n8 * ctx->cc + act - 1) / act}};
    for (auto& e : bufs) {
        if (!e.b) continue;
        if (dry_bytes) *dry_bytes += (e.n * sizeof(float) + 255) & ~(size_t)255;
        else if ((st = dalloc(ctx, p, e.b, e.n)) != UFVC_OK) return st;
    }
    return UFVC_OK;
}

// slot: a batched call's chunk position (every position of a batch has its own buffers)
static ufvc_status get_plan(ufvc_ctx* ctx, int W, int H, bool for_decode, Plan** out, int slot = 0) {
    const long long key = ((long long)slot << 40) | ((long long)W << 20) | H;
    Plan* p;
    auto it = ctx->plans.find(key);
    if (it == ctx->plans.end()) {
        p = new Plan();
        init_plan_shape(ctx, p, W, H);
        ctx->plans[key] = p;
    } else {
        p = it->second;
    }
    ufvc_status st = plan_buffers(ctx, p, !for_decode && !p->enc_ready, for_decode && !p->dec_ready, nullptr);
    if (st) return st;
    if (!for_decode && !p->enc_ready) {
        // z^ RMS thresholds for this shape: T_k = floor(npos * exp(2 t_k)), FP64 on the host
        std::vector<uint64_t> zt(kBins - 1);
        const double npos = (double)p->Hz * p->Wz;
        for (int k = 0; k < kBins - 1; ++k) zt[k] = (uint64_t)std::floor(npos * std::exp(2.0 * ctx->tabs.log_thr[k]));
        CK(cudaMemcpy(p->zthr, zt.data(), zt.size() * 8, cudaMemcpyHostToDevice));
        if (ctx->cfg.precision != UFVC_FP32) {
            CK(cudaMemset(p->y_bf, 0, (size_t)p->Hye * p->Wye * ctx->arch.cy * 2));
            CK(cudaMemset(p->hb_bf, 0, (size_t)p->hhe * p->whe * ctx->arch.cz * 2));
        }
        p->enc_ready = true;
    }
    if (for_decode && !p->dec_ready) p->dec_ready = true;
    if (for_decode && ctx->color != UFVC_COLOR_RGB && !p->fstage &&
        (st = dalloc(ctx, p, &p->fstage, (size_t)ctx->N * p->H * p->W * 3)) != UFVC_OK)
        return st;
    if (ctx->tc_on && !p->t_enc_ready) {  // the zero context lives with the encoder half: allocate it first
        if ((st = tc_buffers(ctx, p, true, nullptr)) != UFVC_OK) return st;
        CK(cudaMemset(p->t_zero, 0, (size_t)4 * p->Hy * p->Wy * ctx->cc * (ctx->cfg.precision == UFVC_FP32 ? 4 : 2)));
        p->t_enc_ready = true;
    }
    if (ctx->tc_on && for_decode && !p->t_dec_ready) {
        if ((st = tc_buffers(ctx, p, false, nullptr)) != UFVC_OK) return st;
        p->t_dec_ready = true;
    }
    if (ctx->pm_on && (for_decode ? !p->pm_dec_ready : !p->pm_enc_ready)) {
        if ((st = pm_buffers(ctx, p, !for_decode, nullptr)) != UFVC_OK) return st;
        (for_decode ? p->pm_dec_ready : p->pm_enc_ready) = true;
    }
    *out = p;
    return UFVC_OK;
}

// Device bytes one W x H plan of ctx takes once it has encoded and decoded: its buffers plus the
// split-K workspaces of the hyper-synthesis (one per direction).
size_t ufvc::ctx_plan_bytes(const ufvc_ctx* ctx, int W, int H) {
    Plan tmp;
    init_plan_shape(ctx, &tmp, W, H);
    size_t bytes = 0;
    plan_buffers(const_cast<ufvc_ctx*>(ctx), &tmp, true, true, &bytes);
    const Arch& a = ctx->arch;
    auto ws = [&](int h, int w, int k, int cout, int cin, const LayerW& L) {
        ConvDesc d;
        d.H = h; d.W = w; d.k = k; d.stride = 1; d.Cout = cout; d.Cin = ceil_div(cin, 16) * 16; d.groups = 1;
        d.wtf = L.wtf;  // the TF32 GEMM's planes and K-range sums where the layer has it
        return conv_simt_workspace(d) * sizeof(float);
    };
    size_t hs = std::max({ws(tmp.Hz, tmp.Wz, 3, 4 * a.cz, a.cz, ctx->enc[L_S1]),
                          ws(2 * tmp.Hz, 2 * tmp.Wz, 3, 4 * a.cz, a.cz, ctx->enc[L_S2]),
                          ws(tmp.Hy, tmp.Wy, 1, 2 * a.cy, a.cz, ctx->enc[L_S3])});
    if (ctx->color != UFVC_COLOR_RGB) bytes += ((size_t)ctx->N * H * W * 3 * sizeof(float) + 255) & ~(size_t)255;
    if (ctx->tc_on) {
        tc_buffers(const_cast<ufvc_ctx*>(ctx), &tmp, true, &bytes);
        tc_buffers(const_cast<ufvc_ctx*>(ctx), &tmp, false, &bytes);
    }
    if (ctx->pm_on) {
        pm_buffers(const_cast<ufvc_ctx*>(ctx), &tmp, true, &bytes);
        pm_buffers(const_cast<ufvc_ctx*>(ctx), &tmp, false, &bytes);
        if (ctx->cfg.precision == UFVC_FP32)
            hs = std::max({hs, ws(tmp.Hy, tmp.Wy, 3, a.cz, a.cy + a.cz, LayerW{}), ws(tmp.Hy, tmp.Wy, 1, a.cy, a.cz, LayerW{})});
    }
    return bytes + 2 * hs;
}

// ------------------------------------------------------------------------------------------------
// create / destroy
// ------------------------------------------------------------------------------------------------
extern "C" size_t ufvc_weight_count(int arch, int chunk_len) { return weight_count(arch, chunk_len); }

extern "C" ufvc_status ufvc_layer_shape(int arch, int chunk_len, int layer, int* cout, int* k, int* cin) {
    return layer_shape(arch, chunk_len, layer, cout, k, cin) ? UFVC_OK : UFVC_ERR_ARG;
}

extern "C" ufvc_status ufvc_latent_dims(int arch, int width, int height, int* Hy, int* Wy, int* Hz, int* Wz, int* Cy,
                                        int* Cz) {
    Arch a;
    if (!get_arch(arch, &a) || width < 1 || height < 1) return UFVC_ERR_ARG;
    const int hy = ceil_div(height, 16), wy = ceil_div(width, 16);
    if (Hy) *Hy = hy;
    if (Wy) *Wy = wy;
    if (Hz) *Hz = ceil_div(hy, 4);
    if (Wz) *Wz = ceil_div(wy, 4);
    if (Cy) *Cy = a.cy;
    if (Cz) *Cz = a.cz;
    return UFVC_OK;
}

// shape (cout, k, cin), when given, replaces the codec blob's layer table (the progressive-mean blob);
// no_fp8 keeps an FP8 context's layer on bf16 operands
static ufvc_status upload_layer(ufvc_ctx* ctx, LayerW& L, const float* blob, const size_t* offs, int first, int groups,
                                bool tc, bool pixel_shuffle = false, bool final_layer = false,
                                const int* shape = nullptr, bool no_fp8 = false, int gstride = D_NDEC,
                                float tc_scale = 1.0f) {
    int co, k, ci;
    if (shape) { co = shape[0]; k = shape[1]; ci = shape[2]; }
    else layer_shape(ctx->cfg.arch, ctx->N, first, &co, &k, &ci);
    L.cout = co; L.k = k; L.cin = ci; L.cin_p = ceil_div(ci, 16) * 16; L.groups = groups;
    L.w_gs = (long long)k * k * L.cin_p * co;
    L.b_gs = co;
    std::vector<float> w((size_t)groups * L.w_gs, 0.f), b((size_t)groups * co);
    for (int g = 0; g < groups; ++g) {
        const int l = first + g * gstride;
        const float* src = blob + offs[l];
        for (int o = 0; o < co; ++o)
            for (int t = 0; t < k * k; ++t)
                for (int i = 0; i < ci; ++i)
                    w[g * L.w_gs + ((size_t)t * L.cin_p + i) * co + o] = src[((size_t)o * k * k + t) * ci + i];
        for (int o = 0; o < co; ++o) b[(size_t)g * co + o] = src[(size_t)co * k * k * ci + o];
    }
    ufvc_status st;
    if ((st = dalloc(ctx, nullptr, &L.w, w.size())) != UFVC_OK) return st;
    if ((st = dalloc(ctx, nullptr, &L.b, b.size())) != UFVC_OK) return st;
    CK(cudaMemcpy(L.w, w.data(), w.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L.b, b.data(), b.size() * 4, cudaMemcpyHostToDevice));
    if (tc && ctx->cfg.precision != UFVC_FP32) {
        // K-major bf16 copy for tcgen05: [g][cout_pad][tap][cin_tc], zero rows / columns in the padding
        // 64-channel stages; in BF16 a layer with at most 32 input channels (the first) uses 32-channel ones
        L.cin_tc = (ci <= 32 && ctx->cfg.precision == UFVC_BF16) ? 32 : ceil_div(ci, 64) * 64;
        L.cout_pad = co >= 64 ? co : 16;
        L.ps_major = pixel_shuffle && co % 128 == 0;  // runs of 32 channels per sub-pixel in every N tile
        const int cq = co / 4;
        auto row = [&](int o) { return L.ps_major ? (o & 3) * cq + (o >> 2) : o; };
        const size_t K = (size_t)k * k * L.cin_tc;
        std::vector<__nv_bfloat16> wt((size_t)groups * L.cout_pad * K, __float2bfloat16(0.f));
        std::vector<float> bt(b.size());
        for (int g = 0; g < groups; ++g) {
            const float* src = blob + offs[first + g * gstride];
            for (int o = 0; o < co; ++o) {
                for (int t = 0; t < k * k; ++t)
                    for (int i = 0; i < ci; ++i)
                        wt[((size_t)g * L.cout_pad + row(o)) * K + (size_t)t * L.cin_tc + i] =
                            __float2bfloat16(tc_scale * src[((size_t)o * k * k + t) * ci + i]);
                bt[(size_t)g * co + row(o)] = b[(size_t)g * co + o];
            }
        }
        if ((st = dalloc(ctx, nullptr, &L.wtc, wt.size())) != UFVC_OK) return st;
        CK(cudaMemcpy(L.wtc, wt.data(), wt.size() * 2, cudaMemcpyHostToDevice));
        if (L.ps_major) {
            if ((st = dalloc(ctx, nullptr, &L.btc, bt.size())) != UFVC_OK) return st;
            CK(cudaMemcpy(L.btc, bt.data(), bt.size() * 4, cudaMemcpyHostToDevice));
        }
        if (ctx->cfg.precision == UFVC_FP8 && !final_layer && !no_fp8) {
            // E4M3 copy with one scale per output channel (per group): code = e4m3(w / s), s = absmax / 448
            std::vector<uint8_t> w8((size_t)groups * L.cout_pad * K, 0);
            L.wscale.assign((size_t)groups * co, 1.f);
            for (int g = 0; g < groups; ++g) {
                const float* src = blob + offs[first + g * gstride];
                for (int o = 0; o < co; ++o) {
                    float amax = 0.f;
                    for (size_t e = 0; e < (size_t)k * k * ci; ++e) amax = std::max(amax, std::fabs(src[(size_t)o * k * k * ci + e]));
                    const float sc = amax > 0.f ? amax / 448.f : 1.f;
                    L.wscale[(size_t)g * co + row(o)] = sc;
                    for (int t = 0; t < k * k; ++t)
                        for (int i = 0; i < ci; ++i)
                            w8[((size_t)g * L.cout_pad + row(o)) * K + (size_t)t * L.cin_tc + i] = (uint8_t)
                                __nv_cvt_float_to_fp8(src[((size_t)o * k * k + t) * ci + i] / sc, __NV_SATFINITE, __NV_E4M3);
                }
            }
            if ((st = dalloc(ctx, nullptr, &L.w8, w8.size())) != UFVC_OK) return st;
            CK(cudaMemcpy(L.w8, w8.data(), w8.size(), cudaMemcpyHostToDevice));
            if ((st = dalloc(ctx, nullptr, &L.cs8, L.wscale.size())) != UFVC_OK) return st;
        }
        if (final_layer && co == 12 && k == 3 && ci == 64) {
            std::vector<__nv_bfloat16> ws((size_t)groups * 128 * 64, __float2bfloat16(0.f));
            for (int g = 0; g < groups; ++g) {
                const float* src = blob + offs[first + g * gstride];
                for (int c = 0; c < 12; ++c)
                    for (int t = 0; t < 9; ++t)
                        for (int i = 0; i < 64; ++i)
                            ws[((size_t)g * 128 + 32 * (c / 3) + 3 * t + c % 3) * 64 + i] =
                                __float2bfloat16(src[((size_t)c * 9 + t) * 64 + i]);
            }
            if ((st = dalloc(ctx, nullptr, &L.wsc, ws.size())) != UFVC_OK) return st;
            CK(cudaMemcpy(L.wsc, ws.data(), ws.size() * 2, cudaMemcpyHostToDevice));
        }
    }
    return UFVC_OK;
}

// A depth-wise 3x3 layer (blob kernel [C][3][3][1] + bias [C], per group) as float [g][9][C] taps and [g][C]
// biases for the depth-wise kernel (every precision).
static ufvc_status upload_dw(ufvc_ctx* ctx, LayerW& L, const float* blob, const size_t* offs, int first, int groups,
                             int gstride, int C) {
    L.cout = C; L.k = 3; L.cin = 1; L.groups = groups;
    std::vector<float> w((size_t)groups * 9 * C), b((size_t)groups * C);
    for (int g = 0; g < groups; ++g) {
        const float* src = blob + offs[first + g * gstride];
        for (int c = 0; c < C; ++c) {
            for (int t = 0; t < 9; ++t) w[((size_t)g * 9 + t) * C + c] = src[(size_t)c * 9 + t];
            b[(size_t)g * C + c] = src[(size_t)C * 9 + c];
        }
    }
    ufvc_status st;
    if ((st = dalloc(ctx, nullptr, &L.w, w.size())) != UFVC_OK) return st;
    if ((st = dalloc(ctx, nullptr, &L.b, b.size())) != UFVC_OK) return st;
    CK(cudaMemcpy(L.w, w.data(), w.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L.b, b.data(), b.size() * 4, cudaMemcpyHostToDevice));
    return UFVC_OK;
}

// The DC-block model's layers: shared ones into ctx->dcl (and the hyperprior into ctx->enc[L_H1..L_S3], the
// prior's context layer into ctx->tl[TL_PC], so that the hyperprior code serves both models), frame ones
// grouped into ctx->dcf.
static ufvc_status upload_dc(ufvc_ctx* ctx, const float* weights) {
    const int N = ctx->N, nl = kDcShared + kDcPerFrame * N;
    std::vector<size_t> offs(nl);
    size_t off = 0;
    for (int l = 0; l < nl; ++l) {
        int co, k, ci;
        dc_layer_shape(N, l, &co, &k, &ci);
        offs[l] = off;
        off += (size_t)co * k * k * ci + co;
    }
    ufvc_status st;
    ctx->dcl.assign(kDcShared, LayerW());
    for (int l = 0; l < kDcShared; ++l) {
        int sh[3];
        dc_layer_shape(N, l, &sh[0], &sh[1], &sh[2]);
        if (sh[2] == 1) {
            st = upload_dw(ctx, ctx->dcl[l], weights, offs.data(), l, 1, 1, sh[0]);
        } else if (l >= DC_H1 && l <= DC_S3) {  // S1..S3: the deterministic FP32 path, as in the plain model
            st = upload_layer(ctx, ctx->enc[L_H1 + (l - DC_H1)], weights, offs.data(), l, 1, l <= DC_H2, false, false,
                              sh, true, 1);
        } else if (l == DC_PC) {
            st = upload_layer(ctx, ctx->tl[TL_PC], weights, offs.data(), l, 1, true, false, false, sh, true, 1);
        } else {  // the patch embedding's bf16 input carries kS2dInScale
            st = upload_layer(ctx, ctx->dcl[l], weights, offs.data(), l, 1, true, l == DC_DU, false, sh, true, 1,
                              l == DC_PE ? 1.0f / kS2dInScale : 1.0f);
        }
        if (st != UFVC_OK) return st;
    }
    for (int j = 0; j < kDcPerFrame; ++j) {
        int sh[3];
        dc_layer_shape(N, kDcShared + j, &sh[0], &sh[1], &sh[2]);
        st = sh[2] == 1 ? upload_dw(ctx, ctx->dcf[j], weights, offs.data(), kDcShared + j, N, kDcPerFrame, sh[0])
                        : upload_layer(ctx, ctx->dcf[j], weights, offs.data(), kDcShared + j, N, true, false, false, sh,
                                       true, kDcPerFrame);
        if (st != UFVC_OK) return st;
    }
    ctx->dcm = true;
    ctx->tc_on = true;
    ctx->cc = kDcCc;
    return UFVC_OK;
}

// The TF32 parts of a float: hi(x) = x rounded to the nearest TF32 value (the 13 low fraction bits rounded
// away, halves away from zero), lo(x) = hi(x - hi(x)).
static float tf32_hi(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    std::memcpy(&x, &u, 4);
    return x;
}

// A hyper-synthesis layer's weights for the three-product TF32 GEMM: K index (tap, part, c) holds
// (hi, lo, hi)[part] of w[o][tap][c], against the input planes (hi, hi, lo) (conv_tf32.cu).  Layers the GEMM
// does not take (Cin not a multiple of 32, Cout not a multiple of 256) keep only the SIMT weights.
static ufvc_status upload_tf32(ufvc_ctx* ctx, LayerW& L, const float* src) {
    const int co = L.cout, kk = L.k * L.k, ci = L.cin;
    if (ci % 32 != 0 || ci != L.cin_p || co % 256 != 0 || L.groups != 1) return UFVC_OK;
    std::vector<float> w((size_t)co * kk * 3 * ci);
    for (int o = 0; o < co; ++o)
        for (int t = 0; t < kk; ++t)
            for (int c = 0; c < ci; ++c) {
                const float v = src[((size_t)o * kk + t) * ci + c];
                const float hi = tf32_hi(v), lo = tf32_hi(v - hi);
                float* row = &w[((size_t)o * kk + t) * 3 * ci];
                row[c] = hi;
                row[ci + c] = lo;
                row[2 * ci + c] = hi;
            }
    ufvc_status st;
    if ((st = dalloc(ctx, nullptr, &L.wtf, w.size())) != UFVC_OK) return st;
    CK(cudaMemcpy(L.wtf, w.data(), w.size() * 4, cudaMemcpyHostToDevice));
    return UFVC_OK;
}

// A1 (3x3, stride 2, 3N -> e0) regrouped for space-to-depth input: super-pixel (Y, X) holds input pixels
// (2Y + dy, 2X + dx) as channels [2 dy + dx][32].  Output pixel (oh, ow) reads input rows 2 oh - 1 .. 2 oh + 1,
// i.e. sub-row 1 of super-row oh - 1 and both sub-rows of super-row oh: tap (sy, sx) of the 2x2 form at
// super offsets (sy - 1, sx - 1) carries original tap (ky, kx) = (2 sy + dy - 1, 2 sx + dx - 1) where that
// lies in 0..2, zero elsewhere.  K steps (tap, 64-channel chunk = sub-row dy): taps (0, 0) and (0, 1) have
// no dy = 0 weights, so steps 0 and 2 are skipped.
static ufvc_status upload_a1_s2d(ufvc_ctx* ctx, const float* src) {
    const LayerW& A1 = ctx->enc[L_A1];
    const int co = A1.cout, ci = A1.cin;  // ci = 3N <= 32
    LayerW& L = ctx->a1s2d;
    L.cout = co; L.k = 2; L.cin = 128; L.cin_p = 128; L.groups = 1;
    L.b = A1.b; L.b_gs = A1.b_gs;
    L.cin_tc = 128; L.cout_pad = co;
    L.kmask = 0xFAull;
    const size_t K = 4 * 128;
    std::vector<__nv_bfloat16> wt((size_t)co * K, __float2bfloat16(0.f));
    for (int o = 0; o < co; ++o)
        for (int sy = 0; sy < 2; ++sy)
            for (int sx = 0; sx < 2; ++sx)
                for (int dy = 0; dy < 2; ++dy)
                    for (int dx = 0; dx < 2; ++dx) {
                        const int ky = 2 * sy + dy - 1, kx = 2 * sx + dx - 1;
                        if (ky < 0 || kx < 0) continue;
                        for (int c = 0; c < ci; ++c)  // the input carries kS2dInScale
                            wt[(size_t)o * K + (sy * 2 + sx) * 128 + (dy * 2 + dx) * 32 + c] =
                                __float2bfloat16(src[((size_t)o * 9 + ky * 3 + kx) * ci + c] / kS2dInScale);
                    }
    ufvc_status st;
    if ((st = dalloc(ctx, nullptr, &L.wtc, wt.size())) != UFVC_OK) return st;
    CK(cudaMemcpy(L.wtc, wt.data(), wt.size() * 2, cudaMemcpyHostToDevice));
    return UFVC_OK;
}

extern "C" void ufvc_destroy(ufvc_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->cfg.device);
    if (!ctx->borrowed) cudaDeviceSynchronize();  // a clone's owner has synchronised its stream
    for (auto& kv : ctx->plans) free_plan(kv.second);
    if (!ctx->borrowed) {
        for (auto* Ls : {&ctx->enc[0], &ctx->dec[0]}) {
            const int nl = Ls == &ctx->enc[0] ? L_NENC : D_NDEC;
            for (int l = 0; l < nl; ++l) {
                LayerW& L = Ls[l];
                cudaFree(L.w); cudaFree(L.b); cudaFree(L.wtc); cudaFree(L.btc); cudaFree(L.wsc);
                cudaFree(L.w8); cudaFree(L.cs8); cudaFree(L.wtf);
            }
        }
        for (LayerW& L : ctx->pm) { cudaFree(L.w); cudaFree(L.b); cudaFree(L.wtc); }
        for (LayerW* L : {&ctx->tl[0], &ctx->tl[1], &ctx->tl[2], &ctx->tl[3], &ctx->tl[4], &ctx->tdf}) {
            cudaFree(L->w); cudaFree(L->b); cudaFree(L->wtc); cudaFree(L->btc);
        }
        for (LayerW& L : ctx->dcl) { cudaFree(L.w); cudaFree(L.b); cudaFree(L.wtc); cudaFree(L.btc); }
        for (LayerW& L : ctx->dcf) { cudaFree(L.w); cudaFree(L.b); cudaFree(L.wtc); cudaFree(L.btc); }
        cudaFree(ctx->a1s2d.wtc);  // (its bias is enc[L_A1]'s)
        cudaFree(ctx->first_w);
        cudaFree(ctx->d_packed); cudaFree(ctx->d_dec); cudaFree(ctx->d_thr); cudaFree(ctx->d_qstep);
        cudaFree(ctx->d_qinv);
    }
    cudaFree(ctx->d_status);
    cudaFree(ctx->r_scr); cudaFree(ctx->r_ctl);
    cudaFree(ctx->st_frames); cudaFree(ctx->st_bits); cudaFree(ctx->st_nbytes);
    cudaFree(ctx->ws_stage.p);
    for (auto& e : ctx->prof) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
    delete ctx;
}

extern "C" ufvc_status ufvc_create(const ufvc_config* cfg, const float* weights, size_t n_weights, ufvc_ctx** out) {
    if (!cfg || !weights || !out) return UFVC_ERR_ARG;
    Arch a;
    if (!get_arch(cfg->arch, &a) || cfg->chunk_len < 1 || cfg->chunk_len > 16 || cfg->lanes < 1 ||
        cfg->lanes > 65536 || cfg->precision < 0 || cfg->precision > 2)
        return UFVC_ERR_ARG;
    if (n_weights != weight_count(cfg->arch, cfg->chunk_len)) return UFVC_ERR_ARG;
    // the tensor-core path stages K in 64-channel chunks: every activation width must be a multiple of
    // 64, which holds for the 1080p-family widths only (the tiny widths include 96)
    if (cfg->precision != UFVC_FP32 && cfg->arch == 0) return UFVC_ERR_UNSUPPORTED;
    if (cfg->precision == UFVC_FP8 && cfg->arch == 2) return UFVC_ERR_UNSUPPORTED;
    ufvc_ctx* ctx = new ufvc_ctx();
    ctx->cfg = *cfg;
    ctx->arch = a;
    ctx->N = cfg->chunk_len;
    auto bail = [&](ufvc_status s) { ufvc_destroy(ctx); return s; };
    if (cudaSetDevice(cfg->device) != cudaSuccess) return bail(UFVC_ERR_CUDA);
    build_host_tables(ctx->tabs);
    ufvc_status st;
    if ((st = dalloc(ctx, nullptr, &ctx->d_packed, ctx->tabs.packed.size())) != UFVC_OK) return bail(st);
    if ((st = dalloc(ctx, nullptr, &ctx->d_dec, ctx->tabs.dec.size())) != UFVC_OK) return bail(st);
    if (cudaMemcpy(ctx->d_dec, ctx->tabs.dec.data(), ctx->tabs.dec.size(), cudaMemcpyHostToDevice))
        return bail(UFVC_ERR_CUDA);
    if ((st = dalloc(ctx, nullptr, &ctx->d_thr, ctx->tabs.thr.size())) != UFVC_OK) return bail(st);
    if ((st = dalloc(ctx, nullptr, &ctx->d_qstep, 64)) != UFVC_OK) return bail(st);
    if ((st = dalloc(ctx, nullptr, &ctx->d_qinv, 64)) != UFVC_OK) return bail(st);
    if ((st = dalloc(ctx, nullptr, &ctx->d_status, 1)) != UFVC_OK) return bail(st);
    if (cudaMemcpy(ctx->d_packed, ctx->tabs.packed.data(), ctx->tabs.packed.size() * 4, cudaMemcpyHostToDevice) ||
        cudaMemcpy(ctx->d_thr, ctx->tabs.thr.data(), ctx->tabs.thr.size() * 4, cudaMemcpyHostToDevice) ||
        cudaMemcpy(ctx->d_qstep, ctx->tabs.qstep.data(), 64 * 4, cudaMemcpyHostToDevice) ||
        cudaMemcpy(ctx->d_qinv, ctx->tabs.qinv.data(), 64 * 4, cudaMemcpyHostToDevice) ||
        cudaMemset(ctx->d_status, 0, 4))
        return bail(UFVC_ERR_CUDA);
    if (cfg->arch == 2) {
        if ((st = upload_dc(ctx, weights)) != UFVC_OK) return bail(st);
        *out = ctx;
        return UFVC_OK;
    }
    // weight blob offsets
    const int nl = L_NENC + D_NDEC * ctx->N;
    std::vector<size_t> offs(nl);
    size_t off = 0;
    for (int l = 0; l < nl; ++l) {
        int co, k, ci;
        layer_shape(cfg->arch, ctx->N, l, &co, &k, &ci);
        offs[l] = off;
        off += (size_t)co * k * k * ci + co;
    }
    for (int l = 0; l < L_NENC; ++l)
        if ((st = upload_layer(ctx, ctx->enc[l], weights, offs.data(), l, 1, l <= L_H2)) != UFVC_OK) return bail(st);
    for (int j = 0; j < D_NDEC; ++j)
        if ((st = upload_layer(ctx, ctx->dec[j], weights, offs.data(), L_NENC + j, ctx->N, true,
                                   j == D_D0 || j == D_U1 || j == D_U2, j == D_U3)) != UFVC_OK)
            return bail(st);
    if (cfg->precision == UFVC_BF16 && 3 * ctx->N <= 32 && (st = upload_a1_s2d(ctx, weights + offs[L_A1])) != UFVC_OK)
        return bail(st);
    if (cfg->arch == 1)  // the hyper-synthesis on the tensor cores (TF32, three products), every precision
        for (int l : {L_S1, L_S2, L_S3})
            if ((st = upload_tf32(ctx, ctx->enc[l], weights + offs[l])) != UFVC_OK) return bail(st);
    if ((cfg->precision == UFVC_BF16 || cfg->precision == UFVC_FP8) && first_layer_ct(ctx->N) &&
        ctx->enc[L_A1].cout == 64 && ctx->enc[L_A1].k == 3) {
        // the frame-byte kernel's input is x * kS2dInScale, like the space-to-depth pack's
        const int pitch = first_layer_pitch(ctx->N);
        std::vector<uint16_t> img(first_layer_weight_bytes(pitch) / 2);
        first_layer_weights(weights + offs[L_A1], ctx->N, 1.0f / kS2dInScale, pitch, img.data());
        uint16_t* dimg = nullptr;
        if ((st = dalloc(ctx, nullptr, &dimg, img.size())) != UFVC_OK) return bail(st);
        ctx->first_w = dimg;
        if (cudaMemcpy(dimg, img.data(), img.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(UFVC_ERR_CUDA);
    }
    *out = ctx;
    return UFVC_OK;
}

// A context that shares base's weights and tables (read-only on the device) but has its own plans,
// workspaces, staging and status word, so that it can run concurrently with base on another stream.
// base must outlive it.
int ufvc::ctx_color(const ufvc_ctx* ctx) { return ctx->color; }

ufvc_ctx* ufvc::ctx_clone_shared(const ufvc_ctx* base) {
    if (!base || base->borrowed) return nullptr;
    if (cudaSetDevice(base->cfg.device) != cudaSuccess) return nullptr;
    auto* c = new ufvc_ctx();
    c->cfg = base->cfg;
    c->arch = base->arch;
    c->N = base->N;
    c->tabs = base->tabs;
    c->d_packed = base->d_packed;
    c->d_dec = base->d_dec;
    c->table_spin = base->table_spin;
    c->conv_pairs = base->conv_pairs;
    c->fp8_ready = base->fp8_ready;  // the calibration as it stands (the layers' scales are shared)
    for (int t = 0; t < T_NT; ++t) c->act_scale[t] = base->act_scale[t];
    c->d_thr = base->d_thr;
    c->d_qstep = base->d_qstep;
    c->d_qinv = base->d_qinv;
    for (int l = 0; l < L_NENC; ++l) c->enc[l] = base->enc[l];
    for (int l = 0; l < D_NDEC; ++l) c->dec[l] = base->dec[l];
    c->a1s2d = base->a1s2d;
    c->first_w = base->first_w;
    for (int l = 0; l < kMeanLayers; ++l) c->pm[l] = base->pm[l];
    c->pm_on = base->pm_on;
    c->color = base->color;
    for (int l = 0; l < TL_N; ++l) c->tl[l] = base->tl[l];
    c->tdf = base->tdf;
    c->tc_on = base->tc_on;
    c->cc = base->cc;
    c->dcm = base->dcm;
    c->dcl = base->dcl;
    for (int j = 0; j < kDcPerFrame; ++j) c->dcf[j] = base->dcf[j];
    c->borrowed = true;
    if (cudaMalloc(&c->d_status, 4) != cudaSuccess || cudaMemset(c->d_status, 0, 4) != cudaSuccess) {
        cudaFree(c->d_status);
        delete c;
        return nullptr;
    }
    return c;
}

extern "C" const char* ufvc_last_error(const ufvc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

static bool use_tc(const ufvc_ctx* ctx, const LayerW& L) { return ctx->cfg.precision != UFVC_FP32 && L.wtc; }

static ufvc_status conv(ufvc_ctx* ctx, const LayerW& L, const void* in, int H, int W, int stride, int act, int mode,
                        void* out, int out_h, int out_w, cudaStream_t s, const void* res, float* out2, int split,
                        long long in_gs, long long out_gs, long long res_gs, int groups, bool out_f32,
                        const EntParams* ent) {
    ConvDesc d;
    if (ent) {
        d.ent_idx = ent->idx; d.ent_y = ent->y; d.ent_rhat = ent->rhat; d.ent_qp_dev = ent->qp_dev;
        d.ent_qp = ent->qp; d.ent_keep_ls = ent->keep_ls ? 1 : 0; d.ent_thr = ctx->d_thr; d.ent_qinv = ctx->d_qinv;
    }
    d.in = in; d.in_gs = in_gs; d.H = H; d.W = W;
    d.w = L.w; d.w_gs = L.w_gs; d.b = L.b; d.b_gs = L.b_gs;
    d.Cout = L.cout; d.k = L.k; d.stride = stride; d.mode = mode; d.act = act;
    d.out = out; d.out_gs = out_gs; d.out_h = out_h; d.out_w = out_w;
    d.res = res; d.res_gs = res_gs; d.out2 = out2; d.split = split; d.groups = groups;
    if (use_tc(ctx, L)) {
        d.Cin = L.cin_tc; d.wtc = L.wtc; d.cout_pad = L.cout_pad; d.out_f32 = out_f32; d.err = ctx->d_status;
        d.btc = L.btc; d.ps_major = L.ps_major; d.wsc = L.wsc; d.kmask = L.kmask; d.pairs = ctx->conv_pairs;
        if (ctx->cfg.precision == UFVC_FP8 && L.w8) {
            d.w8 = L.w8; d.cscale = L.cs8; d.out_inv = L.out_inv; d.res_s = L.res_s;
        }
        const size_t tneed = conv_tc_workspace(d);  // split-K range sums (layers with few tiles)
        if (tneed) {
            Workspace* ws = ctx->cur_ws;
            if (tneed > ws->cap) {  // first use of this shape: grow (cudaFree waits for the old buffer's users)
                cudaFree(ws->p);
                ws->p = nullptr;
                ws->cap = 0;
                CK(cudaMalloc(&ws->p, tneed * sizeof(float)));
                ws->cap = tneed;
            }
            d.tc_ws = ws->p;
            d.tc_ws_cap = ws->cap;
        }
        int extra = 0;
        const cudaError_t e = launch_conv_tc(d, s, &extra);
        if (e != cudaSuccess) {
            ctx->err = std::string("tensor-core conv launch: ") + cudaGetErrorString(e);
            return UFVC_ERR_CUDA;
        }
        ctx->conv_launches += 1 + extra;
        return UFVC_OK;
    }
    d.Cin = L.cin_p;
    d.wtf = L.wtf;
    const size_t need = conv_simt_workspace(d);
    if (need) {
        Workspace* ws = ctx->cur_ws;
        if (need > ws->cap) {  // first use of this shape: grow (cudaFree waits for the old buffer's users)
            cudaFree(ws->p);
            ws->p = nullptr;
            ws->cap = 0;
            CK(cudaMalloc(&ws->p, need * sizeof(float)));
            ws->cap = need;
        }
        d.ws = ws->p;
        d.ws_cap = ws->cap;
    }
    CK(launch_conv_simt(d, s, &ctx->conv_launches));
    return UFVC_OK;
}

#define RUN(x)                          \
    do {                                \
        ufvc_status st_ = (x);          \
        if (st_ != UFVC_OK) return st_; \
    } while (0)

extern "C" size_t ufvc_max_bitstream_bytes(const ufvc_ctx* ctx, int width, int height) {
    if (!ctx || width < 1 || height < 1) return 0;
    const int hy = ceil_div(height, 16), wy = ceil_div(width, 16);
    const size_t ny = (size_t)hy * wy * ctx->arch.cy;
    const size_t nz = (size_t)ceil_div(hy, 4) * ceil_div(wy, 4) * ctx->arch.cz;
    const size_t K = ctx->cfg.lanes, Kz = K < nz ? K : nz;
    const size_t hdr = (20 + (size_t)ctx->arch.cz + 3) & ~(size_t)3;
    return hdr + (4 * Kz + 2 * (nz + 2 * Kz) + 3) + (4 * K + 2 * (ny + 2 * K) + 3);
}

extern "C" ufvc_status ufvc_sync_status(ufvc_ctx* ctx, void* stream) {
    if (!ctx) return UFVC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaStreamSynchronize(s));
    int v = 0;
    CK(cudaMemcpy(&v, ctx->d_status, 4, cudaMemcpyDeviceToHost));
    CK(cudaMemset(ctx->d_status, 0, 4));
    if (v != 0) ctx->err = "device status " + std::to_string(v);
    return (ufvc_status)v;
}

// ------------------------------------------------------------------------------------------------
// pipeline stages
// ------------------------------------------------------------------------------------------------
// An FP8 context computes with calibrated activation scales (ufvc_calibrate_fp8)
static bool fp8_unready(ufvc_ctx* ctx) { return ctx->cfg.precision == UFVC_FP8 && !ctx->fp8_ready; }

static bool check_shape(ufvc_ctx* ctx, int n_frames, int width, int height) {
    return n_frames == ctx->N && width >= 1 && height >= 1 && width <= 65535 && height <= 65535;
}

// hyper-synthesis: zhat (int16) -> mu, logsig; deterministic FP32 path in every precision
// cin (temporal context C_i, [2Hy][2Wy][Cc]) and pc_tmp ([Hy][Wy][Cz] float): the prior's features get
// PC(C_i) added before S3 (both null without the temporal context)
static ufvc_status run_hyper_synthesis(ufvc_ctx* ctx, Plan* p, const int16_t* zhat, float* zf, float* s1, float* s2,
                                       float* mu, float* ls, cudaStream_t s, const void* cin = nullptr,
                                       float* pc_tmp = nullptr, const EntParams* ent = nullptr) {
    const Arch& a = ctx->arch;
    prof_begin(ctx, "hyper_synthesis", s);
    const int nl0 = ctx->conv_launches;
    launch_i16_to_f32(zhat, p->nz, zf, s);
    RUN(conv(ctx, ctx->enc[L_S1], zf, p->Hz, p->Wz, 1, 1, OUT_PS, s1, 2 * p->Hz, 2 * p->Wz, s));
    RUN(conv(ctx, ctx->enc[L_S2], s1, 2 * p->Hz, 2 * p->Wz, 1, 1, OUT_PS, s2, p->Hy, p->Wy, s));  // crop
    if (cin) {
        RUN(conv(ctx, ctx->tl[TL_PC], cin, 2 * p->Hy, 2 * p->Wy, 2, 0, OUT_NHWC, pc_tmp, p->Hy, p->Wy, s, nullptr,
                 nullptr, 0, 0, 0, 0, 1, true));
        launch_add_f32(s2, pc_tmp, (size_t)p->Hy * p->Wy * a.cz, s);
    }
    RUN(conv(ctx, ctx->enc[L_S3], s2, p->Hy, p->Wy, 1, 0, OUT_NHWC, mu, p->Hy, p->Wy, s, nullptr, ls, a.cy, 0, 0, 0, 1,
             false, ent));
    // the conversion (+ the context addition) and every kernel of the layers, split-K reductions included
    prof_end(ctx, s, 1 + (cin ? 1 : 0) + (ctx->conv_launches - nl0));
    return UFVC_OK;
}

// The chunk feature F_i = GELU(PS(FD(y^))) + FC(C_i) and, with cout, the next context C_{i+1} = GELU(CG(F_i))
// (temporal context; y^ and the contexts in the activation type).
static ufvc_status run_chunk_feature(ufvc_ctx* ctx, Plan* p, const void* yhat, const void* cin, float* F, void* cout,
                                     cudaStream_t s) {
    const int H8 = 2 * p->Hy, W8 = 2 * p->Wy;
    prof_begin(ctx, "chunk_context", s);
    RUN(conv(ctx, ctx->tl[TL_FD], yhat, p->Hy, p->Wy, 1, 1, OUT_PS, F, H8, W8, s));
    RUN(conv(ctx, ctx->tl[TL_FC], cin, H8, W8, 1, 0, OUT_NHWC, F, H8, W8, s, F));
    if (cout) RUN(conv(ctx, ctx->tl[TL_CG], F, H8, W8, 1, 1, OUT_NHWC, cout, H8, W8, s));
    prof_end(ctx, s, cout ? 3 : 2);
    return UFVC_OK;
}

// Progressive means (Sec. 3.4, Fig. 4c): after the single parameter pass, the means of partitions 1, 2, 3,
// each from the partitions before it and the hyper-synthesis features s (see progressive.cu).  Encoder
// (y != null): quantises partition 0 with mu^0 and partition k with mu^k, writing r^; decoder: r^ is the
// decoded one.  Both leave in mu the mean every element is coded with (y^ = r^ q + mu).  The mean
// network runs on the tensor cores (bf16 operands, also in FP8 contexts) or, in FP32 precision, on
// the SIMT kernel.  in / h / muk: the plan's buffers of this direction.
static ufvc_status run_progressive(ufvc_ctx* ctx, int Hy, int Wy, const float* y, int16_t* rhat, float* mu,
                                   const float* sfeat, const int* qp_dev, int qp_host, const int* ver_dev, float* in,
                                   float* h, float* muk, cudaStream_t s) {
    const Arch& a = ctx->arch;
    const bool f32 = ctx->cfg.precision == UFVC_FP32;
    prof_begin(ctx, "progressive_means", s);
    launch_pm_init(y, rhat, mu, sfeat, Hy, Wy, a.cy, a.cz, ctx->d_qstep, ctx->d_qinv, qp_dev, qp_host, in, f32, s);
    for (int k = 1; k <= 3; ++k) {
        RUN(conv(ctx, ctx->pm[2 * k - 2], in, Hy, Wy, 1, 1, OUT_NHWC, h, Hy, Wy, s));
        RUN(conv(ctx, ctx->pm[2 * k - 1], h, Hy, Wy, 1, 0, OUT_NHWC, muk, Hy, Wy, s, nullptr, nullptr, 0, 0, 0, 0, 1,
                 true));
        launch_pm_step(k, y, rhat, mu, muk, Hy, Wy, a.cy, a.cz, ctx->d_qstep, ctx->d_qinv, qp_dev, qp_host, ver_dev,
                       in, f32, s);
    }
    prof_end(ctx, s, 10);
    return UFVC_OK;
}

// One DC block (PWa, DW, PWb, PWc, PWd) on x in place: y = x + PWb(GELU(DW(PWa(x)))), x = y + PWd(GELU(PWc(y))).
// groups > 1: one block per frame position (own weights), x / t1 / t2 with gs elements per group, t3 gs3.
static ufvc_status run_dc_block(ufvc_ctx* ctx, const LayerW* L, void* x, int H, int W, int groups, long long gs,
                                long long gs3, void* t1, void* t2, void* t3, cudaStream_t s) {
    const bool f32 = ctx->cfg.precision == UFVC_FP32;
    const long long ig = groups > 1 ? gs : 0, ig3 = groups > 1 ? gs3 : 0;
    RUN(conv(ctx, L[0], x, H, W, 1, 0, OUT_NHWC, t1, H, W, s, nullptr, nullptr, 0, ig, ig, 0, groups));
    launch_dw_conv(t1, groups, H, W, L[1].cout, ig, L[1].w, L[1].b, t2, f32, s);
    RUN(conv(ctx, L[2], t2, H, W, 1, 0, OUT_NHWC, x, H, W, s, x, nullptr, 0, ig, ig, ig, groups));
    RUN(conv(ctx, L[3], x, H, W, 1, 1, OUT_NHWC, t3, H, W, s, nullptr, nullptr, 0, ig, ig3, 0, groups));
    RUN(conv(ctx, L[4], t3, H, W, 1, 0, OUT_NHWC, x, H, W, s, x, nullptr, 0, ig3, ig, ig, groups));
    return UFVC_OK;
}

// DC-block model, chunk decoder: F = GELU(PS(DU(y^))) + FC(C_i), then 7 blocks (t1..t3: block scratch).
static ufvc_status run_dc_trunk(ufvc_ctx* ctx, Plan* p, const void* yhat, const void* cin, void* F, void* t1, void* t2,
                                void* t3, cudaStream_t s) {
    const int H8 = p->h3, W8 = p->w3;
    prof_begin(ctx, "dc.chunk_decoder", s);
    RUN(conv(ctx, ctx->dcl[DC_DU], yhat, p->Hy, p->Wy, 1, 1, OUT_PS, F, H8, W8, s));
    RUN(conv(ctx, ctx->dcl[DC_FC], cin, H8, W8, 1, 0, OUT_NHWC, F, H8, W8, s, F));
    for (int b = 0; b < 7; ++b) RUN(run_dc_block(ctx, &ctx->dcl[DC_D0 + 5 * b], F, H8, W8, 1, 0, 0, t1, t2, t3, s));
    prof_end(ctx, s, 2 + 7 * 5);
    return UFVC_OK;
}

// DC-block model, context generation in place on F: 11 blocks, C_{i+1} = GO(.).
static ufvc_status run_dc_context(ufvc_ctx* ctx, Plan* p, void* F, void* cout, void* t1, void* t2, void* t3,
                                  cudaStream_t s) {
    const int H8 = p->h3, W8 = p->w3;
    prof_begin(ctx, "dc.context", s);
    for (int b = 0; b < 11; ++b) RUN(run_dc_block(ctx, &ctx->dcl[DC_G0 + 5 * b], F, H8, W8, 1, 0, 0, t1, t2, t3, s));
    RUN(conv(ctx, ctx->dcl[DC_GO], F, H8, W8, 1, 0, OUT_NHWC, cout, H8, W8, s));
    prof_end(ctx, s, 11 * 5 + 1);
    return UFVC_OK;
}

// DC-block model, frame decoders (grouped over the frame positions) from F to frames in final_mode.
static ufvc_status run_dc_frames(ufvc_ctx* ctx, Plan* p, const void* F, void* frames_out, int final_mode,
                                 cudaStream_t s) {
    const int H8 = p->h3, W8 = p->w3, N = ctx->N;
    const long long P = (long long)H8 * W8, gsf = P * kDcCf, gs3 = P * 2 * kDcCf, gso = P * 192;
    prof_begin(ctx, "dc.frame_decoders", s);
    RUN(conv(ctx, ctx->dcf[0], F, H8, W8, 1, 0, OUT_NHWC, p->dc_hf, H8, W8, s, nullptr, nullptr, 0, 0, gsf, 0, N));
    for (int b = 0; b < 3; ++b)
        RUN(run_dc_block(ctx, &ctx->dcf[1 + 5 * b], p->dc_hf, H8, W8, N, gsf, gs3, p->dc_f1, p->dc_f2, p->dc_f3, s));
    RUN(conv(ctx, ctx->dcf[kDcPerFrame - 1], p->dc_hf, H8, W8, 1, 0, OUT_NHWC, p->dc_o, H8, W8, s, nullptr, nullptr, 0,
             gsf, gso, 0, N, true));
    const bool conv_out = ctx->color != UFVC_COLOR_RGB;
    launch_ps8_out(p->dc_o, N, H8, W8, p->H, p->W, conv_out ? (void*)p->fstage : frames_out,
                   !conv_out && final_mode == OUT_PS_FINAL_U8, s);
    if (conv_out) launch_color_out(ctx->color, final_mode == OUT_PS_FINAL_F32, p->fstage, N, p->H, p->W, frames_out, s);
    prof_end(ctx, s, 2 + 3 * 5 + 1 + (conv_out ? 1 : 0));
    return UFVC_OK;
}

// DC-block model, patch embedding and chunk encoder: frames -> y (float).
static ufvc_status run_dc_encoder(ufvc_ctx* ctx, Plan* p, const uint8_t* frames, const void* cin, cudaStream_t s) {
    const int H8 = p->h3, W8 = p->w3;
    const bool f32 = ctx->cfg.precision == UFVC_FP32;
    prof_begin(ctx, "pack", s);
    launch_pack_s2d8(frames, ctx->N, p->H, p->W, H8, W8, p->dc_x0, f32, ctx->color, s);
    prof_end(ctx, s, 1);
    prof_begin(ctx, "analysis", s);
    RUN(conv(ctx, ctx->dcl[DC_PE], p->dc_x0, H8, W8, 1, 0, OUT_NHWC, p->dc_h, H8, W8, s));
    RUN(conv(ctx, ctx->dcl[DC_EC], cin, H8, W8, 1, 0, OUT_NHWC, p->dc_h, H8, W8, s, p->dc_h));
    for (int b = 0; b < 6; ++b)
        RUN(run_dc_block(ctx, &ctx->dcl[DC_E0 + 5 * b], p->dc_h, H8, W8, 1, 0, 0, p->dc_t1e, p->dc_t2e, p->dc_t3e, s));
    RUN(conv(ctx, ctx->dcl[DC_ED], p->dc_h, H8, W8, 2, 0, OUT_NHWC, p->y, p->Hy, p->Wy, s, nullptr, nullptr, 0, 0, 0, 0,
             1, true));
    prof_end(ctx, s, 2 + 6 * 5 + 1);
    return UFVC_OK;
}

// FP8 calibration run (FP32 path): record max |x| of activation tensor t
static void probe(ufvc_ctx* ctx, int t, const float* x, size_t n, cudaStream_t s) {
    if (ctx->amax) launch_absmax(x, n, ctx->amax + t, s);
}

// The plain model's analysis: pack, A1..A3, EC(C_i) with the temporal context, the cross-frame interaction,
// A4 -> y (float in every precision: it feeds the quantiser).
static ufvc_status run_plain_analysis(ufvc_ctx* ctx, Plan* p, const uint8_t* frames, const void* cin, cudaStream_t s) {
    const Arch& a = ctx->arch;
    const bool fp8 = ctx->cfg.precision == UFVC_FP8;
    const bool s2d = ctx->cfg.precision == UFVC_BF16 && ctx->a1s2d.wtc != nullptr && p->C0p == 32;
    // BF16 / FP8 frames in RGB, YUV444 or YUV420 with even N <= 8: A1 reads the frame bytes itself (no pack)
    const bool first = ctx->cfg.precision != UFVC_FP32 && ctx->first_w != nullptr && ctx->color != UFVC_COLOR_RGB_BT709;
    if (first) {
        prof_begin(ctx, "A1", s);
        // (an FP8 context's A1 computes with bf16 operands and writes the E4M3 codes A2 reads)
        CK(launch_first_layer(frames, ctx->color, ctx->N, p->H, p->W, p->h1, p->w1, ctx->first_w, ctx->enc[L_A1].b,
                              p->a1, fp8 ? 1.f / ctx->act_scale[T_A1] : 0.f, ctx->d_status, s));
    } else {
        prof_begin(ctx, "pack", s);
        if (ctx->cfg.precision == UFVC_FP32)
            launch_pack(frames, ctx->N, p->H, p->W, p->Hp, p->Wp, p->C0p, p->x, s, ctx->color);
        else if (fp8)
            launch_pack_fp8(frames, ctx->N, p->H, p->W, p->Hp, p->Wp, reinterpret_cast<uint8_t*>(p->x), s, ctx->color);
        else
            launch_pack_bf16(frames, ctx->N, p->H, p->W, p->Hp, p->Wp, p->C0p, reinterpret_cast<__nv_bfloat16*>(p->x), s,
                             s2d, ctx->color);
        prof_end(ctx, s, 1);
        prof_begin(ctx, "A1", s);
        if (s2d)  // the same layer as a 2x2 stride-1 convolution over the space-to-depth input
            RUN(conv(ctx, ctx->a1s2d, p->x, p->Hp / 2, p->Wp / 2, 1, 1, OUT_NHWC, p->a1, p->h1, p->w1, s));
        else
            RUN(conv(ctx, ctx->enc[L_A1], p->x, p->Hp, p->Wp, 2, 1, OUT_NHWC, p->a1, p->h1, p->w1, s));
    }
    prof_end(ctx, s, 1);
    prof_begin(ctx, "analysis", s);
    probe(ctx, T_A1, p->a1, (size_t)p->h1 * p->w1 * a.e0, s);
    RUN(conv(ctx, ctx->enc[L_A2], p->a1, p->h1, p->w1, 2, 1, OUT_NHWC, p->a2, p->h2, p->w2, s));
    probe(ctx, T_A2, p->a2, (size_t)p->h2 * p->w2 * a.e1, s);
    RUN(conv(ctx, ctx->enc[L_A3], p->a2, p->h2, p->w2, 2, 1, OUT_NHWC, p->a3, p->h3, p->w3, s));
    probe(ctx, T_A3, p->a3, (size_t)p->h3 * p->w3 * a.e2, s);
    if (cin)  // temporal context: the patch-embedded features + EC(C_i), in place
        RUN(conv(ctx, ctx->tl[TL_EC], cin, p->h3, p->w3, 1, 0, OUT_NHWC, p->a3, p->h3, p->w3, s, p->a3));
    RUN(conv(ctx, ctx->enc[L_XA], p->a3, p->h3, p->w3, 1, 1, OUT_NHWC, p->xt, p->h3, p->w3, s));
    probe(ctx, T_XT, p->xt, (size_t)p->h3 * p->w3 * a.e2, s);
    // cross-frame interaction residual, in place
    RUN(conv(ctx, ctx->enc[L_XB], p->xt, p->h3, p->w3, 1, 0, OUT_NHWC, p->a3, p->h3, p->w3, s, p->a3));
    probe(ctx, T_A3R, p->a3, (size_t)p->h3 * p->w3 * a.e2, s);
    // y is float in every precision (it feeds the quantiser)
    RUN(conv(ctx, ctx->enc[L_A4], p->a3, p->h3, p->w3, 2, 0, OUT_NHWC, p->y, p->Hy, p->Wy, s, nullptr, nullptr, 0, 0, 0,
             0, 1, true));
    probe(ctx, T_Y, p->y, p->ny, s);
    prof_end(ctx, s, cin ? 6 : 5);
    return UFVC_OK;
}

static ufvc_status run_encoder_front(ufvc_ctx* ctx, Plan* p, const uint8_t* frames, int qp, cudaStream_t s) {
    const Arch& a = ctx->arch;
    const bool fp8 = ctx->cfg.precision == UFVC_FP8;
    ctx->cur_ws = &p->ws_enc;
    const void* cin = ctx->tc_on ? (ctx->cur_cin ? ctx->cur_cin : (const void*)p->t_zero) : nullptr;
    if (ctx->dcm) RUN(run_dc_encoder(ctx, p, frames, cin, s));
    else RUN(run_plain_analysis(ctx, p, frames, cin, s));
    prof_begin(ctx, "hyper_analysis", s);
    const int nl_ha = ctx->conv_launches;
    if (use_tc(ctx, ctx->enc[L_H1])) {
        // tensor cores: only the encoder computes z (z^ travels in the bit-stream), so the hyper-analysis
        // needs no bit-exact twin on the decoder side
        if (fp8)
            launch_f32_to_e4m3_rows(p->y, p->Hy, p->Wy, a.cy, 1.f / ctx->act_scale[T_Y],
                                    reinterpret_cast<uint8_t*>(p->y_bf), p->Wye, s);
        else
            launch_f32_to_bf16_rows(p->y, p->Hy, p->Wy, a.cy, p->y_bf, p->Wye, s);
        RUN(conv(ctx, ctx->enc[L_H1], p->y_bf, p->Hye, p->Wye, 2, 1, OUT_NHWC, p->hb_bf, p->hhe, p->whe, s));
        RUN(conv(ctx, ctx->enc[L_H2], p->hb_bf, p->hhe, p->whe, 2, 0, OUT_NHWC, p->z, p->Hz, p->Wz, s, nullptr,
                 nullptr, 0, 0, 0, 0, 1, true));
        launch_zquant(p->z, p->Hz * p->Wz, a.cz, p->zthr, p->zhat, p->iz, s);
        prof_end(ctx, s, 2 + (ctx->conv_launches - nl_ha));  // the conversion, z^ and every conv kernel
    } else {
        RUN(conv(ctx, ctx->enc[L_H1], p->y, p->Hy, p->Wy, 2, 1, OUT_NHWC, p->hb, p->hh, p->wh, s));
        probe(ctx, T_HB, p->hb, (size_t)p->hh * p->wh * a.cz, s);
        RUN(conv(ctx, ctx->enc[L_H2], p->hb, p->hh, p->wh, 2, 0, OUT_NHWC, p->z, p->Hz, p->Wz, s));
        launch_zquant(p->z, p->Hz * p->Wz, a.cz, p->zthr, p->zhat, p->iz, s);
        prof_end(ctx, s, 1 + (ctx->conv_launches - nl_ha));
    }
    // the last hyper-synthesis layer also quantises the latent and forms its scale indices
    const EntParams ent{p->idx, p->y, p->rhat, nullptr, qp, true};
    RUN(run_hyper_synthesis(ctx, p, p->zhat, p->zf, p->s1, p->s2, p->mu, p->ls, s, cin, p->t_pc_e, &ent));
    if (ctx->pm_on)
        RUN(run_progressive(ctx, p->Hy, p->Wy, p->y, p->rhat, p->mu, p->s2, nullptr, qp, nullptr, p->pm_in_e, p->pm_h_e,
                            p->pm_mu_e, s));
    if (cin && ctx->cur_cout) {  // the encoder tracks the decoder's context from its own y^ = r^ q + mu
        const bool f32 = ctx->cfg.precision == UFVC_FP32;
        launch_dequant(p->rhat, p->mu, p->ny, ctx->d_qstep, nullptr, f32 ? p->t_yh_e : nullptr,
                       f32 ? nullptr : reinterpret_cast<__nv_bfloat16*>(p->t_yh_e), s, nullptr, 0.f, qp);
        if (ctx->dcm) {  // the encoder runs the decoder's trunk and context generation on its own scratch
            RUN(run_dc_trunk(ctx, p, p->t_yh_e, cin, p->dc_h, p->dc_t1e, p->dc_t2e, p->dc_t3e, s));
            RUN(run_dc_context(ctx, p, p->dc_h, ctx->cur_cout, p->dc_t1e, p->dc_t2e, p->dc_t3e, s));
        } else {
            RUN(run_chunk_feature(ctx, p, p->t_yh_e, cin, p->t_F_e, ctx->cur_cout, s));
        }
    }
    return UFVC_OK;
}

// yhat: float [Hy][Wy][Cy] in FP32 precision, bf16 otherwise
// F: the chunk feature (temporal context), added to every frame decoder's D0 output through its DF_f
static ufvc_status run_decoders(ufvc_ctx* ctx, Plan* p, const void* yhat, void* frames_out, int final_mode,
                                cudaStream_t s, const void* F = nullptr) {
    const Arch& a = ctx->arch;
    const int N = ctx->N;
    const int h1 = 2 * p->Hy, w1 = 2 * p->Wy, h2 = 4 * p->Hy, w2 = 4 * p->Wy, h3 = 8 * p->Hy, w3 = 8 * p->Wy;
    const long long g1 = (long long)h1 * w1 * a.cd1, g2 = (long long)h2 * w2 * a.cd2, g3 = (long long)h3 * w3 * a.cd2;
    const long long gf = (long long)p->H * p->W * 3;
    prof_begin(ctx, "dec.D0", s);
    RUN(conv(ctx, ctx->dec[D_D0], yhat, p->Hy, p->Wy, 1, 1, OUT_PS, p->bufA, h1, w1, s, nullptr, nullptr, 0, 0, g1, 0,
             N));
    if (F)
        RUN(conv(ctx, ctx->tdf, F, h1, w1, 1, 0, OUT_NHWC, p->bufA, h1, w1, s, p->bufA, nullptr, 0, 0, g1, g1, N));
    probe(ctx, T_D0, (const float*)p->bufA, (size_t)N * h1 * w1 * a.cd1, s);
    prof_end(ctx, s, F ? 2 : 1);
    prof_begin(ctx, "dec.R1", s);
    RUN(conv(ctx, ctx->dec[D_R1A], p->bufA, h1, w1, 1, 1, OUT_NHWC, p->bufT, h1, w1, s, nullptr, nullptr, 0, g1, g1, 0,
             N));
    probe(ctx, T_R1A, (const float*)p->bufT, (size_t)N * h1 * w1 * a.cd1, s);
    RUN(conv(ctx, ctx->dec[D_R1B], p->bufT, h1, w1, 1, 0, OUT_NHWC, p->bufA, h1, w1, s, p->bufA, nullptr, 0, g1, g1,
             g1, N));
    probe(ctx, T_R1B, (const float*)p->bufA, (size_t)N * h1 * w1 * a.cd1, s);
    prof_end(ctx, s, 2);
    prof_begin(ctx, "dec.U1", s);
    RUN(conv(ctx, ctx->dec[D_U1], p->bufA, h1, w1, 1, 1, OUT_PS, p->bufB, h2, w2, s, nullptr, nullptr, 0, g1, g2, 0, N));
    probe(ctx, T_U1, (const float*)p->bufB, (size_t)N * h2 * w2 * a.cd2, s);
    prof_end(ctx, s, 1);
    prof_begin(ctx, "dec.R2", s);
    RUN(conv(ctx, ctx->dec[D_R2A], p->bufB, h2, w2, 1, 1, OUT_NHWC, p->bufT2, h2, w2, s, nullptr, nullptr, 0, g2, g2, 0,
             N));
    probe(ctx, T_R2A, (const float*)p->bufT2, (size_t)N * h2 * w2 * a.cd2, s);
    RUN(conv(ctx, ctx->dec[D_R2B], p->bufT2, h2, w2, 1, 0, OUT_NHWC, p->bufB, h2, w2, s, p->bufB, nullptr, 0, g2, g2,
             g2, N));
    probe(ctx, T_R2B, (const float*)p->bufB, (size_t)N * h2 * w2 * a.cd2, s);
    prof_end(ctx, s, 2);
    prof_begin(ctx, "dec.U2", s);
    RUN(conv(ctx, ctx->dec[D_U2], p->bufB, h2, w2, 1, 1, OUT_PS, p->bufC, h3, w3, s, nullptr, nullptr, 0, g2, g3, 0, N));
    prof_end(ctx, s, 1);
    prof_begin(ctx, "dec.U3", s);
    // colour formats other than RGB: x^ as float into the plan's staging, then the format conversion
    const bool conv_out = ctx->color != UFVC_COLOR_RGB && (final_mode == OUT_PS_FINAL_U8 || final_mode == OUT_PS_FINAL_F32);
    RUN(conv(ctx, ctx->dec[D_U3], p->bufC, h3, w3, 1, 0, conv_out ? OUT_PS_FINAL_F32 : final_mode,
             conv_out ? (void*)p->fstage : frames_out, p->H, p->W, s, nullptr, nullptr, 0, g3, gf, 0, N));
    prof_end(ctx, s, 1);
    if (conv_out) {
        prof_begin(ctx, "color_out", s);
        launch_color_out(ctx->color, final_mode == OUT_PS_FINAL_F32, p->fstage, N, p->H, p->W, frames_out, s);
        prof_end(ctx, s, 1);
    }
    return UFVC_OK;
}

// ------------------------------------------------------------------------------------------------
// chunk encode / decode
// ------------------------------------------------------------------------------------------------
// A batch of B chunks of one size: each chunk's analysis, hyperprior and entropy parameters run in its own
// plan (batch position b), then the rANS coding of all 2B sections is one launch.
static ufvc_status encode_batch(ufvc_ctx* ctx, int B, const uint8_t* const* frames, int width, int height,
                                const int* qps, uint8_t* const* bits, size_t capacity, uint64_t* const* nbytes,
                                cudaStream_t s) {
    Plan* plans[kRansMaxStreams];
    for (int b = 0; b < B; ++b) {
        RUN(get_plan(ctx, width, height, false, &plans[b], b));
        RUN(run_encoder_front(ctx, plans[b], frames[b], qps[b], s));
    }
    // both sections of every chunk coded, laid out and the headers written in one launch
    prof_begin(ctx, "rans_encode", s);
    RansEncJob j{};
    const int version = 1 + (ctx->pm_on ? 1 : 0) + (ctx->tc_on ? 2 : 0);
    for (int b = 0; b < B; ++b) {
        Plan* p = plans[b];
        j.s[2 * b] = RansEncSec{p->zhat, p->iz, ctx->arch.cz, (uint32_t)p->nz, p->Kz, p->scr_z, p->cap_z, b};
        j.s[2 * b + 1] = RansEncSec{p->rhat, p->idx, 0, (uint32_t)p->ny, ctx->cfg.lanes, p->scr_y, p->cap_y, b};
        RansEncStream& o = j.st[b];
        o.out = bits[b];
        o.capacity = capacity;
        o.nbytes = nbytes[b];
        o.base = p->hdr;
        o.hdr_len = (int)p->hdr;
        const uint32_t fields[] = {'U', 'F', 'V', 'C', (uint32_t)version, (uint32_t)ctx->cfg.arch, (uint32_t)ctx->N,
                                   (uint32_t)qps[b]};
        for (int i = 0; i < 8; ++i) o.hdr20[i] = (uint8_t)fields[i];
        for (int i = 0; i < 2; ++i) {
            o.hdr20[8 + i] = (uint8_t)(width >> (8 * i));
            o.hdr20[10 + i] = (uint8_t)(height >> (8 * i));
        }
        for (int i = 0; i < 4; ++i) {
            o.hdr20[12 + i] = (uint8_t)((uint32_t)ctx->cfg.lanes >> (8 * i));
            o.hdr20[16 + i] = (uint8_t)((uint32_t)p->Kz >> (8 * i));
        }
        o.iz = p->iz;
        o.cz = ctx->arch.cz;
    }
    j.nsec = 2 * B;
    j.nstreams = B;
    j.ctl = plans[0]->ctl;
    j.status = ctx->d_status;
    j.spin = ctx->table_spin;
    CK(launch_rans_encode(j, ctx->d_packed, s));
    prof_end(ctx, s, 1);
    CK(cudaGetLastError());
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_encode_chunk(ufvc_ctx* ctx, const uint8_t* d_frames, int n_frames, int width, int height,
                                         int qp, uint8_t* d_bits, size_t capacity, uint64_t* d_nbytes, void* stream) {
    if (!ctx || !d_frames || !d_bits || !d_nbytes || !check_shape(ctx, n_frames, width, height) || qp < 0 || qp > 63)
        return fail(ctx, UFVC_ERR_ARG, "encode_chunk: bad argument");
    if (fp8_unready(ctx)) return fail(ctx, UFVC_ERR_ARG, "encode_chunk: FP8 context not calibrated (ufvc_calibrate_fp8)");
    CK(cudaSetDevice(ctx->cfg.device));
    return encode_batch(ctx, 1, &d_frames, width, height, &qp, &d_bits, capacity, &d_nbytes, (cudaStream_t)stream);
}

// nbytes: the stream size, or (with d_nbytes) the readable capacity, the size then being read on the device
static ufvc_status decode_batch(ufvc_ctx* ctx, int B, const uint8_t* const* bits, size_t nbytes, void* const* frames,
                                int final_mode, int width, int height, cudaStream_t s,
                                const uint64_t* const* d_nbytes = nullptr) {
    Plan* plans[kRansMaxDecSec];
    for (int b = 0; b < B; ++b) RUN(get_plan(ctx, width, height, true, &plans[b], b));
    const Arch& a = ctx->arch;
    const bool fp32 = ctx->cfg.precision == UFVC_FP32, fp8 = ctx->cfg.precision == UFVC_FP8;
    // z^ sections: each chunk's header is checked in the same launch (its scale indices are the section's
    // tables)
    prof_begin(ctx, "rans_decode_z", s);
    RansDecJob jz{};
    for (int b = 0; b < B; ++b) {
        Plan* p = plans[b];
        RansDecSec& e = jz.s[b];
        e.bits = bits[b];
        e.nbytes = nbytes;
        e.sec_off = p->hdr;
        e.idx = bits[b] + 20;
        e.next_off = p->next_z;
        e.sym = p->dzhat;
        e.qp_out = p->qp_dev;
        e.ver_out = p->ver_dev;
    }
    jz.nsec = B;
    jz.idx_period = a.cz;
    jz.n = (uint32_t)plans[0]->nz;
    jz.K = plans[0]->Kz;
    jz.out = kDecSym;
    jz.hdr_cz = a.cz;
    jz.arch = ctx->cfg.arch;
    jz.N = ctx->N;
    jz.W = width;
    jz.H = height;
    jz.Ky = ctx->cfg.lanes;
    jz.allow_pm = ctx->pm_on;
    jz.temporal = ctx->tc_on;
    jz.status = ctx->d_status;
    jz.spin = ctx->table_spin;
    CK(launch_rans_decode(jz, ctx->d_dec, s));
    prof_end(ctx, s, 1);
    const void* cin = nullptr;
    for (int b = 0; b < B; ++b) {
        Plan* p = plans[b];
        ctx->cur_ws = &p->ws_dec;
        cin = ctx->tc_on ? (ctx->cur_cin ? ctx->cur_cin : (const void*)p->t_zero) : nullptr;
        // the last hyper-synthesis layer also forms the scale indices (at the rate the header carries)
        const EntParams ent{p->didx, nullptr, nullptr, p->qp_dev, 0, false};
        RUN(run_hyper_synthesis(ctx, p, p->dzhat, p->dzf, p->ds1, p->ds2, p->dmu, p->dls, s, cin, p->t_pc_d, &ent));
    }
    // y^ sections, each ending exactly at its stream's end; with the single-pass means the decoder writes
    // y^ = r^ q + mu itself, the progressive means need r^ first
    prof_begin(ctx, "rans_decode_y", s);
    RansDecJob jy{};
    for (int b = 0; b < B; ++b) {
        Plan* p = plans[b];
        RansDecSec& e = jy.s[b];
        e.bits = bits[b];
        e.nbytes = nbytes;
        e.sec_off_dev = p->next_z;
        e.expect_end = d_nbytes ? 0 : nbytes;
        e.expect_end_dev = d_nbytes ? d_nbytes[b] : nullptr;
        e.idx = p->didx;
        e.sym = p->drhat;
        e.yout = fp32 ? (void*)p->yhat : (void*)p->yhat_bf;
        e.mu = p->dmu;
        e.qp_dev = p->qp_dev;
    }
    jy.nsec = B;
    jy.n = (uint32_t)plans[0]->ny;
    jy.K = ctx->cfg.lanes;
    jy.out = ctx->pm_on ? kDecSym : fp32 ? kDecF32 : fp8 ? kDecE4M3 : kDecBf16;
    jy.qstep_all = ctx->d_qstep;
    jy.inv8 = fp8 ? 1.f / ctx->act_scale[T_YHAT] : 0.f;
    jy.status = ctx->d_status;
    jy.spin = ctx->table_spin;
    CK(launch_rans_decode(jy, ctx->d_dec, s));
    prof_end(ctx, s, 1);
    for (int b = 0; b < B; ++b) {
        Plan* p = plans[b];
        if (ctx->pm_on) {  // a version-1 stream leaves the means of the single pass (the steps check the version)
            RUN(run_progressive(ctx, p->Hy, p->Wy, nullptr, p->drhat, p->dmu, p->ds2, p->qp_dev, 0, p->ver_dev,
                                p->pm_in_d, p->pm_h_d, p->pm_mu_d, s));
            prof_begin(ctx, "dequant", s);
            launch_dequant(p->drhat, p->dmu, p->ny, ctx->d_qstep, p->qp_dev, fp32 ? p->yhat : nullptr,
                           fp32 || fp8 ? nullptr : p->yhat_bf, s, fp8 ? reinterpret_cast<uint8_t*>(p->yhat_bf) : nullptr,
                           fp8 ? 1.f / ctx->act_scale[T_YHAT] : 0.f);
            prof_end(ctx, s, 1);
        }
        if (fp32) probe(ctx, T_YHAT, p->yhat, p->ny, s);
        const void* yh = fp32 ? (const void*)p->yhat : (const void*)p->yhat_bf;
        if (ctx->dcm) {  // chunk decoder, frame decoders, then the context generation in place on F
            RUN(run_dc_trunk(ctx, p, yh, cin, p->dc_F, p->dc_t1d, p->dc_t2d, p->dc_t3d, s));
            RUN(run_dc_frames(ctx, p, p->dc_F, frames[b], final_mode, s));
            if (ctx->cur_cout) RUN(run_dc_context(ctx, p, p->dc_F, ctx->cur_cout, p->dc_t1d, p->dc_t2d, p->dc_t3d, s));
            continue;
        }
        if (cin) RUN(run_chunk_feature(ctx, p, yh, cin, p->t_F_d, ctx->cur_cout, s));
        RUN(run_decoders(ctx, p, yh, frames[b], final_mode, s, cin ? (const void*)p->t_F_d : nullptr));
    }
    CK(cudaGetLastError());
    return UFVC_OK;
}

static ufvc_status decode_impl(ufvc_ctx* ctx, const uint8_t* d_bits, size_t nbytes, void* d_frames, int final_mode,
                               int n_frames, int width, int height, void* stream, const uint64_t* d_nbytes = nullptr) {
    if (!ctx || !d_bits || !d_frames || !check_shape(ctx, n_frames, width, height) || nbytes == 0)
        return fail(ctx, UFVC_ERR_ARG, "decode_chunk: bad argument");
    if (fp8_unready(ctx)) return fail(ctx, UFVC_ERR_ARG, "decode_chunk: FP8 context not calibrated (ufvc_calibrate_fp8)");
    CK(cudaSetDevice(ctx->cfg.device));
    return decode_batch(ctx, 1, &d_bits, nbytes, &d_frames, final_mode, width, height, (cudaStream_t)stream,
                        d_nbytes ? &d_nbytes : nullptr);
}

// Batched calls (serving): B chunks of one size, each with its own buffers, their rANS sections coded in one
// launch.  Not for contexts that carry a temporal context (each stream has its own).
static bool batch_ok(ufvc_ctx* ctx, int batch) {
    return batch >= 1 && batch <= kRansMaxDecSec && (batch == 1 || (!ctx->tc_on && !ctx->dcm));
}

extern "C" ufvc_status ufvc_encode_chunks(ufvc_ctx* ctx, int batch, const uint8_t* const* d_frames, int n_frames,
                                          int width, int height, const int* qps, uint8_t* const* d_bits,
                                          size_t capacity, uint64_t* const* d_nbytes, void* stream) {
    if (!ctx || !d_frames || !d_bits || !d_nbytes || !qps || !check_shape(ctx, n_frames, width, height))
        return fail(ctx, UFVC_ERR_ARG, "encode_chunks: bad argument");
    if (!batch_ok(ctx, batch))
        return fail(ctx, batch >= 1 && batch <= kRansMaxDecSec ? UFVC_ERR_UNSUPPORTED : UFVC_ERR_ARG,
                    "encode_chunks: batch must be 1..8, and 1 for a context with a temporal context");
    for (int b = 0; b < batch; ++b)
        if (!d_frames[b] || !d_bits[b] || !d_nbytes[b] || qps[b] < 0 || qps[b] > 63)
            return fail(ctx, UFVC_ERR_ARG, "encode_chunks: bad argument");
    if (fp8_unready(ctx)) return fail(ctx, UFVC_ERR_ARG, "encode_chunks: FP8 context not calibrated (ufvc_calibrate_fp8)");
    CK(cudaSetDevice(ctx->cfg.device));
    return encode_batch(ctx, batch, d_frames, width, height, qps, d_bits, capacity, d_nbytes, (cudaStream_t)stream);
}

extern "C" ufvc_status ufvc_decode_chunks(ufvc_ctx* ctx, int batch, const uint8_t* const* d_bits, size_t capacity,
                                          const uint64_t* const* d_nbytes, uint8_t* const* d_frames, int n_frames,
                                          int width, int height, void* stream) {
    if (!ctx || !d_frames || !d_bits || !d_nbytes || !check_shape(ctx, n_frames, width, height) || capacity == 0)
        return fail(ctx, UFVC_ERR_ARG, "decode_chunks: bad argument");
    if (!batch_ok(ctx, batch))
        return fail(ctx, batch >= 1 && batch <= kRansMaxDecSec ? UFVC_ERR_UNSUPPORTED : UFVC_ERR_ARG,
                    "decode_chunks: batch must be 1..8, and 1 for a context with a temporal context");
    for (int b = 0; b < batch; ++b)
        if (!d_frames[b] || !d_bits[b] || !d_nbytes[b]) return fail(ctx, UFVC_ERR_ARG, "decode_chunks: bad argument");
    if (fp8_unready(ctx)) return fail(ctx, UFVC_ERR_ARG, "decode_chunks: FP8 context not calibrated (ufvc_calibrate_fp8)");
    CK(cudaSetDevice(ctx->cfg.device));
    void* fr[kRansMaxDecSec];
    for (int b = 0; b < batch; ++b) fr[b] = d_frames[b];
    return decode_batch(ctx, batch, d_bits, capacity, fr, OUT_PS_FINAL_U8, width, height, (cudaStream_t)stream,
                        d_nbytes);
}

extern "C" ufvc_status ufvc_decode_chunk(ufvc_ctx* ctx, const uint8_t* d_bits, size_t nbytes, uint8_t* d_frames,
                                         int n_frames, int width, int height, void* stream) {
    return decode_impl(ctx, d_bits, nbytes, d_frames, OUT_PS_FINAL_U8, n_frames, width, height, stream);
}

extern "C" ufvc_status ufvc_decode_chunk_f32(ufvc_ctx* ctx, const uint8_t* d_bits, size_t nbytes, float* d_frames,
                                             int n_frames, int width, int height, void* stream) {
    return decode_impl(ctx, d_bits, nbytes, d_frames, OUT_PS_FINAL_F32, n_frames, width, height, stream);
}

extern "C" ufvc_status ufvc_decode_chunk_dev(ufvc_ctx* ctx, const uint8_t* d_bits, size_t capacity,
                                             const uint64_t* d_nbytes, uint8_t* d_frames, int n_frames, int width,
                                             int height, void* stream) {
    if (!d_nbytes) return fail(ctx, UFVC_ERR_ARG, "decode_chunk_dev: null size");
    return decode_impl(ctx, d_bits, capacity, d_frames, OUT_PS_FINAL_U8, n_frames, width, height, stream, d_nbytes);
}

// ------------------------------------------------------------------------------------------------
// host-buffer variants
// ------------------------------------------------------------------------------------------------
static ufvc_status ensure_staging(ufvc_ctx* ctx, size_t frames_sz, size_t bits_sz) {
    if (frames_sz > ctx->st_frames_sz) {
        cudaFree(ctx->st_frames);
        ctx->st_frames = nullptr;
        ufvc_status st = dalloc(ctx, nullptr, &ctx->st_frames, frames_sz);
        if (st) return st;
        ctx->st_frames_sz = frames_sz;
    }
    if (bits_sz > ctx->st_bits_sz) {
        cudaFree(ctx->st_bits);
        ctx->st_bits = nullptr;
        ufvc_status st = dalloc(ctx, nullptr, &ctx->st_bits, bits_sz);
        if (st) return st;
        ctx->st_bits_sz = bits_sz;
    }
    if (!ctx->st_nbytes) {
        ufvc_status st = dalloc(ctx, nullptr, &ctx->st_nbytes, 1);
        if (st) return st;
    }
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_encode_chunk_host(ufvc_ctx* ctx, const uint8_t* h_frames, int n_frames, int width,
                                              int height, int qp, uint8_t* h_bits, size_t capacity, size_t* nbytes,
                                              void* stream) {
    if (!ctx || !h_frames || !h_bits || !nbytes || !check_shape(ctx, n_frames, width, height))
        return fail(ctx, UFVC_ERR_ARG, "encode_chunk_host: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->cfg.device));
    const size_t fsz = (size_t)n_frames * frame_bytes(ctx->color, width, height);
    const size_t bmax = ufvc_max_bitstream_bytes(ctx, width, height);
    ufvc_status st = ensure_staging(ctx, fsz, bmax);
    if (st) return st;
    CK(cudaMemcpyAsync(ctx->st_frames, h_frames, fsz, cudaMemcpyHostToDevice, s));
    st = ufvc_encode_chunk(ctx, ctx->st_frames, n_frames, width, height, qp, ctx->st_bits, bmax, ctx->st_nbytes, stream);
    if (st) return st;
    uint64_t nb = 0;
    CK(cudaMemcpyAsync(&nb, ctx->st_nbytes, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *nbytes = nb;
    if (nb > capacity) return fail(ctx, UFVC_ERR_CAPACITY, "encode_chunk_host: capacity");
    CK(cudaMemcpyAsync(h_bits, ctx->st_bits, nb, cudaMemcpyDeviceToHost, s));
    return ufvc_sync_status(ctx, stream);
}

extern "C" ufvc_status ufvc_decode_chunk_host(ufvc_ctx* ctx, const uint8_t* h_bits, size_t nbytes, uint8_t* h_frames,
                                              int n_frames, int width, int height, void* stream) {
    if (!ctx || !h_bits || !h_frames || !check_shape(ctx, n_frames, width, height) || nbytes == 0)
        return fail(ctx, UFVC_ERR_ARG, "decode_chunk_host: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->cfg.device));
    const size_t fsz = (size_t)n_frames * frame_bytes(ctx->color, width, height);
    ufvc_status st = ensure_staging(ctx, fsz, nbytes);
    if (st) return st;
    CK(cudaMemcpyAsync(ctx->st_bits, h_bits, nbytes, cudaMemcpyHostToDevice, s));
    st = ufvc_decode_chunk(ctx, ctx->st_bits, nbytes, ctx->st_frames, n_frames, width, height, stream);
    if (st) return st;
    CK(cudaMemcpyAsync(h_frames, ctx->st_frames, fsz, cudaMemcpyDeviceToHost, s));
    return ufvc_sync_status(ctx, stream);
}

// ------------------------------------------------------------------------------------------------
// stage entry points
// ------------------------------------------------------------------------------------------------
extern "C" ufvc_status ufvc_encode_stages(ufvc_ctx* ctx, const uint8_t* d_frames, int width, int height, int qp,
                                          float* d_y, int16_t* d_zhat, uint8_t* d_iz, float* d_mu, float* d_logsig,
                                          int16_t* d_rhat, uint8_t* d_idx, void* stream) {
    if (!ctx || !d_frames || !check_shape(ctx, ctx->N, width, height) || qp < 0 || qp > 63)
        return fail(ctx, UFVC_ERR_ARG, "encode_stages: bad argument");
    if (fp8_unready(ctx)) return fail(ctx, UFVC_ERR_ARG, "encode_stages: FP8 context not calibrated (ufvc_calibrate_fp8)");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->cfg.device));
    Plan* p;
    ufvc_status st = get_plan(ctx, width, height, false, &p);
    if (st) return st;

    RUN(run_encoder_front(ctx, p, d_frames, qp, s));
    const Arch& a = ctx->arch;
    if (d_y) CK(cudaMemcpyAsync(d_y, p->y, p->ny * 4, cudaMemcpyDeviceToDevice, s));
    if (d_zhat) CK(cudaMemcpyAsync(d_zhat, p->zhat, p->nz * 2, cudaMemcpyDeviceToDevice, s));
    if (d_iz) CK(cudaMemcpyAsync(d_iz, p->iz, a.cz, cudaMemcpyDeviceToDevice, s));
    if (d_mu) CK(cudaMemcpyAsync(d_mu, p->mu, p->ny * 4, cudaMemcpyDeviceToDevice, s));
    if (d_logsig) CK(cudaMemcpyAsync(d_logsig, p->ls, p->ny * 4, cudaMemcpyDeviceToDevice, s));
    if (d_rhat) CK(cudaMemcpyAsync(d_rhat, p->rhat, p->ny * 2, cudaMemcpyDeviceToDevice, s));
    if (d_idx) CK(cudaMemcpyAsync(d_idx, p->idx, p->ny, cudaMemcpyDeviceToDevice, s));
    CK(cudaGetLastError());
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_hyper_synthesis(ufvc_ctx* ctx, const int16_t* d_zhat, int Hz, int Wz, int Hy, int Wy,
                                            float* d_mu, float* d_logsig, void* stream) {
    if (!ctx || !d_zhat || !d_mu || !d_logsig || Hz < 1 || Wz < 1 || Hy < 1 || Wy < 1 || 4 * Hz < Hy || 4 * Wz < Wy)
        return fail(ctx, UFVC_ERR_ARG, "hyper_synthesis: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->cfg.device));
    const Arch& a = ctx->arch;
    Plan tmp;
    tmp.Hz = Hz; tmp.Wz = Wz; tmp.Hy = Hy; tmp.Wy = Wy;
    tmp.nz = (size_t)Hz * Wz * a.cz;
    float *zf, *s1, *s2;
    ufvc_status st;
    if ((st = dalloc(ctx, &tmp, &zf, tmp.nz)) || (st = dalloc(ctx, &tmp, &s1, 4 * tmp.nz)) ||
        (st = dalloc(ctx, &tmp, &s2, (size_t)Hy * Wy * a.cz))) {
        for (void* v : tmp.allocs) cudaFree(v);
        return st;
    }

    ctx->cur_ws = &ctx->ws_stage;
    st = run_hyper_synthesis(ctx, &tmp, d_zhat, zf, s1, s2, d_mu, d_logsig, s);
    cudaError_t e = cudaStreamSynchronize(s);
    for (void* v : tmp.allocs) cudaFree(v);
    if (st) return st;
    if (e != cudaSuccess) return fail(ctx, UFVC_ERR_CUDA, cudaGetErrorString(e));
    return UFVC_OK;
}

extern "C" size_t ufvc_mean_weight_count(int arch) { return mean_weight_count(arch); }

extern "C" size_t ufvc_temporal_weight_count(int arch, int chunk_len) { return temporal_weight_count(arch, chunk_len); }

extern "C" ufvc_status ufvc_set_temporal_context(ufvc_ctx* ctx, const float* weights, size_t n_weights) {
    if (!ctx || !weights) return fail(ctx, UFVC_ERR_ARG, "set_temporal_context: bad argument");
    if (ctx->borrowed) return fail(ctx, UFVC_ERR_ARG, "set_temporal_context: context shares another's weights");
    if (ctx->tc_on) return fail(ctx, UFVC_ERR_ARG, "set_temporal_context: already set (the DC-block model has its own)");
    if (ctx->cfg.precision == UFVC_FP8)
        return fail(ctx, UFVC_ERR_UNSUPPORTED, "set_temporal_context: not available in FP8 contexts");
    if (n_weights != temporal_weight_count(ctx->cfg.arch, ctx->N))
        return fail(ctx, UFVC_ERR_ARG, "set_temporal_context: weight count");
    CK(cudaSetDevice(ctx->cfg.device));
    const int nl = TL_N + ctx->N;
    std::vector<size_t> offs(nl);
    size_t off = 0;
    for (int l = 0; l < nl; ++l) {
        int co, k, ci;
        temporal_layer_shape(ctx->cfg.arch, ctx->N, l, &co, &k, &ci);
        offs[l] = off;
        off += (size_t)co * k * k * ci + co;
    }
    for (int l = 0; l <= TL_N; ++l) {  // the five shared layers, then DF grouped over the frame positions
        int sh[3];
        temporal_layer_shape(ctx->cfg.arch, ctx->N, l, &sh[0], &sh[1], &sh[2]);
        LayerW& L = l < TL_N ? ctx->tl[l] : ctx->tdf;
        ufvc_status st = upload_layer(ctx, L, weights, offs.data(), l, l < TL_N ? 1 : ctx->N, true, l == TL_FD, false,
                                      sh, true, 1);
        if (st != UFVC_OK) return st;
    }
    ctx->tc_on = true;
    return UFVC_OK;
}

extern "C" size_t ufvc_context_bytes(const ufvc_ctx* ctx, int width, int height) {
    if (!ctx || width < 1 || height < 1) return 0;
    const size_t es = ctx->cfg.precision == UFVC_FP32 ? 4 : 2;
    return (size_t)((height + 15) / 16 * 2) * ((width + 15) / 16 * 2) * ctx->cc * es;
}

// runs fn with the call's context buffers installed (temporal-context contexts only)
template <class Fn>
static ufvc_status with_context(ufvc_ctx* ctx, const void* d_ctx_in, void* d_ctx_out, const char* what, Fn fn) {
    if (!ctx) return UFVC_ERR_ARG;
    if (!ctx->tc_on) return fail(ctx, UFVC_ERR_ARG, (std::string(what) + ": no temporal context (ufvc_set_temporal_context)").c_str());
    if (((uintptr_t)d_ctx_in & 15) || ((uintptr_t)d_ctx_out & 15))
        return fail(ctx, UFVC_ERR_ARG, (std::string(what) + ": context buffers must be 16-byte aligned").c_str());
    if (d_ctx_in && d_ctx_in == d_ctx_out)
        return fail(ctx, UFVC_ERR_ARG, (std::string(what) + ": context in and out must differ").c_str());
    ctx->cur_cin = d_ctx_in;
    ctx->cur_cout = d_ctx_out;
    const ufvc_status st = fn();
    ctx->cur_cin = nullptr;
    ctx->cur_cout = nullptr;
    return st;
}

extern "C" ufvc_status ufvc_encode_chunk_tc(ufvc_ctx* ctx, const uint8_t* d_frames, int n_frames, int width,
                                            int height, int qp, uint8_t* d_bits, size_t capacity, uint64_t* d_nbytes,
                                            const void* d_ctx_in, void* d_ctx_out, void* stream) {
    return with_context(ctx, d_ctx_in, d_ctx_out, "encode_chunk_tc", [&] {
        return ufvc_encode_chunk(ctx, d_frames, n_frames, width, height, qp, d_bits, capacity, d_nbytes, stream);
    });
}

extern "C" ufvc_status ufvc_decode_chunk_tc(ufvc_ctx* ctx, const uint8_t* d_bits, size_t nbytes, const uint64_t* d_nbytes,
                                            void* d_frames, int f32, int n_frames, int width, int height,
                                            const void* d_ctx_in, void* d_ctx_out, void* stream) {
    return with_context(ctx, d_ctx_in, d_ctx_out, "decode_chunk_tc", [&] {
        return decode_impl(ctx, d_bits, nbytes, d_frames, f32 ? OUT_PS_FINAL_F32 : OUT_PS_FINAL_U8, n_frames, width,
                           height, stream, d_nbytes);
    });
}

extern "C" ufvc_status ufvc_encode_stages_tc(ufvc_ctx* ctx, const uint8_t* d_frames, int width, int height, int qp,
                                             const void* d_ctx_in, float* d_y, int16_t* d_zhat, uint8_t* d_iz,
                                             float* d_mu, float* d_logsig, int16_t* d_rhat, uint8_t* d_idx,
                                             void* stream) {
    return with_context(ctx, d_ctx_in, nullptr, "encode_stages_tc", [&] {
        return ufvc_encode_stages(ctx, d_frames, width, height, qp, d_y, d_zhat, d_iz, d_mu, d_logsig, d_rhat, d_idx,
                                  stream);
    });
}

extern "C" size_t ufvc_frame_bytes(int format, int width, int height) {
    if (format < UFVC_COLOR_RGB || format > UFVC_COLOR_YUV420P || width < 1 || height < 1) return 0;
    return frame_bytes(format, width, height);
}

extern "C" ufvc_status ufvc_set_color_format(ufvc_ctx* ctx, int format) {
    if (!ctx || format < UFVC_COLOR_RGB || format > UFVC_COLOR_YUV420P)
        return fail(ctx, UFVC_ERR_ARG, "set_color_format: unknown format");
    ctx->color = format;
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_set_progressive_means(ufvc_ctx* ctx, const float* weights, size_t n_weights) {
    if (!ctx || !weights) return fail(ctx, UFVC_ERR_ARG, "set_progressive_means: bad argument");
    if (ctx->borrowed) return fail(ctx, UFVC_ERR_ARG, "set_progressive_means: context shares another's weights");
    if (ctx->pm_on) return fail(ctx, UFVC_ERR_ARG, "set_progressive_means: already set");
    if (n_weights != mean_weight_count(ctx->cfg.arch)) return fail(ctx, UFVC_ERR_ARG, "set_progressive_means: weight count");
    CK(cudaSetDevice(ctx->cfg.device));
    size_t offs[kMeanLayers], off = 0;
    for (int l = 0; l < kMeanLayers; ++l) {
        int sh[3];
        mean_layer_shape(ctx->cfg.arch, l, &sh[0], &sh[1], &sh[2]);
        offs[l] = off;
        off += (size_t)sh[0] * sh[1] * sh[1] * sh[2] + sh[0];
    }
    for (int l = 0; l < kMeanLayers; ++l) {
        int sh[3];
        mean_layer_shape(ctx->cfg.arch, l, &sh[0], &sh[1], &sh[2]);
        ufvc_status st = upload_layer(ctx, ctx->pm[l], weights, offs, l, 1, true, false, false, sh, true);
        if (st != UFVC_OK) return st;
    }
    ctx->pm_on = true;
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_progressive_means(ufvc_ctx* ctx, const float* d_y, const int16_t* d_rhat_in,
                                              const float* d_mu0, const float* d_s, int Hy, int Wy, int qp,
                                              int16_t* d_rhat, float* d_mu, float* d_yhat, void* stream) {
    if (!ctx || !d_mu0 || !d_s || !d_rhat || !d_mu || !d_yhat || (!d_y && !d_rhat_in) || Hy < 1 || Wy < 1 || qp < 0 ||
        qp > 63)
        return fail(ctx, UFVC_ERR_ARG, "progressive_means: bad argument");
    if (!ctx->pm_on) return fail(ctx, UFVC_ERR_ARG, "progressive_means: no mean network (ufvc_set_progressive_means)");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->cfg.device));
    const Arch& a = ctx->arch;
    Plan tmp;
    tmp.Hy = Hy; tmp.Wy = Wy;
    const size_t ny = (size_t)Hy * Wy * a.cy;
    int* qpd = nullptr;
    ufvc_status st;
    if ((st = pm_buffers(ctx, &tmp, true, nullptr)) || (st = dalloc(ctx, &tmp, &qpd, 1))) {
        for (void* v : tmp.allocs) cudaFree(v);
        return st;
    }
    ctx->cur_ws = &ctx->ws_stage;
    cudaError_t e = cudaMemcpyAsync(d_mu, d_mu0, ny * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && !d_y) e = cudaMemcpyAsync(d_rhat, d_rhat_in, ny * 2, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(qpd, &qp, 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        st = run_progressive(ctx, Hy, Wy, d_y, d_rhat, d_mu, d_s, nullptr, qp, nullptr, tmp.pm_in_e, tmp.pm_h_e,
                             tmp.pm_mu_e, s);
        if (st == UFVC_OK) launch_dequant(d_rhat, d_mu, ny, ctx->d_qstep, qpd, d_yhat, nullptr, s);
        e = cudaStreamSynchronize(s);
    }
    for (void* v : tmp.allocs) cudaFree(v);
    if (st) return st;
    if (e != cudaSuccess) return fail(ctx, UFVC_ERR_CUDA, cudaGetErrorString(e));
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_quantize(ufvc_ctx* ctx, const float* d_y, const float* d_mu, const float* d_logsig,
                                     size_t n, int qp, int16_t* d_rhat, uint8_t* d_idx, void* stream) {
    if (!ctx || !d_y || !d_mu || !d_logsig || !d_rhat || !d_idx || qp < 0 || qp > 63)
        return fail(ctx, UFVC_ERR_ARG, "quantize: bad argument");
    CK(cudaSetDevice(ctx->cfg.device));
    if (n) launch_quantize(d_y, d_mu, d_logsig, n, ctx->d_thr, ctx->d_qinv, nullptr, qp, d_rhat, d_idx, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_synthesize(ufvc_ctx* ctx, const float* d_yhat, int width, int height, float* d_frames,
                                       void* stream) {
    if (!ctx || !d_yhat || !d_frames || !check_shape(ctx, ctx->N, width, height))
        return fail(ctx, UFVC_ERR_ARG, "synthesize: bad argument");
    if (fp8_unready(ctx)) return fail(ctx, UFVC_ERR_ARG, "synthesize: FP8 context not calibrated (ufvc_calibrate_fp8)");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->cfg.device));
    Plan* p;
    ufvc_status st = get_plan(ctx, width, height, true, &p);
    if (st) return st;

    ctx->cur_ws = &p->ws_dec;
    if (ctx->cfg.precision == UFVC_FP32) {
        RUN(run_decoders(ctx, p, d_yhat, d_frames, OUT_PS_FINAL_F32, s));
    } else {
        if (ctx->cfg.precision == UFVC_FP8)
            launch_f32_to_e4m3_rows(d_yhat, p->Hy, p->Wy, ctx->arch.cy, 1.f / ctx->act_scale[T_YHAT],
                                    reinterpret_cast<uint8_t*>(p->yhat_bf), p->Wy, s);
        else
            launch_f32_to_bf16(d_yhat, p->ny, p->yhat_bf, s);
        RUN(run_decoders(ctx, p, p->yhat_bf, d_frames, OUT_PS_FINAL_F32, s));
    }
    CK(cudaGetLastError());
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_conv_layer(ufvc_ctx* ctx, int layer, const void* d_in, int H, int W, int stride, int act,
                                       int mode, void* d_out, int out_h, int out_w, void* stream) {
    if (!ctx || !d_in || !d_out || layer < 0 || layer >= L_NENC + D_NDEC * ctx->N || H < 1 || W < 1 ||
        (stride != 1 && stride != 2) || mode < 0 || mode > 3 || out_h < 1 || out_w < 1)
        return fail(ctx, UFVC_ERR_ARG, "conv_layer: bad argument");
    if (fp8_unready(ctx)) return fail(ctx, UFVC_ERR_ARG, "conv_layer: FP8 context not calibrated (ufvc_calibrate_fp8)");
    CK(cudaSetDevice(ctx->cfg.device));
    LayerW L;
    int g = 0;
    if (layer < L_NENC) {
        L = ctx->enc[layer];
    } else {
        g = (layer - L_NENC) / D_NDEC;
        L = ctx->dec[(layer - L_NENC) % D_NDEC];
        L.w += g * L.w_gs;
        L.b += g * L.b_gs;
        if (L.wtc) L.wtc += (size_t)g * L.cout_pad * L.k * L.k * L.cin_tc;
        if (L.btc) L.btc += g * L.b_gs;
        if (L.wsc) L.wsc += (size_t)g * 128 * 64;
        if (L.w8) L.w8 += (size_t)g * L.cout_pad * L.k * L.k * L.cin_tc;
        if (L.cs8) L.cs8 += g * L.b_gs;
    }
    L.groups = 1;
    const int m = (mode == 0 || mode == 3) ? OUT_NHWC : mode == 1 ? OUT_PS : OUT_PS_FINAL_F32;
    if (use_tc(ctx, L) && L.ps_major && m != OUT_PS)
        return fail(ctx, UFVC_ERR_ARG, "conv_layer: this layer's tensor-core weights are laid out for pixel shuffle");
    ctx->cur_ws = &ctx->ws_stage;
    RUN(conv(ctx, L, d_in, H, W, stride, act, m, d_out, out_h, out_w, (cudaStream_t)stream,
             mode == 3 ? d_out : nullptr));  // mode 3: the residual is d_out's content, updated in place
    CK(cudaGetLastError());
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_set_conv_pairs(ufvc_ctx* ctx, int enable) {
    if (!ctx || (enable != 0 && enable != 1)) return fail(ctx, UFVC_ERR_ARG, "set_conv_pairs: bad argument");
    ctx->conv_pairs = enable;
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_set_table_wait_limit(ufvc_ctx* ctx, long long cycles) {
    if (!ctx || cycles < 0) return fail(ctx, UFVC_ERR_ARG, "set_table_wait_limit: bad argument");
    ctx->table_spin = cycles;
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_first_layer(ufvc_ctx* ctx, const uint8_t* d_frames, int width, int height, int kernel,
                                        void* d_out, void* stream) {
    if (!ctx || !d_frames || !d_out || width < 1 || height < 1 || width > 65535 || height > 65535 || kernel < 0 ||
        kernel > 2)
        return fail(ctx, UFVC_ERR_ARG, "first_layer: bad argument");
    if (!ctx->first_w || ctx->color == UFVC_COLOR_RGB_BT709)
        return fail(ctx, UFVC_ERR_UNSUPPORTED,
                    "first_layer: this context's first layer does not read frame bytes (needs BF16 or FP8, an even "
                    "chunk length of at most 8 and colour format RGB, YUV444P or YUV420P)");
    if (kernel == 2 && !first_layer_tma_ok(ctx->color, width, d_frames))
        return fail(ctx, UFVC_ERR_ARG,
                    "first_layer: the TMA kernel needs interleaved RGB frames with rows of a multiple of 16 bytes "
                    "at a 16-byte aligned address");
    CK(cudaSetDevice(ctx->cfg.device));
    const int Ho = conv_out(ceil_div(height, 16) * 16, 3, 2), Wo = conv_out(ceil_div(width, 16) * 16, 3, 2);
    CK(launch_first_layer(d_frames, ctx->color, ctx->N, height, width, Ho, Wo, ctx->first_w, ctx->enc[L_A1].b, d_out,
                          0.f, ctx->d_status, (cudaStream_t)stream, kernel));
    CK(cudaGetLastError());
    return UFVC_OK;
}

static ufvc_status ensure_rans_scratch(ufvc_ctx* ctx, size_t words) {
    if (words > ctx->r_scr_words) {
        cudaFree(ctx->r_scr);
        ctx->r_scr = nullptr;
        ufvc_status st = dalloc(ctx, nullptr, &ctx->r_scr, words);
        if (st) return st;
        ctx->r_scr_words = words;
    }
    if (!ctx->r_ctl) {
        ufvc_status st = dalloc(ctx, nullptr, &ctx->r_ctl, 1);
        if (st) return st;
        if (cudaMemset(ctx->r_ctl, 0, sizeof(RansCtl)) != cudaSuccess) return UFVC_ERR_CUDA;
    }
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_rans_encode(ufvc_ctx* ctx, const int16_t* d_sym, const uint8_t* d_idx, size_t n, int lanes,
                                        uint8_t* d_out, size_t capacity, uint64_t* d_nbytes, void* stream) {
    if (!ctx || (!d_sym && n) || (!d_idx && n) || !d_out || !d_nbytes || lanes < 1 || lanes > 65536 ||
        n > 0x7FFFFFFFull)
        return fail(ctx, UFVC_ERR_ARG, "rans_encode: bad argument");
    CK(cudaSetDevice(ctx->cfg.device));
    const int cap_lane = (int)(n / lanes + 3);
    ufvc_status st = ensure_rans_scratch(ctx, (size_t)lanes * cap_lane);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    RansEncJob j{};
    j.s[0] = RansEncSec{d_sym, d_idx, 0, (uint32_t)n, lanes, ctx->r_scr, cap_lane, 0};
    j.nsec = 1;
    j.st[0].out = d_out;
    j.st[0].capacity = capacity;
    j.st[0].nbytes = d_nbytes;
    j.nstreams = 1;
    j.ctl = ctx->r_ctl;
    j.status = ctx->d_status;
    j.spin = ctx->table_spin;
    prof_begin(ctx, "rans_encode", s);
    CK(launch_rans_encode(j, ctx->d_packed, s));
    prof_end(ctx, s, 1);
    CK(cudaGetLastError());
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_rans_decode(ufvc_ctx* ctx, const uint8_t* d_in, size_t nbytes, const uint8_t* d_idx,
                                        size_t n, int lanes, int16_t* d_sym, void* stream) {
    if (!ctx || !d_in || (!d_idx && n) || (!d_sym && n) || lanes < 1 || lanes > 65536 || n > 0x7FFFFFFFull)
        return fail(ctx, UFVC_ERR_ARG, "rans_decode: bad argument");
    CK(cudaSetDevice(ctx->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    RansDecJob j{};
    j.s[0].bits = d_in;
    j.s[0].nbytes = nbytes;
    j.s[0].idx = d_idx;
    j.s[0].sym = d_sym;
    j.nsec = 1;
    j.n = (uint32_t)n;
    j.K = lanes;
    j.out = kDecSym;
    j.status = ctx->d_status;
    j.spin = ctx->table_spin;
    prof_begin(ctx, "rans_decode", s);
    CK(launch_rans_decode(j, ctx->d_dec, s));
    prof_end(ctx, s, 1);
    CK(cudaGetLastError());
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_get_tables(const ufvc_ctx* ctx, uint32_t* freq, uint32_t* cum, int qp, float* thr) {
    if (qp < 0 || qp > 63) return UFVC_ERR_ARG;
    HostTables local;
    if (!ctx) build_host_tables(local);  // no context: build on the host, no device involved
    const HostTables& t = ctx ? ctx->tabs : local;
    if (freq) memcpy(freq, t.freq.data(), t.freq.size() * 4);
    if (cum) memcpy(cum, t.cum.data(), t.cum.size() * 4);
    if (thr) memcpy(thr, &t.thr[qp * (kBins - 1)], (kBins - 1) * 4);
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_set_profiling(ufvc_ctx* ctx, int enable) {
    if (!ctx) return UFVC_ERR_ARG;
    ctx->prof_on = enable != 0;

    return UFVC_OK;
}

extern "C" ufvc_status ufvc_get_profile(ufvc_ctx* ctx, char* names, float* ms, int* launches, int max, int* count) {
    if (!ctx || !count) return UFVC_ERR_ARG;
    int n = 0;
    for (size_t i = 0; i < ctx->prof_n && n < max; ++i, ++n) {
        ProfEntry& e = ctx->prof[i];
        CK(cudaEventSynchronize(e.b));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, e.a, e.b));
        if (names) snprintf(names + 32 * n, 32, "%s", e.name);
        if (ms) ms[n] = t;
        if (launches) launches[n] = e.launches;
    }
    *count = n;
    ctx->prof_n = 0;  // entries accumulate over calls until read
    return UFVC_OK;
}

// ------------------------------------------------------------------------------------------------
// read-only access to context internals for other translation units of the library
// ------------------------------------------------------------------------------------------------
namespace ufvc {
const uint32_t* ctx_packed_tables(const ufvc_ctx* c) { return c->d_packed; }
long long ctx_table_spin(const ufvc_ctx* c) { return c->table_spin; }
bool ctx_temporal(const ufvc_ctx* c) { return c->tc_on; }
int* ctx_status_word(ufvc_ctx* c) { return c->d_status; }
int ctx_device(const ufvc_ctx* c) { return c->cfg.device; }
void ctx_set_error(ufvc_ctx* c, const char* msg) { c->err = msg; }
}  // namespace ufvc

// FP8 layer roles: input, output (-1: bf16 / float output) and residual activation tensors
static void fp8_roles(bool enc, int l, int* tin, int* tout, int* tres) {
    static const int E[L_NENC][3] = {{T_X, T_A1, -1},  {T_A1, T_A2, -1}, {T_A2, T_A3, -1}, {T_A3, T_XT, -1},
                                     {T_XT, T_A3R, T_A3}, {T_A3R, -1, -1}, {T_Y, T_HB, -1},  {T_HB, -1, -1},
                                     {-1, -1, -1},      {-1, -1, -1},     {-1, -1, -1}};
    static const int D[D_NDEC][3] = {{T_YHAT, T_D0, -1}, {T_D0, T_R1A, -1}, {T_R1A, T_R1B, T_D0}, {T_R1B, T_U1, -1},
                                     {T_U1, T_R2A, -1},  {T_R2A, T_R2B, T_U1}, {T_R2B, -1, -1},   {-1, -1, -1}};
    const int* r = enc ? E[l] : D[l];
    *tin = r[0]; *tout = r[1]; *tres = r[2];
}

extern "C" ufvc_status ufvc_calibrate_fp8(ufvc_ctx* ctx, const uint8_t* d_frames, int n_frames, int width,
                                          int height, int qp, void* stream) {
    if (!ctx || !d_frames || !check_shape(ctx, n_frames, width, height) || qp < 0 || qp > 63)
        return fail(ctx, UFVC_ERR_ARG, "calibrate_fp8: bad argument");
    if (ctx->cfg.precision != UFVC_FP8) return fail(ctx, UFVC_ERR_ARG, "calibrate_fp8: not an FP8 context");
    CK(cudaSetDevice(ctx->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    // the FP32 path of the same weights (a clone sharing them) codes the chunk and records the maxima
    ufvc_ctx* c = ctx_clone_shared(ctx);
    if (!c) return fail(ctx, UFVC_ERR_OOM, "calibrate_fp8: context clone failed");
    c->cfg.precision = UFVC_FP32;
    // the frame-byte A1 kernel and the space-to-depth A1 write bf16 / E4M3 activations: the FP32 run takes
    // the packed input and A1's FP32 weights instead
    c->first_w = nullptr;
    c->a1s2d = LayerW{};
    const size_t cap = ufvc_max_bitstream_bytes(ctx, width, height);
    uint8_t *bits = nullptr, *out = nullptr;
    uint64_t* nb = nullptr;
    ufvc_status st = UFVC_OK;
    float amax[T_NT] = {};
    if (cudaMalloc(&c->amax, T_NT * sizeof(float)) != cudaSuccess || cudaMemset(c->amax, 0, T_NT * 4) != cudaSuccess ||
        cudaMalloc(&bits, cap) != cudaSuccess || cudaMalloc(&nb, 8) != cudaSuccess ||
        cudaMalloc(&out, (size_t)n_frames * width * height * 3) != cudaSuccess) {
        cudaGetLastError();
        st = UFVC_ERR_OOM;
    }
    if (st == UFVC_OK) st = ufvc_encode_chunk(c, d_frames, n_frames, width, height, qp, bits, cap, nb, stream);
    if (st == UFVC_OK) st = ufvc_sync_status(c, stream);
    uint64_t n = 0;
    if (st == UFVC_OK && cudaMemcpy(&n, nb, 8, cudaMemcpyDeviceToHost) != cudaSuccess) st = UFVC_ERR_CUDA;
    if (st == UFVC_OK) st = ufvc_decode_chunk(c, bits, n, out, n_frames, width, height, stream);
    if (st == UFVC_OK) st = ufvc_sync_status(c, stream);
    if (st == UFVC_OK && cudaMemcpy(amax, c->amax, sizeof(amax), cudaMemcpyDeviceToHost) != cudaSuccess)
        st = UFVC_ERR_CUDA;
    if (st != UFVC_OK) ctx->err = std::string("calibrate_fp8: FP32 run failed: ") + c->err;
    cudaFree(c->amax);
    c->amax = nullptr;
    cudaFree(bits);
    cudaFree(nb);
    cudaFree(out);
    ufvc_destroy(c);
    (void)s;
    if (st != UFVC_OK) return st;
    for (int t = 0; t < T_NT; ++t) ctx->act_scale[t] = amax[t] > 0.f ? amax[t] / 448.f : 1.f / 448.f;
    ctx->act_scale[T_X] = 1.f / 448.f;
    // per-layer accumulator scales and output / residual scales
    for (int pass = 0; pass < 2; ++pass) {
        const int nl = pass == 0 ? L_NENC : D_NDEC;
        for (int l = 0; l < nl; ++l) {
            LayerW& L = pass == 0 ? ctx->enc[l] : ctx->dec[l];
            if (!L.w8) continue;
            int tin, tout, tres;
            fp8_roles(pass == 0, l, &tin, &tout, &tres);
            std::vector<float> cs(L.wscale.size());
            for (size_t i = 0; i < cs.size(); ++i) cs[i] = ctx->act_scale[tin] * L.wscale[i];
            CK(cudaMemcpy(L.cs8, cs.data(), cs.size() * 4, cudaMemcpyHostToDevice));
            L.out_inv = tout >= 0 ? 1.f / ctx->act_scale[tout] : 0.f;
            L.res_s = tres >= 0 ? ctx->act_scale[tres] : 0.f;
        }
    }
    ctx->fp8_ready = true;
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_get_fp8_scales(const ufvc_ctx* ctx, float* act_scales, int n) {
    if (!ctx || !act_scales || n < (int)T_NT || ctx->cfg.precision != UFVC_FP8 || !ctx->fp8_ready) return UFVC_ERR_ARG;
    for (int t = 0; t < T_NT; ++t) act_scales[t] = ctx->act_scale[t];
    return UFVC_OK;
}
