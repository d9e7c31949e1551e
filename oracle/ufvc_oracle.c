/*
 * ufvc_oracle.c -- plain, slow, FP64 CPU oracle of the chunk-coding path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code, header, table or constant generator with the CUDA library:
 * everything here is written out again from the paper and from the readings listed below.
 *
 * What it follows (paper "Ultra-Fast Neural Video Compression"):
 *   Sec. 3.1 (Overview, Fig. 3): a chunk X_i of N frames is patch-embedded, encoded into ONE latent y_i,
 *     quantised to y^_i, converted into a bit-stream, parsed back and decoded; qp_i sets the rate.
 *   Sec. 3.2: N frame-specific decoders, one per temporal position, reconstruct all frames in parallel.
 *   Sec. 3.4 (Fig. 4c): r^ = round(y - mu), coded with the scale sigma only; y^ = r^ + mu; the scales of
 *     ALL latent elements come from one parameter-estimation pass, so the whole latent is entropy
 *     coded in a single step.
 * The paper shows the module internals only in figures.  The plain architecture used here (strided
 * 3x3 convs + GELU, one residual cross-frame interaction block, a 2-layer hyper-analysis, a 3-layer
 * hyper-synthesis emitting (mu, log sigma), and conv/residual/pixel-shuffle decoders) and every
 * numeric convention (scale bins, CDF construction, rANS parameters, bit-stream layout) are the
 * readings stated beside each function.
 *
 * Precision: all convolutions, GELU and hyper-synthesis in FP64 with the float32 weights promoted to
 * double; CDF tables built in FP64 with libm erf/erfc; rANS in exact integers.
 *
 * Parity status of each function: pinned by tests under tests/ (brute force, closed forms, library
 * cross-checks, exact bit counts), except the rate-distortion behaviour of the random-weight codec,
 * which no published value can pin ("parity unpinned": random weights have no meaningful R-D).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_CAPACITY 2
#define ORC_ERR_CORRUPT 3
#define ORC_ERR_OOM 4

#define NBINS 64          /* scale bins */
#define RMAX 255          /* |r^| <= 255 */
#define NSYM 511          /* symbols -255..255 */
#define PROB_BITS 16
#define PROB_M (1u << PROB_BITS)
#define RANS_L (1u << 16) /* lower bound of the 32-bit rANS state */
#define ORC_CF 64         /* temporal chunk feature channels */
#define ORC_CC 64         /* temporal context channels */
/* DC-block model widths: chunk modules, frame decoders, context, latent, hyper-latent */
#define DC_C 512
#define DC_CF 256
#define DC_CC 128
#define DC_CY 256
#define DC_CZ 128

/* ------------------------------------------------------------------------------------------------ */
/* Architecture (plain reading of Fig. 3; widths per workload)                                      */
/* ------------------------------------------------------------------------------------------------ */
typedef struct { int e0, e1, e2, cy, cz, cd1, cd2; } arch_t;

static int get_arch(int arch, arch_t* a) {
    if (arch == 0) { arch_t t = {64, 96, 128, 128, 64, 128, 64}; *a = t; return ORC_OK; }
    if (arch == 1) { arch_t t = {64, 128, 192, 256, 128, 128, 64}; *a = t; return ORC_OK; }
    if (arch == 2) { arch_t t = {0, 0, 0, 256, 128, 0, 0}; *a = t; return ORC_OK; }  /* DC-block model */
    return ORC_ERR_ARG;
}

static int dc_hyper_layer(int l);  /* DC-block model: blob index of hyperprior layer l = 6..10 */
static void dc_layer_ptr(int N, const float* blob, int l, const float** w, const float** b);
size_t orc_dc_weight_count(int N);

/* Layer l of the blob: (cout, k, cin).  Encoder/hyper layers 0..10, then 8 per frame. */
int orc_layer_shape(int arch, int N, int l, int* cout, int* k, int* cin) {
    arch_t a;
    if (arch == 2 || get_arch(arch, &a) || N < 1 || l < 0 || l >= 11 + 8 * N) return ORC_ERR_ARG;
    int t[11][3] = {{a.e0, 3, 3 * N}, {a.e1, 3, a.e0}, {a.e2, 3, a.e1}, {a.e2, 3, a.e2}, {a.e2, 1, a.e2},
                    {a.cy, 3, a.e2},  {a.cz, 3, a.cy}, {a.cz, 3, a.cz}, {4 * a.cz, 3, a.cz},
                    {4 * a.cz, 3, a.cz}, {2 * a.cy, 1, a.cz}};
    int d[8][3] = {{4 * a.cd1, 3, a.cy}, {a.cd1, 3, a.cd1}, {a.cd1, 3, a.cd1}, {4 * a.cd2, 3, a.cd1},
                   {a.cd2, 3, a.cd2},    {a.cd2, 3, a.cd2}, {4 * a.cd2, 3, a.cd2}, {12, 3, a.cd2}};
    const int* r = (l < 11) ? t[l] : d[(l - 11) % 8];
    *cout = r[0]; *k = r[1]; *cin = r[2];
    return ORC_OK;
}

size_t orc_weight_count(int arch, int N) {
    if (arch == 2) return orc_dc_weight_count(N);
    size_t n = 0;
    int co, k, ci;
    for (int l = 0; l < 11 + 8 * N; l++) {
        if (orc_layer_shape(arch, N, l, &co, &k, &ci)) return 0;
        n += (size_t)co * k * k * ci + co;
    }
    return n;
}

/* Pointers to layer l's kernel [Cout][k][k][Cin] and bias [Cout] inside the blob. */
static void layer_ptr(int arch, int N, const float* blob, int l, const float** w, const float** b) {
    if (arch == 2) { dc_layer_ptr(N, blob, dc_hyper_layer(l), w, b); return; }  /* hyperprior layers only */
    size_t off = 0;
    int co, k, ci;
    for (int i = 0; i < l; i++) {
        orc_layer_shape(arch, N, i, &co, &k, &ci);
        off += (size_t)co * k * k * ci + co;
    }
    orc_layer_shape(arch, N, l, &co, &k, &ci);
    *w = blob + off;
    *b = blob + off + (size_t)co * k * k * ci;
}

/* ------------------------------------------------------------------------------------------------ */
/* Network primitives                                                                               */
/* ------------------------------------------------------------------------------------------------ */

/* 2-D convolution, NHWC, zero padding k/2, stride s:
 *   out[oh][ow][co] = b[co] + sum_{ky,kx,ci} w[co][ky][kx][ci] * in[oh*s+ky-k/2][ow*s+kx-k/2][ci]
 * (terms outside the input are zero).  Ho = (H + 2*(k/2) - k)/s + 1. */
void orc_conv2d(const double* in, int H, int W, int Cin, const float* w, const float* b, int Cout, int k,
                int s, double* out) {
    int p = k / 2;
    int Ho = (H + 2 * p - k) / s + 1, Wo = (W + 2 * p - k) / s + 1;
    double* wd = (double*)malloc(sizeof(double) * (size_t)Cout * k * k * Cin);
    for (size_t i = 0; i < (size_t)Cout * k * k * Cin; i++) wd[i] = (double)w[i];
#pragma omp parallel for collapse(2) schedule(static)
    for (int oh = 0; oh < Ho; oh++)
        for (int ow = 0; ow < Wo; ow++) {
            double* o = out + ((size_t)oh * Wo + ow) * Cout;
            for (int co = 0; co < Cout; co++) {
                double acc = (double)b[co];
                for (int ky = 0; ky < k; ky++) {
                    int ih = oh * s + ky - p;
                    if (ih < 0 || ih >= H) continue;
                    for (int kx = 0; kx < k; kx++) {
                        int iw = ow * s + kx - p;
                        if (iw < 0 || iw >= W) continue;
                        const double* x = in + ((size_t)ih * W + iw) * Cin;
                        const double* wk = wd + (((size_t)co * k + ky) * k + kx) * Cin;
                        for (int ci = 0; ci < Cin; ci++) acc += wk[ci] * x[ci];
                    }
                }
                o[co] = acc;
            }
        }
    free(wd);
}

/* GELU, exact erf form: x * Phi(x) = 0.5 x (1 + erf(x / sqrt 2)). */
double orc_gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }

static void gelu_inplace(double* x, size_t n) {
    for (size_t i = 0; i < n; i++) x[i] = orc_gelu(x[i]);
}

/* Pixel shuffle x2 (NHWC): out[2h+dy][2w+dx][c] = in[h][w][4c + 2dy + dx]; in has 4C channels. */
void orc_pixel_shuffle(const double* in, int H, int W, int C, double* out) {
    for (int h = 0; h < H; h++)
        for (int w = 0; w < W; w++)
            for (int c = 0; c < C; c++)
                for (int dy = 0; dy < 2; dy++)
                    for (int dx = 0; dx < 2; dx++)
                        out[(((size_t)(2 * h + dy)) * (2 * W) + (2 * w + dx)) * C + c] =
                            in[((size_t)h * W + w) * 4 * C + 4 * c + 2 * dy + dx];
}

static double* dalloc(size_t n) { return (double*)calloc(n ? n : 1, sizeof(double)); }
static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

static int conv_out(int x, int k, int s) { return (x + 2 * (k / 2) - k) / s + 1; }

/* ------------------------------------------------------------------------------------------------ */
/* Analysis (patchify + chunk encoder + cross-frame interaction), Sec. 3.1, Fig. 3                 */
/* ------------------------------------------------------------------------------------------------ */

/* ------------------------------------------------------------------------------------------------ */
/* Colour interface (Appendix: YUV444 is the model's input and output; RGB and YUV420 are converted)   */
/* ------------------------------------------------------------------------------------------------ */
/* Formats: 0 = RGB u8 interleaved [N][H][W][3], the channels fed to the network as they are;
 * 1 = RGB u8 interleaved, converted to YUV444 with BT.709 (full range, chroma centred at 0.5) before the
 *     network and back after it;  2 = YUV444 u8 planar [N][3][H][W];  3 = YUV420 u8 planar per frame
 *     (Y [H][W], then U and V [ceil(H/2)][ceil(W/2)]), chroma replicated over its 2x2 block on input
 *     and averaged over the block's pixels inside the frame on output.
 * BT.709 on [0, 1] values: Y = 0.2126 R + 0.7152 G + 0.0722 B, U = (B - Y) / 1.8556 + 0.5,
 * V = (R - Y) / 1.5748 + 0.5; inverse R = Y + 1.5748 (V - 0.5), B = Y + 1.8556 (U - 0.5),
 * G = (Y - 0.2126 R - 0.0722 B) / 0.7152. */
size_t orc_frame_bytes(int fmt, int H, int W) {
    if (fmt == 3) return (size_t)H * W + 2 * (size_t)((H + 1) / 2) * ((W + 1) / 2);
    return (size_t)3 * H * W;
}

static void bt709_fwd(double r, double g, double b, double* o) {
    double y = 0.2126 * r + 0.7152 * g + 0.0722 * b;
    o[0] = y;
    o[1] = (b - y) / 1.8556 + 0.5;
    o[2] = (r - y) / 1.5748 + 0.5;
}

static void bt709_inv(const double* yuv, double* rgb) {
    double r = yuv[0] + 1.5748 * (yuv[2] - 0.5);
    double b = yuv[0] + 1.8556 * (yuv[1] - 0.5);
    rgb[0] = r;
    rgb[1] = (yuv[0] - 0.2126 * r - 0.0722 * b) / 0.7152;
    rgb[2] = b;
}

/* Caller's frames -> the network's channels in [0, 1]: x [N][H][W][3]. */
int orc_color_in(int fmt, const uint8_t* frames, int N, int H, int W, double* x) {
    if (fmt < 0 || fmt > 3 || N < 1 || H < 1 || W < 1) return ORC_ERR_ARG;
    const size_t fb = orc_frame_bytes(fmt, H, W);
    const int Wc = (W + 1) / 2, Hc = (H + 1) / 2;
    for (int n = 0; n < N; n++) {
        const uint8_t* f = frames + n * fb;
        for (int h = 0; h < H; h++)
            for (int w = 0; w < W; w++) {
                double* o = x + (((size_t)n * H + h) * W + w) * 3;
                const size_t i = (size_t)h * W + w;
                if (fmt == 0 || fmt == 1) {
                    double r = f[3 * i] / 255.0, g = f[3 * i + 1] / 255.0, b = f[3 * i + 2] / 255.0;
                    if (fmt == 0) { o[0] = r; o[1] = g; o[2] = b; }
                    else bt709_fwd(r, g, b, o);
                } else if (fmt == 2) {
                    for (int c = 0; c < 3; c++) o[c] = f[(size_t)c * H * W + i] / 255.0;
                } else {
                    const size_t ci = (size_t)(h / 2) * Wc + w / 2;
                    o[0] = f[i] / 255.0;
                    o[1] = f[(size_t)H * W + ci] / 255.0;
                    o[2] = f[(size_t)H * W + (size_t)Hc * Wc + ci] / 255.0;
                }
            }
    }
    return ORC_OK;
}

/* The network's reconstruction x [N][H][W][3] (already clamped to [0, 1]) -> the caller's format, as
 * values in [0, 1] laid out like the format's bytes (out: N * frame_bytes doubles).  BT.709 results are
 * clamped to [0, 1] again; YUV420 chroma is the mean of the 2x2 block's pixels that lie in the frame. */
int orc_color_out(int fmt, const double* x, int N, int H, int W, double* out) {
    if (fmt < 0 || fmt > 3 || N < 1 || H < 1 || W < 1) return ORC_ERR_ARG;
    const size_t fb = orc_frame_bytes(fmt, H, W);
    const int Wc = (W + 1) / 2, Hc = (H + 1) / 2;
    for (int n = 0; n < N; n++) {
        double* f = out + n * fb;
        const double* xf = x + (size_t)n * H * W * 3;
        if (fmt == 3) {
            for (size_t i = 0; i < (size_t)H * W; i++) f[i] = xf[3 * i];
            for (int hc = 0; hc < Hc; hc++)
                for (int wc = 0; wc < Wc; wc++)
                    for (int c = 1; c < 3; c++) {
                        double s = 0.0;
                        int cnt = 0;
                        for (int dy = 0; dy < 2; dy++)
                            for (int dx = 0; dx < 2; dx++) {
                                int h = 2 * hc + dy, w = 2 * wc + dx;
                                if (h < H && w < W) { s += xf[((size_t)h * W + w) * 3 + c]; cnt++; }
                            }
                        f[(size_t)H * W + (size_t)(c - 1) * Hc * Wc + (size_t)hc * Wc + wc] = s / cnt;
                    }
            continue;
        }
        for (size_t i = 0; i < (size_t)H * W; i++) {
            const double* v = xf + 3 * i;
            if (fmt == 0) { f[3 * i] = v[0]; f[3 * i + 1] = v[1]; f[3 * i + 2] = v[2]; }
            else if (fmt == 1) {
                double rgb[3];
                bt709_inv(v, rgb);
                for (int c = 0; c < 3; c++) f[3 * i + c] = clampd(rgb[c], 0.0, 1.0);
            } else {
                for (int c = 0; c < 3; c++) f[(size_t)c * H * W + i] = v[c];
            }
        }
    }
    return ORC_OK;
}

/* Chunk -> latent y [Hy][Wy][Cy] from the network's input channels x [N][H][W][3] in [0, 1]: frame n
 * -> channels 3n..3n+2, replicate-padded to multiples of 16.  Then A1..A3 (3x3 stride 2 + GELU), the
 * interaction block h + Xb(GELU(Xa(h))), A4 (3x3 stride 2). */
static int analysis_core(int arch, int N, const double* xin, int H, int W, const float* wts, const double* add_h3,
                         double* y);

int orc_analysis_x(int arch, int N, const double* xin, int H, int W, const float* wts, double* y) {
    return analysis_core(arch, N, xin, H, W, wts, NULL, y);
}

/* add_h3 (optional, [H/8][W/8][e2] of the padded size): added to the A3 output before the interaction
 * block (the temporal-context conditioning of the chunk encoder). */
static int analysis_core(int arch, int N, const double* xin, int H, int W, const float* wts, const double* add_h3,
                         double* y) {
    arch_t a;
    if (get_arch(arch, &a) || N < 1 || H < 1 || W < 1) return ORC_ERR_ARG;
    int Hp = (H + 15) / 16 * 16, Wp = (W + 15) / 16 * 16, C0 = 3 * N;
    double* x = dalloc((size_t)Hp * Wp * C0);
    for (int h = 0; h < Hp; h++)
        for (int w = 0; w < Wp; w++)
            for (int n = 0; n < N; n++)
                for (int c = 0; c < 3; c++) {
                    int sh = h < H ? h : H - 1, sw = w < W ? w : W - 1;
                    x[((size_t)h * Wp + w) * C0 + 3 * n + c] = xin[(((size_t)n * H + sh) * W + sw) * 3 + c];
                }
    const float *wk, *bk;
    int h1 = conv_out(Hp, 3, 2), w1 = conv_out(Wp, 3, 2);
    double* t1 = dalloc((size_t)h1 * w1 * a.e0);
    layer_ptr(arch, N, wts, 0, &wk, &bk);
    orc_conv2d(x, Hp, Wp, C0, wk, bk, a.e0, 3, 2, t1);
    gelu_inplace(t1, (size_t)h1 * w1 * a.e0);
    int h2 = conv_out(h1, 3, 2), w2 = conv_out(w1, 3, 2);
    double* t2 = dalloc((size_t)h2 * w2 * a.e1);
    layer_ptr(arch, N, wts, 1, &wk, &bk);
    orc_conv2d(t1, h1, w1, a.e0, wk, bk, a.e1, 3, 2, t2);
    gelu_inplace(t2, (size_t)h2 * w2 * a.e1);
    int h3 = conv_out(h2, 3, 2), w3 = conv_out(w2, 3, 2);
    size_t n3 = (size_t)h3 * w3 * a.e2;
    double* t3 = dalloc(n3);
    layer_ptr(arch, N, wts, 2, &wk, &bk);
    orc_conv2d(t2, h2, w2, a.e1, wk, bk, a.e2, 3, 2, t3);
    gelu_inplace(t3, n3);
    if (add_h3)
        for (size_t i = 0; i < n3; i++) t3[i] += add_h3[i];
    /* cross-frame interaction: h + Xb(GELU(Xa(h))) */
    double* u = dalloc(n3);
    double* v = dalloc(n3);
    layer_ptr(arch, N, wts, 3, &wk, &bk);
    orc_conv2d(t3, h3, w3, a.e2, wk, bk, a.e2, 3, 1, u);
    gelu_inplace(u, n3);
    layer_ptr(arch, N, wts, 4, &wk, &bk);
    orc_conv2d(u, h3, w3, a.e2, wk, bk, a.e2, 1, 1, v);
    for (size_t i = 0; i < n3; i++) t3[i] += v[i];
    layer_ptr(arch, N, wts, 5, &wk, &bk);
    orc_conv2d(t3, h3, w3, a.e2, wk, bk, a.cy, 3, 2, y);
    free(x); free(t1); free(t2); free(t3); free(u); free(v);
    return ORC_OK;
}

/* The same from RGB u8 frames [N][H][W][3] fed as they are (format 0): x = frames / 255. */
int orc_analysis(int arch, int N, const uint8_t* frames, int H, int W, const float* wts, double* y) {
    if (N < 1 || H < 1 || W < 1) return ORC_ERR_ARG;
    double* x = dalloc((size_t)N * H * W * 3);
    orc_color_in(0, frames, N, H, W, x);
    int rc = orc_analysis_x(arch, N, x, H, W, wts, y);
    free(x);
    return rc;
}

/* Hyper-analysis: z = H2(GELU(H1(y))), both 3x3 stride 2.  z: [ceil(Hy/4)][ceil(Wy/4)][Cz]. */
int orc_hyper_analysis(int arch, int N, const double* y, int Hy, int Wy, const float* wts, double* z) {
    arch_t a;
    if (get_arch(arch, &a)) return ORC_ERR_ARG;
    const float *wk, *bk;
    int h1 = conv_out(Hy, 3, 2), w1 = conv_out(Wy, 3, 2);
    double* t = dalloc((size_t)h1 * w1 * a.cz);
    layer_ptr(arch, N, wts, 6, &wk, &bk);
    orc_conv2d(y, Hy, Wy, a.cy, wk, bk, a.cz, 3, 2, t);
    gelu_inplace(t, (size_t)h1 * w1 * a.cz);
    layer_ptr(arch, N, wts, 7, &wk, &bk);
    orc_conv2d(t, h1, w1, a.cz, wk, bk, a.cz, 3, 2, z);
    free(t);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------------ */
/* Scale bins, thresholds and CDF tables                                                            */
/* ------------------------------------------------------------------------------------------------ */

/* Scale bin k = 0..63: s_k = exp(ln 0.11 + k (ln 64 - ln 0.11) / 63) (64 log-spaced bins on [0.11, 64]). */
double orc_scale(int k) { return exp(log(0.11) + k * (log(64.0) - log(0.11)) / 63.0); }

/* Log-domain decision threshold between bins k-1 and k (k = 1..63): the midpoint of their logs. */
double orc_log_threshold(int k) { return 0.5 * (log(orc_scale(k - 1)) + log(orc_scale(k))); }

/* Quantisation step for qp in [0, 63]: q = 2^((qp - 32) / 8); qp = 32 gives q = 1. */
double orc_qstep(int qp) { return pow(2.0, (qp - 32) / 8.0); }

/* FP32 thresholds used to index log sigma at rate qp: thr[k-1] = float(t_k + ln q), k = 1..63.
 * The element's scale relative to the quantisation step is sigma/q, so ln(sigma/q) > t_k  <=>
 * ln sigma > t_k + ln q. */
void orc_thresholds(int qp, float* thr) {
    double lq = log(orc_qstep(qp));
    for (int k = 1; k < NBINS; k++) thr[k - 1] = (float)(orc_log_threshold(k) + lq);
}

/* Integer CDF table for bin k: a zero-mean Gaussian of std s = s_k discretised on the integers,
 * |r| <= 255, tails beyond +-254.5 folded into the end symbols:
 *   p_0 = erf(0.5 / (s sqrt2)),  p_r = (erfc((|r|-0.5)/(s sqrt2)) - erfc((|r|+0.5)/(s sqrt2))) / 2
 *   for 0 < |r| < 255, p_{+-255} = erfc(254.5 / (s sqrt2)) / 2;
 *   f_r = 1 + floor(p_r (2^16 - 511)), then f_0 += 2^16 - sum f (the mode takes the rounding deficit).
 * freq[k*511 + (r+255)] = f_r; cum[k*512 + j] = sum_{i<j} f.  Built in FP64. */
void orc_build_tables(uint32_t* freq, uint32_t* cum) {
    const double budget = (double)(PROB_M - NSYM);
    for (int k = 0; k < NBINS; k++) {
        double s = orc_scale(k), d = s * sqrt(2.0);
        uint32_t* f = freq + (size_t)k * NSYM;
        for (int r = 0; r <= RMAX; r++) {
            double p;
            if (r == 0) p = erf(0.5 / d);
            else if (r < RMAX) p = 0.5 * (erfc((r - 0.5) / d) - erfc((r + 0.5) / d));
            else p = 0.5 * erfc((RMAX - 0.5) / d);
            uint32_t fr = 1u + (uint32_t)floor(p * budget);
            f[RMAX + r] = fr;
            f[RMAX - r] = fr;
        }
        uint32_t sum = 0;
        for (int i = 0; i < NSYM; i++) sum += f[i];
        f[RMAX] += PROB_M - sum;
        uint32_t* c = cum + (size_t)k * (NSYM + 1);
        c[0] = 0;
        for (int i = 0; i < NSYM; i++) c[i + 1] = c[i] + f[i];
    }
}

/* ------------------------------------------------------------------------------------------------ */
/* Quantisation (Sec. 3.4: r^ = round(y - mu), y^ = r^ + mu) and scale indexing                      */
/* ------------------------------------------------------------------------------------------------ */


/* Hyper-latent: z^ = clamp(rint(z), -255, 255).  Per channel c, the scale index used to code z^ is the
 * nearest log bin of the channel's RMS: iz[c] = #{k : t_k < ln sqrt(S_c / n)}, S_c = sum z^^2 over the
 * n = Hz*Wz positions (S_c = 0 gives bin 0). */
int orc_quantize_z(const double* z, int npos, int cz, int16_t* zhat, uint8_t* iz) {
    for (size_t i = 0; i < (size_t)npos * cz; i++) zhat[i] = (int16_t)clampd(rint(z[i]), -RMAX, RMAX);
    for (int c = 0; c < cz; c++) {
        double S = 0.0;
        for (int p = 0; p < npos; p++) {
            double v = zhat[(size_t)p * cz + c];
            S += v * v;
        }
        int idx = 0;
        if (S > 0.0) {
            double lr = 0.5 * log(S / npos);
            for (int k = 1; k < NBINS; k++) idx += orc_log_threshold(k) < lr;
        }
        iz[c] = (uint8_t)idx;
    }
    return ORC_OK;
}

/* Hyper-synthesis (single-step parameter estimation, Sec. 3.4): from z^ alone, one pass gives mu and
 * log sigma for every latent element.  S1, S2: 3x3 conv Cz -> 4Cz, pixel shuffle x2, GELU; crop to
 * (Hy, Wy); S3: 1x1 conv Cz -> 2Cy; channels [0, Cy) are mu, [Cy, 2Cy) are log sigma. */
static int hyper_synthesis_core(int arch, int N, const int16_t* zhat, int Hz, int Wz, int Hy, int Wy,
                                const float* wts, const double* add_s, double* mu, double* logsig, double* s_out);

int orc_hyper_synthesis_s(int arch, int N, const int16_t* zhat, int Hz, int Wz, int Hy, int Wy,
                          const float* wts, double* mu, double* logsig, double* s_out) {
    return hyper_synthesis_core(arch, N, zhat, Hz, Wz, Hy, Wy, wts, NULL, mu, logsig, s_out);
}

/* The same pass with the temporal context's term added to the features before S3. */
int orc_hyper_synthesis_add(int arch, int N, const int16_t* zhat, int Hz, int Wz, int Hy, int Wy, const float* wts,
                            const double* add_s, double* mu, double* logsig, double* s_out) {
    return hyper_synthesis_core(arch, N, zhat, Hz, Wz, Hy, Wy, wts, add_s, mu, logsig, s_out);
}

/* add_s (optional, [Hy][Wy][Cz]): added to the S2 features before S3 (the prior's temporal context). */
static int hyper_synthesis_core(int arch, int N, const int16_t* zhat, int Hz, int Wz, int Hy, int Wy,
                                const float* wts, const double* add_s, double* mu, double* logsig, double* s_out) {
    arch_t a;
    if (get_arch(arch, &a) || 4 * Hz < Hy || 4 * Wz < Wy) return ORC_ERR_ARG;
    const float *wk, *bk;
    int cz = a.cz;
    double* zd = dalloc((size_t)Hz * Wz * cz);
    for (size_t i = 0; i < (size_t)Hz * Wz * cz; i++) zd[i] = zhat[i];
    double* t = dalloc((size_t)Hz * Wz * 4 * cz);
    double* s1 = dalloc((size_t)4 * Hz * Wz * cz);
    layer_ptr(arch, N, wts, 8, &wk, &bk);
    orc_conv2d(zd, Hz, Wz, cz, wk, bk, 4 * cz, 3, 1, t);
    orc_pixel_shuffle(t, Hz, Wz, cz, s1);
    gelu_inplace(s1, (size_t)4 * Hz * Wz * cz);
    int H1 = 2 * Hz, W1 = 2 * Wz;
    double* t2 = dalloc((size_t)H1 * W1 * 4 * cz);
    double* s2 = dalloc((size_t)4 * H1 * W1 * cz);
    layer_ptr(arch, N, wts, 9, &wk, &bk);
    orc_conv2d(s1, H1, W1, cz, wk, bk, 4 * cz, 3, 1, t2);
    orc_pixel_shuffle(t2, H1, W1, cz, s2);
    gelu_inplace(s2, (size_t)4 * H1 * W1 * cz);
    /* crop (2H1 x 2W1) -> (Hy x Wy) */
    double* s2c = dalloc((size_t)Hy * Wy * cz);
    for (int h = 0; h < Hy; h++)
        memcpy(s2c + (size_t)h * Wy * cz, s2 + (size_t)h * (2 * W1) * cz, sizeof(double) * Wy * cz);
    if (add_s)
        for (size_t i = 0; i < (size_t)Hy * Wy * cz; i++) s2c[i] += add_s[i];
    double* p = dalloc((size_t)Hy * Wy * 2 * a.cy);
    layer_ptr(arch, N, wts, 10, &wk, &bk);
    orc_conv2d(s2c, Hy, Wy, cz, wk, bk, 2 * a.cy, 1, 1, p);
    for (size_t i = 0; i < (size_t)Hy * Wy; i++) {
        memcpy(mu + i * a.cy, p + i * 2 * a.cy, sizeof(double) * a.cy);
        memcpy(logsig + i * a.cy, p + i * 2 * a.cy + a.cy, sizeof(double) * a.cy);
    }
    if (s_out) memcpy(s_out, s2c, sizeof(double) * Hy * Wy * cz);
    free(zd); free(t); free(s1); free(t2); free(s2); free(s2c); free(p);
    return ORC_OK;
}

/* The same pass without the feature map.  s_out of orc_hyper_synthesis_s, when not NULL, receives the
 * S2 output s = [Hy][Wy][Cz] (after GELU and crop): the prior that the progressive mean steps read. */
int orc_hyper_synthesis(int arch, int N, const int16_t* zhat, int Hz, int Wz, int Hy, int Wy,
                        const float* wts, double* mu, double* logsig) {
    return orc_hyper_synthesis_s(arch, N, zhat, Hz, Wz, Hy, Wy, wts, mu, logsig, NULL);
}

/* Latent quantisation at rate qp: r^ = clamp(rint((y - mu) / q), -255, 255) and the scale index
 * idx = #{k : thr_qp[k] < log sigma} with the FP32 thresholds of orc_thresholds (the comparison is
 * strict, so a value equal to a threshold goes to the lower bin). */
int orc_quantize_y(const double* y, const double* mu, const double* logsig, size_t n, int qp,
                   int16_t* rhat, uint8_t* idx) {
    if (qp < 0 || qp > 63) return ORC_ERR_ARG;
    double q = orc_qstep(qp);
    float thr[NBINS - 1];
    orc_thresholds(qp, thr);
    for (size_t i = 0; i < n; i++) {
        rhat[i] = (int16_t)clampd(rint((y[i] - mu[i]) / q), -RMAX, RMAX);
        int k = 0;
        for (int j = 0; j < NBINS - 1; j++) k += (double)thr[j] < logsig[i];
        idx[i] = (uint8_t)k;
    }
    return ORC_OK;
}

/* Index only (used by the decoder, which has log sigma but no y). */
int orc_scale_index(const double* logsig, size_t n, int qp, uint8_t* idx) {
    if (qp < 0 || qp > 63) return ORC_ERR_ARG;
    float thr[NBINS - 1];
    orc_thresholds(qp, thr);
    for (size_t i = 0; i < n; i++) {
        int k = 0;
        for (int j = 0; j < NBINS - 1; j++) k += (double)thr[j] < logsig[i];
        idx[i] = (uint8_t)k;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------------ */
/* Progressive means (Sec. 3.4, Fig. 4a and 4c)                                                      */
/* ------------------------------------------------------------------------------------------------ */
/* The latent is split into four partitions, quadtree-like in space and channel.  The parameter
 * network gives the scales of ALL four partitions and the means of partition 0 in one pass (the
 * hyper-synthesis above: mu^0 and log sigma); the means of partitions 1, 2, 3 are then estimated one
 * partition at a time, each from the partitions already reconstructed.  The bit-stream depends on the
 * scales only, so the whole latent is still entropy coded in one step.
 *
 * Reading of the partition (the paper shows it only as a figure): channels are split into four
 * consecutive groups g = c / (Cy / 4); inside each 2x2 spatial block the position t = 2 (h mod 2) +
 * (w mod 2); element (h, w, c) belongs to partition (t + g) mod 4.  Every partition thus holds one
 * position of every 2x2 block in every channel group, a different one per group. */
int orc_partition(int h, int w, int c, int cy) {
    int g = c / (cy / 4);
    int t = 2 * (h % 2) + (w % 2);
    return (t + g) % 4;
}

void orc_partition_map(int Hy, int Wy, int cy, uint8_t* out) {
    for (int h = 0; h < Hy; h++)
        for (int w = 0; w < Wy; w++)
            for (int c = 0; c < cy; c++) out[((size_t)h * Wy + w) * cy + c] = (uint8_t)orc_partition(h, w, c, cy);
}

/* Reading of the mean-estimation network of step k = 1..3 (figure only in the paper): its input is the
 * reconstructed latent restricted to partitions 0..k-1 (zero elsewhere), Cy channels, followed by the
 * prior s, Cz channels; Pk_a: 3x3 conv (Cy + Cz -> Cz) + GELU; Pk_b: 1x1 conv (Cz -> Cy) gives mu^k.
 * Blob (separate from the codec's): P1a, P1b, P2a, P2b, P3a, P3b, each kernel [Cout][k][k][Cin] then
 * bias [Cout]. */
int orc_mean_layer_shape(int arch, int l, int* cout, int* k, int* cin) {
    arch_t a;
    if (get_arch(arch, &a) || l < 0 || l >= 6) return ORC_ERR_ARG;
    if (l % 2 == 0) { *cout = a.cz; *k = 3; *cin = a.cy + a.cz; }
    else            { *cout = a.cy; *k = 1; *cin = a.cz; }
    return ORC_OK;
}

size_t orc_mean_weight_count(int arch) {
    size_t n = 0;
    int co, k, ci;
    for (int l = 0; l < 6; l++) {
        if (orc_mean_layer_shape(arch, l, &co, &k, &ci)) return 0;
        n += (size_t)co * k * k * ci + co;
    }
    return n;
}

static void mean_layer_ptr(int arch, const float* blob, int l, const float** w, const float** b) {
    size_t off = 0;
    int co, k, ci;
    for (int i = 0; i < l; i++) {
        orc_mean_layer_shape(arch, i, &co, &k, &ci);
        off += (size_t)co * k * k * ci + co;
    }
    orc_mean_layer_shape(arch, l, &co, &k, &ci);
    *w = blob + off;
    *b = blob + off + (size_t)co * k * k * ci;
}

/* Step k (1..3): mu_k [Hy][Wy][Cy] from yhat (only its partitions < k are read) and s [Hy][Wy][Cz]. */
int orc_mean_step(int arch, int k, const double* yhat, const double* s, int Hy, int Wy, const float* pm,
                  double* mu_k) {
    arch_t a;
    if (get_arch(arch, &a) || k < 1 || k > 3 || a.cy % 4) return ORC_ERR_ARG;
    const int cin = a.cy + a.cz;
    const size_t npix = (size_t)Hy * Wy;
    double* in = dalloc(npix * cin);
    for (int h = 0; h < Hy; h++)
        for (int w = 0; w < Wy; w++) {
            size_t pix = (size_t)h * Wy + w;
            for (int c = 0; c < a.cy; c++)
                in[pix * cin + c] = orc_partition(h, w, c, a.cy) < k ? yhat[pix * a.cy + c] : 0.0;
            for (int c = 0; c < a.cz; c++) in[pix * cin + a.cy + c] = s[pix * a.cz + c];
        }
    const float *wk, *bk;
    double* t = dalloc(npix * a.cz);
    mean_layer_ptr(arch, pm, 2 * (k - 1), &wk, &bk);
    orc_conv2d(in, Hy, Wy, cin, wk, bk, a.cz, 3, 1, t);
    gelu_inplace(t, npix * a.cz);
    mean_layer_ptr(arch, pm, 2 * (k - 1) + 1, &wk, &bk);
    orc_conv2d(t, Hy, Wy, a.cz, wk, bk, a.cy, 1, 1, mu_k);
    free(in); free(t);
    return ORC_OK;
}

/* The four steps, in the paper's order.  Encoder (y != NULL): for partition 0, r^ = clamp(rint((y -
 * mu^0) / q)); then for k = 1..3, mu^k from the partitions before k and, on partition k, r^ =
 * clamp(rint((y - mu^k) / q)).  Decoder (y == NULL): rhat is given (decoded in one step) and only the
 * reconstruction runs.  Both: y^ = r^ q + mu on each partition with that partition's mean, so the
 * decoder repeats the encoder's means exactly.  mu_used[i] receives the mean element i was coded with
 * (mu^0 on partition 0, mu^k on partition k); yhat receives the reconstructed latent. */
int orc_progressive_means(int arch, const double* y, int16_t* rhat, const double* mu0, const double* s, int Hy,
                          int Wy, int qp, const float* pm, double* yhat, double* mu_used) {
    arch_t a;
    if (get_arch(arch, &a) || qp < 0 || qp > 63 || !pm || a.cy % 4) return ORC_ERR_ARG;
    const double q = orc_qstep(qp);
    const size_t ny = (size_t)Hy * Wy * a.cy;
    double* muk = dalloc(ny);
    for (size_t i = 0; i < ny; i++) yhat[i] = 0.0;
    for (int k = 0; k < 4; k++) {
        if (k > 0) orc_mean_step(arch, k, yhat, s, Hy, Wy, pm, muk);
        for (int h = 0; h < Hy; h++)
            for (int w = 0; w < Wy; w++)
                for (int c = 0; c < a.cy; c++) {
                    if (orc_partition(h, w, c, a.cy) != k) continue;
                    size_t i = ((size_t)h * Wy + w) * a.cy + c;
                    double m = k == 0 ? mu0[i] : muk[i];
                    if (y) rhat[i] = (int16_t)clampd(rint((y[i] - m) / q), -RMAX, RMAX);
                    yhat[i] = rhat[i] * q + m;
                    mu_used[i] = m;
                }
    }
    free(muk);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------------ */
/* Interleaved rANS (single consolidated coding step over the whole latent, Sec. 3.4)               */
/* ------------------------------------------------------------------------------------------------ */
/* Reading: 32-bit state x in [2^16, 2^32), probabilities with 16-bit precision (M = 2^16), 16-bit
 * output words (Duda's rANS with Giesen's interleaving).  K lanes: element i goes to lane i mod K; lane
 * j codes its elements i = j, j+K, j+2K, ... .  Encoding runs each lane backwards (last element first)
 * starting from x = 2^16:
 *     if x >= f * 2^16: emit x & 0xFFFF, x >>= 16           (at most one word per symbol)
 *     x = floor(x / f) * 2^16 + (x mod f) + c
 * then flushes x as two words.  A lane's stream is stored in decoding order: the final state's high
 * half, its low half, then the renormalisation words newest first.  Decoding runs forwards:
 *     x = (w0 << 16) | w1;  per symbol: slot = x & 0xFFFF, s = the symbol with c_s <= slot < c_s + f_s,
 *     x = f_s (x >> 16) + slot - c_s;  if x < 2^16: x = (x << 16) | next word
 * and a valid lane ends with x == 2^16 having consumed exactly its words.
 *
 * Tables are generic for testing: symbol value v uses slot v + offset of table t (freq[t*nsym + slot],
 * cum[t*(nsym+1) + slot]); the codec uses nsym = 511, offset = 255.
 *
 * Section layout: K little-endian u32 word counts, then the K lane streams back to back (u16 words),
 * zero-padded to a multiple of 4 bytes.  Returns the section size in bytes (0 on capacity error). */
size_t orc_rans_encode(const int16_t* sym, const uint8_t* tab, size_t n, int K, const uint32_t* freq,
                       const uint32_t* cum, int nsym, int offset, uint8_t* out, size_t cap) {
    if (K < 1) return 0;
    size_t per_lane = n / K + 1 + 2;
    uint16_t* buf = (uint16_t*)malloc(sizeof(uint16_t) * per_lane);
    size_t head = (size_t)K * 4, pos = head;
    if (cap < head) { free(buf); return 0; }
    for (int j = 0; j < K; j++) {
        size_t cnt = (j < (long long)n) ? (n - j + K - 1) / K : 0; /* elements of lane j */
        size_t wp = per_lane;                                     /* fill buf from the back */
        uint32_t x = RANS_L;
        for (size_t m = cnt; m-- > 0;) {
            size_t i = (size_t)j + m * K;
            int slot = sym[i] + offset;
            uint32_t f = freq[(size_t)tab[i] * nsym + slot];
            uint32_t c = cum[(size_t)tab[i] * (nsym + 1) + slot];
            if ((uint64_t)x >= (uint64_t)f << 16) {
                buf[--wp] = (uint16_t)(x & 0xFFFF);
                x >>= 16;
            }
            x = (x / f) * PROB_M + (x % f) + c;
        }
        buf[--wp] = (uint16_t)(x & 0xFFFF);
        buf[--wp] = (uint16_t)(x >> 16);
        uint32_t words = (uint32_t)(per_lane - wp);
        if (pos + 2 * (size_t)words > cap) { free(buf); return 0; }
        out[4 * j + 0] = (uint8_t)(words & 0xFF);
        out[4 * j + 1] = (uint8_t)((words >> 8) & 0xFF);
        out[4 * j + 2] = (uint8_t)((words >> 16) & 0xFF);
        out[4 * j + 3] = (uint8_t)(words >> 24);
        for (uint32_t w = 0; w < words; w++) {
            uint16_t v = buf[wp + w];
            out[pos++] = (uint8_t)(v & 0xFF);
            out[pos++] = (uint8_t)(v >> 8);
        }
    }
    while (pos % 4) {
        if (pos >= cap) { free(buf); return 0; }
        out[pos++] = 0;
    }
    free(buf);
    return pos;
}

/* Decode a section produced by orc_rans_encode.  avail = bytes available from `in`.  Writes the n
 * symbols and *used = section size in bytes.  Returns ORC_ERR_CORRUPT if a lane's counts, words or
 * final state are inconsistent. */
int orc_rans_decode(const uint8_t* in, size_t avail, const uint8_t* tab, size_t n, int K, const uint32_t* freq,
                    const uint32_t* cum, int nsym, int offset, int16_t* sym, size_t* used) {
    if (K < 1 || avail < (size_t)K * 4) return ORC_ERR_CORRUPT;
    size_t pos = (size_t)K * 4;
    for (int j = 0; j < K; j++) {
        uint32_t words = (uint32_t)in[4 * j] | ((uint32_t)in[4 * j + 1] << 8) | ((uint32_t)in[4 * j + 2] << 16) |
                         ((uint32_t)in[4 * j + 3] << 24);
        size_t cnt = (j < (long long)n) ? (n - j + K - 1) / K : 0;
        if (words < 2 || words > cnt + 2 || pos + 2 * (size_t)words > avail) return ORC_ERR_CORRUPT;
        const uint8_t* p = in + pos;
        uint32_t r = 0;
#define NEXTW() ((uint32_t)p[2 * r] | ((uint32_t)p[2 * r + 1] << 8))
        uint32_t x = NEXTW() << 16;
        r++;
        x |= NEXTW();
        r++;
        for (size_t m = 0; m < cnt; m++) {
            size_t i = (size_t)j + m * K;
            const uint32_t* c = cum + (size_t)tab[i] * (nsym + 1);
            uint32_t slot = x & 0xFFFF;
            int s = 0;
            while (s + 1 < nsym && c[s + 1] <= slot) s++; /* linear search: plain, slow, obvious */
            uint32_t f = c[s + 1] - c[s];
            x = f * (x >> 16) + slot - c[s];
            if (x < RANS_L) {
                if (r >= words) return ORC_ERR_CORRUPT;
                x = (x << 16) | NEXTW();
                r++;
            }
            sym[i] = (int16_t)(s - offset);
        }
#undef NEXTW
        if (x != RANS_L || r != words) return ORC_ERR_CORRUPT;
        pos += 2 * (size_t)words;
    }
    while (pos % 4) pos++;
    if (pos > avail) return ORC_ERR_CORRUPT;
    *used = pos;
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------------ */
/* Frame-specific synthesis (Sec. 3.2): N decoders, decoder f reconstructs frame f from y^            */
/* ------------------------------------------------------------------------------------------------ */

/* Decoder f: D0 3x3 Cy->4Cd1, PS, GELU; R1: h + R1b(GELU(R1a(h))); U1 3x3 Cd1->4Cd2, PS, GELU;
 * R2: h + R2b(GELU(R2a(h))); U2 3x3 Cd2->4Cd2, PS, GELU; U3 3x3 Cd2->12, PS -> o (3 channels);
 * x^ = clamp(0.5 + o, 0, 1), cropped to H x W.  frames: [N][H][W][3] doubles in [0, 1]. */
static int synthesis_core(int arch, int N, const double* yhat, int Hy, int Wy, int H, int W, const float* wts,
                          const double* F, const float* tw, double* frames);

int orc_synthesis(int arch, int N, const double* yhat, int Hy, int Wy, int H, int W, const float* wts,
                  double* frames) {
    return synthesis_core(arch, N, yhat, Hy, Wy, H, W, wts, NULL, NULL, frames);
}

static void temporal_layer_ptr(int arch, int N, const float* blob, int l, const float** w, const float** b);

/* F (optional, the chunk feature [2Hy][2Wy][Cf]) with the temporal blob tw: each frame decoder adds its
 * own 1x1 projection DF_f(F) to its D0 output. */
static int synthesis_core(int arch, int N, const double* yhat, int Hy, int Wy, int H, int W, const float* wts,
                          const double* F, const float* tw, double* frames) {
    arch_t a;
    if (get_arch(arch, &a) || 16 * Hy < H || 16 * Wy < W) return ORC_ERR_ARG;
    for (int f = 0; f < N; f++) {
        const float *wk, *bk;
        int base = 11 + 8 * f;
        int h = Hy, w = Wy;
        /* D0 */
        double* t = dalloc((size_t)h * w * 4 * a.cd1);
        layer_ptr(arch, N, wts, base + 0, &wk, &bk);
        orc_conv2d(yhat, h, w, a.cy, wk, bk, 4 * a.cd1, 3, 1, t);
        double* h1 = dalloc((size_t)4 * h * w * a.cd1);
        orc_pixel_shuffle(t, h, w, a.cd1, h1);
        free(t);
        h *= 2; w *= 2;
        size_t n1 = (size_t)h * w * a.cd1;
        gelu_inplace(h1, n1);
        if (F && tw) {
            const float *wd, *bd;
            double* df = dalloc(n1);
            temporal_layer_ptr(arch, N, tw, 5 + f, &wd, &bd);
            orc_conv2d(F, h, w, ORC_CF, wd, bd, a.cd1, 1, 1, df);
            for (size_t i = 0; i < n1; i++) h1[i] += df[i];
            free(df);
        }
        /* R1 */
        double* u = dalloc(n1);
        double* v = dalloc(n1);
        layer_ptr(arch, N, wts, base + 1, &wk, &bk);
        orc_conv2d(h1, h, w, a.cd1, wk, bk, a.cd1, 3, 1, u);
        gelu_inplace(u, n1);
        layer_ptr(arch, N, wts, base + 2, &wk, &bk);
        orc_conv2d(u, h, w, a.cd1, wk, bk, a.cd1, 3, 1, v);
        for (size_t i = 0; i < n1; i++) h1[i] += v[i];
        free(u); free(v);
        /* U1 */
        t = dalloc((size_t)h * w * 4 * a.cd2);
        layer_ptr(arch, N, wts, base + 3, &wk, &bk);
        orc_conv2d(h1, h, w, a.cd1, wk, bk, 4 * a.cd2, 3, 1, t);
        double* h2 = dalloc((size_t)4 * h * w * a.cd2);
        orc_pixel_shuffle(t, h, w, a.cd2, h2);
        free(t); free(h1);
        h *= 2; w *= 2;
        size_t n2 = (size_t)h * w * a.cd2;
        gelu_inplace(h2, n2);
        /* R2 */
        u = dalloc(n2);
        v = dalloc(n2);
        layer_ptr(arch, N, wts, base + 4, &wk, &bk);
        orc_conv2d(h2, h, w, a.cd2, wk, bk, a.cd2, 3, 1, u);
        gelu_inplace(u, n2);
        layer_ptr(arch, N, wts, base + 5, &wk, &bk);
        orc_conv2d(u, h, w, a.cd2, wk, bk, a.cd2, 3, 1, v);
        for (size_t i = 0; i < n2; i++) h2[i] += v[i];
        free(u); free(v);
        /* U2 */
        t = dalloc((size_t)h * w * 4 * a.cd2);
        layer_ptr(arch, N, wts, base + 6, &wk, &bk);
        orc_conv2d(h2, h, w, a.cd2, wk, bk, 4 * a.cd2, 3, 1, t);
        double* h3 = dalloc((size_t)4 * h * w * a.cd2);
        orc_pixel_shuffle(t, h, w, a.cd2, h3);
        free(t); free(h2);
        h *= 2; w *= 2;
        gelu_inplace(h3, (size_t)h * w * a.cd2);
        /* U3 */
        t = dalloc((size_t)h * w * 12);
        layer_ptr(arch, N, wts, base + 7, &wk, &bk);
        orc_conv2d(h3, h, w, a.cd2, wk, bk, 12, 3, 1, t);
        double* o = dalloc((size_t)4 * h * w * 3);
        orc_pixel_shuffle(t, h, w, 3, o);
        free(t); free(h3);
        h *= 2; w *= 2;
        for (int yy = 0; yy < H; yy++)
            for (int xx = 0; xx < W; xx++)
                for (int c = 0; c < 3; c++)
                    frames[(((size_t)f * H + yy) * W + xx) * 3 + c] =
                        clampd(0.5 + o[((size_t)yy * w + xx) * 3 + c], 0.0, 1.0);
        free(o);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------------ */
/* Temporal chunk context (Sec. 3.1, Fig. 3; Sec. 3.3)                                              */
/* ------------------------------------------------------------------------------------------------ */
/* Chunk i is coded conditioned on a context C_i generated from chunk i-1's decoded feature.  Reading of
 * the figure on the plain layers (Cf = Cc = 64 channels, all at 1/8 of the padded frame size):
 *   chunk feature   F_i     = GELU(PS(FD(y^_i))) + FC(C_i)       FD 3x3 Cy -> 4 Cf, FC 1x1 Cc -> Cf
 *   next context    C_{i+1} = GELU(CG(F_i))                      CG 3x3 Cf -> Cc
 *   encoder         A3 output + EC(C_i) before the interaction   EC 1x1 Cc -> e2
 *   prior           S2 features + PC(C_i) before S3              PC 3x3 stride 2 Cc -> Cz
 *   frame decoder f D0 output + DF_f(F_i)                        DF_f 1x1 Cf -> Cd1
 * The first chunk of a stream uses C_0 = 0.  Blob: EC, FD, FC, CG, PC, then DF_f for f = 0..N-1, each
 * kernel [Cout][k][k][Cin] then bias [Cout]. */
int orc_temporal_layer_shape(int arch, int N, int l, int* cout, int* k, int* cin) {
    arch_t a;
    if (get_arch(arch, &a) || N < 1 || l < 0 || l >= 5 + N) return ORC_ERR_ARG;
    int t[5][3] = {{a.e2, 1, ORC_CC}, {4 * ORC_CF, 3, a.cy}, {ORC_CF, 1, ORC_CC}, {ORC_CC, 3, ORC_CF},
                   {a.cz, 3, ORC_CC}};
    if (l < 5) { *cout = t[l][0]; *k = t[l][1]; *cin = t[l][2]; }
    else { *cout = a.cd1; *k = 1; *cin = ORC_CF; }
    return ORC_OK;
}

size_t orc_temporal_weight_count(int arch, int N) {
    size_t n = 0;
    int co, k, ci;
    for (int l = 0; l < 5 + N; l++) {
        if (orc_temporal_layer_shape(arch, N, l, &co, &k, &ci)) return 0;
        n += (size_t)co * k * k * ci + co;
    }
    return n;
}

static void temporal_layer_ptr(int arch, int N, const float* blob, int l, const float** w, const float** b) {
    size_t off = 0;
    int co, k, ci;
    for (int i = 0; i < l; i++) {
        orc_temporal_layer_shape(arch, N, i, &co, &k, &ci);
        off += (size_t)co * k * k * ci + co;
    }
    orc_temporal_layer_shape(arch, N, l, &co, &k, &ci);
    *w = blob + off;
    *b = blob + off + (size_t)co * k * k * ci;
}

/* Context dims: [H8][W8][Cc] with H8, W8 = the padded frame size / 8 (= 2 Hy, 2 Wy). */
int orc_context_dims(int arch, int H, int W, int* H8, int* W8, int* Cc) {
    arch_t a;
    if (get_arch(arch, &a) || H < 1 || W < 1) return ORC_ERR_ARG;
    *H8 = (H + 15) / 16 * 2;
    *W8 = (W + 15) / 16 * 2;
    *Cc = arch == 2 ? DC_CC : ORC_CC;
    return ORC_OK;
}

/* One 1x1 / 3x3 temporal layer l on x [H][W][cin] (c == NULL stands for the all-zero first context). */
static void temporal_conv(int arch, int N, const float* tw, int l, const double* x, int H, int W, int stride,
                          double* out) {
    const float *wk, *bk;
    int co, k, ci;
    orc_temporal_layer_shape(arch, N, l, &co, &k, &ci);
    temporal_layer_ptr(arch, N, tw, l, &wk, &bk);
    if (x) {
        orc_conv2d(x, H, W, ci, wk, bk, co, k, stride, out);
    } else {
        int Ho = conv_out(H, k, stride), Wo = conv_out(W, k, stride);
        for (size_t i = 0; i < (size_t)Ho * Wo; i++)
            for (int c = 0; c < co; c++) out[i * co + c] = bk[c];
    }
}

/* F_i from y^_i [Hy][Wy][Cy] and C_i (NULL: zero), F: [2Hy][2Wy][Cf]. */
int orc_chunk_feature(int arch, int N, const double* yhat, int Hy, int Wy, const float* tw, const double* c_in,
                      double* F) {
    arch_t a;
    if (get_arch(arch, &a) || !tw) return ORC_ERR_ARG;
    const size_t n8 = (size_t)4 * Hy * Wy;
    double* t = dalloc(n8 * ORC_CF);
    double* fc = dalloc(n8 * ORC_CF);
    temporal_conv(arch, N, tw, 1, yhat, Hy, Wy, 1, t);
    orc_pixel_shuffle(t, Hy, Wy, ORC_CF, F);
    gelu_inplace(F, n8 * ORC_CF);
    temporal_conv(arch, N, tw, 2, c_in, 2 * Hy, 2 * Wy, 1, fc);
    for (size_t i = 0; i < n8 * ORC_CF; i++) F[i] += fc[i];
    free(t); free(fc);
    return ORC_OK;
}

/* C_{i+1} = GELU(CG(F_i)), [H8][W8][Cc]. */
int orc_context_next(int arch, int N, const double* F, int H8, int W8, const float* tw, double* c_out) {
    if (!tw) return ORC_ERR_ARG;
    temporal_conv(arch, N, tw, 3, F, H8, W8, 1, c_out);
    gelu_inplace(c_out, (size_t)H8 * W8 * ORC_CC);
    return ORC_OK;
}

/* The conditioning terms from C_i: EC(C_i) [H8][W8][e2] (encoder) and PC(C_i) [H8/2][W8/2][Cz] (prior). */
int orc_context_terms(int arch, int N, const double* c_in, int H8, int W8, const float* tw, double* ec, double* pc) {
    if (!tw) return ORC_ERR_ARG;
    if (ec) temporal_conv(arch, N, tw, 0, c_in, H8, W8, 1, ec);
    if (pc) temporal_conv(arch, N, tw, 4, c_in, H8, W8, 2, pc);
    return ORC_OK;
}

/* Frame-specific synthesis with the chunk feature (temporal mode). */
int orc_synthesis_f(int arch, int N, const double* yhat, int Hy, int Wy, int H, int W, const float* wts,
                    const double* F, const float* tw, double* frames) {
    if (!F || !tw) return ORC_ERR_ARG;
    return synthesis_core(arch, N, yhat, Hy, Wy, H, W, wts, F, tw, frames);
}

/* ------------------------------------------------------------------------------------------------ */
/* DC-block model (Appendix: all modules built from depth-wise convolution blocks; HT-S block counts) */
/* ------------------------------------------------------------------------------------------------ */
/* Reading of the appendix figure and counts (widths are not given; they are chosen so that the model
 * costs about the paper's 211 G MACs per 1080p frame for N = 8):
 *   DC block of width C:  y = x + PWb(GELU(DW(PWa(x)))),  out = y + PWd(GELU(PWc(y)))
 *     PWa, PWb 1x1 C -> C; DW 3x3 depth-wise (one 3x3 filter per channel); PWc 1x1 C -> 2C; PWd 2C -> C
 *   at 1/8 of the padded frame size (H8 x W8):
 *   patch embedding  x = PE(s2d8(frames))          s2d8: channel (3n + c) 64 + 8 dy + dx, PE 1x1 -> C
 *   chunk encoder    x += EC(C_i); 6 DC blocks; y = ED(x)   (ED 3x3 stride 2, C -> Cy)
 *   hyperprior       as the plain model's (H1, H2, S1, S2, S3), with PC(C_i) (3x3 stride 2, Cc -> Cz)
 *                    added to the S2 features before S3
 *   chunk decoder    x = GELU(PS(DU(y^))) + FC(C_i)  (DU 1x1 Cy -> 4C), 7 DC blocks -> F_i
 *   context          11 DC blocks on F_i, C_{i+1} = GO(.)  (GO 1x1 C -> Cc)
 *   frame decoder f  FP_f (1x1 C -> Cf), 3 DC blocks at Cf, FO_f (1x1 Cf -> 192), pixel shuffle x8,
 *                    x^ = clamp(0.5 + o, 0, 1), cropped
 * C = 512, Cf = 256, Cc = 128, Cy = 256, Cz = 128; C_0 = 0.  Blob order: PE, EC, 6 x [PWa DW PWb PWc PWd],
 * ED, H1, H2, S1, S2, S3, PC, DU, FC, 7 x [...], 11 x [...], GO, then per frame FP_f, 3 x [...] at Cf,
 * FO_f; a depth-wise layer is stored as kernel [C][3][3][1] + bias [C]. */
#define DC_SHARED 132  /* layers before the frame decoders */
#define DC_PER_FRAME 17

/* block layer j (0..4) of width c: (cout, k, cin) */
static void dc_block_shape(int c, int j, int* co, int* k, int* ci) {
    const int t[5][3] = {{c, 1, c}, {c, 3, 1}, {c, 1, c}, {2 * c, 1, c}, {c, 1, 2 * c}};
    *co = t[j][0]; *k = t[j][1]; *ci = t[j][2];
}

int orc_dc_layer_shape(int N, int l, int* cout, int* k, int* cin) {
    if (N < 1 || l < 0 || l >= DC_SHARED + DC_PER_FRAME * N) return ORC_ERR_ARG;
    if (l >= DC_SHARED) {
        int j = (l - DC_SHARED) % DC_PER_FRAME;
        if (j == 0) { *cout = DC_CF; *k = 1; *cin = DC_C; }
        else if (j == 16) { *cout = 192; *k = 1; *cin = DC_CF; }
        else dc_block_shape(DC_CF, (j - 1) % 5, cout, k, cin);
        return ORC_OK;
    }
    if (l == 0) { *cout = DC_C; *k = 1; *cin = 3 * N * 64; }
    else if (l == 1) { *cout = DC_C; *k = 1; *cin = DC_CC; }
    else if (l < 32) dc_block_shape(DC_C, (l - 2) % 5, cout, k, cin);
    else if (l == 32) { *cout = DC_CY; *k = 3; *cin = DC_C; }
    else if (l == 33) { *cout = DC_CZ; *k = 3; *cin = DC_CY; }
    else if (l == 34) { *cout = DC_CZ; *k = 3; *cin = DC_CZ; }
    else if (l == 35 || l == 36) { *cout = 4 * DC_CZ; *k = 3; *cin = DC_CZ; }
    else if (l == 37) { *cout = 2 * DC_CY; *k = 1; *cin = DC_CZ; }
    else if (l == 38) { *cout = DC_CZ; *k = 3; *cin = DC_CC; }
    else if (l == 39) { *cout = 4 * DC_C; *k = 1; *cin = DC_CY; }
    else if (l == 40) { *cout = DC_C; *k = 1; *cin = DC_CC; }
    else if (l < 131) dc_block_shape(DC_C, (l - 41) % 5, cout, k, cin);
    else { *cout = DC_CC; *k = 1; *cin = DC_C; }
    return ORC_OK;
}

size_t orc_dc_weight_count(int N) {
    size_t n = 0;
    int co, k, ci;
    for (int l = 0; l < DC_SHARED + DC_PER_FRAME * N; l++) {
        if (orc_dc_layer_shape(N, l, &co, &k, &ci)) return 0;
        n += (size_t)co * k * k * ci + co;
    }
    return n;
}

static int dc_hyper_layer(int l) { return 33 + (l - 6); }  /* H1 H2 S1 S2 S3 */

static void dc_layer_ptr(int N, const float* blob, int l, const float** w, const float** b) {
    size_t off = 0;
    int co, k, ci;
    for (int i = 0; i < l; i++) {
        orc_dc_layer_shape(N, i, &co, &k, &ci);
        off += (size_t)co * k * k * ci + co;
    }
    orc_dc_layer_shape(N, l, &co, &k, &ci);
    *w = blob + off;
    *b = blob + off + (size_t)co * k * k * ci;
}

/* Depth-wise 3x3 convolution, zero padding 1: out[h][w][c] = b[c] + sum w[c][ky][kx] x[h+ky-1][w+kx-1][c]. */
void orc_dw_conv(const double* x, int H, int W, int C, const float* w, const float* b, double* out) {
    #pragma omp parallel for
    for (int h = 0; h < H; h++)
        for (int ww = 0; ww < W; ww++)
            for (int c = 0; c < C; c++) {
                double acc = b[c];
                for (int ky = 0; ky < 3; ky++)
                    for (int kx = 0; kx < 3; kx++) {
                        int ih = h + ky - 1, iw = ww + kx - 1;
                        if (ih < 0 || ih >= H || iw < 0 || iw >= W) continue;
                        acc += (double)w[(size_t)c * 9 + ky * 3 + kx] * x[((size_t)ih * W + iw) * C + c];
                    }
                out[((size_t)h * W + ww) * C + c] = acc;
            }
}

/* One DC block of width c on x [H][W][c] in place; its five layers start at blob layer l0. */
static void dc_block(int N, const float* wts, int l0, double* x, int H, int W, int c) {
    const size_t n = (size_t)H * W;
    const float *wk, *bk;
    double* t = dalloc(n * c);
    double* u = dalloc(n * c);
    double* v = dalloc(n * 2 * c);
    dc_layer_ptr(N, wts, l0, &wk, &bk);
    orc_conv2d(x, H, W, c, wk, bk, c, 1, 1, t);
    dc_layer_ptr(N, wts, l0 + 1, &wk, &bk);
    orc_dw_conv(t, H, W, c, wk, bk, u);
    gelu_inplace(u, n * c);
    dc_layer_ptr(N, wts, l0 + 2, &wk, &bk);
    orc_conv2d(u, H, W, c, wk, bk, c, 1, 1, t);
    for (size_t i = 0; i < n * c; i++) x[i] += t[i];
    dc_layer_ptr(N, wts, l0 + 3, &wk, &bk);
    orc_conv2d(x, H, W, c, wk, bk, 2 * c, 1, 1, v);
    gelu_inplace(v, n * 2 * c);
    dc_layer_ptr(N, wts, l0 + 4, &wk, &bk);
    orc_conv2d(v, H, W, 2 * c, wk, bk, c, 1, 1, t);
    for (size_t i = 0; i < n * c; i++) x[i] += t[i];
    free(t); free(u); free(v);
}

/* c_in NULL stands for the all-zero first context: a 1x1 / stride-2 3x3 layer of it is its bias. */
static void dc_context_layer(int N, const float* wts, int l, const double* c_in, int H8, int W8, int stride,
                             double* out) {
    const float *wk, *bk;
    int co, k, ci;
    orc_dc_layer_shape(N, l, &co, &k, &ci);
    dc_layer_ptr(N, wts, l, &wk, &bk);
    if (c_in) {
        orc_conv2d(c_in, H8, W8, ci, wk, bk, co, k, stride, out);
    } else {
        int Ho = conv_out(H8, k, stride), Wo = conv_out(W8, k, stride);
        for (size_t i = 0; i < (size_t)Ho * Wo; i++)
            for (int c = 0; c < co; c++) out[i * co + c] = bk[c];
    }
}

/* Chunk encoder: frames (network channels x [N][H][W][3] in [0, 1]) -> y [H8/2][W8/2][Cy]. */
int orc_dc_analysis(int N, const double* xin, int H, int W, const float* wts, const double* c_in, double* y) {
    const int Hp = (H + 15) / 16 * 16, Wp = (W + 15) / 16 * 16, H8 = Hp / 8, W8 = Wp / 8, C0 = 3 * N * 64;
    const size_t n8 = (size_t)H8 * W8;
    double* p = dalloc(n8 * C0);
    for (int h = 0; h < Hp; h++)
        for (int w = 0; w < Wp; w++) {
            const int sh = h < H ? h : H - 1, sw = w < W ? w : W - 1;
            for (int n = 0; n < N; n++)
                for (int c = 0; c < 3; c++)
                    p[((size_t)(h / 8) * W8 + w / 8) * C0 + (3 * n + c) * 64 + 8 * (h % 8) + (w % 8)] =
                        xin[(((size_t)n * H + sh) * W + sw) * 3 + c];
        }
    const float *wk, *bk;
    double* x = dalloc(n8 * DC_C);
    double* e = dalloc(n8 * DC_C);
    dc_layer_ptr(N, wts, 0, &wk, &bk);
    orc_conv2d(p, H8, W8, C0, wk, bk, DC_C, 1, 1, x);
    dc_context_layer(N, wts, 1, c_in, H8, W8, 1, e);
    for (size_t i = 0; i < n8 * DC_C; i++) x[i] += e[i];
    for (int b = 0; b < 6; b++) dc_block(N, wts, 2 + 5 * b, x, H8, W8, DC_C);
    dc_layer_ptr(N, wts, 32, &wk, &bk);
    orc_conv2d(x, H8, W8, DC_C, wk, bk, DC_CY, 3, 2, y);
    free(p); free(x); free(e);
    return ORC_OK;
}

/* The prior's context term PC(C_i) [H8/2][W8/2][Cz]. */
int orc_dc_prior_term(int N, const double* c_in, int H8, int W8, const float* wts, double* pc) {
    dc_context_layer(N, wts, 38, c_in, H8, W8, 2, pc);
    return ORC_OK;
}

/* Chunk decoder and context generation: y^ [Hy][Wy][Cy] -> F [2Hy][2Wy][C] and (c_out) C_{i+1} [.][.][Cc]. */
int orc_dc_trunk(int N, const double* yhat, int Hy, int Wy, const float* wts, const double* c_in, double* F,
                 double* c_out) {
    const int H8 = 2 * Hy, W8 = 2 * Wy;
    const size_t n8 = (size_t)H8 * W8;
    const float *wk, *bk;
    double* t = dalloc((size_t)Hy * Wy * 4 * DC_C);
    double* e = dalloc(n8 * DC_C);
    dc_layer_ptr(N, wts, 39, &wk, &bk);
    orc_conv2d(yhat, Hy, Wy, DC_CY, wk, bk, 4 * DC_C, 1, 1, t);
    orc_pixel_shuffle(t, Hy, Wy, DC_C, F);
    gelu_inplace(F, n8 * DC_C);
    dc_context_layer(N, wts, 40, c_in, H8, W8, 1, e);
    for (size_t i = 0; i < n8 * DC_C; i++) F[i] += e[i];
    for (int b = 0; b < 7; b++) dc_block(N, wts, 41 + 5 * b, F, H8, W8, DC_C);
    if (c_out) {
        double* g = dalloc(n8 * DC_C);
        memcpy(g, F, sizeof(double) * n8 * DC_C);
        for (int b = 0; b < 11; b++) dc_block(N, wts, 76 + 5 * b, g, H8, W8, DC_C);
        dc_layer_ptr(N, wts, 131, &wk, &bk);
        orc_conv2d(g, H8, W8, DC_C, wk, bk, DC_CC, 1, 1, c_out);
        free(g);
    }
    free(t); free(e);
    return ORC_OK;
}

/* Frame decoders: F [H8][W8][C] -> frames [N][H][W][3] in [0, 1]. */
int orc_dc_frames(int N, const double* F, int H8, int W8, int H, int W, const float* wts, double* frames) {
    const size_t n8 = (size_t)H8 * W8;
    for (int f = 0; f < N; f++) {
        const int l0 = DC_SHARED + DC_PER_FRAME * f;
        const float *wk, *bk;
        double* h = dalloc(n8 * DC_CF);
        double* o = dalloc(n8 * 192);
        dc_layer_ptr(N, wts, l0, &wk, &bk);
        orc_conv2d(F, H8, W8, DC_C, wk, bk, DC_CF, 1, 1, h);
        for (int b = 0; b < 3; b++) dc_block(N, wts, l0 + 1 + 5 * b, h, H8, W8, DC_CF);
        dc_layer_ptr(N, wts, l0 + 16, &wk, &bk);
        orc_conv2d(h, H8, W8, DC_CF, wk, bk, 192, 1, 1, o);
        /* pixel shuffle x8: out[8h + dy][8w + dx][c] = o[h][w][64 c + 8 dy + dx] */
        for (int yy = 0; yy < H; yy++)
            for (int xx = 0; xx < W; xx++)
                for (int c = 0; c < 3; c++)
                    frames[(((size_t)f * H + yy) * W + xx) * 3 + c] =
                        clampd(0.5 + o[((size_t)(yy / 8) * W8 + xx / 8) * 192 + 64 * c + 8 * (yy % 8) + (xx % 8)],
                               0.0, 1.0);
        free(h); free(o);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------------ */
/* Whole chunk: encode and decode with the bit-stream container                                     */
/* ------------------------------------------------------------------------------------------------ */
/* Container (little-endian): "UFVC", u8 version, u8 arch, u8 N, u8 qp, u16 W, u16 H, u32 K,
 * u32 Kz, Cz bytes iz[c]; zero-padded to a multiple of 4; then the z^ section (Kz lanes, Kz = min(K,
 * n_z)), then the y^ section (K lanes).  Both sections as in orc_rans_encode.  Version 1: every mean
 * comes from the single parameter pass; version 2: partitions 1..3 take the progressive means
 * (orc_progressive_means), which the decoder must then repeat with the same mean-network weights. */

static void put16(uint8_t* p, uint32_t v) { p[0] = v & 0xFF; p[1] = (v >> 8) & 0xFF; }
static void put32(uint8_t* p, uint32_t v) { put16(p, v & 0xFFFF); put16(p + 2, v >> 16); }
static uint32_t get16(const uint8_t* p) { return (uint32_t)p[0] | ((uint32_t)p[1] << 8); }
static uint32_t get32(const uint8_t* p) { return get16(p) | (get16(p + 2) << 16); }

typedef struct {
    double* y;        /* [Hy][Wy][Cy] */
    double* z;        /* [Hz][Wz][Cz] */
    int16_t* zhat;
    uint8_t* iz;      /* [Cz] */
    double* mu;
    double* logsig;
    int16_t* rhat;
    uint8_t* idx;
    double* s;        /* [Hy][Wy][Cz] prior of the mean steps */
    double* yhat;     /* [Hy][Wy][Cy] the encoder's reconstruction */
} orc_debug;

int orc_latent_dims(int arch, int H, int W, int* Hy, int* Wy, int* Hz, int* Wz, int* Cy, int* Cz) {
    arch_t a;
    if (get_arch(arch, &a) || H < 1 || W < 1) return ORC_ERR_ARG;
    int hp = (H + 15) / 16 * 16, wp = (W + 15) / 16 * 16;
    *Hy = hp / 16; *Wy = wp / 16;
    *Hz = (*Hy + 3) / 4; *Wz = (*Wy + 3) / 4;
    /* two stride-2 convs with padding 1 give ceil(ceil(x/2)/2) = ceil(x/4) */
    *Cy = a.cy; *Cz = a.cz;
    return ORC_OK;
}

/* Coding options: pm = the mean-network blob (progressive means) or NULL; tw = the temporal-context blob
 * or NULL; c_in = C_i [H8][W8][Cc] (NULL: the first chunk, C = 0); c_out = C_{i+1} (may be NULL).
 * Container version = 1 + (pm != NULL) + 2 (tw != NULL). */
typedef struct {
    const float* pm;
    const float* tw;
    const double* c_in;
    double* c_out;
} orc_opts;

int orc_encode_chunk_opts(int arch, int N, const uint8_t* frames, int H, int W, int qp, int K, const float* wts,
                          const orc_opts* o, uint8_t* out, size_t cap, size_t* nbytes, orc_debug* dbg);

int orc_encode_chunk(int arch, int N, const uint8_t* frames, int H, int W, int qp, int K, const float* wts,
                     const float* pm, uint8_t* out, size_t cap, size_t* nbytes, orc_debug* dbg) {
    orc_opts o = {pm, NULL, NULL, NULL};
    return orc_encode_chunk_opts(arch, N, frames, H, W, qp, K, wts, &o, out, cap, nbytes, dbg);
}

int orc_encode_chunk_opts(int arch, int N, const uint8_t* frames, int H, int W, int qp, int K, const float* wts,
                          const orc_opts* o, uint8_t* out, size_t cap, size_t* nbytes, orc_debug* dbg) {
    const float* pm = o->pm;
    const float* tw = o->tw;
    int Hy, Wy, Hz, Wz, Cy, Cz;
    if (orc_latent_dims(arch, H, W, &Hy, &Wy, &Hz, &Wz, &Cy, &Cz) || N < 1 || N > 255 || qp < 0 || qp > 63 ||
        K < 1 || W > 65535 || H > 65535)
        return ORC_ERR_ARG;
    size_t ny = (size_t)Hy * Wy * Cy, nz = (size_t)Hz * Wz * Cz;
    double* y = dalloc(ny);
    double* z = dalloc(nz);
    int16_t* zhat = (int16_t*)malloc(2 * nz);
    uint8_t iz[256];
    double* mu = dalloc(ny);
    double* ls = dalloc(ny);
    int16_t* rhat = (int16_t*)malloc(2 * ny);
    uint8_t* idx = (uint8_t*)malloc(ny);
    uint8_t* zidx = (uint8_t*)malloc(nz);
    uint32_t* freq = (uint32_t*)malloc(sizeof(uint32_t) * NBINS * NSYM);
    uint32_t* cum = (uint32_t*)malloc(sizeof(uint32_t) * NBINS * (NSYM + 1));
    double* sp = dalloc((size_t)Hy * Wy * Cz);
    double* yh = dalloc(ny);
    double* xin = dalloc((size_t)N * H * W * 3);
    int e2 = 0, k_, c_;
    orc_layer_shape(arch, N, 2, &e2, &k_, &c_);  /* A3's width: the encoder features at 1/8 */
    double* ec = tw ? dalloc((size_t)4 * Hy * Wy * e2) : NULL;
    const int dcm = arch == 2;  /* the DC-block model carries its temporal context itself */
    double* pc = (tw || dcm) ? dalloc((size_t)Hy * Wy * Cz) : NULL;
    int rc = ORC_OK;
    orc_build_tables(freq, cum);
    orc_color_in(0, frames, N, H, W, xin);
    if (dcm) {
        orc_dc_prior_term(N, o->c_in, 2 * Hy, 2 * Wy, wts, pc);
        orc_dc_analysis(N, xin, H, W, wts, o->c_in, y);
    } else {
        if (tw) orc_context_terms(arch, N, o->c_in, 2 * Hy, 2 * Wy, tw, ec, pc);
        analysis_core(arch, N, xin, H, W, wts, ec, y);
    }
    orc_hyper_analysis(arch, N, y, Hy, Wy, wts, z);
    orc_quantize_z(z, Hz * Wz, Cz, zhat, iz);
    hyper_synthesis_core(arch, N, zhat, Hz, Wz, Hy, Wy, wts, pc, mu, ls, sp);
    orc_quantize_y(y, mu, ls, ny, qp, rhat, idx);
    if (pm) {
        double* mu0 = dalloc(ny);
        memcpy(mu0, mu, sizeof(double) * ny);
        rc = orc_progressive_means(arch, y, rhat, mu0, sp, Hy, Wy, qp, pm, yh, mu);
        free(mu0);
        if (rc) goto done;
    } else {
        double q = orc_qstep(qp);
        for (size_t i = 0; i < ny; i++) yh[i] = rhat[i] * q + mu[i];
    }
    if (dcm && o->c_out) {  /* the encoder runs the decoder's trunk to track the context */
        double* F = dalloc((size_t)4 * Hy * Wy * DC_C);
        orc_dc_trunk(N, yh, Hy, Wy, wts, o->c_in, F, o->c_out);
        free(F);
    } else if (tw && o->c_out) {  /* the encoder tracks the decoder's context: F and C_{i+1} from its own y^ */
        double* F = dalloc((size_t)4 * Hy * Wy * ORC_CF);
        orc_chunk_feature(arch, N, yh, Hy, Wy, tw, o->c_in, F);
        orc_context_next(arch, N, F, 2 * Hy, 2 * Wy, tw, o->c_out);
        free(F);
    }
    for (size_t i = 0; i < nz; i++) zidx[i] = iz[i % Cz];
    size_t hdr = (20 + (size_t)Cz + 3) / 4 * 4;
    int Kz = (size_t)K < nz ? K : (int)nz;
    if (cap < hdr) { rc = ORC_ERR_CAPACITY; goto done; }
    memset(out, 0, hdr);
    memcpy(out, "UFVC", 4);
    out[4] = (uint8_t)(1 + (pm ? 1 : 0) + ((tw || dcm) ? 2 : 0)); out[5] = (uint8_t)arch; out[6] = (uint8_t)N; out[7] = (uint8_t)qp;
    put16(out + 8, (uint32_t)W); put16(out + 10, (uint32_t)H);
    put32(out + 12, (uint32_t)K); put32(out + 16, (uint32_t)Kz);
    memcpy(out + 20, iz, Cz);
    size_t s1 = orc_rans_encode(zhat, zidx, nz, Kz, freq, cum, NSYM, RMAX, out + hdr, cap - hdr);
    if (!s1) { rc = ORC_ERR_CAPACITY; goto done; }
    size_t s2 = orc_rans_encode(rhat, idx, ny, K, freq, cum, NSYM, RMAX, out + hdr + s1, cap - hdr - s1);
    if (!s2) { rc = ORC_ERR_CAPACITY; goto done; }
    *nbytes = hdr + s1 + s2;
    if (dbg) {
        if (dbg->y) memcpy(dbg->y, y, sizeof(double) * ny);
        if (dbg->z) memcpy(dbg->z, z, sizeof(double) * nz);
        if (dbg->zhat) memcpy(dbg->zhat, zhat, 2 * nz);
        if (dbg->iz) memcpy(dbg->iz, iz, Cz);
        if (dbg->mu) memcpy(dbg->mu, mu, sizeof(double) * ny);
        if (dbg->logsig) memcpy(dbg->logsig, ls, sizeof(double) * ny);
        if (dbg->rhat) memcpy(dbg->rhat, rhat, 2 * ny);
        if (dbg->idx) memcpy(dbg->idx, idx, ny);
        if (dbg->s) memcpy(dbg->s, sp, sizeof(double) * Hy * Wy * Cz);
        if (dbg->yhat) memcpy(dbg->yhat, yh, sizeof(double) * ny);
    }
done:
    free(y); free(z); free(zhat); free(mu); free(ls); free(rhat); free(idx); free(zidx); free(freq); free(cum);
    free(sp); free(yh); free(xin); free(ec); free(pc);
    return rc;
}

/* Decode: parse the container, decode z^ (single step), hyper-synthesis -> mu, log sigma -> indices,
 * decode r^ for the whole latent in one step, y^ = r^ q + mu (version 2: the progressive means, which
 * need the mean-network blob pm), then the N frame-specific decoders.
 * frames_out: [N][H][W][3] doubles in [0, 1]; yhat_out (optional): [Hy][Wy][Cy]. */
int orc_decode_chunk_opts(int arch, int N, const uint8_t* bits, size_t nbytes, int H, int W, const float* wts,
                          const orc_opts* o, double* frames_out, double* yhat_out);

int orc_decode_chunk(int arch, int N, const uint8_t* bits, size_t nbytes, int H, int W, const float* wts,
                     const float* pm, double* frames_out, double* yhat_out) {
    orc_opts o = {pm, NULL, NULL, NULL};
    return orc_decode_chunk_opts(arch, N, bits, nbytes, H, W, wts, &o, frames_out, yhat_out);
}

/* Version 3 / 4 (temporal context) streams need o->tw and decode against o->c_in; versions 1 / 2 need
 * tw == NULL.  With tw, c_out receives C_{i+1}. */
int orc_decode_chunk_opts(int arch, int N, const uint8_t* bits, size_t nbytes, int H, int W, const float* wts,
                          const orc_opts* o, double* frames_out, double* yhat_out) {
    const float* pm = o->pm;
    const float* tw = o->tw;
    int Hy, Wy, Hz, Wz, Cy, Cz;
    if (orc_latent_dims(arch, H, W, &Hy, &Wy, &Hz, &Wz, &Cy, &Cz)) return ORC_ERR_ARG;
    size_t hdr = (20 + (size_t)Cz + 3) / 4 * 4;
    if (nbytes < hdr || memcmp(bits, "UFVC", 4) || bits[4] < 1 || bits[4] > 4) return ORC_ERR_CORRUPT;
    const int v_pm = bits[4] == 2 || bits[4] == 4, v_tc = bits[4] >= 3, dcm = arch == 2;
    if ((v_pm && !pm) || (v_tc != (tw != NULL || dcm))) return ORC_ERR_ARG;
    if (bits[5] != arch || bits[6] != N || get16(bits + 8) != (uint32_t)W || get16(bits + 10) != (uint32_t)H)
        return ORC_ERR_ARG;
    int qp = bits[7];
    int K = (int)get32(bits + 12), Kz = (int)get32(bits + 16);
    size_t ny = (size_t)Hy * Wy * Cy, nz = (size_t)Hz * Wz * Cz;
    if (qp > 63 || K < 1 || Kz != ((size_t)K < nz ? K : (int)nz)) return ORC_ERR_CORRUPT;
    for (int c = 0; c < Cz; c++)
        if (bits[20 + c] >= NBINS) return ORC_ERR_CORRUPT;
    uint32_t* freq = (uint32_t*)malloc(sizeof(uint32_t) * NBINS * NSYM);
    uint32_t* cum = (uint32_t*)malloc(sizeof(uint32_t) * NBINS * (NSYM + 1));
    orc_build_tables(freq, cum);
    int16_t* zhat = (int16_t*)malloc(2 * nz);
    uint8_t* zidx = (uint8_t*)malloc(nz);
    for (size_t i = 0; i < nz; i++) zidx[i] = bits[20 + i % Cz];
    double* mu = dalloc(ny);
    double* ls = dalloc(ny);
    uint8_t* idx = (uint8_t*)malloc(ny);
    int16_t* rhat = (int16_t*)malloc(2 * ny);
    double* yhat = dalloc(ny);
    double* sp = dalloc((size_t)Hy * Wy * Cz);
    double* pc = (tw || dcm) ? dalloc((size_t)Hy * Wy * Cz) : NULL;
    double* F = (tw || dcm) ? dalloc((size_t)4 * Hy * Wy * (dcm ? DC_C : ORC_CF)) : NULL;
    size_t used1 = 0, used2 = 0;
    int rc = orc_rans_decode(bits + hdr, nbytes - hdr, zidx, nz, Kz, freq, cum, NSYM, RMAX, zhat, &used1);
    if (rc) goto done;
    if (dcm) orc_dc_prior_term(N, o->c_in, 2 * Hy, 2 * Wy, wts, pc);
    else if (tw) orc_context_terms(arch, N, o->c_in, 2 * Hy, 2 * Wy, tw, NULL, pc);
    hyper_synthesis_core(arch, N, zhat, Hz, Wz, Hy, Wy, wts, pc, mu, ls, sp);
    orc_scale_index(ls, ny, qp, idx);
    rc = orc_rans_decode(bits + hdr + used1, nbytes - hdr - used1, idx, ny, K, freq, cum, NSYM, RMAX, rhat, &used2);
    if (rc) goto done;
    if (hdr + used1 + used2 != nbytes) { rc = ORC_ERR_CORRUPT; goto done; }
    if (v_pm) {
        double* mu_used = dalloc(ny);
        rc = orc_progressive_means(arch, NULL, rhat, mu, sp, Hy, Wy, qp, pm, yhat, mu_used);
        free(mu_used);
        if (rc) goto done;
    } else {
        double q = orc_qstep(qp);
        for (size_t i = 0; i < ny; i++) yhat[i] = rhat[i] * q + mu[i];
    }
    if (yhat_out) memcpy(yhat_out, yhat, sizeof(double) * ny);
    if (dcm) {
        orc_dc_trunk(N, yhat, Hy, Wy, wts, o->c_in, F, o->c_out);
        if (frames_out) orc_dc_frames(N, F, 2 * Hy, 2 * Wy, H, W, wts, frames_out);
    } else {
        if (tw) {
            orc_chunk_feature(arch, N, yhat, Hy, Wy, tw, o->c_in, F);
            if (o->c_out) orc_context_next(arch, N, F, 2 * Hy, 2 * Wy, tw, o->c_out);
        }
        if (frames_out) synthesis_core(arch, N, yhat, Hy, Wy, H, W, wts, F, tw, frames_out);
    }
done:
    free(freq); free(cum); free(zhat); free(zidx); free(mu); free(ls); free(idx); free(rhat); free(yhat); free(sp);
    free(pc); free(F);
    return rc;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
