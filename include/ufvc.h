/*
 * ufvc.h -- C ABI of the B300 (sm_103a) chunk-coding library libufvc.so.
 *
 * The library codes one chunk of N video frames through ONE shared latent, following the paper
 * "Ultra-Fast Neural Video Compression" (DCVC-UF):
 *   Sec. 3.1, Fig. 3  -- chunk X_i = {x_i,0..x_i,N-1} -> patch embedding -> chunk encoder with
 *                        cross-frame interaction -> latent y_i -> quantised y^_i -> bit-stream; qp_i
 *                        is the rate input;
 *   Sec. 3.2          -- N frame-specific decoders reconstruct all frames of the chunk in parallel;
 *   Sec. 3.4, Fig. 4c -- r^ = round(y - mu) is entropy coded with the scale sigma only, y^ = r^ + mu,
 *                        and the scales of ALL latent elements come from one parameter-estimation
 *                        pass, so the whole latent is entropy coded in a single step.
 * The module internals are figure-only in the paper; this library implements the plain reading
 * (strided 3x3 convolutions + GELU, one residual cross-frame interaction block, a hyperprior whose
 * synthesis outputs (mu, log sigma), and conv / residual / pixel-shuffle decoders), a 64-bin scale
 * index into fixed 16-bit integer Gaussian CDF tables, and K interleaved rANS lanes.
 *
 * Conventions (all entry points):
 *   - Every buffer is owned by the caller.  "d_" pointers are CUDA device pointers on the context's
 *     device; "h_" pointers are host pointers.  The library keeps no pointer after a call returns,
 *     except that asynchronous work on the given stream reads / writes the buffers until it completes.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream.  Calls are
 *     stream-ordered and asynchronous unless documented otherwise.
 *   - Argument errors are detected on the host and returned before any launch (UFVC_ERR_ARG).
 *     Errors found on the device (corrupt bit-stream, too-small capacity) set a status word in the
 *     context; ufvc_sync_status() synchronises the stream and returns (and clears) it.
 *   - A context is not thread-safe: use one per host thread, or lock around calls.
 *   - Layouts are NHWC with the channel fastest.  Frames are uint8 RGB [N][H][W][3].
 */
#ifndef UFVC_H
#define UFVC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ufvc_ctx ufvc_ctx;
typedef struct ufvc_server ufvc_server;

typedef enum {
    UFVC_OK = 0,
    UFVC_ERR_ARG = 1,          /* invalid argument (checked on the host, nothing launched) */
    UFVC_ERR_CAPACITY = 2,     /* output buffer too small for the bit-stream */
    UFVC_ERR_CORRUPT = 3,      /* bit-stream header / lane counts / lane final state inconsistent */
    UFVC_ERR_OOM = 4,          /* device allocation failed */
    UFVC_ERR_CUDA = 5,         /* a CUDA call failed (see ufvc_last_error) */
    UFVC_ERR_TIMEOUT = 6,      /* a bounded device or host wait gave up */
    UFVC_ERR_UNSUPPORTED = 7,  /* configuration not supported on this device */
    UFVC_PENDING = 8           /* serving: request not finished yet */
} ufvc_status;

typedef enum {
    UFVC_FP32 = 0,  /* every convolution in FP32 on CUDA cores (deterministic) */
    UFVC_BF16 = 1,  /* analysis, hyper-analysis and decoder convolutions: BF16 operands on tcgen05
                       tensor cores, FP32 accumulation in TMEM; the entropy-parameter path (hyper-
                       synthesis) stays deterministic FP32.  arch 1 and 2 (all activation widths
                       multiples of 64); arch 0 gives UFVC_ERR_UNSUPPORTED */
    UFVC_FP8 = 2    /* as BF16 but the tensor-core layers (all except the final frame layer, which
                       stays BF16) take E4M3 operands: weights with one scale per output channel
                       (absmax / 448), activations with one scale per tensor from
                       ufvc_calibrate_fp8; FP32 accumulation.  Needs calibration before use.
                       arch 1 only */
} ufvc_precision;

typedef struct {
    int arch;        /* 0: tiny widths (analysis 64/96/128, Cy=128, Cz=64);
                        1: 1080p-family widths (analysis 64/128/192, Cy=256, Cz=128);
                        2: the DC-block model at the paper's HT-S block counts (Appendix): every
                           module built from depth-wise convolution blocks, Cy=256, Cz=128, with the
                           temporal chunk context built in (see "DC-block model" below) */
    int chunk_len;   /* N, frames per chunk (1..16); N frame-specific decoders */
    int lanes;       /* K, interleaved rANS lanes of the latent section (1..65536) */
    int precision;   /* ufvc_precision */
    int device;      /* CUDA device ordinal */
} ufvc_config;

/* Number of float32 weights the architecture needs (the blob layout is documented at
 * ufvc_create). */
size_t ufvc_weight_count(int arch, int chunk_len);

/* Create a context: copies the weights to the device, builds the CDF and threshold tables on the
 * host in FP64 and uploads them.  `weights` is a host float32 blob: for each layer in the order
 *   A1 A2 A3 Xa Xb A4 H1 H2 S1 S2 S3, then for f = 0..N-1: D0 R1a R1b U1 R2a R2b U2 U3,
 * the kernel [Cout][k][k][Cin] followed by the bias [Cout] (shapes: see ufvc_layer_shape).
 * Returns UFVC_ERR_ARG if n_weights != ufvc_weight_count(arch, chunk_len).
 *
 * DC-block model (arch 2).  A DC block of width C is y = x + PWb(GELU(DW(PWa(x)))), then
 * y + PWd(GELU(PWc(y))) with PWa, PWb 1x1 C -> C, DW a 3x3 depth-wise layer (one filter per channel,
 * stored as kernel [C][3][3][1]), PWc 1x1 C -> 2C, PWd 1x1 2C -> C (a reading of the paper's block
 * figure).  At 1/8 of the padded frame size: patch embedding PE (1x1 over the 8x8 space-to-depth of the
 * N stacked frames, channel (3n + c) 64 + 8 dy + dx), EC(C_i), 6 blocks at 512, ED (3x3 stride 2) -> y;
 * the plain hyperprior with PC(C_i) added before S3; chunk decoder GELU(PS(DU(y^))) + FC(C_i), 7 blocks
 * -> F; context generation: 11 blocks on F, GO (1x1) -> C_{i+1} (128 channels); frame decoder f: FP_f
 * (1x1 512 -> 256), 3 blocks at 256, FO_f (1x1 -> 192), pixel shuffle x8, x^ = clamp(0.5 + o, 0, 1).
 * Blob order: PE, EC, 6 x [PWa DW PWb PWc PWd], ED, H1, H2, S1, S2, S3, PC, DU, FC, 7 x [...],
 * 11 x [...], GO, then per frame FP, 3 x [...], FO.  The context is always carried: the plain chunk
 * calls code a stream's first chunk, the _tc calls carry C_i (ufvc_context_bytes: 128 channels).
 * BF16 and FP32 only. */
ufvc_status ufvc_create(const ufvc_config* cfg, const float* weights, size_t n_weights, ufvc_ctx** out);
void ufvc_destroy(ufvc_ctx* ctx);

/* Shape (Cout, k, Cin) of blob layer l (0-based, order above). */
ufvc_status ufvc_layer_shape(int arch, int chunk_len, int layer, int* cout, int* k, int* cin);

/* Latent geometry of a W x H chunk: frames are replicate-padded to multiples of 16; the latent is
 * [Hy][Wy][Cy] with Hy = ceil(H/16), Wy = ceil(W/16); the hyper-latent [Hz][Wz][Cz] with
 * Hz = ceil(Hy/4), Wz = ceil(Wy/4). */
ufvc_status ufvc_latent_dims(int arch, int width, int height, int* Hy, int* Wy, int* Hz, int* Wz, int* Cy,
                             int* Cz);

/* Upper bound of the bit-stream size of one W x H chunk (header + two sections, at most one 16-bit
 * word per symbol plus two flush words and one 32-bit count per lane). */
size_t ufvc_max_bitstream_bytes(const ufvc_ctx* ctx, int width, int height);

/* Encode one chunk (Sec. 3.1 / 3.4).  d_frames: device uint8 [N][H][W][3], N = chunk_len.
 * qp in [0, 63] sets the quantisation step q = 2^((qp-32)/8).  The bit-stream is written to d_bits
 * (capacity bytes) and its size to *d_nbytes (device uint64).  If the stream would not fit,
 * nothing past `capacity` is written and the status word becomes UFVC_ERR_CAPACITY.
 * Bit-stream layout: "UFVC", u8 version (1, + 1 with progressive means, + 2 with the temporal context;
 * see ufvc_set_progressive_means and ufvc_set_temporal_context),
 * u8 arch, u8 N, u8 qp, u16 W, u16 H, u32 K, u32 Kz,
 * Cz bytes of per-channel hyper-latent scale indices, zero padding to 4 bytes; then the z^ section
 * (Kz = min(K, #z^) lanes) and the y^ section (K lanes), each = K u32 lane word counts followed by
 * the lane streams (u16 words in decoding order), zero-padded to 4 bytes.  Little-endian. */
ufvc_status ufvc_encode_chunk(ufvc_ctx* ctx, const uint8_t* d_frames, int n_frames, int width, int height,
                              int qp, uint8_t* d_bits, size_t capacity, uint64_t* d_nbytes, void* stream);

/* Decode one chunk: one entropy-decoding step for z^, the hyper-synthesis (mu, log sigma for every
 * latent element in one pass), one entropy-decoding step for the whole latent, y^ = r^ q + mu, then
 * the N frame-specific decoders (Sec. 3.2) in parallel.  nbytes = the stream size (the number the
 * encoder wrote); n_frames / width / height must match the header (else status UFVC_ERR_ARG on the
 * device).  d_frames: device uint8 [N][H][W][3], x^ = clamp(0.5 + o, 0, 1) scaled by 255 and rounded
 * half-to-even.  The _f32 variant writes x^ in [0, 1] as float32 instead. */
ufvc_status ufvc_decode_chunk(ufvc_ctx* ctx, const uint8_t* d_bits, size_t nbytes, uint8_t* d_frames,
                              int n_frames, int width, int height, void* stream);
ufvc_status ufvc_decode_chunk_f32(ufvc_ctx* ctx, const uint8_t* d_bits, size_t nbytes, float* d_frames,
                                  int n_frames, int width, int height, void* stream);

/* As ufvc_decode_chunk for a bit-stream whose size is known only on the device, as ufvc_encode_chunk
 * left it in *d_nbytes: reads stay within `capacity` bytes of d_bits and the stream must end exactly
 * at *d_nbytes (else status UFVC_ERR_CORRUPT).  Nothing is read back to the host, so the call can be
 * captured in a CUDA graph and replayed for every stream that the same buffers carry. */
ufvc_status ufvc_decode_chunk_dev(ufvc_ctx* ctx, const uint8_t* d_bits, size_t capacity, const uint64_t* d_nbytes,
                                  uint8_t* d_frames, int n_frames, int width, int height, void* stream);

/* Host-buffer variants (the call a user without device buffers makes): copy h_frames / h_bits to a
 * context-owned device staging area, run the chunk on `stream`, copy the result back, synchronise.
 * *nbytes receives the stream size.  Return the device status of the call. */
ufvc_status ufvc_encode_chunk_host(ufvc_ctx* ctx, const uint8_t* h_frames, int n_frames, int width, int height,
                                   int qp, uint8_t* h_bits, size_t capacity, size_t* nbytes, void* stream);
ufvc_status ufvc_decode_chunk_host(ufvc_ctx* ctx, const uint8_t* h_bits, size_t nbytes, uint8_t* h_frames,
                                   int n_frames, int width, int height, void* stream);

/* ---- pipelined host-buffer round trips (streaming callers) ----
 * A pipeline of `depth` slots (1..16) of device buffers, one context sharing ctx's weights and tables
 * (own plans and status word), one compute stream and four copy streams; ctx must outlive it and stay
 * unchanged meanwhile.  ufvc_pipe_submit enqueues one chunk's round trip on slot ticket % depth and
 * returns at once: h_frames (ctx's colour format) to the device, ufvc_encode_chunk, the whole bit-stream
 * buffer (`capacity` bytes, at least ufvc_max_bitstream_bytes) to h_bits, that host copy back to the
 * device, ufvc_decode_chunk_dev of it, and the decoded frames to h_out (skipped when h_out is NULL).
 * The kernels run one chunk at a time on the compute stream; a ticket's decode is enqueued after the
 * next ticket's encode, or after the second next one's with depth >= 5 (or by its wait), so the copies of
 * the other tickets and the bit-stream's trip through the host overlap the kernels.  Host buffers must stay valid and unchanged until the
 * ticket has been waited for; page-locked host memory makes the copies asynchronous.  *ticket gets
 * consecutive numbers from 0.  UFVC_ERR_ARG if ticket t - depth has not been waited for yet,
 * UFVC_ERR_CAPACITY if capacity is too small.  ufvc_pipe_wait blocks until the ticket's round trip has
 * completed and returns its device status; *nbytes gets the stream size (the first *nbytes bytes of
 * h_bits are the bit-stream).  Each ticket is waited for once. */
typedef struct ufvc_pipe ufvc_pipe;
ufvc_status ufvc_pipe_create(ufvc_ctx* ctx, int depth, ufvc_pipe** out);
ufvc_status ufvc_pipe_submit(ufvc_pipe* pipe, const uint8_t* h_frames, int n_frames, int width, int height, int qp,
                             uint8_t* h_bits, size_t capacity, uint8_t* h_out, long long* ticket);
ufvc_status ufvc_pipe_wait(ufvc_pipe* pipe, long long ticket, size_t* nbytes);
void ufvc_pipe_destroy(ufvc_pipe* pipe);

/* Batched chunk calls for serving (the paper has no counterpart: it codes chunk after chunk).  `batch`
 * (1..8) chunks of the same size, each with its own buffers (host arrays of `batch` device pointers; the
 * encoder takes one rate per chunk in qps, the decoder reads each stream's size from d_nbytes[b] on the
 * device, as ufvc_decode_chunk_dev does).  Every chunk runs its own analysis, hyperprior and synthesis
 * launches; the entropy coding of all chunks is shared: one launch codes and lays out the 2 x batch
 * sections, one launch decodes the batch's z^ sections and one its y^ sections, so the latency-bound lane
 * chains of the chunks run side by side on the SMs instead of one after another.  The bit-streams and
 * frames are byte for byte those of the single-chunk calls.  Each batch position has its own per-size
 * buffers (allocated on first use).  UFVC_ERR_UNSUPPORTED for batch > 1 in a context with a temporal
 * context (every stream carries its own). */
ufvc_status ufvc_encode_chunks(ufvc_ctx* ctx, int batch, const uint8_t* const* d_frames, int n_frames, int width,
                               int height, const int* qps, uint8_t* const* d_bits, size_t capacity,
                               uint64_t* const* d_nbytes, void* stream);
ufvc_status ufvc_decode_chunks(ufvc_ctx* ctx, int batch, const uint8_t* const* d_bits, size_t capacity,
                               const uint64_t* const* d_nbytes, uint8_t* const* d_frames, int n_frames, int width,
                               int height, void* stream);

/* Synchronise `stream`, then return and clear the device status word (UFVC_OK if no device-side
 * error was recorded since the last call). */
ufvc_status ufvc_sync_status(ufvc_ctx* ctx, void* stream);

/* ---- stage entry points (tests and benchmarks call these; same kernels as the chunk calls) ---- */

/* Encoder front half: d_y float32 [Hy][Wy][Cy] (latent before quantisation), d_zhat int16
 * [Hz][Wz][Cz] (z^ = clamp(rint(z), -255, 255)), d_iz uint8 [Cz] (per-channel z^ scale index),
 * d_mu / d_logsig float32 [Hy][Wy][Cy], d_rhat int16 and d_idx uint8 [Hy][Wy][Cy].  Any output
 * pointer may be NULL. */
ufvc_status ufvc_encode_stages(ufvc_ctx* ctx, const uint8_t* d_frames, int width, int height, int qp, float* d_y,
                               int16_t* d_zhat, uint8_t* d_iz, float* d_mu, float* d_logsig, int16_t* d_rhat,
                               uint8_t* d_idx, void* stream);

/* Hyper-synthesis alone (single-step parameter estimation, Sec. 3.4), deterministic FP32 with a fixed
 * reduction order: d_zhat int16 [Hz][Wz][Cz] -> d_mu, d_logsig float32 [Hy][Wy][Cy]. */
ufvc_status ufvc_hyper_synthesis(ufvc_ctx* ctx, const int16_t* d_zhat, int Hz, int Wz, int Hy, int Wy,
                                 float* d_mu, float* d_logsig, void* stream);

/* ---- colour interface (Appendix: the model reads and writes YUV444; RGB and YUV420 are converted) ----
 * The frame buffers of the chunk calls (d_frames / h_frames of encode and decode) hold N frames in the
 * context's colour format, ufvc_frame_bytes(format, W, H) bytes each (float32 values in [0, 1] instead of
 * bytes for ufvc_decode_chunk_f32):
 *   UFVC_COLOR_RGB       RGB interleaved [H][W][3], fed to the network as its three channels (default);
 *   UFVC_COLOR_RGB_BT709 RGB interleaved [H][W][3], converted to YUV444 with BT.709 (full range, chroma
 *                        centred at 0.5: Y = 0.2126 R + 0.7152 G + 0.0722 B, U = (B - Y) / 1.8556 + 0.5,
 *                        V = (R - Y) / 1.5748 + 0.5) before the network and back (clamped) after it;
 *   UFVC_COLOR_YUV444P   YUV444 planar [3][H][W];
 *   UFVC_COLOR_YUV420P   YUV420 planar: Y [H][W], U and V [ceil(H/2)][ceil(W/2)]; each chroma sample
 *                        serves its 2x2 block on input, and on output is the mean of the block's pixels
 *                        inside the frame.
 * Decoded values are x^ = clamp(0.5 + o, 0, 1) converted to the format; bytes are rint(255 v).  The
 * bit-stream does not record the format: it codes the network's channels, and the decoding context's
 * format decides the output conversion. */
typedef enum { UFVC_COLOR_RGB = 0, UFVC_COLOR_RGB_BT709 = 1, UFVC_COLOR_YUV444P = 2, UFVC_COLOR_YUV420P = 3 } ufvc_color;

/* Bytes of one frame of width x height in `format` (0 for an unknown format). */
size_t ufvc_frame_bytes(int format, int width, int height);

/* Set the context's colour format (ufvc_color); it applies to the calls that follow.  UFVC_ERR_ARG for an
 * unknown format.  No device work. */
ufvc_status ufvc_set_color_format(ufvc_ctx* ctx, int format);

/* ---- temporal chunk context (Sec. 3.1, Fig. 3) ----
 * Chunk i of a stream is coded conditioned on a context C_i that the decoder generated from chunk i-1:
 * the chunk feature F_i = GELU(PS(FD(y^_i))) + FC(C_i) (64 channels at 1/8 of the padded frame size) feeds
 * the frame-specific decoders (each adds its 1x1 projection DF_f(F_i) to its first layer's output) and
 * gives the next context C_{i+1} = GELU(CG(F_i)) (64 channels at 1/8 size).  The encoder adds EC(C_i)
 * (1x1) to its patch-embedded features before the cross-frame interaction, and the prior adds PC(C_i)
 * (3x3 stride 2) to the hyper-synthesis features before their last layer, so the scales depend on C_i:
 * a chunk decodes only against the context its encoder used.  The encoder recomputes F_i and C_{i+1} from
 * its own y^ = r^ q + mu, so it tracks the decoder's context exactly (same kernels, same inputs; the
 * context is in the context's activation type, so a stream decodes in a context of the same precision).
 * A stream's first chunk uses C_0 = 0.  Layer shapes (a reading of the figure on the plain layers):
 * EC 1x1 64 -> e2, FD 3x3 Cy -> 256 (pixel shuffle), FC 1x1 64 -> 64, CG 3x3 64 -> 64, PC 3x3/2 64 -> Cz,
 * DF_f 1x1 64 -> Cd1.  Streams coded this way have container version 3 (4 with progressive means). */

/* Floats of the temporal blob: EC FD FC CG PC, then DF_f for f = 0..chunk_len-1, each the kernel
 * [Cout][k][k][Cin] followed by the bias [Cout]. */
size_t ufvc_temporal_weight_count(int arch, int chunk_len);

/* Give the context the temporal-context layers (host blob, uploaded; the caller keeps it).  From then on
 * every chunk call codes version-3/4 streams; ufvc_encode_chunk / ufvc_decode_chunk act as a stream's
 * first chunk (C = 0, next context discarded) and the _tc calls below carry the context.  A context
 * without it reports UFVC_ERR_UNSUPPORTED (status word) for version 3/4 and one with it for version 1/2.
 * Not for FP8 contexts (UFVC_ERR_UNSUPPORTED).  Call once, before the context is shared. */
ufvc_status ufvc_set_temporal_context(ufvc_ctx* ctx, const float* weights, size_t n_weights);

/* Bytes of one context buffer for width x height chunks: [ceil(H/16) 2][ceil(W/16) 2][64] of bf16 (BF16
 * contexts) or float32 (FP32 contexts). */
size_t ufvc_context_bytes(const ufvc_ctx* ctx, int width, int height);

/* Chunk calls with the stream's context: d_ctx_in = C_i (device, ufvc_context_bytes; NULL for the first
 * chunk of a stream), d_ctx_out = receives C_{i+1} (NULL: not wanted).  Both 16-byte aligned and distinct;
 * the caller owns them (double-buffer them across chunks).  Otherwise as ufvc_encode_chunk /
 * ufvc_decode_chunk(_f32) (f32 != 0: float frames); with d_nbytes (device) the stream size is read on the
 * device and nbytes is the readable capacity, as in ufvc_decode_chunk_dev.  UFVC_ERR_ARG without
 * ufvc_set_temporal_context. */
ufvc_status ufvc_encode_chunk_tc(ufvc_ctx* ctx, const uint8_t* d_frames, int n_frames, int width, int height, int qp,
                                 uint8_t* d_bits, size_t capacity, uint64_t* d_nbytes, const void* d_ctx_in,
                                 void* d_ctx_out, void* stream);
ufvc_status ufvc_decode_chunk_tc(ufvc_ctx* ctx, const uint8_t* d_bits, size_t nbytes, const uint64_t* d_nbytes,
                                 void* d_frames, int f32, int n_frames, int width, int height, const void* d_ctx_in,
                                 void* d_ctx_out, void* stream);
/* ufvc_encode_stages against the context C_i (d_ctx_in, NULL = first chunk). */
ufvc_status ufvc_encode_stages_tc(ufvc_ctx* ctx, const uint8_t* d_frames, int width, int height, int qp,
                                  const void* d_ctx_in, float* d_y, int16_t* d_zhat, uint8_t* d_iz, float* d_mu,
                                  float* d_logsig, int16_t* d_rhat, uint8_t* d_idx, void* stream);

/* ---- progressive means (Sec. 3.4, Fig. 4a and 4c) ----
 * The latent is split into four partitions: channel group g = c / (Cy / 4), position t = 2 (h mod 2)
 * + (w mod 2) in its 2x2 block, partition (t + g) mod 4 (a reading of the paper's figure).  The single
 * parameter pass gives every scale and the means of partition 0; the means of partitions 1, 2, 3 then
 * come one partition at a time from a small network over the partitions already reconstructed and the
 * hyper-synthesis features s (S2's output, [Hy][Wy][Cz]):
 *     mu^k = P_k,b(GELU(P_k,a([y^ on partitions < k, zero elsewhere ; s])))     k = 1, 2, 3
 * with P_k,a a 3x3 convolution Cy + Cz -> Cz and P_k,b a 1x1 convolution Cz -> Cy.  Partition k is
 * quantised with mu^k (r^ = clamp(rint((y - mu^k) / q))) and reconstructed as y^ = r^ q + mu^k.  The
 * scales, and so the single entropy-coding step, are unchanged; the decoder repeats the steps after
 * it and reproduces the encoder's means exactly (same kernels, same inputs). */

/* Number of floats of the mean-network blob: for P1a P1b P2a P2b P3a P3b the kernel [Cout][k][k][Cin]
 * followed by the bias [Cout]. */
size_t ufvc_mean_weight_count(int arch);

/* Give the context the mean network (host float32 blob of ufvc_mean_weight_count(arch) floats; it is
 * uploaded, the caller keeps ownership).  From then on ufvc_encode_chunk writes version-2 streams, and
 * the decode calls accept version 1 (single-pass means) and version 2.  A context without it reports
 * UFVC_ERR_UNSUPPORTED (status word) for a version-2 stream.  Call once, before the context is shared
 * (servers, clones); UFVC_ERR_ARG on a count mismatch or a second call.  The mean network runs on bf16
 * operands on the tensor cores in BF16 and FP8 contexts and on the FP32 SIMT kernel in FP32 contexts. */
ufvc_status ufvc_set_progressive_means(ufvc_ctx* ctx, const float* weights, size_t n_weights);

/* The progressive steps alone, for tests.  Encoder form (d_y != NULL): d_y, d_mu0 float32 [Hy][Wy][Cy],
 * d_s float32 [Hy][Wy][Cz] -> d_rhat int16 (every partition quantised with its mean), d_mu float32 (the
 * mean each element is coded with), d_yhat float32 = r^ q + mu.  Decoder form (d_y == NULL): d_rhat_in
 * gives r^ (copied to d_rhat).  Synchronises `stream`; needs ufvc_set_progressive_means. */
ufvc_status ufvc_progressive_means(ufvc_ctx* ctx, const float* d_y, const int16_t* d_rhat_in, const float* d_mu0,
                                   const float* d_s, int Hy, int Wy, int qp, int16_t* d_rhat, float* d_mu,
                                   float* d_yhat, void* stream);

/* Quantise + scale index (Sec. 3.4): r^ = clamp(rint((y - mu) / q), -255, 255) (FP32, no FMA
 * contraction), idx = #{k : thr_qp[k] < log sigma}.  n elements, all device buffers. */
ufvc_status ufvc_quantize(ufvc_ctx* ctx, const float* d_y, const float* d_mu, const float* d_logsig, size_t n,
                          int qp, int16_t* d_rhat, uint8_t* d_idx, void* stream);

/* Frame-specific synthesis (Sec. 3.2) from a dequantised latent d_yhat float32 [Hy][Wy][Cy] to
 * d_frames float32 [N][H][W][3] in [0, 1]. */
ufvc_status ufvc_synthesize(ufvc_ctx* ctx, const float* d_yhat, int width, int height, float* d_frames,
                            void* stream);

/* One rANS section (the single consolidated coding step, Sec. 3.4) over n symbols with the context's
 * 64 Gaussian tables: symbol i in [-255, 255] uses table d_idx[i] (0..63) and goes to lane i mod
 * lanes.  Encode writes the section (lanes u32 word counts + lane streams, zero-padded to 4 bytes)
 * to d_out and its byte size to *d_nbytes; decode reads a section of at most `nbytes` bytes.
 * Errors (capacity / corrupt) go to the status word. */
ufvc_status ufvc_rans_encode(ufvc_ctx* ctx, const int16_t* d_sym, const uint8_t* d_idx, size_t n, int lanes,
                             uint8_t* d_out, size_t capacity, uint64_t* d_nbytes, void* stream);
ufvc_status ufvc_rans_decode(ufvc_ctx* ctx, const uint8_t* d_in, size_t nbytes, const uint8_t* d_idx, size_t n,
                             int lanes, int16_t* d_sym, void* stream);

/* One convolution of the context's weights, for layer-level tests: blob layer `layer` (decoder layers
 * of frame f are 11 + 8 f + j) applied to d_in [H][W][Cin_s] with zero padding k/2 and `stride`;
 * act = 1 applies GELU; mode 0 writes NHWC [out_h][out_w][Cout], mode 1 pixel-shuffles x2 into
 * [out_h][out_w][Cout/4] (positions outside out_h x out_w are dropped), mode 2 writes
 * clamp(0.5 + o, 0, 1) pixel-shuffled as float, mode 3 writes NHWC like mode 0 plus the residual that
 * d_out holds on entry, in place (as the decoders' second residual-block convolutions R1b and R2b run,
 * Sec. 3.2; d_out in the tensor layout of d_out for mode 0).  In FP32 precision (and for the hyper-synthesis
 * layers S1 S2 S3) tensors are float with Cin_s = Cin rounded up to 16; otherwise they are bf16 with
 * Cin_s rounded up to 64 (32 for a layer with at most 32 input channels, i.e. the first layer for
 * N <= 10) and the layer runs on the tensor cores (stride 2 needs even H and W).  In FP8 precision the
 * tensors are E4M3 codes of the calibrated scales (Cin_s rounded up to 64).  The tensor-core weights of the
 * pixel-shuffle decoder layers (D0, U1, U2) are stored for mode 1 only: another mode on them returns
 * UFVC_ERR_ARG. */
ufvc_status ufvc_conv_layer(ufvc_ctx* ctx, int layer, const void* d_in, int H, int W, int stride, int act, int mode,
                            void* d_out, int out_h, int out_w, void* stream);

/* Test hook for the timeout path of the entropy kernels (the paper has no counterpart: a library
 * facility).  Every rANS encode and decode launch first copies the coding tables into shared memory and
 * waits for the copy for a bounded time; `cycles` sets that bound in SM clocks (0 restores the default,
 * about 2 s).  A wait that runs out records UFVC_ERR_TIMEOUT in the status word (ufvc_sync_status),
 * the kernel returns without coding, an encoder's lanes are laid out empty, and the context stays usable.
 * Synchronous, no device work. */
ufvc_status ufvc_set_table_wait_limit(ufvc_ctx* ctx, long long cycles);

/* Kernel selection for the decoders' pixel-shuffle layers (D0, U1, U2 at 256 accumulator columns, Sec. 3.2
 * frame decoders) on the tensor cores: enable = 1 (the default) runs them on pairs of SMs that share one
 * MMA of 256 pixels (each SM loads its 128 pixels and half of the weights), 0 on one SM per 128-pixel tile.
 * Both compute every output from the same bf16 operands with FP32 accumulation; layer outputs agree to
 * the accumulation order.  UFVC_ERR_ARG for other values.  Synchronous, no device work. */
ufvc_status ufvc_set_conv_pairs(ufvc_ctx* ctx, int enable);

/* The first analysis layer read straight from the frame bytes (the patch embedding of the stacked chunk,
 * Sec. 3.1: frame n's three channels become channels 3n .. 3n+2 of one input, replicate-padded to a
 * multiple of 16, then A1 = 3x3 stride-2 convolution + GELU), as the BF16 and FP8 chunk encoders run it
 * (the FP8 encoder with the same bf16 operands, writing E4M3 codes instead): d_frames
 * holds N frames in the context's colour format (RGB, YUV444P or YUV420P; YUV420 chroma repeated over
 * its 2x2 block), d_out receives bf16 NHWC [ceil16(H)/2][ceil16(W)/2][64].  The bytes enter as v / 256
 * (exact in bf16) and the bf16 weights carry 256 / 255, so the operands are bf16(w * 256 / 255) and
 * v / 256.  kernel: 0 = the kernel the chunk encoder picks, 1 = the register-staged kernel (every
 * format and width), 2 = the TMA-window kernel (interleaved RGB whose rows are a multiple of 16 bytes
 * and start 16-byte aligned; UFVC_ERR_ARG otherwise).  UFVC_ERR_UNSUPPORTED for contexts whose first
 * layer does not read the frame bytes (FP32, an odd chunk length or one above 8, or BT.709 RGB
 * input).  Asynchronous on `stream`; device-side errors go to the status word. */
ufvc_status ufvc_first_layer(ufvc_ctx* ctx, const uint8_t* d_frames, int width, int height, int kernel, void* d_out,
                             void* stream);

/* Allocation-free variant of ufvc_rans_encode (the paper has no counterpart: this is a library
 * facility).  Same arguments, same output bytes, same error reporting, but it never allocates:
 * ufvc_rans_encode may call cudaMalloc for its staging rows, which callers in real-time loops that cannot
 * absorb cudaMalloc's implicit device synchronisation, and callers whose device memory belongs to their
 * own pool allocator, cannot accept.  The staging space is one fixed 24 MiB array per device, held by
 * every GPU that loads this library until the process exits; a call needs 8448 bytes for its layout
 * control block plus 2 * lanes * (n / lanes + 3) bytes of staging rows (rounded up to 256), which allows
 * roughly 12.5 million symbols, and returns UFVC_ERR_ARG (message in ufvc_last_error) beyond that.  The
 * first call on a device looks up the array's device address (cudaGetSymbolAddress, with that device
 * current); make that first call before any stream capture.  All calls on a device share the array and it
 * keeps the last call's contents; each call clears the control block on `stream` before its launch (a
 * memset, not an allocation), and the rows need no clearing.  Calls whose work can overlap on the GPU
 * (different streams, or the same stream without ordering) race. */
ufvc_status ufvc_rans_encode_noalloc(ufvc_ctx* ctx, const int16_t* d_sym, const uint8_t* d_idx, size_t n, int lanes,
                                     uint8_t* d_out, size_t capacity, uint64_t* d_nbytes, void* stream);

/* Host copies of the tables the context uses: freq / cum uint32 [64][511] / [64][512] (may be NULL),
 * thr float32 [63] for rate qp (may be NULL).  No device work.  ctx may be NULL: the tables are then
 * built on the host (FP64) without touching any device. */
ufvc_status ufvc_get_tables(const ufvc_ctx* ctx, uint32_t* freq, uint32_t* cum, int qp, float* thr);

/* Per-stage device timing of the chunk calls, measured with CUDA events on the calling stream.
 * enable != 0 turns recording on (and discards unread entries).  Entries accumulate over calls;
 * ufvc_get_profile waits for them, copies up to `max`: names (NUL-terminated, 32 bytes each),
 * milliseconds and kernel launches per stage, returns the count in *count, and starts a new list. */
ufvc_status ufvc_set_profiling(ufvc_ctx* ctx, int enable);
ufvc_status ufvc_get_profile(ufvc_ctx* ctx, char* names, float* ms, int* launches, int max, int* count);

/* Human-readable description of the last error on this context ("" if none). */
const char* ufvc_last_error(const ufvc_ctx* ctx);

/* FP8 calibration: the FP32 path of the context's weights codes the given chunk (device frames, as for
 * ufvc_encode_chunk) and every activation tensor of the E4M3 layers gets the scale absmax / 448 (the
 * packed input in [0, 1] uses 1 / 448).  Only for precision UFVC_FP8; synchronises `stream`.  Until it
 * has run, an FP8 context refuses the chunk calls with UFVC_ERR_ARG.  Calibrating again replaces the
 * scales. */
ufvc_status ufvc_calibrate_fp8(ufvc_ctx* ctx, const uint8_t* d_frames, int n_frames, int width, int height, int qp,
                               void* stream);
/* The calibrated activation scales, n >= 15 entries: packed input, A1, A2, A3, interaction hidden,
 * A3 + interaction, y (hyper-analysis input), H1, y^, D0, R1a, R1b, U1, R2a, R2b. */
ufvc_status ufvc_get_fp8_scales(const ufvc_ctx* ctx, float* act_scales, int n);

/* ------------------------------------------------------------------------------------------------
 * Serving: continuous batching of chunk requests from many streams (the cross-chunk overlap that
 * Sec. 4 leaves as potential; the paper's own pipeline codes one chunk at a time).
 *
 * A server owns one weight copy and a pool of execution slots.  A slot is a context sharing those
 * weights, a CUDA stream, device staging buffers for one frame size, and the CUDA graphs of its
 * encode and decode calls (captured after the slot's first direct run).  Each stream (a video, opened
 * with its frame size and qp) owns device-resident buffers: the input chunk, its latest bit-stream
 * (bytes + size) and the latest decoded chunk.  A host scheduler thread admits queued requests as
 * slots free up: a request runs on an idle slot of its frame size, or on a new slot if the pool has
 * room and the HBM cap allows the slot's footprint (idle slots of other sizes are released to make
 * room); requests of one stream run in submission order; requests on different slots overlap on the
 * device.  Queued requests of the same frame size and operation (and rate, for encodes) that are
 * admitted together run as one batch on one slot (ufvc_encode_chunks / ufvc_decode_chunks: their rANS
 * sections share launches), up to the slot's batch size (4 chunks up to 1080p, 1 above; 1 with the
 * temporal context, where every stream carries its own).  Results are identical to the single-context
 * calls (same kernels, same arithmetic).
 *
 * All server calls are thread-safe.  Device pointers returned by ufvc_server_stream_buffers stay valid
 * until the server is destroyed; the input buffer must not be modified while an encode request of the
 * stream is queued or running, and the outputs are stable once the request completed.
 * ------------------------------------------------------------------------------------------------ */
typedef struct ufvc_server ufvc_server;

typedef enum { UFVC_OP_ENCODE = 0, UFVC_OP_DECODE = 1 } ufvc_op;

typedef struct {
    int status;          /* ufvc_status of the request (UFVC_PENDING while queued or running) */
    int op;              /* ufvc_op */
    int stream_id;
    int slot;            /* slot that ran it (-1 while queued) */
    double submit_ms;    /* host steady-clock times, milliseconds since the server was created */
    double start_ms;     /* launched on a slot */
    double done_ms;      /* completion observed by the scheduler */
    uint64_t nbytes;     /* encode: bit-stream size (read back at completion); decode: the size decoded */
    int batch;           /* requests in the batch it ran in (1: alone) */
} ufvc_result;

typedef struct {
    int slots;                /* slots alive */
    int busy_slots;
    int queued;               /* requests waiting for a slot */
    int graphs;               /* CUDA graphs instantiated */
    uint64_t completed;       /* requests finished */
    size_t hbm_used;          /* bytes held: streams' buffers + slots' footprints */
    size_t hbm_cap;
    uint64_t batches;         /* launches of two or more requests at once */
    uint64_t batched;         /* requests that ran in such batches */
} ufvc_server_stats;

/* cfg / weights as for ufvc_create.  hbm_cap_bytes bounds the device bytes the server holds besides
 * its weight copy (0: no cap); max_slots bounds concurrent requests (>= 1). */
ufvc_status ufvc_server_create(const ufvc_config* cfg, const float* weights, size_t n_weights, size_t hbm_cap_bytes,
                               int max_slots, ufvc_server** out);
/* Waits for all requests, then frees everything. */
void ufvc_server_destroy(ufvc_server* srv);
/* A new stream of width x height chunks at rate qp; its buffers count against the HBM cap
 * (UFVC_ERR_OOM if they do not fit). */
ufvc_status ufvc_server_open_stream(ufvc_server* srv, int width, int height, int qp, int* stream_id);
/* The stream's device buffers (any pointer argument may be NULL): d_frames_in [N][H][W][3] uint8 (the
 * caller writes the chunk to encode there), d_bits / *d_nbytes (the latest bit-stream, capacity bytes),
 * d_frames_out [N][H][W][3] uint8 (the latest decoded chunk). */
ufvc_status ufvc_server_stream_buffers(ufvc_server* srv, int stream_id, uint8_t** d_frames_in, uint8_t** d_bits,
                                       uint64_t** d_nbytes, size_t* capacity, uint8_t** d_frames_out);
/* Queue a request; returns at once with its ticket.  ENCODE codes the stream's input buffer into its
 * bit-stream buffers; DECODE decodes the stream's latest bit-stream into its output buffer. */
ufvc_status ufvc_server_submit(ufvc_server* srv, int stream_id, int op, uint64_t* ticket);
/* Queue n requests at once (request i: stream_ids[i], ops[i]; its ticket in tickets[i]), all or none
 * (UFVC_ERR_ARG if any is invalid).  The scheduler sees them together, so same-shape requests among them
 * whose streams are free run as batches (ufvc_result.batch). */
ufvc_status ufvc_server_submit_many(ufvc_server* srv, int n, const int* stream_ids, const int* ops,
                                    uint64_t* tickets);
/* The request's result; returns UFVC_PENDING while it is queued or running, else its status. */
ufvc_status ufvc_server_poll(ufvc_server* srv, uint64_t ticket, ufvc_result* out);
/* Blocks until the request completed (timeout_ms < 0: no limit; UFVC_PENDING on timeout). */
ufvc_status ufvc_server_wait(ufvc_server* srv, uint64_t ticket, double timeout_ms, ufvc_result* out);
ufvc_status ufvc_server_stats_get(ufvc_server* srv, ufvc_server_stats* out);
/* Message of the last server-level error ("" if none). */
const char* ufvc_server_last_error(const ufvc_server* srv);

/* Optional networks of the served codec (as ufvc_set_temporal_context / ufvc_set_progressive_means), set
 * before the first stream is opened (UFVC_ERR_ARG afterwards).  With the temporal context every stream
 * carries its own coding state on the device: the encoder's and the decoder's context, advanced by each
 * of the stream's encode and decode requests in submission order (the first chunk uses C_0 = 0); the
 * stream's chunks therefore have to be encoded and decoded in order, as for a single context.  A stream
 * holds only its latest bit-stream, so each ENCODE has to be followed by its DECODE before the stream's
 * next ENCODE when the server decodes the stream: a DECODE whose bit-stream is not the chunk after the
 * last one the stream's decoder decoded finishes with UFVC_ERR_ARG (nothing runs, both contexts unchanged). */
ufvc_status ufvc_server_set_temporal_context(ufvc_server* srv, const float* weights, size_t n_weights);
/* An FP8 server's activation scales (as ufvc_calibrate_fp8 on the server's own context, synchronous), set
 * before the first stream is opened (UFVC_ERR_ARG afterwards); until then an FP8 server's requests finish
 * with UFVC_ERR_ARG. */
ufvc_status ufvc_server_calibrate_fp8(ufvc_server* srv, const uint8_t* d_frames, int n_frames, int width, int height,
                                      int qp);
ufvc_status ufvc_server_set_progressive_means(ufvc_server* srv, const float* weights, size_t n_weights);

#ifdef __cplusplus
}
#endif

#endif /* UFVC_H */
