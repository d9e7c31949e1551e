// Elementwise and entropy-coding kernels.
//
//  * pack          : chunk frames uint8 [N][H][W][3] -> /255, replicate pad to x16, frames stacked into
//                    channels (frame n -> channels 3n..3n+2), zero channels up to the padded count
//                    (the patch-embedding input of Sec. 3.1).
//  * zquant        : z^ = clamp(rint(z), +-255) and the per-channel scale index of z^.
//  * quantize      : r^ = clamp(rint((y - mu) / q), +-255) and the scale index of log sigma (Sec. 3.4).
//  * rANS          : K interleaved lanes, the whole latent coded in one step (Sec. 3.4): element i goes
//                    to lane i mod K; 32-bit state in [2^16, 2^32), 16-bit probabilities, 16-bit words,
//                    at most one renormalisation word per symbol.
#include "ufvc_internal.h"

#include <cub/block/block_scan.cuh>

namespace ufvc {

__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, 0, code); }

// ------------------------------------------------------------------------------------------------
// pack
// ------------------------------------------------------------------------------------------------
__global__ void pack_kernel(const uint8_t* __restrict__ frames, int N, int H, int W, int Hp, int Wp, int Cp,
                            float* __restrict__ x) {
    const size_t pix = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= (size_t)Hp * Wp) return;
    const int h = (int)(pix / Wp), w = (int)(pix % Wp);
    const int sh = h < H ? h : H - 1, sw = w < W ? w : W - 1;
    float* o = x + pix * Cp;
    for (int c0 = 0; c0 < Cp; c0 += 4) {
        float v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = c0 + j, n = c / 3;
            v[j] = (n < N) ? frames[(((size_t)n * H + sh) * W + sw) * 3 + (c - 3 * n)] / 255.0f : 0.0f;
        }
        *reinterpret_cast<float4*>(o + c0) = make_float4(v[0], v[1], v[2], v[3]);
    }
}

void launch_pack(const uint8_t* frames, int N, int H, int W, int Hp, int Wp, int Cp, float* x, cudaStream_t s) {
    const size_t npix = (size_t)Hp * Wp;
    pack_kernel<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(frames, N, H, W, Hp, Wp, Cp, x);
}

// bf16 variant for the tensor-core path: one thread per (pixel, 8-channel group), 16-byte stores
__global__ void pack_bf16_kernel(const uint8_t* __restrict__ frames, int N, int H, int W, int Hp, int Wp, int Cp,
                                 __nv_bfloat16* __restrict__ x) {
    const int groups = Cp / 8;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)Hp * Wp * groups) return;
    const size_t pix = i / groups;
    const int c0 = (int)(i % groups) * 8;
    const int h = (int)(pix / Wp), w = (int)(pix % Wp);
    const int sh = h < H ? h : H - 1, sw = w < W ? w : W - 1;
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = c0 + j, n = c / 3;
        const float f = (n < N) ? frames[(((size_t)n * H + sh) * W + sw) * 3 + (c - 3 * n)] / 255.0f : 0.0f;
        v[j] = __float2bfloat16_rn(f);
    }
    *reinterpret_cast<uint4*>(x + pix * Cp + c0) = *reinterpret_cast<const uint4*>(v);
}

void launch_pack_bf16(const uint8_t* frames, int N, int H, int W, int Hp, int Wp, int Cp, __nv_bfloat16* x,
                      cudaStream_t s) {
    const size_t n = (size_t)Hp * Wp * (Cp / 8);
    pack_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(frames, N, H, W, Hp, Wp, Cp, x);
}

// ------------------------------------------------------------------------------------------------
// z^ quantisation and per-channel index.  iz[c] = #{k : S_c > T_k}, S_c = sum z^^2 (exact integer),
// T_k = floor(npos * exp(2 t_k)) precomputed on the host in FP64: S_c > npos e^{2 t_k} <=>
// ln sqrt(S_c / npos) > t_k, i.e. the nearest log bin of the channel's RMS.
// ------------------------------------------------------------------------------------------------
__global__ void zquant_kernel(const float* __restrict__ z, int npos, int cz, const uint64_t* __restrict__ zthr,
                              int16_t* __restrict__ zhat, uint8_t* __restrict__ iz) {
    const int c = blockIdx.x;
    unsigned long long S = 0;
    for (int p = threadIdx.x; p < npos; p += blockDim.x) {
        const float v = fminf(fmaxf(rintf(z[(size_t)p * cz + c]), -255.0f), 255.0f);
        const int q = (int)v;
        zhat[(size_t)p * cz + c] = (int16_t)q;
        S += (unsigned long long)(q * q);
    }
    __shared__ unsigned long long red[256];
    red[threadIdx.x] = S;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int k = 0;
        for (int j = 0; j < kBins - 1; ++j) k += red[0] > zthr[j];
        iz[c] = (uint8_t)k;
    }
}

void launch_zquant(const float* z, int npos, int cz, const uint64_t* zthr, int16_t* zhat, uint8_t* iz,
                   cudaStream_t s) {
    zquant_kernel<<<cz, 256, 0, s>>>(z, npos, cz, zthr, zhat, iz);
}

// ------------------------------------------------------------------------------------------------
// quantize / scale index
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ int count_below(const float* thr, float v) {
    // #{k : thr[k] < v} for the 63 ascending thresholds (binary search)
    int lo = 0, hi = kBins - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (thr[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void quantize_kernel(const float* __restrict__ y, const float* __restrict__ mu,
                                const float* __restrict__ logsig, size_t n, const float* __restrict__ thr_all,
                                const float* __restrict__ qinv_all, const int* qp_dev, int qp_host,
                                int16_t* __restrict__ rhat, uint8_t* __restrict__ idx) {
    __shared__ float thr[kBins - 1];
    const int qp = qp_dev ? *qp_dev : qp_host;
    if (threadIdx.x < kBins - 1) thr[threadIdx.x] = thr_all[qp * (kBins - 1) + threadIdx.x];
    __syncthreads();
    const float qinv = qinv_all[qp];
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        if (rhat) {
            // explicit round-to-nearest ops: no FMA contraction, same result on every launch
            const float r = rintf(__fmul_rn(__fsub_rn(y[i], mu[i]), qinv));
            rhat[i] = (int16_t)fminf(fmaxf(r, -255.0f), 255.0f);
        }
        idx[i] = (uint8_t)count_below(thr, logsig[i]);
    }
}

static unsigned grid_for(size_t n, int per_block) {
    size_t g = (n + per_block - 1) / per_block;
    if (g > 148 * 16) g = 148 * 16;
    return (unsigned)(g ? g : 1);
}

void launch_quantize(const float* y, const float* mu, const float* logsig, size_t n, const float* thr_all,
                     const float* qinv_all, const int* qp_dev, int qp_host, int16_t* rhat, uint8_t* idx,
                     cudaStream_t s) {
    quantize_kernel<<<grid_for(n, 256), 256, 0, s>>>(y, mu, logsig, n, thr_all, qinv_all, qp_dev, qp_host, rhat, idx);
}

void launch_scale_index(const float* logsig, size_t n, const float* thr_all, const int* qp_dev, uint8_t* idx,
                        cudaStream_t s) {
    quantize_kernel<<<grid_for(n, 256), 256, 0, s>>>(nullptr, nullptr, logsig, n, thr_all, thr_all, qp_dev, 0,
                                                    nullptr, idx);
}

__global__ void i16_to_f32_kernel(const int16_t* a, size_t n, float* out) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (float)a[i];
}

void launch_i16_to_f32(const int16_t* a, size_t n, float* out, cudaStream_t s) {
    i16_to_f32_kernel<<<grid_for(n, 256), 256, 0, s>>>(a, n, out);
}

__global__ void f32_to_bf16_kernel(const float* a, size_t n, __nv_bfloat16* out) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(a[i]);
}

void launch_f32_to_bf16(const float* a, size_t n, __nv_bfloat16* out, cudaStream_t s) {
    f32_to_bf16_kernel<<<grid_for(n, 256), 256, 0, s>>>(a, n, out);
}

// ------------------------------------------------------------------------------------------------
// rANS encode: one thread per lane, lanes of up to two sections in one launch.  Each lane runs its
// elements backwards (last first) and writes its words backwards into its scratch row, so that the
// row's tail [cap_lane - words, cap_lane) is the lane stream in decoding order.
// ------------------------------------------------------------------------------------------------
struct RansSecPair { RansSection s[2]; int nsec; };

__global__ void rans_encode_kernel(const RansSecPair P, const uint32_t* __restrict__ tables) {
    extern __shared__ uint32_t tab[];  // [64][511] (freq << 16) | cum
    for (int i = threadIdx.x; i < kBins * kNsym; i += blockDim.x) tab[i] = tables[i];
    __syncthreads();
    int lane = blockIdx.x * blockDim.x + threadIdx.x;
    int si = 0;
    if (lane >= P.s[0].K) { lane -= P.s[0].K; si = 1; }
    if (si >= P.nsec) return;
    const RansSection& S = P.s[si];
    if (lane >= S.K) return;
    const size_t n = S.n, K = (size_t)S.K;
    const size_t cnt = (size_t)lane < n ? (n - lane + K - 1) / K : 0;
    uint16_t* row = S.scratch + (size_t)lane * S.cap_lane;
    int wp = S.cap_lane;
    uint32_t x = kRansL;
    for (size_t m = cnt; m-- > 0;) {
        const size_t i = (size_t)lane + m * K;
        int t = S.idx_period ? S.idx[i % S.idx_period] : S.idx[i];
        int v = S.sym[i];
        if (t >= kBins || v < -kRmax || v > kRmax) {  // caller error: never index outside the tables
            set_status(S.status, UFVC_ERR_ARG);
            t = 0;
            v = 0;
        }
        const uint32_t e = tab[t * kNsym + (v + kRmax)];
        const uint32_t f = e >> 16, c = e & 0xFFFFu;
        if (x >= (f << 16)) {  // f << 16 < 2^32 as f <= 65026
            row[--wp] = (uint16_t)(x & 0xFFFFu);
            x >>= 16;
        }
        const uint32_t q = x / f;
        x = (q << 16) + (x - q * f) + c;
    }
    row[--wp] = (uint16_t)(x & 0xFFFFu);
    row[--wp] = (uint16_t)(x >> 16);
    S.counts[lane] = (uint32_t)(S.cap_lane - wp);
}

void launch_rans_encode(const RansSection* secs, int nsec, const uint32_t* packed_tables, cudaStream_t s) {
    RansSecPair P{};
    P.nsec = nsec;
    int total = 0;
    for (int i = 0; i < nsec; ++i) { P.s[i] = secs[i]; total += secs[i].K; }
    const int smem = kBins * kNsym * 4;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(rans_encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr = true;
    }
    const int threads = 64;
    rans_encode_kernel<<<(total + threads - 1) / threads, threads, smem, s>>>(P, packed_tables);
}

// ------------------------------------------------------------------------------------------------
// rANS finalize: single block scans the lane counts of each section, writes them and the section
// padding, and records each lane's destination byte offset; then a copy kernel moves the words.
// Nothing is written at or past `capacity`.
// ------------------------------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
using BlockScanU64 = cub::BlockScan<unsigned long long, kScanThreads>;

__global__ void __launch_bounds__(kScanThreads) rans_finalize_kernel(const RansSecPair P, uint8_t* out,
                                                                     size_t hdr_bytes, size_t capacity,
                                                                     uint64_t* nbytes, uint64_t* off_ws,
                                                                     int* status) {
    __shared__ typename BlockScanU64::TempStorage tmp;
    __shared__ unsigned long long base_sh;
    if (threadIdx.x == 0) base_sh = hdr_bytes;
    __syncthreads();
    size_t ws_base = 0;
    for (int si = 0; si < P.nsec; ++si) {
        const RansSection& S = P.s[si];
        const int K = S.K;
        const int per = (K + kScanThreads - 1) / kScanThreads;
        const int j0 = threadIdx.x * per;
        unsigned long long local = 0;
        for (int j = j0; j < j0 + per && j < K; ++j) local += S.counts[j];
        unsigned long long excl, total;
        BlockScanU64(tmp).ExclusiveSum(local, excl, total);
        const unsigned long long base = base_sh;
        const unsigned long long words_at = base + 4ull * K;
        for (int j = j0; j < j0 + per && j < K; ++j) {
            const uint32_t c = S.counts[j];
            off_ws[ws_base + j] = words_at + 2ull * excl;
            excl += c;
            const size_t cp = base + 4ull * j;
            if (cp + 4 <= capacity) {
                out[cp] = c & 0xFF; out[cp + 1] = (c >> 8) & 0xFF; out[cp + 2] = (c >> 16) & 0xFF; out[cp + 3] = c >> 24;
            }
        }
        const unsigned long long end = words_at + 2ull * total;
        const unsigned long long end4 = (end + 3) & ~3ull;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (unsigned long long b = end; b < end4; ++b)
                if (b < capacity) out[b] = 0;
            base_sh = end4;
        }
        __syncthreads();
        ws_base += K;
    }
    if (threadIdx.x == 0) {
        *nbytes = base_sh;
        if (base_sh > capacity) set_status(status, UFVC_ERR_CAPACITY);
    }
}

__global__ void rans_copy_kernel(const RansSecPair P, uint8_t* out, size_t capacity, const uint64_t* off_ws) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, l = threadIdx.x & 31;
    int lane = warp, si = 0;
    size_t ws = 0;
    if (lane >= P.s[0].K) { lane -= P.s[0].K; si = 1; ws = P.s[0].K; }
    if (si >= P.nsec || lane >= P.s[si].K) return;
    const RansSection& S = P.s[si];
    const uint32_t words = S.counts[lane];
    const uint16_t* src = S.scratch + (size_t)lane * S.cap_lane + (S.cap_lane - words);
    const uint64_t dst = off_ws[ws + lane];
    if (dst + 2ull * words > capacity) return;  // status already records the capacity error
    uint16_t* d = reinterpret_cast<uint16_t*>(out + dst);
    for (uint32_t w = l; w < words; w += 32) d[w] = src[w];
}

void launch_rans_finalize(const RansSection* secs, int nsec, uint8_t* out, size_t hdr_bytes, size_t capacity,
                          uint64_t* nbytes, uint64_t* offsets_ws, int* status, cudaStream_t s) {
    RansSecPair P{};
    P.nsec = nsec;
    int total = 0;
    for (int i = 0; i < nsec; ++i) { P.s[i] = secs[i]; total += secs[i].K; }
    rans_finalize_kernel<<<1, kScanThreads, 0, s>>>(P, out, hdr_bytes, capacity, nbytes, offsets_ws, status);
    const int threads = 256;
    rans_copy_kernel<<<(unsigned)(((size_t)total * 32 + threads - 1) / threads), threads, 0, s>>>(P, out, capacity,
                                                                                               offsets_ws);
}

// ------------------------------------------------------------------------------------------------
// rANS decode.  parse: single block reads the K lane counts of a section, checks 2 <= words <= n_j + 2
// and that the section fits in the stream, and produces each lane's byte offset.  decode: one thread
// per lane; every read stays inside the lane's words; a lane that ends with a state != 2^16 or with
// unread / missing words marks the stream corrupt.
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kScanThreads) rans_parse_kernel(const RansDecodeJob J, size_t expect_end,
                                                                  int* status) {
    __shared__ typename BlockScanU64::TempStorage tmp;
    __shared__ int bad, prior;
    if (threadIdx.x == 0) { bad = 0; prior = *status; }
    __syncthreads();
    if (prior != 0) return;
    const unsigned long long off = J.sec_off_dev ? *J.sec_off_dev : J.sec_off_host;
    const int K = J.K;
    const size_t n = J.n;
    if (off + 4ull * K > J.nbytes) {
        if (threadIdx.x == 0) set_status(status, UFVC_ERR_CORRUPT);
        return;
    }
    const int per = (K + kScanThreads - 1) / kScanThreads;
    const int j0 = threadIdx.x * per;
    unsigned long long local = 0;
    for (int j = j0; j < j0 + per && j < K; ++j) {
        const uint8_t* p = J.bits + off + 4ull * j;
        const uint32_t c = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
        const size_t cnt = (size_t)j < n ? (n - j + K - 1) / K : 0;
        if (c < 2 || c > cnt + 2) bad = 1;
        local += c;
    }
    unsigned long long excl, total;
    BlockScanU64(tmp).ExclusiveSum(local, excl, total);
    __syncthreads();
    const unsigned long long words_at = off + 4ull * K;
    const unsigned long long end4 = (words_at + 2ull * total + 3) & ~3ull;
    const bool fits = end4 <= J.nbytes && (expect_end == 0 || end4 == expect_end);
    if (bad || !fits) {
        if (threadIdx.x == 0) set_status(status, UFVC_ERR_CORRUPT);
        return;
    }
    for (int j = j0; j < j0 + per && j < K; ++j) {
        const uint8_t* p = J.bits + off + 4ull * j;
        const uint32_t c = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
        J.lane_off[j] = words_at + 2ull * excl;
        J.lane_words[j] = c;
        excl += c;
    }
    if (threadIdx.x == 0 && J.next_off) *J.next_off = end4;
}

void launch_rans_parse(const RansDecodeJob& j, int* status, cudaStream_t s) {
    rans_parse_kernel<<<1, kScanThreads, 0, s>>>(j, 0, status);
}

void launch_rans_parse_expect(const RansDecodeJob& j, size_t expect_end, int* status, cudaStream_t s) {
    rans_parse_kernel<<<1, kScanThreads, 0, s>>>(j, expect_end, status);
}

__global__ void rans_decode_kernel(const RansDecodeJob J, const uint32_t* __restrict__ tables, int* status) {
    extern __shared__ uint32_t tab[];
    for (int i = threadIdx.x; i < kBins * kNsym; i += blockDim.x) tab[i] = tables[i];
    __syncthreads();
    if (*(volatile int*)status != 0) return;
    const int lane = blockIdx.x * blockDim.x + threadIdx.x;
    if (lane >= J.K) return;
    const size_t n = J.n, K = (size_t)J.K;
    const size_t cnt = (size_t)lane < n ? (n - lane + K - 1) / K : 0;
    const uint16_t* wp = reinterpret_cast<const uint16_t*>(J.bits + J.lane_off[lane]);
    const uint32_t words = J.lane_words[lane];
    const float q = (J.yhat || J.yhat_bf16) ? J.qstep_all[*J.qp_dev] : 0.0f;
    uint32_t x = ((uint32_t)wp[0] << 16) | wp[1];
    uint32_t r = 2;
    for (size_t m = 0; m < cnt; ++m) {
        const size_t i = (size_t)lane + m * K;
        int t = J.idx_period ? J.idx[i % J.idx_period] : J.idx[i];
        if (t >= kBins) {
            set_status(status, UFVC_ERR_ARG);
            t = 0;
        }
        const uint32_t* T = tab + t * kNsym;
        const uint32_t slot = x & 0xFFFFu;
        // largest s with cum(s) <= slot
        int lo = 0, hi = kNsym - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((T[mid] & 0xFFFFu) <= slot) lo = mid; else hi = mid - 1;
        }
        const uint32_t e = T[lo];
        x = (e >> 16) * (x >> 16) + slot - (e & 0xFFFFu);
        if (x < kRansL) {
            const uint32_t w = r < words ? wp[r] : 0u;
            x = (x << 16) | w;
            ++r;
        }
        const int sym = lo - kRmax;
        if (J.sym) J.sym[i] = (int16_t)sym;
        if (J.yhat || J.yhat_bf16) {
            const float yv = __fadd_rn(__fmul_rn((float)sym, q), J.mu[i]);
            if (J.yhat) J.yhat[i] = yv;
            if (J.yhat_bf16) J.yhat_bf16[i] = __float2bfloat16_rn(yv);
        }
    }
    if (x != kRansL || r != words) set_status(status, UFVC_ERR_CORRUPT);
}

void launch_rans_decode(const RansDecodeJob& j, const uint32_t* packed_tables, int* status, cudaStream_t s) {
    const int smem = kBins * kNsym * 4;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(rans_decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr = true;
    }
    const int threads = 64;
    rans_decode_kernel<<<(j.K + threads - 1) / threads, threads, smem, s>>>(j, packed_tables, status);
}

// ------------------------------------------------------------------------------------------------
// container header
// ------------------------------------------------------------------------------------------------
__global__ void write_header_kernel(uint8_t* out, int arch, int N, int qp, int W, int H, int K, int Kz,
                                    const uint8_t* iz, int Cz, size_t capacity, int* status) {
    const size_t hdr = (20 + (size_t)Cz + 3) & ~(size_t)3;
    if (hdr > capacity) {
        if (threadIdx.x == 0) set_status(status, UFVC_ERR_CAPACITY);
        return;
    }
    for (int i = threadIdx.x; i < (int)hdr; i += blockDim.x) {
        uint8_t v = 0;
        if (i < 4) v = "UFVC"[i];
        else if (i == 4) v = 1;
        else if (i == 5) v = (uint8_t)arch;
        else if (i == 6) v = (uint8_t)N;
        else if (i == 7) v = (uint8_t)qp;
        else if (i < 10) v = (uint8_t)(W >> (8 * (i - 8)));
        else if (i < 12) v = (uint8_t)(H >> (8 * (i - 10)));
        else if (i < 16) v = (uint8_t)((uint32_t)K >> (8 * (i - 12)));
        else if (i < 20) v = (uint8_t)((uint32_t)Kz >> (8 * (i - 16)));
        else if (i < 20 + Cz) v = iz[i - 20];
        out[i] = v;
    }
}

void launch_write_header(uint8_t* out, int arch, int N, int qp, int W, int H, int K, int Kz, const uint8_t* iz,
                         int Cz, size_t capacity, int* status, cudaStream_t s) {
    write_header_kernel<<<1, 256, 0, s>>>(out, arch, N, qp, W, H, K, Kz, iz, Cz, capacity, status);
}

__global__ void parse_header_kernel(const uint8_t* b, size_t nbytes, int arch, int N, int W, int H, int K, int Kz,
                                    int Cz, int* qp_dev, uint8_t* iz, int* status) {
    if (threadIdx.x != 0) return;
    const size_t hdr = (20 + (size_t)Cz + 3) & ~(size_t)3;
    *qp_dev = 32;
    for (int c = 0; c < Cz; ++c) iz[c] = 0;
    if (nbytes < hdr || b[0] != 'U' || b[1] != 'F' || b[2] != 'V' || b[3] != 'C' || b[4] != 1) {
        set_status(status, UFVC_ERR_CORRUPT);
        return;
    }
    const int w = b[8] | (b[9] << 8), h = b[10] | (b[11] << 8);
    const uint32_t k = b[12] | (b[13] << 8) | (b[14] << 16) | ((uint32_t)b[15] << 24);
    const uint32_t kz = b[16] | (b[17] << 8) | (b[18] << 16) | ((uint32_t)b[19] << 24);
    if (b[5] != arch || b[6] != N || w != W || h != H) { set_status(status, UFVC_ERR_ARG); return; }
    if (b[7] > 63 || k != (uint32_t)K || kz != (uint32_t)Kz) { set_status(status, UFVC_ERR_CORRUPT); return; }
    for (int c = 0; c < Cz; ++c) {
        if (b[20 + c] >= kBins) { set_status(status, UFVC_ERR_CORRUPT); return; }
        iz[c] = b[20 + c];
    }
    *qp_dev = b[7];
}

void launch_parse_header(const uint8_t* bits, size_t nbytes, int arch, int N, int W, int H, int K, int Kz, int Cz,
                         int* qp_dev, uint8_t* iz, int* status, cudaStream_t s) {
    parse_header_kernel<<<1, 32, 0, s>>>(bits, nbytes, arch, N, W, H, K, Kz, Cz, qp_dev, iz, status);
}

}  // namespace ufvc
