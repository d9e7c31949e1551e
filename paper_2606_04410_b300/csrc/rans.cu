// Interleaved rANS coding of whole latent sections in one step (Sec. 3.4: every element of the chunk
// latent is coded with its scale in a single pass), and the bit-stream container around it.
//
// Element i of a section goes to lane i mod K; lane j codes elements j, j + K, j + 2K, ... as one rANS
// chain: 32-bit state in [2^16, 2^32), 16-bit probabilities (M = 2^16), 16-bit words, at most one
// renormalisation word per symbol.  The encoder runs each chain backwards; a lane stream is stored in
// decoding order (final state's high half, low half, then the renormalisation words, last one first).
//
// Section layout: K lane word counts (u32, little endian), the lanes' words in lane order, zero bytes up
// to a multiple of 4.  Container: header ("UFVC", version, arch, N, qp, W u16, H u16, K u32, Kz u32,
// Cz z^ scale indices, zero padding to 4), the z^ section (Kz lanes, one scale index per channel), the
// y^ section (K lanes, one scale index per element).
//
// Kernels (all one thread per lane, the tables in shared memory):
//  * rans_encode_kernel: codes the lanes of one or two sections, then lays them out in the same launch.
//    Blocks take tickets in the order they start; a block publishes its sections' word total and finds
//    the words of all earlier blocks by looking back over their published totals (a block only waits on
//    blocks with smaller tickets, which have started before it), then writes its lanes' counts and
//    copies its lanes' words to their final place.  The first block writes the container header.
//  * rans_decode_kernel: every block reads the section's lane counts itself (its lanes' offsets are
//    prefix sums, the section's end is their total), checks them, then decodes; the z^ section's launch
//    also checks the header and takes its scale indices from it; the y^ section's launch can write
//    y^ = r^ q + mu directly (bf16, float or E4M3) instead of r^.
// Every wait is bounded: a wait that runs out records UFVC_ERR_TIMEOUT and the kernel returns.
#include "ufvc_internal.h"

#include <cuda_fp8.h>

#include <type_traits>

#include "tc_ptx.h"

namespace ufvc {

namespace {

__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, 0, code); }

constexpr int kEncTabBytes = kBins * kNsym * 4;           // packed (freq << 16) | cum, 130816 bytes
constexpr int kEncSmemMax = 232448;                       // dynamic shared memory per block (227 KB)
constexpr int kPF = 16;                                   // symbols fetched ahead per lane
constexpr long long kSpinDefault = 4000000000LL;          // about 2 s at 2 GHz
constexpr uint64_t kFlagAgg = 1ull << 62, kFlagIncl = 2ull << 62, kFlagMask = (1ull << 62) - 1;

__device__ __forceinline__ uint32_t ld_u16(const uint16_t* p) {
    unsigned short v;
    asm volatile("ld.global.nc.u16 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
}
// Predicated loads into a register that keeps its value where the predicate is false: no select (and so
// no wait for the load) where the value is merged.
__device__ __forceinline__ void ld_if_u8(unsigned short& v, const uint8_t* p, bool c) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.global.nc.u8 %0, [%1];\n\t}"
                 : "+h"(v) : "l"(p), "r"((uint32_t)c));
}
__device__ __forceinline__ void ld_if_s16(short& v, const int16_t* p, bool c) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.global.nc.s16 %0, [%1];\n\t}"
                 : "+h"(v) : "l"(p), "r"((uint32_t)c));
}
__device__ __forceinline__ void ld_if_u16(unsigned short& v, const uint16_t* p, bool c) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.global.nc.u16 %0, [%1];\n\t}"
                 : "+h"(v) : "l"(p), "r"((uint32_t)c));
}
__device__ __forceinline__ void ld_if_f32(float& v, const float* p, bool c) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.global.nc.f32 %0, [%1];\n\t}"
                 : "+f"(v) : "l"(p), "r"((uint32_t)c));
}

// Bulk copy of `bytes` (a multiple of 16) from global to shared memory, waited for with a non-blocking
// test for at most `spin` clocks.  On a timeout the issuing thread waits (for at most about 2 s) for its
// copies to land before the block may exit, and false is returned everywhere.
__device__ bool load_table(void* dst, const void* src, int bytes, uint64_t* bar, int* status, long long spin) {
    if (threadIdx.x == 0) {
        ptx::mbar_init(bar, 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ptx::mbar_arrive_expect_tx(bar, (uint32_t)bytes);
        for (int off = 0; off < bytes; off += 32768) {
            const int n = bytes - off < 32768 ? bytes - off : 32768;
            ptx::bulk_load(static_cast<uint8_t*>(dst) + off, static_cast<const uint8_t*>(src) + off, n, bar);
        }
    }
    // a short bound (a test of the timeout path) is polled without blocking; the default one waits in
    // try_wait's own suspended steps
    const bool poll = spin > 0 && spin < kSpinDefault;
    if (spin <= 0) spin = kSpinDefault;
    const long long t0 = clock64();
    while (!(poll ? ptx::mbar_test_wait(bar, 0) : ptx::mbar_try_wait(bar, 0))) {
        if (clock64() - t0 > spin) {
            set_status(status, UFVC_ERR_TIMEOUT);
            if (threadIdx.x == 0) {
                const long long t1 = clock64();
                while (!ptx::mbar_test_wait(bar, 0) && clock64() - t1 < kSpinDefault) {
                }
            }
            return false;
        }
    }
    return true;
}

// Exclusive prefix sum over the block of one u32 per thread (blockDim.x a multiple of 32); *total gets
// the block's sum.  sh: 32 words of shared memory.
__device__ uint32_t block_excl_scan(uint32_t v, uint32_t* total, uint32_t* sh) {
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (l >= o) inc += t;
    }
    if (l == 31) sh[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t s = l < nw ? sh[l] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, s, o);
            if (l >= o) s += t;
        }
        sh[l] = s;  // inclusive over warps
    }
    __syncthreads();
    const uint32_t before = w ? sh[w - 1] : 0u;
    *total = sh[nw - 1];
    __syncthreads();
    return before + inc - v;
}

// Sum over the block of one u64 per thread; every thread gets the result.  sh: 32 u64 of shared memory.
__device__ uint64_t block_sum_u64(uint64_t v, uint64_t* sh) {
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (l == 0) sh[w] = v;
    __syncthreads();
    uint64_t s = 0;
    for (int i = 0; i < nw; ++i) s += sh[i];
    __syncthreads();
    return s;
}

// elements of lane j in a section of n elements and K lanes
__device__ __forceinline__ uint32_t lane_elems(uint32_t n, int K, int j) {
    return (uint32_t)j < n ? (n - (uint32_t)j + (uint32_t)K - 1u) / (uint32_t)K : 0u;
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// encode
// ------------------------------------------------------------------------------------------------
// One encoder step with a float reciprocal instead of an integer division: after renormalisation
// x < f 2^16, so q = floor(x / f) < 2^16.  x and 1/f rounded to float and their rounded product carry a
// relative error below 3 2^-24, i.e. below 0.012 in x / f, so the truncated product is q - 1, q or q + 1,
// and one correction by the sign and size of the remainder r = x - q' f gives q and r exactly (checked
// for every f against integer division).  The reciprocal depends on f alone, off the state chain.
struct EncSym {
    uint32_t f, c;
    float rcp;
};

// 1 / f for the quotient estimate of enc_update: the hardware's approximate reciprocal (within about one
// ulp, relative error near 2^-23; the correctly rounded __frcp_rn took a quarter of the encoder's time).
// With x < f 2^16 after renormalisation the quotient is below 2^16, so float(x) * rcp (three roundings of
// relative size 2^-24 .. 2^-23) is within 2^16 * 2^-21 < 1 of x / f, and the two corrections in
// enc_update return the exact quotient and remainder: the state, and so the stream, do not depend on
// the reciprocal's rounding.
__device__ __forceinline__ float enc_rcp(uint32_t f) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"((float)f));
    return r;
}

__device__ __forceinline__ EncSym enc_sym(uint32_t e) {
    EncSym s;
    s.f = e >> 16;
    s.c = e & 0xFFFFu;
    s.rcp = enc_rcp(s.f);
    return s;
}

__device__ __forceinline__ uint32_t enc_update(uint32_t x, const EncSym& q) {
    uint32_t d = __float2uint_rz(__fmul_rn(__uint2float_rn(x), q.rcp));
    int r = (int)(x - d * q.f);
    const bool lo = r < 0;
    d -= lo ? 1u : 0u;
    r += lo ? (int)q.f : 0;
    const bool hi = r >= (int)q.f;
    d += hi ? 1u : 0u;
    r -= hi ? (int)q.f : 0;
    return (d << 16) + (uint32_t)r + q.c;
}

// STAGE: the lanes' words are staged in shared memory (after the tables) instead of the global rows; the
// block copies them to their place either way.  A block codes S.lpb lanes (its first S.lpb threads); all
// its threads copy.
// HELP (one warp of lanes per block, staged, the latency-bound case): warp 1 serves the coding warp
// through a shared-memory ring of four groups of 16 steps: it loads each element's symbol and scale index,
// checks them and writes the table word ((freq << 16) | cum) and the reciprocal of the frequency, so the
// coding warp's step is the state chain and the store of its renormalisation word.  Hand-over through
// mbarriers with bounded waits.
constexpr int kEncRingBytes = 4 * kPF * 32 * 8;
// the producer's raw rows: per group, 16 rows of 32 indices (32 B) and 32 symbols (64 B), four groups
constexpr int kEncRawGroups = 4;
constexpr int kEncRawBytes = kEncRawGroups * kPF * 96;
constexpr int kEncHelpExtra = kEncRingBytes + 128 + kEncRawBytes;  // ring, 8 barriers, raw rows
template <bool STAGE, bool HELP = false>
__global__ void __launch_bounds__(512) rans_encode_kernel(const RansEncJob J, const uint32_t* __restrict__ tables) {
    extern __shared__ __align__(16) uint32_t tab[];  // [64][511] (freq << 16) | cum, then the staged words
    __shared__ uint64_t bar;
    __shared__ uint32_t scan_sh[32];
    __shared__ int ticket_sh, last_sh, abort_sh;
    __shared__ unsigned long long pre_sh, base_sh;
    RansCtl* ctl = J.ctl;
    const int BT = blockDim.x;
    uint16_t* stage = reinterpret_cast<uint16_t*>(reinterpret_cast<uint8_t*>(tab) + kEncTabBytes);
    const bool loaded = __syncthreads_and(load_table(tab, tables, kEncTabBytes, &bar, J.status, J.spin));
    if (loaded) pdl_trigger();  // the tables are constants: loaded while the previous kernel finishes
    pdl_wait();                 // the symbols, the control block and the output are touched below only
    if (threadIdx.x == 0) {
        ticket_sh = loaded ? (int)atomicAdd(&ctl->ticket, 1u) : -1;
        abort_sh = 0;
    }
    __syncthreads();
    const int t = ticket_sh;
    if (!loaded || t < 0 || t >= J.grid) goto done;
    {
        int si = 0;  // the section of this ticket (sections take consecutive ticket ranges)
        while (si + 1 < J.nsec && t >= J.s[si + 1].first) ++si;
        const RansEncSec& S = J.s[si];
        const RansEncStream& O = J.st[S.stream];
        const int T = S.lpb;         // this section's lanes per block
        const int bs = t - S.first;  // block within the section
        const int lane = bs * T + threadIdx.x;
        const bool live = (int)threadIdx.x < T && lane < S.K;
        const uint32_t cnt = live ? lane_elems(S.n, S.K, lane) : 0u;
        uint16_t* row = STAGE ? stage + (size_t)(live ? threadIdx.x : 0) * S.cap_lane
                              : S.rows + (size_t)(live ? lane : 0) * S.cap_lane;
        uint32_t words = 0;
        // HELP: whole groups of 16 steps below the lanes' common element count, coded from the ring
        uint32_t ngr = 0, cmin = 0;
        int hx_wp = S.cap_lane;
        uint32_t hx_x = kRansL, hx_bad = 0;
        if constexpr (HELP) {
            static_assert(STAGE, "serving warp: staged words");
            __shared__ uint32_t ngr_sh, cmin_sh;
            const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
            uint2* ring = reinterpret_cast<uint2*>(reinterpret_cast<uint8_t*>(stage) + J.stage_bytes);
            uint64_t* hb = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(ring) + kEncRingBytes);
            // raw rows of group g in slot g % 4: indices [16][32] u8, then symbols [16][32] s16
            uint8_t* raw = reinterpret_cast<uint8_t*>(hb) + 128;
            if (threadIdx.x == 0) {
                for (int k = 0; k < 8; ++k) ptx::mbar_init(&hb[k], 1);  // full[4], empty[4]
                ptx::fence_mbar_init();
            }
            if (w == 0) {
                const uint32_t cm = __reduce_min_sync(0xffffffffu, live ? cnt : 0u);
                const bool f = S.idx_period == 0 && __all_sync(0xffffffffu, live);
                if (l == 0) {
                    cmin_sh = cm;
                    ngr_sh = f ? cm / kPF : 0u;
                }
            }
            __syncthreads();
            ngr = ngr_sh;
            cmin = cmin_sh;
            auto hwait = [&](uint64_t* b, uint32_t par) {
                const long long t0 = clock64();
                while (!ptx::mbar_try_wait(b, par))
                    if (clock64() - t0 > kSpinDefault) {
                        set_status(J.status, UFVC_ERR_TIMEOUT);
                        return false;
                    }
                return true;
            };
            const int K = S.K;
            const size_t lane0 = (size_t)bs * T;
            if (w == 1) {
                // ---- producer: group g holds the elements m = cmin - 1 - 16 g - u of the warp's lanes.  When
                //      the rows are 16-byte aligned, each row of a group (32 indices, 32 symbols) arrives by a
                //      bulk copy issued four groups ahead, so the loads' latency overlaps the coding; else
                //      the lanes load their elements directly
                const bool bulk = ((reinterpret_cast<uintptr_t>(S.idx) | reinterpret_cast<uintptr_t>(S.sym)) & 15) == 0 &&
                                  (K & 15) == 0 && (lane0 & 15) == 0;
                // lane l copies 16 bytes of the index rows (row l / 2, half l & 1) and 32 bytes of the symbol
                // rows (row l / 2, quarters 2 (l & 1) and 2 (l & 1) + 1) of group g into raw slot g % 4
                auto issue = [&](uint32_t g) {
                    if (g < ngr) {
                        uint8_t* dst = raw + (g % kEncRawGroups) * (kPF * 96);
                        const int u = l >> 1, h = l & 1;
                        const size_t e = lane0 + (size_t)(cmin - 1 - kPF * g - u) * K;
                        ptx::cp_async16(dst + u * 32 + 16 * h, S.idx + e + 16 * h);
                        ptx::cp_async16(dst + kPF * 32 + u * 64 + 32 * h, S.sym + e + 16 * h);
                        ptx::cp_async16(dst + kPF * 32 + u * 64 + 32 * h + 16, S.sym + e + 16 * h + 8);
                    }
                    ptx::cp_async_commit();  // (an empty group past the last keeps the count)
                };
                if (bulk)
                    for (uint32_t g = 0; g < (uint32_t)kEncRawGroups; ++g) issue(g);
                uint32_t bad = 0;
                for (uint32_t g = 0; g < ngr; ++g) {
                    const int b = (int)(g & 3);
                    const uint32_t use = g >> 2;
                    uint32_t tv[kPF];
                    int sv[kPF];
                    if (bulk) {
                        ptx::cp_async_wait<kEncRawGroups - 1>();  // this lane's copies of group g have landed
                        __syncwarp();                              // and every lane's
                        const uint8_t* src = raw + (g % kEncRawGroups) * (kPF * 96);
#pragma unroll
                        for (int u = 0; u < kPF; ++u) {
                            tv[u] = src[u * 32 + l];
                            sv[u] = reinterpret_cast<const int16_t*>(src + kPF * 32)[u * 32 + l];
                        }
                        __syncwarp();  // the slot is read: group g + 4 may overwrite it
                        issue(g + kEncRawGroups);
                    } else {
#pragma unroll
                        for (int u = 0; u < kPF; ++u) {
                            const size_t e = lane0 + l + (size_t)(cmin - 1 - kPF * g - u) * K;
                            tv[u] = __ldg(S.idx + e);
                            sv[u] = __ldg(S.sym + e);
                        }
                    }
                    if (use > 0 && !__all_sync(0xffffffffu, hwait(&hb[4 + b], (use - 1) & 1))) break;
#pragma unroll
                    for (int u = 0; u < kPF; ++u) {
                        const uint32_t v = (uint32_t)(sv[u] + kRmax);
                        const bool ok = tv[u] < (uint32_t)kBins && v < (uint32_t)kNsym;
                        bad |= !ok;
                        const uint32_t ent = tab[ok ? tv[u] * kNsym + v : kRmax];
                        ring[(b * kPF + u) * 32 + l] = make_uint2(ent, __float_as_uint(enc_rcp(ent >> 16)));
                    }
                    __syncwarp();
                    if (l == 0) ptx::mbar_arrive(&hb[b]);
                }
                if (bulk) ptx::cp_async_wait<0>();  // nothing in flight when the block's shared memory is freed
                if (bad) set_status(J.status, UFVC_ERR_ARG);
            } else if (w == 0 && ngr > 0) {
                // ---- coding warp: first the top element of the lanes that have one more, then the groups
                uint16_t* hrow = stage + (size_t)threadIdx.x * S.cap_lane;
                if (cnt > cmin) {
                    const size_t e = lane0 + l + (size_t)cmin * K;
                    const uint32_t tt = __ldg(S.idx + e), v = (uint32_t)(__ldg(S.sym + e) + kRmax);
                    const bool ok = tt < (uint32_t)kBins && v < (uint32_t)kNsym;
                    hx_bad |= !ok;
                    const EncSym q = enc_sym(tab[ok ? tt * kNsym + v : kRmax]);
                    const bool o = hx_x >= (q.f << 16);
                    if (o) hrow[--hx_wp] = (uint16_t)hx_x;
                    hx_x = o ? hx_x >> 16 : hx_x;
                    hx_x = enc_update(hx_x, q);
                }
                for (uint32_t g = 0; g < ngr; ++g) {
                    const int b = (int)(g & 3);
                    const uint32_t use = g >> 2;
                    if (!__all_sync(0xffffffffu, hwait(&hb[b], use & 1))) break;
                    uint2 rv[kPF];
#pragma unroll
                    for (int u = 0; u < kPF; ++u) rv[u] = ring[(b * kPF + u) * 32 + l];
#pragma unroll
                    for (int u = 0; u < kPF; ++u) {
                        EncSym q;
                        q.f = rv[u].x >> 16;
                        q.c = rv[u].x & 0xFFFFu;
                        q.rcp = __uint_as_float(rv[u].y);
                        const bool o = hx_x >= (q.f << 16);
                        if (o) hrow[--hx_wp] = (uint16_t)hx_x;
                        hx_x = o ? hx_x >> 16 : hx_x;
                        hx_x = enc_update(hx_x, q);
                    }
                    __syncwarp();
                    if (l == 0) ptx::mbar_arrive(&hb[4 + b]);
                }
            }
        }
        if (live) {
            int wp = S.cap_lane;
            uint32_t x = kRansL, bad = 0;
            if (HELP && ngr > 0) {  // continue below the ring's groups
                wp = hx_wp;
                x = hx_x;
                bad = hx_bad;
            }
            const int K = S.K, per = S.idx_period;
            // per-channel tables: index of element lane + m K is (lane + m K) mod per, stepped down by K mod per
            const int kmod = per ? K % per : 0;
            int ip = per && cnt ? (int)(((uint64_t)lane + (uint64_t)(cnt - 1) * K) % (uint64_t)per) : 0;
            // the loaded values stay untouched until their step: any arithmetic on them here would wait for
            // the load, and the loads are predicated so that nothing merges them either
            unsigned short tc[kPF], tn[kPF];
            short vc[kPF], vn[kPF];
            uint32_t fe = (uint32_t)lane + (cnt ? (cnt - 1u) * (uint32_t)K : 0u);  // element of the next fetch
            auto fetch = [&](int mtop, unsigned short* td, short* vd) {
#pragma unroll
                for (int u = 0; u < kPF; ++u) {
                    const bool ok = mtop - u >= 0;
                    td[u] = 0;
                    vd[u] = 0;
                    ld_if_u8(td[u], per ? S.idx + ip : S.idx + fe, ok);
                    ld_if_s16(vd[u], S.sym + fe, ok);
                    if (per) {  // (uniform per block: one section per block)
                        const int nip = ip - kmod;
                        ip = ok ? (nip < 0 ? nip + per : nip) : ip;
                    }
                    fe -= ok ? (uint32_t)K : 0u;
                }
            };
            // The renormalisation words of a group are kept in registers and stored after the group: a
            // store reads its registers late (the rows are scattered, one per lane), and the state chain
            // must not wait for that before it overwrites its own registers.
            uint32_t wbuf[kPF];
            uint32_t emit = 0;  // bit u: step u of the group emitted wbuf[u]
            auto step = [&](int u, uint32_t tt, int sv) {
                const uint32_t v = (uint32_t)(sv + kRmax);  // (tt, sv: the raw loaded index and symbol)
                const bool ok = tt < (uint32_t)kBins && v < (uint32_t)kNsym;
                bad |= !ok;
                const EncSym q = enc_sym(tab[ok ? tt * kNsym + v : kRmax]);
                const bool o = x >= (q.f << 16);
                if (STAGE) {  // shared memory: stored at once
                    if (o) row[--wp] = (uint16_t)x;
                } else {
                    wbuf[u] = x & 0xFFFFu;
                    emit |= o ? 1u << u : 0u;
                }
                x = o ? x >> 16 : x;
                x = enc_update(x, q);
            };
            auto flush = [&]() {  // the group's words, in emission order, backwards into the row
                if constexpr (!STAGE) {
#pragma unroll
                    for (int u = 0; u < kPF; ++u)
                        if (emit & (1u << u)) row[--wp] = (uint16_t)wbuf[u];
                    emit = 0;
                }
            };
            const int top = (HELP && ngr > 0) ? (int)(cmin - kPF * ngr) - 1 : (int)cnt - 1;
            if (HELP && ngr > 0) fe = (uint32_t)lane + (top > 0 ? (uint32_t)top * (uint32_t)K : 0u);
            fetch(top, tc, vc);
            int mtop = top;
            for (; mtop >= kPF - 1; mtop -= kPF) {  // whole groups of kPF symbols
                fetch(mtop - kPF, tn, vn);
#pragma unroll
                for (int u = 0; u < kPF; ++u) step(u, tc[u], vc[u]);
                flush();
#pragma unroll
                for (int u = 0; u < kPF; ++u) { tc[u] = tn[u]; vc[u] = vn[u]; }
            }
#pragma unroll
            for (int u = 0; u < kPF; ++u)  // the remaining mtop + 1 < kPF symbols
                if (u <= mtop) step(u, tc[u], vc[u]);
            flush();
            if (bad) set_status(J.status, UFVC_ERR_ARG);
            row[--wp] = (uint16_t)(x & 0xFFFFu);
            row[--wp] = (uint16_t)(x >> 16);
            words = (uint32_t)(S.cap_lane - wp);
        }
        // ---- layout: this block's word prefix within its section.  Warp 0 looks back over the published
        //      totals of the section's earlier blocks 32 at a time: it sums aggregates down to the nearest
        //      block that published its inclusive prefix (waiting, bounded, where one has not published yet)
        uint32_t agg;
        const uint32_t excl = block_excl_scan(words, &agg, scan_sh);
        if (threadIdx.x < 32) {
            const int l = threadIdx.x;
            const int first = S.first;  // the section's first ticket
            uint64_t pre = 0;
            bool ok = true;
            if (l == 0) ptx::st_release_u64(&ctl->flag[t], (t == first ? kFlagIncl : kFlagAgg) | agg);
            const long long t0 = clock64();
            for (int j = t - 1; j >= first && ok;) {
                const int jj = j - l;
                const uint64_t f = jj >= first ? ptx::ld_acquire_u64(&ctl->flag[jj]) : kFlagIncl;  // start: 0
                const unsigned incl = __ballot_sync(0xffffffffu, (f & kFlagIncl) != 0);
                const unsigned pub = __ballot_sync(0xffffffffu, (f & (kFlagIncl | kFlagAgg)) != 0);
                const int ni = incl ? __ffs(incl) - 1 : 31;  // the window's last lane to add
                const unsigned need = ni == 31 ? 0xffffffffu : (2u << ni) - 1u;
                if ((pub & need) != need) {  // a block in the window has not published yet: poll again
                    ok = __all_sync(0xffffffffu, clock64() - t0 <= kSpinDefault);
                    continue;
                }
                uint64_t v = l <= ni ? (f & kFlagMask) : 0ull;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                pre += v;
                if (incl) break;
                j -= 32;
            }
            if (l == 0) {
                if (ok && t != first) ptx::st_release_u64(&ctl->flag[t], kFlagIncl | (pre + agg));
                uint64_t base = O.base;
                if (ok && S.prev >= 0) {  // the y^ section follows the z^ section: its total is the last z^ block's
                    const RansEncSec& P = J.s[S.prev];
                    const int lz = P.first + P.nblk - 1;
                    uint64_t f;
                    while (!((f = ptx::ld_acquire_u64(&ctl->flag[lz])) & kFlagIncl))
                        if (clock64() - t0 > kSpinDefault) { ok = false; break; }
                    if (ok) base = (O.base + 4ull * P.K + 2ull * (f & kFlagMask) + 3ull) & ~3ull;
                }
                if (!ok) {
                    set_status(J.status, UFVC_ERR_TIMEOUT);
                    abort_sh = 1;
                }
                pre_sh = pre;
                base_sh = base;
            }
        }
        __syncthreads();
        if (abort_sh) goto done;
        {
            const uint64_t base = base_sh, words_at = base + 4ull * S.K;
            const uint64_t off = words_at + 2ull * (pre_sh + excl);
            uint8_t* out = O.out;
            const uint64_t cap = O.capacity;
            if (live && base + 4ull * lane + 4 <= cap) {
                uint8_t* c = out + base + 4ull * lane;
                c[0] = words & 0xFF; c[1] = (words >> 8) & 0xFF; c[2] = (words >> 16) & 0xFF; c[3] = words >> 24;
            }
            // the block's lanes' words, one warp per lane at a time, eight loads in flight per thread
            // (offsets and counts through shared memory, in the tables' place)
            uint64_t* offs = reinterpret_cast<uint64_t*>(tab);
            uint32_t* cnts = reinterpret_cast<uint32_t*>(offs + T);
            __syncthreads();
            if ((int)threadIdx.x < T) {
                offs[threadIdx.x] = off;
                cnts[threadIdx.x] = live ? words : 0u;
            }
            __syncthreads();
            const int l = threadIdx.x & 31;
            for (int k = threadIdx.x >> 5; k < T; k += BT >> 5) {
                const uint32_t wk = cnts[k];
                const uint64_t ok_ = offs[k];
                if (wk == 0 || ok_ + 2ull * wk > cap) continue;
                const uint16_t* src = (STAGE ? stage + (size_t)k * S.cap_lane
                                             : S.rows + (size_t)(bs * T + k) * S.cap_lane) + (S.cap_lane - wk);
                uint16_t* dst = reinterpret_cast<uint16_t*>(out + ok_);
                for (uint32_t w0 = l; w0 < wk; w0 += 32 * 8) {
                    uint16_t v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) v[u] = w0 + 32u * u < wk ? src[w0 + 32u * u] : (uint16_t)0;
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (w0 + 32u * u < wk) dst[w0 + 32u * u] = v[u];
                }
            }
            if (bs == S.nblk - 1 && threadIdx.x == 0) {  // the section's last block: padding, and the size
                const uint64_t end = words_at + 2ull * (pre_sh + agg), end4 = (end + 3) & ~3ull;
                for (uint64_t b = end; b < end4; ++b)
                    if (b < cap) out[b] = 0;
                if (S.last) {
                    *O.nbytes = end4;
                    if (end4 > cap) set_status(J.status, UFVC_ERR_CAPACITY);
                }
            }
            if (bs == 0 && S.prev < 0 && O.hdr_len > 0) {  // the stream's container header
                if ((uint64_t)O.hdr_len > cap) {
                    if (threadIdx.x == 0) set_status(J.status, UFVC_ERR_CAPACITY);
                } else {
                    for (int i = threadIdx.x; i < O.hdr_len; i += BT)
                        out[i] = i < 20 ? O.hdr20[i] : i < 20 + O.cz ? O.iz[i - 20] : 0;
                }
            }
        }
    }
done:
    // the last block to finish resets the control block for the next launch
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last_sh = atomicAdd(&ctl->done, 1u) == (unsigned)(J.grid - 1);
    }
    __syncthreads();
    if (last_sh) {
        for (int i = threadIdx.x; i < J.grid && i < kRansMaxBlocks; i += BT) ctl->flag[i] = 0;
        if (threadIdx.x == 0) {
            ctl->ticket = 0;
            ctl->done = 0;
        }
        __threadfence();
    }
}

// Threads per block (lanes per block) for the job's sections: the smallest multiple of 32 for which their
// blocks fit in one wave of one block per SM, at most 512 (more sections or lanes then take more than one
// wave: a block only ever waits on blocks that started before it).
static int enc_threads(const RansEncJob& j, int sms) {
    for (int T = 32; T < 512; T += 32) {
        int b = 0;
        for (int i = 0; i < j.nsec; ++i) b += (j.s[i].K + T - 1) / T;
        if (b <= sms) return T;
    }
    return 512;
}

cudaError_t launch_rans_encode(RansEncJob& j, const uint32_t* packed_tables, cudaStream_t s) {
    if (j.nsec < 1 || j.nsec > kRansMaxEncSec || j.nstreams < 1 || j.nstreams > kRansMaxStreams)
        return cudaErrorInvalidValue;
    int T = enc_threads(j, sm_count());
    // few lanes per SM (the latency-bound case): one warp of lanes per block with its serving warp, when
    // the blocks stay within the control block and the words, the ring and the tables fit
    bool help = false;
    size_t st_help = 0;  // the staged words' bytes the serving-warp layout was checked with
    if (T <= 64) {
        int b32 = 0, cap32 = 0;
        for (int i = 0; i < j.nsec; ++i) {
            b32 += (j.s[i].K + 31) / 32;
            cap32 = j.s[i].cap_lane > cap32 ? j.s[i].cap_lane : cap32;
        }
        const size_t st32 = ((size_t)32 * cap32 * 2 + 15) & ~(size_t)15;
        help = b32 <= kRansMaxBlocks && kEncTabBytes + st32 + kEncHelpExtra <= (size_t)kEncSmemMax;
        if (help) {
            T = 32;
            st_help = st32;
        }
    }
    j.lpb = T;
    j.grid = 0;
    size_t stage_max = 0;  // the largest block's staged words
    for (int i = 0; i < j.nsec; ++i) {
        RansEncSec& e = j.s[i];
        if (e.K < 1 || e.stream < 0 || e.stream >= j.nstreams) return cudaErrorInvalidValue;
        // with serving warps (one warp of lanes per block), a section with per-channel tables (the z^
        // section: 16 steps per lane, no serving warp) takes up to 512 lanes per block, so that its few
        // blocks leave the SMs to the long y^ blocks instead of holding 128 of them at the start
        e.lpb = T;
        if (help && e.idx_period > 0) {  // (its rows must fit in the staged words checked above)
            int l = (e.K + 31) / 32 * 32;
            l = l < 512 ? l : 512;
            const long long fit = (long long)(st_help / (2ull * (e.cap_lane > 0 ? e.cap_lane : 1))) / 32 * 32;
            l = l < fit ? l : (int)fit;
            e.lpb = l > 32 ? l : 32;
        }
        j.lpb = e.lpb > j.lpb ? e.lpb : j.lpb;
        e.nblk = (e.K + e.lpb - 1) / e.lpb;
        e.first = j.grid;
        j.grid += e.nblk;
        // a stream's sections are consecutive: the one before it in the same stream, and whether it ends it
        e.prev = i > 0 && j.s[i - 1].stream == e.stream ? i - 1 : -1;
        e.last = i + 1 == j.nsec || j.s[i + 1].stream != e.stream;
        if (e.prev >= 0 && j.s[e.prev].prev >= 0) return cudaErrorInvalidValue;  // at most two per stream
        const size_t st = (size_t)e.lpb * e.cap_lane * 2;
        stage_max = st > stage_max ? st : stage_max;
    }
    if (j.grid > kRansMaxBlocks) return cudaErrorInvalidValue;
    // the words go through shared memory when every lane's row fits there beside the tables; then the
    // block needs few threads to copy them, else 512 copy from the global rows
    const size_t stage = (stage_max + 15) & ~(size_t)15;
    const bool staged = kEncTabBytes + stage <= (size_t)kEncSmemMax;
    if (!staged && help) return cudaErrorInvalidValue;  // (help was chosen with the rows fitting)
    const int BT = staged ? (j.lpb < 128 ? 128 : j.lpb) : 512;
    j.stage_bytes = (int)stage;
    // the shared memory holds the tables (then the lanes' offsets and counts, 12 bytes each) and the stage
    // (HELP: then the ring, its barriers and the producer's raw rows)
    const int smem = (int)(kEncTabBytes + (staged ? stage : 0) + (help ? kEncHelpExtra : 0));
    const void* kern = help     ? (const void*)rans_encode_kernel<true, true>
                       : staged ? (const void*)rans_encode_kernel<true>
                                : (const void*)rans_encode_kernel<false>;
    cudaError_t e = smem_optin(kern, smem);
    if (e != cudaSuccess) return e;
    if (help)
        return launch_pdl(rans_encode_kernel<true, true>, dim3(j.grid), dim3(BT), (size_t)smem, s, j, packed_tables);
    if (staged) return launch_pdl(rans_encode_kernel<true>, dim3(j.grid), dim3(BT), (size_t)smem, s, j, packed_tables);
    return launch_pdl(rans_encode_kernel<false>, dim3(j.grid), dim3(BT), (size_t)smem, s, j, packed_tables);
}

size_t rans_ctl_bytes() { return sizeof(RansCtl); }

// ------------------------------------------------------------------------------------------------
// decode
// ------------------------------------------------------------------------------------------------
// Decoding tables (built on the host, build_decode_tables): for table t and bucket b of 256 slots a
// 64-bit entry, low word s0 | f0 << 9 | d << 25, high word c0 | f1 << 16, where s0 owns the bucket's
// first slot outside the unit-frequency end runs, c0 = cum(s0), f0 = freq(s0), f1 = freq(s0 + 1) and
// d = min(127, the last symbol of the bucket - s0); then per table A | B << 16, the lengths of the end runs
// (symbols 0 .. A-1 and 511-B .. 510 have frequency 1, so there the symbol is the slot, resp. the slot
// - 65025); then cum(s) as u16 [64][512] for the few slots past s0 + 1 (bisection).
constexpr int kDecEntBytes = kBins * 256 * 8;
constexpr int kDecRunBytes = kBins * 4;
constexpr int kDecCumBytes = kBins * 512 * 2;
constexpr int kDecTabBytes = kDecEntBytes + kDecRunBytes + kDecCumBytes;  // 196864
// after the tables: the section's lane counts, brought in by one bulk copy when they fit (K <= 4096), then
// one output tile of 16 steps x 32 lanes (int16) per warp
constexpr int kDecCntBytes = 4 * 4096 + 32;
constexpr int kDecTileOff = kDecTabBytes + kDecCntBytes;
constexpr int kDecMaxWarps = 16;
constexpr int kDecSmemBytes = kDecTileOff + kDecMaxWarps * 16 * 32 * 2;

// HELP (one warp of lanes per block, the latency-bound case): three more warps serve the decoding warp
// through shared memory, in groups of 16 steps: warp 1 stages the lanes' scale indices in a ring four
// groups ahead, warp 3 copies each lane's next stream words into a window one group ahead (so a
// renormalisation reads its word from shared memory, off the global-load latency), and warp 2 takes the
// symbols from a ring and writes y^ = r^ q + mu (or r^) as 16-byte vectors; the decoding warp issues
// little besides the state chain.  The hand-overs are mbarriers with bounded waits.
template <int OUT, bool PER, bool HELP = false>
__global__ void __launch_bounds__(512) rans_decode_kernel(const RansDecJob J, const uint8_t* __restrict__ tables) {
    extern __shared__ __align__(16) uint8_t dsm[];
    const uint2* ent = reinterpret_cast<const uint2*>(dsm);
    const uint32_t* runs = reinterpret_cast<const uint32_t*>(dsm + kDecEntBytes);
    const uint16_t* cum = reinterpret_cast<const uint16_t*>(dsm + kDecEntBytes + kDecRunBytes);
    __shared__ uint64_t bar;
    __shared__ uint32_t scan_sh[32];
    __shared__ uint64_t red_sh[32];
    __shared__ int bad_sh;
    const int si = blockIdx.x / J.bps, blk = blockIdx.x - si * J.bps;  // section, block within it
    const RansDecSec& S = J.s[si];
    const bool loaded = __syncthreads_and(load_table(dsm, tables, kDecTabBytes, &bar, J.status, J.spin));
    if (loaded) pdl_trigger();
    pdl_wait();
    // the rate and version the later kernels read are always written (defaults unless the header is good)
    if (J.hdr_cz > 0 && blk == 0 && threadIdx.x == 0) {
        *S.qp_out = 32;
        *S.ver_out = 1;
    }
    if (threadIdx.x == 0) bad_sh = *(volatile int*)J.status != 0;  // an earlier stage failed: nothing to do
    __syncthreads();
    if (!loaded || bad_sh) return;
    const uint8_t* bits = S.bits;
    const uint64_t nbytes = S.nbytes;
    // T: lanes per block (its first T threads); NT: all threads (HELP: the two serving warps besides)
    const int K = J.K, T = HELP ? 32 : (int)blockDim.x, NT = blockDim.x;
    // ---- container header (the z^ section's launch): every block checks it; block 0 publishes the rate
    //      and the version for the later kernels
    if (J.hdr_cz > 0) {
        const uint64_t hdr = (20ull + J.hdr_cz + 3) & ~3ull;
        const bool whole = nbytes >= hdr;
        bool iz_bad = false;  // the scale indices, checked by all threads
        for (int c = threadIdx.x; whole && c < J.hdr_cz; c += NT) iz_bad |= bits[20 + c] >= kBins;
        iz_bad = __syncthreads_or(iz_bad);
        if (threadIdx.x == 0) {
            int st = 0, qp = 32, ver = 1;
            if (!whole || bits[0] != 'U' || bits[1] != 'F' || bits[2] != 'V' || bits[3] != 'C' || bits[4] < 1 ||
                bits[4] > 4) {
                st = UFVC_ERR_CORRUPT;
            } else {
                const int v_pm = bits[4] == 2 || bits[4] == 4, v_tc = bits[4] >= 3;
                const int w = bits[8] | (bits[9] << 8), h = bits[10] | (bits[11] << 8);
                const uint32_t k = bits[12] | (bits[13] << 8) | (bits[14] << 16) | ((uint32_t)bits[15] << 24);
                const uint32_t kz = bits[16] | (bits[17] << 8) | (bits[18] << 16) | ((uint32_t)bits[19] << 24);
                if ((v_pm && !J.allow_pm) || v_tc != J.temporal) st = UFVC_ERR_UNSUPPORTED;
                else if (bits[5] != J.arch || bits[6] != J.N || w != J.W || h != J.H) st = UFVC_ERR_ARG;
                else if (bits[7] > 63 || k != (uint32_t)J.Ky || kz != (uint32_t)K || iz_bad) st = UFVC_ERR_CORRUPT;
                if (!st) {
                    qp = bits[7];
                    ver = v_pm ? 2 : 1;
                }
            }
            if (st) {
                set_status(J.status, st);
                bad_sh = 1;
            }
            if (blk == 0) {
                *S.qp_out = qp;
                *S.ver_out = ver;
            }
        }
        __syncthreads();
        if (bad_sh) return;
    }
    // ---- the section's lane counts: prefix before this block's first lane, and the total
    const uint64_t sec = S.sec_off_dev ? *S.sec_off_dev : S.sec_off;
    if (sec + 4ull * K > nbytes) {
        if (threadIdx.x == 0) set_status(J.status, UFVC_ERR_CORRUPT);
        return;
    }
    const int first = blk * T;
    const uint8_t* cb = bits + sec;
    // the counts' 16-byte aligned superset, when it fits in shared memory and lies inside the stream
    const uintptr_t lo = reinterpret_cast<uintptr_t>(cb) & ~(uintptr_t)15;
    const uintptr_t hi = (reinterpret_cast<uintptr_t>(cb) + 4ull * K + 15) & ~(uintptr_t)15;
    const bool in_smem = hi - lo <= (uintptr_t)kDecCntBytes && lo >= reinterpret_cast<uintptr_t>(bits) &&
                         hi <= reinterpret_cast<uintptr_t>(bits) + nbytes;
    const uint32_t* csm = reinterpret_cast<const uint32_t*>(dsm + kDecTabBytes + (reinterpret_cast<uintptr_t>(cb) - lo));
    if (in_smem) {
        if (threadIdx.x == 0) {
            ptx::mbar_arrive_expect_tx(&bar, (uint32_t)(hi - lo));
            ptx::bulk_load(dsm + kDecTabBytes, reinterpret_cast<const void*>(lo), (uint32_t)(hi - lo), &bar);
        }
        const long long t0 = clock64();
        bool got = true;
        while (!ptx::mbar_test_wait(&bar, 1))
            if (clock64() - t0 > kSpinDefault) { got = false; break; }
        if (!__syncthreads_and(got)) {
            if (threadIdx.x == 0) {
                set_status(J.status, UFVC_ERR_TIMEOUT);
                const long long t1 = clock64();  // the copy in flight lands before the block exits
                while (!ptx::mbar_test_wait(&bar, 1) && clock64() - t1 < kSpinDefault) {
                }
            }
            return;
        }
    }
    const bool al = (reinterpret_cast<uintptr_t>(cb) & 3) == 0;
    auto count_at = [&](int j) -> uint32_t {
        if (in_smem) return csm[j];
        if (al) return __ldg(reinterpret_cast<const uint32_t*>(cb) + j);
        const uint8_t* p = cb + 4ull * j;
        return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
    };
    uint64_t pre = 0, tot = 0;
    for (int j0 = threadIdx.x; j0 < K; j0 += 16 * NT) {  // sixteen loads in flight per thread
        uint32_t c[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) c[k] = j0 + k * NT < K ? count_at(j0 + k * NT) : 0u;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            tot += c[k];
            pre += j0 + k * NT < first ? c[k] : 0u;
        }
    }
    pre = block_sum_u64(pre, red_sh);
    tot = block_sum_u64(tot, red_sh);
    const uint64_t words_at = sec + 4ull * K;
    const uint64_t end4 = (words_at + 2ull * tot + 3ull) & ~3ull;
    const uint64_t expect = S.expect_end_dev ? *S.expect_end_dev : S.expect_end;
    if (end4 > nbytes || (expect != 0 && end4 != expect)) {
        if (threadIdx.x == 0) set_status(J.status, UFVC_ERR_CORRUPT);
        return;
    }
    if (blk == 0 && threadIdx.x == 0 && S.next_off) *S.next_off = end4;
    const int lane = first + threadIdx.x;
    const bool inl = (int)threadIdx.x < T && lane < K;
    const uint32_t words = inl ? count_at(lane) : 0u;
    uint32_t btot;
    const uint32_t excl = block_excl_scan(words, &btot, scan_sh);
    // From here on a warp steps in lock-step (the rare bisection below is a lane's own branch; the warp
    // reconverges after it): lanes past K, and
    // lanes with a bad count, take part without coding; a warp with no lane left returns.
    if (!HELP && __all_sync(0xffffffffu, !inl)) return;  // (HELP: the block's lanes are its warp 0, all < K)
    const uint32_t n = J.n, cnt = inl ? lane_elems(n, K, lane) : 0u;
    const bool okc = inl && words >= 2 && words <= cnt + 2;  // every read below stays inside the lane's words
    if (inl && !okc) set_status(J.status, UFVC_ERR_CORRUPT);
    const uint32_t mine = okc ? cnt : 0u;
    const uint32_t cmax = __reduce_max_sync(0xffffffffu, mine);
    const uint32_t nw = okc ? words : 2u;
    const uint16_t* wp = reinterpret_cast<const uint16_t*>(bits + words_at + 2ull * (pre + excl));
    if (!okc) wp = reinterpret_cast<const uint16_t*>(S.bits);  // not read (every step of this lane is idle)
    // the lane's words in decoding order: the state, then one word per renormalisation
    uint32_t x = okc ? (ld_u16(wp) << 16) | ld_u16(wp + 1) : kRansL;
    uint32_t r = 2;                                                        // next word to read
    uint32_t w0 = okc ? ld_u16(wp + (2 < nw ? 2 : nw - 1)) : 0u;          // words r and r + 1, fetched ahead
    unsigned short w1 = okc ? (unsigned short)ld_u16(wp + (3 < nw ? 3 : nw - 1)) : (unsigned short)0;
    float q = 0.f;
    if (OUT != kDecSym) q = J.qstep_all[S.qp_dev ? *S.qp_dev : J.qp_host];
    const int per = J.idx_period;
    const int kmod = PER ? K % per : 0;
    int ip = PER && okc ? lane % per : 0;
    const uint32_t cmin = __reduce_min_sync(0xffffffffu, okc ? cnt : 0xFFFFFFFFu);  // every lane has these
    unsigned short tc[kPF], tn[kPF];
    float mc[kPF], mn[kPF];
    uint32_t fi = (uint32_t)lane;  // element of the next fetch (sections hold fewer than 2^31 elements)
    bool tile_mode = false;        // the fast path below reads mu itself
    auto fetch = [&](uint32_t m0, unsigned short* td, float* md) {
#pragma unroll
        for (int u = 0; u < kPF; ++u) {
            const bool ok = m0 + (uint32_t)u < mine;
            td[u] = 0;
            md[u] = 0.f;
            ld_if_u8(td[u], PER ? S.idx + ip : S.idx + fi, ok);
            if (OUT != kDecSym && !tile_mode) ld_if_f32(md[u], S.mu + fi, ok);
            if (PER) {
                const int nip = ip + kmod;
                ip = ok ? (nip >= per ? nip - per : nip) : ip;
            }
            fi += ok ? (uint32_t)K : 0u;
        }
    };
    uint32_t bad = 0;
    uint32_t i = (uint32_t)lane;  // element of the next output
    // the lane's words staged in shared memory (HELP groups): word r is win_cur[r + woff]
    const uint16_t* win_cur = nullptr;
    int woff = 0;
    // one symbol of this lane where act (ALL: known to hold for every lane of the warp; SMW: the words come
    // from the shared-memory window, else from the lane's global row through w0 / w1); returns it
    auto decode = [&](uint32_t t, bool act, auto all, auto smw) -> uint32_t {
        if constexpr (decltype(all)::value) act = true;
        bad |= t;
        t &= (uint32_t)(kBins - 1);
        const uint32_t slot = x & 0xFFFFu, xh = x >> 16;
        const uint2 e = ent[t * 256 + (slot >> 8)];
        const uint32_t ab = runs[t];
        const bool tl = slot < (ab & 0xFFFFu), tr = slot >= kProbM - (ab >> 16);
        const uint32_t s0 = e.x & 511u, c0 = e.y & 0xFFFFu, f0 = (e.x >> 9) & 0xFFFFu;
        const uint32_t f1 = e.y >> 16, b1 = c0 + f0;
        // the next state for both candidates, s0 and s0 + 1, computed before the choice (off the chain)
        const uint32_t xn0 = f0 * xh + (slot - c0), xn1 = f1 * xh + (slot - b1);
        const bool h = slot >= b1;
        uint32_t xn = h ? xn1 : xn0;
        uint32_t s = s0 + (h ? 1u : 0u);
        xn = tl || tr ? xh : xn;  // the tails: f = 1, c = slot
        s = tl ? slot : tr ? slot - (kProbM - kNsym) : s;
        const uint32_t d = e.x >> 25;
        const bool far = act && d >= 2u && slot >= b1 + f1 && !tl && !tr;
        {  // (a lane's own branch: a warp vote before it cost more on the chain than the rare divergence)
            if (far) {  // the slot lies past s0 + 1: bisection over the bucket's remaining symbols
                const uint16_t* C = cum + t * 512;
                uint32_t lo = s0 + 2, hi = s0 + (d < 127u ? d : 255u);
                hi = hi < (uint32_t)(kNsym - 1) ? hi : (uint32_t)(kNsym - 1);
                while (lo < hi) {
                    const uint32_t mid = (lo + hi + 1) >> 1;
                    if (C[mid] <= slot) lo = mid; else hi = mid - 1;
                }
                s = lo;
                const uint32_t c = C[lo];
                const uint32_t f = (lo + 1 < (uint32_t)kNsym ? (uint32_t)C[lo + 1] : kProbM) - c;
                xn = f * xh + slot - c;
            }
        }
        if (act) {
            const bool rn = xn < kRansL;
            x = rn ? (xn << 16) | w0 : xn;
            r += rn ? 1u : 0u;
            if constexpr (decltype(smw)::value) {
                w0 = win_cur[(int)r + woff];  // needed at the next renormalisation only
            } else {
                w0 = rn ? (uint32_t)w1 : w0;
                ld_if_u16(w1, wp + (r + 1 < nw ? r + 1 : nw - 1), rn);
            }
        }
        return s;
    };
    auto yval = [&](int v, float mu) { return __fadd_rn(__fmul_rn((float)v, q), mu); };
    // the generic path's output: one element
    auto put = [&](uint32_t s, float mu) {
        const int v = (int)s - kRmax;
        if (OUT == kDecSym) {
            S.sym[i] = (int16_t)v;
        } else {
            const float yv = yval(v, mu);
            if (OUT == kDecBf16) reinterpret_cast<__nv_bfloat16*>(S.yout)[i] = __float2bfloat16_rn(yv);
            else if (OUT == kDecF32) reinterpret_cast<float*>(S.yout)[i] = yv;
            else reinterpret_cast<uint8_t*>(S.yout)[i] =
                (uint8_t)__nv_cvt_float_to_fp8(yv * J.inv8, __NV_SATFINITE, __NV_E4M3);
        }
        i += (uint32_t)K;
    };
    // the lane's stream is read sequentially: the line 64 words ahead goes to L1 at every group
    auto ahead = [&]() {
        if (okc) asm volatile("prefetch.global.L1 [%0];" ::"l"(wp + (r + 64 < nw ? r + 64 : nw - 1)));
    };
    std::true_type every;
    std::false_type some;
    uint32_t m0 = 0;
    const uintptr_t outp = OUT == kDecSym ? reinterpret_cast<uintptr_t>(S.sym) : reinterpret_cast<uintptr_t>(S.yout);
    if constexpr (HELP) {
        // rings of four groups: indices [4][16 steps][32 lanes] u8, symbols [4][16][32] int16; barriers
        // t_full, t_empty, s_full, s_empty (four each), then w_full, pub (two each), one arrival per phase;
        // each lane's words for a group in a window [2][32 lanes][17] u32 (34 words), and the read positions
        // the decoding warp publishes [2][32]
        uint8_t* ring_t = dsm + kDecTileOff;
        int16_t* ring_s = reinterpret_cast<int16_t*>(dsm + kDecTileOff + 2048);
        uint64_t* hb = reinterpret_cast<uint64_t*>(dsm + kDecTileOff + 6144);
        uint32_t* rpos = reinterpret_cast<uint32_t*>(dsm + kDecTileOff + 6144 + 20 * 8);
        uint32_t* win32 = reinterpret_cast<uint32_t*>(dsm + kDecTileOff + 6144 + 20 * 8 + 256);
        __shared__ uint32_t ngr_sh;
        __shared__ uint64_t lstart[32];  // the lanes' first words, counted from the section's words
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        if (threadIdx.x == 0) {
            for (int k = 0; k < 20; ++k) ptx::mbar_init(&hb[k], 1);
            ptx::fence_mbar_init();
        }
        if (w == 0) {  // whole groups of 16 steps that every lane of the warp codes, with aligned rows
            const bool f = !PER && (K & 15) == 0 && (outp & 15) == 0 &&
                           (reinterpret_cast<uintptr_t>(S.idx) & 15) == 0 &&
                           (reinterpret_cast<uintptr_t>(bits) & 3) == 0 &&
                           (OUT == kDecSym || (reinterpret_cast<uintptr_t>(S.mu) & 15) == 0) &&
                           __all_sync(0xffffffffu, okc && cmin >= (uint32_t)kPF);
            if (l == 0) ngr_sh = f ? cmin / kPF : 0u;
            lstart[l] = pre + excl;
        }
        __syncthreads();
        const uint32_t ngr = ngr_sh;
        auto hwait = [&](uint64_t* b, uint32_t par) {
            const long long t0 = clock64();
            while (!ptx::mbar_try_wait(b, par))
                if (clock64() - t0 > kSpinDefault) {
                    set_status(J.status, UFVC_ERR_TIMEOUT);
                    return false;
                }
            return true;
        };
        if (w == 1) {
            // ---- index stage: lane l copies 16 indices of step 16 g + l / 2 (lanes 16 (l & 1) ..)
            const int u = l >> 1, h = l & 1;
            uint32_t badv = 0;
            for (uint32_t g = 0; g < ngr; ++g) {
                const int b = (int)(g & 3);
                const uint32_t use = g >> 2;
                const uint4 v = __ldg(reinterpret_cast<const uint4*>(S.idx + first + 16 * h + (size_t)(kPF * g + u) * K));
                badv |= (v.x | v.y | v.z | v.w) & 0xC0C0C0C0u;  // an index of 64 or more
                bool ok = true;
                if (use > 0) ok = hwait(&hb[4 + b], (use - 1) & 1);
                if (!__all_sync(0xffffffffu, ok)) break;
                *reinterpret_cast<uint4*>(ring_t + b * 512 + u * 32 + 16 * h) = v;
                __syncwarp();
                if (l == 0) ptx::mbar_arrive(&hb[b]);
            }
            if (badv) set_status(J.status, UFVC_ERR_ARG);
            return;
        }
        if (w == 2) {
            // ---- output: lane l writes elements 16 (l & 1) .. + 15 of step 16 g + l / 2, mu read a group ahead
            const int lr = l >> 1, lh = l & 1;
            float mv[16];
            auto load_mu = [&](uint32_t g) {
                if (OUT == kDecSym) return;
                const bool ok = g < ngr;
                const float4* pm = reinterpret_cast<const float4*>(S.mu + first + 16u * lh + (size_t)(kPF * g + lr) * K);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (ok) v = __ldg(pm + k);
                    mv[4 * k] = v.x; mv[4 * k + 1] = v.y; mv[4 * k + 2] = v.z; mv[4 * k + 3] = v.w;
                }
            };
            load_mu(0);
            for (uint32_t g = 0; g < ngr; ++g) {
                const int b = (int)(g & 3);
                const uint32_t use = g >> 2;
                if (!__all_sync(0xffffffffu, hwait(&hb[8 + b], use & 1))) break;
                const uint4* src = reinterpret_cast<const uint4*>(ring_s + b * 512 + lr * 32 + 16 * lh);
                const uint4 a = src[0], c2 = src[1];
                __syncwarp();
                if (l == 0) ptx::mbar_arrive(&hb[12 + b]);  // the slot is free again
                const size_t e0 = first + 16u * lh + (size_t)(kPF * g + lr) * K;
                const uint32_t wv[8] = {a.x, a.y, a.z, a.w, c2.x, c2.y, c2.z, c2.w};
                if (OUT == kDecSym) {
                    uint4* dst = reinterpret_cast<uint4*>(S.sym + e0);
                    dst[0] = a;
                    dst[1] = c2;
                } else {
                    float y[16];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        y[2 * k] = yval((int)(int16_t)(wv[k] & 0xFFFFu), mv[2 * k]);
                        y[2 * k + 1] = yval((int)(int16_t)(wv[k] >> 16), mv[2 * k + 1]);
                    }
                    if (OUT == kDecBf16) {
                        uint32_t pk[8];
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const __nv_bfloat162 hv = __floats2bfloat162_rn(y[2 * k], y[2 * k + 1]);
                            pk[k] = *reinterpret_cast<const uint32_t*>(&hv);
                        }
                        uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(S.yout) + e0);
                        dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                    } else if (OUT == kDecF32) {
                        float4* dst = reinterpret_cast<float4*>(reinterpret_cast<float*>(S.yout) + e0);
#pragma unroll
                        for (int k = 0; k < 4; ++k) dst[k] = make_float4(y[4 * k], y[4 * k + 1], y[4 * k + 2], y[4 * k + 3]);
                    } else {
                        uint32_t pk[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            uint32_t wd = 0;
#pragma unroll
                            for (int b2 = 0; b2 < 4; ++b2)
                                wd |= (uint32_t)__nv_cvt_float_to_fp8(y[4 * k + b2] * J.inv8, __NV_SATFINITE, __NV_E4M3)
                                      << (8 * b2);
                            pk[k] = wd;
                        }
                        *reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(S.yout) + e0) =
                            make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    }
                }
                load_mu(g + 1);
            }
            return;
        }
        if (w == 3) {
            // ---- word stage: group g reads the lane's words R_g .. R_g + 15, R_g <= R_{g-1} + 16, so the
            //      window of words R_{g-1} .. R_{g-1} + 31 (R_{-1} = 2, the first after the state) serves
            //      it; R_{g-1} is published by the decoding warp when group g - 1 starts, which leaves the
            //      whole of group g - 1 for the copy.  Whole u32 from the 4-byte boundary at or below.
            const uint64_t wbase = words_at + 2ull * lstart[l];  // the lane's words, bytes from `bits`
            for (uint32_t g = 0; g < ngr; ++g) {
                uint32_t rp = 2;
                if (g > 0) {
                    if (!__all_sync(0xffffffffu, hwait(&hb[18 + ((g - 1) & 1)], ((g - 1) >> 1) & 1))) break;
                    rp = rpos[((g - 1) & 1) * 32 + l];
                }
                const uint64_t b0 = (wbase + 2ull * rp) & ~3ull;
                uint32_t* dst = win32 + ((g & 1) * 32 + l) * 17;
#pragma unroll
                for (int k = 0; k < 17; ++k) {
                    const uint64_t o = b0 + 4ull * k;
                    uint32_t v = 0;
                    if (o + 4 <= nbytes) v = __ldg(reinterpret_cast<const uint32_t*>(bits + o));
                    dst[k] = v;
                }
                __syncwarp();
                if (l == 0) ptx::mbar_arrive(&hb[16 + (g & 1)]);
            }
            return;
        }
        // ---- warp 0: the state chains, 16 steps per group, indices and words from shared memory, symbols
        //      into the ring
        uint32_t rprev = 2;  // R_{g-1}: the window of group g starts there
        for (uint32_t g = 0; g < ngr; ++g) {
            const int b = (int)(g & 3);
            const uint32_t use = g >> 2;
            bool ok = hwait(&hb[b], use & 1);
            if (use > 0 && ok) ok = hwait(&hb[12 + b], (use - 1) & 1);
            if (ok) ok = hwait(&hb[16 + (g & 1)], (g >> 1) & 1);
            if (!__all_sync(0xffffffffu, ok)) return;
            // this group's window; publish R_g for the next one
            const uint64_t A = words_at / 2 + lstart[l] + rprev;  // (words_at is a multiple of 4)
            woff = (int)(A & 1) - (int)rprev;
            win_cur = reinterpret_cast<const uint16_t*>(win32 + ((g & 1) * 32 + l) * 17);
            rpos[(g & 1) * 32 + l] = r;
            __syncwarp();
            if (l == 0) ptx::mbar_arrive(&hb[18 + (g & 1)]);
            rprev = r;
            const uint8_t* tr = ring_t + b * 512 + l;
            int16_t* sr = ring_s + b * 512 + l;
            uint32_t tv[kPF];
#pragma unroll
            for (int u = 0; u < kPF; ++u) tv[u] = tr[u * 32];
#pragma unroll
            for (int u = 0; u < kPF; ++u)
                sr[u * 32] = (int16_t)((int)decode(tv[u], true, every, every) - kRmax);
            __syncwarp();
            if (l == 0) {
                ptx::mbar_arrive(&hb[4 + b]);  // indices consumed
                ptx::mbar_arrive(&hb[8 + b]);  // symbols ready
            }
        }
        m0 = kPF * ngr;
        fi = (uint32_t)lane + m0 * (uint32_t)K;
        i = fi;
        // the generic path reads the lane's words from its global row: w0 = word r (already held), w1 = r + 1
        if (ngr > 0) w1 = (unsigned short)ld_u16(wp + (r + 1 < nw ? r + 1 : nw - 1));
    }
    // Fast path, for a warp of 32 lanes in range with good counts and 16-byte aligned rows: the symbols of
    // a group go to a shared-memory tile [16 steps][32 lanes] (one store each, off the state chain), then
    // the warp writes the group's 16 rows of 32 consecutive elements as 16-byte vectors, y^ = r^ q + mu
    // computed there from mu read a group ahead.  Lane l writes elements 16 (l & 1) .. + 15 of row l / 2.
    const uint32_t j0 = (uint32_t)(lane & ~31);
    const bool fast = !HELP && !PER && (K & 15) == 0 && (outp & 15) == 0 &&
                      (OUT == kDecSym || (reinterpret_cast<uintptr_t>(S.mu) & 15) == 0) &&
                      __all_sync(0xffffffffu, okc && cmin >= (uint32_t)kPF);
    if (fast) {
        int16_t* tile = reinterpret_cast<int16_t*>(dsm + kDecTileOff) + (threadIdx.x >> 5) * (kPF * 32);
        const int lr = (int)(threadIdx.x & 31) >> 1, lh = (int)(threadIdx.x & 1);
        float mv[16];
        auto load_mu = [&](uint32_t g0) {  // mu of the lane's 16 flush elements of group g0 (if it is whole)
            if (OUT == kDecSym) return;
            const bool ok = g0 + kPF <= cmin;
            const float4* p = reinterpret_cast<const float4*>(S.mu + j0 + 16u * lh + (size_t)(g0 + lr) * K);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (ok) v = __ldg(p + k);
                mv[4 * k] = v.x; mv[4 * k + 1] = v.y; mv[4 * k + 2] = v.z; mv[4 * k + 3] = v.w;
            }
        };
        auto flush = [&](uint32_t g0) {
            __syncwarp();
            const uint4* src = reinterpret_cast<const uint4*>(tile + lr * 32 + 16 * lh);
            const uint4 a = src[0], b = src[1];
            const size_t e0 = j0 + 16u * lh + (size_t)(g0 + lr) * K;
            const uint32_t wv[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
            if (OUT == kDecSym) {
                uint4* dst = reinterpret_cast<uint4*>(S.sym + e0);
                dst[0] = a;
                dst[1] = b;
            } else {
                float y[16];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    y[2 * k] = yval((int)(int16_t)(wv[k] & 0xFFFFu), mv[2 * k]);
                    y[2 * k + 1] = yval((int)(int16_t)(wv[k] >> 16), mv[2 * k + 1]);
                }
                if (OUT == kDecBf16) {
                    uint32_t pk[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const __nv_bfloat162 hv = __floats2bfloat162_rn(y[2 * k], y[2 * k + 1]);
                        pk[k] = *reinterpret_cast<const uint32_t*>(&hv);
                    }
                    uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(S.yout) + e0);
                    dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                } else if (OUT == kDecF32) {
                    float4* dst = reinterpret_cast<float4*>(reinterpret_cast<float*>(S.yout) + e0);
#pragma unroll
                    for (int k = 0; k < 4; ++k) dst[k] = make_float4(y[4 * k], y[4 * k + 1], y[4 * k + 2], y[4 * k + 3]);
                } else {
                    uint32_t pk[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        uint32_t w = 0;
#pragma unroll
                        for (int b2 = 0; b2 < 4; ++b2)
                            w |= (uint32_t)__nv_cvt_float_to_fp8(y[4 * k + b2] * J.inv8, __NV_SATFINITE, __NV_E4M3)
                                 << (8 * b2);
                        pk[k] = w;
                    }
                    *reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(S.yout) + e0) =
                        make_uint4(pk[0], pk[1], pk[2], pk[3]);
                }
            }
            __syncwarp();
        };
        tile_mode = true;
        fetch(0, tc, mc);
        load_mu(0);
        for (; m0 + kPF <= cmin; m0 += kPF) {
            ahead();
            fetch(m0 + kPF, tn, mn);
#pragma unroll
            for (int u = 0; u < kPF; ++u)
                tile[u * 32 + (threadIdx.x & 31)] = (int16_t)((int)decode(tc[u], true, every, some) - kRmax);
            flush(m0);
            load_mu(m0 + kPF);
#pragma unroll
            for (int u = 0; u < kPF; ++u) tc[u] = tn[u];
        }
        // the generic path takes the rest from m0: its fetch position and first output element
        tile_mode = false;
        fi = (uint32_t)lane + m0 * (uint32_t)K;
        i = fi;
        if (PER) ip = (int)(((uint64_t)lane + (uint64_t)m0 * K) % (uint64_t)per);
    }
    fetch(m0, tc, mc);
    for (; m0 + kPF <= cmin; m0 += kPF) {  // whole groups that every live lane of the warp codes
        ahead();
        fetch(m0 + kPF, tn, mn);
#pragma unroll
        for (int u = 0; u < kPF; ++u) {
            const bool act = okc;
            const uint32_t sy = decode(tc[u], act, some, some);
            if (act) put(sy, mc[u]);
        }
#pragma unroll
        for (int u = 0; u < kPF; ++u) { tc[u] = tn[u]; mc[u] = mn[u]; }
    }
    for (; m0 < cmax; m0 += kPF) {  // the rest: at most a group and a bit, lanes predicated
        ahead();
        fetch(m0 + kPF, tn, mn);
#pragma unroll
        for (int u = 0; u < kPF; ++u)
            if (m0 + u < cmax) {
                const bool act = m0 + u < mine;
                const uint32_t sy = decode(tc[u], act, some, some);
                if (act) put(sy, mc[u]);
            }
#pragma unroll
        for (int u = 0; u < kPF; ++u) { tc[u] = tn[u]; mc[u] = mn[u]; }
    }
    bad = bad >= (uint32_t)kBins;
    if (bad) set_status(J.status, UFVC_ERR_ARG);
    if (okc && (x != kRansL || r != words)) set_status(J.status, UFVC_ERR_CORRUPT);
}

// Threads per block for a section of K lanes: the lanes spread over one wave of one block per SM
// (the tables take 192 KB of shared memory), whole warps, at most 512 (K <= 65536 needs 448).
static int dec_threads(int K, int sms) {
    int T = 32 * ((K + 32 * sms - 1) / (32 * sms));
    return T < 32 ? 32 : T > 512 ? 512 : T;
}

template <int OUT, bool PER>
static cudaError_t launch_dec_t(const RansDecJob& j, const uint8_t* tables, cudaStream_t s) {
    if (!PER && j.threads == 32) {  // one warp of lanes per block: three serving warps beside it
        cudaError_t e = smem_optin((const void*)rans_decode_kernel<OUT, PER, true>, kDecSmemBytes);
        if (e != cudaSuccess) return e;
        return launch_pdl(rans_decode_kernel<OUT, PER, true>, dim3(j.bps * j.nsec), dim3(128), (size_t)kDecSmemBytes,
                          s, j, tables);
    }
    cudaError_t e = smem_optin((const void*)rans_decode_kernel<OUT, PER>, kDecSmemBytes);
    if (e != cudaSuccess) return e;
    return launch_pdl(rans_decode_kernel<OUT, PER>, dim3(j.bps * j.nsec), dim3(j.threads), (size_t)kDecSmemBytes, s,
                      j, tables);
}

cudaError_t launch_rans_decode(RansDecJob& j, const uint8_t* dec_tables, cudaStream_t s) {
    if (j.K < 1 || j.K > 65536 || j.nsec < 1 || j.nsec > kRansMaxDecSec) return cudaErrorInvalidValue;
    // the lanes of all sections spread over one wave of one block per SM
    j.threads = dec_threads(j.K * j.nsec, sm_count());
    // per-channel tables (the z^ section: a few steps per lane) in blocks of up to 512 lanes: each block's
    // fixed costs (the tables' copy, the header, the scan of the lane counts) then count a few times
    // instead of once per warp of lanes
    if (j.idx_period) j.threads = 512;
    if (j.threads > j.K) j.threads = (j.K + 31) / 32 * 32;
    j.bps = (j.K + j.threads - 1) / j.threads;
    if (j.idx_period) {
        if (j.out != kDecSym) return cudaErrorInvalidValue;
        return launch_dec_t<kDecSym, true>(j, dec_tables, s);
    }
    switch (j.out) {
        case kDecSym: return launch_dec_t<kDecSym, false>(j, dec_tables, s);
        case kDecBf16: return launch_dec_t<kDecBf16, false>(j, dec_tables, s);
        case kDecF32: return launch_dec_t<kDecF32, false>(j, dec_tables, s);
        case kDecE4M3: return launch_dec_t<kDecE4M3, false>(j, dec_tables, s);
        default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------------------------------------
// host: decoding tables from the integer CDF tables
// ------------------------------------------------------------------------------------------------
void build_decode_tables(const std::vector<uint32_t>& cum_all, std::vector<uint8_t>& out) {
    out.assign(kDecTabBytes, 0);
    uint64_t* ent = reinterpret_cast<uint64_t*>(out.data());
    uint32_t* runs = reinterpret_cast<uint32_t*>(out.data() + kDecEntBytes);
    uint16_t* c16 = reinterpret_cast<uint16_t*>(out.data() + kDecEntBytes + kDecRunBytes);
    for (int k = 0; k < kBins; ++k) {
        const uint32_t* c = &cum_all[(size_t)k * (kNsym + 1)];  // c[0] = 0 .. c[511] = 65536
        auto freq = [&](int s) { return c[s + 1] - c[s]; };
        uint32_t A = 0, B = 0;
        while (A < (uint32_t)kNsym && freq((int)A) == 1) ++A;
        while (B < (uint32_t)kNsym && freq(kNsym - 1 - (int)B) == 1) ++B;
        runs[k] = A | (B << 16);
        for (int s = 0; s < kNsym; ++s) c16[k * 512 + s] = (uint16_t)c[s];
        // owner of a slot: the s with c[s] <= slot < c[s + 1]
        auto owner = [&](uint32_t slot) {
            int lo = 0, hi = kNsym - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (c[mid] <= slot) lo = mid; else hi = mid - 1;
            }
            return lo;
        };
        for (int b = 0; b < 256; ++b) {
            // the bucket's slots outside the end runs
            const uint32_t lo = std::max<uint32_t>((uint32_t)b << 8, A);
            const uint32_t hi = std::min<uint32_t>((uint32_t)(b + 1) << 8, kProbM - B);
            uint64_t e = 0;
            if (lo < hi) {
                const int s0 = owner(lo), sl = owner(hi - 1);
                const uint32_t f0 = freq(s0), f1 = s0 + 1 < kNsym ? freq(s0 + 1) : 0u;
                const uint32_t d = (uint32_t)std::min(127, sl - s0);
                const uint32_t lw = (uint32_t)s0 | (f0 << 9) | (d << 25);
                const uint32_t hw = c[s0] | (f1 << 16);
                e = (uint64_t)lw | ((uint64_t)hw << 32);
            }
            ent[k * 256 + b] = e;
        }
    }
}

}  // namespace ufvc
