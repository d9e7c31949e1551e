// Host-side FP64 construction of the entropy-coding tables and the architecture table.
//
// Scale bins (64, log-spaced on [0.11, 64]), the per-qp FP32 index thresholds and the 16-bit integer
// Gaussian CDF tables are built once per context in double precision, so no GPU step needs FP64.
// The paper's streamlined entropy model (Sec. 3.4) codes each element with its scale only; these
// tables turn a scale index into integer frequencies for the rANS coder.
#include "ufvc_internal.h"

#include <algorithm>
#include <cmath>

namespace ufvc {

static double bin_scale(int k) {
    const double lo = std::log(0.11), hi = std::log(64.0);
    return std::exp(lo + (hi - lo) * k / 63.0);
}

double qstep_fp64(int qp) { return std::exp2((qp - 32) / 8.0); }

void build_host_tables(HostTables& t) {
    t.freq.assign(kBins * kNsym, 0);
    t.cum.assign(kBins * (kNsym + 1), 0);
    t.packed.assign(kBins * kNsym, 0);
    t.thr.assign(64 * (kBins - 1), 0.f);
    t.qstep.assign(64, 0.f);
    t.qinv.assign(64, 0.f);
    t.log_thr.assign(kBins - 1, 0.0);

    // log-domain decision thresholds between neighbouring bins (geometric midpoints)
    for (int k = 1; k < kBins; ++k) t.log_thr[k - 1] = 0.5 * (std::log(bin_scale(k - 1)) + std::log(bin_scale(k)));
    for (int qp = 0; qp < 64; ++qp) {
        const double q = qstep_fp64(qp);
        t.qstep[qp] = (float)q;
        t.qinv[qp] = (float)(1.0 / q);
        const double lq = std::log(q);
        for (int k = 1; k < kBins; ++k) t.thr[qp * (kBins - 1) + k - 1] = (float)(t.log_thr[k - 1] + lq);
    }

    // Each table: mass of N(0, s^2) on [r - 1/2, r + 1/2), the mass beyond +-254.5 folded into +-255;
    // frequency = 1 + floor(mass * (2^16 - 511)); the mode (r = 0) absorbs the rounding deficit.
    const double budget = double(kProbM - kNsym);
    for (int k = 0; k < kBins; ++k) {
        const double inv = 1.0 / (bin_scale(k) * std::sqrt(2.0));
        uint32_t* f = &t.freq[k * kNsym];
        for (int r = 0; r <= kRmax; ++r) {
            double mass;
            if (r == 0)
                mass = std::erf(0.5 * inv);
            else if (r < kRmax)
                mass = 0.5 * (std::erfc((r - 0.5) * inv) - std::erfc((r + 0.5) * inv));
            else
                mass = 0.5 * std::erfc((kRmax - 0.5) * inv);
            const uint32_t v = 1u + (uint32_t)std::floor(mass * budget);
            f[kRmax + r] = v;
            f[kRmax - r] = v;
        }
        uint32_t total = 0;
        for (int i = 0; i < kNsym; ++i) total += f[i];
        f[kRmax] += kProbM - total;
        uint32_t* c = &t.cum[k * (kNsym + 1)];
        c[0] = 0;
        for (int i = 0; i < kNsym; ++i) c[i + 1] = c[i] + f[i];
        for (int i = 0; i < kNsym; ++i) t.packed[k * kNsym + i] = (f[i] << 16) | c[i];
    }
    build_decode_tables(t.cum, t.dec);
}

// ---------------------------------------------------------------------------------------------
// Architecture: analysis widths e0..e2, latent Cy, hyper-latent Cz, decoder widths Cd1, Cd2.
// ---------------------------------------------------------------------------------------------
bool get_arch(int arch, Arch* a) {
    if (arch == 0) { *a = Arch{64, 96, 128, 128, 64, 128, 64}; return true; }
    if (arch == 1) { *a = Arch{64, 128, 192, 256, 128, 128, 64}; return true; }
    if (arch == 2) { *a = Arch{0, 0, 0, kDcCy, kDcCz, 0, 0}; return true; }  // DC-block model
    return false;
}

// DC-block model (arch 2): blob layer l -> (cout, k, cin); depth-wise layers have cin = 1.  Shared layers:
// PE, EC, 6 encoder blocks, ED, H1, H2, S1, S2, S3, PC, DU, FC, 7 decoder blocks, 11 context blocks, GO;
// then per frame FP, 3 blocks at the frame width, FO.  A block is PWa, DW, PWb, PWc, PWd.
static void dc_block_shape(int c, int j, int* co, int* k, int* ci) {
    const int t[5][3] = {{c, 1, c}, {c, 3, 1}, {c, 1, c}, {2 * c, 1, c}, {c, 1, 2 * c}};
    *co = t[j][0]; *k = t[j][1]; *ci = t[j][2];
}

bool dc_layer_shape(int N, int l, int* cout, int* k, int* cin) {
    if (N < 1 || l < 0 || l >= kDcShared + kDcPerFrame * N) return false;
    if (l >= kDcShared) {
        const int j = (l - kDcShared) % kDcPerFrame;
        if (j == 0) { *cout = kDcCf; *k = 1; *cin = kDcC; }
        else if (j == kDcPerFrame - 1) { *cout = 192; *k = 1; *cin = kDcCf; }
        else dc_block_shape(kDcCf, (j - 1) % 5, cout, k, cin);
        return true;
    }
    if (l == DC_PE) { *cout = kDcC; *k = 1; *cin = 3 * N * 64; }
    else if (l == DC_EC || l == DC_FC) { *cout = kDcC; *k = 1; *cin = kDcCc; }
    else if (l < DC_ED) dc_block_shape(kDcC, (l - DC_E0) % 5, cout, k, cin);
    else if (l == DC_ED) { *cout = kDcCy; *k = 3; *cin = kDcC; }
    else if (l == DC_H1) { *cout = kDcCz; *k = 3; *cin = kDcCy; }
    else if (l == DC_H2) { *cout = kDcCz; *k = 3; *cin = kDcCz; }
    else if (l == DC_S1 || l == DC_S2) { *cout = 4 * kDcCz; *k = 3; *cin = kDcCz; }
    else if (l == DC_S3) { *cout = 2 * kDcCy; *k = 1; *cin = kDcCz; }
    else if (l == DC_PC) { *cout = kDcCz; *k = 3; *cin = kDcCc; }
    else if (l == DC_DU) { *cout = 4 * kDcC; *k = 1; *cin = kDcCy; }
    else if (l < DC_GO) dc_block_shape(kDcC, (l - DC_D0) % 5, cout, k, cin);
    else { *cout = kDcCc; *k = 1; *cin = kDcC; }
    return true;
}

bool layer_shape(int arch, int N, int l, int* cout, int* k, int* cin) {
    if (arch == 2) return dc_layer_shape(N, l, cout, k, cin);
    Arch a;
    if (!get_arch(arch, &a) || N < 1 || l < 0 || l >= L_NENC + D_NDEC * N) return false;
    if (l < L_NENC) {
        const int t[L_NENC][3] = {{a.e0, 3, 3 * N},     {a.e1, 3, a.e0},      {a.e2, 3, a.e1},
                                  {a.e2, 3, a.e2},      {a.e2, 1, a.e2},      {a.cy, 3, a.e2},
                                  {a.cz, 3, a.cy},      {a.cz, 3, a.cz},      {4 * a.cz, 3, a.cz},
                                  {4 * a.cz, 3, a.cz},  {2 * a.cy, 1, a.cz}};
        *cout = t[l][0]; *k = t[l][1]; *cin = t[l][2];
    } else {
        const int d[D_NDEC][3] = {{4 * a.cd1, 3, a.cy}, {a.cd1, 3, a.cd1},    {a.cd1, 3, a.cd1},
                                  {4 * a.cd2, 3, a.cd1}, {a.cd2, 3, a.cd2},   {a.cd2, 3, a.cd2},
                                  {4 * a.cd2, 3, a.cd2}, {12, 3, a.cd2}};
        const int j = (l - L_NENC) % D_NDEC;
        *cout = d[j][0]; *k = d[j][1]; *cin = d[j][2];
    }
    return true;
}

size_t weight_count(int arch, int N) {
    size_t n = 0;
    int co, k, ci;
    if (arch == 2) {
        for (int l = 0; l < kDcShared + kDcPerFrame * N; ++l) {
            if (!dc_layer_shape(N, l, &co, &k, &ci)) return 0;
            n += (size_t)co * k * k * ci + co;
        }
        return n;
    }
    for (int l = 0; l < L_NENC + D_NDEC * N; ++l) {
        if (!layer_shape(arch, N, l, &co, &k, &ci)) return 0;
        n += (size_t)co * k * k * ci + co;
    }
    return n;
}

// Progressive-mean layers of step k = 1..3: P_k,a (3x3, Cy + Cz -> Cz, GELU) then P_k,b (1x1, Cz -> Cy).
bool mean_layer_shape(int arch, int l, int* cout, int* k, int* cin) {
    Arch a;
    if (!get_arch(arch, &a) || l < 0 || l >= kMeanLayers) return false;
    if (l % 2 == 0) { *cout = a.cz; *k = 3; *cin = a.cy + a.cz; }
    else            { *cout = a.cy; *k = 1; *cin = a.cz; }
    return true;
}

// Temporal chunk context (Cf = Cc = 64): EC (1x1, Cc -> e2), FD (3x3, Cy -> 4 Cf), FC (1x1, Cc -> Cf),
// CG (3x3, Cf -> Cc), PC (3x3 stride 2, Cc -> Cz), then DF_f (1x1, Cf -> Cd1) for each frame position f.
bool temporal_layer_shape(int arch, int N, int l, int* cout, int* k, int* cin) {
    Arch a;
    if (!get_arch(arch, &a) || N < 1 || l < 0 || l >= TL_N + N) return false;
    const int t[TL_N][3] = {{a.e2, 1, kCc}, {4 * kCf, 3, a.cy}, {kCf, 1, kCc}, {kCc, 3, kCf}, {a.cz, 3, kCc}};
    if (l < TL_N) { *cout = t[l][0]; *k = t[l][1]; *cin = t[l][2]; }
    else { *cout = a.cd1; *k = 1; *cin = kCf; }
    return true;
}

size_t temporal_weight_count(int arch, int N) {
    size_t n = 0;
    int co, k, ci;
    for (int l = 0; l < TL_N + N; ++l) {
        if (!temporal_layer_shape(arch, N, l, &co, &k, &ci)) return 0;
        n += (size_t)co * k * k * ci + co;
    }
    return n;
}

size_t mean_weight_count(int arch) {
    size_t n = 0;
    int co, k, ci;
    for (int l = 0; l < kMeanLayers; ++l) {
        if (!mean_layer_shape(arch, l, &co, &k, &ci)) return 0;
        n += (size_t)co * k * k * ci + co;
    }
    return n;
}

}  // namespace ufvc
