// Allocation-free variant of the rANS section encoder (ufvc_rans_encode_noalloc).
//
// ufvc_rans_encode needs scratch memory beyond its inputs and outputs: every lane writes its words into a
// row of a staging buffer before they are laid out, and the blocks publish their word totals in a small
// control block.  That entry point allocates them with cudaMalloc the first time a size is seen.  Some
// callers cannot let a library allocate: real-time loops where cudaMalloc's implicit device
// synchronisation would stall other work, and hosts whose device memory is wholly owned by their own pool
// allocator.  For them this file keeps the scratch in one file-scope __device__ array of fixed size, which
// every GPU that loads the library holds until the process exits, and the entry point below performs no
// allocation of any kind.
#include "ufvc_internal.h"

#include <mutex>

namespace {

constexpr size_t kScratchBytes = 24ull << 20;  // 24 MiB per device
constexpr int kMaxDevices = 64;

// Layout of one call: the layout control block (tickets and published block totals, cleared before every
// launch), then the lane rows (u16 x lanes x (n / lanes + 3)), each part 256-byte aligned.
static __device__ __align__(256) unsigned char g_rans_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

extern "C" ufvc_status ufvc_rans_encode_noalloc(ufvc_ctx* ctx, const int16_t* d_sym, const uint8_t* d_idx, size_t n,
                                                int lanes, uint8_t* d_out, size_t capacity, uint64_t* d_nbytes,
                                                void* stream) {
    if (!ctx) return UFVC_ERR_ARG;
    if ((!d_sym && n) || (!d_idx && n) || !d_out || !d_nbytes || lanes < 1 || lanes > 65536) {
        ufvc::ctx_set_error(ctx, "rans_encode_noalloc: bad argument");
        return UFVC_ERR_ARG;
    }
    // n above half the array can never fit (two bytes per symbol); refusing it first also keeps the
    // size arithmetic below from wrapping and the per-lane row length within an int
    if (n > kScratchBytes / 2) {
        ufvc::ctx_set_error(ctx, "rans_encode_noalloc: n exceeds the 24 MiB static scratch (at most about 12.5 "
                                 "million symbols); use ufvc_rans_encode");
        return UFVC_ERR_ARG;
    }
    const size_t cap_lane = n / (size_t)lanes + 3;
    const size_t ctl_bytes = align256(ufvc::rans_ctl_bytes());
    const size_t need = ctl_bytes + (size_t)lanes * cap_lane * 2;
    if (need > kScratchBytes) {
        ufvc::ctx_set_error(ctx, "rans_encode_noalloc: n + 3 * lanes exceeds the 24 MiB static scratch "
                                 "(at most about 12.5 million symbols); use ufvc_rans_encode");
        return UFVC_ERR_ARG;
    }
    const int dev = ufvc::ctx_device(ctx);
    if (dev < 0 || dev >= kMaxDevices) {
        ufvc::ctx_set_error(ctx, "rans_encode_noalloc: device ordinal out of range");
        return UFVC_ERR_ARG;
    }
    cudaError_t e = cudaSetDevice(dev);
    if (e != cudaSuccess) {
        ufvc::ctx_set_error(ctx, cudaGetErrorString(e));
        return UFVC_ERR_CUDA;
    }
    void* base = nullptr;
    {
        // once per device, with that device current: the array's device address (the host-side symbol
        // is only a stand-in and must never be handed to a kernel)
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_rans_scratch);
            if (e != cudaSuccess || !p) {
                ufvc::ctx_set_error(ctx, e != cudaSuccess ? cudaGetErrorString(e) : "cudaGetSymbolAddress: null");
                return UFVC_ERR_CUDA;
            }
            g_scratch_addr[dev] = p;
        }
        base = g_scratch_addr[dev];
    }
    // The control block must start at zero: it is cleared on the stream before the launch (a memset, no
    // allocation).  The rows hold nothing the call reads before writing it.
    unsigned char* b = static_cast<unsigned char*>(base);
    ufvc::RansCtl* ctl = reinterpret_cast<ufvc::RansCtl*>(b);
    uint16_t* rows = reinterpret_cast<uint16_t*>(b + ctl_bytes);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = cudaMemsetAsync(ctl, 0, ufvc::rans_ctl_bytes(), s);
    if (e != cudaSuccess) {
        ufvc::ctx_set_error(ctx, cudaGetErrorString(e));
        return UFVC_ERR_CUDA;
    }
    ufvc::RansEncJob j{};
    j.s[0] = ufvc::RansEncSec{d_sym, d_idx, 0, (uint32_t)n, lanes, rows, (int)cap_lane, 0};
    j.nsec = 1;
    j.st[0].out = d_out;
    j.st[0].capacity = capacity;
    j.st[0].nbytes = d_nbytes;
    j.nstreams = 1;
    j.ctl = ctl;
    j.status = ufvc::ctx_status_word(ctx);
    j.spin = ufvc::ctx_table_spin(ctx);
    e = ufvc::launch_rans_encode(j, ufvc::ctx_packed_tables(ctx), s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        ufvc::ctx_set_error(ctx, cudaGetErrorString(e));
        return UFVC_ERR_CUDA;
    }
    return UFVC_OK;
}
