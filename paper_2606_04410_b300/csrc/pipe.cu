// Pipelined host-buffer round trips (ufvc_pipe_*): chunks streamed through host memory.
//
// A pipeline owns `depth` slots.  A slot is a context that shares the caller's weights and tables
// (ctx_clone_shared: own plans, workspaces and status word), a non-blocking CUDA stream, device buffers
// for one chunk (frames in, bit-stream, the bit-stream as read back from the host, frames out), a pinned
// word for the stream size and a completion event.  ufvc_pipe_submit enqueues one round trip on the slot
// of its ticket (ticket % depth) and returns without waiting:
//   H2D frames -> ufvc_encode_chunk -> D2H bit-stream buffer (whole capacity) and size
//   -> H2D of that host copy -> ufvc_decode_chunk_dev (size read on the device) -> D2H frames.
// Each step's copies therefore cross the host link like the synchronous host-buffer calls, but the
// copies of one slot overlap the kernels of the others.  ufvc_pipe_wait synchronises the ticket's event
// and returns its stream size and the slot's device status.
#include "ufvc_internal.h"

#include <vector>

using namespace ufvc;

struct PipeSlot {
    ufvc_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    uint8_t *d_frames = nullptr, *d_bits = nullptr, *d_bits2 = nullptr, *d_out = nullptr;
    uint64_t* d_nbytes = nullptr;
    uint64_t* h_nbytes = nullptr;  // pinned
    size_t in_cap = 0, out_cap = 0, bits_cap = 0, bits2_cap = 0;
    long long ticket = -1;  // last ticket submitted here
    bool waited = true;     // that ticket has been waited for
};

struct ufvc_pipe {
    ufvc_ctx* base = nullptr;
    std::vector<PipeSlot> slots;
    long long next = 0;
};

static void free_slot(PipeSlot& s) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    cudaFree(s.d_frames); cudaFree(s.d_bits); cudaFree(s.d_bits2); cudaFree(s.d_out); cudaFree(s.d_nbytes);
    cudaFreeHost(s.h_nbytes);
    if (s.done) cudaEventDestroy(s.done);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.ctx) ufvc_destroy(s.ctx);
    s = PipeSlot();
}

extern "C" ufvc_status ufvc_pipe_create(ufvc_ctx* ctx, int depth, ufvc_pipe** out) {
    if (!ctx || !out || depth < 1 || depth > 16) return UFVC_ERR_ARG;
    if (cudaSetDevice(ctx_device(ctx)) != cudaSuccess) return UFVC_ERR_CUDA;
    ufvc_pipe* p = new ufvc_pipe();
    p->base = ctx;
    p->slots.resize(depth);
    for (PipeSlot& s : p->slots) {
        s.ctx = ctx_clone_shared(ctx);
        if (!s.ctx || cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMalloc(&s.d_nbytes, 8) != cudaSuccess || cudaMallocHost(&s.h_nbytes, 8) != cudaSuccess) {
            cudaGetLastError();
            for (PipeSlot& t : p->slots) free_slot(t);
            delete p;
            return UFVC_ERR_OOM;
        }
        *s.h_nbytes = 0;
    }
    *out = p;
    return UFVC_OK;
}

extern "C" void ufvc_pipe_destroy(ufvc_pipe* p) {
    if (!p) return;
    cudaSetDevice(ctx_device(p->base));
    for (PipeSlot& s : p->slots) free_slot(s);
    delete p;
}

static ufvc_status grow(uint8_t** buf, size_t* cap, size_t need) {
    if (need <= *cap) return UFVC_OK;
    cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    if (cudaMalloc(buf, need) != cudaSuccess) {
        cudaGetLastError();
        return UFVC_ERR_OOM;
    }
    *cap = need;
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_pipe_submit(ufvc_pipe* p, const uint8_t* h_frames, int n_frames, int width, int height,
                                        int qp, uint8_t* h_bits, size_t capacity, uint8_t* h_out, long long* ticket) {
    if (!p || !h_frames || !h_bits || !ticket) return UFVC_ERR_ARG;
    const long long t = p->next;
    PipeSlot& s = p->slots[t % (long long)p->slots.size()];
    if (!s.waited) return UFVC_ERR_ARG;  // wait for ticket t - depth first
    if (cudaSetDevice(ctx_device(p->base)) != cudaSuccess) return UFVC_ERR_CUDA;
    const size_t bmax = ufvc_max_bitstream_bytes(s.ctx, width, height);
    if (bmax == 0) return UFVC_ERR_ARG;
    if (capacity < bmax) return UFVC_ERR_CAPACITY;
    const size_t fsz = (size_t)n_frames * frame_bytes(ctx_color(s.ctx), width, height);
    ufvc_status st;
    if ((st = grow(&s.d_frames, &s.in_cap, fsz)) || (st = grow(&s.d_out, &s.out_cap, fsz)) ||
        (st = grow(&s.d_bits, &s.bits_cap, bmax)) || (st = grow(&s.d_bits2, &s.bits2_cap, bmax)))
        return st;
    cudaStream_t q = s.stream;
    if (cudaMemcpyAsync(s.d_frames, h_frames, fsz, cudaMemcpyHostToDevice, q) != cudaSuccess) return UFVC_ERR_CUDA;
    if ((st = ufvc_encode_chunk(s.ctx, s.d_frames, n_frames, width, height, qp, s.d_bits, bmax, s.d_nbytes, q)))
        return st;
    if (cudaMemcpyAsync(s.h_nbytes, s.d_nbytes, 8, cudaMemcpyDeviceToHost, q) != cudaSuccess ||
        cudaMemcpyAsync(h_bits, s.d_bits, bmax, cudaMemcpyDeviceToHost, q) != cudaSuccess)
        return UFVC_ERR_CUDA;
    if (h_out) {
        // the decoder side reads the bit-stream from the host copy, as a separate receiver would
        if (cudaMemcpyAsync(s.d_bits2, h_bits, bmax, cudaMemcpyHostToDevice, q) != cudaSuccess) return UFVC_ERR_CUDA;
        if ((st = ufvc_decode_chunk_dev(s.ctx, s.d_bits2, bmax, s.d_nbytes, s.d_out, n_frames, width, height, q)))
            return st;
        if (cudaMemcpyAsync(h_out, s.d_out, fsz, cudaMemcpyDeviceToHost, q) != cudaSuccess) return UFVC_ERR_CUDA;
    }
    if (cudaEventRecord(s.done, q) != cudaSuccess) return UFVC_ERR_CUDA;
    s.ticket = t;
    s.waited = false;
    p->next = t + 1;
    *ticket = t;
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_pipe_wait(ufvc_pipe* p, long long ticket, size_t* nbytes) {
    if (!p || ticket < 0) return UFVC_ERR_ARG;
    PipeSlot& s = p->slots[ticket % (long long)p->slots.size()];
    if (s.ticket != ticket || s.waited) return UFVC_ERR_ARG;
    if (cudaSetDevice(ctx_device(p->base)) != cudaSuccess) return UFVC_ERR_CUDA;
    if (cudaEventSynchronize(s.done) != cudaSuccess) return UFVC_ERR_CUDA;
    s.waited = true;
    if (nbytes) *nbytes = (size_t)*s.h_nbytes;
    return ufvc_sync_status(s.ctx, s.stream);
}
