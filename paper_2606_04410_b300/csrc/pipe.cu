// Pipelined host-buffer round trips (ufvc_pipe_*): chunks streamed through host memory.
//
// A pipeline owns one context that shares the caller's weights and tables (ctx_clone_shared: own plans,
// workspaces and status word), one compute stream, four copy streams (frames in, bit-stream out,
// bit-stream back in, frames out) and `depth` slots of device buffers for one chunk each (frames in,
// bit-stream, the bit-stream as read back from the host, frames out) with pinned words for the stream
// size and the status.  Ticket t uses slot t % depth:
//   frames in (copy stream)  ->  encode (compute)  ->  bit-stream buffer and size out, then that host copy
//   back in (copy streams)  ->  ufvc_decode_chunk_dev (compute, size read on the device)  ->  frames out.
// All kernels run on the one compute stream, one chunk's kernels at a time, as on a single context: the
// decode of ticket t is enqueued after the encode of ticket t + lag (by that submit, or by the wait of
// ticket t), so the compute stream never stands still while a bit-stream crosses the host link, and the
// copies of the other tickets overlap it.  lag = 2 with five slots or more (the bit-stream's copies out
// and back in queue on the copy engines behind 50 MB frame copies, and one encode of slack was not always
// enough: 1.76 against 1.86 ms per 1080p step), else 1 (with fewer slots the host, which reuses a slot
// only after its ticket's frames are back, would wait on decodes held back: four slots 1.93 ms, three
// 3.37 ms with lag 2).  Each encode and each decode moves the status word into the
// slot's mapped pinned status word and clears it, by a one-thread kernel (a copy there would queue on the
// copy engine behind the frame copies and stall the compute stream), so every ticket reports its own
// device status.
#include "ufvc_internal.h"

#include <deque>
#include <vector>

using namespace ufvc;

struct PipeSlot {
    uint8_t *d_frames = nullptr, *d_bits = nullptr, *d_bits2 = nullptr, *d_out = nullptr;
    uint64_t* d_nbytes = nullptr;
    uint64_t* h_nbytes = nullptr;  // pinned
    int* h_status = nullptr;       // pinned and mapped: [0] the encode's status, [1] the decode's
    int* hd_status = nullptr;      // its device address
    cudaEvent_t in = nullptr, enc = nullptr, bits_out = nullptr, bits_in = nullptr, dec = nullptr, done = nullptr;
    size_t in_cap = 0, out_cap = 0, bits_cap = 0, bits2_cap = 0;
    // the ticket last submitted here, and what its decode needs (enqueued later)
    long long ticket = -1;
    bool waited = true;
    uint8_t* h_out = nullptr;
    size_t bmax = 0, fsz = 0;
    int n_frames = 0, width = 0, height = 0;
};

struct ufvc_pipe {
    ufvc_ctx* base = nullptr;
    ufvc_ctx* ctx = nullptr;
    cudaStream_t cs = nullptr, in_frames = nullptr, out_bits = nullptr, in_bits = nullptr, out_frames = nullptr;
    std::vector<PipeSlot> slots;
    long long next = 0;
    std::deque<long long> pending;  // tickets whose decodes are not enqueued yet, oldest first
    size_t lag = 1;                 // encodes between a ticket's encode and its decode on the compute stream
};

static void free_slot(PipeSlot& s) {
    cudaFree(s.d_frames); cudaFree(s.d_bits); cudaFree(s.d_bits2); cudaFree(s.d_out); cudaFree(s.d_nbytes);
    cudaFreeHost(s.h_nbytes);
    cudaFreeHost(s.h_status);
    for (cudaEvent_t e : {s.in, s.enc, s.bits_out, s.bits_in, s.dec, s.done})
        if (e) cudaEventDestroy(e);
    s = PipeSlot();
}

static void free_pipe(ufvc_pipe* p) {
    for (cudaStream_t q : {p->cs, p->in_frames, p->out_bits, p->in_bits, p->out_frames})
        if (q) cudaStreamSynchronize(q);
    for (PipeSlot& s : p->slots) free_slot(s);
    for (cudaStream_t q : {p->cs, p->in_frames, p->out_bits, p->in_bits, p->out_frames})
        if (q) cudaStreamDestroy(q);
    if (p->ctx) ufvc_destroy(p->ctx);
    delete p;
}

extern "C" ufvc_status ufvc_pipe_create(ufvc_ctx* ctx, int depth, ufvc_pipe** out) {
    if (!ctx || !out || depth < 1 || depth > 16) return UFVC_ERR_ARG;
    if (cudaSetDevice(ctx_device(ctx)) != cudaSuccess) return UFVC_ERR_CUDA;
    ufvc_pipe* p = new ufvc_pipe();
    p->base = ctx;
    p->slots.resize(depth);
    p->lag = depth >= 5 ? 2 : 1;
    bool ok = (p->ctx = ctx_clone_shared(ctx)) != nullptr;
    for (cudaStream_t* q : {&p->cs, &p->in_frames, &p->out_bits, &p->in_bits, &p->out_frames})
        ok = ok && cudaStreamCreateWithFlags(q, cudaStreamNonBlocking) == cudaSuccess;
    for (PipeSlot& s : p->slots) {
        ok = ok && cudaMalloc(&s.d_nbytes, 8) == cudaSuccess && cudaMallocHost(&s.h_nbytes, 8) == cudaSuccess &&
             cudaHostAlloc(&s.h_status, 8, cudaHostAllocMapped) == cudaSuccess &&
             cudaHostGetDevicePointer(reinterpret_cast<void**>(&s.hd_status), s.h_status, 0) == cudaSuccess;
        for (cudaEvent_t* e : {&s.in, &s.enc, &s.bits_out, &s.bits_in, &s.dec, &s.done})
            ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
        if (ok) {
            *s.h_nbytes = 0;
            s.h_status[0] = s.h_status[1] = 0;
        }
    }
    if (!ok) {
        cudaGetLastError();
        free_pipe(p);
        return UFVC_ERR_OOM;
    }
    *out = p;
    return UFVC_OK;
}

extern "C" void ufvc_pipe_destroy(ufvc_pipe* p) {
    if (!p) return;
    cudaSetDevice(ctx_device(p->base));
    free_pipe(p);
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

__global__ void status_take_kernel(int* status, int* dst) {
    *dst = *status;
    *status = 0;
}

// the status word after a group of kernels into the slot's pinned word i, then cleared (compute stream)
static ufvc_status take_status(ufvc_pipe* p, PipeSlot& s, int i) {
    status_take_kernel<<<1, 1, 0, p->cs>>>(ctx_status_word(p->ctx), s.hd_status + i);
    return cudaGetLastError() == cudaSuccess ? UFVC_OK : UFVC_ERR_CUDA;
}

// the decode of ticket t (its bit-stream back on the device) and its frames out
static ufvc_status enqueue_decode(ufvc_pipe* p, long long t) {
    PipeSlot& s = p->slots[t % (long long)p->slots.size()];
    ufvc_status st;
    if (cudaStreamWaitEvent(p->cs, s.bits_in, 0) != cudaSuccess) return UFVC_ERR_CUDA;
    if ((st = ufvc_decode_chunk_dev(p->ctx, s.d_bits2, s.bmax, s.d_nbytes, s.d_out, s.n_frames, s.width, s.height,
                                    p->cs)))
        return st;
    if ((st = take_status(p, s, 1))) return st;
    if (cudaEventRecord(s.dec, p->cs) != cudaSuccess || cudaStreamWaitEvent(p->out_frames, s.dec, 0) != cudaSuccess ||
        cudaMemcpyAsync(s.h_out, s.d_out, s.fsz, cudaMemcpyDeviceToHost, p->out_frames) != cudaSuccess ||
        cudaEventRecord(s.done, p->out_frames) != cudaSuccess)
        return UFVC_ERR_CUDA;
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_pipe_submit(ufvc_pipe* p, const uint8_t* h_frames, int n_frames, int width, int height,
                                        int qp, uint8_t* h_bits, size_t capacity, uint8_t* h_out, long long* ticket) {
    if (!p || !h_frames || !h_bits || !ticket) return UFVC_ERR_ARG;
    const long long t = p->next;
    PipeSlot& s = p->slots[t % (long long)p->slots.size()];
    if (!s.waited) return UFVC_ERR_ARG;  // wait for ticket t - depth first
    if (cudaSetDevice(ctx_device(p->base)) != cudaSuccess) return UFVC_ERR_CUDA;
    const size_t bmax = ufvc_max_bitstream_bytes(p->ctx, width, height);
    if (bmax == 0) return UFVC_ERR_ARG;
    if (capacity < bmax) return UFVC_ERR_CAPACITY;
    const size_t fsz = (size_t)n_frames * frame_bytes(ctx_color(p->ctx), width, height);
    ufvc_status st;
    if ((st = grow(&s.d_frames, &s.in_cap, fsz)) || (st = grow(&s.d_out, &s.out_cap, fsz)) ||
        (st = grow(&s.d_bits, &s.bits_cap, bmax)) || (st = grow(&s.d_bits2, &s.bits2_cap, bmax)))
        return st;
    s.h_status[0] = s.h_status[1] = 0;
    // frames in; the encode on the compute stream once they have landed
    if (cudaMemcpyAsync(s.d_frames, h_frames, fsz, cudaMemcpyHostToDevice, p->in_frames) != cudaSuccess ||
        cudaEventRecord(s.in, p->in_frames) != cudaSuccess || cudaStreamWaitEvent(p->cs, s.in, 0) != cudaSuccess)
        return UFVC_ERR_CUDA;
    if ((st = ufvc_encode_chunk(p->ctx, s.d_frames, n_frames, width, height, qp, s.d_bits, bmax, s.d_nbytes, p->cs)))
        return st;
    if ((st = take_status(p, s, 0))) return st;
    // the bit-stream buffer and its size out; the host copy back in (the decoder side reads the bit-stream
    // from the host, as a separate receiver would)
    if (cudaEventRecord(s.enc, p->cs) != cudaSuccess || cudaStreamWaitEvent(p->out_bits, s.enc, 0) != cudaSuccess ||
        cudaMemcpyAsync(s.h_nbytes, s.d_nbytes, 8, cudaMemcpyDeviceToHost, p->out_bits) != cudaSuccess ||
        cudaMemcpyAsync(h_bits, s.d_bits, bmax, cudaMemcpyDeviceToHost, p->out_bits) != cudaSuccess ||
        cudaEventRecord(s.bits_out, p->out_bits) != cudaSuccess)
        return UFVC_ERR_CUDA;
    s.ticket = t;
    s.waited = false;
    s.h_out = h_out;
    s.bmax = bmax;
    s.fsz = fsz;
    s.n_frames = n_frames;
    s.width = width;
    s.height = height;
    if (h_out) {
        if (cudaStreamWaitEvent(p->in_bits, s.bits_out, 0) != cudaSuccess ||
            cudaMemcpyAsync(s.d_bits2, h_bits, bmax, cudaMemcpyHostToDevice, p->in_bits) != cudaSuccess ||
            cudaEventRecord(s.bits_in, p->in_bits) != cudaSuccess)
            return UFVC_ERR_CUDA;
    } else if (cudaEventRecord(s.done, p->out_bits) != cudaSuccess) {
        return UFVC_ERR_CUDA;
    }
    p->next = t + 1;
    *ticket = t;
    // the decode of the ticket lag encodes back goes after this encode on the compute stream
    if (h_out) p->pending.push_back(t);
    while (p->pending.size() > p->lag) {
        const long long u = p->pending.front();
        p->pending.pop_front();
        if ((st = enqueue_decode(p, u))) return st;
    }
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_pipe_wait(ufvc_pipe* p, long long ticket, size_t* nbytes) {
    if (!p || ticket < 0) return UFVC_ERR_ARG;
    PipeSlot& s = p->slots[ticket % (long long)p->slots.size()];
    if (s.ticket != ticket || s.waited) return UFVC_ERR_ARG;
    if (cudaSetDevice(ctx_device(p->base)) != cudaSuccess) return UFVC_ERR_CUDA;
    while (!p->pending.empty() && p->pending.front() <= ticket) {  // its decode waits for no later encode
        const long long u = p->pending.front();
        p->pending.pop_front();
        const ufvc_status st = enqueue_decode(p, u);
        if (st) return st;
    }
    if (cudaEventSynchronize(s.done) != cudaSuccess) return UFVC_ERR_CUDA;
    s.waited = true;
    if (nbytes) *nbytes = (size_t)*s.h_nbytes;
    return (ufvc_status)(s.h_status[0] ? s.h_status[0] : s.h_status[1]);
}
