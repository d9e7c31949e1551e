// Serving loop: continuous batching of chunk encode / decode requests from many streams.
//
// The paper codes one chunk at a time and names overlapping work across chunks as potential (Sec. 4);
// this is that overlap for a server.  A host scheduler thread owns a pool of slots.  A slot is a
// context that shares the server's weights (ctx_clone_shared), a non-blocking CUDA stream, staging
// buffers for one frame size, and CUDA graphs of its encode (per qp) and decode calls, captured after
// the slot's first direct run of that call.  Requests queue per arrival; the scheduler admits a
// request when its stream has nothing earlier queued or running and a slot of its frame size is idle,
// or a new slot fits under the slot count and the HBM cap (idle slots of other sizes are released,
// least recently used first, to make room).  Work on different slots overlaps on the device; the
// scheduler notices completions through per-slot events and reads each slot context's status word.
//
// Every slot computes with the same kernels as a single context, and none of them depends on what
// runs beside it, so a request's bit-stream and frames are the same alone and in a mix.
//
// With the temporal chunk context (ufvc_server_set_temporal_context, or the DC-block model, which always
// has it) each stream also owns its coding
// state on the device: the encoder's and the decoder's context C_i.  A request copies the stream's
// context into the slot's input buffer (zeros for the stream's first chunk, which equals C_0 = 0),
// runs, and copies the slot's output context back, so the slot's graphs keep fixed pointers and a
// stream's chunks form one context chain whatever slots they run on.
#include "ufvc_internal.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>

using namespace ufvc;

namespace {

using Clock = std::chrono::steady_clock;

// dst[0, n) = src[0, n) with n = min(*n_dev, cap) read on the device (both 16-byte aligned)
__global__ void copy_sized_kernel(uint8_t* dst, const uint8_t* src, const uint64_t* n_dev, size_t cap) {
    size_t n = (size_t)*n_dev;
    if (n > cap) n = cap;
    const size_t n16 = n / 16;
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = tid; i < n16; i += stride)
        reinterpret_cast<uint4*>(dst)[i] = reinterpret_cast<const uint4*>(src)[i];
    if (tid < n - n16 * 16) dst[n16 * 16 + tid] = src[n16 * 16 + tid];
}

void copy_sized(uint8_t* dst, const uint8_t* src, const uint64_t* n_dev, size_t cap, cudaStream_t s) {
    const size_t blocks = std::min<size_t>((cap / 16 + 255) / 256 + 1, 1184);
    copy_sized_kernel<<<(unsigned)blocks, 256, 0, s>>>(dst, src, n_dev, cap);
}

struct StreamBuf {
    int W = 0, H = 0, qp = 32;
    uint8_t *in = nullptr, *bits = nullptr, *out = nullptr;
    uint64_t* nbytes = nullptr;
    size_t cap = 0, frame_bytes = 0, bytes = 0;
    bool running = false, has_bits = false;
    // temporal context: the encoder's and the decoder's C_i, and how many chunks each side has coded
    void *ctx_enc = nullptr, *ctx_dec = nullptr;
    size_t ctx_bytes = 0;
    uint64_t enc_chunks = 0, dec_chunks = 0;
};

struct Req {
    uint64_t ticket = 0;
    ufvc_result res{};
};

struct Slot {
    int id = 0, W = 0, H = 0;
    ufvc_ctx* ctx = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    uint8_t *frames = nullptr, *bits = nullptr, *out = nullptr;
    uint64_t* nbytes = nullptr;
    void *cin = nullptr, *cout = nullptr;  // temporal context in / out of the slot's calls
    size_t cap = 0, footprint = 0;
    bool busy = false;
    uint64_t ticket = 0;
    int launch_status = UFVC_OK;
    double last_used = 0;
    // graphs: encode per qp, decode; ran[] = the call ran directly once (its buffers exist)
    std::map<int, cudaGraphExec_t> g_enc;
    cudaGraphExec_t g_dec = nullptr;
    std::unordered_set<int> enc_ran, enc_nograph;
    bool dec_ran = false, dec_nograph = false;
};

}  // namespace

struct ufvc_server {
    ufvc_config cfg{};
    int device = 0, N = 0;
    ufvc_ctx* base = nullptr;
    size_t cap = 0, used = 0;
    int max_slots = 1, next_slot_id = 0;
    std::atomic<int> graphs{0};
    uint64_t completed = 0, next_ticket = 1;
    bool temporal = false;  // streams carry the temporal chunk context
    std::vector<Slot*> slots;
    std::vector<std::unique_ptr<StreamBuf>> streams;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Req> reqs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    Clock::time_point t0;
    std::string err;

    double now_ms() const { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }
};

namespace {

void destroy_slot(ufvc_server* S, Slot* sl) {
    cudaStreamSynchronize(sl->st);
    for (auto& kv : sl->g_enc) cudaGraphExecDestroy(kv.second);
    if (sl->g_dec) cudaGraphExecDestroy(sl->g_dec);
    ufvc_destroy(sl->ctx);
    cudaFree(sl->cin);
    cudaFree(sl->cout);
    cudaFree(sl->frames);
    cudaFree(sl->bits);
    cudaFree(sl->out);
    cudaFree(sl->nbytes);
    cudaEventDestroy(sl->ev);
    cudaStreamDestroy(sl->st);
    S->used -= sl->footprint;
    delete sl;
}

// Release the least recently used idle slot whose size differs from (W, H) (any idle slot if
// any_size); false if there is none.
bool evict_one(ufvc_server* S, int W, int H, bool any_size) {
    Slot* victim = nullptr;
    for (Slot* sl : S->slots)
        if (!sl->busy && (any_size || sl->W != W || sl->H != H) && (!victim || sl->last_used < victim->last_used))
            victim = sl;
    if (!victim) return false;
    S->slots.erase(std::find(S->slots.begin(), S->slots.end(), victim));
    destroy_slot(S, victim);
    return true;
}

Slot* make_slot(ufvc_server* S, int W, int H) {
    const size_t frame_bytes = (size_t)S->N * W * H * 3;
    const size_t cap = ufvc_max_bitstream_bytes(S->base, W, H);
    const size_t cb = S->temporal ? ufvc_context_bytes(S->base, W, H) : 0;
    // plan buffers + workspaces + staging + a margin for the rANS scratch, graphs and allocator rounding
    const size_t fp = ctx_plan_bytes(S->base, W, H) + 2 * frame_bytes + cap + 2 * cb + (64ull << 20);
    if ((int)S->slots.size() >= S->max_slots && !evict_one(S, W, H, false)) return nullptr;
    while (S->cap && S->used + fp > S->cap)
        if (!evict_one(S, W, H, false)) return nullptr;
    auto* sl = new Slot();
    sl->id = S->next_slot_id++;
    sl->W = W;
    sl->H = H;
    sl->cap = cap;
    sl->footprint = fp;
    sl->ctx = ctx_clone_shared(S->base);
    bool ok = sl->ctx && cudaStreamCreateWithFlags(&sl->st, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&sl->ev, cudaEventDisableTiming) == cudaSuccess &&
              cudaMalloc(&sl->frames, frame_bytes) == cudaSuccess && cudaMalloc(&sl->bits, cap) == cudaSuccess &&
              cudaMalloc(&sl->out, frame_bytes) == cudaSuccess && cudaMalloc(&sl->nbytes, 8) == cudaSuccess &&
              (!cb || (cudaMalloc(&sl->cin, cb) == cudaSuccess && cudaMalloc(&sl->cout, cb) == cudaSuccess));
    if (!ok) {
        S->err = "server: slot creation failed";
        cudaGetLastError();
        if (sl->ctx) ufvc_destroy(sl->ctx);
        if (sl->st) cudaStreamDestroy(sl->st);
        if (sl->ev) cudaEventDestroy(sl->ev);
        cudaFree(sl->cin);
        cudaFree(sl->cout);
        cudaFree(sl->frames);
        cudaFree(sl->bits);
        cudaFree(sl->out);
        cudaFree(sl->nbytes);
        delete sl;
        return nullptr;
    }
    S->used += fp;
    S->slots.push_back(sl);
    return sl;
}

// Run fn directly, or as the slot's graph for this call: the first run is direct (it creates the
// plan's buffers), the second is captured into a graph that later requests replay.  A call that cannot
// be captured keeps running directly.
template <class F>
ufvc_status run_call(ufvc_server* S, Slot* sl, cudaGraphExec_t* g, bool* ran, bool* nograph, F&& fn) {
    if (*g) return cudaGraphLaunch(*g, sl->st) == cudaSuccess ? UFVC_OK : UFVC_ERR_CUDA;
    if (!*ran || *nograph) {
        const ufvc_status st = fn();
        if (st == UFVC_OK) *ran = true;
        return st;
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(sl->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        *nograph = true;
        return fn();
    }
    const ufvc_status st = fn();
    const cudaError_t e = cudaStreamEndCapture(sl->st, &graph);
    if (st == UFVC_OK && e == cudaSuccess && graph &&
        cudaGraphInstantiate(g, graph, 0) == cudaSuccess) {
        cudaGraphDestroy(graph);
        ++S->graphs;
        return cudaGraphLaunch(*g, sl->st) == cudaSuccess ? UFVC_OK : UFVC_ERR_CUDA;
    }
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    *g = nullptr;
    *nograph = true;
    return fn();
}

// Launch request r of stream sb on slot sl (called without the lock; only the worker touches slots).
void launch(ufvc_server* S, Slot* sl, StreamBuf* sb, int op) {
    ufvc_status st = UFVC_OK;
    const int N = S->N, W = sb->W, H = sb->H;
    // the stream's context into the slot (zeros before its first chunk: C_0 = 0)
    auto ctx_in = [&](const void* c, uint64_t chunks) {
        if (!S->temporal) return;
        if (chunks) cudaMemcpyAsync(sl->cin, c, sb->ctx_bytes, cudaMemcpyDeviceToDevice, sl->st);
        else cudaMemsetAsync(sl->cin, 0, sb->ctx_bytes, sl->st);
    };
    if (op == UFVC_OP_ENCODE) {
        cudaMemcpyAsync(sl->frames, sb->in, sb->frame_bytes, cudaMemcpyDeviceToDevice, sl->st);
        ctx_in(sb->ctx_enc, sb->enc_chunks);
        auto it = sl->g_enc.find(sb->qp);
        cudaGraphExec_t g = it == sl->g_enc.end() ? nullptr : it->second;
        bool ran = sl->enc_ran.count(sb->qp) != 0, nograph = sl->enc_nograph.count(sb->qp) != 0;
        st = run_call(S, sl, &g, &ran, &nograph, [&] {
            if (S->temporal)
                return ufvc_encode_chunk_tc(sl->ctx, sl->frames, N, W, H, sb->qp, sl->bits, sl->cap, sl->nbytes,
                                            sl->cin, sl->cout, sl->st);
            return ufvc_encode_chunk(sl->ctx, sl->frames, N, W, H, sb->qp, sl->bits, sl->cap, sl->nbytes, sl->st);
        });
        if (g) sl->g_enc[sb->qp] = g;
        if (ran) sl->enc_ran.insert(sb->qp);
        if (nograph) sl->enc_nograph.insert(sb->qp);
        if (st == UFVC_OK) {
            copy_sized(sb->bits, sl->bits, sl->nbytes, sb->cap, sl->st);
            cudaMemcpyAsync(sb->nbytes, sl->nbytes, 8, cudaMemcpyDeviceToDevice, sl->st);
            if (S->temporal) {
                cudaMemcpyAsync(sb->ctx_enc, sl->cout, sb->ctx_bytes, cudaMemcpyDeviceToDevice, sl->st);
                ++sb->enc_chunks;
            }
        }
    } else {
        copy_sized(sl->bits, sb->bits, sb->nbytes, sl->cap, sl->st);
        cudaMemcpyAsync(sl->nbytes, sb->nbytes, 8, cudaMemcpyDeviceToDevice, sl->st);
        ctx_in(sb->ctx_dec, sb->dec_chunks);
        st = run_call(S, sl, &sl->g_dec, &sl->dec_ran, &sl->dec_nograph, [&] {
            if (S->temporal)
                return ufvc_decode_chunk_tc(sl->ctx, sl->bits, sl->cap, sl->nbytes, sl->out, 0, N, W, H, sl->cin,
                                            sl->cout, sl->st);
            return ufvc_decode_chunk_dev(sl->ctx, sl->bits, sl->cap, sl->nbytes, sl->out, N, W, H, sl->st);
        });
        if (st == UFVC_OK) {
            cudaMemcpyAsync(sb->out, sl->out, sb->frame_bytes, cudaMemcpyDeviceToDevice, sl->st);
            if (S->temporal) {
                cudaMemcpyAsync(sb->ctx_dec, sl->cout, sb->ctx_bytes, cudaMemcpyDeviceToDevice, sl->st);
                ++sb->dec_chunks;
            }
        }
    }
    if (st == UFVC_OK && cudaGetLastError() != cudaSuccess) st = UFVC_ERR_CUDA;
    sl->launch_status = st;
    cudaEventRecord(sl->ev, sl->st);
}

void finish(ufvc_server* S, Slot* sl) {
    Req& r = S->reqs[sl->ticket];
    StreamBuf* sb = S->streams[r.res.stream_id].get();
    ufvc_status st = (ufvc_status)sl->launch_status;
    const ufvc_status dev = ufvc_sync_status(sl->ctx, sl->st);  // the slot's work is complete: no wait
    if (st == UFVC_OK) st = dev;
    if (st == UFVC_OK) {
        uint64_t nb = 0;
        if (cudaMemcpy(&nb, r.res.op == UFVC_OP_ENCODE ? sb->nbytes : sl->nbytes, 8, cudaMemcpyDeviceToHost) ==
            cudaSuccess)
            r.res.nbytes = nb;
        if (r.res.op == UFVC_OP_ENCODE) sb->has_bits = true;
    }
    r.res.status = st;
    r.res.done_ms = S->now_ms();
    sl->busy = false;
    sl->last_used = r.res.done_ms;
    sb->running = false;
    ++S->completed;
    S->cv_done.notify_all();
}

// Admit queued requests in arrival order; a stream's later requests wait behind its earlier ones.
// Returns the launches to make (the caller launches them without holding the lock).
std::vector<std::pair<Slot*, uint64_t>> admit(ufvc_server* S) {
    std::vector<std::pair<Slot*, uint64_t>> todo;
    std::unordered_set<int> blocked;
    for (auto it = S->queue.begin(); it != S->queue.end();) {
        Req& r = S->reqs[*it];
        StreamBuf* sb = S->streams[r.res.stream_id].get();
        if (sb->running || blocked.count(r.res.stream_id)) {
            blocked.insert(r.res.stream_id);
            ++it;
            continue;
        }
        if (r.res.op == UFVC_OP_DECODE && !sb->has_bits) {  // nothing encoded yet on this stream
            r.res.status = UFVC_ERR_ARG;
            r.res.done_ms = S->now_ms();
            ++S->completed;
            S->cv_done.notify_all();
            it = S->queue.erase(it);
            continue;
        }
        Slot* sl = nullptr;
        for (Slot* c : S->slots)
            if (!c->busy && c->W == sb->W && c->H == sb->H) { sl = c; break; }
        if (!sl) sl = make_slot(S, sb->W, sb->H);
        if (!sl) {
            blocked.insert(r.res.stream_id);
            ++it;
            continue;
        }
        sl->busy = true;
        sl->ticket = r.ticket;
        sb->running = true;
        r.res.slot = sl->id;
        r.res.start_ms = S->now_ms();
        todo.emplace_back(sl, r.ticket);
        it = S->queue.erase(it);
    }
    return todo;
}

void worker_main(ufvc_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        bool busy = false;
        for (Slot* sl : S->slots) {
            if (!sl->busy) continue;
            const cudaError_t q = cudaEventQuery(sl->ev);
            if (q == cudaErrorNotReady) { busy = true; continue; }
            if (q != cudaSuccess) cudaGetLastError();
            finish(S, sl);
        }
        auto todo = admit(S);
        if (!todo.empty()) {
            std::vector<std::pair<Slot*, std::pair<StreamBuf*, int>>> work;
            for (auto& t : todo) {
                const Req& r = S->reqs[t.second];
                work.push_back({t.first, {S->streams[r.res.stream_id].get(), r.res.op}});
            }
            lk.unlock();
            for (auto& w : work) launch(S, w.first, w.second.first, w.second.second);
            lk.lock();
            continue;
        }
        if (S->stop && S->queue.empty() && !busy) break;
        if (busy) S->cv_work.wait_for(lk, std::chrono::microseconds(20));
        else S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
    }
}

}  // namespace

extern "C" ufvc_status ufvc_server_create(const ufvc_config* cfg, const float* weights, size_t n_weights,
                                          size_t hbm_cap_bytes, int max_slots, ufvc_server** out) {
    if (!cfg || !out || max_slots < 1) return UFVC_ERR_ARG;
    *out = nullptr;
    auto* S = new ufvc_server();
    S->cfg = *cfg;
    S->device = cfg->device;
    S->N = cfg->chunk_len;
    S->cap = hbm_cap_bytes;
    S->max_slots = max_slots;
    S->t0 = Clock::now();
    const ufvc_status st = ufvc_create(cfg, weights, n_weights, &S->base);
    if (st != UFVC_OK) {
        delete S;
        return st;
    }
    S->temporal = ctx_temporal(S->base);  // the DC-block model carries its context from the start
    S->worker = std::thread(worker_main, S);
    *out = S;
    return UFVC_OK;
}

extern "C" void ufvc_server_destroy(ufvc_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    S->worker.join();
    cudaSetDevice(S->device);
    for (Slot* sl : S->slots) destroy_slot(S, sl);
    for (auto& sb : S->streams) {
        cudaFree(sb->in);
        cudaFree(sb->bits);
        cudaFree(sb->out);
        cudaFree(sb->nbytes);
        cudaFree(sb->ctx_enc);
        cudaFree(sb->ctx_dec);
    }
    ufvc_destroy(S->base);
    delete S;
}

extern "C" ufvc_status ufvc_server_open_stream(ufvc_server* S, int width, int height, int qp, int* stream_id) {
    if (!S || !stream_id || width < 16 || height < 16 || width > 65535 || height > 65535 || qp < 0 || qp > 63)
        return UFVC_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto sb = std::make_unique<StreamBuf>();
    sb->W = width;
    sb->H = height;
    sb->qp = qp;
    sb->frame_bytes = (size_t)S->N * width * height * 3;
    sb->cap = ufvc_max_bitstream_bytes(S->base, width, height);
    sb->ctx_bytes = S->temporal ? ufvc_context_bytes(S->base, width, height) : 0;
    sb->bytes = 2 * sb->frame_bytes + sb->cap + 256 + 2 * sb->ctx_bytes;
    if (S->cap && S->used + sb->bytes > S->cap) {
        S->err = "server: stream buffers exceed the HBM cap";
        return UFVC_ERR_OOM;
    }
    if (cudaSetDevice(S->device) != cudaSuccess || cudaMalloc(&sb->in, sb->frame_bytes) != cudaSuccess ||
        cudaMalloc(&sb->bits, sb->cap) != cudaSuccess || cudaMalloc(&sb->out, sb->frame_bytes) != cudaSuccess ||
        cudaMalloc(&sb->nbytes, 8) != cudaSuccess || cudaMemset(sb->nbytes, 0, 8) != cudaSuccess ||
        (sb->ctx_bytes && (cudaMalloc(&sb->ctx_enc, sb->ctx_bytes) != cudaSuccess ||
                           cudaMalloc(&sb->ctx_dec, sb->ctx_bytes) != cudaSuccess))) {
        cudaGetLastError();
        cudaFree(sb->ctx_enc);
        cudaFree(sb->ctx_dec);
        cudaFree(sb->in);
        cudaFree(sb->bits);
        cudaFree(sb->out);
        cudaFree(sb->nbytes);
        S->err = "server: stream buffer allocation failed";
        return UFVC_ERR_OOM;
    }
    S->used += sb->bytes;
    *stream_id = (int)S->streams.size();
    S->streams.push_back(std::move(sb));
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_server_stream_buffers(ufvc_server* S, int stream_id, uint8_t** d_frames_in,
                                                  uint8_t** d_bits, uint64_t** d_nbytes, size_t* capacity,
                                                  uint8_t** d_frames_out) {
    if (!S) return UFVC_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (stream_id < 0 || stream_id >= (int)S->streams.size()) return UFVC_ERR_ARG;
    StreamBuf* sb = S->streams[stream_id].get();
    if (d_frames_in) *d_frames_in = sb->in;
    if (d_bits) *d_bits = sb->bits;
    if (d_nbytes) *d_nbytes = sb->nbytes;
    if (capacity) *capacity = sb->cap;
    if (d_frames_out) *d_frames_out = sb->out;
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_server_submit(ufvc_server* S, int stream_id, int op, uint64_t* ticket) {
    if (!S || !ticket || (op != UFVC_OP_ENCODE && op != UFVC_OP_DECODE)) return UFVC_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (stream_id < 0 || stream_id >= (int)S->streams.size() || S->stop) return UFVC_ERR_ARG;
        Req r;
        r.ticket = S->next_ticket++;
        r.res.status = UFVC_PENDING;
        r.res.op = op;
        r.res.stream_id = stream_id;
        r.res.slot = -1;
        r.res.submit_ms = S->now_ms();
        S->reqs[r.ticket] = r;
        S->queue.push_back(r.ticket);
        *ticket = r.ticket;
    }
    S->cv_work.notify_one();
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_server_poll(ufvc_server* S, uint64_t ticket, ufvc_result* out) {
    if (!S) return UFVC_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return UFVC_ERR_ARG;
    if (out) *out = it->second.res;
    return (ufvc_status)it->second.res.status;
}

extern "C" ufvc_status ufvc_server_wait(ufvc_server* S, uint64_t ticket, double timeout_ms, ufvc_result* out) {
    if (!S) return UFVC_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return UFVC_ERR_ARG;
    auto done = [&] { return it->second.res.status != UFVC_PENDING; };
    if (timeout_ms < 0) S->cv_done.wait(lk, done);
    else S->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), done);
    if (out) *out = it->second.res;
    return (ufvc_status)it->second.res.status;
}

extern "C" ufvc_status ufvc_server_stats_get(ufvc_server* S, ufvc_server_stats* out) {
    if (!S || !out) return UFVC_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    out->slots = (int)S->slots.size();
    out->busy_slots = 0;
    for (Slot* sl : S->slots) out->busy_slots += sl->busy;
    out->queued = (int)S->queue.size();
    out->graphs = S->graphs;
    out->completed = S->completed;
    out->hbm_used = S->used;
    out->hbm_cap = S->cap;
    return UFVC_OK;
}

extern "C" const char* ufvc_server_last_error(const ufvc_server* S) { return S ? S->err.c_str() : "null server"; }

// The optional networks are set on the server's weight copy before any slot clones it.
template <class Fn>
static ufvc_status server_configure(ufvc_server* S, const char* what, Fn fn) {
    if (!S) return UFVC_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->streams.empty() || !S->slots.empty()) {
        S->err = std::string(what) + ": only before the first stream is opened";
        return UFVC_ERR_ARG;
    }
    const ufvc_status st = fn();
    if (st != UFVC_OK) S->err = std::string(what) + ": " + ufvc_last_error(S->base);
    return st;
}

extern "C" ufvc_status ufvc_server_set_temporal_context(ufvc_server* S, const float* weights, size_t n_weights) {
    return server_configure(S, "server_set_temporal_context", [&] {
        const ufvc_status st = ufvc_set_temporal_context(S->base, weights, n_weights);
        if (st == UFVC_OK) S->temporal = true;
        return st;
    });
}

extern "C" ufvc_status ufvc_server_set_progressive_means(ufvc_server* S, const float* weights, size_t n_weights) {
    return server_configure(S, "server_set_progressive_means",
                            [&] { return ufvc_set_progressive_means(S->base, weights, n_weights); });
}
