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
// Same-shape work is batched: requests of one frame size and operation (and rate, for encodes) that are
// admitted together run on one slot as one batched call (ufvc_encode_chunks / ufvc_decode_chunks), whose
// entropy-coding launches carry every chunk of the batch; the slot keeps one graph per batch size.
//
// Every slot computes with the same kernels as a single context, and none of them depends on what
// runs beside it or in its batch, so a request's bit-stream and frames are the same alone and in a mix.
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

constexpr int kMaxBatch = 4;

struct Slot {
    int id = 0, W = 0, H = 0, bmax = 1;  // bmax: the slot's batch size
    ufvc_ctx* ctx = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    uint8_t *frames[kMaxBatch] = {}, *bits[kMaxBatch] = {}, *out[kMaxBatch] = {};
    uint64_t* nbytes = nullptr;  // [kMaxBatch]
    void *cin = nullptr, *cout = nullptr;  // temporal context in / out of the slot's calls
    size_t cap = 0, footprint = 0;
    bool busy = false;
    std::vector<uint64_t> tickets;  // the batch running on the slot
    int launch_status = UFVC_OK;
    double last_used = 0;
    // graphs: encode per (batch, qp), decode per batch; ran = the call ran directly once (its buffers exist)
    std::map<int, cudaGraphExec_t> g_enc, g_dec;
    std::unordered_set<int> enc_ran, enc_nograph, dec_ran, dec_nograph;
};

// frame sizes up to 1080p batch four chunks, larger ones run alone; the temporal context runs alone
int batch_size(bool temporal, int W, int H) {
    if (temporal) return 1;
    const long long b = 4ll * 1920 * 1088 / ((long long)W * H);
    return b < 1 ? 1 : b > kMaxBatch ? kMaxBatch : (int)b;
}

}  // namespace

struct ufvc_server {
    ufvc_config cfg{};
    int device = 0, N = 0;
    ufvc_ctx* base = nullptr;
    size_t cap = 0, used = 0;
    int max_slots = 1, next_slot_id = 0;
    std::atomic<int> graphs{0};
    uint64_t completed = 0, next_ticket = 1, batches = 0, batched = 0;
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
    for (auto& kv : sl->g_dec) cudaGraphExecDestroy(kv.second);
    ufvc_destroy(sl->ctx);
    cudaFree(sl->cin);
    cudaFree(sl->cout);
    for (int b = 0; b < kMaxBatch; ++b) {
        cudaFree(sl->frames[b]);
        cudaFree(sl->bits[b]);
        cudaFree(sl->out[b]);
    }
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
    const int bmax = batch_size(S->temporal, W, H);
    // per batch position: plan buffers + workspaces + staging; a margin for the rANS scratch, graphs and
    // allocator rounding
    const size_t fp = bmax * (ctx_plan_bytes(S->base, W, H) + 2 * frame_bytes + cap) + 2 * cb + (64ull << 20);
    if ((int)S->slots.size() >= S->max_slots && !evict_one(S, W, H, false)) return nullptr;
    while (S->cap && S->used + fp > S->cap)
        if (!evict_one(S, W, H, false)) return nullptr;
    auto* sl = new Slot();
    sl->id = S->next_slot_id++;
    sl->W = W;
    sl->H = H;
    sl->bmax = bmax;
    sl->cap = cap;
    sl->footprint = fp;
    sl->ctx = ctx_clone_shared(S->base);
    bool ok = sl->ctx && cudaStreamCreateWithFlags(&sl->st, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&sl->ev, cudaEventDisableTiming) == cudaSuccess &&
              cudaMalloc(&sl->nbytes, 8 * kMaxBatch) == cudaSuccess &&
              (!cb || (cudaMalloc(&sl->cin, cb) == cudaSuccess && cudaMalloc(&sl->cout, cb) == cudaSuccess));
    for (int b = 0; ok && b < bmax; ++b)
        ok = cudaMalloc(&sl->frames[b], frame_bytes) == cudaSuccess && cudaMalloc(&sl->bits[b], cap) == cudaSuccess &&
             cudaMalloc(&sl->out[b], frame_bytes) == cudaSuccess;
    if (!ok) {
        S->err = "server: slot creation failed";
        cudaGetLastError();
        if (sl->ctx) ufvc_destroy(sl->ctx);
        if (sl->st) cudaStreamDestroy(sl->st);
        if (sl->ev) cudaEventDestroy(sl->ev);
        cudaFree(sl->cin);
        cudaFree(sl->cout);
        for (int b = 0; b < kMaxBatch; ++b) {
            cudaFree(sl->frames[b]);
            cudaFree(sl->bits[b]);
            cudaFree(sl->out[b]);
        }
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

// Launch the batch of requests (streams sbs, one operation) on slot sl (called without the lock; only the
// worker touches slots).  A batch of one with the temporal context runs the context calls; every other
// batch runs the batched calls, whose results equal the single-chunk calls'.
void launch(ufvc_server* S, Slot* sl, const std::vector<StreamBuf*>& sbs, int op) {
    ufvc_status st = UFVC_OK;
    const int N = S->N, B = (int)sbs.size(), W = sbs[0]->W, H = sbs[0]->H, qp = sbs[0]->qp;
    StreamBuf* sb = sbs[0];
    // the stream's context into the slot (zeros before its first chunk: C_0 = 0)
    auto ctx_in = [&](const void* c, uint64_t chunks) {
        if (!S->temporal) return;
        if (chunks) cudaMemcpyAsync(sl->cin, c, sb->ctx_bytes, cudaMemcpyDeviceToDevice, sl->st);
        else cudaMemsetAsync(sl->cin, 0, sb->ctx_bytes, sl->st);
    };
    const uint8_t* frames[kMaxBatch];
    const uint8_t* bits_in[kMaxBatch];
    uint8_t* bits[kMaxBatch];
    uint8_t* outs[kMaxBatch];
    uint64_t* nbs[kMaxBatch];
    const uint64_t* nbs_in[kMaxBatch];
    int qps[kMaxBatch];
    for (int b = 0; b < B; ++b) {
        frames[b] = sl->frames[b];
        bits[b] = sl->bits[b];
        bits_in[b] = sl->bits[b];
        outs[b] = sl->out[b];
        nbs[b] = sl->nbytes + b;
        nbs_in[b] = sl->nbytes + b;
        qps[b] = qp;
    }
    if (op == UFVC_OP_ENCODE) {
        for (int b = 0; b < B; ++b)
            cudaMemcpyAsync(sl->frames[b], sbs[b]->in, sb->frame_bytes, cudaMemcpyDeviceToDevice, sl->st);
        ctx_in(sb->ctx_enc, sb->enc_chunks);
        const int key = B * 64 + qp;
        auto it = sl->g_enc.find(key);
        cudaGraphExec_t g = it == sl->g_enc.end() ? nullptr : it->second;
        bool ran = sl->enc_ran.count(key) != 0, nograph = sl->enc_nograph.count(key) != 0;
        st = run_call(S, sl, &g, &ran, &nograph, [&] {
            if (S->temporal)
                return ufvc_encode_chunk_tc(sl->ctx, sl->frames[0], N, W, H, qp, sl->bits[0], sl->cap, sl->nbytes,
                                            sl->cin, sl->cout, sl->st);
            return ufvc_encode_chunks(sl->ctx, B, frames, N, W, H, qps, bits, sl->cap, nbs, sl->st);
        });
        if (g) sl->g_enc[key] = g;
        if (ran) sl->enc_ran.insert(key);
        if (nograph) sl->enc_nograph.insert(key);
        if (st == UFVC_OK) {
            for (int b = 0; b < B; ++b) {
                copy_sized(sbs[b]->bits, sl->bits[b], sl->nbytes + b, sbs[b]->cap, sl->st);
                cudaMemcpyAsync(sbs[b]->nbytes, sl->nbytes + b, 8, cudaMemcpyDeviceToDevice, sl->st);
            }
            if (S->temporal) {
                cudaMemcpyAsync(sb->ctx_enc, sl->cout, sb->ctx_bytes, cudaMemcpyDeviceToDevice, sl->st);
                ++sb->enc_chunks;
            }
        }
    } else {
        for (int b = 0; b < B; ++b) {
            copy_sized(sl->bits[b], sbs[b]->bits, sbs[b]->nbytes, sl->cap, sl->st);
            cudaMemcpyAsync(sl->nbytes + b, sbs[b]->nbytes, 8, cudaMemcpyDeviceToDevice, sl->st);
        }
        ctx_in(sb->ctx_dec, sb->dec_chunks);
        auto it = sl->g_dec.find(B);
        cudaGraphExec_t g = it == sl->g_dec.end() ? nullptr : it->second;
        bool ran = sl->dec_ran.count(B) != 0, nograph = sl->dec_nograph.count(B) != 0;
        st = run_call(S, sl, &g, &ran, &nograph, [&] {
            if (S->temporal)
                return ufvc_decode_chunk_tc(sl->ctx, sl->bits[0], sl->cap, sl->nbytes, sl->out[0], 0, N, W, H,
                                            sl->cin, sl->cout, sl->st);
            return ufvc_decode_chunks(sl->ctx, B, bits_in, sl->cap, nbs_in, outs, N, W, H, sl->st);
        });
        if (g) sl->g_dec[B] = g;
        if (ran) sl->dec_ran.insert(B);
        if (nograph) sl->dec_nograph.insert(B);
        if (st == UFVC_OK) {
            for (int b = 0; b < B; ++b)
                cudaMemcpyAsync(sbs[b]->out, sl->out[b], sb->frame_bytes, cudaMemcpyDeviceToDevice, sl->st);
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
    ufvc_status st = (ufvc_status)sl->launch_status;
    const ufvc_status dev = ufvc_sync_status(sl->ctx, sl->st);  // the slot's work is complete: no wait
    if (st == UFVC_OK) st = dev;
    const double done = S->now_ms();
    const int B = (int)sl->tickets.size();
    uint64_t nb[kMaxBatch] = {};
    if (st == UFVC_OK && cudaMemcpy(nb, sl->nbytes, 8 * B, cudaMemcpyDeviceToHost) != cudaSuccess) st = UFVC_ERR_CUDA;
    for (int b = 0; b < B; ++b) {
        Req& r = S->reqs[sl->tickets[b]];
        StreamBuf* sb = S->streams[r.res.stream_id].get();
        if (st == UFVC_OK) {
            r.res.nbytes = nb[b];
            if (r.res.op == UFVC_OP_ENCODE) sb->has_bits = true;
        }
        r.res.status = st;
        r.res.done_ms = done;
        sb->running = false;
        ++S->completed;
    }
    if (B > 1) {
        ++S->batches;
        S->batched += B;
    }
    sl->tickets.clear();
    sl->busy = false;
    sl->last_used = done;
    S->cv_done.notify_all();
}

// Admit queued requests in arrival order; a stream's later requests wait behind its earlier ones.  A slot
// takes the first admissible request and, up to its batch size, the later queued ones of the same frame
// size and operation (and rate, for encodes) whose streams are free.  Returns the launches to make (the
// caller launches them without holding the lock).
struct Launch {
    Slot* sl;
    std::vector<StreamBuf*> sbs;
    int op;
};

std::vector<Launch> admit(ufvc_server* S) {
    std::vector<Launch> todo;
    std::unordered_set<int> blocked;
    double t_adm = 0;  // a batch's requests start together
    auto take = [&](Req& r, StreamBuf* sb, Slot* sl) {
        sl->tickets.push_back(r.ticket);
        sb->running = true;
        r.res.slot = sl->id;
        r.res.start_ms = t_adm;
    };
    auto fail_no_bits = [&](Req& r) {  // a decode with no bit-stream it can decode
        r.res.status = UFVC_ERR_ARG;
        r.res.done_ms = S->now_ms();
        ++S->completed;
        S->cv_done.notify_all();
    };
    for (auto it = S->queue.begin(); it != S->queue.end();) {
        Req& r = S->reqs[*it];
        StreamBuf* sb = S->streams[r.res.stream_id].get();
        if (sb->running || blocked.count(r.res.stream_id)) {
            blocked.insert(r.res.stream_id);
            ++it;
            continue;
        }
        // a decode needs a bit-stream; with the temporal context it must be the chunk that follows the
        // last one this stream's decoder decoded (the stream holds only its latest bit-stream, so a chunk
        // encoded over an undecoded one has lost its predecessor for the decoder's context chain)
        if (r.res.op == UFVC_OP_DECODE &&
            (!sb->has_bits || (S->temporal && sb->dec_chunks + 1 != sb->enc_chunks))) {
            fail_no_bits(r);
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
        Launch l{sl, {sb}, r.res.op};
        t_adm = S->now_ms();
        take(r, sb, sl);
        it = S->queue.erase(it);
        // the batch's other members: later queued requests of the same shape and operation
        std::unordered_set<int> seen(blocked);
        for (auto jt = it; jt != S->queue.end() && (int)l.sbs.size() < sl->bmax;) {
            Req& q = S->reqs[*jt];
            StreamBuf* qb = S->streams[q.res.stream_id].get();
            const bool free = !qb->running && !seen.count(q.res.stream_id);
            seen.insert(q.res.stream_id);  // a stream's later requests stay behind this one
            if (free && q.res.op == l.op && qb->W == sb->W && qb->H == sb->H &&
                (q.res.op == UFVC_OP_DECODE ? qb->has_bits : qb->qp == sb->qp)) {
                take(q, qb, sl);
                l.sbs.push_back(qb);
                jt = S->queue.erase(jt);
                continue;
            }
            ++jt;
        }
        for (size_t b = 0; b < l.sbs.size(); ++b) S->reqs[sl->tickets[b]].res.batch = (int)l.sbs.size();
        todo.push_back(std::move(l));
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
            lk.unlock();
            for (auto& l : todo) launch(S, l.sl, l.sbs, l.op);
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

extern "C" ufvc_status ufvc_server_submit_many(ufvc_server* S, int n, const int* stream_ids, const int* ops,
                                               uint64_t* tickets) {
    if (!S || n < 0 || (n && (!stream_ids || !ops || !tickets))) return UFVC_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return UFVC_ERR_ARG;
        for (int i = 0; i < n; ++i)  // all or nothing
            if (stream_ids[i] < 0 || stream_ids[i] >= (int)S->streams.size() ||
                (ops[i] != UFVC_OP_ENCODE && ops[i] != UFVC_OP_DECODE))
                return UFVC_ERR_ARG;
        for (int i = 0; i < n; ++i) {
            Req r;
            r.ticket = S->next_ticket++;
            r.res.status = UFVC_PENDING;
            r.res.op = ops[i];
            r.res.stream_id = stream_ids[i];
            r.res.slot = -1;
            r.res.submit_ms = S->now_ms();
            S->reqs[r.ticket] = r;
            S->queue.push_back(r.ticket);
            tickets[i] = r.ticket;
        }
    }
    S->cv_work.notify_one();
    return UFVC_OK;
}

extern "C" ufvc_status ufvc_server_submit(ufvc_server* S, int stream_id, int op, uint64_t* ticket) {
    return ufvc_server_submit_many(S, 1, &stream_id, &op, ticket);
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
    out->batches = S->batches;
    out->batched = S->batched;
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

extern "C" ufvc_status ufvc_server_calibrate_fp8(ufvc_server* S, const uint8_t* d_frames, int n_frames, int width,
                                                 int height, int qp) {
    return server_configure(S, "server_calibrate_fp8", [&] {
        const ufvc_status st = ufvc_calibrate_fp8(S->base, d_frames, n_frames, width, height, qp, nullptr);
        if (st == UFVC_OK) return ufvc_sync_status(S->base, nullptr);
        return st;
    });
}

extern "C" ufvc_status ufvc_server_set_progressive_means(ufvc_server* S, const float* weights, size_t n_weights) {
    return server_configure(S, "server_set_progressive_means",
                            [&] { return ufvc_set_progressive_means(S->base, weights, n_weights); });
}
