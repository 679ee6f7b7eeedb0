// Continuous-batching serving engine and the launch-variant autotuner.
//
// Serving: requests (host headers + host id buffer, any loaded ruleset) are queued by
// tang_serve_submit. A worker thread owns a set of device slots (header + id buffers of
// max_batch packets, a stream, pinned staging), each admitted against the context's memory
// pool when the engine starts. Whenever a slot is free it packs queued requests of one ruleset
// (FIFO order, up to max_batch packets; a larger request is split across launches), stages them
// H2D, classifies them and copies the ids back on the slot's stream. Slots run concurrently on
// their own streams, so requests that arrive while others are on the GPU are admitted as soon as
// a slot frees up and their copies and kernels overlap with the work already in flight.
#include <algorithm>
#include <chrono>
#include <cstring>

#include "internal.h"

namespace tang {

struct Request {
    uint64_t id;
    uint32_t rs;
    const tang_header *h;
    uint32_t n;
    uint32_t *ids;
    uint32_t next = 0;        // first packet not yet dispatched
    uint32_t outstanding = 0; // launches in flight
    double submit_s = 0, start_s = 0, done_s = 0;
    bool done = false;
    int rc = TANG_OK;
};

struct Piece {
    Request *req;
    uint32_t off, n, slot_off;
};

struct ServeSlot {
    void *d_h = nullptr, *d_ids = nullptr;
    tang_header *p_h = nullptr;
    uint32_t *p_ids = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    std::vector<Piece> pieces;
};

struct ServeEngine {
    tang_ctx *ctx;
    tang_serve_cfg cfg;
    std::vector<ServeSlot> slots;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> reqs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    bool slot_finished = false;  // set by a stream callback: some slot's work completed
    uint64_t next_id = 1;
};

double now_s() { return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count(); }

int enqueue_classify_path(tang_ctx *ctx, uint32_t rs, const tang_header *h, uint32_t n, uint32_t *ids, uint32_t path,
                          cudaStream_t st);

// Runs on a CUDA driver thread after a slot's D2H copy: wakes the worker (no CUDA calls here).
static void CUDART_CB slot_done(void *arg) {
    ServeEngine *E = static_cast<ServeEngine *>(arg);
    {
        std::lock_guard<std::mutex> g(E->mu);
        E->slot_finished = true;
    }
    E->cv_work.notify_one();
}

// The worker. The engine lock guards the queue and the requests' bookkeeping only; host copies
// (staging headers, delivering ids) and CUDA calls run outside it, so submitters and pollers
// are not held up by the copies.
static void serve_loop(ServeEngine *E) {
    tang_ctx *ctx = E->ctx;
    cudaSetDevice(ctx->device);
    std::vector<ServeSlot *> finished, launched;
    std::vector<uint32_t> launched_rs;
    std::unique_lock<std::mutex> lk(E->mu);
    while (true) {
        // 1. slots whose work completed (their pieces are read below without the lock)
        finished.clear();
        for (auto &s : E->slots)
            if (s.busy && cudaEventQuery(s.ev) == cudaSuccess) finished.push_back(&s);
        E->slot_finished = false;
        // 2. pack queued requests of one ruleset (FIFO, up to max_batch) into each free slot
        launched.clear();
        launched_rs.clear();
        const double t_pack = now_s();
        for (auto &s : E->slots) {
            if (s.busy || E->queue.empty()) continue;
            const uint32_t rs = E->queue.front()->rs;
            uint32_t used = 0;
            for (auto it = E->queue.begin(); it != E->queue.end() && used < E->cfg.max_batch;) {
                Request *r = *it;
                if (r->rs != rs) {
                    ++it;
                    continue;
                }
                const uint32_t take = std::min(E->cfg.max_batch - used, r->n - r->next);
                if (r->next == 0) r->start_s = t_pack;
                s.pieces.push_back(Piece{r, r->next, take, used});
                r->next += take;
                r->outstanding++;
                used += take;
                if (r->next == r->n)
                    it = E->queue.erase(it);
                else
                    break;  // the slot is full
            }
            if (used == 0) continue;
            s.busy = true;
            launched.push_back(&s);
            launched_rs.push_back(rs);
        }
        lk.unlock();
        // 3. deliver the finished slots' ids to their requests
        for (ServeSlot *s : finished)
            for (const Piece &p : s->pieces)
                std::memcpy(p.req->ids + p.off, s->p_ids + p.slot_off, sizeof(uint32_t) * p.n);
        // 4. stage and launch the packed slots: H2D, classify, D2H, then a completion callback
        for (size_t k = 0; k < launched.size(); ++k) {
            ServeSlot &s = *launched[k];
            uint32_t used = 0;
            for (const Piece &p : s.pieces) {
                std::memcpy(s.p_h + p.slot_off, p.req->h + p.off, sizeof(tang_header) * p.n);
                used = std::max(used, p.slot_off + p.n);
            }
            cudaMemcpyAsync(s.d_h, s.p_h, sizeof(tang_header) * used, cudaMemcpyHostToDevice, s.st);
            const int rc = enqueue_classify_path(ctx, launched_rs[k], static_cast<tang_header *>(s.d_h), used,
                                                 static_cast<uint32_t *>(s.d_ids), E->cfg.path, s.st);
            if (rc)
                for (const Piece &p : s.pieces) p.req->rc = rc;
            cudaMemcpyAsync(s.p_ids, s.d_ids, sizeof(uint32_t) * used, cudaMemcpyDeviceToHost, s.st);
            cudaEventRecord(s.ev, s.st);
            cudaLaunchHostFunc(s.st, slot_done, E);
        }
        lk.lock();
        // 5. bookkeeping of the delivered pieces; free their slots
        if (!finished.empty()) {
            const double t = now_s();
            for (ServeSlot *s : finished) {
                for (const Piece &p : s->pieces)
                    if (--p.req->outstanding == 0 && p.req->next == p.req->n) {
                        p.req->done = true;
                        p.req->done_s = t;
                    }
                s->pieces.clear();
                s->busy = false;
            }
            E->cv_done.notify_all();
            continue;  // a slot is free: look at the queue again at once
        }
        bool any_busy = false;
        for (auto &s : E->slots) any_busy |= s.busy;
        if (E->stop && E->queue.empty() && !any_busy) break;
        if (!launched.empty()) continue;
        // 6. sleep until a slot completes or the engine stops. An idle GPU takes new work at once;
        // while launches are in flight, requests arriving within a short window are batched into
        // one launch instead of one small launch each (many small concurrent kernels contend for
        // the SMs and lengthen every request's latency)
        if (any_busy)
            E->cv_work.wait_for(lk, std::chrono::microseconds(100), [&] { return E->slot_finished || E->stop; });
        else
            E->cv_work.wait_for(lk, std::chrono::milliseconds(5),
                                [&] { return E->slot_finished || E->stop || !E->queue.empty(); });
    }
}

}  // namespace tang

using namespace tang;

extern "C" {

int tang_serve_start(tang_ctx *ctx, const tang_serve_cfg *cfg) {
    if (!ctx || !cfg) return TANG_EINVAL;
    if (ctx->serve) return set_err(ctx, TANG_EINVAL, "serving engine already running");
    const uint32_t path = cfg->path & TANG_PATH_MASK;
    if (path != TANG_PATH_FUSED_BF16 && path != TANG_PATH_FUSED_FP8 && path != TANG_PATH_NO_NN)
        return set_err(ctx, TANG_EINVAL, "serving supports the fused and no-network paths (no shared scratch)");
    if (cfg->max_batch == 0 || cfg->max_inflight == 0) return set_err(ctx, TANG_EINVAL, "empty serving configuration");
    cudaSetDevice(ctx->device);
    ServeEngine *E = new ServeEngine();
    E->ctx = ctx;
    E->cfg = *cfg;
    E->cfg.path = path;
    // admit as many slots as the memory pool allows (at least one)
    for (uint32_t k = 0; k < cfg->max_inflight; ++k) {
        ServeSlot s;
        if (ctx_alloc(ctx, sizeof(tang_header) * size_t(cfg->max_batch), &s.d_h)) break;
        if (ctx_alloc(ctx, sizeof(uint32_t) * size_t(cfg->max_batch), &s.d_ids)) {
            ctx_free(ctx, s.d_h);
            break;
        }
        if (cudaMallocHost(reinterpret_cast<void **>(&s.p_h), sizeof(tang_header) * size_t(cfg->max_batch)) != cudaSuccess ||
            cudaMallocHost(reinterpret_cast<void **>(&s.p_ids), sizeof(uint32_t) * size_t(cfg->max_batch)) != cudaSuccess ||
            cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess) {
            ctx_free(ctx, s.d_h);
            ctx_free(ctx, s.d_ids);
            break;
        }
        E->slots.push_back(s);
    }
    ctx->err.clear();
    if (E->slots.empty()) {
        delete E;
        return set_err(ctx, TANG_ENOMEM, "no serving slot fits in the memory pool");
    }
    ctx->serve = E;
    E->worker = std::thread(serve_loop, E);
    return TANG_OK;
}

int tang_serve_submit(tang_ctx *ctx, uint32_t rs, const tang_header *h, uint32_t n, uint32_t *ids, uint64_t *req_id) {
    if (!ctx || !req_id || (n && (!h || !ids))) return TANG_EINVAL;
    ServeEngine *E = ctx->serve;
    if (!E) return set_err(ctx, TANG_EINVAL, "serving engine not started");
    if (ctx->rulesets.find(rs) == ctx->rulesets.end()) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rs);
    Request *r = new Request();
    r->rs = rs;
    r->h = h;
    r->n = n;
    r->ids = ids;
    r->submit_s = now_s();
    std::lock_guard<std::mutex> g(E->mu);
    r->id = E->next_id++;
    E->reqs[r->id] = r;
    if (n == 0) {
        r->done = true;
        r->start_s = r->done_s = r->submit_s;
    } else {
        E->queue.push_back(r);
        E->cv_work.notify_one();
    }
    *req_id = r->id;
    return TANG_OK;
}

int tang_serve_poll(tang_ctx *ctx, uint64_t req_id, int wait_ms, tang_req_stats *stats) {
    if (!ctx) return TANG_EINVAL;
    ServeEngine *E = ctx->serve;
    if (!E) return set_err(ctx, TANG_EINVAL, "serving engine not started");
    std::unique_lock<std::mutex> lk(E->mu);
    auto it = E->reqs.find(req_id);
    if (it == E->reqs.end()) return set_err(ctx, TANG_ENOTFOUND, "unknown request %llu", (unsigned long long)req_id);
    Request *r = it->second;
    if (!r->done && wait_ms > 0)
        E->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return r->done; });
    if (!r->done) return TANG_EAGAIN;
    if (stats) {
        stats->submit_s = r->submit_s;
        stats->start_s = r->start_s;
        stats->done_s = r->done_s;
    }
    const int rc = r->rc;
    E->reqs.erase(it);
    delete r;
    if (rc) return set_err(ctx, rc, "request failed: %s", ctx->err.c_str());
    return TANG_OK;
}

int tang_serve_stop(tang_ctx *ctx) {
    if (!ctx || !ctx->serve) return TANG_OK;
    ServeEngine *E = ctx->serve;
    {
        std::lock_guard<std::mutex> g(E->mu);
        E->stop = true;
        E->cv_work.notify_all();
    }
    if (E->worker.joinable()) E->worker.join();
    for (auto &s : E->slots) {
        cudaStreamSynchronize(s.st);
        ctx_free(ctx, s.d_h);
        ctx_free(ctx, s.d_ids);
        cudaFreeHost(s.p_h);
        cudaFreeHost(s.p_ids);
        cudaStreamDestroy(s.st);
        cudaEventDestroy(s.ev);
    }
    for (auto &kv : E->reqs) delete kv.second;
    delete E;
    ctx->serve = nullptr;
    return TANG_OK;
}

}  // extern "C"
