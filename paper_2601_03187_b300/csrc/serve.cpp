// Continuous-batching serving engine.
//
// Requests (host headers + host id buffer, any loaded ruleset) are queued by tang_serve_submit.
// A worker thread owns up to max_inflight slots (a stream, pinned staging of max_batch packets).
// A slot's device buffers (headers and ids of max_batch packets) are admitted against the
// context's memory pool (or the device's free memory when the pool is unbounded) only when work
// needs another slot, and given back once the slot has been idle for a while, so the number of
// slots in flight follows the memory that rulesets, models and other callers leave free: a
// ruleset loaded while serving runs lowers it, an unloaded one raises it. Whenever an admitted
// slot is free it packs queued requests of one ruleset (FIFO order, up to max_batch packets; a
// larger request is split across launches), stages them H2D, classifies them and copies the ids
// back on the slot's stream. Slots run concurrently on their own streams, so requests that arrive
// while others are on the GPU are admitted as soon as a slot and memory free up, and their copies
// and kernels overlap with the work already in flight.
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
    void *d_h = nullptr, *d_ids = nullptr;  // admitted device buffers (null while not admitted)
    tang_header *p_h = nullptr;
    uint32_t *p_ids = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    double idle_since = 0;
    std::vector<Piece> pieces;
};

// A slot that has held no work for this long gives its device buffers back to the pool.
constexpr double kSlotIdleRelease = 0.02;
// Admission retries while nothing is in flight that could free memory, before queued requests
// fail with TANG_ENOMEM.
constexpr double kAdmitGiveUp = 1.0;

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
    // admission counters (tang_serve_info)
    uint32_t admitted = 0, admitted_peak = 0;
    uint64_t refusals = 0, launches = 0, packets = 0;
    double refused_since = 0;    // first refusal while nothing was in flight (0: none)
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
    const size_t bytes_h = sizeof(tang_header) * size_t(E->cfg.max_batch), bytes_ids = sizeof(uint32_t) * size_t(E->cfg.max_batch);
    std::vector<ServeSlot *> finished, launched, release;
    std::vector<uint32_t> launched_rs;
    std::unique_lock<std::mutex> lk(E->mu);
    while (true) {
        const double t_now = now_s();
        // 1. slots whose work completed (their pieces are read below without the lock)
        finished.clear();
        for (auto &s : E->slots)
            if (s.busy && cudaEventQuery(s.ev) == cudaSuccess) finished.push_back(&s);
        E->slot_finished = false;
        // 2. pack queued requests of one ruleset (FIFO, up to max_batch) into each free admitted
        // slot; note whether queued work wants one more slot admitted, and which idle slots give
        // their memory back
        launched.clear();
        launched_rs.clear();
        release.clear();
        ServeSlot *admit = nullptr;
        for (auto &s : E->slots) {
            if (s.busy) continue;
            if (!s.d_h) {
                if (!admit && !E->queue.empty()) admit = &s;
                continue;
            }
            if (E->queue.empty()) {
                if (t_now - s.idle_since > kSlotIdleRelease) release.push_back(&s);
                continue;
            }
            const uint32_t rs = E->queue.front()->rs;
            uint32_t used = 0;
            for (auto it = E->queue.begin(); it != E->queue.end() && used < E->cfg.max_batch;) {
                Request *r = *it;
                if (r->rs != rs) {
                    ++it;
                    continue;
                }
                const uint32_t take = std::min(E->cfg.max_batch - used, r->n - r->next);
                if (r->next == 0) r->start_s = t_now;
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
            E->launches++;
            E->packets += used;
        }
        if (!launched.empty()) admit = nullptr;  // admit only when every admitted slot is busy
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
        // 5. admission of one more slot against the pool / free device memory, and the release
        // of long-idle slots (memory calls outside the engine lock)
        bool admitted_now = false, refused_now = false;
        if (admit) {
            void *dh = nullptr, *di = nullptr;
            if (ctx_try_alloc(ctx, bytes_h, &dh) == TANG_OK && ctx_try_alloc(ctx, bytes_ids, &di) == TANG_OK) {
                admit->d_h = dh;
                admit->d_ids = di;
                admitted_now = true;
            } else {
                ctx_free(ctx, dh);
                refused_now = true;
            }
        }
        for (ServeSlot *s : release) {
            ctx_free(ctx, s->d_h);
            ctx_free(ctx, s->d_ids);
            s->d_h = s->d_ids = nullptr;
        }
        lk.lock();
        if (admitted_now) {
            E->admitted_peak = std::max(E->admitted_peak, ++E->admitted);
            E->refused_since = 0;
            admit->idle_since = now_s();
        }
        E->admitted -= uint32_t(release.size());
        bool any_busy = false;
        for (auto &s : E->slots) any_busy |= s.busy;
        if (refused_now) {
            E->refusals++;
            // with nothing in flight, no memory will come back from this engine: give up on the
            // queued requests after a bounded wait (another caller may still free memory)
            if (!any_busy && finished.empty() && E->admitted == 0) {
                if (E->refused_since == 0) E->refused_since = t_now;
                if (t_now - E->refused_since > kAdmitGiveUp) {
                    for (Request *r : E->queue) {
                        r->rc = TANG_ENOMEM;
                        r->next = r->n;
                        if (r->outstanding == 0) {
                            r->done = true;
                            r->done_s = t_now;
                        }
                    }
                    E->queue.clear();
                    E->refused_since = 0;
                    E->cv_done.notify_all();
                }
            }
        }
        // 6. bookkeeping of the delivered pieces; free their slots
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
                s->idle_since = t;
            }
            E->cv_done.notify_all();
            continue;  // a slot is free: look at the queue again at once
        }
        if (E->stop && E->queue.empty() && !any_busy) break;
        if (!launched.empty() || admitted_now) continue;
        // 7. sleep until a slot completes or the engine stops. An idle GPU takes new work at once;
        // while launches are in flight, requests arriving within a short window are batched into
        // one launch instead of one small launch each (many small concurrent kernels contend for
        // the SMs and lengthen every request's latency). After a refused admission the engine
        // waits for a slot to complete (its memory may then be reused) or retries within 1 ms.
        if (any_busy)
            E->cv_work.wait_for(lk, std::chrono::microseconds(refused_now ? 1000 : 100),
                                [&] { return E->slot_finished || E->stop; });
        else
            E->cv_work.wait_for(lk, std::chrono::milliseconds(refused_now ? 1 : 5),
                                [&] { return E->slot_finished || E->stop || (!refused_now && !E->queue.empty()); });
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
    if (cfg->max_batch == 0 || cfg->max_inflight == 0 || cfg->max_inflight > 64)
        return set_err(ctx, TANG_EINVAL, "serving needs 1-64 slots of at least one packet");
    cudaSetDevice(ctx->device);
    ServeEngine *E = new ServeEngine();
    E->ctx = ctx;
    E->cfg = *cfg;
    E->cfg.path = path;
    // A slot's device buffers are admitted when work needs them; one slot must fit the pool (or
    // the device) at all. Streams, events and pinned staging exist for every slot from the start.
    const size_t slot_bytes = (sizeof(tang_header) + sizeof(uint32_t)) * size_t(cfg->max_batch);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    if ((ctx->cap && slot_bytes > ctx->cap) || slot_bytes > total_b) {
        delete E;
        return set_err(ctx, TANG_ENOMEM, "a serving slot of %zu bytes does not fit the memory pool", slot_bytes);
    }
    E->slots.resize(cfg->max_inflight);
    for (auto &s : E->slots) {
        if (cudaMallocHost(reinterpret_cast<void **>(&s.p_h), sizeof(tang_header) * size_t(cfg->max_batch)) != cudaSuccess ||
            cudaMallocHost(reinterpret_cast<void **>(&s.p_ids), sizeof(uint32_t) * size_t(cfg->max_batch)) != cudaSuccess ||
            cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            for (auto &t : E->slots) {
                if (t.p_h) cudaFreeHost(t.p_h);
                if (t.p_ids) cudaFreeHost(t.p_ids);
                if (t.st) cudaStreamDestroy(t.st);
                if (t.ev) cudaEventDestroy(t.ev);
            }
            delete E;
            return set_err(ctx, TANG_ENOMEM, "pinned staging, streams or events for %u slots could not be created",
                           cfg->max_inflight);
        }
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

int tang_serve_info_get(tang_ctx *ctx, tang_serve_info *out) {
    if (!ctx || !out) return TANG_EINVAL;
    ServeEngine *E = ctx->serve;
    if (!E) return set_err(ctx, TANG_EINVAL, "serving engine not started");
    std::lock_guard<std::mutex> g(E->mu);
    out->slots_max = uint32_t(E->slots.size());
    out->slots_admitted = E->admitted;
    out->slots_admitted_peak = E->admitted_peak;
    uint32_t busy = 0;
    for (auto &s : E->slots) busy += s.busy;
    out->slots_busy = busy;
    out->admissions_refused = E->refusals;
    out->launches = E->launches;
    out->packets = E->packets;
    out->slot_bytes = (sizeof(tang_header) + sizeof(uint32_t)) * uint64_t(E->cfg.max_batch);
    out->queued = uint32_t(E->queue.size());
    out->reserved = 0;
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
        if (s.d_h) ctx_free(ctx, s.d_h);
        if (s.d_ids) ctx_free(ctx, s.d_ids);
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
