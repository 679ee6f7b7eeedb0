// The paper's CPU-GPU hybrid streaming framework (§5.1.2, Fig. 4), built as a comparison
// pipeline beside this library's all-GPU path. Headers are batched on the host and sent to the
// GPU; each batch is split into segments, one per CUDA stream, and the network alone runs on
// them (the tensor-core kernel without its search warps, or the FP32 kernels); the predicted
// tuples come back to pinned host memory, and a pool of host threads runs the tuple-space search
// while the GPU works on the next batch (two buffers, as the paper's double buffering). The
// search is this library's exact one (conflict sets) or, with TANG_SEARCH_PAPER, the paper's own
// post-verification; it reads a host snapshot of the device tables taken at the start of the
// call, so it probes exactly what the search kernels probe.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

using namespace tang;

namespace tang {
uint64_t fmix64_host(uint64_t k);
}

namespace {

// Host copy of one ruleset's device tables.
struct HostTables {
    std::vector<TupleDesc> tuples;
    std::vector<Slot> slots;
    std::vector<DRule> rules;
    std::vector<uint32_t> cwords;
    std::vector<uint16_t> order;
    uint32_t T = 0, cw = 1;
};

int snapshot(tang_ctx *ctx, const Ruleset &rs, HostTables &ht) {
    Tables d{};
    cudaStream_t st = ctx->stream;
    if (cudaMemcpyAsync(&d, rs.d_desc, sizeof(d), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return set_err(ctx, TANG_EDEVICE, "hybrid: reading the table descriptor failed");
    ht.T = d.T;
    ht.cw = d.cw;
    ht.tuples.resize(d.T);
    ht.order.resize(d.T);
    ht.rules.resize(d.pool_size);
    ht.slots.resize(rs.slot_capacity);
    ht.cwords.resize(d.cw > 1 ? size_t(rs.cword_rows) * d.cw : 0);
    cudaMemcpyAsync(ht.tuples.data(), d.tuples, sizeof(TupleDesc) * d.T, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(ht.order.data(), d.order, sizeof(uint16_t) * d.T, cudaMemcpyDeviceToHost, st);
    if (d.pool_size) cudaMemcpyAsync(ht.rules.data(), d.rules, sizeof(DRule) * d.pool_size, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(ht.slots.data(), d.slots, sizeof(Slot) * ht.slots.size(), cudaMemcpyDeviceToHost, st);
    if (!ht.cwords.empty())
        cudaMemcpyAsync(ht.cwords.data(), d.cwords, 4 * ht.cwords.size(), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "hybrid: table snapshot failed");
    return TANG_OK;
}

struct HBest {
    uint32_t prio, id, pos, tuple;
};
struct HCount {
    uint64_t packets = 0, matched = 0, nn_correct = 0, pred_hit = 0, fallback = 0, probes = 0, rule_reads = 0,
             slot_reads = 0;
};

inline bool h_beats(uint32_t prio, uint32_t id, const HBest &b) { return prio < b.prio || (prio == b.prio && id < b.id); }

inline bool h_match(const DRule &r, const tang_header &h) {
    const uint32_t m = r.meta;
    bool ok = ((h.sip ^ r.sip) & prefix_mask(meta_sip_len(m))) == 0;
    ok = ok && ((h.dip ^ r.dip) & prefix_mask(meta_dip_len(m))) == 0;
    ok = ok && h.sp >= (r.sp & 0xFFFFu) && h.sp <= (r.sp >> 16);
    ok = ok && h.dp >= (r.dp & 0xFFFFu) && h.dp <= (r.dp >> 16);
    return ok && (!meta_proto_exact(m) || h.proto == meta_proto(m));
}

// One tuple probe (§4.3 truncation, then the run under the key in (priority, id) order).
bool h_probe(const HostTables &ht, uint32_t t, const tang_header &h, HBest &best, HCount &c) {
    const TupleDesc &d = ht.tuples[t];
    const uint32_t ks = h.sip & d.mask_s, kd = h.dip & d.mask_d;
    const uint32_t start = uint32_t(fmix64_host((uint64_t(ks) << 32) | kd)) & d.slot_mask;
    for (uint32_t i = 0; i <= d.max_probe; ++i) {
        const Slot &s = ht.slots[d.slot_base + ((start + i) & d.slot_mask)];
        c.slot_reads++;
        if (s.start == kEmpty) return false;
        if (s.ks == ks && s.kd == kd) {
            for (uint32_t j = 0; j < s.len; ++j) {
                const DRule &r = ht.rules[s.start + j];
                c.rule_reads++;
                if (!h_beats(r.prio, r.id, best)) return false;
                if (h_match(r, h)) {
                    best = HBest{r.prio, r.id, s.start + j, t};
                    return true;
                }
            }
            return false;
        }
    }
    return false;
}

// The two-stage search of §5.1.1 on the host: predicted tuple first; then, exact, the tuples of
// the hit's conflict set or, after a miss, all tuples in ascending best (priority, id); in paper
// mode a hit ends the search.
uint32_t h_search(const HostTables &ht, const tang_header &h, int pred, bool paper, HCount &c) {
    HBest best{0xFFFFFFFFu, 0xFFFFFFFFu, kEmpty, 0};
    bool hit = false;
    if (uint32_t(pred) < ht.T) {
        c.probes++;
        hit = h_probe(ht, uint32_t(pred), h, best, c);
    }
    c.packets++;
    c.pred_hit += hit;
    c.fallback += !hit;
    if (!(hit && paper)) {
        const uint32_t *cfw = nullptr;
        uint32_t cf0 = 0;
        if (hit) {
            const uint32_t cf = ht.rules[best.pos].cf;
            if (ht.cw == 1)
                cf0 = cf;
            else
                cfw = ht.cwords.data() + size_t(cf) * ht.cw;
        }
        for (uint32_t k = 0; k < ht.T; ++k) {
            const uint32_t t = ht.order[k];
            if (int(t) == pred) continue;
            if (hit) {
                const uint32_t w = cfw ? cfw[t >> 5] : cf0;
                if (!((w >> (t & 31)) & 1u)) continue;
            }
            const TupleDesc &d = ht.tuples[t];
            if (!h_beats(d.min_prio, d.min_id, best)) break;
            c.probes++;
            h_probe(ht, t, h, best, c);
        }
    }
    if (best.id != 0xFFFFFFFFu) {
        c.matched++;
        c.nn_correct += int(best.tuple) == pred;
    }
    return best.id;
}

// Host threads that search one batch at a time, each a static slice of it.
class SearchPool {
  public:
    SearchPool(const HostTables &ht, unsigned n, bool paper) : ht_(ht), paper_(paper), counts_(n) {
        for (unsigned i = 0; i < n; ++i) threads_.emplace_back([this, i, n] { run(i, n); });
    }
    ~SearchPool() {
        {
            std::lock_guard<std::mutex> g(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto &t : threads_) t.join();
    }
    // Search headers[0..n) with predictions pred[0..n) into ids; returns when done.
    void search(const tang_header *headers, const int32_t *pred, uint32_t n, uint32_t *ids) {
        std::unique_lock<std::mutex> lk(mu_);
        h_ = headers;
        pred_ = pred;
        n_ = n;
        ids_ = ids;
        done_ = 0;
        ++gen_;
        cv_.notify_all();
        done_cv_.wait(lk, [&] { return done_ == threads_.size(); });
    }
    HCount total() const {
        HCount s;
        for (const HCount &c : counts_) {
            s.packets += c.packets;
            s.matched += c.matched;
            s.nn_correct += c.nn_correct;
            s.pred_hit += c.pred_hit;
            s.fallback += c.fallback;
            s.probes += c.probes;
            s.rule_reads += c.rule_reads;
            s.slot_reads += c.slot_reads;
        }
        return s;
    }

  private:
    void run(unsigned idx, unsigned n_threads) {
        uint64_t seen = 0;
        for (;;) {
            const tang_header *h;
            const int32_t *pred;
            uint32_t n;
            uint32_t *ids;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
                if (stop_) return;
                seen = gen_;
                h = h_;
                pred = pred_;
                n = n_;
                ids = ids_;
            }
            const uint32_t per = (n + n_threads - 1) / n_threads;
            const uint32_t b = std::min(n, idx * per), e = std::min(n, b + per);
            HCount &c = counts_[idx];
            for (uint32_t i = b; i < e; ++i) ids[i] = h_search(ht_, h[i], pred[i], paper_, c);
            {
                std::lock_guard<std::mutex> g(mu_);
                ++done_;
            }
            done_cv_.notify_one();
        }
    }
    const HostTables &ht_;
    const bool paper_;
    std::vector<HCount> counts_;
    std::vector<std::thread> threads_;
    std::mutex mu_;
    std::condition_variable cv_, done_cv_;
    uint64_t gen_ = 0;
    size_t done_ = 0;
    bool stop_ = false;
    const tang_header *h_ = nullptr;
    const int32_t *pred_ = nullptr;
    uint32_t n_ = 0;
    uint32_t *ids_ = nullptr;
};

}  // namespace

extern "C" int tang_classify_hybrid(tang_ctx *ctx, uint32_t rsh, const tang_header *headers, uint32_t n, uint32_t *ids,
                                    const tang_hybrid_cfg *cfg, tang_stats *stats) {
    const NvtxRange nvtx_range("tang_classify_hybrid");
    if (!ctx || !cfg) return set_err(ctx, TANG_EINVAL, "null argument");
    auto it = ctx->rulesets.find(rsh);
    if (it == ctx->rulesets.end()) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    Ruleset &rs = *it->second;
    if (n && (!headers || !ids)) return set_err(ctx, TANG_EINVAL, "null buffer");
    if (cfg->flags & ~uint32_t(TANG_SEARCH_PAPER)) return set_err(ctx, TANG_EINVAL, "unknown hybrid flags");
    const int prec = int(cfg->precision);
    if (prec != TANG_FP32 && prec != TANG_BF16 && prec != TANG_FP8) return set_err(ctx, TANG_EINVAL, "bad precision");
    if (!rs.model) return set_err(ctx, TANG_EINVAL, "ruleset %u has no model", rsh);
    if (prec != TANG_FP32 && !rs.model->d_wbf16) return set_err(ctx, TANG_EUNSUPPORTED, "no tensor-core copy of the model");
    if (prec == TANG_FP8 && !rs.model->has_fp8) return set_err(ctx, TANG_EINVAL, "FP8 needs a calibrated model");
    const uint32_t batch = cfg->batch ? cfg->batch : 8192;
    const uint32_t n_streams = std::max(1u, std::min(cfg->streams ? cfg->streams : 4u, 16u));
    const unsigned n_threads = cfg->threads ? cfg->threads : std::max(1u, std::thread::hardware_concurrency());
    if (batch > (1u << 24)) return set_err(ctx, TANG_EINVAL, "batch too large");
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (n == 0) return TANG_OK;
    cudaSetDevice(ctx->device);
    if (rs.has_update && cudaStreamWaitEvent(ctx->stream, rs.last_update, 0) != cudaSuccess)
        return set_err(ctx, TANG_EDEVICE, "hybrid: waiting for updates failed");
    HostTables ht;
    int rc = snapshot(ctx, rs, ht);
    if (rc) return rc;

    // two batch buffers on both sides; FP32 inference needs its own scratch per segment
    tang_header *dh = nullptr;
    int32_t *dt = nullptr;
    void *ph = nullptr, *pt = nullptr;
    if ((rc = ctx_alloc(ctx, 2 * size_t(batch) * sizeof(tang_header), (void **)&dh))) return rc;
    if ((rc = ctx_alloc(ctx, 2 * size_t(batch) * sizeof(int32_t), (void **)&dt))) {
        ctx_free(ctx, dh);
        return rc;
    }
    std::vector<cudaStream_t> streams(n_streams, nullptr);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    auto cleanup = [&]() {
        for (cudaStream_t s : streams)
            if (s) cudaStreamSynchronize(s);
        for (cudaStream_t s : streams)
            if (s) cudaStreamDestroy(s);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (ph) cudaFreeHost(ph);
        if (pt) cudaFreeHost(pt);
        ctx_free(ctx, dh);
        ctx_free(ctx, dt);
    };
    bool ok = cudaMallocHost(&ph, 2 * size_t(batch) * sizeof(tang_header)) == cudaSuccess &&
              cudaMallocHost(&pt, 2 * size_t(batch) * sizeof(int32_t)) == cudaSuccess;
    for (uint32_t s = 0; ok && s < n_streams; ++s) ok = cudaStreamCreateWithFlags(&streams[s], cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; ok && k < 2; ++k) ok = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming) == cudaSuccess;
    if (ok)  // the first segments must see the table and model state of the context stream
        for (uint32_t s = 0; ok && s < n_streams; ++s) {
            cudaEvent_t e;
            ok = cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventRecord(e, ctx->stream) == cudaSuccess && cudaStreamWaitEvent(streams[s], e, 0) == cudaSuccess;
            cudaEventDestroy(e);
        }
    if (!ok) {
        cleanup();
        return set_err(ctx, TANG_EDEVICE, "hybrid: pinned buffers, streams or events could not be created");
    }
    tang_header *host_h = static_cast<tang_header *>(ph);
    int32_t *host_t = static_cast<int32_t *>(pt);
    const bool paper = (cfg->flags & TANG_SEARCH_PAPER) != 0;
    const TuneEntry *tune = nullptr;
    {
        SearchPool pool(ht, n_threads, paper);
        const uint32_t nb = (n + batch - 1) / batch;
        // GPU side of batch b into buffer b & 1: per segment H2D, the network, D2H of predictions
        auto gpu_batch = [&](uint32_t b) -> int {
            const uint32_t k = b & 1, b0 = b * batch, rows = std::min(batch, n - b0);
            std::memcpy(host_h + size_t(k) * batch, headers + b0, sizeof(tang_header) * rows);
            const uint32_t seg = (rows + n_streams - 1) / n_streams;
            for (uint32_t s = 0; s < n_streams; ++s) {
                const uint32_t s0 = s * seg, sr = s0 < rows ? std::min(seg, rows - s0) : 0;
                if (!sr) continue;
                tang_header *d_seg = dh + size_t(k) * batch + s0;
                int32_t *t_seg = dt + size_t(k) * batch + s0;
                // the FP32 kernels share the context's scratch buffer: their segments run in order
                // on one stream; the tensor-core kernel keeps its state on chip and overlaps
                cudaStream_t sst = prec == TANG_FP32 ? streams[0] : streams[s];
                cudaMemcpyAsync(d_seg, host_h + size_t(k) * batch + s0, sizeof(tang_header) * sr, cudaMemcpyHostToDevice,
                                sst);
                int r = prec == TANG_FP32 ? mlp_fp32_forward(ctx, *rs.model, d_seg, sr, nullptr, t_seg, sst)
                                          : tc_launch(ctx, rs, d_seg, sr, nullptr, nullptr, t_seg, prec, false, nullptr,
                                                      sst, tune, 0);
                if (r) return r;
                cudaMemcpyAsync(host_t + size_t(k) * batch + s0, t_seg, sizeof(int32_t) * sr, cudaMemcpyDeviceToHost, sst);
            }
            // the batch is complete when every stream has finished its segment
            for (uint32_t s = 1; s < n_streams; ++s) {
                cudaEvent_t e;
                cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
                cudaEventRecord(e, streams[s]);
                cudaStreamWaitEvent(streams[0], e, 0);
                cudaEventDestroy(e);
            }
            cudaEventRecord(ev[k], streams[0]);
            return TANG_OK;
        };
        auto cpu_batch = [&](uint32_t b) {
            const uint32_t k = b & 1, b0 = b * batch, rows = std::min(batch, n - b0);
            cudaEventSynchronize(ev[k]);
            pool.search(host_h + size_t(k) * batch, host_t + size_t(k) * batch, rows, ids + b0);
        };
        for (uint32_t b = 0; b < nb && rc == TANG_OK; ++b) {
            // the GPU takes batch b while the host threads search batch b - 1
            rc = gpu_batch(b);
            if (rc == TANG_OK && b > 0) cpu_batch(b - 1);
        }
        if (rc == TANG_OK) cpu_batch(nb - 1);
        if (stats && rc == TANG_OK) {
            const HCount c = pool.total();
            stats->packets = c.packets;
            stats->matched = c.matched;
            stats->nn_correct = c.nn_correct;
            stats->pred_hit = c.pred_hit;
            stats->fallback = c.fallback;
            stats->probes = c.probes;
            stats->rule_reads = c.rule_reads;
            stats->slot_reads = c.slot_reads;
        }
    }
    cleanup();
    if (rc) return rc;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "hybrid pipeline: %s", cudaGetErrorString(e));
    return TANG_OK;
}
