// C-ABI entry points: context and memory admission, rulesets, models, classification
// (device-resident, graph-replayed, or host-streamed through pinned buffers), updates.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace tang {

int set_err(tang_ctx *ctx, int code, const char *fmt, ...) {
    if (!ctx) return code;
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
    return code;
}

int ctx_alloc(tang_ctx *ctx, size_t bytes, void **p) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    std::lock_guard<std::mutex> g(ctx->alloc_mu);
    if (ctx->cap && ctx->used + bytes > ctx->cap)
        return set_err(ctx, TANG_ENOMEM, "memory pool: %zu bytes requested, %zu of %zu in use", bytes, ctx->used,
                       ctx->cap);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_err(ctx, TANG_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    ctx->allocs[*p] = bytes;
    ctx->used += bytes;
    return TANG_OK;
}

int ctx_try_alloc(tang_ctx *ctx, size_t bytes, void **p) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    std::lock_guard<std::mutex> g(ctx->alloc_mu);
    if (ctx->cap && ctx->used + bytes > ctx->cap) return TANG_ENOMEM;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return TANG_ENOMEM;
    }
    ctx->allocs[*p] = bytes;
    ctx->used += bytes;
    return TANG_OK;
}

void ctx_free(tang_ctx *ctx, void *p) {
    if (!p) return;
    std::lock_guard<std::mutex> g(ctx->alloc_mu);
    auto it = ctx->allocs.find(p);
    if (it != ctx->allocs.end()) {
        ctx->used -= it->second;
        ctx->allocs.erase(it);
    }
    cudaFree(p);
}

static void drop_graphs(tang_ctx *ctx) {
    for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
    ctx->graphs.clear();
}

int ensure_scratch(tang_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->scratch_bytes) return TANG_OK;
    cudaDeviceSynchronize();
    drop_graphs(ctx);  // graphs captured the old scratch address
    ctx_free(ctx, ctx->scratch);
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
    int rc = ctx_alloc(ctx, bytes, &ctx->scratch);
    if (rc) return rc;
    ctx->scratch_bytes = bytes;
    return TANG_OK;
}

bool GraphKey::operator<(const GraphKey &o) const {
    if (rs != o.rs) return rs < o.rs;
    if (path != o.path) return path < o.path;
    if (n != o.n) return n < o.n;
    if (h != o.h) return h < o.h;
    if (ids != o.ids) return ids < o.ids;
    return stream < o.stream;
}

}  // namespace tang

using namespace tang;

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// After a synchronisation point: report (and clear) error bits set by bounded device waits.
int tang::check_device_error(tang_ctx *ctx) {
    int bits = 0;
    if (cudaMemcpy(&bits, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return set_err(ctx, TANG_EDEVICE, "reading the device error word failed");
    if (bits) {
        cudaMemset(ctx->d_err, 0, sizeof(int));
        if (bits & kErrIndex)
            return set_err(ctx, TANG_EDEVICE, "a table index was out of range; the access was skipped (checked build, "
                                              "error bits 0x%x)", bits);
        return set_err(ctx, TANG_ETIMEOUT, "a device wait ran out of time (error bits 0x%x)", bits);
    }
    return TANG_OK;
}

// Search mode bits requested by TANG_SEARCH_* flags.
int tang::search_mode_of(uint32_t flags) {
    return ((flags & TANG_SEARCH_PAPER) ? kSearchPaper : 0) | ((flags & TANG_SEARCH_SERIAL) ? kSearchSerial : 0);
}

// Kernel variant requested by flag bits: 5 = the N=256 fused kernel on one SM, 6 = on CTA pairs,
// 7 = network and search as two kernels (fused paths), 0 = tuned or library default.
static int variant_of(uint32_t flags) {
    if ((flags & TANG_VARIANT_MASK) == TANG_FUSED_SPLIT) return kVariantSplit;
    if (flags & TANG_FUSED_PAIR) return 6;
    if (flags & TANG_FUSED_N256) return 5;
    return 0;
}

static Ruleset *find_rs(tang_ctx *ctx, uint32_t rs) {
    auto it = ctx->rulesets.find(rs);
    return it == ctx->rulesets.end() ? nullptr : it->second.get();
}

// Checked builds synchronise after every classify and search call (unless the stream is being
// captured) and report the device error word, so that an index found out of range surfaces at the
// call that formed it; other builds check it at the calls that synchronise anyway.
int tang::checked_sync(tang_ctx *ctx, cudaStream_t st) {
#ifdef TANG_CHECKED
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
        if (cudaStreamSynchronize(st) != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "stream synchronise failed");
        return check_device_error(ctx);
    }
#else
    (void)ctx;
    (void)st;
#endif
    return TANG_OK;
}

void tang::note_classify(Ruleset &rs, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return;  // work captured into a graph runs when the graph is launched, under the caller's ordering
    }
    std::lock_guard<std::mutex> g(rs.inflight_mu);
    for (auto &e : rs.inflight)
        if (e.first == st) {
            cudaEventRecord(e.second, st);
            return;
        }
    if (rs.inflight.size() >= 16) {
        // forget streams whose last classification has completed
        std::vector<std::pair<cudaStream_t, cudaEvent_t>> keep;
        for (auto &e : rs.inflight) {
            if (cudaEventQuery(e.second) == cudaSuccess)
                cudaEventDestroy(e.second);
            else
                keep.push_back(e);
        }
        cudaGetLastError();
        rs.inflight.swap(keep);
    }
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        // no event: fall back to waiting here, so an update can never overtake this classification
        cudaGetLastError();
        cudaStreamSynchronize(st);
        return;
    }
    cudaEventRecord(ev, st);
    rs.inflight.emplace_back(st, ev);
}

int tang::wait_classifies(tang_ctx *ctx, Ruleset &rs, cudaStream_t st) {
    std::lock_guard<std::mutex> g(rs.inflight_mu);
    for (auto &e : rs.inflight) CK(cudaStreamWaitEvent(st, e.second, 0));
    return TANG_OK;
}

static void free_inflight(Ruleset &rs) {
    std::lock_guard<std::mutex> g(rs.inflight_mu);
    for (auto &e : rs.inflight) cudaEventDestroy(e.second);
    rs.inflight.clear();
}

int tang_checked_build(void) {
#ifdef TANG_CHECKED
    return 1;
#else
    return 0;
#endif
}

int tang_debug_set_pool_view(tang_ctx *ctx, uint32_t rsh, uint32_t n) {
    if (!ctx) return TANG_EINVAL;
    Ruleset *rs = find_rs(ctx, rsh);
    if (!rs) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    cudaSetDevice(ctx->device);
    return tss_set_pool_view(ctx, *rs, n);
}

extern "C" {

int tang_create(int device, size_t pool_bytes, tang_ctx **out) {
    if (!out) return TANG_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return TANG_EDEVICE;
    }
    tang_ctx *ctx = new tang_ctx();
    ctx->device = device;
    ctx->cap = pool_bytes;
    if (cudaSetDevice(device) != cudaSuccess) {
        delete ctx;
        return TANG_EDEVICE;
    }
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->copy_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->copy_out, cudaStreamNonBlocking) != cudaSuccess) {
        delete ctx;
        return TANG_EDEVICE;
    }
    if (ctx_alloc(ctx, sizeof(DevStats), (void **)&ctx->d_stats) != TANG_OK ||
        ctx_alloc(ctx, sizeof(int), (void **)&ctx->d_err) != TANG_OK || cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess) {
        tang_destroy(ctx);
        return TANG_ENOMEM;
    }
    if (noalloc_prepare(ctx) != TANG_OK) {
        tang_destroy(ctx);
        return TANG_EDEVICE;
    }
    *out = ctx;
    return TANG_OK;
}

int tang_serve_stop(tang_ctx *ctx);
void tang_model_free(tang_ctx *ctx, DeviceModel *m);

void tang_destroy(tang_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    tang_serve_stop(ctx);
    cudaDeviceSynchronize();
    drop_graphs(ctx);
    for (auto &kv : ctx->rulesets) {
        tss_free(ctx, *kv.second);
        if (kv.second->model) tang_model_free(ctx, kv.second->model.get());
        if (kv.second->last_update) cudaEventDestroy(kv.second->last_update);
        free_inflight(*kv.second);
    }
    ctx->rulesets.clear();
    ctx_free(ctx, ctx->scratch);
    ctx_free(ctx, ctx->d_stats);
    ctx_free(ctx, ctx->d_err);
    ctx_free(ctx, ctx->dev_h);
    ctx_free(ctx, ctx->dev_ids);
    if (ctx->pinned_h) cudaFreeHost(ctx->pinned_h);
    if (ctx->pinned_ids) cudaFreeHost(ctx->pinned_ids);
    for (auto &kv : std::unordered_map<void *, size_t>(ctx->allocs)) cudaFree(kv.first);
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    if (ctx->copy_in) cudaStreamDestroy(ctx->copy_in);
    if (ctx->copy_out) cudaStreamDestroy(ctx->copy_out);
    delete ctx;
}

const char *tang_last_error(tang_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int tang_memory_usage(tang_ctx *ctx, size_t *used, size_t *cap) {
    if (!ctx) return TANG_EINVAL;
    std::lock_guard<std::mutex> g(ctx->alloc_mu);
    if (used) *used = ctx->used;
    if (cap) *cap = ctx->cap;
    return TANG_OK;
}

int tang_load_ruleset(tang_ctx *ctx, const tang_rule *rules, uint32_t n, uint32_t *rs_out) {
    const NvtxRange nvtx_range("tang_load_ruleset");
    if (!ctx || !rs_out || (n && !rules)) return set_err(ctx, TANG_EINVAL, "null argument");
    cudaSetDevice(ctx->device);
    auto t0 = std::chrono::steady_clock::now();
    std::unique_ptr<Ruleset> rs(new Ruleset());
    int rc = tss_build(ctx, *rs, rules, n);
    if (rc) return rc;
    rc = tss_upload(ctx, *rs, ctx->stream);
    if (rc) {
        tss_free(ctx, *rs);
        return rc;
    }
    CK(cudaEventCreateWithFlags(&rs->last_update, cudaEventDisableTiming));
    rs->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    rs->handle = ctx->next_rs++;
    *rs_out = rs->handle;
    ctx->rulesets[rs->handle] = std::move(rs);
    return TANG_OK;
}

int tang_unload_ruleset(tang_ctx *ctx, uint32_t rsh) {
    if (!ctx) return TANG_EINVAL;
    Ruleset *rs = find_rs(ctx, rsh);
    if (!rs) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    drop_graphs(ctx);
    tss_free(ctx, *rs);
    if (rs->model) tang_model_free(ctx, rs->model.get());
    if (rs->last_update) cudaEventDestroy(rs->last_update);
    free_inflight(*rs);
    ctx->rulesets.erase(rsh);
    return TANG_OK;
}

int tang_ruleset_info_get(tang_ctx *ctx, uint32_t rsh, tang_ruleset_info *out) {
    if (!ctx || !out) return TANG_EINVAL;
    Ruleset *rs = find_rs(ctx, rsh);
    if (!rs) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    out->n_rules = rs->host.live;
    out->n_tuples = uint32_t(rs->host.tuples.size());
    out->conflict_words = rs->host.cw;
    uint32_t keys = 0;
    for (auto &t : rs->host.tuples) keys += t.n_keys;
    out->n_keys = keys;
    out->device_bytes = uint64_t(sizeof(TupleDesc)) * kMaxTuples + uint64_t(sizeof(Slot)) * rs->slot_capacity +
                        uint64_t(sizeof(DRule)) * rs->rule_capacity + uint64_t(4) * rs->cword_capacity +
                        2 * kMaxTuples + sizeof(Tables);
    out->build_ms = rs->build_ms;
    return TANG_OK;
}

int tang_tuple_get(tang_ctx *ctx, uint32_t rsh, uint32_t t, uint32_t *sl, uint32_t *dl, uint32_t *mp, uint32_t *mi) {
    if (!ctx) return TANG_EINVAL;
    Ruleset *rs = find_rs(ctx, rsh);
    if (!rs) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    if (t >= rs->host.tuples.size()) return set_err(ctx, TANG_EINVAL, "tuple %u out of range", t);
    const HostTuple &h = rs->host.tuples[t];
    if (sl) *sl = h.ls;
    if (dl) *dl = h.ld;
    if (mp) *mp = h.min_prio;
    if (mi) *mi = h.min_id;
    return TANG_OK;
}

int tang_rule_conflicts(tang_ctx *ctx, uint32_t rsh, uint32_t id, uint32_t *tuple, uint32_t *words) {
    if (!ctx) return TANG_EINVAL;
    Ruleset *rs = find_rs(ctx, rsh);
    if (!rs) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    auto it = rs->host.pos_of_id.find(id);
    if (it == rs->host.pos_of_id.end()) return set_err(ctx, TANG_ENOTFOUND, "rule id %u is not live", id);
    cudaSetDevice(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream));
    DRule r;
    CK(cudaMemcpy(&r, rs->d_rules + it->second, sizeof(DRule), cudaMemcpyDeviceToHost));
    if (tuple) *tuple = meta_tuple(r.meta);
    if (words) {
        if (rs->host.cw == 1)
            words[0] = r.cf;
        else
            CK(cudaMemcpy(words, rs->d_cwords + size_t(r.cf) * rs->host.cw, 4 * rs->host.cw, cudaMemcpyDeviceToHost));
    }
    return TANG_OK;
}

// ---------------------------------------------------------------------------------------
// Model
// ---------------------------------------------------------------------------------------
void tang_model_free(tang_ctx *ctx, DeviceModel *m) {
    ctx_free(ctx, m->d_params);
    ctx_free(ctx, m->d_wbf16);
    ctx_free(ctx, m->d_wfp8);
    ctx_free(ctx, m->d_wscale8);
    ctx_free(ctx, m->d_bias_tc);
    ctx_free(ctx, m->d_fold8);
    ctx_free(ctx, m->d_l0);
    free(m->tmap256);
    m->d_params = nullptr;
}

// Bytes of a buffer allocated through ctx_alloc (0 if unknown or null).
static size_t alloc_size(tang_ctx *ctx, const void *p) {
    if (!p) return 0;
    std::lock_guard<std::mutex> g(ctx->alloc_mu);
    auto it = ctx->allocs.find(const_cast<void *>(p));
    return it == ctx->allocs.end() ? 0 : it->second;
}

static int check_cuda(tang_ctx *ctx, const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "%s: %s", what, cudaGetErrorString(e));
    return TANG_OK;
}

// Hot swap of a model between graph replays: when the new model has the live one's shape and
// buffer set, its device copies are written over the live buffers, so every pointer and tensor
// map that launches (and captured CUDA graphs) hold stays valid. All device work is drained
// first, so no kernel reads a half-written model. Returns false (nothing changed) otherwise.
static bool swap_in_place(tang_ctx *ctx, DeviceModel &live, const DeviceModel &next) {
    if (live.S != next.S || live.N != next.N || live.blocks != next.blocks || live.C != next.C ||
        live.Cpad != next.Cpad || live.has_fp8 != next.has_fp8)
        return false;
    const void *dst[] = {live.d_params, live.d_wbf16, live.d_wfp8, live.d_wscale8, live.d_bias_tc, live.d_fold8, live.d_l0};
    const void *src[] = {next.d_params, next.d_wbf16, next.d_wfp8, next.d_wscale8, next.d_bias_tc, next.d_fold8, next.d_l0};
    for (int k = 0; k < 7; ++k)
        if ((dst[k] == nullptr) != (src[k] == nullptr) || alloc_size(ctx, dst[k]) != alloc_size(ctx, src[k])) return false;
    cudaDeviceSynchronize();
    for (int k = 0; k < 7; ++k)
        if (dst[k]) cudaMemcpyAsync(const_cast<void *>(dst[k]), src[k], alloc_size(ctx, src[k]), cudaMemcpyDeviceToDevice,
                                    ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    live.host_params = next.host_params;
    std::memcpy(live.act_amax, next.act_amax, sizeof(live.act_amax));
    std::memcpy(live.act_scale, next.act_scale, sizeof(live.act_scale));
    return true;
}

int tang_load_model(tang_ctx *ctx, uint32_t rsh, const void *blob, size_t bytes) {
    const NvtxRange nvtx_range("tang_load_model");
    if (!ctx || !blob) return set_err(ctx, TANG_EINVAL, "null argument");
    Ruleset *rs = find_rs(ctx, rsh);
    if (!rs) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    if (bytes < sizeof(tang_model_header)) return set_err(ctx, TANG_EINVAL, "model blob too small");
    tang_model_header hd;
    std::memcpy(&hd, blob, sizeof(hd));
    if (hd.magic != TANG_MODEL_MAGIC || hd.version != 1) return set_err(ctx, TANG_EINVAL, "bad model magic/version");
    const uint32_t T = uint32_t(rs->host.tuples.size());
    if (hd.S != 7) return set_err(ctx, TANG_EINVAL, "model input width %u != 7", hd.S);
    if (hd.C != T) return set_err(ctx, TANG_EINVAL, "model classes %u != ruleset tuples %u", hd.C, T);
    if (hd.N == 0 || hd.N > 4096 || hd.blocks > 31) return set_err(ctx, TANG_EINVAL, "unsupported model shape");
    const size_t n_amax = 2 * size_t(hd.blocks) + 1;
    const size_t n_params = size_t(hd.S) * hd.N + hd.N + size_t(hd.blocks) * (2 * size_t(hd.N) * hd.N + 2 * hd.N) +
                            size_t(hd.N) * hd.C + hd.C;
    const size_t want = sizeof(hd) + 4 * n_amax + 4 * n_params;
    if (bytes != want) return set_err(ctx, TANG_EINVAL, "model blob has %zu bytes, expected %zu", bytes, want);
    cudaSetDevice(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream));
    std::unique_ptr<DeviceModel> m(new DeviceModel());
    m->S = hd.S;
    m->N = hd.N;
    m->blocks = hd.blocks;
    m->C = hd.C;
    m->Cpad = std::max<uint32_t>(32, (hd.C + 31) / 32 * 32);
    const float *amax = reinterpret_cast<const float *>(static_cast<const uint8_t *>(blob) + sizeof(hd));
    bool calibrated = true;
    for (size_t i = 0; i < n_amax; ++i) {
        m->act_amax[i] = amax[i];
        if (!(amax[i] > 0.f) || !std::isfinite(amax[i])) calibrated = false;
    }
    m->has_fp8 = calibrated;
    m->host_params.resize(n_params);
    std::memcpy(m->host_params.data(), amax + n_amax, 4 * n_params);
    for (float v : m->host_params)
        if (!std::isfinite(v)) return set_err(ctx, TANG_EINVAL, "model blob holds a non-finite parameter");
    int rc = ctx_alloc(ctx, 4 * n_params, (void **)&m->d_params);
    if (rc) return rc;
    CK(cudaMemcpy(m->d_params, m->host_params.data(), 4 * n_params, cudaMemcpyHostToDevice));
    const float *p = m->d_params;
    const uint32_t N = hd.N;
    m->W0 = p;
    p += size_t(hd.S) * N;
    m->b0 = p;
    p += N;
    for (uint32_t b = 0; b < hd.blocks; ++b) {
        m->W1.push_back(p);
        p += size_t(N) * N;
        m->b1.push_back(p);
        p += N;
        m->W2.push_back(p);
        p += size_t(N) * N;
        m->b2.push_back(p);
        p += N;
    }
    m->Wc = p;
    p += size_t(N) * hd.C;
    m->bc = p;
    if (N == 512 || N == 256) {  // tensor-core copies (tc_prepare_model checks the remaining limits)
        rc = tc_prepare_model(ctx, *m);
        if (rc) {
            tang_model_free(ctx, m.get());
            return rc;
        }
    }
    if (rs->model && swap_in_place(ctx, *rs->model, *m)) {
        // the live buffers now hold the new weights; the staging copy goes
        tang_model_free(ctx, m.get());
        return check_cuda(ctx, "model swap");
    }
    cudaDeviceSynchronize();
    drop_graphs(ctx);  // graphs captured the old model's buffers
    if (rs->model) tang_model_free(ctx, rs->model.get());
    rs->model = std::move(m);
    return TANG_OK;
}

// ---------------------------------------------------------------------------------------
// Classification
// ---------------------------------------------------------------------------------------
static int run_infer(tang_ctx *ctx, Ruleset &rs, const tang_header *h, uint32_t n, float *logits, int32_t *tuple,
                     int precision, cudaStream_t st, int variant = 0) {
    if (!rs.model) return set_err(ctx, TANG_EINVAL, "ruleset %u has no model", rs.handle);
    if (precision == TANG_FP32) return mlp_fp32_forward(ctx, *rs.model, h, n, logits, tuple, st);
    if (!rs.model->d_wbf16) return set_err(ctx, TANG_EUNSUPPORTED, "tensor-core path needs N == 256 or 512 and 1 <= blocks <= 31");
    if (precision == TANG_FP8 && !rs.model->has_fp8)
        return set_err(ctx, TANG_EINVAL, "FP8 path needs a calibrated model (act_amax)");
    const TuneEntry *tune = nullptr;
    auto it = rs.tune.find(precision == TANG_FP8 ? TANG_PATH_STAGED_FP8 : TANG_PATH_STAGED_BF16);
    if (it != rs.tune.end()) tune = &it->second;
    return tc_launch(ctx, rs, h, n, nullptr, logits, tuple, precision, false, nullptr, st, tune, variant);
}

// Enqueue the device-resident classification of one batch on `st` (no synchronisation).
static int enqueue_classify(tang_ctx *ctx, Ruleset &rs, const tang_header *h, uint32_t n, uint32_t *ids,
                            uint32_t path, DevStats *stats, cudaStream_t st, int variant = 0, int smode = 0) {
    if (n == 0) return TANG_OK;
    const int cw = int(rs.host.cw);
    const TuneEntry *tune = nullptr;
    auto it = rs.tune.find(path);
    if (it != rs.tune.end()) tune = &it->second;
    switch (path) {
        case TANG_PATH_NO_NN: {
            cudaError_t e = launch_search(rs.d_desc, uint32_t(rs.host.tuples.size()), cw, h, nullptr, n, ids, stats,
                                          tune, st, smode);
            if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "search: %s", cudaGetErrorString(e));
            return TANG_OK;
        }
        case TANG_PATH_PLAIN_FP32:
        case TANG_PATH_STAGED_BF16:
        case TANG_PATH_STAGED_FP8: {
            if (!rs.model) return set_err(ctx, TANG_EINVAL, "ruleset %u has no model", rs.handle);
            const int prec = path == TANG_PATH_PLAIN_FP32 ? TANG_FP32 : path == TANG_PATH_STAGED_BF16 ? TANG_BF16 : TANG_FP8;
            // the predicted tuples live after the network's own scratch
            const uint32_t chunk = 1u << 22;
            for (uint32_t c0 = 0; c0 < n; c0 += chunk) {
                const uint32_t rows = std::min(chunk, n - c0);
                const size_t fwd = prec == TANG_FP32
                                       ? size_t((std::min<uint32_t>(rows, 262144) + 127) / 128 * 128) *
                                             (8 + 2 * rs.model->N + rs.model->C) * sizeof(float)
                                       : 0;
                const size_t off = (fwd + 255) / 256 * 256;
                int rc = ensure_scratch(ctx, off + size_t(chunk) * sizeof(int32_t));
                if (rc) return rc;
                int32_t *tup = reinterpret_cast<int32_t *>(static_cast<uint8_t *>(ctx->scratch) + off);
                rc = run_infer(ctx, rs, h + c0, rows, nullptr, tup, prec, st, variant);
                if (rc) return rc;
                cudaError_t e = launch_search(rs.d_desc, uint32_t(rs.host.tuples.size()), cw, h + c0, tup, rows,
                                              ids + c0, stats, tune, st, smode);
                if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "search: %s", cudaGetErrorString(e));
            }
            return TANG_OK;
        }
        case TANG_PATH_FUSED_BF16:
        case TANG_PATH_FUSED_FP8: {
            if (!rs.model) return set_err(ctx, TANG_EINVAL, "ruleset %u has no model", rs.handle);
            if (!rs.model->d_wbf16) return set_err(ctx, TANG_EUNSUPPORTED, "tensor-core path needs N == 256 or 512 and 1 <= blocks <= 31");
            const int prec = path == TANG_PATH_FUSED_BF16 ? TANG_BF16 : TANG_FP8;
            if (prec == TANG_FP8 && !rs.model->has_fp8)
                return set_err(ctx, TANG_EINVAL, "FP8 path needs a calibrated model (act_amax)");
            if ((variant ? variant : tune ? tune->fused_variant : 0) == kVariantSplit) {
                // the network kernel leaves each packet's predicted tuple in ids; the search kernel
                // reads it there and overwrites it with the rule id (no scratch memory)
                int rc = tc_launch(ctx, rs, h, n, nullptr, nullptr, reinterpret_cast<int32_t *>(ids), prec, false,
                                   nullptr, st, nullptr, 0);
                if (rc) return rc;
                cudaError_t e = launch_search(rs.d_desc, uint32_t(rs.host.tuples.size()), cw, h, nullptr, n, ids,
                                              stats, nullptr, st, smode | kSearchPredInIds);
                if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "search: %s", cudaGetErrorString(e));
                return TANG_OK;
            }
            return tc_launch(ctx, rs, h, n, ids, nullptr, nullptr, prec, true, stats, st, tune, variant, smode);
        }
        default:
            return set_err(ctx, TANG_EINVAL, "unknown path %u", path);
    }
}

static int classify_host(tang_ctx *ctx, Ruleset &rs, const tang_header *h, uint32_t n, uint32_t *ids, uint32_t path,
                         DevStats *stats, int variant, int smode);


int tang_classify(tang_ctx *ctx, uint32_t rsh, const tang_header *headers, uint32_t n, uint32_t *ids, uint32_t flags,
                  void *stream, tang_stats *stats) {
    const NvtxRange nvtx_range("tang_classify");
    if (!ctx) return TANG_EINVAL;
    Ruleset *rs = find_rs(ctx, rsh);
    if (!rs) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    if (n && (!headers || !ids)) return set_err(ctx, TANG_EINVAL, "null buffer");
    if ((reinterpret_cast<uintptr_t>(headers) & 15) || (reinterpret_cast<uintptr_t>(ids) & 3))
        return set_err(ctx, TANG_EINVAL, "headers must be 16-byte aligned and ids 4-byte aligned");
    const uint32_t path = flags & TANG_PATH_MASK;
    const int variant = variant_of(flags);
    const int smode = search_mode_of(flags);
    cudaSetDevice(ctx->device);
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
    DevStats *dst = stats ? ctx->d_stats : nullptr;
    if (dst) CK(cudaMemsetAsync(dst, 0, sizeof(DevStats), st));
    int rc;
    if (flags & TANG_MEM_HOST) {
        rc = classify_host(ctx, *rs, headers, n, ids, path, dst, variant, smode);
    } else {
        if (rs->has_update) CK(cudaStreamWaitEvent(st, rs->last_update, 0));
        if ((flags & TANG_GRAPH) && !dst && n) {
            GraphKey key{rsh, path | uint32_t(variant) << 8 | uint32_t(smode) << 16, n, headers, ids, (void *)st};
            auto it = ctx->graphs.find(key);
            if (it == ctx->graphs.end()) {
                // First call for this key: run eagerly (this sizes any scratch, so nothing
                // allocates or synchronises inside the capture), then capture for later calls.
                rc = enqueue_classify(ctx, *rs, headers, n, ids, path, nullptr, st, variant, smode);
                if (rc) return rc;
                CK(cudaStreamSynchronize(st));
                // capture on a private stream so the caller's stream may be the legacy one
                cudaStream_t cap;
                CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
                CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
                rc = enqueue_classify(ctx, *rs, headers, n, ids, path, nullptr, cap, variant, smode);
                cudaGraph_t g = nullptr;
                cudaError_t e = cudaStreamEndCapture(cap, &g);
                cudaStreamDestroy(cap);
                if (rc) {
                    if (g) cudaGraphDestroy(g);
                    return rc;
                }
                if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "graph capture: %s", cudaGetErrorString(e));
                cudaGraphExec_t ex = nullptr;
                e = cudaGraphInstantiate(&ex, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "graph instantiate: %s", cudaGetErrorString(e));
                ctx->graphs.emplace(key, ex);
            } else {
                CK(cudaGraphLaunch(it->second, st));
            }
            rc = TANG_OK;
        } else {
            rc = enqueue_classify(ctx, *rs, headers, n, ids, path, dst, st, variant, smode);
        }
        if (rc == TANG_OK && n) note_classify(*rs, st);
    }
    if (rc) return rc;
    if (stats) {
        DevStats hs;
        CK(cudaMemcpyAsync(&hs, dst, sizeof(hs), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        stats->packets = hs.packets;
        stats->matched = hs.matched;
        stats->nn_correct = hs.nn_correct;
        stats->pred_hit = hs.pred_hit;
        stats->fallback = hs.fallback;
        stats->probes = hs.probes;
        stats->rule_reads = hs.rule_reads;
        stats->slot_reads = hs.slot_reads;
    }
    if (stats || (flags & TANG_MEM_HOST)) return check_device_error(ctx);
    return checked_sync(ctx, st);
}

// Host-streamed classification: chunks flow H2D (copy_in stream) -> compute (ctx stream) ->
// D2H (copy_out stream) through two device buffers, so copies of one chunk overlap the
// compute of the next. Pageable user buffers are staged through pinned buffers by this thread.
static int classify_host(tang_ctx *ctx, Ruleset &rs, const tang_header *h, uint32_t n, uint32_t *ids, uint32_t path,
                         DevStats *stats, int variant, int smode) {
    if (n == 0) return TANG_OK;
    const uint32_t chunk = std::min<uint32_t>(n, 1u << 20);
    if (ctx->dev_pkts < chunk) {
        cudaDeviceSynchronize();
        ctx_free(ctx, ctx->dev_h);
        ctx_free(ctx, ctx->dev_ids);
        ctx->dev_h = ctx->dev_ids = nullptr;
        ctx->dev_pkts = 0;
        int rc = ctx_alloc(ctx, 2 * size_t(chunk) * sizeof(tang_header), &ctx->dev_h);
        if (!rc) rc = ctx_alloc(ctx, 2 * size_t(chunk) * sizeof(uint32_t), &ctx->dev_ids);
        if (rc) return rc;
        ctx->dev_pkts = chunk;
    }
    cudaPointerAttributes ah{}, ai{};
    bool pinned = cudaPointerGetAttributes(&ah, h) == cudaSuccess && ah.type == cudaMemoryTypeHost &&
                  cudaPointerGetAttributes(&ai, ids) == cudaSuccess && ai.type == cudaMemoryTypeHost;
    cudaGetLastError();
    if (!pinned && ctx->pinned_pkts < chunk) {
        if (ctx->pinned_h) cudaFreeHost(ctx->pinned_h);
        if (ctx->pinned_ids) cudaFreeHost(ctx->pinned_ids);
        ctx->pinned_h = ctx->pinned_ids = nullptr;
        ctx->pinned_pkts = 0;
        CK(cudaMallocHost(&ctx->pinned_h, 2 * size_t(chunk) * sizeof(tang_header)));
        CK(cudaMallocHost(&ctx->pinned_ids, 2 * size_t(chunk) * sizeof(uint32_t)));
        ctx->pinned_pkts = chunk;
    }
    tang_header *dh = static_cast<tang_header *>(ctx->dev_h);
    uint32_t *di = static_cast<uint32_t *>(ctx->dev_ids);
    tang_header *ph = static_cast<tang_header *>(ctx->pinned_h);
    uint32_t *pi = static_cast<uint32_t *>(ctx->pinned_ids);
    cudaEvent_t ev_in[2], ev_comp[2], ev_out[2];
    for (int b = 0; b < 2; ++b) {
        cudaEventCreateWithFlags(&ev_in[b], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&ev_comp[b], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&ev_out[b], cudaEventDisableTiming);
    }
    if (rs.has_update) cudaStreamWaitEvent(ctx->stream, rs.last_update, 0);
    int rc = TANG_OK;
    const uint32_t nchunks = (n + chunk - 1) / chunk;
    uint32_t drained = 0;  // chunks whose ids were copied back to pageable user memory
    auto drain = [&](uint32_t c) {
        const uint32_t b = c & 1, c0 = c * chunk, rows = std::min(chunk, n - c0);
        cudaEventSynchronize(ev_out[b]);
        if (!pinned) std::memcpy(ids + c0, pi + size_t(b) * chunk, sizeof(uint32_t) * rows);
    };
    for (uint32_t c = 0; c < nchunks && rc == TANG_OK; ++c) {
        const uint32_t b = c & 1, c0 = c * chunk, rows = std::min(chunk, n - c0);
        const tang_header *src = h + c0;
        if (c >= 2) {
            // buffer b was used by chunk c-2: its results must be out before reuse
            if (!pinned) {
                drain(c - 2);
                drained = c - 1;
            }
            cudaStreamWaitEvent(ctx->copy_in, ev_out[b], 0);
        }
        if (!pinned) {
            if (c >= 2) cudaEventSynchronize(ev_in[b]);
            std::memcpy(ph + size_t(b) * chunk, src, sizeof(tang_header) * rows);
            src = ph + size_t(b) * chunk;
        }
        cudaMemcpyAsync(dh + size_t(b) * chunk, src, sizeof(tang_header) * rows, cudaMemcpyHostToDevice, ctx->copy_in);
        cudaEventRecord(ev_in[b], ctx->copy_in);
        cudaStreamWaitEvent(ctx->stream, ev_in[b], 0);
        rc = enqueue_classify(ctx, rs, dh + size_t(b) * chunk, rows, di + size_t(b) * chunk, path, stats, ctx->stream,
                              variant, smode);
        cudaEventRecord(ev_comp[b], ctx->stream);
        cudaStreamWaitEvent(ctx->copy_out, ev_comp[b], 0);
        uint32_t *dst = pinned ? ids + c0 : pi + size_t(b) * chunk;
        cudaMemcpyAsync(dst, di + size_t(b) * chunk, sizeof(uint32_t) * rows, cudaMemcpyDeviceToHost, ctx->copy_out);
        cudaEventRecord(ev_out[b], ctx->copy_out);
    }
    if (rc == TANG_OK) {
        if (!pinned)
            for (uint32_t c = drained; c < nchunks; ++c) drain(c);
        cudaStreamSynchronize(ctx->copy_out);
        cudaStreamSynchronize(ctx->stream);
    } else {
        cudaStreamSynchronize(ctx->copy_out);
        cudaStreamSynchronize(ctx->stream);
    }
    for (int b = 0; b < 2; ++b) {
        cudaEventDestroy(ev_in[b]);
        cudaEventDestroy(ev_comp[b]);
        cudaEventDestroy(ev_out[b]);
    }
    cudaError_t e = cudaGetLastError();
    if (rc == TANG_OK && e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "host pipeline: %s", cudaGetErrorString(e));
    return rc;
}

int tang_infer(tang_ctx *ctx, uint32_t rsh, const tang_header *d_headers, uint32_t n, float *d_logits,
               int32_t *d_tuple, int precision, void *stream) {
    const NvtxRange nvtx_range("tang_infer");
    if (!ctx) return TANG_EINVAL;
    Ruleset *rs = find_rs(ctx, rsh);
    if (!rs) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    if (n == 0) return TANG_OK;
    if (!d_headers || (reinterpret_cast<uintptr_t>(d_headers) & 15)) return set_err(ctx, TANG_EINVAL, "bad headers");
    cudaSetDevice(ctx->device);
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
    const int variant = variant_of(uint32_t(precision));
    return run_infer(ctx, *rs, d_headers, n, d_logits, d_tuple, precision & 0xF, st, variant);
}

int tang_search(tang_ctx *ctx, uint32_t rsh, const tang_header *d_headers, const int32_t *d_tuple, uint32_t n,
                uint32_t *d_ids, void *stream, tang_stats *stats) {
    return tang_search_ex(ctx, rsh, d_headers, d_tuple, n, d_ids, 0, stream, stats);
}

int tang_search_ex(tang_ctx *ctx, uint32_t rsh, const tang_header *d_headers, const int32_t *d_tuple, uint32_t n,
                   uint32_t *d_ids, uint32_t flags, void *stream, tang_stats *stats) {
    const NvtxRange nvtx_range("tang_search_ex");
    if (!ctx) return TANG_EINVAL;
    Ruleset *rs = find_rs(ctx, rsh);
    if (!rs) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    if (n && (!d_headers || !d_ids || (reinterpret_cast<uintptr_t>(d_headers) & 15)))
        return set_err(ctx, TANG_EINVAL, "bad buffers");
    cudaSetDevice(ctx->device);
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
    if (rs->has_update) CK(cudaStreamWaitEvent(st, rs->last_update, 0));
    DevStats *dst = stats ? ctx->d_stats : nullptr;
    if (dst) CK(cudaMemsetAsync(dst, 0, sizeof(DevStats), st));
    if (flags & ~uint32_t(TANG_SEARCH_PAPER | TANG_SEARCH_SERIAL))
        return set_err(ctx, TANG_EINVAL, "unknown search flags 0x%x", flags);
    CK(launch_search(rs->d_desc, uint32_t(rs->host.tuples.size()), rs->host.cw, d_headers, d_tuple, n, d_ids, dst,
                     nullptr, st, search_mode_of(flags)));
    if (n) note_classify(*rs, st);
    if (stats) {
        DevStats hs;
        CK(cudaMemcpyAsync(&hs, dst, sizeof(hs), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        std::memcpy(stats, &hs, sizeof(hs));
        return check_device_error(ctx);
    }
    return checked_sync(ctx, st);
}

int tang_insert_rule(tang_ctx *ctx, uint32_t rsh, const tang_rule *rule) {
    const NvtxRange nvtx_range("tang_insert_rule");
    if (!ctx || !rule) return set_err(ctx, TANG_EINVAL, "null argument");
    Ruleset *rs = find_rs(ctx, rsh);
    if (!rs) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    cudaSetDevice(ctx->device);
    // classifications already issued on other streams read the tables this call rewrites in place
    int rc = wait_classifies(ctx, *rs, ctx->stream);
    if (!rc) rc = tss_insert(ctx, *rs, *rule, ctx->stream);
    if (rc) return rc;
    CK(cudaEventRecord(rs->last_update, ctx->stream));
    rs->has_update = true;
    return TANG_OK;
}

int tang_delete_rule(tang_ctx *ctx, uint32_t rsh, uint32_t id) {
    const NvtxRange nvtx_range("tang_delete_rule");
    if (!ctx) return TANG_EINVAL;
    Ruleset *rs = find_rs(ctx, rsh);
    if (!rs) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    cudaSetDevice(ctx->device);
    int rc = wait_classifies(ctx, *rs, ctx->stream);
    if (!rc) rc = tss_delete(ctx, *rs, id, ctx->stream);
    if (rc) return rc;
    CK(cudaEventRecord(rs->last_update, ctx->stream));
    rs->has_update = true;
    return TANG_OK;
}

int tang_suboptimal_count(tang_ctx *ctx, uint32_t rsh, uint64_t *count) {
    if (!ctx || !count) return TANG_EINVAL;
    Ruleset *rs = find_rs(ctx, rsh);
    if (!rs) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    *count = rs->host.suboptimal;
    return TANG_OK;
}

double tang_now(void) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // extern "C"

namespace tang {
// Device-resident classification of one batch on `st` (serving engine, autotuner).
int enqueue_classify_path(tang_ctx *ctx, uint32_t rsh, const tang_header *h, uint32_t n, uint32_t *ids, uint32_t path,
                          cudaStream_t st) {
    Ruleset *rs = find_rs(ctx, rsh);
    if (!rs) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    if (rs->has_update) CK(cudaStreamWaitEvent(st, rs->last_update, 0));
    const int rc = enqueue_classify(ctx, *rs, h, n, ids, path, nullptr, st);
    if (rc == TANG_OK && n) note_classify(*rs, st);
    return rc;
}
void drop_graphs_of(tang_ctx *ctx) { drop_graphs(ctx); }
}  // namespace tang
