// Launch-shape autotuner: times the candidate launch shapes of a path on a caller-supplied
// device batch and keeps the fastest per (ruleset, path). Candidates:
//   search kernel (no-network, staged and plain paths): threads per block x blocks per SM;
//   fused kernel: one CTA per SM or CTA pairs, and the number of persistent CTAs (one per SM, or a
//   divisor-friendly subset so that the tile count spreads evenly); also the split form, the
//   network kernel and then the search kernel with the whole GPU (it wins when the ruleset holds
//   long runs, which the fused kernel's 128 search threads per SM scan slowly).
#include <algorithm>

#include "internal.h"

namespace tang {
int enqueue_classify_path(tang_ctx *ctx, uint32_t rs, const tang_header *h, uint32_t n, uint32_t *ids, uint32_t path,
                          cudaStream_t st);
void drop_graphs_of(tang_ctx *ctx);
}  // namespace tang

using namespace tang;

extern "C" int tang_autotune(tang_ctx *ctx, uint32_t rsh, const tang_header *d_headers, uint32_t n, uint32_t flags) {
    if (!ctx) return TANG_EINVAL;
    auto it = ctx->rulesets.find(rsh);
    if (it == ctx->rulesets.end()) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    if (n == 0 || !d_headers || (reinterpret_cast<uintptr_t>(d_headers) & 15))
        return set_err(ctx, TANG_EINVAL, "autotune needs a non-empty, 16-byte aligned device batch");
    Ruleset &rs = *it->second;
    const uint32_t path = flags & TANG_PATH_MASK;
    cudaSetDevice(ctx->device);
    std::vector<TuneEntry> cands;
    if (path == TANG_PATH_FUSED_BF16 || path == TANG_PATH_FUSED_FP8) {
        if (!rs.model) return set_err(ctx, TANG_EINVAL, "ruleset %u has no model", rsh);
        const int sms = ctx->sm_count;
        const uint32_t tiles = (n + 127) / 128;
        std::vector<int> grids = {sms};
        // the largest grid <= #SMs that divides the tile count evenly, if it is close to #SMs
        for (int g = sms - 1; g >= sms * 7 / 8; --g)
            if (tiles % uint32_t(g) == 0) {
                grids.push_back(g);
                break;
            }
        for (int v : {5, 6})
            for (int g : grids) {
                TuneEntry e;
                e.fused_variant = v;
                e.fused_grid = g;
                cands.push_back(e);
            }
        TuneEntry split;
        split.fused_variant = kVariantSplit;
        cands.push_back(split);
    } else {
        for (int th : {128, 256, 512})
            for (int bps : {2, 4, 8, 16}) {
                if (th * bps > 2048) continue;
                TuneEntry e;
                e.search_threads = th;
                e.search_bps = bps;
                cands.push_back(e);
            }
    }
    uint32_t *d_ids = nullptr;
    int rc = ctx_alloc(ctx, sizeof(uint32_t) * size_t(n), (void **)&d_ids);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    TuneEntry best;
    float best_ms = 1e30f;
    const TuneEntry saved = rs.tune.count(path) ? rs.tune[path] : TuneEntry{};
    for (const TuneEntry &c : cands) {
        rs.tune[path] = c;
        rc = enqueue_classify_path(ctx, rsh, d_headers, n, d_ids, path, ctx->stream);  // warm-up
        if (rc) break;
        const int reps = 3;
        cudaEventRecord(e0, ctx->stream);
        for (int r = 0; r < reps && !rc; ++r) rc = enqueue_classify_path(ctx, rsh, d_headers, n, d_ids, path, ctx->stream);
        cudaEventRecord(e1, ctx->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = set_err(ctx, TANG_EDEVICE, "autotune timing failed");
        if (rc) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx_free(ctx, d_ids);
    if (rc) {
        rs.tune[path] = saved;
        return rc;
    }
    best.ms = best_ms;
    rs.tune[path] = best;
    drop_graphs_of(ctx);  // graphs captured the previous launch shape
    return TANG_OK;
}

extern "C" int tang_autotune_set(tang_ctx *ctx, uint32_t rsh, uint32_t path, int variant, int grid, int search_threads,
                                 int search_bps) {
    if (!ctx) return TANG_EINVAL;
    auto it = ctx->rulesets.find(rsh);
    if (it == ctx->rulesets.end()) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    const uint32_t p = path & TANG_PATH_MASK;
    const bool fused = p == TANG_PATH_FUSED_BF16 || p == TANG_PATH_FUSED_FP8;
    const bool v_ok = variant == 0 || variant == 5 || variant == 6 || (variant == kVariantSplit && fused);
    if (!v_ok || grid < 0 || grid > ctx->sm_count)
        return set_err(ctx, TANG_EINVAL, "variant %d / grid %d out of range for path %u", variant, grid, p);
    const bool th_ok = search_threads == 0 || search_threads == 128 || search_threads == 256 || search_threads == 512;
    if (!th_ok || search_bps < 0 || search_bps > 16 || search_threads * search_bps > 2048)
        return set_err(ctx, TANG_EINVAL, "search launch %d threads x %d blocks per SM out of range", search_threads,
                       search_bps);
    TuneEntry e;
    e.fused_variant = variant;
    e.fused_grid = grid;
    e.search_threads = search_threads;
    e.search_bps = search_bps;
    it->second->tune[path & TANG_PATH_MASK] = e;
    drop_graphs_of(ctx);  // graphs captured the previous launch shape
    return TANG_OK;
}

extern "C" int tang_autotune_get(tang_ctx *ctx, uint32_t rsh, uint32_t path, int *variant, int *grid, int *search_threads,
                                 int *search_bps, float *ms) {
    if (!ctx) return TANG_EINVAL;
    auto it = ctx->rulesets.find(rsh);
    if (it == ctx->rulesets.end()) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    auto t = it->second->tune.find(path & TANG_PATH_MASK);
    const TuneEntry e = t == it->second->tune.end() ? TuneEntry{} : t->second;
    if (variant) *variant = e.fused_variant;
    if (grid) *grid = e.fused_grid;
    if (search_threads) *search_threads = e.search_threads;
    if (search_bps) *search_bps = e.search_bps;
    if (ms) *ms = e.ms;
    return TANG_OK;
}
