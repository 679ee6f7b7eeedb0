// Deferred update (§5.2.2): the throughput monitor and its trigger (tau), the choice between
// incremental training and full retraining (theta, on the counter of rules that restricted
// insertion placed in a tuple whose lengths differ from theirs), incremental training from the
// deployed model, the full rebuild of the tuple space, and the hot swap of the new weights.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

using namespace tang;

extern "C" void tang_model_free(tang_ctx *ctx, DeviceModel *m);

namespace tang {
void drop_graphs_of(tang_ctx *ctx);
}

static Ruleset *du_find(tang_ctx *ctx, uint32_t rsh) {
    auto it = ctx->rulesets.find(rsh);
    return it == ctx->rulesets.end() ? nullptr : it->second.get();
}

extern "C" {

int tang_du_decide(const tang_du_cfg *cfg, double th_base, double th_cur, uint64_t suboptimal) {
    if (!cfg || !(cfg->tau >= 0.0) || !std::isfinite(cfg->tau)) return TANG_EINVAL;
    if (!(th_base > 0.0) || !(th_cur >= 0.0) || !std::isfinite(th_base) || !std::isfinite(th_cur)) return TANG_DU_NONE;
    // §5.2.2: a deferred update when the windowed throughput has dropped by more than tau relative
    // to the first window after the last full retraining ...
    if (!(1.0 - th_cur / th_base > cfg->tau)) return TANG_DU_NONE;
    // ... a full retraining when more than theta rules sit in tuples that do not match their
    // lengths, incremental training otherwise
    return suboptimal > cfg->theta ? TANG_DU_RETRAIN : TANG_DU_INCREMENTAL;
}

int tang_du_observe(tang_ctx *ctx, uint32_t rsh, uint64_t packets, double cost) {
    if (!ctx) return TANG_EINVAL;
    Ruleset *rs = du_find(ctx, rsh);
    if (!rs) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    if (!(cost >= 0.0) || !std::isfinite(cost)) return set_err(ctx, TANG_EINVAL, "window cost must be finite and >= 0");
    rs->du_packets += packets;
    rs->du_cost += cost;
    return TANG_OK;
}

int tang_du_close_window(tang_ctx *ctx, uint32_t rsh, const tang_du_cfg *cfg, tang_du_window *out) {
    if (!ctx || !cfg || !out) return set_err(ctx, TANG_EINVAL, "null argument");
    Ruleset *rs = du_find(ctx, rsh);
    if (!rs) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    if (rs->du_packets == 0 || !(rs->du_cost > 0.0))
        return set_err(ctx, TANG_EINVAL, "the window holds no observation (packets and cost must be > 0)");
    const double th = double(rs->du_packets) / rs->du_cost;
    out->window = rs->du_windows;
    if (rs->du_windows == 0) rs->du_th_base = th;
    out->th_cur = th;
    out->th_base = rs->du_th_base;
    out->suboptimal = rs->host.suboptimal;
    const int d = rs->du_windows == 0 ? TANG_DU_NONE : tang_du_decide(cfg, rs->du_th_base, th, rs->host.suboptimal);
    if (d < 0) return set_err(ctx, d, "bad deferred-update configuration");
    out->decision = d;
    rs->du_windows++;
    rs->du_packets = 0;
    rs->du_cost = 0.0;
    return TANG_OK;
}

int tang_finetune(tang_ctx *ctx, uint32_t rsh, const tang_header *samples, uint32_t n, const tang_train_cfg *cfg,
                  void *blob, size_t *bytes, tang_train_report *report) {
    const NvtxRange nvtx_range("tang_finetune");
    if (!ctx || !samples || !cfg || !bytes || n == 0) return set_err(ctx, TANG_EINVAL, "bad argument");
    Ruleset *rs = du_find(ctx, rsh);
    if (!rs) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    if (!rs->model) return set_err(ctx, TANG_EINVAL, "ruleset %u has no model to train from", rsh);
    cudaSetDevice(ctx->device);
    std::vector<uint8_t> out;
    int rc = train_run(ctx, *rs, samples, n, *cfg, out, report, rs->model.get());
    if (rc) return rc;
    const size_t have = *bytes;
    *bytes = out.size();
    if (blob && have >= out.size()) std::memcpy(blob, out.data(), out.size());
    return TANG_OK;
}

int tang_rebuild_ruleset(tang_ctx *ctx, uint32_t rsh, int *model_kept) {
    const NvtxRange nvtx_range("tang_rebuild_ruleset");
    if (!ctx) return TANG_EINVAL;
    Ruleset *rs = du_find(ctx, rsh);
    if (!rs) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    cudaSetDevice(ctx->device);
    bool same = false;
    int rc = tss_rebuild(ctx, *rs, same);
    if (rc) return rc;
    // a model whose class list no longer matches the tuples goes, with the graphs that use it
    if (!same && rs->model) {
        drop_graphs_of(ctx);
        tang_model_free(ctx, rs->model.get());
        rs->model.reset();
    }
    if (model_kept) *model_kept = rs->model ? 1 : 0;
    rs->has_update = false;
    rs->du_packets = 0;
    rs->du_cost = 0.0;
    rs->du_windows = 0;  // the next closed window is the new baseline
    rs->du_th_base = 0.0;
    return TANG_OK;
}

int tang_du_apply(tang_ctx *ctx, uint32_t rsh, int decision, const tang_header *samples, uint32_t n,
                  const tang_train_cfg *cfg, tang_train_report *report) {
    const NvtxRange nvtx_range("tang_du_apply");
    if (!ctx) return TANG_EINVAL;
    Ruleset *rs = du_find(ctx, rsh);
    if (!rs) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    if (decision == TANG_DU_NONE) return TANG_OK;
    if (decision != TANG_DU_INCREMENTAL && decision != TANG_DU_RETRAIN)
        return set_err(ctx, TANG_EINVAL, "unknown deferred-update decision %d", decision);
    if (!samples || !cfg || n == 0) return set_err(ctx, TANG_EINVAL, "training samples and configuration required");
    cudaSetDevice(ctx->device);
    std::vector<uint8_t> blob;
    int rc;
    if (decision == TANG_DU_INCREMENTAL) {
        if (!rs->model) return set_err(ctx, TANG_EINVAL, "incremental training needs a loaded model");
        rc = train_run(ctx, *rs, samples, n, *cfg, blob, report, rs->model.get());
    } else {
        if ((rc = tang_rebuild_ruleset(ctx, rsh, nullptr))) return rc;
        // full retraining trains from scratch even when the tuple list survived the rebuild
        rc = train_run(ctx, *rs, samples, n, *cfg, blob, report, nullptr);
    }
    if (rc) return rc;
    return tang_load_model(ctx, rsh, blob.data(), blob.size());
}

int tang_export_rules(tang_ctx *ctx, uint32_t rsh, tang_rule *out, uint32_t cap, uint32_t *n_out) {
    if (!ctx || !n_out) return TANG_EINVAL;
    Ruleset *rs = du_find(ctx, rsh);
    if (!rs) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    const HostTSS &H = rs->host;
    *n_out = uint32_t(H.pos_of_id.size());
    if (!out) return TANG_OK;
    if (cap < *n_out) return set_err(ctx, TANG_EINVAL, "export needs room for %u rules", *n_out);
    std::vector<const DRule *> live;
    live.reserve(H.pos_of_id.size());
    for (const auto &kv : H.pos_of_id) live.push_back(&H.pool[kv.second]);
    std::sort(live.begin(), live.end(), [](const DRule *a, const DRule *b) {
        return a->prio < b->prio || (a->prio == b->prio && a->id < b->id);
    });
    for (size_t i = 0; i < live.size(); ++i) {
        const DRule &d = *live[i];
        tang_rule r{};
        r.sip = d.sip;
        r.dip = d.dip;
        r.sp_lo = uint16_t(d.sp & 0xFFFFu);
        r.sp_hi = uint16_t(d.sp >> 16);
        r.dp_lo = uint16_t(d.dp & 0xFFFFu);
        r.dp_hi = uint16_t(d.dp >> 16);
        r.sip_len = uint8_t(meta_sip_len(d.meta));
        r.dip_len = uint8_t(meta_dip_len(d.meta));
        r.proto_wild = meta_proto_exact(d.meta) ? 0 : 1;
        r.proto = uint8_t(meta_proto(d.meta));
        r.priority = d.prio;
        r.id = d.id;
        out[i] = r;
    }
    return TANG_OK;
}

int tang_graph_count(tang_ctx *ctx, uint32_t *count) {
    if (!ctx || !count) return TANG_EINVAL;
    *count = uint32_t(ctx->graphs.size());
    return TANG_OK;
}

}  // extern "C"
