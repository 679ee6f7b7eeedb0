// Host side of the tuple space: construction (§4.3), device upload, and the immediate-update
// path (§5.2.1: delete, and insertion restricted to existing tuples).
//
// The host keeps a mirror of the device tables (tuples, slots, rule pool without the conflict
// words) so that inserts and deletes are decided on the host and applied to the device with a
// few stream-ordered copies and small kernels. Conflict sets live only on the device.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <numeric>
#include <unordered_set>

#include "internal.h"

namespace tang {

// MurmurHash3's 64-bit finalizer (fmix64, Austin Appleby, public domain); the device copy is in
// search_dev.cuh. Results of the classifier do not depend on the hash.
uint64_t fmix64_host(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

static uint32_t next_pow2(uint32_t v) {
    uint32_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

static inline bool key_less(uint32_t pa, uint32_t ia, uint32_t pb, uint32_t ib) {
    return pa < pb || (pa == pb && ia < ib);
}

static DRule to_drule(const tang_rule &r, uint32_t tuple) {
    DRule d;
    d.sip = r.sip & prefix_mask(r.sip_len);
    d.dip = r.dip & prefix_mask(r.dip_len);
    d.sp = uint32_t(r.sp_lo) | (uint32_t(r.sp_hi) << 16);
    d.dp = uint32_t(r.dp_lo) | (uint32_t(r.dp_hi) << 16);
    d.meta = make_meta(r.sip_len, r.dip_len, r.proto_wild ? 0u : 1u, r.proto_wild ? 0u : r.proto, tuple);
    d.prio = r.priority;
    d.id = r.id;
    d.cf = 0;
    return d;
}

static int validate_rule(tang_ctx *ctx, const tang_rule &r) {
    if (r.sip_len > 32 || r.dip_len > 32) return set_err(ctx, TANG_EINVAL, "rule %u: prefix length > 32", r.id);
    if (r.sp_lo > r.sp_hi || r.dp_lo > r.dp_hi) return set_err(ctx, TANG_EINVAL, "rule %u: port range lo > hi", r.id);
    if (r.id == TANG_NO_MATCH) return set_err(ctx, TANG_EINVAL, "rule id 0xFFFFFFFF is reserved");
    if (r.priority == 0xFFFFFFFFu) return set_err(ctx, TANG_EINVAL, "rule %u: priority 0xFFFFFFFF is reserved", r.id);
    if (r.reserved != 0) return set_err(ctx, TANG_EINVAL, "rule %u: reserved field must be 0", r.id);
    return TANG_OK;
}

// Linear probing on the host mirror. Returns the slot index (absolute) holding (ks, kd) or the
// first empty slot of the probe sequence if absent (found = false). dist = probe distance.
static uint32_t host_find(const HostTSS &H, const HostTuple &t, uint32_t ks, uint32_t kd, bool &found,
                          uint32_t &dist) {
    uint32_t mask = t.cap - 1;
    uint32_t h = uint32_t(fmix64_host((uint64_t(ks) << 32) | kd)) & mask;
    for (uint32_t i = 0; i <= mask; ++i) {
        const Slot &s = H.slots[t.slot_base + ((h + i) & mask)];
        if (s.start == kEmpty) {
            found = false;
            dist = i;
            return t.slot_base + ((h + i) & mask);
        }
        if (s.ks == ks && s.kd == kd) {
            found = true;
            dist = i;
            return t.slot_base + ((h + i) & mask);
        }
    }
    found = false;
    dist = t.cap;
    return kEmpty;  // table full (never happens: load factor is kept <= 3/4)
}

static void recompute_order(HostTSS &H) {
    uint32_t T = uint32_t(H.tuples.size());
    H.order.resize(T);
    std::iota(H.order.begin(), H.order.end(), 0);
    std::stable_sort(H.order.begin(), H.order.end(), [&](uint16_t a, uint16_t b) {
        const HostTuple &x = H.tuples[a], &y = H.tuples[b];
        return key_less(x.min_prio, x.min_id, y.min_prio, y.min_id);
    });
}

int tss_build(tang_ctx *ctx, Ruleset &rs, const tang_rule *rules, uint32_t n) {
    HostTSS &H = rs.host;
    for (uint32_t i = 0; i < n; ++i) {
        int rc = validate_rule(ctx, rules[i]);
        if (rc) return rc;
    }
    std::vector<uint32_t> ord(n);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](uint32_t a, uint32_t b) {
        return key_less(rules[a].priority, rules[a].id, rules[b].priority, rules[b].id);
    });
    {
        std::vector<uint32_t> ids(n);
        for (uint32_t i = 0; i < n; ++i) ids[i] = rules[i].id;
        std::sort(ids.begin(), ids.end());
        for (uint32_t i = 1; i < n; ++i)
            if (ids[i] == ids[i - 1]) return set_err(ctx, TANG_EEXIST, "duplicate rule id %u", ids[i]);
    }
    // Tuples in order of first appearance over the priority order (§4.3, Table 1 numbering).
    std::memset(H.tuple_of_len, 0xFF, sizeof(H.tuple_of_len));
    H.tuples.clear();
    auto add_tuple = [&](uint32_t ls, uint32_t ld) {
        HostTuple t{};
        t.ls = ls;
        t.ld = ld;
        t.min_prio = t.min_id = 0xFFFFFFFFu;
        H.tuple_of_len[ls][ld] = int16_t(H.tuples.size());
        H.tuples.push_back(t);
    };
    for (uint32_t k = 0; k < n; ++k) {
        const tang_rule &r = rules[ord[k]];
        if (H.tuple_of_len[r.sip_len][r.dip_len] < 0) {
            if (H.tuples.size() >= kMaxTuples) return set_err(ctx, TANG_ETABLEFULL, "more than %u tuples", kMaxTuples);
            add_tuple(r.sip_len, r.dip_len);
        }
    }
    if (H.tuple_of_len[0][0] < 0) add_tuple(0, 0);
    const uint32_t T = uint32_t(H.tuples.size());
    H.cw = (T + 31) / 32;

    // Group rules by (tuple, truncated key); within a key keep the priority order.
    struct Ent {
        uint32_t t, ks, kd, rank;
    };
    std::vector<Ent> ents(n);
    for (uint32_t k = 0; k < n; ++k) {
        const tang_rule &r = rules[ord[k]];
        uint32_t t = uint32_t(H.tuple_of_len[r.sip_len][r.dip_len]);
        const HostTuple &ht = H.tuples[t];
        ents[k] = {t, r.sip & prefix_mask(ht.ls), r.dip & prefix_mask(ht.ld), k};
    }
    std::sort(ents.begin(), ents.end(), [](const Ent &a, const Ent &b) {
        if (a.t != b.t) return a.t < b.t;
        if (a.ks != b.ks) return a.ks < b.ks;
        if (a.kd != b.kd) return a.kd < b.kd;
        return a.rank < b.rank;
    });
    std::vector<uint32_t> keys_per_tuple(T, 0);
    for (uint32_t k = 0; k < n; ++k)
        if (k == 0 || ents[k].t != ents[k - 1].t || ents[k].ks != ents[k - 1].ks || ents[k].kd != ents[k - 1].kd)
            keys_per_tuple[ents[k].t]++;
    uint32_t slot_total = 0;
    for (uint32_t t = 0; t < T; ++t) {
        H.tuples[t].cap = next_pow2(std::max(4u, 2 * keys_per_tuple[t]));
        H.tuples[t].slot_base = slot_total;
        slot_total += H.tuples[t].cap;
    }
    H.slots.assign(slot_total, Slot{0, 0, kEmpty, 0});
    H.run_cap.assign(slot_total, 0);
    H.pool.clear();
    H.pool.reserve(n);
    H.pos_of_id.clear();
    H.pos_of_id.reserve(size_t(n) * 2);
    for (uint32_t k = 0; k < n;) {
        uint32_t e = k;
        while (e < n && ents[e].t == ents[k].t && ents[e].ks == ents[k].ks && ents[e].kd == ents[k].kd) ++e;
        HostTuple &ht = H.tuples[ents[k].t];
        bool found;
        uint32_t dist;
        uint32_t s = host_find(H, ht, ents[k].ks, ents[k].kd, found, dist);
        H.slots[s] = Slot{ents[k].ks, ents[k].kd, uint32_t(H.pool.size()), e - k};
        H.run_cap[s] = e - k;
        ht.n_keys++;
        ht.max_probe = std::max(ht.max_probe, dist);
        for (uint32_t j = k; j < e; ++j) {
            const tang_rule &r = rules[ord[ents[j].rank]];
            H.pos_of_id[r.id] = uint32_t(H.pool.size());
            H.pool.push_back(to_drule(r, ents[k].t));
            ht.n_rules++;
            if (key_less(r.priority, r.id, ht.min_prio, ht.min_id)) {
                ht.min_prio = r.priority;
                ht.min_id = r.id;
            }
        }
        k = e;
    }
    H.live = n;
    H.suboptimal = 0;
    recompute_order(H);
    return TANG_OK;
}

static void fill_desc(const HostTSS &H, std::vector<TupleDesc> &out) {
    out.resize(H.tuples.size());
    for (size_t t = 0; t < H.tuples.size(); ++t) {
        const HostTuple &h = H.tuples[t];
        out[t] = TupleDesc{prefix_mask(h.ls), prefix_mask(h.ld), h.slot_base, h.cap - 1,
                           h.min_prio,        h.min_id,        h.max_probe, h.n_rules};
    }
}

#define CKR(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static int upload_desc(tang_ctx *ctx, Ruleset &rs, cudaStream_t st) {
    rs.h_desc.tuples = rs.d_tuples;
    rs.h_desc.slots = rs.d_slots;
    rs.h_desc.rules = rs.d_rules;
    rs.h_desc.cwords = rs.d_cwords;
    rs.h_desc.order = rs.d_order;
    rs.h_desc.T = uint32_t(rs.host.tuples.size());
    rs.h_desc.cw = rs.host.cw;
    rs.h_desc.pool_size = rs.pool_view != kEmpty ? rs.pool_view : uint32_t(rs.host.pool.size());
    rs.h_desc.slot_cap = rs.slot_capacity;
    rs.h_desc.cword_rows = rs.host.cw > 1 ? rs.cword_capacity / rs.host.cw : 0;
    rs.h_desc.err = ctx->d_err;
    CKR(cudaMemcpyAsync(rs.d_desc, &rs.h_desc, sizeof(Tables), cudaMemcpyHostToDevice, st));
    return TANG_OK;
}

// Test hook: make the device descriptor state a pool size of n (kEmpty: the real size again).
int tss_set_pool_view(tang_ctx *ctx, Ruleset &rs, uint32_t n) {
    rs.pool_view = n;
    int rc = upload_desc(ctx, rs, ctx->stream);
    if (!rc) CKR(cudaStreamSynchronize(ctx->stream));
    return rc;
}

int tss_upload(tang_ctx *ctx, Ruleset &rs, cudaStream_t st) {
    HostTSS &H = rs.host;
    const uint32_t T = uint32_t(H.tuples.size());
    const uint32_t n = uint32_t(H.pool.size());
    rs.slot_capacity = uint32_t(H.slots.size()) * 2 + 4096;
    rs.rule_capacity = n + n / 4 + 4096;
    int rc;
    if ((rc = ctx_alloc(ctx, sizeof(TupleDesc) * kMaxTuples, (void **)&rs.d_tuples))) return rc;
    if ((rc = ctx_alloc(ctx, sizeof(Slot) * size_t(rs.slot_capacity), (void **)&rs.d_slots))) return rc;
    if ((rc = ctx_alloc(ctx, sizeof(DRule) * size_t(rs.rule_capacity), (void **)&rs.d_rules))) return rc;
    if ((rc = ctx_alloc(ctx, sizeof(uint16_t) * kMaxTuples, (void **)&rs.d_order))) return rc;
    if ((rc = ctx_alloc(ctx, sizeof(Tables), (void **)&rs.d_desc))) return rc;
    if (H.cw > 1) {
        rs.cword_capacity = rs.rule_capacity * H.cw;  // in words
        if ((rc = ctx_alloc(ctx, sizeof(uint32_t) * size_t(rs.cword_capacity), (void **)&rs.d_cwords))) return rc;
        CKR(cudaMemsetAsync(rs.d_cwords, 0, sizeof(uint32_t) * size_t(rs.cword_capacity), st));
        rs.cword_rows = n;
        // every rule owns the conflict row of its build position; inserts take new rows
        for (uint32_t p = 0; p < n; ++p) H.pool[p].cf = p;
    }
    std::vector<TupleDesc> td;
    fill_desc(H, td);
    CKR(cudaMemcpyAsync(rs.d_tuples, td.data(), sizeof(TupleDesc) * T, cudaMemcpyHostToDevice, st));
    CKR(cudaMemsetAsync(rs.d_slots, 0xFF, sizeof(Slot) * size_t(rs.slot_capacity), st));
    if (!H.slots.empty())
        CKR(cudaMemcpyAsync(rs.d_slots, H.slots.data(), sizeof(Slot) * H.slots.size(), cudaMemcpyHostToDevice, st));
    if (n) CKR(cudaMemcpyAsync(rs.d_rules, H.pool.data(), sizeof(DRule) * n, cudaMemcpyHostToDevice, st));
    CKR(cudaMemcpyAsync(rs.d_order, H.order.data(), sizeof(uint16_t) * T, cudaMemcpyHostToDevice, st));
    if ((rc = upload_desc(ctx, rs, st))) return rc;

    // Conflict sets: brute force over better rules on the GPU, in priority order.
    if (n) {
        std::vector<uint32_t> ord(n);
        std::iota(ord.begin(), ord.end(), 0);
        std::sort(ord.begin(), ord.end(), [&](uint32_t a, uint32_t b) {
            return key_less(H.pool[a].prio, H.pool[a].id, H.pool[b].prio, H.pool[b].id);
        });
        std::vector<DRule> sorted(n);
        for (uint32_t k = 0; k < n; ++k) sorted[k] = H.pool[ord[k]];
        DRule *d_sorted = nullptr;
        uint32_t *d_pos = nullptr;
        if ((rc = ctx_alloc(ctx, sizeof(DRule) * n, (void **)&d_sorted))) return rc;
        if ((rc = ctx_alloc(ctx, sizeof(uint32_t) * n, (void **)&d_pos))) {
            ctx_free(ctx, d_sorted);
            return rc;
        }
        CKR(cudaMemcpyAsync(d_sorted, sorted.data(), sizeof(DRule) * n, cudaMemcpyHostToDevice, st));
        CKR(cudaMemcpyAsync(d_pos, ord.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice, st));
        CKR(launch_conflict_build(d_sorted, d_pos, n, rs.d_rules, rs.d_cwords, H.cw, T, st));
        CKR(cudaStreamSynchronize(st));
        ctx_free(ctx, d_sorted);
        ctx_free(ctx, d_pos);
    }
    CKR(cudaStreamSynchronize(st));
    return TANG_OK;
}

void tss_free(tang_ctx *ctx, Ruleset &rs) {
    ctx_free(ctx, rs.d_tuples);
    ctx_free(ctx, rs.d_slots);
    ctx_free(ctx, rs.d_rules);
    ctx_free(ctx, rs.d_cwords);
    ctx_free(ctx, rs.d_order);
    ctx_free(ctx, rs.d_desc);
    rs.d_tuples = nullptr;
    rs.d_slots = nullptr;
    rs.d_rules = nullptr;
    rs.d_cwords = nullptr;
    rs.d_order = nullptr;
    rs.d_desc = nullptr;
}

// Full rebuild of the tuple space over the live rules (the TSS step of §5.2.2's full retraining):
// tuples are recomputed from the rules' own lengths, so rules that restricted insertion placed in
// a coarser tuple move to their exact one, tuples may appear or disappear, and the counter of such
// rules restarts at zero. The ruleset keeps its device descriptor (kernels and captured graphs
// reach the tables through it); only the arrays it points to are replaced. same_tuples reports
// whether the new tuple list (lengths in index order) equals the old one.
int tss_rebuild(tang_ctx *ctx, Ruleset &rs, bool &same_tuples) {
    const HostTSS &H = rs.host;
    std::vector<tang_rule> live;
    live.reserve(H.live);
    for (const auto &kv : H.pos_of_id) {
        const DRule &d = H.pool[kv.second];
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
        live.push_back(r);
    }
    Ruleset fresh;
    int rc = tss_build(ctx, fresh, live.data(), uint32_t(live.size()));
    if (!rc) rc = tss_upload(ctx, fresh, ctx->stream);
    if (rc) {
        tss_free(ctx, fresh);
        return rc;
    }
    same_tuples = fresh.host.tuples.size() == H.tuples.size();
    for (size_t t = 0; same_tuples && t < H.tuples.size(); ++t)
        same_tuples = fresh.host.tuples[t].ls == H.tuples[t].ls && fresh.host.tuples[t].ld == H.tuples[t].ld;
    // no kernel may still read the old arrays
    CKR(cudaDeviceSynchronize());
    Tables *desc = rs.d_desc;
    rs.d_desc = nullptr;
    tss_free(ctx, rs);
    rs.host = std::move(fresh.host);
    rs.d_tuples = fresh.d_tuples;
    rs.d_slots = fresh.d_slots;
    rs.d_rules = fresh.d_rules;
    rs.d_cwords = fresh.d_cwords;
    rs.d_order = fresh.d_order;
    rs.slot_capacity = fresh.slot_capacity;
    rs.rule_capacity = fresh.rule_capacity;
    rs.cword_capacity = fresh.cword_capacity;
    rs.cword_rows = fresh.cword_rows;
    ctx_free(ctx, fresh.d_desc);
    rs.d_desc = desc;
    if ((rc = upload_desc(ctx, rs, ctx->stream))) return rc;
    CKR(cudaStreamSynchronize(ctx->stream));
    return TANG_OK;
}

// ---------------------------------------------------------------------------------------
// Immediate update (§5.2.1)
// ---------------------------------------------------------------------------------------

// Grow a device array to hold at least `need` elements (copying `used` of them). The tables'
// descriptor is re-uploaded by the caller, so captured graphs keep working.
template <typename T>
static int grow(tang_ctx *ctx, T **arr, uint32_t &capacity, uint32_t used, uint32_t need, cudaStream_t st,
                int fill) {
    if (need <= capacity) return TANG_OK;
    uint32_t cap2 = std::max(need, capacity + capacity / 2 + 1024);
    T *fresh = nullptr;
    int rc = ctx_alloc(ctx, sizeof(T) * size_t(cap2), (void **)&fresh);
    if (rc) return rc;
    if (fill >= 0) CKR(cudaMemsetAsync(fresh, fill, sizeof(T) * size_t(cap2), st));
    if (used) CKR(cudaMemcpyAsync(fresh, *arr, sizeof(T) * size_t(used), cudaMemcpyDeviceToDevice, st));
    CKR(cudaStreamSynchronize(st));
    ctx_free(ctx, *arr);
    *arr = fresh;
    capacity = cap2;
    return TANG_OK;
}

static int upload_tuple(tang_ctx *ctx, Ruleset &rs, uint32_t t, cudaStream_t st) {
    const HostTuple &h = rs.host.tuples[t];
    TupleDesc d{prefix_mask(h.ls), prefix_mask(h.ld), h.slot_base, h.cap - 1, h.min_prio, h.min_id, h.max_probe,
                h.n_rules};
    CKR(cudaMemcpyAsync(rs.d_tuples + t, &d, sizeof(d), cudaMemcpyHostToDevice, st));
    return TANG_OK;
}

static int upload_slot(tang_ctx *ctx, Ruleset &rs, uint32_t s, cudaStream_t st) {
    CKR(cudaMemcpyAsync(rs.d_slots + s, &rs.host.slots[s], sizeof(Slot), cudaMemcpyHostToDevice, st));
    return TANG_OK;
}

// Move tuple t's table to a fresh region twice as large (keys re-inserted).
static int rehash_tuple(tang_ctx *ctx, Ruleset &rs, uint32_t t, cudaStream_t st) {
    HostTSS &H = rs.host;
    HostTuple &ht = H.tuples[t];
    uint32_t old_base = ht.slot_base, old_cap = ht.cap;
    uint32_t new_cap = old_cap * 2;
    uint32_t new_base = uint32_t(H.slots.size());
    int rc = grow(ctx, &rs.d_slots, rs.slot_capacity, uint32_t(H.slots.size()), new_base + new_cap, st, 0xFF);
    if (rc) return rc;
    H.slots.resize(new_base + new_cap, Slot{0, 0, kEmpty, 0});
    H.run_cap.resize(new_base + new_cap, 0);
    ht.slot_base = new_base;
    ht.cap = new_cap;
    ht.max_probe = 0;
    for (uint32_t i = 0; i < old_cap; ++i) {
        Slot s = H.slots[old_base + i];
        if (s.start == kEmpty) continue;
        bool found;
        uint32_t dist;
        uint32_t at = host_find(H, ht, s.ks, s.kd, found, dist);
        H.slots[at] = s;
        H.run_cap[at] = H.run_cap[old_base + i];
        ht.max_probe = std::max(ht.max_probe, dist);
    }
    CKR(cudaMemcpyAsync(rs.d_slots + new_base, H.slots.data() + new_base, sizeof(Slot) * new_cap,
                        cudaMemcpyHostToDevice, st));
    return TANG_OK;
}

int tss_insert(tang_ctx *ctx, Ruleset &rs, const tang_rule &r, cudaStream_t st) {
    HostTSS &H = rs.host;
    int rc = validate_rule(ctx, r);
    if (rc) return rc;
    if (H.pos_of_id.count(r.id)) return set_err(ctx, TANG_EEXIST, "rule id %u is already live", r.id);
    // §5.2.1: exact lengths, else the first tuple of maximal length sum with l^T <= l^R.
    int t = H.tuple_of_len[r.sip_len][r.dip_len];
    if (t < 0) {
        int best_sum = -1;
        for (uint32_t i = 0; i < H.tuples.size(); ++i) {
            const HostTuple &ht = H.tuples[i];
            if (ht.ls <= r.sip_len && ht.ld <= r.dip_len && int(ht.ls + ht.ld) > best_sum) {
                best_sum = int(ht.ls + ht.ld);
                t = int(i);
            }
        }
        if (t < 0) return set_err(ctx, TANG_EINVAL, "no tuple can hold rule %u", r.id);
        H.suboptimal++;
    }
    HostTuple &ht = H.tuples[t];
    uint32_t ks = r.sip & prefix_mask(ht.ls), kd = r.dip & prefix_mask(ht.ld);
    bool found;
    uint32_t dist;
    uint32_t s = host_find(H, ht, ks, kd, found, dist);
    if (!found && (ht.n_keys + 1) * 4 > ht.cap * 3) {
        if ((rc = rehash_tuple(ctx, rs, uint32_t(t), st))) return rc;
        s = host_find(H, ht, ks, kd, found, dist);
    }
    if (!found) {
        H.slots[s] = Slot{ks, kd, uint32_t(H.pool.size()), 0};
        H.run_cap[s] = 0;
        ht.n_keys++;
        ht.max_probe = std::max(ht.max_probe, dist);
    }
    Slot &slot = H.slots[s];
    DRule nr = to_drule(r, uint32_t(t));
    // position inside the run, kept in (priority, id) order
    uint32_t p = 0;
    while (p < slot.len && key_less(H.pool[slot.start + p].prio, H.pool[slot.start + p].id, nr.prio, nr.id)) ++p;
    if (slot.len == H.run_cap[s]) {
        // relocate the run to the end of the pool with room to grow
        uint32_t cap2 = std::max(4u, H.run_cap[s] * 2);
        uint32_t from = slot.start, to = uint32_t(H.pool.size());
        uint32_t used = uint32_t(H.pool.size());
        if ((rc = grow(ctx, &rs.d_rules, rs.rule_capacity, used, to + cap2, st, -1))) return rc;
        DRule dead;
        std::memset(&dead, 0xFF, sizeof(dead));
        H.pool.resize(to + cap2, dead);
        if (slot.len) {
            CKR(launch_run_copy(rs.d_rules, from, to, slot.len, st));
            for (uint32_t j = 0; j < slot.len; ++j) {
                H.pool[to + j] = H.pool[from + j];
                H.pos_of_id[H.pool[to + j].id] = to + j;
                H.pool[from + j] = dead;
            }
            CKR(cudaMemsetAsync(rs.d_rules + from, 0xFF, sizeof(DRule) * slot.len, st));
        }
        CKR(cudaMemsetAsync(rs.d_rules + to + slot.len, 0xFF, sizeof(DRule) * (cap2 - slot.len), st));
        slot.start = to;
        H.run_cap[s] = cap2;
    }
    // shift the tail of the run up by one and write the new rule
    if (p < slot.len) CKR(launch_run_shift(rs.d_rules, slot.start, slot.len, p, +1, st));
    for (uint32_t j = slot.len; j > p; --j) {
        H.pool[slot.start + j] = H.pool[slot.start + j - 1];
        H.pos_of_id[H.pool[slot.start + j].id] = slot.start + j;
    }
    uint32_t new_pos = slot.start + p;
    if (H.cw > 1) {
        // a fresh conflict row for the new rule (rows are never reused)
        uint32_t row = rs.cword_rows;
        if ((rc = grow(ctx, &rs.d_cwords, rs.cword_capacity, rs.cword_rows * H.cw, (row + 1) * H.cw, st, 0)))
            return rc;
        CKR(cudaMemsetAsync(rs.d_cwords + size_t(row) * H.cw, 0, sizeof(uint32_t) * H.cw, st));
        nr.cf = row;
        rs.cword_rows = row + 1;
    }
    H.pool[new_pos] = nr;
    H.pos_of_id[nr.id] = new_pos;
    CKR(cudaMemcpyAsync(rs.d_rules + new_pos, &H.pool[new_pos], sizeof(DRule), cudaMemcpyHostToDevice, st));
    slot.len++;
    if ((rc = upload_slot(ctx, rs, s, st))) return rc;
    ht.n_rules++;
    bool order_changed = false;
    if (key_less(nr.prio, nr.id, ht.min_prio, ht.min_id)) {
        ht.min_prio = nr.prio;
        ht.min_id = nr.id;
        order_changed = true;
    }
    if ((rc = upload_tuple(ctx, rs, uint32_t(t), st))) return rc;
    if (order_changed) {
        recompute_order(H);
        CKR(cudaMemcpyAsync(rs.d_order, H.order.data(), sizeof(uint16_t) * H.order.size(), cudaMemcpyHostToDevice,
                            st));
    }
    H.live++;
    if ((rc = upload_desc(ctx, rs, st))) return rc;
    CKR(launch_conflict_insert(rs.d_desc, uint32_t(H.pool.size()), new_pos, H.cw, st));
    return TANG_OK;
}

int tss_delete(tang_ctx *ctx, Ruleset &rs, uint32_t id, cudaStream_t st) {
    HostTSS &H = rs.host;
    auto it = H.pos_of_id.find(id);
    if (it == H.pos_of_id.end()) return set_err(ctx, TANG_ENOTFOUND, "rule id %u is not live", id);
    uint32_t pos = it->second;
    DRule r = H.pool[pos];
    uint32_t t = meta_tuple(r.meta);
    HostTuple &ht = H.tuples[t];
    uint32_t ks = r.sip & prefix_mask(ht.ls), kd = r.dip & prefix_mask(ht.ld);
    bool found;
    uint32_t dist;
    uint32_t s = host_find(H, ht, ks, kd, found, dist);
    if (!found) return set_err(ctx, TANG_EDEVICE, "internal: rule %u has no slot", id);
    Slot &slot = H.slots[s];
    uint32_t p = pos - slot.start;
    if (p + 1 < slot.len) CKR(launch_run_shift(rs.d_rules, slot.start, slot.len, p, -1, st));
    for (uint32_t j = p; j + 1 < slot.len; ++j) {
        H.pool[slot.start + j] = H.pool[slot.start + j + 1];
        H.pos_of_id[H.pool[slot.start + j].id] = slot.start + j;
    }
    std::memset(&H.pool[slot.start + slot.len - 1], 0xFF, sizeof(DRule));
    CKR(cudaMemsetAsync(rs.d_rules + slot.start + slot.len - 1, 0xFF, sizeof(DRule), st));
    H.pos_of_id.erase(it);
    slot.len--;
    int rc;
    if ((rc = upload_slot(ctx, rs, s, st))) return rc;
    ht.n_rules--;
    if ((rc = upload_tuple(ctx, rs, t, st))) return rc;
    H.live--;
    return TANG_OK;
}

}  // namespace tang
