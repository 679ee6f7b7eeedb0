// Device functions of the exact tuple-space search (stage 2 of §5.1.1), shared by the staged
// search kernel (search.cu) and the fused classification kernel (mlp_tc256.cu).
#pragma once

#include "internal.h"

namespace tang {

// Checked builds (TANG_CHECKED) test every table index against its table's size before the
// access; an index out of range sets kErrIndex in the context's error word and the access is
// skipped (the lookup then ends as if it had found nothing). Other builds compile the test out.
#ifdef TANG_CHECKED
#define TANG_INDEX_OK(tb, cond) ((cond) || (atomicOr((tb).err, kErrIndex), false))
#else
#define TANG_INDEX_OK(tb, cond) true
#endif

// MurmurHash3 fmix64 finalizer (Austin Appleby, public domain); same as fmix64_host().
__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

struct Hdr {
    uint32_t sip, dip, sp, dp, proto;
};

__device__ __forceinline__ Hdr load_header(const tang_header *h) {
    uint4 v = __ldg(reinterpret_cast<const uint4 *>(h));
    return Hdr{v.x, v.y, v.z & 0xFFFFu, v.z >> 16, v.w & 0xFFu};
}
// Header read with the evict-first (streaming) cache hint: packet headers are read once or twice
// and should not displace the hash tables from L2.
__device__ __forceinline__ Hdr load_header_stream(const tang_header *h) {
    uint4 v = __ldcs(reinterpret_cast<const uint4 *>(h));
    return Hdr{v.x, v.y, v.z & 0xFFFFu, v.z >> 16, v.w & 0xFFu};
}

__device__ __forceinline__ DRule load_rule(const DRule *r) {
    uint4 a = __ldg(reinterpret_cast<const uint4 *>(r));
    uint4 b = __ldg(reinterpret_cast<const uint4 *>(r) + 1);
    return DRule{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
}

// Rule conditions of §2.1 on the rule's own prefix lengths (also for rules truncated into a
// coarser tuple by restricted insertion).
__device__ __forceinline__ bool rule_match(const DRule &r, const Hdr &h) {
    uint32_t m = r.meta;
    bool ok = ((h.sip ^ r.sip) & prefix_mask(meta_sip_len(m))) == 0;
    ok &= ((h.dip ^ r.dip) & prefix_mask(meta_dip_len(m))) == 0;
    ok &= (h.sp >= (r.sp & 0xFFFFu)) & (h.sp <= (r.sp >> 16));
    ok &= (h.dp >= (r.dp & 0xFFFFu)) & (h.dp <= (r.dp >> 16));
    ok &= (!meta_proto_exact(m)) | (h.proto == meta_proto(m));
    return ok;
}

// The best match found so far, ordered by (priority, id).
struct Best {
    uint32_t prio, id, pos, cf, tuple;
};

__device__ __forceinline__ bool beats(uint32_t prio, uint32_t id, const Best &b) {
    return prio < b.prio || (prio == b.prio && id < b.id);
}

struct Counters {
    uint32_t probes, rule_reads, slot_reads;
};

// A thread scans the first kCoopAfter rules of a run itself; if the scan has not ended there, the
// rest of the run is scanned by the lanes of the warp together (scan_run_coop). Most scans end
// within a few rules (at the first match or the first rule that cannot beat the current best).
constexpr uint32_t kCoopAfter = 32;

// Scan the runs (or run remainders) of every lane of the calling group (the lanes that are
// executing this call together) cooperatively: for each member's run in turn, the group reads consecutive rules of it
// in one coalesced step per group size (lane of rank k takes rule base + k), and two ballots find
// the first rule in run order that matches or that no longer beats the member's current best (the
// run is priority-sorted, so the scan ends there). Each lane gets its own run's outcome: the
// same rule, the same improvement of `best` and the same count of rule reads as a serial scan.
// Control flow is uniform across the group, so every shuffle and ballot sees all its lanes.
__device__ __forceinline__ bool scan_run_coop(const Tables &tb, uint32_t run_start, uint32_t run_len, uint32_t t,
                                           const Hdr &h, Best &best, Counters &c) {
    const uint32_t grp = __activemask();
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t rank = __popc(grp & ((1u << lane) - 1u));
    const uint32_t g = __popc(grp);
    bool mine = false;
    for (uint32_t pending = grp; pending; pending &= pending - 1) {
        const int leader = __ffs(pending) - 1;
        const uint32_t start = __shfl_sync(grp, run_start, leader), len = __shfl_sync(grp, run_len, leader);
        const Hdr hl{__shfl_sync(grp, h.sip, leader), __shfl_sync(grp, h.dip, leader), __shfl_sync(grp, h.sp, leader),
                     __shfl_sync(grp, h.dp, leader), __shfl_sync(grp, h.proto, leader)};
        const uint32_t bprio = __shfl_sync(grp, best.prio, leader), bid = __shfl_sync(grp, best.id, leader);
        uint32_t reads = len, found = kEmpty;  // found: run index of the matching rule
        for (uint32_t base = 0; base < len; base += g) {
            const uint32_t j = base + rank;
            bool stop = false, match = false;
            DRule r{};
            if (j < len) {
                if (TANG_INDEX_OK(tb, start + j < tb.pool_size)) {
                    r = load_rule(tb.rules + start + j);
                    stop = !(r.prio < bprio || (r.prio == bprio && r.id < bid));
                    match = !stop && rule_match(r, hl);
                } else {
                    stop = true;  // checked build: index out of range, the access is skipped
                }
            }
            const uint32_t ev = __ballot_sync(grp, stop || match);
            if (ev) {
                const int first = __ffs(ev) - 1;  // lowest lane = lowest rank = earliest rule
                const uint32_t jf = base + __popc(grp & ((1u << first) - 1u));
                reads = jf + 1;
                if (__shfl_sync(grp, uint32_t(match), first)) {
                    found = jf;
                    const uint32_t fprio = __shfl_sync(grp, r.prio, first), fid = __shfl_sync(grp, r.id, first),
                                   fcf = __shfl_sync(grp, r.cf, first);
                    if (int(lane) == leader) best = Best{fprio, fid, start + jf, fcf, t};
                }
                break;
            }
        }
        if (int(lane) == leader) {
            c.rule_reads += reads;
            mine = found != kEmpty;
        }
    }
    return mine;
}

// Probe tuple t with the header truncated to the tuple's lengths (§4.3); scan the run under
// that key in (priority, id) order and stop at the first match or at the first rule that does
// not beat the current best. Returns true if `best` improved.
__device__ __forceinline__ bool probe_tuple(const Tables &tb, const TupleDesc &d, uint32_t t, const Hdr &h,
                                            Best &best, Counters &c, bool coop) {
    const uint32_t ks = h.sip & d.mask_s, kd = h.dip & d.mask_d;
    const uint32_t start = uint32_t(fmix64((uint64_t(ks) << 32) | kd)) & d.slot_mask;
    for (uint32_t i = 0; i <= d.max_probe; ++i) {
        const uint32_t si = d.slot_base + ((start + i) & d.slot_mask);
        if (!TANG_INDEX_OK(tb, si < tb.slot_cap)) return false;
        uint4 s = __ldg(reinterpret_cast<const uint4 *>(tb.slots + si));
        c.slot_reads++;
        if (s.z == kEmpty) return false;
        if (s.x == ks && s.y == kd) {
            const uint32_t serial_len = coop && s.w > kCoopAfter ? kCoopAfter : s.w;
            for (uint32_t j = 0; j < serial_len; ++j) {
                if (!TANG_INDEX_OK(tb, s.z + j < tb.pool_size)) return false;
                DRule r = load_rule(tb.rules + s.z + j);
                c.rule_reads++;
                if (!beats(r.prio, r.id, best)) return false;
                if (rule_match(r, h)) {
                    best = Best{r.prio, r.id, s.z + j, r.cf, t};
                    return true;
                }
            }
            if (serial_len < s.w) return scan_run_coop(tb, s.z + serial_len, s.w - serial_len, t, h, best, c);
            return false;
        }
    }
    return false;
}

// Full exact search of one header. `tuples` / `order` may point to shared-memory copies.
// pred outside [0, T) means "no prediction". Returns true if the predicted tuple held a match.
// mode bit kSearchPaper: the post-verification exactly as §5.1.1 states it, kept for measurement:
// a match in the predicted tuple is returned without the conflict-set probes (so it may be a
// lower-priority rule, the uncorrected case of §5.1.1 and §8); a miss still searches the remaining
// tuples in order. Bit kSearchSerial: every run is scanned by its own thread (no cooperative scan
// of long runs), for measurement; the result is the same. (The bits are defined in internal.h.)
__device__ __forceinline__ bool search_packet(const Tables &tb, const TupleDesc *tuples, const uint16_t *order,
                                              const Hdr &h, int pred, Best &best, Counters &c, int mode = 0) {
    const uint32_t T = tb.T;
    const bool paper = (mode & kSearchPaper) != 0, coop = (mode & kSearchSerial) == 0;
    best = Best{0xFFFFFFFFu, 0xFFFFFFFFu, kEmpty, 0u, 0u};
    bool hit = false;
    if (uint32_t(pred) < T) {
        c.probes++;
        hit = probe_tuple(tb, tuples[pred], uint32_t(pred), h, best, c, coop);
        if (hit && paper) return true;
    }
    // After a hit r: only tuples in conflict(r) can hold a better match. After a miss: all.
    uint32_t cf0 = 0xFFFFFFFFu;
    const uint32_t *cfw = nullptr;
    if (hit) {
        if (tb.cw == 1)
            cf0 = best.cf;
        else if (TANG_INDEX_OK(tb, best.cf < tb.cword_rows))
            cfw = tb.cwords + size_t(best.cf) * tb.cw;
        else
            return hit;
    }
    for (uint32_t k = 0; k < T; ++k) {
        const uint32_t t = order[k];
        if (!TANG_INDEX_OK(tb, t < T)) break;
        if (int(t) == pred) continue;
        if (hit) {
            uint32_t w = cfw ? __ldg(cfw + (t >> 5)) : cf0;
            if (!((w >> (t & 31)) & 1u)) continue;
        }
        const TupleDesc d = tuples[t];
        // tuples come in ascending best (priority, id): none from here on can win
        if (!beats(d.min_prio, d.min_id, best)) break;
        c.probes++;
        probe_tuple(tb, d, t, h, best, c, coop);
    }
    return hit;
}

}  // namespace tang
