// Stage-2 kernels: exact tuple-space search (§5.1.1 two-stage classification with the
// conflict-set certificate), conflict-set construction and maintenance, and the run edits of the
// immediate-update path (§5.2.1).
#include "search_dev.cuh"

namespace tang {

constexpr int kSmemTuples = 64;  // tuple descriptors staged in shared memory when T <= 64

__device__ __forceinline__ void warp_add(unsigned long long *dst, uint32_t v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, (unsigned long long)v);
}

// One thread per packet; grid-stride. Tuple descriptors and the search order are staged in
// shared memory (T <= 64), so a probe costs one slot load plus one 32-byte load per rule read.
template <int THREADS, bool STATS>
__global__ void __launch_bounds__(THREADS) k_search(const Tables *__restrict__ desc, const tang_header *__restrict__ hdr,
                                                const int32_t *__restrict__ pred, uint32_t n,
                                                uint32_t *__restrict__ ids, DevStats *stats, int mode) {
    __shared__ TupleDesc s_tuples[kSmemTuples];
    __shared__ uint16_t s_order[kSmemTuples];
    const Tables tb = *desc;
    const TupleDesc *tuples = tb.tuples;
    const uint16_t *order = tb.order;
    if (tb.T <= kSmemTuples) {
        for (uint32_t i = threadIdx.x; i < tb.T; i += blockDim.x) {
            s_tuples[i] = tb.tuples[i];
            s_order[i] = tb.order[i];
        }
        __syncthreads();
        tuples = s_tuples;
        order = s_order;
    }
    uint32_t st_pk = 0, st_match = 0, st_correct = 0, st_hit = 0, st_fb = 0;
    Counters c{0, 0, 0};
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const Hdr h = load_header(hdr + i);
        // the prediction: from its own array, from this packet's entry of ids (read before the
        // same thread overwrites it), or none
        const int p = pred ? __ldg(pred + i) : (mode & kSearchPredInIds) ? int(ids[i]) : -1;
        Best best;
        const bool hit = search_packet(tb, tuples, order, h, p, best, c, mode & (kSearchPaper | kSearchSerial));
        ids[i] = best.id;
        if (STATS) {
            st_pk++;
            const bool m = best.id != 0xFFFFFFFFu;
            st_match += m;
            st_correct += m && int(best.tuple) == p;
            st_hit += hit;
            st_fb += !hit;
        }
    }
    if (STATS) {
        warp_add(&stats->packets, st_pk);
        warp_add(&stats->matched, st_match);
        warp_add(&stats->nn_correct, st_correct);
        warp_add(&stats->pred_hit, st_hit);
        warp_add(&stats->fallback, st_fb);
        warp_add(&stats->probes, c.probes);
        warp_add(&stats->rule_reads, c.rule_reads);
        warp_add(&stats->slot_reads, c.slot_reads);
    }
}

cudaError_t launch_search(const Tables *d_desc, uint32_t T, uint32_t cw, const tang_header *h, const int32_t *tuple,
                          uint32_t n, uint32_t *ids, DevStats *stats, const TuneEntry *tune, cudaStream_t st,
                          int mode) {
    (void)T;
    (void)cw;
    if (n == 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int threads = tune && tune->search_threads ? tune->search_threads : 256;
    const int bps = tune && tune->search_bps ? tune->search_bps : 8;
    uint32_t blocks = (n + threads - 1) / threads;
    const uint32_t cap = uint32_t(sms) * uint32_t(bps);
    if (blocks > cap) blocks = cap;
#define TANG_SEARCH_LAUNCH(TH)                                                                     \
    if (stats)                                                                                     \
        k_search<TH, true><<<blocks, TH, 0, st>>>(d_desc, h, tuple, n, ids, stats, mode);                 \
    else                                                                                           \
        k_search<TH, false><<<blocks, TH, 0, st>>>(d_desc, h, tuple, n, ids, stats, mode);
    if (threads == 128) {
        TANG_SEARCH_LAUNCH(128)
    } else if (threads == 512) {
        TANG_SEARCH_LAUNCH(512)
    } else {
        TANG_SEARCH_LAUNCH(256)
    }
#undef TANG_SEARCH_LAUNCH
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Conflict sets: conflict(r) = { tuple(r') : r' beats r and r' overlaps r }.
// ---------------------------------------------------------------------------------------

// Two rules share a header: prefixes agree on the shorter length, port ranges intersect,
// protocols agree unless one is a wildcard.
__device__ __forceinline__ bool rules_overlap(const DRule &a, const DRule &b) {
    const uint32_t ls = min(meta_sip_len(a.meta), meta_sip_len(b.meta));
    const uint32_t ld = min(meta_dip_len(a.meta), meta_dip_len(b.meta));
    bool ok = ((a.sip ^ b.sip) & prefix_mask(ls)) == 0;
    ok &= ((a.dip ^ b.dip) & prefix_mask(ld)) == 0;
    ok &= ((a.sp & 0xFFFFu) <= (b.sp >> 16)) & ((b.sp & 0xFFFFu) <= (a.sp >> 16));
    ok &= ((a.dp & 0xFFFFu) <= (b.dp >> 16)) & ((b.dp & 0xFFFFu) <= (a.dp >> 16));
    ok &= !(meta_proto_exact(a.meta) & meta_proto_exact(b.meta) & (meta_proto(a.meta) != meta_proto(b.meta)));
    return ok;
}

// Rules are given in ascending (priority, id): every j < i beats i. Block b owns 256
// consecutive rules (heaviest chunks first) and streams all better rules through shared
// memory. A thread stops early once its set holds every tuple.
__global__ void __launch_bounds__(256) k_conflict_build(const DRule *__restrict__ sorted,
                                                        const uint32_t *__restrict__ sorted_pos, uint32_t n,
                                                        DRule *pool, uint32_t *cwords, uint32_t cw, uint32_t full) {
    __shared__ DRule tile[256];
    const uint32_t chunk = gridDim.x - 1 - blockIdx.x;
    const uint32_t i = chunk * 256 + threadIdx.x;
    const bool valid = i < n;
    DRule me = valid ? sorted[i] : DRule{0, 0, 0, 0, 0, 0, 0, 0};
    uint32_t cf = 0;
    bool done = !valid;
    const uint32_t jend = min(n, chunk * 256 + 256);
    for (uint32_t j0 = 0; j0 < jend; j0 += 256) {
        if (__syncthreads_and(done)) break;
        if (j0 + threadIdx.x < jend) tile[threadIdx.x] = sorted[j0 + threadIdx.x];
        __syncthreads();
        if (!done) {
            const uint32_t lim = i > j0 ? min(256u, i - j0) : 0u;
            for (uint32_t jj = 0; jj < lim; ++jj) {
                const DRule &o = tile[jj];
                if (rules_overlap(me, o)) {
                    const uint32_t t = meta_tuple(o.meta);
                    if (cw == 1)
                        cf |= 1u << t;
                    else
                        atomicOr(cwords + size_t(me.cf) * cw + (t >> 5), 1u << (t & 31));
                }
            }
            if (cw == 1 && cf == full) done = true;
        }
    }
    if (valid && cw == 1) pool[sorted_pos[i]].cf = cf;
}

cudaError_t launch_conflict_build(const DRule *sorted, const uint32_t *sorted_pos, uint32_t n, DRule *pool,
                                  uint32_t *cwords, uint32_t cw, uint32_t T, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const uint32_t full = T >= 32 ? 0xFFFFFFFFu : ((1u << T) - 1u);
    k_conflict_build<<<(n + 255) / 256, 256, 0, st>>>(sorted, sorted_pos, n, pool, cwords, cw, full);
    return cudaGetLastError();
}

// Insert maintenance: the new rule at `new_pos` gets the tuples of every better overlapping
// rule; every worse overlapping rule gets the new rule's tuple. Dead records have priority
// 0xFFFFFFFF and never beat anything.
__global__ void k_conflict_insert(const Tables *__restrict__ desc, uint32_t pool_size, uint32_t new_pos,
                                  uint32_t cw) {
    const Tables tb = *desc;
    const DRule nr = tb.rules[new_pos];
    const uint32_t tn = meta_tuple(nr.meta);
    uint32_t mine = 0;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < pool_size; p += gridDim.x * blockDim.x) {
        if (p == new_pos) continue;
        const DRule r = tb.rules[p];
        if (r.prio == 0xFFFFFFFFu) continue;
        if (!rules_overlap(r, nr)) continue;
        const uint32_t t = meta_tuple(r.meta);
        if (r.prio < nr.prio || (r.prio == nr.prio && r.id < nr.id)) {
            if (cw == 1)
                mine |= 1u << t;
            else
                atomicOr(tb.cwords + size_t(nr.cf) * cw + (t >> 5), 1u << (t & 31));
        } else {
            if (cw == 1)
                atomicOr(&tb.rules[p].cf, 1u << tn);
            else
                atomicOr(tb.cwords + size_t(r.cf) * cw + (tn >> 5), 1u << (tn & 31));
        }
    }
    if (cw == 1) {
        for (int o = 16; o; o >>= 1) mine |= __shfl_xor_sync(0xFFFFFFFFu, mine, o);
        if ((threadIdx.x & 31) == 0 && mine) atomicOr(&tb.rules[new_pos].cf, mine);
    }
}

cudaError_t launch_conflict_insert(const Tables *d_desc, uint32_t pool_size, uint32_t new_pos, uint32_t cw,
                                   cudaStream_t st) {
    uint32_t blocks = (pool_size + 255) / 256;
    if (blocks > 1184) blocks = 1184;
    if (blocks == 0) blocks = 1;
    k_conflict_insert<<<blocks, 256, 0, st>>>(d_desc, pool_size, new_pos, cw);
    return cudaGetLastError();
}

// Shift the tail of a run by one record: dir > 0 moves [pos, len) up (insert at pos), dir < 0
// moves [pos+1, len) down (delete at pos). One block; chunks are processed in the order that
// never overwrites an unread record, with a barrier between each chunk's reads and writes.
__global__ void k_run_shift(DRule *pool, uint32_t start, uint32_t len, uint32_t pos, int dir) {
    DRule *run = pool + start;
    if (dir > 0) {
        for (int64_t hi = len; hi > int64_t(pos); hi -= blockDim.x) {
            const int64_t lo = hi - int64_t(blockDim.x) > int64_t(pos) ? hi - int64_t(blockDim.x) : int64_t(pos);
            const int64_t k = lo + threadIdx.x;
            DRule v;
            const bool act = k < hi;
            if (act) v = run[k];
            __syncthreads();
            if (act) run[k + 1] = v;
            __syncthreads();
        }
    } else {
        for (int64_t lo = int64_t(pos) + 1; lo < int64_t(len); lo += blockDim.x) {
            const int64_t hi = lo + int64_t(blockDim.x) < int64_t(len) ? lo + int64_t(blockDim.x) : int64_t(len);
            const int64_t k = lo + threadIdx.x;
            DRule v;
            const bool act = k < hi;
            if (act) v = run[k];
            __syncthreads();
            if (act) run[k - 1] = v;
            __syncthreads();
        }
    }
}

cudaError_t launch_run_shift(DRule *pool, uint32_t start, uint32_t len, uint32_t pos, int dir, cudaStream_t st) {
    k_run_shift<<<1, 256, 0, st>>>(pool, start, len, pos, dir);
    return cudaGetLastError();
}

__global__ void k_run_copy(DRule *pool, uint32_t from, uint32_t to, uint32_t len) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < len; k += gridDim.x * blockDim.x)
        pool[to + k] = pool[from + k];
}

cudaError_t launch_run_copy(DRule *pool, uint32_t from, uint32_t to, uint32_t len, cudaStream_t st) {
    if (len == 0) return cudaSuccess;
    uint32_t blocks = (len + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    k_run_copy<<<blocks, 256, 0, st>>>(pool, from, to, len);
    return cudaGetLastError();
}

}  // namespace tang
