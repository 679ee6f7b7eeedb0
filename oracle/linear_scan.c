/*
 * ORACLE (test infrastructure only) -- plain CPU packet classification by linear scan.
 *
 * Computes the definition of §2.1 of the paper: a packet P is classified to the
 * highest-priority rule R whose every field condition holds:
 *   - SIP / DIP: prefix match on the rule's own prefix length (length 0 matches all),
 *   - SP / DP:   inclusive range lo <= p <= hi,
 *   - PRO:       exact match, or wildcard.
 * Priority: a smaller number is a higher priority (Table 1); equal priorities are ordered by
 * rule id. A packet that no rule matches gets 0xFFFFFFFF.
 *
 * Rules are sorted once by (priority, id) and scanned in that order; the first match is the
 * answer. Nothing here is shared with the CUDA path: the record layouts are re-declared below.
 * Only tests, the smoke check and the benchmark's CPU-baseline leg may load this file.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint32_t sip, dip;
    uint16_t sp, dp;
    uint8_t proto, pad[3];
} o_header;

typedef struct {
    uint32_t sip, dip;
    uint16_t sp_lo, sp_hi, dp_lo, dp_hi;
    uint8_t sip_len, dip_len, proto, proto_wild;
    uint32_t priority, id, reserved;
} o_rule;

_Static_assert(sizeof(o_header) == 16, "header is 16 bytes");
_Static_assert(sizeof(o_rule) == 32, "rule is 32 bytes");

#define O_NO_MATCH 0xFFFFFFFFu

/* Top `len` bits set. len == 0 gives 0 (a 32-bit shift by 32 would be undefined). */
static uint32_t prefix_mask(unsigned len) {
    if (len == 0) return 0u;
    return 0xFFFFFFFFu << (32u - len);
}

static int rule_matches(const o_rule *r, const o_header *p) {
    if (((p->sip ^ r->sip) & prefix_mask(r->sip_len)) != 0) return 0;
    if (((p->dip ^ r->dip) & prefix_mask(r->dip_len)) != 0) return 0;
    if (p->sp < r->sp_lo || p->sp > r->sp_hi) return 0;
    if (p->dp < r->dp_lo || p->dp > r->dp_hi) return 0;
    if (!r->proto_wild && p->proto != r->proto) return 0;
    return 1;
}

typedef struct {
    uint32_t priority, id;
    uint64_t index; /* position in the caller's array */
} o_order;

static int order_cmp(const void *a, const void *b) {
    const o_order *x = (const o_order *)a, *y = (const o_order *)b;
    if (x->priority != y->priority) return x->priority < y->priority ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

typedef struct {
    const o_rule *sorted;
    const uint64_t *orig_index;
    uint64_t n_rules;
    const o_header *packets;
    uint64_t begin, end;
    uint32_t *out_id;
    int64_t *out_index;
} o_job;

static void *scan_range(void *arg) {
    o_job *job = (o_job *)arg;
    for (uint64_t i = job->begin; i < job->end; ++i) {
        uint32_t id = O_NO_MATCH;
        int64_t idx = -1;
        for (uint64_t k = 0; k < job->n_rules; ++k) {
            if (rule_matches(&job->sorted[k], &job->packets[i])) {
                id = job->sorted[k].id;
                idx = (int64_t)job->orig_index[k];
                break;
            }
        }
        job->out_id[i] = id;
        if (job->out_index) job->out_index[i] = idx;
    }
    return NULL;
}

/*
 * Classify n packets. out_id[i] = id of the matched rule or 0xFFFFFFFF; out_index (may be NULL)
 * receives the matched rule's position in `rules`, or -1. `threads` <= 0 means 1.
 * Returns 0, or -1 on allocation failure.
 */
int oracle_classify(const o_rule *rules, uint64_t n_rules, const o_header *packets, uint64_t n,
                    uint32_t *out_id, int64_t *out_index, int threads) {
    if (threads <= 0) threads = 1;
    o_order *ord = (o_order *)malloc(sizeof(o_order) * (n_rules ? n_rules : 1));
    o_rule *sorted = (o_rule *)malloc(sizeof(o_rule) * (n_rules ? n_rules : 1));
    uint64_t *orig = (uint64_t *)malloc(sizeof(uint64_t) * (n_rules ? n_rules : 1));
    if (!ord || !sorted || !orig) {
        free(ord); free(sorted); free(orig);
        return -1;
    }
    for (uint64_t k = 0; k < n_rules; ++k) {
        ord[k].priority = rules[k].priority;
        ord[k].id = rules[k].id;
        ord[k].index = k;
    }
    qsort(ord, n_rules, sizeof(o_order), order_cmp);
    for (uint64_t k = 0; k < n_rules; ++k) {
        sorted[k] = rules[ord[k].index];
        orig[k] = ord[k].index;
    }
    free(ord);

    if ((uint64_t)threads > n) threads = n ? (int)n : 1;
    pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * threads);
    o_job *jobs = (o_job *)malloc(sizeof(o_job) * threads);
    if (!tid || !jobs) {
        free(tid); free(jobs); free(sorted); free(orig);
        return -1;
    }
    uint64_t chunk = (n + threads - 1) / threads;
    for (int t = 0; t < threads; ++t) {
        jobs[t].sorted = sorted;
        jobs[t].orig_index = orig;
        jobs[t].n_rules = n_rules;
        jobs[t].packets = packets;
        jobs[t].begin = (uint64_t)t * chunk < n ? (uint64_t)t * chunk : n;
        jobs[t].end = jobs[t].begin + chunk < n ? jobs[t].begin + chunk : n;
        jobs[t].out_id = out_id;
        jobs[t].out_index = out_index;
    }
    int spawned = 0;
    for (int t = 1; t < threads; ++t) {
        if (pthread_create(&tid[t], NULL, scan_range, &jobs[t]) != 0) break;
        spawned = t;
    }
    scan_range(&jobs[0]);
    for (int t = 1; t <= spawned; ++t) pthread_join(tid[t], NULL);
    for (int t = spawned + 1; t < threads; ++t) scan_range(&jobs[t]); /* threads that failed to spawn */
    free(tid); free(jobs); free(sorted); free(orig);
    return 0;
}
