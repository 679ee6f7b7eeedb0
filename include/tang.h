/*
 * tang.h -- C ABI of the B300 (sm_103a) TaNG packet classifier.
 *
 * TaNG classifies a packet header against a multi-field ruleset in two stages (§5.1.1): a
 * residual MLP (§6.1) predicts the tuple of the tuple space (§4.3) that holds the answer, then
 * that tuple's hash table is probed, the candidates are verified field by field, and the
 * highest-priority matching rule is returned. This library makes the post-verification exact
 * (the paper's is not: §5.1.1, §8): after a hit in the predicted tuple it also probes every tuple
 * that holds a better rule overlapping the hit, and after a miss it searches all other tuples in
 * ascending order of their best priority. The returned rule id is therefore always the one the
 * definition of §2.1 gives, whatever the network predicts.
 *
 * Conventions for every entry point:
 *   - Return value: TANG_OK (0) or a negative TANG_E* code. No C++ exception crosses the ABI.
 *     tang_last_error(ctx) describes the last failure on that context (thread-unsafe string).
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA global memory on the
 *     context's device. Entry points that accept either say so and take a TANG_MEM_* flag.
 *   - The caller owns every buffer it passes in; the library copies what it keeps.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the context's own stream.
 *     Device-side work is enqueued on that stream; results are valid once it is synchronised
 *     unless the call says it synchronises itself.
 *   - A context is single-threaded: do not call into one context from two threads at once
 *     (the serving engine's own thread is the exception and is internal).
 */
#ifndef TANG_H
#define TANG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------------------------------
 * Records (§2.1). All fields little-endian, host byte order (no network byte order).
 * ------------------------------------------------------------------------------------- */

/* One 5-field packet header, 16 bytes. */
typedef struct tang_header {
    uint32_t sip, dip; /* source / destination IPv4 address */
    uint16_t sp, dp;   /* source / destination port */
    uint8_t proto;     /* IP protocol */
    uint8_t pad[3];    /* ignored */
} tang_header;

/* One rule, 32 bytes. SIP/DIP are prefixes of length 0..32 (bits below the length are
 * ignored); SP/DP are inclusive ranges lo <= p <= hi; the protocol matches exactly unless
 * proto_wild != 0. A smaller `priority` is a higher priority (Table 1); equal priorities are
 * ordered by `id`. `id` must be unique within a ruleset and != TANG_NO_MATCH. */
typedef struct tang_rule {
    uint32_t sip, dip;
    uint16_t sp_lo, sp_hi, dp_lo, dp_hi;
    uint8_t sip_len, dip_len, proto, proto_wild;
    uint32_t priority, id;
    uint32_t reserved; /* must be 0 */
} tang_rule;

#define TANG_NO_MATCH 0xFFFFFFFFu /* id returned when no rule matches */

/* Error codes. */
#define TANG_OK 0
#define TANG_EINVAL (-1)       /* bad argument, malformed rule or model blob */
#define TANG_ENOMEM (-2)       /* device allocation failed or the memory pool refused it */
#define TANG_ETABLEFULL (-3)   /* a table cannot grow (e.g. more than 2047 tuples) */
#define TANG_ENOTFOUND (-4)    /* unknown ruleset handle or rule id */
#define TANG_EDEVICE (-5)      /* a CUDA call failed */
#define TANG_ETIMEOUT (-6)     /* a bounded wait ran out */
#define TANG_EUNSUPPORTED (-7) /* valid request this build cannot serve (e.g. shape too large) */
#define TANG_EEXIST (-8)       /* duplicate rule id */
#define TANG_EAGAIN (-9)       /* request not finished yet (serving poll) */

/* ---------------------------------------------------------------------------------------
 * Context
 * ------------------------------------------------------------------------------------- */
typedef struct tang_ctx tang_ctx;

/* Create a context on CUDA device `device`. Every device allocation the context makes
 * (tables, model weights, scratch, serving buffers) is admitted against `pool_bytes`; 0 means
 * "no cap". Errors: TANG_EINVAL, TANG_EDEVICE. */
int tang_create(int device, size_t pool_bytes, tang_ctx **out);

/* Synchronise, stop the serving engine, free everything. NULL is ignored. */
void tang_destroy(tang_ctx *ctx);

/* Text of the last error on this context ("" if none). Owned by the context. */
const char *tang_last_error(tang_ctx *ctx);

/* Device bytes currently admitted against the pool, and the cap (0 = none). */
int tang_memory_usage(tang_ctx *ctx, size_t *used, size_t *cap);

/* ---------------------------------------------------------------------------------------
 * Rulesets: tuple space (§4.3) + exactness certificate
 * ------------------------------------------------------------------------------------- */

/* Build the tuple space of `n` host rules and upload it. Tuples are the distinct
 * (sip_len, dip_len) pairs (§4.3: 5-field tuples are built from SIP and DIP), indexed in
 * order of first appearance over the rules sorted by (priority, id); a (0,0) tuple is
 * appended if absent so that restricted insertion (§5.2.1) always has a candidate.
 * Each tuple gets an open-addressing hash table keyed by the header truncated to the
 * tuple's lengths; the rules under one key form a run sorted by (priority, id).
 * Per rule, the conflict set (tuples holding a better rule that overlaps it) is computed
 * on the GPU. n may be 0. Synchronous. On success *rs_out is the ruleset handle.
 * Errors: TANG_EINVAL (len > 32, lo > hi, id == TANG_NO_MATCH), TANG_EEXIST (duplicate id),
 * TANG_ETABLEFULL (> 2047 tuples), TANG_ENOMEM. */
int tang_load_ruleset(tang_ctx *ctx, const tang_rule *rules, uint32_t n, uint32_t *rs_out);

/* Free a ruleset and its model. */
int tang_unload_ruleset(tang_ctx *ctx, uint32_t rs);

typedef struct tang_ruleset_info {
    uint32_t n_rules;      /* live rules */
    uint32_t n_tuples;     /* T: the network's class count C must equal this */
    uint32_t conflict_words; /* 32-bit words per conflict set: ceil(T/32) */
    uint32_t n_keys;       /* distinct (tuple, key) runs */
    uint64_t device_bytes; /* bytes held by the tables (not the model) */
    double build_ms;       /* host build + upload + conflict kernel */
} tang_ruleset_info;

int tang_ruleset_info_get(tang_ctx *ctx, uint32_t rs, tang_ruleset_info *out);

/* Tuple t's prefix lengths and best (priority, id), for t < n_tuples; host outputs. */
int tang_tuple_get(tang_ctx *ctx, uint32_t rs, uint32_t t, uint32_t *sip_len, uint32_t *dip_len,
                   uint32_t *min_priority, uint32_t *min_id);

/* For a rule id: the tuple it is stored in and its conflict set (conflict_words words,
 * bit t set if tuple t holds a better rule that overlaps this rule). Host outputs.
 * Synchronises the context stream. TANG_ENOTFOUND for an unknown id. */
int tang_rule_conflicts(tang_ctx *ctx, uint32_t rs, uint32_t id, uint32_t *tuple, uint32_t *words);

/* ---------------------------------------------------------------------------------------
 * Model (§6.1): input FC (S=7 -> N) + k residual blocks (Eq. 1) + output FC (N -> C)
 * ------------------------------------------------------------------------------------- */

/* Precisions of the network's N x N layers. */
#define TANG_FP32 0 /* FP32 CUDA-core GEMMs */
#define TANG_BF16 1 /* tcgen05 BF16 MMA, FP32 accumulation */
#define TANG_FP8 2  /* tcgen05 FP8 E4M3 MMA, FP32 accumulation; weight scales per hidden layer and per output column of the output layer, power-of-two activation scales per layer input */

/* Model blob (little-endian), produced by tang_train() or by the caller:
 *   tang_model_header
 *   float act_amax[2*blocks + 1]  -- max |activation| entering each tensor-core layer, in
 *                                    order h0, u1, h1, u2, h2, ..., uk, hk (used for FP8;
 *                                    all zero = "not calibrated", FP8 then refused)
 *   float params[] in this order, each row-major with the x.W convention of Eq. 1
 *     W0[S][N] b0[N]  { W1[N][N] b1[N] W2[N][N] b2[N] } x blocks  Wc[N][C] bc[C]
 * W0 acts on the raw 16-bit segment values of §6.2 (SIP hi, SIP lo, DIP hi, DIP lo, SP, DP,
 * PRO). */
#define TANG_MODEL_MAGIC 0x474E4154u /* "TANG" */
typedef struct tang_model_header {
    uint32_t magic;   /* TANG_MODEL_MAGIC */
    uint32_t version; /* 1 */
    uint32_t S, N, blocks, C;
    uint32_t reserved[10];
} tang_model_header; /* 64 bytes */

/* Validate and upload a model for ruleset `rs`; keeps an FP32 copy and derives the BF16 and
 * (if calibrated) FP8 copies. Requires C == n_tuples, S == 7. The tensor-core paths further
 * require N == 256 or 512 and 1 <= blocks <= 31 (other shapes use the FP32 path only); the
 * fused kernel takes any C (its output layer runs in 256-column chunks).
 * Replaces a previous model of the ruleset. Synchronous: waits for all work on the device.
 * Hot swap (§5.2.2 deploys retrained weights while classification goes on): when the previous
 * model has the same S, N, blocks, C and FP8 calibration state, the new weights are written into
 * its device buffers, so CUDA graphs captured with TANG_GRAPH stay valid and their next replay
 * uses the new model; otherwise the graphs are dropped and re-captured on their next call.
 * Errors: TANG_EINVAL (bad magic, sizes, C != T), TANG_ENOMEM. */
int tang_load_model(tang_ctx *ctx, uint32_t rs, const void *blob, size_t bytes);

/* ---------------------------------------------------------------------------------------
 * Classification (§5.1.1)
 * ------------------------------------------------------------------------------------- */

/* Path selection (flags & TANG_PATH_MASK). */
#define TANG_PATH_FUSED_BF16 0x0 /* one persistent kernel: encode + BF16 MLP + search */
#define TANG_PATH_FUSED_FP8 0x1  /* same with FP8 layers */
#define TANG_PATH_PLAIN_FP32 0x2 /* one kernel per stage, FP32 CUDA-core MLP */
#define TANG_PATH_STAGED_BF16 0x3 /* BF16 MLP kernel, then a separate search kernel */
#define TANG_PATH_NO_NN 0x4      /* no network: every tuple in ascending best priority */
#define TANG_PATH_STAGED_FP8 0x5
#define TANG_PATH_MASK 0xF
/* Where `headers` / `ids` live. */
#define TANG_MEM_DEVICE 0x00      /* both device pointers */
#define TANG_MEM_HOST 0x10        /* both host pointers (pageable or pinned); the call pipelines
                                     H2D, compute and D2H on side streams and returns when `ids`
                                     is filled (synchronous) */
/* Other flags. */
#define TANG_GRAPH 0x100          /* DEVICE mode: capture the launch sequence in a CUDA graph
                                     keyed by (ruleset, path, n, pointers, stream) and replay it */
/* Tensor-core kernel variant (fused and staged paths, and tang_infer's precision argument);
 * no bit = the autotuned choice, else the library default. */
#define TANG_FUSED_N256 0x2000    /* one CTA per SM, 256-wide MMAs, single-buffered accumulator */
#define TANG_FUSED_PAIR 0x1000    /* the same kernel on CTA pairs (cta_group::2): every MMA covers two
                                     SMs' tiles (M = 256) and each SM streams half of each weight tile */
#define TANG_FUSED_SPLIT 0x3000   /* fused paths only: the same network (the N=256 kernel without its
                                     search warps) writes each packet's predicted tuple into `ids`,
                                     then the search kernel, with the whole GPU, reads it there and
                                     overwrites it with the rule id. No scratch memory. Faster than the
                                     one persistent kernel (128 search threads per SM) when the ruleset
                                     holds long runs under one key; the autotuner measures both. */
#define TANG_VARIANT_MASK 0x3000
/* Post-verification exactly as §5.1.1 prints it, for measurement only: a match in the predicted
 * tuple is returned at once, without the conflict-set probes, so a packet can get a
 * lower-priority rule when the network predicts a wrong tuple that also holds a match (the case
 * §5.1.1 and §8 leave uncorrected); a miss still searches the other tuples in order. Combines
 * with every path; the default (flag clear) is the exact search. */
#define TANG_SEARCH_PAPER 0x4000
/* Scan every rule run with one thread, as the first builds did, instead of letting the lanes of a
 * warp scan a long run (past its first 32 rules under one key) together with coalesced reads; for
 * measurement. Ids and counters are the same either way. Combines with every path. */
#define TANG_SEARCH_SERIAL 0x8000

typedef struct tang_stats {
    uint64_t packets;       /* packets classified */
    uint64_t matched;       /* packets with a matching rule */
    uint64_t nn_correct;    /* matched packets whose predicted tuple holds the answer */
    uint64_t pred_hit;      /* predicted tuple had a matching rule */
    uint64_t fallback;      /* predicted tuple had no match: ordered search of the rest */
    uint64_t probes;        /* tuple hash-table probes (predicted tuple counts as one) */
    uint64_t rule_reads;    /* rule records compared */
    uint64_t slot_reads;    /* hash slots read */
} tang_stats;

/* Classify n headers into rule ids (ids[i] = matching rule's id or TANG_NO_MATCH).
 * The rule id never depends on the path or precision (exact post-verification).
 * DEVICE mode: asynchronous on `stream`. HOST mode: synchronous.
 * `stats` (may be NULL) receives counters for this call; passing it synchronises.
 * n == 0 is allowed. Errors: TANG_ENOTFOUND (rs), TANG_EINVAL (path needs a model that
 * is not loaded, bad flags, unaligned pointer), TANG_EUNSUPPORTED, TANG_EDEVICE. */
int tang_classify(tang_ctx *ctx, uint32_t rs, const tang_header *headers, uint32_t n, uint32_t *ids,
                  uint32_t flags, void *stream, tang_stats *stats);

/* Stage 1 alone (§5.1.1): run the network of ruleset rs over n device headers.
 * d_logits (device, n x C float, row-major; may be NULL) receives the output layer's logits;
 * d_tuple (device, n int32; may be NULL) the argmax (lowest index on ties).
 * precision: TANG_FP32 / TANG_BF16 / TANG_FP8, optionally OR-ed with a TANG_FUSED_* variant bit.
 * Asynchronous on `stream`. */
int tang_infer(tang_ctx *ctx, uint32_t rs, const tang_header *d_headers, uint32_t n, float *d_logits,
               int32_t *d_tuple, int precision, void *stream);

/* Stage 2 alone: exact search of n device headers given predicted tuples d_tuple (device,
 * n int32; NULL = no prediction, i.e. the ordered search over all tuples). Values outside
 * [0, T) are treated as "no prediction". Writes d_ids (device). `stats` as in classify. */
int tang_search(tang_ctx *ctx, uint32_t rs, const tang_header *d_headers, const int32_t *d_tuple, uint32_t n,
                uint32_t *d_ids, void *stream, tang_stats *stats);

/* tang_search with flags: 0 (exact search, same as tang_search), TANG_SEARCH_PAPER and / or
 * TANG_SEARCH_SERIAL.
 * Errors as tang_search, plus TANG_EINVAL for unknown flag bits. */
int tang_search_ex(tang_ctx *ctx, uint32_t rs, const tang_header *d_headers, const int32_t *d_tuple, uint32_t n,
                   uint32_t *d_ids, uint32_t flags, void *stream, tang_stats *stats);

/* Number of CUDA graphs the context holds for TANG_GRAPH replays. They are dropped when a
 * ruleset is unloaded, the scratch buffer grows, or a model of another shape replaces a
 * ruleset's model; a same-shape model swap (tang_load_model) keeps them. */
int tang_graph_count(tang_ctx *ctx, uint32_t *count);

/* The paper's CPU-GPU hybrid streaming framework (§5.1.2, Fig. 4), as a comparison pipeline:
 * host headers are batched; each batch is split into `streams` segments on as many CUDA streams;
 * the GPU runs only the network on them (stage 1; predicted tuples back to pinned host memory),
 * and `threads` host threads run the tuple-space search (stage 2) on a snapshot of the device
 * tables taken at the start of the call, double-buffered against the GPU's next batch.
 * The search is exact (flags 0, same ids as tang_classify) or the paper's own post-verification
 * (TANG_SEARCH_PAPER). headers / ids are host memory; synchronous. */
typedef struct tang_hybrid_cfg {
    uint32_t batch;     /* packets per batch (paper: 8192; 0 = 8192) */
    uint32_t streams;   /* CUDA streams per batch (paper: 4; 0 = 4; at most 16). FP32 runs its
                           segments in order on one stream (its kernels share a scratch buffer) */
    uint32_t threads;   /* host search threads (0 = all hardware threads) */
    uint32_t precision; /* TANG_FP32, TANG_BF16 or TANG_FP8 network */
    uint32_t flags;     /* 0 or TANG_SEARCH_PAPER */
    uint32_t reserved[3];
} tang_hybrid_cfg;
/* Errors: TANG_EINVAL (no model, bad precision or flags), TANG_EUNSUPPORTED (no tensor-core copy
 * for BF16/FP8), TANG_ENOTFOUND, TANG_ENOMEM, TANG_EDEVICE. `stats` (may be NULL) counts the
 * host search's work as tang_classify's counters do. */
int tang_classify_hybrid(tang_ctx *ctx, uint32_t rs, const tang_header *headers, uint32_t n, uint32_t *ids,
                         const tang_hybrid_cfg *cfg, tang_stats *stats);

/* Staged BF16 classification (the tensor-core network kernel, then the search kernel) for
 * callers that must not allocate device memory during a call: code running inside a custom
 * allocator or allocation hook, processes whose device memory is fixed at start-up, and
 * latency-bound loops that cannot take the device synchronisation cudaMalloc implies.
 * tang_classify may grow the context's scratch buffer with cudaMalloc; this entry point instead
 * passes the predicted tuples between the two kernels through a static device array of
 * TANG_NOALLOC_MAX_PACKETS int32 entries (4 MiB). The array belongs to the library's device
 * module: a GPU holds it from the moment that module is loaded there (at the latest when a
 * context is created on it) until the process exits. tang_create looks up the array's device
 * address, so this call loads no module and calls no cudaMalloc, cudaFree or allocating library
 * routine.
 * The paper has no counterpart; it is an addition of this library.
 *   d_headers: n device headers, 16-byte aligned; d_ids: n device outputs (same ids as
 *   tang_classify). Requires a loaded model with a tensor-core copy (see tang_load_model).
 *   All calls share the one array: calls whose kernels overlap on the GPU (on different
 *   streams, or from different contexts on the same device) race and must be serialised.
 *   Asynchronous on `stream` (NULL = the context's stream).
 * Errors: TANG_EINVAL (n > TANG_NOALLOC_MAX_PACKETS, unaligned or null buffers, no model),
 * TANG_EUNSUPPORTED (the model has no tensor-core copy), TANG_ENOTFOUND, TANG_EDEVICE. */
#define TANG_NOALLOC_MAX_PACKETS 1048576u
int tang_classify_noalloc(tang_ctx *ctx, uint32_t rs, const tang_header *d_headers, uint32_t n, uint32_t *d_ids,
                          void *stream);

/* ---------------------------------------------------------------------------------------
 * Immediate update (§5.2.1). Stream-ordered: every classify issued after the call (on any
 * stream) sees it, and it waits for every classification already issued against the ruleset
 * (on any stream) before it rewrites the tables, so those see the ruleset as it was. Work
 * captured into a CUDA graph by the caller is ordered by the caller. Neither call creates or
 * removes a tuple, so a loaded model stays valid.
 * ------------------------------------------------------------------------------------- */

/* Insert into the tuple with the rule's exact lengths, else into the first tuple of largest
 * length sum among those with lengths <= the rule's (the rule is truncated into it; its own
 * lengths are still verified). Updates the conflict sets of the affected rules on the GPU.
 * Errors: TANG_EINVAL, TANG_EEXIST (id already live), TANG_ENOMEM. */
int tang_insert_rule(tang_ctx *ctx, uint32_t rs, const tang_rule *rule);

/* Remove a live rule. Conflict sets of other rules are left as supersets (still exact).
 * Errors: TANG_ENOTFOUND. */
int tang_delete_rule(tang_ctx *ctx, uint32_t rs, uint32_t id);

/* The live rules of ruleset rs (after any inserts and deletes), in ascending (priority, id), as
 * host records: prefix values carry only their top `len` bits, the protocol of a wildcard rule is
 * 0. With out == NULL only *n_out (the live count) is set; else cap must be >= that count.
 * Together with a model blob this checkpoints a ruleset: tang_load_ruleset of the export builds
 * the same classifier (restricted-insertion placements become exact ones, as in a rebuild).
 * Errors: TANG_ENOTFOUND, TANG_EINVAL (cap too small). */
int tang_export_rules(tang_ctx *ctx, uint32_t rs, tang_rule *out, uint32_t cap, uint32_t *n_out);

/* Rules inserted since load whose lengths differ from their tuple's (the deferred-update
 * counter of §5.2.2). */
int tang_suboptimal_count(tang_ctx *ctx, uint32_t rs, uint64_t *count);


/* ---------------------------------------------------------------------------------------
 * Training (§6.2), all on the GPU with this library's own forward/backward kernels
 * ------------------------------------------------------------------------------------- */

typedef struct tang_train_cfg {
    uint32_t N;             /* neurons per FC layer (paper: 512) */
    uint32_t blocks;        /* residual blocks (paper: 6) */
    uint32_t batch;         /* minibatch (paper: 8192) */
    uint32_t epochs;        /* epochs per round (paper: 1000) */
    uint32_t max_rounds;    /* rounds of the alpha schedule */
    uint32_t decay_every;   /* epochs between lr decays (paper: 200) */
    float lr;               /* initial Adam learning rate (paper: 1e-3) */
    float decay;            /* lr factor per decay (paper: 0.1) */
    uint32_t alpha;         /* class-balance threshold (paper: 1000), x10 per failed round */
    float beta;             /* accuracy threshold (paper: 0.95) */
    float holdout;          /* fraction of labelled samples held out for the accuracy check */
    float time_budget_s;    /* stop training after this many seconds (0 = no limit) */
    uint64_t seed;          /* initialisation, shuffling, oversampling */
} tang_train_cfg;

typedef struct tang_train_report {
    uint32_t rounds, epochs_run, samples_labelled, samples_trained, classes_empty;
    uint32_t alpha_final;
    float final_loss, holdout_accuracy, train_seconds;
} tang_train_report;

/* Label n host sample headers with the tuple of their exact match (unmatched samples are
 * dropped), oversample every class below alpha, and train the network of §6.1 on it with
 * cross-entropy and Adam; repeat rounds with alpha x10 while holdout accuracy < beta (§6.2).
 * On success writes a model blob (calibrated FP8 amax included) to `blob` if *bytes is large
 * enough, and always sets *bytes to the blob size (call with blob == NULL to size it).
 * report may be NULL. Synchronous. */
int tang_train(tang_ctx *ctx, uint32_t rs, const tang_header *samples, uint32_t n, const tang_train_cfg *cfg,
               void *blob, size_t *bytes, tang_train_report *report);

/* Forward + backward of the mean cross-entropy for one batch, on the GPU (the trainer's
 * kernels), for gradient checks. params/grads are host float arrays in the blob's parameter
 * order (sizes from S, N, blocks, C); headers/labels are host arrays of n entries; features
 * are the raw segments times `input_scale`. Writes *loss and grads. Synchronous. */
int tang_loss_grad(tang_ctx *ctx, uint32_t S, uint32_t N, uint32_t blocks, uint32_t C, const float *params,
                   const tang_header *headers, const int32_t *labels, uint32_t n, float input_scale,
                   float *loss, float *grads);

/* One Adam step (bias-corrected, step number t >= 1) over `count` host floats on the GPU. */
int tang_adam_step(tang_ctx *ctx, float *params, const float *grads, float *m, float *v, uint64_t count,
                   uint32_t t, float lr, float beta1, float beta2, float eps);

/* ---------------------------------------------------------------------------------------
 * Deferred update (§5.2.2). A monitor on the search engine measures throughput per window;
 * th_base is the first window closed after the last full retraining (or after load). When
 * 1 - th_cur / th_base > tau, a deferred update is due: a full retraining if more than theta
 * rules were inserted into a tuple whose lengths differ from theirs since the last full
 * retraining (the tang_suboptimal_count counter), incremental training otherwise.
 * ------------------------------------------------------------------------------------- */
#define TANG_DU_NONE 0
#define TANG_DU_INCREMENTAL 1
#define TANG_DU_RETRAIN 2

typedef struct tang_du_cfg {
    double tau;     /* relative throughput drop that triggers (the paper's experiment: 0.05) */
    uint64_t theta; /* counter value above which the update is a full retraining (paper: 10,000) */
} tang_du_cfg;

typedef struct tang_du_window {
    uint64_t window;     /* index of the window just closed; 0 = the baseline window */
    double th_cur;       /* its throughput: packets / cost */
    double th_base;      /* baseline throughput */
    uint64_t suboptimal; /* the counter when the window closed */
    int decision;        /* TANG_DU_*; always TANG_DU_NONE for the baseline window */
} tang_du_window;

/* The decision rule alone: TANG_DU_NONE when th_base <= 0 or the drop 1 - th_cur / th_base
 * does not exceed tau; else TANG_DU_RETRAIN when suboptimal > theta, else TANG_DU_INCREMENTAL.
 * Needs no context and no GPU. Returns TANG_EINVAL for a NULL cfg or a negative/non-finite tau. */
int tang_du_decide(const tang_du_cfg *cfg, double th_base, double th_cur, uint64_t suboptimal);

/* Add an observation to ruleset rs's open window: `packets` classified at `cost` (any unit
 * that grows with the search engine's work: seconds of the search kernel, or memory accesses
 * from tang_stats; throughput is packets / cost, and only ratios of it matter). */
int tang_du_observe(tang_ctx *ctx, uint32_t rs, uint64_t packets, double cost);

/* Close the open window, evaluate the trigger and fill *out. The first window after load or
 * after a full retraining becomes th_base. Errors: TANG_EINVAL (empty window, bad cfg). */
int tang_du_close_window(tang_ctx *ctx, uint32_t rs, const tang_du_cfg *cfg, tang_du_window *out);

/* Incremental training (§5.2.2): like tang_train, but the network starts from the ruleset's
 * loaded model (its N and blocks; cfg->N and cfg->blocks are ignored) and the samples are
 * labelled on the current tuple space, so the model follows the rules inserted and deleted
 * since it was trained. Writes a blob as tang_train does; load it with tang_load_model (a hot
 * swap, since the shape is unchanged). Errors: TANG_EINVAL (no model, or the model no longer
 * fits the tuple count), and those of tang_train. */
int tang_finetune(tang_ctx *ctx, uint32_t rs, const tang_header *samples, uint32_t n, const tang_train_cfg *cfg,
                  void *blob, size_t *bytes, tang_train_report *report);

/* Full rebuild of ruleset rs's tuple space over its live rules (the first step of a full
 * retraining, §5.2.2): every rule moves to the tuple of its own lengths, tuples may appear or
 * disappear (so T may change), conflict sets are recomputed, and the suboptimal counter and
 * the monitor's baseline are reset. If the tuple list changed, the model is dropped (its
 * classes no longer match) together with the context's graphs; *model_kept (may be NULL)
 * says which happened. Synchronous. Errors: TANG_ENOMEM, TANG_ETABLEFULL. */
int tang_rebuild_ruleset(tang_ctx *ctx, uint32_t rs, int *model_kept);

/* Carry out a decision of tang_du_close_window: TANG_DU_NONE does nothing;
 * TANG_DU_INCREMENTAL = tang_finetune + tang_load_model (hot swap); TANG_DU_RETRAIN =
 * tang_rebuild_ruleset + tang_train from scratch (cfg's N and blocks) + tang_load_model.
 * `samples` are recent packet headers (host, n of them); cfg->time_budget_s caps the training
 * time. Synchronous. */
int tang_du_apply(tang_ctx *ctx, uint32_t rs, int decision, const tang_header *samples, uint32_t n,
                  const tang_train_cfg *cfg, tang_train_report *report);

/* Failure-path self-test of the bounded device waits (an addition of this library; the paper
 * has none). Every persistent kernel here waits on barriers with a time limit; when one runs
 * out, the kernel records it in the context's device error word, its other waits give up, and
 * the next synchronising call returns TANG_ETIMEOUT. This launches a one-block kernel whose
 * first warp waits on a barrier that nothing completes, with a limit of `limit_ms` (1-2000),
 * while a second warp waits on another with a 10 s limit and leaves on the first warp's abort
 * flag. Returns TANG_ETIMEOUT when the wait ran out as designed; the error word is then clear
 * and the context usable. *elapsed_ms (may be NULL) receives the kernel's duration.
 * Synchronous. Errors: TANG_EINVAL (limit out of range), TANG_EDEVICE. */
int tang_selftest_wait_timeout(tang_ctx *ctx, uint32_t limit_ms, float *elapsed_ms);

/* Checked builds. A library compiled with TANG_CHECKED (paper_2601_03187_b300/build.py
 * --checked, libtang_checked.so) tests every table index its search code forms (slot, rule
 * pool, conflict-word row, tuple order) against the table's size before the access. An index
 * out of range is not accessed; the lookup ends as if it had found nothing, and the next
 * synchronising call returns TANG_EDEVICE. In other builds the tests are compiled out.
 * tang_checked_build returns 1 for a checked build, else 0. */
int tang_checked_build(void);

/* Test hook for the checked build: the ruleset's device descriptor states a rule-pool size of
 * `n` (0xFFFFFFFF: the real size again), so that rule indices at or past n count as out of
 * range while the memory they address stays allocated. Classification results are undefined
 * until the real size is restored. Synchronous. Errors: TANG_ENOTFOUND, TANG_EDEVICE. */
int tang_debug_set_pool_view(tang_ctx *ctx, uint32_t rs, uint32_t n);

/* ---------------------------------------------------------------------------------------
 * Autotuning and serving
 * ------------------------------------------------------------------------------------- */

/* Time the launch variants of a path on `n` device headers and keep the fastest per
 * (ruleset, path): for the fused paths the tensor-core kernel variant (one CTA per SM, CTA
 * pairs, or network and search as two kernels) and its persistent CTA count, for the
 * search-kernel paths the block size and blocks per SM. Drops captured graphs
 * (they hold the previous launch shape). Synchronous. */
int tang_autotune(tang_ctx *ctx, uint32_t rs, const tang_header *d_headers, uint32_t n, uint32_t flags);

/* The launch shape tang_autotune chose for (rs, path): variant = the fused kernel variant
 * (0 = library default, 5 = the N=256 kernel on one SM, 6 = the same on CTA pairs, 7 = the
 * network and the search as two kernels, TANG_FUSED_SPLIT; fused paths only),
 * grid = persistent CTAs (0 = one per SM), search_threads / search_bps = the search kernel's
 * block size and blocks per SM (0 = default), ms = the time per call measured for the choice
 * (0 if the path was never tuned). Outputs may be NULL. */
int tang_autotune_get(tang_ctx *ctx, uint32_t rs, uint32_t path, int *variant, int *grid, int *search_threads,
                      int *search_bps, float *ms);

/* Set the launch shape of (rs, path) as tang_autotune would, e.g. one saved from
 * tang_autotune_get in an earlier process, so that a restart needs no new tuning. Values as in
 * tang_autotune_get (0 = default for each): variant 0, 5 or 6 (7 on fused paths), grid 0 to the SM count,
 * search_threads 0 / 128 / 256 / 512, search_bps 0-16 with threads x blocks <= 2048. Drops
 * captured graphs. Errors: TANG_ENOTFOUND, TANG_EINVAL (a value out of range). */
int tang_autotune_set(tang_ctx *ctx, uint32_t rs, uint32_t path, int variant, int grid, int search_threads,
                      int search_bps);

typedef struct tang_serve_cfg {
    uint32_t max_inflight;   /* requests on the GPU at once (slots) */
    uint32_t max_batch;      /* packets per GPU launch (requests are packed up to this) */
    uint32_t path;           /* TANG_PATH_* used for every launch */
    uint32_t reserved;
} tang_serve_cfg;

typedef struct tang_req_stats {
    double submit_s, start_s, done_s; /* seconds on the context's monotonic clock */
} tang_req_stats;

/* Start the continuous-batching engine: a host thread packs queued requests (of any
 * rulesets) into GPU launches as slots and memory free up, overlaps their work on several
 * streams, and completes requests out of order. Memory admission: a slot's device buffers
 * ((16 + 4) * max_batch bytes) are taken from the context's pool (from the device's free memory
 * when the pool is unbounded) only when queued work finds every admitted slot busy, and given
 * back after the slot has been idle for 20 ms; a refused admission waits for a slot to finish.
 * So the slots in flight follow the free memory: rulesets or models loaded while the engine runs
 * lower them, unloads raise them. When no slot can be admitted with nothing in flight for 1 s,
 * the queued requests complete with TANG_ENOMEM. Pinned staging, streams and events for
 * max_inflight slots are created here.
 * Errors: TANG_EINVAL (engine running, path other than fused or no-network, max_inflight not in
 * 1..64, max_batch 0), TANG_ENOMEM (one slot exceeds the pool or the device). */
int tang_serve_start(tang_ctx *ctx, const tang_serve_cfg *cfg);
/* Queue a request of n host headers against ruleset rs; ids (host, n entries) is written
 * before the request completes. Both buffers must stay valid until then. */
int tang_serve_submit(tang_ctx *ctx, uint32_t rs, const tang_header *headers, uint32_t n, uint32_t *ids,
                      uint64_t *req_id);
/* TANG_OK when done (stats filled, may be NULL), TANG_EAGAIN while pending after waiting up
 * to wait_ms, TANG_ENOTFOUND for an unknown id. A completed id is forgotten after poll. */
int tang_serve_poll(tang_ctx *ctx, uint64_t req_id, int wait_ms, tang_req_stats *stats);
typedef struct tang_serve_info {
    uint32_t slots_max;           /* max_inflight */
    uint32_t slots_admitted;      /* slots holding device buffers now */
    uint32_t slots_admitted_peak; /* most slots held at once since the engine started */
    uint32_t slots_busy;          /* slots with a launch in flight */
    uint64_t admissions_refused;  /* slot admissions refused for lack of memory */
    uint64_t launches, packets;   /* GPU launches issued and packets in them */
    uint64_t slot_bytes;          /* device bytes one admitted slot holds */
    uint32_t queued;              /* requests waiting for a slot */
    uint32_t reserved;
} tang_serve_info;
/* Counters of the running engine. Errors: TANG_EINVAL (no engine). */
int tang_serve_info_get(tang_ctx *ctx, tang_serve_info *out);
/* Drain and stop. */
int tang_serve_stop(tang_ctx *ctx);
/* Seconds on the clock used by tang_req_stats. */
double tang_now(void);

#ifdef __cplusplus
}
#endif

#endif /* TANG_H */
