// Internal declarations of the TaNG B300 library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "tang.h"

namespace tang {

// A named NVTX range around one library call, for profilers' timelines (nearly free when no
// tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr uint32_t kMaxTuples = 2047;  // tuple index is stored in 11 bits of a rule record

// ---------------------------------------------------------------------------------------
// Device records. All are read with 16-byte vector loads, so sizes are multiples of 16.
// ---------------------------------------------------------------------------------------

// One tuple (§4.3): truncation masks, its open-addressing table, its best (priority, id).
struct TupleDesc {
    uint32_t mask_s, mask_d;      // prefix masks of the tuple's SIP / DIP lengths
    uint32_t slot_base, slot_mask; // table = slots[slot_base .. slot_base + slot_mask]
    uint32_t min_prio, min_id;    // best rule of the tuple (a lower bound after deletes)
    uint32_t max_probe;           // longest linear-probe distance of any key in the table
    uint32_t n_rules;             // live rules (0: never probed)
};
static_assert(sizeof(TupleDesc) == 32, "TupleDesc is 32 bytes");

// One hash-table slot: a truncated key and the run of rules stored under it.
struct Slot {
    uint32_t ks, kd;   // truncated SIP / DIP
    uint32_t start;    // first rule of the run in the rule pool; kEmpty = empty slot
    uint32_t len;      // rules in the run (may be 0 after deletes)
};
static_assert(sizeof(Slot) == 16, "Slot is 16 bytes");

// One rule as the search kernels read it (one 32-byte sector).
//   sp / dp: lo | hi << 16
//   meta:    bits 0-5 sip_len, 6-11 dip_len, 12 protocol-exact flag, 13-20 protocol,
//            21-31 tuple index the rule is stored in
//   cf:      conflict set (bit t = tuple t holds a better overlapping rule) when T <= 32,
//            otherwise the index of the rule's row in Tables::cwords
struct DRule {
    uint32_t sip, dip, sp, dp, meta, prio, id, cf;
};
static_assert(sizeof(DRule) == 32, "DRule is 32 bytes");

__host__ __device__ inline uint32_t meta_sip_len(uint32_t m) { return m & 63u; }
__host__ __device__ inline uint32_t meta_dip_len(uint32_t m) { return (m >> 6) & 63u; }
__host__ __device__ inline uint32_t meta_proto_exact(uint32_t m) { return (m >> 12) & 1u; }
__host__ __device__ inline uint32_t meta_proto(uint32_t m) { return (m >> 13) & 255u; }
__host__ __device__ inline uint32_t meta_tuple(uint32_t m) { return m >> 21; }
__host__ __device__ inline uint32_t make_meta(uint32_t sl, uint32_t dl, uint32_t exact, uint32_t proto,
                                              uint32_t tuple) {
    return sl | (dl << 6) | (exact << 12) | (proto << 13) | (tuple << 21);
}
__host__ __device__ inline uint32_t prefix_mask(uint32_t len) { return len == 0 ? 0u : (0xFFFFFFFFu << (32u - len)); }

// Device-resident descriptor of one ruleset's tables. Kernels receive a pointer to it, so the
// arrays can be reallocated (table growth on insert) without re-capturing CUDA graphs.
struct Tables {
    const TupleDesc *tuples;
    const Slot *slots;
    DRule *rules;
    uint32_t *cwords;        // conflict words when T > 32 (row = DRule::cf), else unused
    const uint16_t *order;   // tuple indices in ascending (min_prio, min_id): the search order
    uint32_t T;              // tuples
    uint32_t cw;             // conflict words per rule (ceil(T/32))
    uint32_t pool_size;      // rule pool entries in use (live + dead)
    uint32_t slot_cap;       // slots allocated (bound of every slot index)
    uint32_t cword_rows;     // conflict-word rows allocated (T > 32)
    uint32_t pad;
    int *err;                // the context's device error word (checked builds report into it)
};

// Device error word bits outside the bounded waits': an index the checked build (TANG_CHECKED)
// found out of range; the access was skipped.
constexpr int kErrIndex = 1 << 30;

// Per-call counters (tang_stats in device memory).
struct DevStats {
    unsigned long long packets, matched, nn_correct, pred_hit, fallback, probes, rule_reads, slot_reads;
};

// ---------------------------------------------------------------------------------------
// Host mirror of a ruleset's tuple space (tss_host.cpp)
// ---------------------------------------------------------------------------------------
struct HostTuple {
    uint32_t ls, ld;
    uint32_t slot_base, cap;  // cap is a power of two
    uint32_t n_keys;          // occupied slots (including keys whose run became empty)
    uint32_t min_prio, min_id, max_probe, n_rules;
};

struct HostTSS {
    std::vector<HostTuple> tuples;
    std::vector<Slot> slots;          // mirror of the device slot pool (size = slot pool capacity used)
    std::vector<uint32_t> run_cap;    // capacity reserved for each slot's run in the rule pool
    std::vector<DRule> pool;          // mirror of the device rule pool (cf not mirrored)
    std::unordered_map<uint32_t, uint32_t> pos_of_id;  // live rule id -> pool position
    std::vector<uint16_t> order;      // search order
    uint32_t cw = 1;
    uint32_t live = 0;
    uint64_t suboptimal = 0;          // inserts whose lengths differ from their tuple's (§5.2.2 counter)
    int16_t tuple_of_len[33][33];     // (sip_len, dip_len) -> tuple index or -1
};

// ---------------------------------------------------------------------------------------
// Model
// ---------------------------------------------------------------------------------------
struct DeviceModel {
    uint32_t S = 0, N = 0, blocks = 0, C = 0, Cpad = 0;
    uint32_t layers = 0;              // N x N layers of the tensor-core copies (2 x blocks; 0 = none)
    std::vector<float> host_params;   // blob parameter order
    float *d_params = nullptr;        // same order, FP32 (plain path and layer 0 of every path)
    // FP32 pointers into d_params
    const float *W0 = nullptr, *b0 = nullptr, *Wc = nullptr, *bc = nullptr;
    std::vector<const float *> W1, b1, W2, b2;
    // Tensor-core copies: per N x N layer l (0 .. 2*blocks-1) the transposed weight W^T[n][k]
    // (K-major), then the output layer Wc^T padded to Cpad rows.
    void *d_wbf16 = nullptr;          // __nv_bfloat16
    void *d_wfp8 = nullptr;           // E4M3 bytes, per-output-channel scaled
    float *d_wscale8 = nullptr;       // per layer, per output channel: 1 / weight scale
    float *d_bias_tc = nullptr;       // per layer N (or Cpad) biases, FP32, output layer last
    // N=256 FP8 kernel: per hidden layer l, dq[l][n] * s[l+1], then bias[l][n] * s[l+1], with s the
    // power-of-two activation scale of the layer's output (so the products are exact)
    float *d_fold8 = nullptr;
    // N=256 kernel: layer 0 as a K=64 BF16 contraction, [2][512][64] (unscaled, then times the
    // FP8 input scale s[0]); see tc256_prepare_model
    void *d_l0 = nullptr;
    float act_amax[64] = {0};
    bool has_fp8 = false;
    float act_scale[64] = {0};        // FP8 activation scale per tensor-core layer input
    void *tmap256 = nullptr;          // host-side tensor maps of the fused kernel: [BF16, FP8]
};

struct Ruleset;

// Graph cache entry for TANG_GRAPH.
struct GraphKey {
    uint32_t rs, path, n;
    const void *h;
    const void *ids;
    void *stream;
    bool operator<(const GraphKey &o) const;
};

// Launch shape chosen by the autotuner per (ruleset, path); zeros mean "default".
struct TuneEntry {
    int search_threads = 0;  // threads per block of the search kernel (128 / 256 / 512)
    int search_bps = 0;      // resident blocks per SM the search grid is sized for
    int fused_grid = 0;      // persistent CTAs of the fused kernel (0 = one per SM)
    int fused_variant = 0;   // 0 = library default, 5 = the N=256 fused kernel, 6 = on CTA pairs, 7 = split
    float ms = 0.f;          // best time measured by the tuner
};
// Fused paths run as two kernels: the network writes its predictions into the output ids, the
// search kernel replaces them with rule ids (TANG_FUSED_SPLIT).
constexpr int kVariantSplit = 7;

// Search mode bits: kSearchPaper = the paper's post-verification (no conflict-set probes after a
// hit in the predicted tuple), kSearchSerial = one thread per rule run, kSearchPredInIds (search
// kernel only) = each packet's prediction is read from its own entry of the output ids, which the
// network kernel filled, and then overwritten with the rule id.
constexpr int kSearchPaper = 1, kSearchSerial = 2, kSearchPredInIds = 4;

struct Ruleset {
    uint32_t handle = 0;
    HostTSS host;
    // device arrays
    TupleDesc *d_tuples = nullptr;
    Slot *d_slots = nullptr;
    DRule *d_rules = nullptr;
    uint32_t *d_cwords = nullptr;
    uint16_t *d_order = nullptr;
    uint32_t slot_capacity = 0, rule_capacity = 0, cword_capacity = 0;  // elements (cwords: words)
    uint32_t cword_rows = 0;  // conflict rows handed out (T > 32 only)
    uint32_t pool_view = kEmpty;  // test hook: the pool size the device descriptor states (kEmpty: the real one)
    Tables *d_desc = nullptr;
    Tables h_desc{};
    std::unique_ptr<DeviceModel> model;
    cudaEvent_t last_update = nullptr;  // classify waits on it
    bool has_update = false;
    // One event per stream that has classified against this ruleset, recorded after its latest
    // classification: an update waits for all of them before it touches the tables.
    std::mutex inflight_mu;
    std::vector<std::pair<cudaStream_t, cudaEvent_t>> inflight;
    double build_ms = 0;
    std::map<uint32_t, TuneEntry> tune;  // per path
    // deferred-update monitor (§5.2.2): the open window's packets and cost, and the throughput of
    // the first window closed after the last full retraining (windows == 0: not measured yet)
    uint64_t du_packets = 0;
    double du_cost = 0.0;
    uint64_t du_windows = 0;
    double du_th_base = 0.0;
};

struct ServeEngine;

}  // namespace tang

struct tang_ctx {
    int device = 0;
    size_t cap = 0;
    size_t used = 0;
    std::string err;
    cudaStream_t stream = nullptr;
    std::map<uint32_t, std::unique_ptr<tang::Ruleset>> rulesets;
    uint32_t next_rs = 1;
    std::unordered_map<void *, size_t> allocs;
    std::mutex alloc_mu;
    // scratch for the staged / plain paths (grown on demand)
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    tang::DevStats *d_stats = nullptr;
    int *d_err = nullptr;  // error bits set by kernels whose bounded waits ran out
    std::map<tang::GraphKey, cudaGraphExec_t> graphs;
    // host pipeline
    cudaStream_t copy_in = nullptr, copy_out = nullptr, compute2 = nullptr;
    void *pinned_h = nullptr, *pinned_ids = nullptr;
    size_t pinned_pkts = 0;
    void *dev_h = nullptr, *dev_ids = nullptr;
    size_t dev_pkts = 0;
    int sm_count = 148;
    tang::ServeEngine *serve = nullptr;
    int32_t *noalloc_tuples = nullptr;  // device address of tang_classify_noalloc's static array
};

// ---------------------------------------------------------------------------------------
// Shared helpers
// ---------------------------------------------------------------------------------------
namespace tang {
int set_err(tang_ctx *ctx, int code, const char *fmt, ...);
// After a synchronisation point: TANG_ETIMEOUT (and the error word cleared) if a bounded device
// wait ran out since the last check, else TANG_OK.
int check_device_error(tang_ctx *ctx);
int ctx_alloc(tang_ctx *ctx, size_t bytes, void **p);
// ctx_alloc without touching the context's error text (for the serving engine's own thread).
int ctx_try_alloc(tang_ctx *ctx, size_t bytes, void **p);
void ctx_free(tang_ctx *ctx, void *p);
int ensure_scratch(tang_ctx *ctx, size_t bytes);
// Checked builds: synchronise `st` (unless it is being captured) and report the device error word.
int checked_sync(tang_ctx *ctx, cudaStream_t st);
// Record, on `st`, that a classification against `rs` was enqueued there (no-op while `st` is
// being captured into a graph).
void note_classify(Ruleset &rs, cudaStream_t st);
// Make `st` wait for every classification noted against `rs` (before an update of its tables).
int wait_classifies(tang_ctx *ctx, Ruleset &rs, cudaStream_t st);
// noalloc.cu: resolve the device address of the no-alloc scratch array for ctx->device.
int noalloc_prepare(tang_ctx *ctx);

// tss_host.cpp
int tss_build(tang_ctx *ctx, Ruleset &rs, const tang_rule *rules, uint32_t n);
int tss_upload(tang_ctx *ctx, Ruleset &rs, cudaStream_t st);
int tss_insert(tang_ctx *ctx, Ruleset &rs, const tang_rule &r, cudaStream_t st);
int tss_delete(tang_ctx *ctx, Ruleset &rs, uint32_t id, cudaStream_t st);
void tss_free(tang_ctx *ctx, Ruleset &rs);
int tss_rebuild(tang_ctx *ctx, Ruleset &rs, bool &same_tuples);
int tss_set_pool_view(tang_ctx *ctx, Ruleset &rs, uint32_t n);
uint64_t fmix64_host(uint64_t k);

// search.cu (mode: search_dev.cuh's kSearchPaper / kSearchSerial bits, from the TANG_SEARCH_* flags)
int search_mode_of(uint32_t flags);
cudaError_t launch_conflict_build(const DRule *sorted, const uint32_t *sorted_pos, uint32_t n, DRule *pool,
                                  uint32_t *cwords, uint32_t cw, uint32_t T, cudaStream_t st);
cudaError_t launch_conflict_insert(const Tables *d_desc, uint32_t pool_size, uint32_t new_pos, uint32_t cw,
                                   cudaStream_t st);
cudaError_t launch_run_shift(DRule *pool, uint32_t start, uint32_t len, uint32_t pos, int dir, cudaStream_t st);
cudaError_t launch_run_copy(DRule *pool, uint32_t from, uint32_t to, uint32_t len, cudaStream_t st);
cudaError_t launch_search(const Tables *d_desc, uint32_t T, uint32_t cw, const tang_header *h,
                          const int32_t *tuple, uint32_t n, uint32_t *ids, DevStats *stats, const TuneEntry *tune,
                          cudaStream_t st, int mode = 0);

// mlp_simt.cu (FP32 CUDA-core kernels: plain path and trainer)
cudaError_t launch_encode(const tang_header *h, uint32_t n, float *X, uint32_t ldx, float scale, cudaStream_t st);
cudaError_t launch_sgemm(int ta, int tb, int M, int N, int K, const float *A, int lda, const float *B, int ldb,
                         float *C, int ldc, const float *bias, const float *resid, int ldr, const float *mask,
                         int ldm, int relu, float beta, cudaStream_t st);
cudaError_t launch_argmax(const float *Z, int ldz, int n, int C, int32_t *out, cudaStream_t st);
int mlp_fp32_forward(tang_ctx *ctx, const DeviceModel &m, const tang_header *h, uint32_t n, float *logits,
                     int32_t *tuple, cudaStream_t st);

// tc_model.cu (host side of the tcgen05 fused kernel in mlp_tc256.cu)
int tc_prepare_model(tang_ctx *ctx, DeviceModel &m);
int tc_launch(tang_ctx *ctx, Ruleset &rs, const tang_header *h, uint32_t n, uint32_t *ids, float *logits,
              int32_t *tuple, int precision, bool fused_search, DevStats *stats, cudaStream_t st,
              const TuneEntry *tune, int variant, int mode = 0);
int tc256_prepare_model(tang_ctx *ctx, DeviceModel &m);

// trainer.cu; init != nullptr starts from that model's parameters (incremental training)
int train_run(tang_ctx *ctx, Ruleset &rs, const tang_header *samples, uint32_t n, const tang_train_cfg &cfg,
              std::vector<uint8_t> &blob, tang_train_report *rep, const DeviceModel *init = nullptr);
}  // namespace tang
