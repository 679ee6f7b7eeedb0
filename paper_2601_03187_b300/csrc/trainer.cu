// Training of TaNG's network (§6.2) on the GPU with this library's own FP32 kernels:
// labelling by the exact tuple-space search, class balancing by oversampling up to alpha,
// minibatch cross-entropy + Adam with a step learning-rate schedule, and rounds with
// alpha x 10 while the held-out accuracy stays below beta.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace tang {

cudaError_t launch_colsum(const float *G, int M, int N, int ldg, float *out, float *part, cudaStream_t st);
cudaError_t launch_softmax_ce(const float *Z, int ldz, int B, int C, const int32_t *y, float *dz, float *row_loss,
                              int32_t *row_ok, cudaStream_t st);
cudaError_t launch_adam(float *p, const float *g, float *m, float *v, size_t count, int t, float lr, float b1,
                        float b2, float eps, cudaStream_t st);
cudaError_t launch_absmax(const float *X, size_t count, unsigned int *out_bits, cudaStream_t st);

// SplitMix64 (Steele, Lea, Flood 2014): the trainer's counter-based random source.
struct SplitMix {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }
    uint32_t below(uint32_t n) { return uint32_t((next() >> 32) * uint64_t(n) >> 32); }
    double uniform() { return double(next() >> 11) * (1.0 / 9007199254740992.0); }
};

__global__ void k_gather(const tang_header *__restrict__ src, const int32_t *__restrict__ lab_src,
                         const uint32_t *__restrict__ idx, uint32_t n, tang_header *__restrict__ dst,
                         int32_t *__restrict__ lab_dst) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t j = idx[i];
        reinterpret_cast<uint4 *>(dst)[i] = reinterpret_cast<const uint4 *>(src)[j];
        lab_dst[i] = lab_src[j];
    }
}

// Parameter/gradient views over one flat buffer in the model blob's order.
struct Views {
    float *W0, *b0, *Wc, *bc;
    std::vector<float *> W1, b1, W2, b2;
};

static size_t param_count(uint32_t S, uint32_t N, uint32_t blocks, uint32_t C) {
    return size_t(S) * N + N + size_t(blocks) * (2 * size_t(N) * N + 2 * N) + size_t(N) * C + C;
}

static Views make_views(float *p, uint32_t S, uint32_t N, uint32_t blocks, uint32_t C) {
    Views v;
    v.W0 = p;
    p += size_t(S) * N;
    v.b0 = p;
    p += N;
    for (uint32_t b = 0; b < blocks; ++b) {
        v.W1.push_back(p);
        p += size_t(N) * N;
        v.b1.push_back(p);
        p += N;
        v.W2.push_back(p);
        p += size_t(N) * N;
        v.b2.push_back(p);
        p += N;
    }
    v.Wc = p;
    p += size_t(N) * C;
    v.bc = p;
    return v;
}

// Device state of one training run: parameters, gradients, Adam moments, activations of a
// batch of up to B rows.
struct Trainer {
    tang_ctx *ctx = nullptr;
    uint32_t S = 7, N = 0, blocks = 0, C = 0, B = 0;
    size_t P = 0;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    float *X = nullptr;               // B x 8
    std::vector<float *> H;           // blocks + 1 buffers of B x N (layer-0 output, block outputs)
    std::vector<float *> U;           // blocks buffers of B x N (first FC of each block)
    float *Z = nullptr, *dZ = nullptr, *G1 = nullptr, *Ga = nullptr, *Gb = nullptr, *part = nullptr;
    float *row_loss = nullptr;
    int32_t *row_ok = nullptr, *labels = nullptr;
    tang_header *hbuf = nullptr;
    std::vector<void *> owned;
    Views pv, gv;

    int alloc(size_t bytes, void **p) {
        int rc = ctx_alloc(ctx, bytes, p);
        if (!rc) owned.push_back(*p);
        return rc;
    }
    ~Trainer() {
        for (void *p : owned) ctx_free(ctx, p);
    }
    int init(tang_ctx *c, uint32_t N_, uint32_t blocks_, uint32_t C_, uint32_t B_) {
        ctx = c;
        N = N_;
        blocks = blocks_;
        C = C_;
        B = B_;
        P = param_count(S, N, blocks, C);
        int rc = 0;
        rc |= alloc(4 * P, (void **)&params);
        rc |= alloc(4 * P, (void **)&grads);
        rc |= alloc(4 * P, (void **)&m);
        rc |= alloc(4 * P, (void **)&v);
        if (rc) return TANG_ENOMEM;
        cudaMemset(m, 0, 4 * P);
        cudaMemset(v, 0, 4 * P);
        const size_t BN = size_t(B) * N;
        rc |= alloc(4 * size_t(B) * 8, (void **)&X);
        H.resize(blocks + 1);
        U.resize(blocks);
        for (auto &p : H) rc |= alloc(4 * BN, (void **)&p);
        for (auto &p : U) rc |= alloc(4 * BN, (void **)&p);
        rc |= alloc(4 * size_t(B) * C, (void **)&Z);
        rc |= alloc(4 * size_t(B) * C, (void **)&dZ);
        rc |= alloc(4 * BN, (void **)&G1);
        rc |= alloc(4 * BN, (void **)&Ga);
        rc |= alloc(4 * BN, (void **)&Gb);
        rc |= alloc(4 * 64 * size_t(std::max(N, C)), (void **)&part);
        rc |= alloc(4 * size_t(B), (void **)&row_loss);
        rc |= alloc(4 * size_t(B), (void **)&row_ok);
        rc |= alloc(4 * size_t(B), (void **)&labels);
        rc |= alloc(sizeof(tang_header) * size_t(B), (void **)&hbuf);
        if (rc) return TANG_ENOMEM;
        pv = make_views(params, S, N, blocks, C);
        gv = make_views(grads, S, N, blocks, C);
        return TANG_OK;
    }

    // Forward of `rows` headers in hbuf; features scaled by `scale` (exact for powers of two).
    cudaError_t forward(uint32_t rows, float scale, cudaStream_t st) {
        const int R = int(rows), n = int(N);
        cudaError_t e = launch_encode(hbuf, rows, X, 8, scale, st);
        if (!e) e = launch_sgemm(0, 0, R, n, int(S), X, 8, pv.W0, n, H[0], n, pv.b0, nullptr, 0, nullptr, 0, 1, 0.f, st);
        for (uint32_t b = 0; b < blocks && !e; ++b) {
            e = launch_sgemm(0, 0, R, n, n, H[b], n, pv.W1[b], n, U[b], n, pv.b1[b], nullptr, 0, nullptr, 0, 1, 0.f, st);
            if (!e) e = launch_sgemm(0, 0, R, n, n, U[b], n, pv.W2[b], n, H[b + 1], n, pv.b2[b], H[b], n, nullptr, 0, 1, 0.f, st);
        }
        if (!e) e = launch_sgemm(0, 0, R, int(C), n, H[blocks], n, pv.Wc, int(C), Z, int(C), pv.bc, nullptr, 0, nullptr, 0, 0, 0.f, st);
        return e;
    }

    // Backward of the mean cross-entropy for labels in `labels` (after forward()).
    cudaError_t backward(uint32_t rows, cudaStream_t st) {
        const int R = int(rows), n = int(N), c = int(C);
        cudaError_t e = launch_softmax_ce(Z, c, R, c, labels, dZ, row_loss, row_ok, st);
        if (!e) e = launch_sgemm(1, 0, n, c, R, H[blocks], n, dZ, c, gv.Wc, c, nullptr, nullptr, 0, nullptr, 0, 0, 0.f, st);
        if (!e) e = launch_colsum(dZ, R, c, c, gv.bc, part, st);
        // g2 of the last block: dZ Wc^T masked by the block output
        float *g2 = Ga, *gnext = Gb;
        if (!e) e = launch_sgemm(0, 1, R, n, c, dZ, c, pv.Wc, c, g2, n, nullptr, nullptr, 0, H[blocks], n, 0, 0.f, st);
        for (int b = int(blocks) - 1; b >= 0 && !e; --b) {
            e = launch_sgemm(1, 0, n, n, R, U[b], n, g2, n, gv.W2[b], n, nullptr, nullptr, 0, nullptr, 0, 0, 0.f, st);
            if (!e) e = launch_colsum(g2, R, n, n, gv.b2[b], part, st);
            if (!e) e = launch_sgemm(0, 1, R, n, n, g2, n, pv.W2[b], n, G1, n, nullptr, nullptr, 0, U[b], n, 0, 0.f, st);
            if (!e) e = launch_sgemm(1, 0, n, n, R, H[b], n, G1, n, gv.W1[b], n, nullptr, nullptr, 0, nullptr, 0, 0, 0.f, st);
            if (!e) e = launch_colsum(G1, R, n, n, gv.b1[b], part, st);
            // gradient into the block input (skip connection adds g2), masked by H[b] > 0
            if (!e) e = launch_sgemm(0, 1, R, n, n, G1, n, pv.W1[b], n, gnext, n, nullptr, g2, n, H[b], n, 0, 0.f, st);
            std::swap(g2, gnext);
        }
        if (!e) e = launch_sgemm(1, 0, int(S), n, R, X, 8, g2, n, gv.W0, n, nullptr, nullptr, 0, nullptr, 0, 0, 0.f, st);
        if (!e) e = launch_colsum(g2, R, n, n, gv.b0, part, st);
        return e;
    }
};

}  // namespace tang

using namespace tang;

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

extern "C" int tang_loss_grad(tang_ctx *ctx, uint32_t S, uint32_t N, uint32_t blocks, uint32_t C, const float *params,
                              const tang_header *headers, const int32_t *labels, uint32_t n, float input_scale,
                              float *loss, float *grads) {
    if (!ctx || !params || !headers || !labels || !loss || !grads || n == 0) return set_err(ctx, TANG_EINVAL, "bad argument");
    if (S != 7 || N == 0 || C == 0) return set_err(ctx, TANG_EINVAL, "bad shape");
    for (uint32_t i = 0; i < n; ++i)
        if (labels[i] < 0 || uint32_t(labels[i]) >= C) return set_err(ctx, TANG_EINVAL, "label out of range");
    cudaSetDevice(ctx->device);
    Trainer tr;
    int rc = tr.init(ctx, N, blocks, C, n);
    if (rc) return rc;
    cudaStream_t st = ctx->stream;
    CK(cudaMemcpyAsync(tr.params, params, 4 * tr.P, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(tr.hbuf, headers, sizeof(tang_header) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(tr.labels, labels, 4 * size_t(n), cudaMemcpyHostToDevice, st));
    CK(tr.forward(n, input_scale, st));
    CK(tr.backward(n, st));
    std::vector<float> rl(n);
    CK(cudaMemcpyAsync(rl.data(), tr.row_loss, 4 * size_t(n), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(grads, tr.grads, 4 * tr.P, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double s = 0;
    for (float x : rl) s += x;
    *loss = float(s / n);
    return TANG_OK;
}

extern "C" int tang_adam_step(tang_ctx *ctx, float *params, const float *grads, float *m, float *v, uint64_t count,
                              uint32_t t, float lr, float beta1, float beta2, float eps) {
    if (!ctx || !params || !grads || !m || !v || t == 0) return set_err(ctx, TANG_EINVAL, "bad argument");
    cudaSetDevice(ctx->device);
    float *d = nullptr;
    int rc = ctx_alloc(ctx, 16 * size_t(count), (void **)&d);
    if (rc) return rc;
    cudaStream_t st = ctx->stream;
    float *dp = d, *dg = d + count, *dm = d + 2 * count, *dv = d + 3 * count;
    cudaMemcpyAsync(dp, params, 4 * count, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dg, grads, 4 * count, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dm, m, 4 * count, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dv, v, 4 * count, cudaMemcpyHostToDevice, st);
    launch_adam(dp, dg, dm, dv, count, int(t), lr, beta1, beta2, eps, st);
    cudaMemcpyAsync(params, dp, 4 * count, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(m, dm, 4 * count, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(v, dv, 4 * count, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    ctx_free(ctx, d);
    if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "adam: %s", cudaGetErrorString(e));
    return TANG_OK;
}

namespace tang {

// A header drawn uniformly inside a rule (wildcard protocol -> uniform byte).
static tang_header inside_rule(const DRule &r, SplitMix &g) {
    tang_header h{};
    const uint32_t ms = prefix_mask(meta_sip_len(r.meta)), md = prefix_mask(meta_dip_len(r.meta));
    h.sip = (r.sip & ms) | (uint32_t(g.next()) & ~ms);
    h.dip = (r.dip & md) | (uint32_t(g.next()) & ~md);
    const uint32_t splo = r.sp & 0xFFFF, sphi = r.sp >> 16, dplo = r.dp & 0xFFFF, dphi = r.dp >> 16;
    h.sp = uint16_t(splo + g.below(sphi - splo + 1));
    h.dp = uint16_t(dplo + g.below(dphi - dplo + 1));
    h.proto = meta_proto_exact(r.meta) ? uint8_t(meta_proto(r.meta)) : uint8_t(g.below(256));
    return h;
}

int train_run(tang_ctx *ctx, Ruleset &rs, const tang_header *samples, uint32_t n, const tang_train_cfg &cfg,
              std::vector<uint8_t> &blob, tang_train_report *rep, const DeviceModel *init) {
    const auto t_start = std::chrono::steady_clock::now();
    auto elapsed = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count(); };
    cudaStream_t st = ctx->stream;
    const uint32_t T = uint32_t(rs.host.tuples.size());
    // incremental training keeps the shape of the model it starts from
    const uint32_t N = init ? init->N : (cfg.N ? cfg.N : 512), blocks = init ? init->blocks : cfg.blocks;
    const uint32_t B = cfg.batch ? cfg.batch : 8192;
    SplitMix rng{cfg.seed * 0x9E3779B97F4A7C15ULL + 12345};
    tang_train_report R{};

    // 1. Label every sample with the tuple of its exact match (§6.2 raw dataset).
    auto label = [&](const std::vector<tang_header> &hs, std::vector<int32_t> &out) -> int {
        out.assign(hs.size(), -1);
        if (hs.empty()) return TANG_OK;
        tang_header *dh = nullptr;
        uint32_t *di = nullptr;
        int rc = ctx_alloc(ctx, sizeof(tang_header) * hs.size(), (void **)&dh);
        if (!rc) rc = ctx_alloc(ctx, 4 * hs.size(), (void **)&di);
        if (rc) {
            ctx_free(ctx, dh);
            return rc;
        }
        std::vector<uint32_t> ids(hs.size());
        cudaMemcpyAsync(dh, hs.data(), sizeof(tang_header) * hs.size(), cudaMemcpyHostToDevice, st);
        launch_search(rs.d_desc, T, rs.host.cw, dh, nullptr, uint32_t(hs.size()), di, nullptr, nullptr, st);
        cudaMemcpyAsync(ids.data(), di, 4 * hs.size(), cudaMemcpyDeviceToHost, st);
        cudaError_t e = cudaStreamSynchronize(st);
        ctx_free(ctx, dh);
        ctx_free(ctx, di);
        if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "labelling: %s", cudaGetErrorString(e));
        for (size_t i = 0; i < hs.size(); ++i) {
            if (ids[i] == TANG_NO_MATCH) continue;
            auto it = rs.host.pos_of_id.find(ids[i]);
            if (it != rs.host.pos_of_id.end()) out[i] = int32_t(meta_tuple(rs.host.pool[it->second].meta));
        }
        return TANG_OK;
    };
    std::vector<tang_header> all(samples, samples + n);
    std::vector<int32_t> lab;
    int rc = label(all, lab);
    if (rc) return rc;
    std::vector<uint32_t> keep;
    for (uint32_t i = 0; i < n; ++i)
        if (lab[i] >= 0) keep.push_back(i);
    R.samples_labelled = uint32_t(keep.size());
    if (keep.empty()) return set_err(ctx, TANG_EINVAL, "no training sample matches a rule");
    // shuffle, then hold out a fraction for the accuracy check
    for (size_t i = keep.size(); i > 1; --i) std::swap(keep[i - 1], keep[rng.below(uint32_t(i))]);
    const size_t n_hold = std::min(keep.size() - 1, size_t(double(keep.size()) * std::max(0.f, cfg.holdout)));
    std::vector<tang_header> hold_h, base_h;
    std::vector<int32_t> hold_y, base_y;
    for (size_t i = 0; i < keep.size(); ++i) {
        (i < n_hold ? hold_h : base_h).push_back(all[keep[i]]);
        (i < n_hold ? hold_y : base_y).push_back(lab[keep[i]]);
    }

    // 2. The network (PyTorch-style uniform init, features prescaled by 2^-16), or, for incremental
    // training (§5.2.2), the deployed model's parameters with the prescale taken back out of W0
    // (exact: a power of two).
    Trainer tr;
    if ((rc = tr.init(ctx, N, blocks, T, B))) return rc;
    if (init) {
        if (init->C != T || init->S != 7 || init->host_params.size() != tr.P)
            return set_err(ctx, TANG_EINVAL, "the loaded model does not fit this ruleset's %u tuples", T);
        std::vector<float> p(init->host_params);
        for (size_t i = 0; i < size_t(7) * N; ++i) p[i] *= 65536.0f;
        CK(cudaMemcpyAsync(tr.params, p.data(), 4 * tr.P, cudaMemcpyHostToDevice, st));
    } else {
        std::vector<float> p(tr.P);
        Views v = make_views(p.data(), 7, N, blocks, T);
        auto fill = [&](float *w, size_t cnt, uint32_t fan_in) {
            const float bound = 1.0f / std::sqrt(float(fan_in));
            for (size_t i = 0; i < cnt; ++i) w[i] = float((rng.uniform() * 2 - 1) * bound);
        };
        fill(v.W0, size_t(7) * N, 7);
        fill(v.b0, N, 7);
        for (uint32_t b = 0; b < blocks; ++b) {
            fill(v.W1[b], size_t(N) * N, N);
            fill(v.b1[b], N, N);
            fill(v.W2[b], size_t(N) * N, N);
            fill(v.b2[b], N, N);
        }
        fill(v.Wc, size_t(N) * T, N);
        fill(v.bc, T, N);
        CK(cudaMemcpyAsync(tr.params, p.data(), 4 * tr.P, cudaMemcpyHostToDevice, st));
    }
    const float scale = 1.0f / 65536.0f;

    // device copies of the training set (grown per round) and of the holdout
    tang_header *d_set = nullptr;
    int32_t *d_lab = nullptr;
    uint32_t *d_idx = nullptr;
    size_t set_cap = 0;
    auto free_set = [&]() {
        ctx_free(ctx, d_set);
        ctx_free(ctx, d_lab);
        ctx_free(ctx, d_idx);
        d_set = nullptr;
        d_lab = nullptr;
        d_idx = nullptr;
        set_cap = 0;
    };
    auto upload_set = [&](const std::vector<tang_header> &h, const std::vector<int32_t> &y) -> int {
        if (h.size() > set_cap) {
            free_set();
            int r = ctx_alloc(ctx, sizeof(tang_header) * h.size(), (void **)&d_set);
            if (!r) r = ctx_alloc(ctx, 4 * h.size(), (void **)&d_lab);
            if (!r) r = ctx_alloc(ctx, 4 * h.size(), (void **)&d_idx);
            if (r) return r;
            set_cap = h.size();
        }
        cudaMemcpyAsync(d_set, h.data(), sizeof(tang_header) * h.size(), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_lab, y.data(), 4 * y.size(), cudaMemcpyHostToDevice, st);
        return TANG_OK;
    };
    // accuracy over a host set, batch by batch
    auto accuracy = [&](const std::vector<tang_header> &h, const std::vector<int32_t> &y) -> double {
        if (h.empty()) return 1.0;
        uint64_t ok = 0;
        std::vector<int32_t> rok(B);
        for (size_t b0 = 0; b0 < h.size(); b0 += B) {
            const uint32_t rows = uint32_t(std::min<size_t>(B, h.size() - b0));
            cudaMemcpyAsync(tr.hbuf, h.data() + b0, sizeof(tang_header) * rows, cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(tr.labels, y.data() + b0, 4 * rows, cudaMemcpyHostToDevice, st);
            tr.forward(rows, scale, st);
            launch_softmax_ce(tr.Z, int(T), int(rows), int(T), tr.labels, tr.dZ, tr.row_loss, tr.row_ok, st);
            cudaMemcpyAsync(rok.data(), tr.row_ok, 4 * rows, cudaMemcpyDeviceToHost, st);
            cudaStreamSynchronize(st);
            for (uint32_t i = 0; i < rows; ++i) ok += rok[i] != 0;
        }
        return double(ok) / double(h.size());
    };

    uint32_t alpha = cfg.alpha;
    uint64_t step = 0;
    bool out_of_time = false;
    double acc = 0.0;
    float last_loss = 0.f;
    for (uint32_t round = 0; round < std::max(1u, cfg.max_rounds) && !out_of_time; ++round) {
        // 3. §6.2 class balance: every class below alpha is oversampled up to alpha.
        std::vector<tang_header> set_h = base_h;
        std::vector<int32_t> set_y = base_y;
        std::vector<std::vector<uint32_t>> by_class(T);
        for (uint32_t i = 0; i < base_y.size(); ++i) by_class[base_y[i]].push_back(i);
        std::vector<uint32_t> empty;
        for (uint32_t c = 0; c < T; ++c) {
            const auto &v = by_class[c];
            if (v.empty()) {
                if (rs.host.tuples[c].n_rules) empty.push_back(c);
                continue;
            }
            for (size_t k = v.size(); k < alpha; ++k) {
                uint32_t j = v[rng.below(uint32_t(v.size()))];
                set_h.push_back(base_h[j]);
                set_y.push_back(c);
            }
        }
        // classes without samples: packets drawn inside the tuple's rules, kept when their
        // exact label is that tuple
        if (!empty.empty()) {
            std::vector<std::vector<uint32_t>> members(T);
            for (auto &kv : rs.host.pos_of_id) members[meta_tuple(rs.host.pool[kv.second].meta)].push_back(kv.second);
            for (auto &mv : members) std::sort(mv.begin(), mv.end());
            std::vector<tang_header> cand;
            std::vector<int32_t> want;
            for (uint32_t c : empty) {
                const auto &mv = members[c];
                if (mv.empty()) continue;
                for (uint32_t k = 0; k < 4 * alpha; ++k) {
                    cand.push_back(inside_rule(rs.host.pool[mv[rng.below(uint32_t(mv.size()))]], rng));
                    want.push_back(int32_t(c));
                }
            }
            std::vector<int32_t> got;
            if ((rc = label(cand, got))) {
                free_set();
                return rc;
            }
            std::vector<uint32_t> added(T, 0);
            for (size_t i = 0; i < cand.size(); ++i)
                if (got[i] == want[i] && added[want[i]] < alpha) {
                    set_h.push_back(cand[i]);
                    set_y.push_back(want[i]);
                    added[want[i]]++;
                }
            for (uint32_t c : empty) R.classes_empty += added[c] == 0;
        }
        if ((rc = upload_set(set_h, set_y))) {
            free_set();
            return rc;
        }
        R.samples_trained = uint32_t(set_h.size());
        // 4. Epochs of shuffled minibatches; lr decays by `decay` every `decay_every` epochs.
        std::vector<uint32_t> perm(set_h.size());
        for (uint32_t ep = 0; ep < std::max(1u, cfg.epochs); ++ep) {
            std::iota(perm.begin(), perm.end(), 0);
            for (size_t i = perm.size(); i > 1; --i) std::swap(perm[i - 1], perm[rng.below(uint32_t(i))]);
            cudaMemcpyAsync(d_idx, perm.data(), 4 * perm.size(), cudaMemcpyHostToDevice, st);
            const float lr = cfg.lr * std::pow(cfg.decay, float(cfg.decay_every ? ep / cfg.decay_every : 0));
            for (size_t b0 = 0; b0 < perm.size(); b0 += B) {
                const uint32_t rows = uint32_t(std::min<size_t>(B, perm.size() - b0));
                k_gather<<<std::min<uint32_t>((rows + 255) / 256, 1184), 256, 0, st>>>(d_set, d_lab, d_idx + b0, rows,
                                                                                      tr.hbuf, tr.labels);
                tr.forward(rows, scale, st);
                tr.backward(rows, st);
                ++step;
                launch_adam(tr.params, tr.grads, tr.m, tr.v, tr.P, int(step), lr, 0.9f, 0.999f, 1e-8f, st);
            }
            R.epochs_run++;
            if (cfg.time_budget_s > 0 && elapsed() > cfg.time_budget_s) {
                out_of_time = true;
                break;
            }
        }
        {
            std::vector<float> rl(B);
            cudaMemcpyAsync(rl.data(), tr.row_loss, 4 * size_t(B), cudaMemcpyDeviceToHost, st);
            CK(cudaStreamSynchronize(st));
            double s = 0;
            const uint32_t rows = uint32_t(std::min<size_t>(B, set_h.size()));
            for (uint32_t i = 0; i < rows; ++i) s += rl[i];
            last_loss = float(s / std::max(1u, rows));
        }
        R.rounds = round + 1;
        acc = accuracy(hold_h.empty() ? base_h : hold_h, hold_h.empty() ? base_y : hold_y);
        R.alpha_final = alpha;
        if (acc >= cfg.beta) break;
        alpha *= 10;
    }
    free_set();

    // 5. Export: parameters with the 2^-16 feature prescale folded into W0 (exact), and the
    // largest activation entering every tensor-core layer over (a sample of) the training set.
    std::vector<float> p(tr.P);
    CK(cudaMemcpy(p.data(), tr.params, 4 * tr.P, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < size_t(7) * N; ++i) p[i] *= scale;
    std::vector<float> amax(2 * blocks + 1, 0.f);
    {
        unsigned int *d_bits = nullptr;
        if ((rc = ctx_alloc(ctx, 4 * amax.size(), (void **)&d_bits))) return rc;
        CK(cudaMemsetAsync(d_bits, 0, 4 * amax.size(), st));
        const size_t lim = std::min<size_t>(base_h.size(), 262144);
        for (size_t b0 = 0; b0 < lim; b0 += B) {
            const uint32_t rows = uint32_t(std::min<size_t>(B, lim - b0));
            cudaMemcpyAsync(tr.hbuf, base_h.data() + b0, sizeof(tang_header) * rows, cudaMemcpyHostToDevice, st);
            tr.forward(rows, scale, st);
            launch_absmax(tr.H[0], size_t(rows) * N, d_bits + 0, st);
            for (uint32_t b = 0; b < blocks; ++b) {
                launch_absmax(tr.U[b], size_t(rows) * N, d_bits + 1 + 2 * b, st);
                launch_absmax(tr.H[b + 1], size_t(rows) * N, d_bits + 2 + 2 * b, st);
            }
        }
        std::vector<unsigned int> bits(amax.size());
        CK(cudaMemcpyAsync(bits.data(), d_bits, 4 * bits.size(), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        ctx_free(ctx, d_bits);
        for (size_t i = 0; i < amax.size(); ++i) {
            float f;
            std::memcpy(&f, &bits[i], 4);
            amax[i] = f > 0.f ? f : 1e-6f;
        }
    }
    tang_model_header hd{};
    hd.magic = TANG_MODEL_MAGIC;
    hd.version = 1;
    hd.S = 7;
    hd.N = N;
    hd.blocks = blocks;
    hd.C = T;
    blob.resize(sizeof(hd) + 4 * amax.size() + 4 * p.size());
    std::memcpy(blob.data(), &hd, sizeof(hd));
    std::memcpy(blob.data() + sizeof(hd), amax.data(), 4 * amax.size());
    std::memcpy(blob.data() + sizeof(hd) + 4 * amax.size(), p.data(), 4 * p.size());
    R.final_loss = last_loss;
    R.holdout_accuracy = float(acc);
    R.train_seconds = float(elapsed());
    if (rep) *rep = R;
    return TANG_OK;
}

}  // namespace tang

extern "C" int tang_train(tang_ctx *ctx, uint32_t rsh, const tang_header *samples, uint32_t n,
                          const tang_train_cfg *cfg, void *blob, size_t *bytes, tang_train_report *report) {
    const NvtxRange nvtx_range("tang_train");
    if (!ctx || !samples || !cfg || !bytes || n == 0) return set_err(ctx, TANG_EINVAL, "bad argument");
    auto it = ctx->rulesets.find(rsh);
    if (it == ctx->rulesets.end()) return set_err(ctx, TANG_ENOTFOUND, "unknown ruleset %u", rsh);
    if (cfg->blocks > 31 || cfg->N > 4096) return set_err(ctx, TANG_EINVAL, "unsupported network shape");
    cudaSetDevice(ctx->device);
    std::vector<uint8_t> out;
    int rc = train_run(ctx, *it->second, samples, n, *cfg, out, report);
    if (rc) return rc;
    const size_t have = *bytes;
    *bytes = out.size();
    if (blob && have >= out.size()) std::memcpy(blob, out.data(), out.size());
    return TANG_OK;
}
