// Host side of the tensor-core path: the model's tensor-core copies (transposed BF16 weights,
// E4M3 weights with their scales, biases, FP8 folded constants), TMA tensor maps, and the
// launch of the fused kernel (mlp_tc256.cu) for the fused, staged and inference-only calls.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "tc_common.cuh"

namespace tang {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// Row-major [rows][cols] matrix of 1- or 2-byte elements, box = 128 bytes x box_rows, 128B swizzle.
int make_tmap(tang_ctx *ctx, CUtensorMap *m, void *base, uint32_t rows, bool f8, uint32_t box_rows, uint32_t cols) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return set_err(ctx, TANG_EDEVICE, "cuTensorMapEncodeTiled unavailable");
    const uint32_t esz = f8 ? 1 : 2;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * esz};
    cuuint32_t box[2] = {128 / esz, box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box,
                     es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_err(ctx, TANG_EDEVICE, "cuTensorMapEncodeTiled failed (%d)", int(r));
    return TANG_OK;
}

// Derive the tensor-core copies of a model: transposed (K-major) BF16 weights, FP8 weights with
// their scales, FP32 biases, FP8 dequantisation factors and activation scales, then the fused
// kernel's tensor maps and layer-0 operands (tc256_prepare_model).
int tc_prepare_model(tang_ctx *ctx, DeviceModel &m) {
    const uint32_t N = m.N, C = m.C;
    // the fused kernel takes width 256 or 512, 1 to 31 residual blocks and any class count (the
    // output layer in 256-row tiles, padded with zero rows past Cpad)
    if ((N != 512 && N != 256) || m.blocks < 1 || m.blocks > 31) return TANG_OK;
    const int nl = int(2 * m.blocks);  // N x N layers
    m.layers = uint32_t(nl);
    const uint32_t Cpad = m.Cpad;  // multiple of 32
    const size_t hid = size_t(nl) * N * N;
    const size_t rows_out = Cpad <= 256 ? Cpad : (Cpad + 255) / 256 * 256;
    const float *hp = m.host_params.data();
    // host views of the FP32 parameters
    const float *p = hp + size_t(7) * N + N;
    std::vector<const float *> W(nl), B(nl);
    for (uint32_t b = 0; b < m.blocks; ++b) {
        W[2 * b] = p;
        p += size_t(N) * N;
        B[2 * b] = p;
        p += N;
        W[2 * b + 1] = p;
        p += size_t(N) * N;
        B[2 * b + 1] = p;
        p += N;
    }
    const float *Wc = p;
    const float *bc = p + size_t(N) * C;
    std::vector<__nv_bfloat16> wb(hid + rows_out * N);
    std::vector<float> bias(size_t(nl) * N + Cpad, 0.f);
    for (int l = 0; l < nl; ++l) {
        for (uint32_t n = 0; n < N; ++n)
            for (uint32_t k = 0; k < N; ++k) wb[size_t(l) * N * N + size_t(n) * N + k] = __float2bfloat16_rn(W[l][size_t(k) * N + n]);
        for (uint32_t n = 0; n < N; ++n) bias[size_t(l) * N + n] = B[l][n];
    }
    for (uint32_t c = 0; c < rows_out; ++c)
        for (uint32_t k = 0; k < N; ++k)
            wb[hid + size_t(c) * N + k] = __float2bfloat16_rn(c < C ? Wc[size_t(k) * C + c] : 0.f);
    for (uint32_t c = 0; c < C; ++c) bias[size_t(nl) * N + c] = bc[c];
    int rc = ctx_alloc(ctx, wb.size() * 2, &m.d_wbf16);
    if (!rc) rc = ctx_alloc(ctx, bias.size() * 4, (void **)&m.d_bias_tc);
    if (rc) return rc;
    cudaMemcpy(m.d_wbf16, wb.data(), wb.size() * 2, cudaMemcpyHostToDevice);
    cudaMemcpy(m.d_bias_tc, bias.data(), bias.size() * 4, cudaMemcpyHostToDevice);

    if (m.has_fp8) {
        // activation scale: the power of two that maps the calibrated max |x| into (224, 448]
        for (int j = 0; j <= nl; ++j) {
            const float amax = m.act_amax[j];
            m.act_scale[j] = std::ldexp(1.0f, int(std::floor(std::log2(448.0 / double(amax)))));
        }
        std::vector<uint8_t> w8(hid + rows_out * N, 0);
        std::vector<float> dq(size_t(nl) * N + Cpad, 0.f);
        // Weight scales: one per hidden layer, 448 / max |W_l| (a single dequantisation factor for
        // the whole layer, so the fused kernel's epilogue needs no per-column scale); one per
        // output column for the output layer, 448 / max |Wc[:, c]|.
        auto amax_of = [&](const float *Wsrc, uint32_t ncols, uint32_t c0, uint32_t c1) {
            float a = 0.f;
            for (uint32_t k = 0; k < N; ++k)
                for (uint32_t n = c0; n < c1; ++n) a = std::max(a, std::fabs(Wsrc[size_t(k) * ncols + n]));
            return a;
        };
        auto quant_col = [&](const float *Wsrc, uint32_t ncols, uint32_t n, size_t dst_row, float sa, float amax,
                             float *dq_out) {
            const float sw = amax > 0.f ? 448.0f / amax : 1.0f;
            for (uint32_t k = 0; k < N; ++k)
                w8[dst_row * N + k] = __nv_cvt_float_to_fp8(Wsrc[size_t(k) * ncols + n] * sw, __NV_SATFINITE, __NV_E4M3);
            *dq_out = 1.0f / (sa * sw);
        };
        for (int l = 0; l < nl; ++l) {
            const float amax = amax_of(W[l], N, 0, N);
            for (uint32_t n = 0; n < N; ++n)
                quant_col(W[l], N, n, size_t(l) * N + n, m.act_scale[l], amax, &dq[size_t(l) * N + n]);
        }
        for (uint32_t c = 0; c < C; ++c)
            quant_col(Wc, C, c, hid / N + c, m.act_scale[nl], amax_of(Wc, C, c, c + 1), &dq[size_t(nl) * N + c]);
        rc = ctx_alloc(ctx, w8.size(), &m.d_wfp8);
        if (!rc) rc = ctx_alloc(ctx, (dq.size() + nl + 1) * 4, (void **)&m.d_wscale8);
        if (rc) return rc;
        cudaMemcpy(m.d_wfp8, w8.data(), w8.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(m.d_wscale8, dq.data(), dq.size() * 4, cudaMemcpyHostToDevice);
        // the nl + 1 activation scales follow the dequantisation factors
        cudaMemcpy(m.d_wscale8 + dq.size(), m.act_scale, (nl + 1) * 4, cudaMemcpyHostToDevice);
        // the output scale s[l+1] folded into each hidden layer's dequantisation factor and bias;
        // s is a power of two, so relu(s * (acc * dq + b)) is bit-identical to the unfolded form
        std::vector<float> fold(size_t(2) * nl * N);
        for (int l = 0; l < nl; ++l)
            for (uint32_t n = 0; n < N; ++n) {
                fold[size_t(l) * N + n] = dq[size_t(l) * N + n] * m.act_scale[l + 1];
                fold[size_t(nl + l) * N + n] = bias[size_t(l) * N + n] * m.act_scale[l + 1];
            }
        if ((rc = ctx_alloc(ctx, fold.size() * 4, (void **)&m.d_fold8))) return rc;
        cudaMemcpy(m.d_fold8, fold.data(), fold.size() * 4, cudaMemcpyHostToDevice);
    }
    if ((rc = tc256_prepare_model(ctx, m))) return rc;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "tc_prepare_model: %s", cudaGetErrorString(e));
    return TANG_OK;
}

int tc256_launch(tang_ctx *ctx, DeviceModel &m, const TcParams &prm, bool f8, cudaStream_t st, int grid_cap, bool pair);

int tc_launch(tang_ctx *ctx, Ruleset &rs, const tang_header *h, uint32_t n, uint32_t *ids, float *logits,
              int32_t *tuple, int precision, bool fused_search, DevStats *stats, cudaStream_t st,
              const TuneEntry *tune, int variant, int mode) {
    if (n == 0) return TANG_OK;
    // variant 0 = the tuned choice, else the library default: 5 = one CTA per SM, 6 = CTA pairs
    const int v = variant ? variant : (tune && tune->fused_variant ? tune->fused_variant : 5);
    if (v != 5 && v != 6) return set_err(ctx, TANG_EINVAL, "unknown tensor-core kernel variant %d", v);
    DeviceModel &m = *rs.model;
    const bool f8 = precision == TANG_FP8;
    if (!m.d_wbf16 || (f8 && !m.d_wfp8)) return set_err(ctx, TANG_EUNSUPPORTED, "no tensor-core copy of this model");
    TcParams prm{};
    prm.headers = h;
    prm.n = n;
    prm.n_tiles = (n + 127) / 128;
    prm.ids = ids;
    prm.logits = logits;
    prm.tuple = tuple;
    prm.tables = rs.d_desc;
    prm.stats = stats;
    prm.err = ctx->d_err;
    prm.bias = m.d_bias_tc;
    prm.dq = f8 ? m.d_wscale8 : nullptr;
    prm.sa = f8 ? m.d_wscale8 + size_t(m.layers) * m.N + m.Cpad : nullptr;
    prm.layers = m.layers;
    prm.fold8 = f8 ? m.d_fold8 : nullptr;
    prm.C = m.C;
    prm.Cpad = m.Cpad;
    prm.fused_search = fused_search && ids ? 1 | (mode << 1) : 0;
    prm.trace = nullptr;
    const int rc = tc256_launch(ctx, m, prm, f8, st, tune ? tune->fused_grid : 0, v == 6);
    if (rc == TANG_EUNSUPPORTED)
        return set_err(ctx, TANG_EUNSUPPORTED, "no tensor-core kernel for a %u-block, %u-class model", m.blocks, m.C);
    return rc;
}

}  // namespace tang
