// Pieces shared by the tensor-core kernel (mlp_tc256.cu) and its host side (tc_model.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "internal.h"

namespace tang {

struct TcParams {
    const tang_header *headers;
    uint32_t n, n_tiles;
    uint32_t *ids;
    float *logits;
    int32_t *tuple;
    const Tables *tables;
    DevStats *stats;
    int *err;
    const float *bias;      // [layers][N] hidden biases, then [Cpad] output biases
    const float *dq;        // FP8 only: per layer and output column 1 / (act scale * weight scale)
    const float *sa;        // FP8 only: [layers + 1] activation scales of the layers' inputs
    const float *fold8;     // FP8 only: [layers][N] dq * s_out, then [layers][N] bias * s_out
    uint32_t C, Cpad;
    uint32_t layers;        // N x N layers (2 x residual blocks)
    int fused_search;       // bit 0: run the search warps; bits 1-2: the search mode (search_packet)
    unsigned long long *trace;  // event timestamps of CTA 0 (trace builds only, else null)
};

// Optional event trace (built with -DTANG_TC_TRACE): clock64() stamps of CTA 0 at fixed slots.
namespace trace {
constexpr int kChunks = 100;                   // first 100 accumulator chunks (about two tiles)
constexpr int kMma = 0;                        // [chunk][12]: start, acc_empty ok, full ok x8, issued
constexpr int kEpi = kMma + kChunks * 12;      // [warp 0/1][chunk][4]: wait, acc_full ok, drained, published
constexpr int kProd = kEpi + 2 * kChunks * 4;  // [load]: empty ok
constexpr int kLoads = 800;
constexpr int kSearch = kProd + kLoads;        // [tile][2]: search warp 0 got the tile, finished it
constexpr int kSearchTiles = 32;
constexpr int kEpiX = kSearch + 2 * kSearchTiles;  // [warp 0/1][chunk][6]: per 32-column half: math, residual, stored
constexpr int kTotal = kEpiX + 2 * kChunks * 6;
}  // namespace trace
#ifdef TANG_TC_TRACE
#define TC_TRACE(slot, limit)                                                        \
    do {                                                                            \
        if (p.trace && blockIdx.x == 0 && (limit)) p.trace[(slot)] = clock64();     \
    } while (0)
#else
#define TC_TRACE(slot, limit) \
    do {                      \
    } while (0)
#endif

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}
// Two FP32 operations in one instruction (the packed f32x2 forms of sm_100 and later): each
// element is rounded to nearest even exactly as the scalar add / fma would round it.
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
    uint64_t d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ float2 f2_unpack(uint64_t v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ float2 add_f2(float2 a, float2 b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_pack(a.x, a.y)), "l"(f2_pack(b.x, b.y)));
    return f2_unpack(d);
}
// a * b + c per element, one rounding each
__device__ __forceinline__ float2 fma_f2(float2 a, float2 b, float2 c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2_pack(a.x, a.y)), "l"(f2_pack(b.x, b.y)), "l"(f2_pack(c.x, c.y)));
    return f2_unpack(d);
}

// Residual additions in one mixed-precision instruction per element (the 16-bit operand widened
// exactly, one rounding of the sum, as the unpack-then-add they replace): c + the BF16 in the low
// or high half of `two`, and c + h * s for the FP16 in the low or high half of `two` and the FP16
// in the low half of `s16`.
__device__ __forceinline__ float add_bf16lo(uint32_t two, float c) {
    float d;
    asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %1;\n\tadd.rn.f32.bf16 %0, lo, %2;\n\t}" : "=f"(d) : "r"(two), "f"(c));
    return d;
}
__device__ __forceinline__ float add_bf16hi(uint32_t two, float c) {
    float d;
    asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %1;\n\tadd.rn.f32.bf16 %0, hi, %2;\n\t}" : "=f"(d) : "r"(two), "f"(c));
    return d;
}
__device__ __forceinline__ float fma_f16lo(uint32_t two, uint32_t s16, float c) {
    float d;
    asm("{\n\t.reg .b16 lo, hi, s, t;\n\tmov.b32 {lo, hi}, %1;\n\tmov.b32 {s, t}, %2;\n\tfma.rn.f32.f16 %0, lo, s, %3;\n\t}"
        : "=f"(d) : "r"(two), "r"(s16), "f"(c));
    return d;
}
__device__ __forceinline__ float fma_f16hi(uint32_t two, uint32_t s16, float c) {
    float d;
    asm("{\n\t.reg .b16 lo, hi, s, t;\n\tmov.b32 {lo, hi}, %1;\n\tmov.b32 {s, t}, %2;\n\tfma.rn.f32.f16 %0, hi, s, %3;\n\t}"
        : "=f"(d) : "r"(two), "r"(s16), "f"(c));
    return d;
}
// Four E4M3 codes (bits 0-7, 8-15 of `two`) as FP16x2, exactly.
__device__ __forceinline__ uint32_t e4m3x2_to_h2(uint32_t two) {
    uint32_t h2;
    asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"(uint16_t(two & 0xFFFFu)));
    return h2;
}

// ReLU, round to nearest even and pack two BF16: lo in bits 0-15, hi in bits 16-31.
__device__ __forceinline__ uint32_t relu_bf16x2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
// ReLU, round to nearest even with saturation at +-448 and pack two E4M3 codes: lo in bits 0-7.
__device__ __forceinline__ uint32_t relu_e4m3x2(float lo, float hi) {
    uint16_t d;
    asm("cvt.rn.satfinite.relu.e4m3x2.f32 %0, %1, %2;" : "=h"(d) : "f"(hi), "f"(lo));
    return d;
}
// Two E4M3 codes (bits 0-7 and 8-15 of `two`) as floats; every E4M3 value is exact in FP16.
__device__ __forceinline__ float2 e4m3x2_to_f2(uint32_t two) {
    uint32_t h2;
    asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"(uint16_t(two & 0xFFFFu)));
    return __half22float2(*reinterpret_cast<const __half2 *>(&h2));
}

// Row-major [rows][cols] weight matrix of 1- or 2-byte elements as a TMA tensor map whose box is
// 128 bytes x box_rows with 128-byte swizzle (cols * element size a multiple of 128).
int make_tmap(tang_ctx *ctx, CUtensorMap *m, void *base, uint32_t rows, bool f8, uint32_t box_rows,
              uint32_t cols = 512);

}  // namespace tang
