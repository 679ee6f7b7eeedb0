// Fused classification kernel on the 5th-generation tensor cores (tcgen05, sm_103a):
// header load + §6.2 encoding + the residual MLP of §6.1 (BF16 or FP8 operands, FP32
// accumulation in tensor memory) + argmax + the exact tuple-space search of §5.1.1, one
// persistent CTA per SM, one 128-packet tile at a time.
//
// Data flow of one tile (M = 128 packets):
//   - layer 0 (7 -> 512) runs on CUDA cores in FP32 (16-bit segments are not exact in BF16);
//     its output x goes to tensor memory (TMEM) as the A operand of the next MMA.
//   - block b, FC1: acc = x . W1 (A from TMEM, B = weight tiles streamed by TMA into shared
//     memory); epilogue: u = ReLU(acc + b1) -> shared memory (128B-swizzled K-major tiles).
//   - block b, FC2: acc = u . W2 (A and B from shared memory); epilogue:
//     x = ReLU(acc + b2 + x), written back into TMEM in place (Eq. 1).
//   - output FC: logits = x . Wc + bc (A from TMEM), argmax -> predicted tuple.
//   - search warps take the predicted tuples and run the exact search while the tensor cores
//     move on to the next tile.
// TMEM (512 columns): two 128-column FP32 accumulators (double-buffered output chunks of 128
// features) + x packed 2 x BF16 (256 columns) or 4 x E4M3 (128 columns) per 32-bit column.
//
// Warp roles (14 warps): 0 TMA producer, 1 MMA issuer (+ TMEM allocation), 2..9 epilogue
// (warp w reads TMEM lanes 32*(w%4)..+31 and one 64-column half of each chunk), 10..13 search.
// Every wait is bounded (2 s of %globaltimer); on timeout the kernel records an error code,
// stops issuing work, drains what it issued and frees TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>
#include <cstring>

#include "search_dev.cuh"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace tang {

namespace tc {
constexpr int kM = 128;            // packets per tile
constexpr int kHid = 512;          // hidden width
constexpr int kLayers = 12;        // N x N layers (6 blocks x 2)
constexpr int kStages = 4;         // weight pipeline depth
constexpr int kStageBytes = 16384; // one 128-row x 128-byte weight tile
constexpr int kThreads = 448;
constexpr int kWarpProd = 0, kWarpMma = 1, kWarpEpi = 2, kNumEpiWarps = 8, kWarpSearch = 10, kNumSearchWarps = 4;
constexpr uint64_t kTimeoutNs = 2000000000ull;
constexpr int kSmemTuples = 64;
constexpr uint32_t kXCol = 256;    // first TMEM column of x

// shared-memory layout (offsets from a 1024-byte aligned base)
constexpr int kOffY = 0;
constexpr int kYBytes = kM * kHid * 2;  // BF16; FP8 uses half of it
constexpr int kOffStage = kOffY + kYBytes;
constexpr int kOffW0 = kOffStage + kStages * kStageBytes;
constexpr int kOffB0 = kOffW0 + 7 * kHid * 4;
constexpr int kOffTup = kOffB0 + kHid * 4;
constexpr int kOffOrd = kOffTup + kSmemTuples * 32;
constexpr int kOffTidx = kOffOrd + kSmemTuples * 2;
constexpr int kOffBar = kOffTidx + 2 * kM * 4;
constexpr int kNumBars = 2 * kStages + 2 + 2 + 8 + 2 + 2 + 1;
constexpr int kOffMisc = kOffBar + kNumBars * 8;
constexpr int kSmemBytes = kOffMisc + 16 + 1024;  // + alignment slack
}  // namespace tc

// CS = CTAs per cluster that share every weight tile: each loads 1/CS of the tile's rows and
// multicasts them to all, so L2 serves each weight line once per cluster instead of once per SM.
template <bool F8, int CS>
__global__ void __launch_bounds__(tc::kThreads, 1)
    k_tc_classify(const __grid_constant__ CUtensorMap tm_hid, const __grid_constant__ CUtensorMap tm_out,
                  const TcParams p) {
    using namespace tc;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sY = smem + kOffY;
    uint8_t *sStage = smem + kOffStage;
    float *sW0 = reinterpret_cast<float *>(smem + kOffW0);
    float *sB0 = reinterpret_cast<float *>(smem + kOffB0);
    TupleDesc *sTup = reinterpret_cast<TupleDesc *>(smem + kOffTup);
    uint16_t *sOrd = reinterpret_cast<uint16_t *>(smem + kOffOrd);
    int32_t *sTidx = reinterpret_cast<int32_t *>(smem + kOffTidx);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kOffBar);
    uint64_t *full = bars, *empty = bars + kStages;
    uint64_t *acc_full = bars + 2 * kStages, *acc_empty = acc_full + 2;
    uint64_t *act = acc_empty + 2;          // 8 barriers, one per K-block of the next layer
    uint64_t *tfull = act + 8, *tempty = tfull + 2, *drain = tempty + 2;
    uint32_t *sTmem = reinterpret_cast<uint32_t *>(smem + kOffMisc);
    volatile int *sAbort = reinterpret_cast<volatile int *>(smem + kOffMisc + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int KB = F8 ? 4 : 8;                 // K-blocks (128-byte rows) per 512-wide layer input
    constexpr int KBW = F8 ? 128 : 64;             // elements per K-block
    constexpr uint32_t kActArrivals = F8 ? 8 : 4;  // epilogue warps writing one K-block
    constexpr uint16_t kMask = uint16_t((1u << CS) - 1);
    const uint32_t crank = CS > 1 ? ptx::cluster_ctarank() : 0;
    // every CTA of a cluster runs the same number of tile rounds (the weight pipeline is shared);
    // rounds past the end run on masked rows
    const uint32_t cbase = blockIdx.x - crank;
    auto round_live = [&](uint32_t k) { return cbase + k * gridDim.x < p.n_tiles; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], CS);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&acc_full[b], 1);
            ptx::mbar_init(&acc_empty[b], kNumEpiWarps);
            ptx::mbar_init(&tfull[b], 4);
            ptx::mbar_init(&tempty[b], kNumSearchWarps);
        }
        for (int k = 0; k < 8; ++k) ptx::mbar_init(&act[k], kActArrivals);
        ptx::mbar_init(drain, 1);
        *sAbort = 0;
        ptx::fence_mbar_init();
    }
    if (warp == kWarpProd && lane == 0) {
        ptx::prefetch_tmap(&tm_hid);
        ptx::prefetch_tmap(&tm_out);
    }
    for (int i = threadIdx.x; i < 7 * kHid; i += kThreads) sW0[i] = p.W0[i];
    for (int i = threadIdx.x; i < kHid; i += kThreads) sB0[i] = p.b0[i];
    const Tables tb = *p.tables;
    const bool tup_smem = tb.T <= uint32_t(kSmemTuples);
    if (tup_smem)
        for (uint32_t i = threadIdx.x; i < tb.T; i += kThreads) {
            sTup[i] = tb.tuples[i];
            sOrd[i] = tb.order[i];
        }
    if (warp == kWarpMma) {
        ptx::tmem_alloc(sTmem, 512);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    if (CS > 1)
        ptx::cluster_sync();  // every CTA's barriers exist before multicast loads and commits land
    else
        __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *sTmem;

    auto fail = [&](int code) {
        atomicOr(p.err, code);
        *sAbort = 1;
    };

    if (warp == kWarpProd) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            uint32_t stage = 0, phase = 0, n_loads = 0;
            bool ok = true;
            const uint32_t hid_rows = 128 / CS, out_rows = p.Cpad / CS;
            for (uint32_t k = 0; round_live(k) && ok; ++k) {
                for (int L = 0; L <= kLayers && ok; ++L) {
                    const int nch = L == kLayers ? 1 : 4;
                    for (int c = 0; c < nch && ok; ++c)
                        for (int kb = 0; kb < KB; ++kb) {
                            if (!ptx::mbar_wait(&empty[stage], phase ^ 1, sAbort, kTimeoutNs)) {
                                fail(1);
                                ok = false;
                                break;
                            }
                            TC_TRACE(trace::kProd + n_loads, n_loads < trace::kLoads);
                            ++n_loads;
                            uint8_t *dst = sStage + stage * kStageBytes;
                            if (L < kLayers) {
                                ptx::mbar_arrive_expect_tx(&full[stage], kStageBytes);
                                if (CS == 1)
                                    ptx::tma_load_2d(dst, &tm_hid, &full[stage], kb * KBW, L * kHid + c * 128);
                                else
                                    ptx::tma_load_2d_mc(dst + crank * hid_rows * 128, &tm_hid, &full[stage], kb * KBW,
                                                        L * kHid + c * 128 + int(crank * hid_rows), kMask);
                            } else {
                                ptx::mbar_arrive_expect_tx(&full[stage], p.Cpad * 128);
                                if (CS == 1)
                                    ptx::tma_load_2d(dst, &tm_out, &full[stage], kb * KBW, 0);
                                else
                                    ptx::tma_load_2d_mc(dst + crank * out_rows * 128, &tm_out, &full[stage], kb * KBW,
                                                        int(crank * out_rows), kMask);
                            }
                            if (++stage == kStages) {
                                stage = 0;
                                phase ^= 1;
                            }
                        }
                }
            }
            // drain: every issued load must land before the CTA may exit (timeout only, no abort)
            volatile int never = 0;
            for (int s = 0; s < kStages; ++s) {
                // the most recent use of stage s was in the phase before the current one for
                // s >= stage, and in the current one for s < stage
                const uint32_t par = s < int(stage) ? phase : phase ^ 1;
                ptx::mbar_wait(&full[s], par, &never, kTimeoutNs);
            }
        }
    } else if (warp == kWarpMma) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc_h = ptx::idesc_make(128, 128, F8);
            const uint32_t idesc_o = ptx::idesc_make(128, p.Cpad, F8);
            const uint32_t y_addr = ptx::smem_u32(sY), st_addr = ptx::smem_u32(sStage);
            uint32_t stage = 0, phase = 0, acc_cnt = 0, lay = 0;
            bool ok = true;
            for (uint32_t k = 0; round_live(k) && ok; ++k) {
                for (int L = 0; L <= kLayers && ok; ++L, ++lay) {
                    const bool a_tmem = (L & 1) == 0;  // FC1 and output layer read x from TMEM
                    const int nch = L == kLayers ? 1 : 4;
                    const uint32_t idesc = L == kLayers ? idesc_o : idesc_h;
                    for (int c = 0; c < nch && ok; ++c, ++acc_cnt) {
                        const uint32_t buf = acc_cnt & 1, use = acc_cnt >> 1;
                        const bool tr = acc_cnt < uint32_t(trace::kChunks);
                        TC_TRACE(trace::kMma + acc_cnt * 12 + 0, tr);
                        if (use > 0 && !ptx::mbar_wait(&acc_empty[buf], (use - 1) & 1, sAbort, kTimeoutNs)) {
                            fail(2);
                            ok = false;
                            break;
                        }
                        TC_TRACE(trace::kMma + acc_cnt * 12 + 1, tr);
                        ptx::tc_fence_after();
                        const uint32_t d = tmem + buf * 128;
                        for (int kb = 0; kb < KB; ++kb) {
                            if (c == 0 && !ptx::mbar_wait(&act[kb], lay & 1, sAbort, kTimeoutNs)) {
                                fail(4);
                                ok = false;
                                break;
                            }
                            if (!ptx::mbar_wait(&full[stage], phase, sAbort, kTimeoutNs)) {
                                fail(8);
                                ok = false;
                                break;
                            }
                            TC_TRACE(trace::kMma + acc_cnt * 12 + 2 + kb, tr);
                            ptx::tc_fence_after();
                            const uint32_t b_base = st_addr + stage * kStageBytes;
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint64_t bd = ptx::sdesc_sw128(b_base + kk * 32);
                                const uint32_t accum = (kb | kk) != 0;
                                if (a_tmem)
                                    ptx::mma_ts(d, tmem + kXCol + kb * 32 + kk * 8, bd, idesc, accum, F8);
                                else
                                    ptx::mma_ss(d, ptx::sdesc_sw128(y_addr + kb * 16384 + kk * 32), bd, idesc, accum, F8);
                            }
                            if (CS == 1)
                                ptx::mma_commit(&empty[stage]);
                            else
                                ptx::mma_commit_mc(&empty[stage], kMask);  // the stage is free in every CTA
                            if (++stage == kStages) {
                                stage = 0;
                                phase ^= 1;
                            }
                        }
                        if (!ok) break;
                        ptx::mma_commit(&acc_full[buf]);
                        TC_TRACE(trace::kMma + acc_cnt * 12 + 10, tr);
                    }
                }
            }
            // wait for every MMA issued by this thread before TMEM is released
            volatile int never = 0;
            ptx::mma_commit(drain);
            ptx::mbar_wait(drain, 0, &never, kTimeoutNs);
        }
    } else if (warp < kWarpSearch) {
        // ---------------- epilogue warps ----------------
        const int ew = warp - kWarpEpi;
        const int q = warp & 3;          // TMEM lane quadrant this warp may access
        const int hc = ew >> 2;          // which 64-column half of every 128-column chunk
        const int r = q * 32 + lane;     // row (packet) of the tile
        const uint32_t lane_base = uint32_t(q * 32) << 16;
        const float *sa = p.sa;
        uint32_t acc_cnt = 0, tcnt = 0;
        bool ok = true;
        // store 32 activations of row r (columns col0 .. col0+31 of the 512-wide layer input)
        // into the swizzled shared-memory operand (u of §6.1 Eq. 1)
        auto store_smem = [&](const uint32_t *w, int col0) {
            if (!F8) {
                const int kb = col0 >> 6, j0 = (col0 & 63) >> 3;  // 16-byte chunk index in the row
                uint8_t *row = sY + kb * 16384 + r * 128;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    *reinterpret_cast<uint4 *>(row + (((j0 + k) ^ (r & 7)) << 4)) =
                        make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
            } else {
                const int kb = col0 >> 7, j0 = (col0 & 127) >> 4;
                uint8_t *row = sY + kb * 16384 + r * 128;
#pragma unroll
                for (int k = 0; k < 2; ++k)
                    *reinterpret_cast<uint4 *>(row + (((j0 + k) ^ (r & 7)) << 4)) =
                        make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
            }
        };
        // x columns col0 .. col0+31 in TMEM
        auto x_col = [&](int col0) -> uint32_t { return tmem + lane_base + kXCol + (F8 ? col0 / 4 : col0 / 2); };
        auto act_arrive = [&](int col0) {
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&act[col0 / KBW]);
        };

        for (uint32_t k = 0; round_live(k) && ok; ++k) {
            const uint32_t tile = blockIdx.x + k * gridDim.x;
            const uint32_t i = tile < p.n_tiles ? tile * kM + r : 0xFFFFFFFFu;
            float f[7];
            {
                uint4 v = i < p.n ? __ldg(reinterpret_cast<const uint4 *>(p.headers + i)) : make_uint4(0, 0, 0, 0);
                f[0] = float(v.x >> 16);
                f[1] = float(v.x & 0xFFFFu);
                f[2] = float(v.y >> 16);
                f[3] = float(v.y & 0xFFFFu);
                f[4] = float(v.z & 0xFFFFu);
                f[5] = float(v.z >> 16);
                f[6] = float(v.w & 0xFFu);
            }
            // ---- layer 0 on CUDA cores: this warp owns the 64-column units hc, hc+2, hc+4, hc+6
            for (int g = 0; g < 4; ++g) {
                const int unit = hc + 2 * g;
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const int col0 = unit * 64 + s * 32;
                    float v[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        float a = sB0[col0 + j];
#pragma unroll
                        for (int t = 0; t < 7; ++t) a = fmaf(f[t], sW0[t * kHid + col0 + j], a);
                        v[j] = fmaxf(a, 0.f);
                    }
                    if (!F8) {
                        uint32_t w[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) w[j] = pack_bf16(v[2 * j], v[2 * j + 1]);
                        ptx::tmem_st16(x_col(col0), w);
                    } else {
                        const float s0 = sa[0];
                        uint32_t w[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            w[j] = pack_e4m3x4(v[4 * j] * s0, v[4 * j + 1] * s0, v[4 * j + 2] * s0, v[4 * j + 3] * s0);
                        ptx::tmem_st8(x_col(col0), w);
                    }
                }
                ptx::tmem_wait_st();
                // one arrival per 64-column unit: a BF16 K-block is one unit (4 arrivals, one per
                // lane quadrant), an FP8 K-block is units 2m and 2m+1 (8 arrivals)
                act_arrive(unit * 64);
            }
            // ---- hidden layers
            for (int L = 0; L < kLayers && ok; ++L) {
                const bool fc2 = (L & 1) != 0;
                const float *bias = p.bias + L * kHid;
                const float *dq = F8 ? p.dq + L * kHid : nullptr;
                const float s_out = F8 ? sa[L + 1] : 1.f;    // scale of the next layer's input
                const float s_res = F8 ? 1.f / sa[L - (fc2 ? 1 : 0)] : 1.f;
                for (int c = 0; c < 4; ++c, ++acc_cnt) {
                    const uint32_t buf = acc_cnt & 1, use = acc_cnt >> 1;
                    const bool tr = lane == 0 && (ew & 3) == 0 && acc_cnt < uint32_t(trace::kChunks);
                    const int tslot = trace::kEpi + ((ew >> 2) * trace::kChunks + int(acc_cnt)) * 4;
                    TC_TRACE(tslot + 0, tr);
                    if (!ptx::mbar_wait(&acc_full[buf], use & 1, sAbort, kTimeoutNs)) {
                        fail(16);
                        ok = false;
                        break;
                    }
                    TC_TRACE(tslot + 1, tr);
                    ptx::tc_fence_after();
                    const int unit = 2 * c + hc;
#pragma unroll
                    for (int s = 0; s < 2; ++s) {
                        const int col0 = unit * 64 + s * 32;
                        uint32_t a[32];
                        ptx::tmem_ld32(tmem + lane_base + buf * 128 + hc * 64 + s * 32, a);
                        uint32_t xr[16];
                        if (fc2) {
                            if (!F8)
                                ptx::tmem_ld16(x_col(col0), xr);
                            else
                                ptx::tmem_ld8(x_col(col0), *reinterpret_cast<uint32_t(*)[8]>(xr));
                        }
                        ptx::tmem_wait_ld();
                        if (s == 1) {
                            ptx::tc_fence_before();
                            __syncwarp();
                            if (lane == 0) ptx::mbar_arrive(&acc_empty[buf]);
                            TC_TRACE(tslot + 2, tr);
                        }
                        float v[32];
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            float y = __uint_as_float(a[j]);
                            y = F8 ? fmaf(y, __ldg(dq + col0 + j), __ldg(bias + col0 + j)) : y + __ldg(bias + col0 + j);
                            v[j] = y;
                        }
                        if (fc2) {
                            if (!F8) {
#pragma unroll
                                for (int j = 0; j < 16; ++j) {
                                    v[2 * j] += __uint_as_float(xr[j] << 16);
                                    v[2 * j + 1] += __uint_as_float(xr[j] & 0xFFFF0000u);
                                }
                            } else {
#pragma unroll
                                for (int j = 0; j < 8; ++j)
#pragma unroll
                                    for (int b = 0; b < 4; ++b) v[4 * j + b] += e4m3_to_f((xr[j] >> (8 * b)) & 0xFFu) * s_res;
                            }
                        }
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = fmaxf(v[j], 0.f);
                        if (!F8) {
                            uint32_t w[16];
#pragma unroll
                            for (int j = 0; j < 16; ++j) w[j] = pack_bf16(v[2 * j], v[2 * j + 1]);
                            if (fc2)
                                ptx::tmem_st16(x_col(col0), w);
                            else
                                store_smem(w, col0);
                        } else {
                            uint32_t w[8];
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                w[j] = pack_e4m3x4(v[4 * j] * s_out, v[4 * j + 1] * s_out, v[4 * j + 2] * s_out,
                                                   v[4 * j + 3] * s_out);
                            if (fc2)
                                ptx::tmem_st8(x_col(col0), w);
                            else
                                store_smem(w, col0);
                        }
                    }
                    if (fc2)
                        ptx::tmem_wait_st();
                    else
                        ptx::fence_proxy_async_smem();
                    act_arrive(unit * 64);
                    TC_TRACE(tslot + 3, tr);
                }
            }
            if (!ok) break;
            // ---- output layer: logits, argmax
            {
                const uint32_t buf = acc_cnt & 1, use = acc_cnt >> 1;
                ++acc_cnt;
                if (!ptx::mbar_wait(&acc_full[buf], use & 1, sAbort, kTimeoutNs)) {
                    fail(32);
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                int arg = 0;
                if (hc == 0) {
                    float best = -INFINITY;
                    const float *bias = p.bias + kLayers * kHid;
                    const float *dq = F8 ? p.dq + kLayers * kHid : nullptr;
                    for (uint32_t c0 = 0; c0 < p.Cpad; c0 += 32) {
                        uint32_t a[32];
                        if (c0 + 32 <= p.Cpad) {
                            ptx::tmem_ld32(tmem + lane_base + buf * 128 + c0, a);
                        } else {
                            uint32_t h16[16];
                            ptx::tmem_ld16(tmem + lane_base + buf * 128 + c0, h16);
#pragma unroll
                            for (int j = 0; j < 16; ++j) a[j] = h16[j];
                        }
                        ptx::tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const uint32_t cc = c0 + j;
                            if (cc >= p.C) break;
                            float z = __uint_as_float(a[j]);
                            z = F8 ? fmaf(z, __ldg(dq + cc), __ldg(bias + cc)) : z + __ldg(bias + cc);
                            if (p.logits && i < p.n) p.logits[size_t(i) * p.C + cc] = z;
                            if (z > best) {
                                best = z;
                                arg = int(cc);
                            }
                        }
                    }
                }
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&acc_empty[buf]);
                if (hc == 0) {
                    if (p.tuple && i < p.n) p.tuple[i] = arg;
                    if (p.fused_search) {
                        const uint32_t t = tcnt & 1, tu = tcnt >> 1;
                        ++tcnt;
                        if (!ptx::mbar_wait(&tempty[t], (tu & 1) ^ 1, sAbort, kTimeoutNs)) {
                            fail(64);
                            ok = false;
                            break;
                        }
                        sTidx[t * kM + r] = arg;
                        __syncwarp();
                        if (lane == 0) ptx::mbar_arrive(&tfull[t]);
                    }
                }
            }
        }
    } else {
        // ---------------- search warps: exact tuple-space search of the predicted tuples ----
        if (p.fused_search) {
            const int r = (warp - kWarpSearch) * 32 + lane;
            const TupleDesc *tuples = tup_smem ? sTup : tb.tuples;
            const uint16_t *order = tup_smem ? sOrd : tb.order;
            uint32_t tcnt = 0;
            uint32_t st_pk = 0, st_match = 0, st_correct = 0, st_hit = 0, st_fb = 0;
            Counters cn{0, 0, 0};
            for (uint32_t k = 0; round_live(k); ++k) {
                const uint32_t tile = blockIdx.x + k * gridDim.x;
                const uint32_t t = tcnt & 1, tu = tcnt >> 1;
                ++tcnt;
                if (!ptx::mbar_wait(&tfull[t], tu & 1, sAbort, kTimeoutNs)) {
                    fail(128);
                    break;
                }
                const int pred = sTidx[t * kM + r];
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&tempty[t]);
                const uint32_t i = tile * kM + r;
                if (tile < p.n_tiles && i < p.n) {
                    const Hdr h = load_header(p.headers + i);
                    Best best;
                    const bool hit = search_packet(tb, tuples, order, h, pred, best, cn, (p.fused_search & 2) != 0);
                    p.ids[i] = best.id;
                    if (p.stats) {
                        st_pk++;
                        const bool m = best.id != 0xFFFFFFFFu;
                        st_match += m;
                        st_correct += m && int(best.tuple) == pred;
                        st_hit += hit;
                        st_fb += !hit;
                    }
                }
            }
            if (p.stats) {
                auto add = [&](unsigned long long *dst, uint32_t v) {
                    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
                    if (lane == 0 && v) atomicAdd(dst, (unsigned long long)v);
                };
                add(&p.stats->packets, st_pk);
                add(&p.stats->matched, st_match);
                add(&p.stats->nn_correct, st_correct);
                add(&p.stats->pred_hit, st_hit);
                add(&p.stats->fallback, st_fb);
                add(&p.stats->probes, cn.probes);
                add(&p.stats->rule_reads, cn.rule_reads);
                add(&p.stats->slot_reads, cn.slot_reads);
            }
        }
    }

    ptx::tc_fence_before();
    if (CS > 1)
        ptx::cluster_sync();  // no CTA leaves while peers may still multicast into it or commit to it
    else
        __syncthreads();
    ptx::tc_fence_after();
    if (warp == kWarpMma) ptx::tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------
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

// Row-major [rows][512] matrix of 1- or 2-byte elements, box = 128 bytes x box_rows, 128B swizzle.
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
// per-output-channel scales, FP32 biases, FP8 dequantisation factors and activation scales.
int tc_prepare_model(tang_ctx *ctx, DeviceModel &m) {
    const uint32_t N = m.N, C = m.C;
    // the N=256 kernel takes width 256 or 512, any block count up to 31 and any class count (in
    // 256-row output tiles, padded with zero rows past Cpad); the N=128 variants only width 512,
    // the paper's 6 blocks and up to 128 classes
    if ((N != 512 && N != 256) || m.blocks < 1 || m.blocks > 31) return TANG_OK;
    const bool narrow = C <= 128 && N == 512;
    const int nl = int(2 * m.blocks);  // N x N layers
    m.layers = uint32_t(nl);
    const uint32_t Cpad = m.Cpad;  // multiple of 32
    const size_t hid = size_t(nl) * N * N;
    const size_t rows_out = Cpad <= 256 ? Cpad : (Cpad + 255) / 256 * 256;
    const float *hp = m.host_params.data();
    // host views of the FP32 parameters
    const float *W0 = hp;
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
    (void)W0;
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
    // one map pair per cluster size 1, 2, 4: a CTA loads 128/CS rows of each hidden tile and
    // Cpad/CS rows of each output tile
    if (narrow) {
        TcMaps *maps = static_cast<TcMaps *>(aligned_alloc(64, 3 * sizeof(TcMaps)));
        m.tmap_bf16 = maps;
        for (int ci = 0; ci < 3; ++ci) {
            const uint32_t cs = 1u << ci;
            if ((rc = make_tmap(ctx, &maps[ci].hid, m.d_wbf16, nl * N, false, 128 / cs))) return rc;
            if ((rc = make_tmap(ctx, &maps[ci].out, static_cast<__nv_bfloat16 *>(m.d_wbf16) + hid, Cpad, false, Cpad / cs)))
                return rc;
        }
    }

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
        if (narrow) {
            TcMaps *m8 = static_cast<TcMaps *>(aligned_alloc(64, 3 * sizeof(TcMaps)));
            m.tmap_fp8 = m8;
            for (int ci = 0; ci < 3; ++ci) {
                const uint32_t cs = 1u << ci;
                if ((rc = make_tmap(ctx, &m8[ci].hid, m.d_wfp8, nl * N, true, 128 / cs))) return rc;
                if ((rc = make_tmap(ctx, &m8[ci].out, static_cast<uint8_t *>(m.d_wfp8) + hid, Cpad, true, Cpad / cs)))
                    return rc;
            }
        }
    }
    if (narrow && nl == tc::kLayers && (rc = tc2_prepare_model(ctx, m))) return rc;
    if ((rc = tc256_prepare_model(ctx, m))) return rc;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "tc_prepare_model: %s", cudaGetErrorString(e));
    return TANG_OK;
}

int tc2_launch(tang_ctx *ctx, DeviceModel &m, const TcParams &prm, bool f8, cudaStream_t st, int grid_cap);
int tc256_launch(tang_ctx *ctx, DeviceModel &m, const TcParams &prm, bool f8, cudaStream_t st, int grid_cap);

// Launch the 1-SM kernel in clusters of CS CTAs: as many clusters as fit on the device at once
// (one CTA per SM), capped by the tile count and the tuned grid.
template <bool F8, int CS>
static int launch_1sm(tang_ctx *ctx, const TcMaps &maps, const TcParams &prm, cudaStream_t st, const TuneEntry *tune) {
    static bool init = false;
    static int max_clusters = 0;
    if (!init) {
        cudaError_t e = cudaFuncSetAttribute(k_tc_classify<F8, CS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             tc::kSmemBytes);
        if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "smem attribute: %s", cudaGetErrorString(e));
        max_clusters = ctx->sm_count / CS;
        if (CS > 1) {
            cudaLaunchConfig_t q = {};
            q.gridDim = dim3(CS * (ctx->sm_count / CS), 1, 1);
            q.blockDim = dim3(tc::kThreads, 1, 1);
            q.dynamicSmemBytes = tc::kSmemBytes;
            cudaLaunchAttribute qa[1];
            qa[0].id = cudaLaunchAttributeClusterDimension;
            qa[0].val.clusterDim.x = CS;
            qa[0].val.clusterDim.y = 1;
            qa[0].val.clusterDim.z = 1;
            q.attrs = qa;
            q.numAttrs = 1;
            int c = 0;
            if (cudaOccupancyMaxActiveClusters(&c, k_tc_classify<F8, CS>, &q) == cudaSuccess && c > 0)
                max_clusters = std::min(max_clusters, c);
            cudaGetLastError();
        }
        init = true;
    }
    uint32_t clusters = uint32_t(max_clusters);
    if (tune && tune->fused_grid > 0) clusters = std::min<uint32_t>(clusters, uint32_t(tune->fused_grid / CS));
    clusters = std::max<uint32_t>(1, std::min<uint32_t>(clusters, (prm.n_tiles + CS - 1) / CS));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CS * clusters, 1, 1);
    cfg.blockDim = dim3(tc::kThreads, 1, 1);
    cfg.dynamicSmemBytes = tc::kSmemBytes;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_tc_classify<F8, CS>, maps.hid, maps.out, prm);
    if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "tc kernel launch: %s", cudaGetErrorString(e));
    return TANG_OK;
}

// Library default variant when neither the caller nor the tuner chose one.
constexpr int kDefaultVariant = 5;  // N=256 kernel (mlp_tc256.cu)

int tc_launch(tang_ctx *ctx, Ruleset &rs, const tang_header *h, uint32_t n, uint32_t *ids, float *logits,
              int32_t *tuple, int precision, bool fused_search, DevStats *stats, cudaStream_t st,
              const TuneEntry *tune, int variant, bool paper) {
    if (n == 0) return TANG_OK;
    DeviceModel &m = *rs.model;
    const bool f8 = precision == TANG_FP8;
    if (!m.d_wbf16 || (f8 && !m.d_wfp8)) return set_err(ctx, TANG_EUNSUPPORTED, "no tensor-core copy of this model");
    TcParams prm{};
    prm.headers = h;
    prm.n = n;
    prm.n_tiles = (n + tc::kM - 1) / tc::kM;
    prm.ids = ids;
    prm.logits = logits;
    prm.tuple = tuple;
    prm.tables = rs.d_desc;
    prm.stats = stats;
    prm.err = ctx->d_err;
    prm.W0 = m.W0;
    prm.b0 = m.b0;
    prm.bias = m.d_bias_tc;
    prm.dq = f8 ? m.d_wscale8 : nullptr;
    prm.sa = f8 ? m.d_wscale8 + size_t(m.layers) * m.N + m.Cpad : nullptr;
    prm.layers = m.layers;
    prm.fold8 = f8 ? m.d_fold8 : nullptr;
    prm.C = m.C;
    prm.Cpad = m.Cpad;
    prm.fused_search = fused_search && ids ? (paper ? 3 : 1) : 0;
    prm.trace = nullptr;
#ifdef TANG_TC_TRACE
    static unsigned long long *d_trace = nullptr;
    if (!d_trace) cudaMalloc(&d_trace, sizeof(unsigned long long) * trace::kTotal);
    cudaMemsetAsync(d_trace, 0, sizeof(unsigned long long) * trace::kTotal, st);
    prm.trace = d_trace;
#endif
    int v = variant ? variant : (tune && tune->fused_variant ? tune->fused_variant : kDefaultVariant);
    // the N=128 variants are built for width 512, 6 blocks and at most 128 classes
    const bool narrow6 = m.N == 512 && m.layers == uint32_t(tc::kLayers) && m.C <= 128;
    if (!narrow6) v = 5;
    if (v == 2 || v == 5) {
        const int rc = v == 2 ? tc2_launch(ctx, m, prm, f8, st, tune ? tune->fused_grid : 0)
                              : tc256_launch(ctx, m, prm, f8, st, tune ? tune->fused_grid : 0);
        if (rc != TANG_EUNSUPPORTED) return rc;  // models without those maps run the 1-SM N=128 kernel
    }
    const TcMaps *maps = static_cast<const TcMaps *>(f8 ? m.tmap_fp8 : m.tmap_bf16);
    if (!narrow6 || !maps)
        return set_err(ctx, TANG_EUNSUPPORTED, "no tensor-core kernel for a %u-block, %u-class model", m.blocks, m.C);
    // variants 1, 3, 4: the 1-SM kernel with weight tiles shared by clusters of 1, 2, 4 CTAs
    const int ci = v == 3 ? 1 : v == 4 ? 2 : 0;
    int rc = ci == 0 ? (f8 ? launch_1sm<true, 1>(ctx, maps[0], prm, st, tune) : launch_1sm<false, 1>(ctx, maps[0], prm, st, tune))
             : ci == 1 ? (f8 ? launch_1sm<true, 2>(ctx, maps[1], prm, st, tune) : launch_1sm<false, 2>(ctx, maps[1], prm, st, tune))
                       : (f8 ? launch_1sm<true, 4>(ctx, maps[2], prm, st, tune) : launch_1sm<false, 4>(ctx, maps[2], prm, st, tune));
    if (rc) return rc;
#ifdef TANG_TC_TRACE
    if (const char *path = getenv("TANG_TC_TRACE_FILE")) {
        std::vector<unsigned long long> hbuf(trace::kTotal);
        cudaMemcpyAsync(hbuf.data(), d_trace, sizeof(unsigned long long) * trace::kTotal, cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        if (FILE *f = fopen(path, "wb")) {
            fwrite(hbuf.data(), sizeof(unsigned long long), hbuf.size(), f);
            fclose(f);
        }
    }
#endif
    return TANG_OK;
}

}  // namespace tang
