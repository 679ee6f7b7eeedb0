// Fused classification kernel, 2-SM variant: a cluster of two CTAs (one per SM) forms a pair
// that runs each MMA with cta_group::2 (M = 256: 128 packets per CTA). Every CTA loads only
// its half of each weight tile (64 of the 128 output features of a chunk), so a CTA streams
// 32 B of weights per tensor-core clock instead of 64 B, and nine 8 KB stages cover about 2.3k
// cycles of L2 latency. The data flow per CTA is the one of the 1-SM kernel (mlp_tc.cu): layer 0
// on CUDA cores, block input x in TMEM as the A operand, FC1 output u in swizzled shared memory,
// double-buffered 128-column accumulators, epilogue warps, in-kernel exact search.
//
// Pair protocol (CTA rank 0 = leader):
//   - both CTAs' producers wait their own `empty` stage barrier, then load their half tile
//     with completion counted on the LEADER's `full` barrier (the leader announces the bytes
//     of both halves);
//   - the leader's MMA thread waits the leader's full / acc_empty / act barriers, issues pair
//     MMAs and commits to `empty` and `acc_full` in both CTAs (multicast);
//   - both CTAs' epilogue warps arrive on the leader's acc_empty and act barriers. Only the act
//     arrivals (which publish freshly written operands) use cluster-scope release; waits and
//     the other arrivals use the default CTA-scope semantics, which is what keeps the pair's
//     handoffs about as cheap as the 1-SM kernel's.
// Every wait is bounded as in the 1-SM kernel; the pair ends with a cluster barrier before TMEM
// is released.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "search_dev.cuh"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace tang {

namespace tc2 {
constexpr int kM = 128;             // packets per CTA (256 per pair)
constexpr int kHid = 512;
constexpr int kLayers = 12;
constexpr int kStages = 9;
constexpr int kStageBytes = 8192;   // 64 rows x 128 bytes: this CTA's half of a weight tile
constexpr int kThreads = 448;
constexpr int kWarpProd = 0, kWarpMma = 1, kWarpEpi = 2, kNumEpiWarps = 8, kWarpSearch = 10, kNumSearchWarps = 4;
constexpr uint64_t kTimeoutNs = 2000000000ull;
constexpr int kSmemTuples = 64;
constexpr uint32_t kXCol = 256;

constexpr int kOffY = 0;
constexpr int kYBytes = kM * kHid * 2;
constexpr int kOffStage = kOffY + kYBytes;
constexpr int kOffW0 = kOffStage + kStages * kStageBytes;
constexpr int kOffB0 = kOffW0 + 7 * kHid * 4;
constexpr int kOffTup = kOffB0 + kHid * 4;
constexpr int kOffOrd = kOffTup + kSmemTuples * 32;
constexpr int kOffTidx = kOffOrd + kSmemTuples * 2;
constexpr int kOffBar = kOffTidx + 2 * kM * 4;
constexpr int kNumBars = 2 * kStages + 2 + 2 + 8 + 2 + 2 + 1;
constexpr int kOffMisc = kOffBar + kNumBars * 8;
constexpr int kSmemBytes = kOffMisc + 16 + 1024;
}  // namespace tc2

template <bool F8>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(tc2::kThreads, 1)
    k_tc2_classify(const __grid_constant__ CUtensorMap tm_hid, const __grid_constant__ CUtensorMap tm_out,
                   const TcParams p) {
    using namespace tc2;
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
    uint64_t *act = acc_empty + 2;
    uint64_t *tfull = act + 8, *tempty = tfull + 2, *drain = tempty + 2;
    uint32_t *sTmem = reinterpret_cast<uint32_t *>(smem + kOffMisc);
    volatile int *sAbort = reinterpret_cast<volatile int *>(smem + kOffMisc + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = ptx::cluster_ctarank();
    const bool leader = rank == 0;
    const uint32_t pair = blockIdx.x >> 1, n_pairs = gridDim.x >> 1;
    constexpr int KB = F8 ? 4 : 8;
    constexpr int KBW = F8 ? 128 : 64;
    constexpr uint32_t kActArrivals = 2 * (F8 ? 8 : 4);  // epilogue warps of both CTAs per K-block

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&acc_full[b], 1);
            ptx::mbar_init(&acc_empty[b], 2 * kNumEpiWarps);
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
        ptx::tmem_alloc_cg2(sTmem, 512);
        ptx::tmem_relinquish_cg2();
    }
    ptx::tc_fence_before();
    ptx::cluster_sync();  // barriers of both CTAs are initialised before any remote arrival
    ptx::tc_fence_after();
    const uint32_t tmem = *sTmem;

    auto fail = [&](int code) {
        atomicOr(p.err, code);
        *sAbort = 1;
    };
    // leader's copies of the barriers both CTAs arrive on
    auto leader_bar = [&](uint64_t *b) { return ptx::mapa(ptx::smem_u32(b), 0); };

    if (warp == kWarpProd) {
        if (lane == 0) {
            uint32_t stage = 0, phase = 0, n_loads = 0;
            bool ok = true;
            const uint32_t out_half = p.Cpad / 2;
            for (uint32_t tile = pair; tile < p.n_tiles && ok; tile += n_pairs) {
                for (int L = 0; L <= kLayers && ok; ++L) {
                    const int nch = L == kLayers ? 1 : 4;
                    for (int c = 0; c < nch && ok; ++c)
                        for (int kb = 0; kb < KB; ++kb) {
                            if (!ptx::mbar_wait(&empty[stage], phase ^ 1, sAbort, kTimeoutNs)) {
                                fail(1);
                                ok = false;
                                break;
                            }
                            TC_TRACE2(trace::kProd + n_loads, n_loads < trace::kLoads);
                            ++n_loads;
                            const uint32_t half_bytes = L < kLayers ? kStageBytes : out_half * 128;
                            if (leader) ptx::mbar_arrive_expect_tx(&full[stage], 2 * half_bytes);
                            if (L < kLayers)
                                ptx::tma_load_2d_cg2(sStage + stage * kStageBytes, &tm_hid, leader_bar(&full[stage]),
                                                     kb * KBW, L * kHid + c * 128 + int(rank) * 64);
                            else
                                ptx::tma_load_2d_cg2(sStage + stage * kStageBytes, &tm_out, leader_bar(&full[stage]),
                                                     kb * KBW, int(rank * out_half));
                            if (++stage == kStages) {
                                stage = 0;
                                phase ^= 1;
                            }
                        }
                }
            }
            if (leader) {
                // every load of both CTAs is counted on the leader's full barriers
                volatile int never = 0;
                for (int s = 0; s < kStages; ++s) {
                    const uint32_t par = s < int(stage) ? phase : phase ^ 1;
                    ptx::mbar_wait(&full[s], par, &never, kTimeoutNs);
                }
            }
        }
    } else if (warp == kWarpMma) {
        if (lane == 0 && leader) {
            const uint32_t idesc_h = ptx::idesc_make(256, 128, F8);
            const uint32_t idesc_o = ptx::idesc_make(256, p.Cpad, F8);
            const uint32_t y_addr = ptx::smem_u32(sY), st_addr = ptx::smem_u32(sStage);
            uint32_t stage = 0, phase = 0, acc_cnt = 0, lay = 0;
            bool ok = true;
            for (uint32_t tile = pair; tile < p.n_tiles && ok; tile += n_pairs) {
                for (int L = 0; L <= kLayers && ok; ++L, ++lay) {
                    const bool a_tmem = (L & 1) == 0;
                    const int nch = L == kLayers ? 1 : 4;
                    const uint32_t idesc = L == kLayers ? idesc_o : idesc_h;
                    for (int c = 0; c < nch && ok; ++c, ++acc_cnt) {
                        const uint32_t buf = acc_cnt & 1, use = acc_cnt >> 1;
                        const bool tr = acc_cnt < uint32_t(trace::kChunks);
                        TC_TRACE2(trace::kMma + acc_cnt * 12 + 0, tr);
                        if (use > 0 && !ptx::mbar_wait(&acc_empty[buf], (use - 1) & 1, sAbort, kTimeoutNs)) {
                            fail(2);
                            ok = false;
                            break;
                        }
                        TC_TRACE2(trace::kMma + acc_cnt * 12 + 1, tr);
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
                            TC_TRACE2(trace::kMma + acc_cnt * 12 + 2 + kb, tr);
                            ptx::tc_fence_after();
                            const uint32_t b_base = st_addr + stage * kStageBytes;
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint64_t bd = ptx::sdesc_sw128(b_base + kk * 32);
                                const uint32_t accum = (kb | kk) != 0;
                                if (a_tmem)
                                    ptx::mma2_ts(d, tmem + kXCol + kb * 32 + kk * 8, bd, idesc, accum, F8);
                                else
                                    ptx::mma2_ss(d, ptx::sdesc_sw128(y_addr + kb * 16384 + kk * 32), bd, idesc, accum,
                                                 F8);
                            }
                            ptx::mma2_commit_mc(&empty[stage], 0x3);
                            if (++stage == kStages) {
                                stage = 0;
                                phase ^= 1;
                            }
                        }
                        if (!ok) break;
                        ptx::mma2_commit_mc(&acc_full[buf], 0x3);
                        TC_TRACE2(trace::kMma + acc_cnt * 12 + 10, tr);
                    }
                }
            }
            volatile int never = 0;
            ptx::mma2_commit_mc(drain, 0x1);
            ptx::mbar_wait(drain, 0, &never, kTimeoutNs);
        }
    } else if (warp < kWarpSearch) {
        const int ew = warp - kWarpEpi;
        const int q = warp & 3;
        const int hc = ew >> 2;
        const int r = q * 32 + lane;
        const uint32_t lane_base = uint32_t(q * 32) << 16;
        const float *sa = p.sa;
        uint32_t acc_cnt = 0, tcnt = 0;
        bool ok = true;
        uint32_t act_remote[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) act_remote[k] = leader_bar(&act[k]);
        const uint32_t acc_empty_remote[2] = {leader_bar(&acc_empty[0]), leader_bar(&acc_empty[1])};
        auto store_smem = [&](const uint32_t *w, int col0) {
            if (!F8) {
                const int kb = col0 >> 6, j0 = (col0 & 63) >> 3;
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
        auto x_col = [&](int col0) -> uint32_t { return tmem + lane_base + kXCol + (F8 ? col0 / 4 : col0 / 2); };
        auto act_arrive = [&](int col0) {
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive_cluster(act_remote[col0 / KBW]);
        };
        for (uint32_t tile = pair; tile < p.n_tiles && ok; tile += n_pairs) {
            const uint32_t i = tile * (2 * kM) + rank * kM + r;
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
                act_arrive(unit * 64);
            }
            for (int L = 0; L < kLayers && ok; ++L) {
                const bool fc2 = (L & 1) != 0;
                const float *bias = p.bias + L * kHid;
                const float *dq = F8 ? p.dq + L * kHid : nullptr;
                const float s_out = F8 ? sa[L + 1] : 1.f;
                const float s_res = F8 ? 1.f / sa[L - (fc2 ? 1 : 0)] : 1.f;
                for (int c = 0; c < 4; ++c, ++acc_cnt) {
                    const uint32_t buf = acc_cnt & 1, use = acc_cnt >> 1;
                    const bool tr = lane == 0 && (ew & 3) == 0 && acc_cnt < uint32_t(trace::kChunks);
                    const int tslot = trace::kEpi + ((ew >> 2) * trace::kChunks + int(acc_cnt)) * 4;
                    TC_TRACE2(tslot + 0, tr);
                    if (!ptx::mbar_wait(&acc_full[buf], use & 1, sAbort, kTimeoutNs)) {
                        fail(16);
                        ok = false;
                        break;
                    }
                    TC_TRACE2(tslot + 1, tr);
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
                            if (lane == 0) ptx::mbar_arrive_remote(acc_empty_remote[buf]);
                            TC_TRACE2(tslot + 2, tr);
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
                    TC_TRACE2(tslot + 3, tr);
                }
            }
            if (!ok) break;
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
                        ptx::tmem_ld32(tmem + lane_base + buf * 128 + c0, a);
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
                if (lane == 0) ptx::mbar_arrive_remote(acc_empty_remote[buf]);
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
        if (p.fused_search) {
            const int r = (warp - kWarpSearch) * 32 + lane;
            const TupleDesc *tuples = tup_smem ? sTup : tb.tuples;
            const uint16_t *order = tup_smem ? sOrd : tb.order;
            uint32_t tcnt = 0;
            uint32_t st_pk = 0, st_match = 0, st_correct = 0, st_hit = 0, st_fb = 0;
            Counters cn{0, 0, 0};
            for (uint32_t tile = pair; tile < p.n_tiles; tile += n_pairs) {
                const uint32_t t = tcnt & 1, tu = tcnt >> 1;
                ++tcnt;
                if (!ptx::mbar_wait(&tfull[t], tu & 1, sAbort, kTimeoutNs)) {
                    fail(128);
                    break;
                }
                const int pred = sTidx[t * kM + r];
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&tempty[t]);
                const uint32_t i = tile * (2 * kM) + rank * kM + r;
                if (i < p.n) {
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
    ptx::cluster_sync();  // the leader's drains cover loads and MMAs that touch the peer
    ptx::tc_fence_after();
    if (warp == kWarpMma) ptx::tmem_dealloc_cg2(tmem, 512);
}

// Tensor maps for the half tiles (64 rows per CTA; Cpad/2 rows of the output layer).
int tc2_prepare_model(tang_ctx *ctx, DeviceModel &m) {
    if (!m.d_wbf16 || m.Cpad % 32 != 0) return TANG_OK;
    const size_t hid = size_t(tc2::kLayers) * m.N * m.N;
    TcMaps *maps = static_cast<TcMaps *>(aligned_alloc(64, sizeof(TcMaps)));
    m.tmap2_bf16 = maps;
    int rc = make_tmap(ctx, &maps->hid, m.d_wbf16, tc2::kLayers * m.N, false, 64);
    if (!rc) rc = make_tmap(ctx, &maps->out, static_cast<__nv_bfloat16 *>(m.d_wbf16) + hid, m.Cpad, false, m.Cpad / 2);
    if (rc) return rc;
    if (m.d_wfp8) {
        TcMaps *m8 = static_cast<TcMaps *>(aligned_alloc(64, sizeof(TcMaps)));
        m.tmap2_fp8 = m8;
        rc = make_tmap(ctx, &m8->hid, m.d_wfp8, tc2::kLayers * m.N, true, 64);
        if (!rc) rc = make_tmap(ctx, &m8->out, static_cast<uint8_t *>(m.d_wfp8) + hid, m.Cpad, true, m.Cpad / 2);
    }
    return rc;
}

// Launch the pair kernel; returns TANG_EUNSUPPORTED when the model has no 2-SM maps.
int tc2_launch(tang_ctx *ctx, DeviceModel &m, const TcParams &prm_in, bool f8, cudaStream_t st, int grid_cap) {
    const TcMaps *maps = static_cast<const TcMaps *>(f8 ? m.tmap2_fp8 : m.tmap2_bf16);
    if (!maps) return TANG_EUNSUPPORTED;
    static bool attr_done[2] = {false, false};
    static int max_pairs[2] = {0, 0};
    if (!attr_done[f8]) {
        cudaError_t e = f8 ? cudaFuncSetAttribute(k_tc2_classify<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  tc2::kSmemBytes)
                           : cudaFuncSetAttribute(k_tc2_classify<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  tc2::kSmemBytes);
        if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "smem attribute (2-SM): %s", cudaGetErrorString(e));
        cudaLaunchConfig_t q = {};
        q.gridDim = dim3(2 * 74, 1, 1);
        q.blockDim = dim3(tc2::kThreads, 1, 1);
        q.dynamicSmemBytes = tc2::kSmemBytes;
        cudaLaunchAttribute qa[1];
        qa[0].id = cudaLaunchAttributeClusterDimension;
        qa[0].val.clusterDim.x = 2;
        qa[0].val.clusterDim.y = 1;
        qa[0].val.clusterDim.z = 1;
        q.attrs = qa;
        q.numAttrs = 1;
        int clusters = 0;
        e = f8 ? cudaOccupancyMaxActiveClusters(&clusters, k_tc2_classify<true>, &q)
               : cudaOccupancyMaxActiveClusters(&clusters, k_tc2_classify<false>, &q);
        if (e != cudaSuccess || clusters <= 0) {
            cudaGetLastError();
            clusters = ctx->sm_count / 2;
        }
        max_pairs[f8] = clusters;
        attr_done[f8] = true;
    }
    TcParams prm = prm_in;
    prm.n_tiles = (prm.n + 2 * tc2::kM - 1) / (2 * tc2::kM);
#ifdef TANG_TC_TRACE
    static unsigned long long *d_trace2 = nullptr;
    if (!d_trace2) cudaMalloc(&d_trace2, sizeof(unsigned long long) * 2 * trace::kTotal);
    cudaMemsetAsync(d_trace2, 0, sizeof(unsigned long long) * 2 * trace::kTotal, st);
    prm.trace = d_trace2;
#endif
    uint32_t pairs = uint32_t(max_pairs[f8]);
    if (grid_cap > 0) pairs = std::min<uint32_t>(pairs, uint32_t(grid_cap / 2));
    pairs = std::max<uint32_t>(1, std::min<uint32_t>(pairs, prm.n_tiles));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * pairs, 1, 1);
    cfg.blockDim = dim3(tc2::kThreads, 1, 1);
    cfg.dynamicSmemBytes = tc2::kSmemBytes;
    cfg.stream = st;
    cudaError_t e = f8 ? cudaLaunchKernelEx(&cfg, k_tc2_classify<true>, maps->hid, maps->out, prm)
                       : cudaLaunchKernelEx(&cfg, k_tc2_classify<false>, maps->hid, maps->out, prm);
    if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "2-SM kernel launch: %s", cudaGetErrorString(e));
#ifdef TANG_TC_TRACE
    if (const char *path = getenv("TANG_TC_TRACE_FILE")) {
        std::vector<unsigned long long> hbuf(2 * trace::kTotal);
        cudaMemcpyAsync(hbuf.data(), d_trace2, sizeof(unsigned long long) * hbuf.size(), cudaMemcpyDeviceToHost, st);
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
