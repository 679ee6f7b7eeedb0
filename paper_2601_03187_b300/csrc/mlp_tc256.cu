// Fused classification kernel with 256-wide MMAs (the default tensor-core variant).
//
// Each tcgen05.mma here is M=128 x N=256 (K=16 BF16 / K=32 E4M3), twice the work per
// instruction of the N=128 kernel in mlp_tc.cu; issuing the same MMA count at N=128 leaves the
// tensor pipe about two-thirds idle. A 256-column FP32 accumulator cannot be double-buffered
// next to the block input x (256 columns of packed BF16) in the 512-column TMEM, so it is
// single-buffered and the epilogue is built to release it quickly: 16 epilogue warps (four per
// TMEM lane quadrant) each pull their 32 rows x 64 columns into registers with two loads and
// release the accumulator at once; bias, residual, ReLU, quantisation and the operand stores
// then overlap the next chunk's MMAs.
//
// Per tile (128 packets): layer 0 on CUDA cores -> x (TMEM); per block: FC1 in two 256-column
// chunks (A = x from TMEM) -> u (swizzled shared memory); FC2 in two chunks (A = u from shared
// memory) -> x = ReLU(acc + b2 + x) in place (Eq. 1); output FC (N = Cpad) + argmax; the exact
// search of §4.1.1 on 2 search warps. Weight tiles are 256 rows x 128 bytes (32 KB), streamed by
// TMA through two stages. All waits are bounded (2 s of %globaltimer) as in the other kernels.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "search_dev.cuh"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace tang {

namespace tc256 {
constexpr int kM = 128;
constexpr int kHid = 512;
constexpr int kLayers = 12;
constexpr int kStages = 2;
constexpr int kStageBytes = 32768;  // 256 rows x 128 bytes
constexpr int kNumEpiWarps = 16;
constexpr int kWarpProd = 0, kWarpMma = 1, kWarpEpi = 2, kWarpSearch = kWarpEpi + kNumEpiWarps, kNumSearchWarps = 2;
constexpr int kThreads = 32 * (kWarpSearch + kNumSearchWarps);  // 640
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
constexpr int kNumBars = 2 * kStages + 1 + 1 + 8 + 2 + 2 + 1;
constexpr int kOffMisc = kOffBar + kNumBars * 8;
constexpr int kSmemBytes = kOffMisc + 16 + 1024;
}  // namespace tc256

// 20 warps: at most 5 per SM sub-partition, whose 16K-entry register file then holds 96 registers
// per thread (5 x 32 x 96 = 15,360).
template <bool F8>
__global__ void __maxnreg__(96)
    k_tc256_classify(const __grid_constant__ CUtensorMap tm_hid, const __grid_constant__ CUtensorMap tm_out,
                     const TcParams p) {
    using namespace tc256;
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
    uint64_t *acc_full = bars + 2 * kStages, *acc_empty = acc_full + 1;
    uint64_t *act = acc_empty + 1;  // 8 barriers, one per K-block of the next layer's input
    uint64_t *tfull = act + 8, *tempty = tfull + 2, *drain = tempty + 2;
    uint32_t *sTmem = reinterpret_cast<uint32_t *>(smem + kOffMisc);
    volatile int *sAbort = reinterpret_cast<volatile int *>(smem + kOffMisc + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int KB = F8 ? 4 : 8;
    constexpr int KBW = F8 ? 128 : 64;
    constexpr uint32_t kActArrivals = F8 ? 8 : 4;  // 64-column units per K-block x 4 lane quadrants

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 1);
        }
        ptx::mbar_init(acc_full, 1);
        ptx::mbar_init(acc_empty, kNumEpiWarps);
        for (int b = 0; b < 2; ++b) {
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
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *sTmem;

    auto fail = [&](int code) {
        atomicOr(p.err, code);
        *sAbort = 1;
    };

    if (warp == kWarpProd) {
        if (lane == 0) {
            uint32_t stage = 0, phase = 0, n_loads = 0;
            bool ok = true;
            for (uint32_t tile = blockIdx.x; tile < p.n_tiles && ok; tile += gridDim.x) {
                for (int L = 0; L <= kLayers && ok; ++L) {
                    const int nch = L == kLayers ? 1 : 2;
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
                                ptx::tma_load_2d(dst, &tm_hid, &full[stage], kb * KBW, L * kHid + c * 256);
                            } else {
                                ptx::mbar_arrive_expect_tx(&full[stage], p.Cpad * 128);
                                ptx::tma_load_2d(dst, &tm_out, &full[stage], kb * KBW, 0);
                            }
                            if (++stage == kStages) {
                                stage = 0;
                                phase ^= 1;
                            }
                        }
                }
            }
            volatile int never = 0;
            for (int s = 0; s < kStages; ++s) {
                const uint32_t par = s < int(stage) ? phase : phase ^ 1;
                ptx::mbar_wait(&full[s], par, &never, kTimeoutNs);
            }
        }
    } else if (warp == kWarpMma) {
        if (lane == 0) {
            const uint32_t idesc_h = ptx::idesc_make(128, 256, F8);
            const uint32_t idesc_o = ptx::idesc_make(128, p.Cpad, F8);
            const uint32_t y_addr = ptx::smem_u32(sY), st_addr = ptx::smem_u32(sStage);
            uint32_t stage = 0, phase = 0, uses = 0, lay = 0;
            bool ok = true;
            for (uint32_t tile = blockIdx.x; tile < p.n_tiles && ok; tile += gridDim.x) {
                for (int L = 0; L <= kLayers && ok; ++L, ++lay) {
                    const bool a_tmem = (L & 1) == 0;  // FC1 and the output layer read x from TMEM
                    const int nch = L == kLayers ? 1 : 2;
                    const uint32_t idesc = L == kLayers ? idesc_o : idesc_h;
                    for (int c = 0; c < nch && ok; ++c, ++uses) {
                        const bool tr = uses < uint32_t(trace::kChunks);
                        TC_TRACE(trace::kMma + uses * 12 + 0, tr);
                        if (uses > 0 && !ptx::mbar_wait(acc_empty, (uses - 1) & 1, sAbort, kTimeoutNs)) {
                            fail(2);
                            ok = false;
                            break;
                        }
                        TC_TRACE(trace::kMma + uses * 12 + 1, tr);
                        ptx::tc_fence_after();
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
                            TC_TRACE(trace::kMma + uses * 12 + 2 + kb, tr);
                            ptx::tc_fence_after();
                            const uint32_t b_base = st_addr + stage * kStageBytes;
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint64_t bd = ptx::sdesc_sw128(b_base + kk * 32);
                                const uint32_t accum = (kb | kk) != 0;
                                if (a_tmem)
                                    ptx::mma_ts(tmem, tmem + kXCol + kb * 32 + kk * 8, bd, idesc, accum, F8);
                                else
                                    ptx::mma_ss(tmem, ptx::sdesc_sw128(y_addr + kb * 16384 + kk * 32), bd, idesc, accum, F8);
                            }
                            ptx::mma_commit(&empty[stage]);
                            if (++stage == kStages) {
                                stage = 0;
                                phase ^= 1;
                            }
                        }
                        if (!ok) break;
                        ptx::mma_commit(acc_full);
                        TC_TRACE(trace::kMma + uses * 12 + 10, tr);
                    }
                }
            }
            volatile int never = 0;
            ptx::mma_commit(drain);
            ptx::mbar_wait(drain, 0, &never, kTimeoutNs);
        }
    } else if (warp < kWarpSearch) {
        // ---------------- 16 epilogue warps ----------------
        const int ew = warp - kWarpEpi;
        const int q = warp & 3;   // TMEM lane quadrant
        const int g = ew >> 2;    // 64-column unit of every 256-column chunk
        const int r = q * 32 + lane;
        const uint32_t lane_base = uint32_t(q * 32) << 16;
        const float *sa = p.sa;
        uint32_t uses = 0, tcnt = 0;
        bool ok = true;
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
            if (lane == 0) ptx::mbar_arrive(&act[col0 / KBW]);
        };
        // ReLU, quantise and store 32 activations (columns col0 ..) of the next layer's input
        auto emit = [&](float *v, int col0, bool to_x, float s_out) {
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = fmaxf(v[j], 0.f);
            if (!F8) {
                uint32_t w[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) w[j] = pack_bf16(v[2 * j], v[2 * j + 1]);
                if (to_x)
                    ptx::tmem_st16(x_col(col0), w);
                else
                    store_smem(w, col0);
            } else {
                uint32_t w[8];
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    w[j] = pack_e4m3x4(v[4 * j] * s_out, v[4 * j + 1] * s_out, v[4 * j + 2] * s_out, v[4 * j + 3] * s_out);
                if (to_x)
                    ptx::tmem_st8(x_col(col0), w);
                else
                    store_smem(w, col0);
            }
        };

        for (uint32_t tile = blockIdx.x; tile < p.n_tiles && ok; tile += gridDim.x) {
            const uint32_t i = tile * kM + r;
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
            // ---- layer 0 (FP32, CUDA cores): units g and g+4 of x
            for (int h = 0; h < 2; ++h) {
                const int unit = g + 4 * h;
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const int col0 = unit * 64 + s * 32;
                    float v[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        float a = sB0[col0 + j];
#pragma unroll
                        for (int t = 0; t < 7; ++t) a = fmaf(f[t], sW0[t * kHid + col0 + j], a);
                        v[j] = a;
                    }
                    emit(v, col0, true, F8 ? sa[0] : 1.f);
                }
                ptx::tmem_wait_st();
                act_arrive(unit * 64);
            }
            // ---- hidden layers, two 256-column chunks each
            for (int L = 0; L < kLayers && ok; ++L) {
                const bool fc2 = (L & 1) != 0;
                const float *bias = p.bias + L * kHid;
                const float *dq = F8 ? p.dq + L * kHid : nullptr;
                const float s_out = F8 ? sa[L + 1] : 1.f;
                const float s_res = F8 ? 1.f / sa[fc2 ? L - 1 : L] : 1.f;
                for (int c = 0; c < 2; ++c, ++uses) {
                    const bool tr = lane == 0 && q == 2 && g < 2 && uses < uint32_t(trace::kChunks);
                    const int tslot = trace::kEpi + (g * trace::kChunks + int(uses)) * 4;
                    TC_TRACE(tslot + 0, tr);
                    if (!ptx::mbar_wait(acc_full, uses & 1, sAbort, kTimeoutNs)) {
                        fail(16);
                        ok = false;
                        break;
                    }
                    TC_TRACE(tslot + 1, tr);
                    ptx::tc_fence_after();
                    const int unit = 4 * c + g;
                    uint32_t a0[32], a1[32];
                    ptx::tmem_ld32(tmem + lane_base + g * 64, a0);
                    ptx::tmem_ld32(tmem + lane_base + g * 64 + 32, a1);
                    ptx::tmem_wait_ld();
                    // the accumulator may take the next chunk's MMAs now
                    ptx::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(acc_empty);
                    TC_TRACE(tslot + 2, tr);
#pragma unroll
                    for (int s = 0; s < 2; ++s) {
                        const int col0 = unit * 64 + s * 32;
                        const uint32_t *a = s == 0 ? a0 : a1;
                        float v[32];
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float y = __uint_as_float(a[j]);
                            v[j] = F8 ? fmaf(y, __ldg(dq + col0 + j), __ldg(bias + col0 + j)) : y + __ldg(bias + col0 + j);
                        }
                        if (fc2) {
                            if (!F8) {
                                uint32_t xr[16];
                                ptx::tmem_ld16(x_col(col0), xr);
                                ptx::tmem_wait_ld();
#pragma unroll
                                for (int j = 0; j < 16; ++j) {
                                    v[2 * j] += __uint_as_float(xr[j] << 16);
                                    v[2 * j + 1] += __uint_as_float(xr[j] & 0xFFFF0000u);
                                }
                            } else {
                                uint32_t xr[8];
                                ptx::tmem_ld8(x_col(col0), xr);
                                ptx::tmem_wait_ld();
#pragma unroll
                                for (int j = 0; j < 8; ++j)
#pragma unroll
                                    for (int b = 0; b < 4; ++b) v[4 * j + b] += e4m3_to_f((xr[j] >> (8 * b)) & 0xFFu) * s_res;
                            }
                        }
                        emit(v, col0, fc2, s_out);
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
            // ---- output layer: logits and argmax on the g == 0 warps
            {
                if (!ptx::mbar_wait(acc_full, uses & 1, sAbort, kTimeoutNs)) {
                    fail(32);
                    ok = false;
                    break;
                }
                ++uses;
                ptx::tc_fence_after();
                int arg = 0;
                if (g == 0) {
                    float best = -INFINITY;
                    const float *bias = p.bias + kLayers * kHid;
                    const float *dq = F8 ? p.dq + kLayers * kHid : nullptr;
                    for (uint32_t c0 = 0; c0 < p.Cpad; c0 += 32) {
                        uint32_t a[32];
                        ptx::tmem_ld32(tmem + lane_base + c0, a);
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
                if (lane == 0) ptx::mbar_arrive(acc_empty);
                if (g == 0) {
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
        // ---------------- search warps ----------------
        if (p.fused_search) {
            const int r = (warp - kWarpSearch) * 32 + lane;
            const TupleDesc *tuples = tup_smem ? sTup : tb.tuples;
            const uint16_t *order = tup_smem ? sOrd : tb.order;
            uint32_t tcnt = 0;
            uint32_t st_pk = 0, st_match = 0, st_correct = 0, st_hit = 0, st_fb = 0;
            Counters cn{0, 0, 0};
            for (uint32_t tile = blockIdx.x; tile < p.n_tiles; tile += gridDim.x) {
                const uint32_t t = tcnt & 1, tu = tcnt >> 1;
                ++tcnt;
                if (!ptx::mbar_wait(&tfull[t], tu & 1, sAbort, kTimeoutNs)) {
                    fail(128);
                    break;
                }
                // each search thread owns rows r and r + 64 of the tile
                const int pred0 = sTidx[t * kM + r], pred1 = sTidx[t * kM + r + 64];
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&tempty[t]);
                for (int h2 = 0; h2 < 2; ++h2) {
                    const uint32_t i = tile * kM + r + 64 * h2;
                    const int pred = h2 ? pred1 : pred0;
                    if (i < p.n) {
                        const Hdr h = load_header(p.headers + i);
                        Best best;
                        const bool hit = search_packet(tb, tuples, order, h, pred, best, cn);
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
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == kWarpMma) ptx::tmem_dealloc(tmem, 512);
}

// 256-row hidden-layer maps (the output-layer map of the 1-SM kernel is reused).
int tc256_prepare_model(tang_ctx *ctx, DeviceModel &m) {
    if (!m.d_wbf16) return TANG_OK;
    TcMaps *maps = static_cast<TcMaps *>(aligned_alloc(64, 2 * sizeof(TcMaps)));
    m.tmap256 = maps;
    const TcMaps *one = static_cast<const TcMaps *>(m.tmap_bf16);
    maps[0].out = one[0].out;
    int rc = make_tmap(ctx, &maps[0].hid, m.d_wbf16, tc256::kLayers * m.N, false, 256);
    if (rc) return rc;
    if (m.d_wfp8) {
        const TcMaps *one8 = static_cast<const TcMaps *>(m.tmap_fp8);
        maps[1].out = one8[0].out;
        rc = make_tmap(ctx, &maps[1].hid, m.d_wfp8, tc256::kLayers * m.N, true, 256);
    }
    return rc;
}

int tc256_launch(tang_ctx *ctx, DeviceModel &m, const TcParams &prm, bool f8, cudaStream_t st, int grid_cap) {
    if (!m.tmap256 || (f8 && !m.d_wfp8)) return TANG_EUNSUPPORTED;
    const TcMaps &maps = static_cast<const TcMaps *>(m.tmap256)[f8 ? 1 : 0];
    static bool attr_done[2] = {false, false};
    if (!attr_done[f8]) {
        cudaError_t e = f8 ? cudaFuncSetAttribute(k_tc256_classify<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  tc256::kSmemBytes)
                           : cudaFuncSetAttribute(k_tc256_classify<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  tc256::kSmemBytes);
        if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "smem attribute (N=256): %s", cudaGetErrorString(e));
        attr_done[f8] = true;
    }
    uint32_t grid = uint32_t(grid_cap > 0 ? grid_cap : ctx->sm_count);
    grid = std::min<uint32_t>(prm.n_tiles, std::min<uint32_t>(grid, uint32_t(ctx->sm_count)));
    TcParams prm_t = prm;
#ifdef TANG_TC_TRACE
    static unsigned long long *d_trace = nullptr;
    if (!d_trace) cudaMalloc(&d_trace, sizeof(unsigned long long) * trace::kTotal);
    cudaMemsetAsync(d_trace, 0, sizeof(unsigned long long) * trace::kTotal, st);
    prm_t.trace = d_trace;
#endif
    if (f8)
        k_tc256_classify<true><<<grid, tc256::kThreads, tc256::kSmemBytes, st>>>(maps.hid, maps.out, prm_t);
    else
        k_tc256_classify<false><<<grid, tc256::kThreads, tc256::kSmemBytes, st>>>(maps.hid, maps.out, prm_t);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "N=256 kernel launch: %s", cudaGetErrorString(e));
#ifdef TANG_TC_TRACE
    if (const char *path = getenv("TANG_TC_TRACE_FILE")) {
        std::vector<unsigned long long> hbuf(trace::kTotal);
        cudaMemcpyAsync(hbuf.data(), d_trace, sizeof(unsigned long long) * hbuf.size(), cudaMemcpyDeviceToHost, st);
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
