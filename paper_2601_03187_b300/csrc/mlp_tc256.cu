// Fused classification kernel with 256-wide MMAs (the default tensor-core variant).
//
// Each tcgen05.mma here is M=128 x N=256 (K=16 BF16 / K=32 E4M3). An N=128 MMA was measured to
// take about as many cycles as an N=256 one, so N=128 chunks would leave the tensor pipe about
// half idle (an earlier N=128 kernel with two accumulators ran at about half this kernel's
// rate). A 256-column FP32 accumulator cannot be double-buffered
// next to the block input x (256 columns of packed BF16) in the 512-column TMEM, so it is
// single-buffered and the epilogue is built to release it quickly: 16 epilogue warps (four per
// TMEM lane quadrant) each pull their 32 rows x 64 columns into registers with two loads and
// release the accumulator at once; bias, residual, ReLU, quantisation and the operand stores
// then overlap the next chunk's MMAs.
//
// Per tile (128 packets), for the paper's width 512: layer 0 on the tensor core -> x (TMEM); per
// block: FC1 in two 256-column chunks (A = x from TMEM) -> u (swizzled shared memory); FC2 in two
// chunks (A = u from shared memory) -> x = ReLU(acc + b2 + x) in place (Eq. 1); output FC in
// 256-column chunks (any tuple count) + argmax; the exact search of §5.1.1 on 4 search warps.
// The width is a template parameter: at 256 every layer is one chunk and u and x take half the
// space.
//
// Layer 0 (7 header fields -> width, FP32 in the other kernels) is one K=48 BF16 contraction per
// 256 columns with FP32 accumulation: every 16-bit field f splits exactly into bytes,
// f = 256 * hi + lo, and every weight and bias into three BF16 parts w1 + w2 + w3 that carry its
// 24 significant bits, so A = [hi(7), lo(7)] x 3 parts, 1 x 3 bias parts, and all products are
// exact. The sum matches the FP32 one up to accumulation order (a few units in the last FP32
// place), far below the BF16 / E4M3 rounding applied next. On CUDA cores the same layer costs a
// uniform broadcast per weight per warp, about 9k cycles per tile at one broadcast per cycle.
//
// Weight tiles are 256 rows x 128 bytes (32 KB), streamed by TMA through three stages (BF16) or
// four (FP8, whose u lives in TMEM), so that at a chunk boundary the next chunk's first
// K-blocks are already in flight while the accumulator changes hands. The epilogue spends few
// instructions per element: vector bias loads, ReLU folded into the packing conversion, and for
// FP8 the output scale folded into the per-column constants (exact, the scales being powers of
// two) and two-at-a-time E4M3 decoding of the residual. All waits are bounded (2 s of
// %globaltimer) as in the other kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "search_dev.cuh"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace tang {

namespace tc256 {
constexpr int kM = 128;
constexpr int kNumEpiWarps = 16;
// Warp groups (4 warps each): 0 = producer (warp 0) and MMA issuer (warp 1); 1..4 = the epilogue;
// 5 = the search. Every sub-partition gets one warp of each group.
constexpr int kWarpProd = 0, kWarpMma = 1, kWarpEpi = 4, kWarpSearch = kWarpEpi + kNumEpiWarps, kNumSearchWarps = 4;
constexpr int kThreads = 32 * (kWarpSearch + kNumSearchWarps);  // 768
// Registers per thread: launched at kRegLaunch, then moved between groups with setmaxnreg so the
// epilogue gets kRegEpi. The shares must add up to the launch total exactly (an increase waits
// until decreases have freed enough), per sub-partition as well as per CTA.
constexpr int kRegLaunch = 80, kRegCtl = 40, kRegEpi = 96, kRegSearch = 56;
static_assert(kRegCtl + 4 * kRegEpi + kRegSearch == 6 * kRegLaunch, "register split must match the launch total");
static_assert(kRegCtl <= kRegLaunch && kRegSearch <= kRegLaunch && kRegEpi >= kRegLaunch,
              "setmaxnreg.dec may only lower and setmaxnreg.inc only raise a warp's registers");
static_assert(kRegCtl % 8 == 0 && kRegEpi % 8 == 0 && kRegSearch % 8 == 0, "setmaxnreg takes multiples of 8");
static_assert(kThreads * kRegLaunch <= 65536, "register file");
constexpr uint64_t kTimeoutNs = 2000000000ull;
constexpr uint32_t kXCol = 256;
// FP8 only: the FC1 output u (E4M3, 4 per 32-bit column: 128 columns at width 512) in the TMEM
// columns BF16's wider x occupies, so that FC2 reads its A operand from TMEM as FC1 does (an
// M=128, N=256 MMA measured 144 cycles with A in TMEM against 171 with A in shared memory)
constexpr uint32_t kUCol = 384;
constexpr int kL0K = 64;     // layer-0 contraction width (48 used, zero padded to one 128-byte row)
constexpr int kL0Kused = 48;
// Column group whose warps combine the partial argmax: its layer-0 units (3 and 7) are the last
// ones the next tile's first MMAs need.
constexpr int kArgG = 3;

// Shared memory: for BF16 u (the FC1 output as swizzled K-blocks of 128 rows x 128 bytes; its
// first 16 KB also hold the next tile's layer-0 operand between the last FC2 and the next FC1
// epilogue), for FP8 (u in TMEM) the layer-0 operand alone; the weight stages, the
// predicted-tuple handoff to the search warps, the barriers, the partial argmax.
// P: the CTA-pair kernel, whose CTAs each hold half of every 256-row weight tile (16 KB stages;
// the freed shared memory buys deeper weight pipelines).
template <bool F8, int HID, bool P = false>
struct Layout {
    static constexpr int kStageBytes = P ? 16384 : 32768;  // 128 / 256 rows x 128 bytes
    static constexpr int kStages = P ? (F8 ? 8 : 6) : (F8 ? 4 : 3);
    static constexpr int kYBytes = F8 ? kM * 128 : kM * HID * 2;
    static constexpr int kOffStage = kYBytes;
    static constexpr int kOffTidx = kOffStage + kStages * kStageBytes;
    static constexpr int kOffBar = kOffTidx + 2 * kM * 4;
    static constexpr int kNumBars = 2 * kStages + 1 + 1 + 8 + 2 + 2 + 1 + 1 + 1;
    static constexpr int kOffMisc = kOffBar + kNumBars * 8;
    // per-row partial argmax of the four column groups ([4][128] floats, then [4][128] ints): in
    // the u buffer's second half for BF16 (idle from the last FC2 to the next tile's FC1 epilogue
    // that writes it), in a region of its own for FP8
    static constexpr int kOffPart = F8 ? kOffMisc + 16 : kYBytes / 2;
    static constexpr int kSmemBytes = (F8 ? kOffPart + 4096 : kOffMisc + 16) + 1024;  // + slack to align the base
    static_assert(kSmemBytes <= 232448, "exceeds the 227 KB of shared memory per CTA");
};
}  // namespace tc256

// 24 warps, launched at 80 registers per thread (6 x 32 x 80 = 15,360 of a sub-partition's 16K);
// after setup the control group drops to 40, the search group to 56 and the epilogue rises to 96.
//
// P (CTA pairs): the kernel runs in clusters of two CTAs on two SMs. Each CTA keeps its own
// 128-packet tile, its own accumulator and x in its TMEM and its own u (BF16: shared memory, FP8: TMEM), but the
// first CTA's MMA warp issues every MMA for both as one cta_group::2 MMA with M = 256: each CTA
// loads only its 128 rows (output columns) of each weight tile, so an SM streams and reads half
// the weight bytes per MMA and issues no MMAs of its own half the time. The barriers the MMAs wait
// on (stages full, accumulator drained, activations published) live in the first CTA and count
// both CTAs' arrivals; the MMA commits arrive in both CTAs.
template <bool F8, int HID, bool P>
__global__ void __launch_bounds__(tc256::kThreads, 1)
    k_tc256_classify(const __grid_constant__ CUtensorMap tm_hid, const __grid_constant__ CUtensorMap tm_out,
                     const __grid_constant__ CUtensorMap tm_l0, const TcParams p) {
    using namespace tc256;
    using Lay = Layout<F8, HID, P>;
    constexpr int kStages = Lay::kStages;
    constexpr int kStageBytes = Lay::kStageBytes;
    constexpr int kPair = P ? 2 : 1;  // CTAs that arrive on the MMA-side barriers
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sY = smem;
    uint8_t *sStage = smem + Lay::kOffStage;
    int32_t *sTidx = reinterpret_cast<int32_t *>(smem + Lay::kOffTidx);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + Lay::kOffBar);
    uint64_t *full = bars, *empty = bars + kStages;
    uint64_t *acc_full = bars + 2 * kStages, *acc_empty = acc_full + 1;
    uint64_t *act = acc_empty + 1;  // 8 barriers, one per K-block of the next layer's input
    uint64_t *tfull = act + 8, *tempty = tfull + 2, *drain = tempty + 2, *part_full = drain + 1;
    uint64_t *feat_full = part_full + 1;  // the layer-0 operand of the current tile is in place
    float *sPartBest = reinterpret_cast<float *>(smem + Lay::kOffPart);
    int32_t *sPartArg = reinterpret_cast<int32_t *>(smem + Lay::kOffPart + 2048);
    uint32_t *sTmem = reinterpret_cast<uint32_t *>(smem + Lay::kOffMisc);
    volatile int *sAbort = reinterpret_cast<volatile int *>(smem + Lay::kOffMisc + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nl = int(p.layers);  // N x N layers: 2 per residual block
    // the output layer in 256-column chunks (Cpad is a multiple of 32; the weight rows are padded
    // to whole 256-row tiles when Cpad > 256, so every tile load is in bounds)
    const int n_oc = int((p.Cpad + 255) >> 8);
    const uint32_t out_box = p.Cpad < 256 ? p.Cpad : 256u;
    constexpr int KBW = F8 ? 128 : 64;  // K per weight stage: 128 bytes of a row
    constexpr int KB = HID / KBW;       // K-blocks per layer
    constexpr int NCH = HID / 256;      // 256-column chunks per layer
    // Arrivals per K-block of the next layer's input: one per 32-column piece x 4 lane quadrants
    // (the hidden-layer epilogue publishes 32 columns at a time; layer 0 arrives twice per
    // 64-column unit)
    constexpr uint32_t kActArrivals = F8 ? 16 : 8;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 1);
        }
        ptx::mbar_init(acc_full, 1);
        ptx::mbar_init(acc_empty, kPair * kNumEpiWarps);
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&tfull[b], 4);
            ptx::mbar_init(&tempty[b], kNumSearchWarps);
        }
        for (int k = 0; k < 8; ++k) ptx::mbar_init(&act[k], kPair * kActArrivals);
        ptx::mbar_init(drain, 1);
        ptx::mbar_init(part_full, 4 * (kNumEpiWarps / 4 - 1));
        ptx::mbar_init(feat_full, kPair * 4);
        *sAbort = 0;
        ptx::fence_mbar_init();
    }
    if (warp == kWarpProd && lane == 0) {
        ptx::prefetch_tmap(&tm_hid);
        ptx::prefetch_tmap(&tm_out);
        ptx::prefetch_tmap(&tm_l0);
    }
    if (warp == kWarpMma) {
        if (P) {
            ptx::tmem_alloc_cg2(sTmem, 512);
            ptx::tmem_relinquish_cg2();
        } else {
            ptx::tmem_alloc(sTmem, 512);
            ptx::tmem_relinquish();
        }
    }
    ptx::tc_fence_before();
    if (P)
        ptx::cluster_sync();  // both CTAs' barriers are initialised before any arrival from the other
    else
        __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *sTmem;
    // Tiles: a CTA pair takes pair-tiles pt = first, first + step, ...; its CTA of rank r works on
    // tile 2 pt + r (past the last tile its rows are all beyond n: computed, never written).
    const uint32_t rank = P ? ptx::cluster_ctarank() : 0u;
    const uint32_t pt_first = P ? blockIdx.x >> 1 : blockIdx.x, pt_step = P ? gridDim.x >> 1 : gridDim.x;
    const uint32_t n_pt = P ? (p.n_tiles + 1) >> 1 : p.n_tiles;
    auto tile_of = [&](uint32_t pt) { return P ? 2 * pt + rank : pt; };
    // shared::cluster address of a barrier in the first CTA of the pair (this CTA's own otherwise)
    auto lead = [&](uint64_t *b) { return P ? ptx::mapa(ptx::smem_u32(b), 0) : ptx::smem_u32(b); };
    // arrival on a barrier the MMA warp waits for
    auto arrive_mma_side = [&](uint64_t *b) {
        if (P)
            ptx::mbar_arrive_cluster(lead(b));
        else
            ptx::mbar_arrive(b);
    };
    // the accumulator release: in a pair a relaxed arrive (see mbar_arrive_cluster_relaxed)
    auto release_acc = [&]() {
        if (P)
            ptx::mbar_arrive_cluster_relaxed(lead(acc_empty));
        else
            ptx::mbar_arrive(acc_empty);
    };
    // waits on barriers that receive arrivals or MMA commits from the other CTA of a pair
    auto wait_x = [&](uint64_t *b, uint32_t parity) {
        return P ? ptx::mbar_wait_cl(b, parity, sAbort, kTimeoutNs) : ptx::mbar_wait(b, parity, sAbort, kTimeoutNs);
    };
    auto fail = [&](int code) {
        atomicOr(p.err, code);
        *sAbort = 1;
    };

    // Each warp group enters its branch whole and first moves its register share (setmaxnreg
    // is executed by all warps of the group at the same point).
    if (warp < kWarpEpi) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegCtl));
    if (warp == kWarpProd) {
        if (lane == 0) {
            uint32_t stage = 0, phase = 0, n_loads = 0;
            bool ok = true;
            auto next_stage = [&]() -> uint8_t * {
                if (!wait_x(&empty[stage], phase ^ 1)) {
                    fail(1);
                    ok = false;
                    return nullptr;
                }
                TC_TRACE(trace::kProd + n_loads, n_loads < trace::kLoads);
                ++n_loads;
                return sStage + stage * kStageBytes;
            };
            auto advance = [&]() {
                if (++stage == kStages) {
                    stage = 0;
                    phase ^= 1;
                }
            };
            // one tile load: the whole box, or (pairs) a box of half its rows for each CTA, whose bytes
            // the first CTA's barrier counts for both; the second CTA's half starts half the MMA's
            // width `n` further (n < rows only in a narrower last output chunk, whose box is then
            // partly unused; the output weights are padded, so it stays in bounds)
            auto load = [&](uint8_t *dst, const CUtensorMap *m, int x, int y, uint32_t rows, uint32_t n) {
                if (P) {
                    if (rank == 0) ptx::mbar_arrive_expect_tx(&full[stage], rows * 128);
                    ptx::tma_load_2d_cg2(dst, m, lead(&full[stage]), x, y + int(rank * n / 2));
                } else {
                    ptx::mbar_arrive_expect_tx(&full[stage], rows * 128);
                    ptx::tma_load_2d(dst, m, &full[stage], x, y);
                }
            };
            for (uint32_t pt = pt_first; pt < n_pt && ok; pt += pt_step) {
                // layer 0: the 256-row chunks of the [HID][64] BF16 operand, one stage each
                for (int c = 0; c < NCH && ok; ++c) {
                    uint8_t *dst = next_stage();
                    if (!dst) break;
                    load(dst, &tm_l0, 0, c * 256, 256, 256);
                    advance();
                }
                for (int L = 0; L <= nl && ok; ++L) {
                    const int nch = L == nl ? n_oc : NCH;
                    for (int c = 0; c < nch && ok; ++c)
                        for (int kb = 0; kb < KB; ++kb) {
                            uint8_t *dst = next_stage();
                            if (!dst) break;
                            if (L < nl)
                                load(dst, &tm_hid, kb * KBW, L * HID + c * 256, 256, 256);
                            else
                                load(dst, &tm_out, kb * KBW, c * 256, out_box,
                                     p.Cpad - 256u * c < 256u ? p.Cpad - 256u * c : 256u);
                            advance();
                        }
                }
            }
            // let the loads still in flight land before the CTA exits (bounded, abort ignored); in a
            // pair both CTAs' loads complete on the first CTA's barriers, and the second CTA stays
            // until the first has seen them (the cluster barrier at the end)
            volatile int never = 0;
            if (rank == 0)
                for (int s = 0; s < kStages; ++s) {
                    const uint32_t par = s < int(stage) ? phase : phase ^ 1;
                    ptx::mbar_wait(&full[s], par, &never, kTimeoutNs);
                }
        }
    } else if (warp == kWarpMma) {
        // The whole warp runs the issuing loop and lane 0 issues every MMA and commit (in a pair,
        // the first CTA's warp, for both CTAs): run by all lanes, the loop's descriptors and TMEM
        // addresses are warp-uniform. Plain loops over register state: this warp's issue rate
        // bounds the tensor pipe's, so it keeps no state in captured lambdas or local memory.
        if (rank == 0) {
            const uint32_t issuer = lane == 0;  // the lane that issues MMAs and commits
            constexpr uint32_t kMmaM = P ? 256 : 128;
            const uint32_t idesc_h = ptx::idesc_make(kMmaM, 256, F8);
            const uint32_t idesc_0 = ptx::idesc_make(kMmaM, 256, false);  // layer 0: BF16 on both paths
            // the second CTA's copy of a barrier (MMA commits arrive in both CTAs of a pair)
            const uint32_t peer_off = P ? ptx::mapa(ptx::smem_u32(bars), 1) - ptx::smem_u32(bars) : 0u;
            const uint32_t y_addr = ptx::smem_u32(sY), st_addr = ptx::smem_u32(sStage);
            const uint64_t a0_desc = ptx::sdesc_sw128(y_addr);
            const uint64_t bd0 = ptx::sdesc_sw128(st_addr);  // stage s: bd0 + s * kStageBytes / 16
            uint32_t stage = 0, phase = 0, uses = 0, lay = 0, ntile = 0;
            int err = 0;
            for (uint32_t pt = pt_first; pt < n_pt && !err; pt += pt_step, ++ntile) {
                // ---- layer 0: A = the header bytes (shared memory), B = the split weights
                for (int c = 0; c < NCH; ++c, ++uses) {
                    TC_TRACE(trace::kMma + uses * 12 + 0, uses < uint32_t(trace::kChunks));
                    if (uses > 0 && !wait_x(acc_empty, (uses - 1) & 1)) {
                        err = 2;
                        break;
                    }
                    TC_TRACE(trace::kMma + uses * 12 + 1, uses < uint32_t(trace::kChunks));
                    if (c == 0 && !wait_x(feat_full, ntile & 1)) {
                        err = 512;
                        break;
                    }
                    if (!wait_x(&full[stage], phase)) {
                        err = 8;
                        break;
                    }
                    TC_TRACE(trace::kMma + uses * 12 + 2, uses < uint32_t(trace::kChunks));
                    ptx::tc_fence_after();
                    const uint64_t bd = ptx::sdesc_sw128(st_addr + stage * kStageBytes);
#pragma unroll
                    for (int kk = 0; kk < kL0Kused / 16; ++kk) {
                        if (P)
                            ptx::mma2_ss_l(issuer, tmem, a0_desc + 2 * kk, bd + 2 * kk, idesc_0, kk != 0, false);
                        else
                            ptx::mma_ss_l(issuer, tmem, a0_desc + 2 * kk, bd + 2 * kk, idesc_0, kk != 0, false);
                    }
                    if (P) {
                        ptx::mma2_commit_l(issuer, ptx::smem_u32(&empty[stage]));
                        ptx::mma2_commit_l(issuer, ptx::smem_u32(&empty[stage]) + peer_off);
                    } else {
                        ptx::mma_commit_l(issuer, &empty[stage]);
                    }
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1;
                    }
                    if (P) {
                        ptx::mma2_commit_l(issuer, ptx::smem_u32(acc_full));
                        ptx::mma2_commit_l(issuer, ptx::smem_u32(acc_full) + peer_off);
                    } else {
                        ptx::mma_commit_l(issuer, acc_full);
                    }
                    TC_TRACE(trace::kMma + uses * 12 + 10, uses < uint32_t(trace::kChunks));
                }
                for (int L = 0; L <= nl && !err; ++L, ++lay) {
                    const bool a_tmem = (L & 1) == 0;  // FC1 and the output layer read x from TMEM
                    const int nch = L == nl ? n_oc : NCH;
                    for (int c = 0; c < nch && !err; ++c, ++uses) {
                        const uint32_t idesc =
                            L == nl ? ptx::idesc_make(kMmaM, p.Cpad - 256u * c < 256u ? p.Cpad - 256u * c : 256u, F8) : idesc_h;
                        TC_TRACE(trace::kMma + uses * 12 + 0, uses < uint32_t(trace::kChunks));
                        if (!wait_x(acc_empty, (uses - 1) & 1)) {
                            err = 2;
                            break;
                        }
                        TC_TRACE(trace::kMma + uses * 12 + 1, uses < uint32_t(trace::kChunks));
                        ptx::tc_fence_after();
                        // The K-block loops, unrolled by four, each body one MMA form. BF16 has one
                        // loop per A source (x in TMEM, u in shared memory); FP8 reads both from TMEM,
                        // so one loop takes the source's base column. Measured against one rolled loop
                        // that chose the form per K-block: +3.5 % (unrolled) then +4-7 % (split) for
                        // BF16, +1 % for FP8 (+4 % more without the choice, network alone); two split
                        // FP8 loops lost 2.5 %, and unrolling all eight BF16 K-blocks lost 8 %.
                        if constexpr (!F8) {
                            if (a_tmem) {
#pragma unroll 4
                                for (int kb = 0; kb < KB; ++kb) {
                                    if (c == 0 && !wait_x(&act[kb], lay & 1)) {
                                        err = 4;
                                        break;
                                    }
                                    if (!wait_x(&full[stage], phase)) {
                                        err = 8;
                                        break;
                                    }
                                    TC_TRACE(trace::kMma + uses * 12 + 2 + kb, uses < uint32_t(trace::kChunks));
                                    ptx::tc_fence_after();
                                    const uint64_t bd = bd0 + uint64_t(stage * (kStageBytes >> 4));
                                    const uint32_t ta = tmem + kXCol + kb * 32;
#pragma unroll
                                    for (int kk = 0; kk < 4; ++kk) {
                                        if (P)
                                            ptx::mma2_ts_l(issuer, tmem, ta + kk * 8, bd + 2 * kk, idesc, (kb | kk) != 0, F8);
                                        else
                                            ptx::mma_ts_l(issuer, tmem, ta + kk * 8, bd + 2 * kk, idesc, (kb | kk) != 0, F8);
                                    }
                                    if (P) {
                                        ptx::mma2_commit_l(issuer, ptx::smem_u32(&empty[stage]));
                                        ptx::mma2_commit_l(issuer, ptx::smem_u32(&empty[stage]) + peer_off);
                                    } else {
                                        ptx::mma_commit_l(issuer, &empty[stage]);
                                    }
                                    if (++stage == kStages) {
                                        stage = 0;
                                        phase ^= 1;
                                    }
                                }
                            } else {
#pragma unroll 4
                                for (int kb = 0; kb < KB; ++kb) {
                                    if (c == 0 && !wait_x(&act[kb], lay & 1)) {
                                        err = 4;
                                        break;
                                    }
                                    if (!wait_x(&full[stage], phase)) {
                                        err = 8;
                                        break;
                                    }
                                    TC_TRACE(trace::kMma + uses * 12 + 2 + kb, uses < uint32_t(trace::kChunks));
                                    ptx::tc_fence_after();
                                    const uint64_t bd = bd0 + uint64_t(stage * (kStageBytes >> 4));
                                    const uint64_t ad = a0_desc + uint64_t(kb) * (16384 >> 4);
#pragma unroll
                                    for (int kk = 0; kk < 4; ++kk) {
                                        if (P)
                                            ptx::mma2_ss_l(issuer, tmem, ad + 2 * kk, bd + 2 * kk, idesc, (kb | kk) != 0, F8);
                                        else
                                            ptx::mma_ss_l(issuer, tmem, ad + 2 * kk, bd + 2 * kk, idesc, (kb | kk) != 0, F8);
                                    }
                                    if (P) {
                                        ptx::mma2_commit_l(issuer, ptx::smem_u32(&empty[stage]));
                                        ptx::mma2_commit_l(issuer, ptx::smem_u32(&empty[stage]) + peer_off);
                                    } else {
                                        ptx::mma_commit_l(issuer, &empty[stage]);
                                    }
                                    if (++stage == kStages) {
                                        stage = 0;
                                        phase ^= 1;
                                    }
                                }
                            }
                        } else {
                            const uint32_t a_base = tmem + (a_tmem ? kXCol : kUCol);  // x (FC1, output) or u (FC2)
#pragma unroll 4
                            for (int kb = 0; kb < KB; ++kb) {
                                if (c == 0 && !wait_x(&act[kb], lay & 1)) {
                                    err = 4;
                                    break;
                                }
                                if (!wait_x(&full[stage], phase)) {
                                    err = 8;
                                    break;
                                }
                                TC_TRACE(trace::kMma + uses * 12 + 2 + kb, uses < uint32_t(trace::kChunks));
                                ptx::tc_fence_after();
                                const uint64_t bd = bd0 + uint64_t(stage * (kStageBytes >> 4));
                                const uint32_t ta = a_base + kb * 32;
#pragma unroll
                                for (int kk = 0; kk < 4; ++kk) {
                                    if (P)
                                        ptx::mma2_ts_l(issuer, tmem, ta + kk * 8, bd + 2 * kk, idesc, (kb | kk) != 0, F8);
                                    else
                                        ptx::mma_ts_l(issuer, tmem, ta + kk * 8, bd + 2 * kk, idesc, (kb | kk) != 0, F8);
                                }
                                if (P) {
                                    ptx::mma2_commit_l(issuer, ptx::smem_u32(&empty[stage]));
                                    ptx::mma2_commit_l(issuer, ptx::smem_u32(&empty[stage]) + peer_off);
                                } else {
                                    ptx::mma_commit_l(issuer, &empty[stage]);
                                }
                                if (++stage == kStages) {
                                    stage = 0;
                                    phase ^= 1;
                                }
                            }
                        }
                        if (err) break;
                        if (P) {
                            ptx::mma2_commit_l(issuer, ptx::smem_u32(acc_full));
                            ptx::mma2_commit_l(issuer, ptx::smem_u32(acc_full) + peer_off);
                        } else {
                            ptx::mma_commit_l(issuer, acc_full);
                        }
                        TC_TRACE(trace::kMma + uses * 12 + 10, uses < uint32_t(trace::kChunks));
                    }
                }
            }
            if (err) fail(err);
            volatile int never = 0;
            if (P)
                ptx::mma2_commit_l(issuer, ptx::smem_u32(drain));
            else
                ptx::mma_commit_l(issuer, drain);
            ptx::mbar_wait(drain, 0, &never, kTimeoutNs);
        }
    }  // warps 2 and 3 of the control group have no role
    } else if (warp < kWarpSearch) {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegEpi));
        // ---------------- 16 epilogue warps ----------------
        const int ew = warp - kWarpEpi;
        const int q = warp & 3;   // TMEM lane quadrant
        const int g = ew >> 2;    // column group: layer 0 unit g of each chunk, hidden layers 32 g.. of each half
        const int r = q * 32 + lane;
        const uint32_t lane_base = uint32_t(q * 32) << 16;
        const float *sa = p.sa;
        uint32_t uses = 0, tcnt = 0;
        bool ok = true;
        // BF16 u: 16 values of row r into the swizzled K-major shared-memory tile FC2 reads
        auto store_smem = [&](const uint32_t *w, int col0) {
            const int kb = col0 >> 6, j0 = (col0 & 63) >> 3;
            uint8_t *row = sY + kb * 16384 + r * 128;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                *reinterpret_cast<uint4 *>(row + (((j0 + k) ^ (r & 7)) << 4)) =
                    make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
        };
        auto x_col = [&](int col0) -> uint32_t { return tmem + lane_base + kXCol + (F8 ? col0 / 4 : col0 / 2); };
        [[maybe_unused]] auto u_col = [&](int col0) -> uint32_t { return tmem + lane_base + kUCol + col0 / 4; };
        auto act_arrive = [&](int col0) {
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) arrive_mma_side(&act[col0 / KBW]);
        };
        // ReLU, round and store 32 activations (columns col0 ..) of the next layer's input; for FP8
        // the values are already in the next layer's scaled units
        auto emit = [&](const float *v, int col0, bool to_x) {
            if (!F8) {
                uint32_t w[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) w[j] = relu_bf16x2(v[2 * j], v[2 * j + 1]);
                if (to_x)
                    ptx::tmem_st16(x_col(col0), w);
                else
                    store_smem(w, col0);
            } else {
                uint32_t w[8];
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    w[j] = relu_e4m3x2(v[4 * j], v[4 * j + 1]) | (relu_e4m3x2(v[4 * j + 2], v[4 * j + 3]) << 16);
                ptx::tmem_st8(to_x ? x_col(col0) : u_col(col0), w);
            }
        };
        // Layer-0 operand of tile t, row r (the g == 0 warps): the header bytes as BF16 in the
        // swizzled K-major layout the MMA reads, [hi(7), lo(7)] three times, then 1, 1, 1, zeros.
        auto write_features = [&](uint32_t t) {
            const uint32_t it = t * kM + r;
            const uint4 hv = it < p.n ? __ldcs(reinterpret_cast<const uint4 *>(p.headers + it)) : make_uint4(0, 0, 0, 0);
            const uint32_t f[7] = {hv.x >> 16, hv.x & 0xFFFFu, hv.y >> 16, hv.y & 0xFFFFu, hv.z & 0xFFFFu, hv.z >> 16,
                                   hv.w & 0xFFu};
            float e[14];
#pragma unroll
            for (int k = 0; k < 7; ++k) {
                e[k] = float(f[k] >> 8);
                e[7 + k] = float(f[k] & 0xFFu);
            }
            uint32_t part[7];  // the 14 byte values as 7 BF16 pairs
#pragma unroll
            for (int k = 0; k < 7; ++k) part[k] = pack_bf16(e[2 * k], e[2 * k + 1]);
            uint32_t w[32];
#pragma unroll
            for (int rep = 0; rep < 3; ++rep)
#pragma unroll
                for (int k = 0; k < 7; ++k) w[7 * rep + k] = part[k];
            w[21] = pack_bf16(1.f, 1.f);
            w[22] = pack_bf16(1.f, 0.f);
#pragma unroll
            for (int k = 23; k < 32; ++k) w[k] = 0u;
            uint8_t *row = sY + r * 128;
#pragma unroll
            for (int j = 0; j < 8; ++j)
                *reinterpret_cast<uint4 *>(row + ((j ^ (r & 7)) << 4)) = make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
            ptx::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) arrive_mma_side(feat_full);
        };

        // Per-column constants of the hidden layers, one per lane: the bias (FP8: b * s_out) of
        // columns 256 c + 32 g + lane and 256 c + 128 + 32 g + lane; for FP8 also the layer's scale
        // dq * s_out, the same for every column (the hidden layers have one weight scale each).
        // Shuffles broadcast them across the warp's rows. They are loaded one chunk ahead: loads
        // issued at the chunk's start stalled the FP8 epilogue, which runs behind the MMAs and so
        // finds its accumulator ready, for an L2 round trip; broadcast loads of whole lines missed
        // the small L1 left beside 231 KB of shared memory in both precisions (about 1k cycles per
        // chunk); broadcast reads from a shared-memory copy were no faster than the shuffles.
        struct ColConst {
            float b0, b1, d;
        };
        auto load_cc = [&](int L, int c) -> ColConst {
            const int col = 256 * c + 32 * g + lane;
            const float *bv = F8 ? p.fold8 + size_t(nl + L) * HID : p.bias + size_t(L) * HID;
            return ColConst{__ldg(bv + col), __ldg(bv + col + 128), F8 ? __ldg(p.fold8 + size_t(L) * HID) : 0.f};
        };
        ColConst next_cc = load_cc(0, 0);
        if (g == 0 && pt_first < n_pt) write_features(tile_of(pt_first));
        for (uint32_t pt = pt_first; pt < n_pt && ok; pt += pt_step) {
            const uint32_t i = tile_of(pt) * kM + r;
            // ---- layer 0 from the accumulator (bias included): units 4c+g of x
            for (int c = 0; c < NCH; ++c, ++uses) {
                if (!wait_x(acc_full, uses & 1)) {
                    fail(16);
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const int unit = 4 * c + g;
                uint32_t a0[32], a1[32];
                ptx::tmem_ld32(tmem + lane_base + g * 64, a0);
                ptx::tmem_ld32(tmem + lane_base + g * 64 + 32, a1);
                ptx::tmem_wait_ld();
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) release_acc();
                emit(reinterpret_cast<const float *>(a0), unit * 64, true);
                emit(reinterpret_cast<const float *>(a1), unit * 64 + 32, true);
                ptx::tmem_wait_st();
                act_arrive(unit * 64);
                act_arrive(unit * 64 + 32);
            }
            if (!ok) break;
            // ---- hidden layers, NCH 256-column chunks each
            for (int L = 0; L < nl && ok; ++L) {
                const bool fc2 = (L & 1) != 0;
                // BF16: v = acc + b. FP8: v = acc * (dq * s_out) + b * s_out, in the output's units.
                // FP8 residual: x is stored in the units of its own layer input (scale s[L-1])
                const float rr = F8 && fc2 ? sa[L + 1] / sa[L - 1] : 1.f;
                // rr as FP16 bits when exact there (a power of two in [2^-24, 2^15]), else 0
                uint32_t rr16 = 0;
                if (F8 && fc2) {
                    const __half h = __float2half_rn(rr);
                    if (__half2float(h) == rr) rr16 = __half_as_ushort(h);
                }
                for (int c = 0; c < NCH; ++c, ++uses) {
                    [[maybe_unused]] const bool tr = lane == 0 && q == 2 && g < 2 && uses < uint32_t(trace::kChunks);
                    [[maybe_unused]] const int tslot = trace::kEpi + (g * trace::kChunks + int(uses)) * 4;
                    TC_TRACE(tslot + 0, tr);
                    // Warp g takes columns 32 g .. 32 g + 31 of each 128-column half of the chunk,
                    // the first half before the second: the first half's K-blocks of the next
                    // layer's input are published about halfway through the chunk's epilogue, so
                    // that the next layer's first MMAs wait less at a layer boundary.
                    // this chunk's column constants, loaded one chunk ago; now the next chunk's
                    const ColConst cc = next_cc;
                    next_cc = c + 1 < NCH ? load_cc(L, c + 1) : load_cc(L + 1 < nl ? L + 1 : 0, 0);
                    if (!wait_x(acc_full, uses & 1)) {
                        fail(16);
                        ok = false;
                        break;
                    }
                    TC_TRACE(tslot + 1, tr);
                    ptx::tc_fence_after();
                    uint32_t a0[32], a1[32];
                    ptx::tmem_ld32(tmem + lane_base + g * 32, a0);
                    ptx::tmem_ld32(tmem + lane_base + 128 + g * 32, a1);
                    ptx::tmem_wait_ld();
                    // the accumulator may take the next chunk's MMAs now
                    ptx::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) release_acc();
                    TC_TRACE(tslot + 2, tr);
#pragma unroll
                    for (int s = 0; s < 2; ++s) {
                        const int col0 = 256 * c + 128 * s + 32 * g;
                        const uint32_t *a = s == 0 ? a0 : a1;
                        const float bl = s == 0 ? cc.b0 : cc.b1;
                        // two columns per packed f32x2 instruction: v = acc + b (BF16), acc * d + b (FP8)
                        float v[32];
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const float2 b = make_float2(__shfl_sync(0xFFFFFFFFu, bl, 2 * j),
                                                         __shfl_sync(0xFFFFFFFFu, bl, 2 * j + 1));
                            const float2 y = make_float2(__uint_as_float(a[2 * j]), __uint_as_float(a[2 * j + 1]));
                            const float2 r = F8 ? fma_f2(y, make_float2(cc.d, cc.d), b) : add_f2(y, b);
                            v[2 * j] = r.x;
                            v[2 * j + 1] = r.y;
                        }
                        TC_TRACE(trace::kEpiX + (g * trace::kChunks + int(uses)) * 6 + 3 * s + 0, tr);
                        if (fc2) {
                            // the residual x, one mixed-precision addition (BF16) or FMA (FP8, the
                            // E4M3 codes widened to FP16 and rr given as FP16) per element
                            if (!F8) {
                                uint32_t xr[16];
                                ptx::tmem_ld16(x_col(col0), xr);
                                ptx::tmem_wait_ld();
#pragma unroll
                                for (int j = 0; j < 16; ++j) {
                                    v[2 * j] = add_bf16lo(xr[j], v[2 * j]);
                                    v[2 * j + 1] = add_bf16hi(xr[j], v[2 * j + 1]);
                                }
                            } else if (rr16) {
                                uint32_t xr[8];
                                ptx::tmem_ld8(x_col(col0), xr);
                                ptx::tmem_wait_ld();
#pragma unroll
                                for (int j = 0; j < 8; ++j) {
                                    const uint32_t h01 = e4m3x2_to_h2(xr[j]), h23 = e4m3x2_to_h2(xr[j] >> 16);
                                    v[4 * j + 0] = fma_f16lo(h01, rr16, v[4 * j + 0]);
                                    v[4 * j + 1] = fma_f16hi(h01, rr16, v[4 * j + 1]);
                                    v[4 * j + 2] = fma_f16lo(h23, rr16, v[4 * j + 2]);
                                    v[4 * j + 3] = fma_f16hi(h23, rr16, v[4 * j + 3]);
                                }
                            } else {  // rr outside FP16's powers of two: widen to FP32
                                uint32_t xr[8];
                                ptx::tmem_ld8(x_col(col0), xr);
                                ptx::tmem_wait_ld();
#pragma unroll
                                for (int j = 0; j < 8; ++j) {
                                    const float2 lo = e4m3x2_to_f2(xr[j]), hi = e4m3x2_to_f2(xr[j] >> 16);
                                    const float2 r0 = fma_f2(lo, make_float2(rr, rr), make_float2(v[4 * j], v[4 * j + 1]));
                                    const float2 r1 = fma_f2(hi, make_float2(rr, rr), make_float2(v[4 * j + 2], v[4 * j + 3]));
                                    v[4 * j + 0] = r0.x;
                                    v[4 * j + 1] = r0.y;
                                    v[4 * j + 2] = r1.x;
                                    v[4 * j + 3] = r1.y;
                                }
                            }
                        }
                        TC_TRACE(trace::kEpiX + (g * trace::kChunks + int(uses)) * 6 + 3 * s + 1, tr);
                        emit(v, col0, fc2);
                        if (fc2 || F8)
                            ptx::tmem_wait_st();
                        else
                            ptx::fence_proxy_async_smem();
                        act_arrive(col0);
                        TC_TRACE(trace::kEpiX + (g * trace::kChunks + int(uses)) * 6 + 3 * s + 2, tr);
                    }
                    TC_TRACE(tslot + 3, tr);
                    // after the last FC2 chunk (its MMAs, the last readers of u, have completed):
                    // the next tile's layer-0 operand
                    if (L == nl - 1 && c == NCH - 1 && g == 0 && pt + pt_step < n_pt) write_features(tile_of(pt + pt_step));
                }
            }
            if (!ok) break;
            // ---- output layer, in 256-column chunks: each column group takes a quarter of every
            // chunk; the kArgG warps combine the four partial maxima per row and hand the
            // prediction on
            {
                float best = -INFINITY;
                int arg = 0;
                const float *bias = p.bias + nl * HID;
                const float *dq = F8 ? p.dq + nl * HID : nullptr;
                for (int oc = 0; oc < n_oc; ++oc) {
                    if (!wait_x(acc_full, uses & 1)) {
                        fail(32);
                        ok = false;
                        break;
                    }
                    ++uses;
                    ptx::tc_fence_after();
                    const uint32_t c_base = 256u * uint32_t(oc);
                    const uint32_t cq = (p.Cpad - c_base < 256u ? p.Cpad - c_base : 256u) / 4;  // a multiple of 8
                    for (uint32_t c0 = uint32_t(g) * cq; c0 < uint32_t(g + 1) * cq; c0 += 8) {
                        uint32_t a[8];
                        ptx::tmem_ld8(tmem + lane_base + c0, a);
                        ptx::tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const uint32_t cc = c_base + c0 + j;
                            if (cc >= p.C) break;
                            float z = __uint_as_float(a[j]);
                            z = F8 ? fmaf(z, __ldg(dq + cc), __ldg(bias + cc)) : z + __ldg(bias + cc);
                            if (p.logits && i < p.n) p.logits[size_t(i) * p.C + cc] = z;
                            if (z > best) {  // this group's columns in increasing order: the first maximum
                                best = z;
                                arg = int(cc);
                            }
                        }
                    }
                    ptx::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) release_acc();
                }
                if (!ok) break;
                const uint32_t t = tcnt & 1, tu = tcnt >> 1;  // this CTA's tile count: barrier parities
                ++tcnt;
                if (g != kArgG) {
                    sPartBest[g * kM + r] = best;
                    sPartArg[g * kM + r] = arg;
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(part_full);
                } else {
                    if (!ptx::mbar_wait(part_full, t, sAbort, kTimeoutNs)) {
                        fail(256);
                        ok = false;
                        break;
                    }
                    // the lowest column among equal maxima, as a serial scan (with several chunks
                    // a group's columns interleave with the others', so ties compare indices)
                    float b = sPartBest[r];
                    int am = sPartArg[r];
#pragma unroll
                    for (int gg = 1; gg < 4; ++gg) {
                        const float bg = gg == kArgG ? best : sPartBest[gg * kM + r];
                        const int ag = gg == kArgG ? arg : sPartArg[gg * kM + r];
                        if (bg > b || (bg == b && ag < am)) {
                            b = bg;
                            am = ag;
                        }
                    }
                    if (p.tuple && i < p.n) p.tuple[i] = am;
                    if (p.fused_search) {
                        if (!ptx::mbar_wait(&tempty[t], (tu & 1) ^ 1, sAbort, kTimeoutNs)) {
                            fail(64);
                            ok = false;
                            break;
                        }
                        sTidx[t * kM + r] = am;
                        __syncwarp();
                        if (lane == 0) ptx::mbar_arrive(&tfull[t]);
                    }
                }
            }
        }
    } else {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegSearch));
        // ---------------- search warps ----------------
        if (p.fused_search) {
            const Tables tb = *p.tables;
            const int r = (warp - kWarpSearch) * 32 + lane;
            uint32_t tcnt = 0;
            uint32_t st_pk = 0, st_match = 0, st_correct = 0, st_hit = 0, st_fb = 0;
            Counters cn{0, 0, 0};
            for (uint32_t pt = pt_first; pt < n_pt; pt += pt_step) {
                const uint32_t t = tcnt & 1, tu = tcnt >> 1;
                ++tcnt;
                if (!ptx::mbar_wait(&tfull[t], tu & 1, sAbort, kTimeoutNs)) {
                    fail(128);
                    break;
                }
                [[maybe_unused]] const bool trs = r == 0 && tcnt <= uint32_t(trace::kSearchTiles);
                TC_TRACE(trace::kSearch + 2 * (tcnt - 1), trs);
                // each search thread owns row r of the tile
                const int pred = sTidx[t * kM + r];
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&tempty[t]);
                const uint32_t i = tile_of(pt) * kM + r;
                if (i < p.n) {
                    // headers and ids stream through L2 with evict-first hints, the tables stay
                    const Hdr h = load_header_stream(p.headers + i);
                    Best best;
                    const bool hit = search_packet(tb, tb.tuples, tb.order, h, pred, best, cn, p.fused_search >> 1);
                    __stcs(p.ids + i, best.id);
                    if (p.stats) {
                        st_pk++;
                        const bool m = best.id != 0xFFFFFFFFu;
                        st_match += m;
                        st_correct += m && int(best.tuple) == pred;
                        st_hit += hit;
                        st_fb += !hit;
                    }
                }
                TC_TRACE(trace::kSearch + 2 * (tcnt - 1) + 1, trs);
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
    if (P)
        ptx::cluster_sync();  // the first CTA's MMAs into this CTA's TMEM and its loads have completed
    else
        __syncthreads();
    ptx::tc_fence_after();
    if (warp == kWarpMma) {
        __syncwarp();  // the issue loop's bounded waits may have left the lanes apart: converge before the warp-wide dealloc
        if (P)
            ptx::tmem_dealloc_cg2(tmem, 512);
        else
            ptx::tmem_dealloc(tmem, 512);
    }
}

namespace {
struct Tc256Maps {
    CUtensorMap hid, out, l0;
};

// Round to the nearest BF16 value, as a float.
float bf16_round_host(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// The layer-0 operand B[n][k] (n < N, k < 64) with sum_k A[k] B[n][k] = s * (b0[n] + sum_t
// f_t W0[t][n]) for A = [hi(7), lo(7)] x 3, 1 x 3, 0 x 19 (f_t = 256 hi_t + lo_t): the weight
// parts scaled by 256 meet the high bytes, the plain parts the low bytes.
void layer0_operand(const float *W0, const float *b0, uint32_t N, float s, __nv_bfloat16 *B) {
    auto split = [](float w, float part[3]) {
        part[0] = bf16_round_host(w);
        const float r1 = w - part[0];  // exact in FP32
        part[1] = bf16_round_host(r1);
        part[2] = bf16_round_host(r1 - part[1]);
    };
    for (uint32_t n = 0; n < N; ++n) {
        __nv_bfloat16 *row = B + size_t(n) * tc256::kL0K;
        for (int k = 0; k < tc256::kL0K; ++k) row[k] = __float2bfloat16_rn(0.f);
        for (int t = 0; t < 7; ++t) {
            float part[3];
            split(W0[size_t(t) * N + n] * s, part);
            for (int pi = 0; pi < 3; ++pi) {
                row[pi * 14 + t] = __float2bfloat16_rn(part[pi] * 256.f);
                row[pi * 14 + 7 + t] = __float2bfloat16_rn(part[pi]);
            }
        }
        float part[3];
        split(b0[n] * s, part);
        for (int pi = 0; pi < 3; ++pi) row[42 + pi] = __float2bfloat16_rn(part[pi]);
    }
}
}  // namespace

// 256-row hidden-layer maps, output-layer maps of up to 256-row tiles, and the layer-0 operands
// with their maps, for width N = 256 or 512.
int tc256_prepare_model(tang_ctx *ctx, DeviceModel &m) {
    if (!m.d_wbf16 || (m.N != 256 && m.N != 512)) return TANG_OK;
    // [BF16, FP8] with whole 256-row boxes, then [BF16, FP8] with half boxes for the CTA pairs
    Tc256Maps *maps = static_cast<Tc256Maps *>(aligned_alloc(64, 4 * sizeof(Tc256Maps)));
    std::memset(static_cast<void *>(maps), 0, 4 * sizeof(Tc256Maps));
    m.tmap256 = maps;
    const uint32_t N = m.N;
    const float *W0 = m.host_params.data(), *b0 = W0 + size_t(7) * N;
    std::vector<__nv_bfloat16> l0(size_t(2) * N * tc256::kL0K);
    layer0_operand(W0, b0, N, 1.f, l0.data());
    if (m.has_fp8) layer0_operand(W0, b0, N, m.act_scale[0], l0.data() + size_t(N) * tc256::kL0K);
    int rc = ctx_alloc(ctx, l0.size() * 2, &m.d_l0);
    if (rc) return rc;
    cudaMemcpy(m.d_l0, l0.data(), l0.size() * 2, cudaMemcpyHostToDevice);
    // output tiles of min(Cpad, 256) rows; past 256 the copies hold whole 256-row tiles
    const size_t hid = size_t(m.layers) * m.N * m.N;
    const uint32_t out_rows = m.Cpad <= 256 ? m.Cpad : (m.Cpad + 255) / 256 * 256, out_box = std::min<uint32_t>(m.Cpad, 256);
    for (uint32_t half = 1; half <= 2; ++half) {  // box rows / half: 1 = whole tiles, 2 = pair halves
        Tc256Maps *mp = maps + (half - 1) * 2;
        if ((rc = make_tmap(ctx, &mp[0].out, static_cast<__nv_bfloat16 *>(m.d_wbf16) + hid, out_rows, false,
                            out_box / half, N)))
            return rc;
        if ((rc = make_tmap(ctx, &mp[0].hid, m.d_wbf16, m.layers * N, false, 256 / half, N))) return rc;
        if ((rc = make_tmap(ctx, &mp[0].l0, m.d_l0, N, false, 256 / half, tc256::kL0K))) return rc;
        if (m.d_wfp8) {
            if ((rc = make_tmap(ctx, &mp[1].out, static_cast<uint8_t *>(m.d_wfp8) + hid, out_rows, true, out_box / half,
                                N)))
                return rc;
            if ((rc = make_tmap(ctx, &mp[1].hid, m.d_wfp8, m.layers * N, true, 256 / half, N))) return rc;
            if ((rc = make_tmap(ctx, &mp[1].l0, static_cast<__nv_bfloat16 *>(m.d_l0) + size_t(N) * tc256::kL0K, N, false,
                                256 / half, tc256::kL0K)))
                return rc;
        }
    }
    return rc;
}

// Pair launches (P) run in clusters of two CTAs: grid = 2 x the pairs that fit at once (one CTA
// per SM), capped by the tuned grid and by the pair-tiles.
template <bool F8, int HID, bool P>
static int tc256_launch_t(tang_ctx *ctx, const Tc256Maps &maps, const TcParams &prm, cudaStream_t st, uint32_t grid) {
    constexpr int kSmem = tc256::Layout<F8, HID, P>::kSmemBytes;
    static bool attr_done = false;
    static uint32_t max_pairs = 0;
    if (!attr_done) {
        // the setmaxnreg split assumes the launch register count it was sized for: with any other
        // count an increase could wait forever, so refuse to launch
        cudaFuncAttributes fa{};
        cudaError_t e = cudaFuncGetAttributes(&fa, k_tc256_classify<F8, HID, P>);
        if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "N=256 kernel attributes: %s", cudaGetErrorString(e));
        if (fa.numRegs != tc256::kRegLaunch)
            return set_err(ctx, TANG_EDEVICE, "N=256 kernel built with %d registers per thread, expected %d", fa.numRegs,
                           tc256::kRegLaunch);
        e = cudaFuncSetAttribute(k_tc256_classify<F8, HID, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "smem attribute (N=256): %s", cudaGetErrorString(e));
        if (P) {
            max_pairs = uint32_t(ctx->sm_count / 2);
            cudaLaunchConfig_t q = {};
            q.gridDim = dim3(2 * max_pairs, 1, 1);
            q.blockDim = dim3(tc256::kThreads, 1, 1);
            q.dynamicSmemBytes = kSmem;
            cudaLaunchAttribute qa[1];
            qa[0].id = cudaLaunchAttributeClusterDimension;
            qa[0].val.clusterDim.x = 2;
            qa[0].val.clusterDim.y = 1;
            qa[0].val.clusterDim.z = 1;
            q.attrs = qa;
            q.numAttrs = 1;
            int c = 0;
            if (cudaOccupancyMaxActiveClusters(&c, k_tc256_classify<F8, HID, P>, &q) == cudaSuccess && c > 0)
                max_pairs = std::min<uint32_t>(max_pairs, uint32_t(c));
            cudaGetLastError();
            if (max_pairs == 0) return set_err(ctx, TANG_EUNSUPPORTED, "no CTA pair fits on this device");
        }
        attr_done = true;
    }
    if (!P) {
        k_tc256_classify<F8, HID, P><<<grid, tc256::kThreads, kSmem, st>>>(maps.hid, maps.out, maps.l0, prm);
    } else {
        const uint32_t pairs = std::max<uint32_t>(1, std::min<uint32_t>({max_pairs, (prm.n_tiles + 1) / 2, (grid + 1) / 2}));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * pairs, 1, 1);
        cfg.blockDim = dim3(tc256::kThreads, 1, 1);
        cfg.dynamicSmemBytes = kSmem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, k_tc256_classify<F8, HID, P>, maps.hid, maps.out, maps.l0, prm);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(ctx, TANG_EDEVICE, "N=256 kernel launch: %s", cudaGetErrorString(e));
    return TANG_OK;
}

int tc256_launch(tang_ctx *ctx, DeviceModel &m, const TcParams &prm, bool f8, cudaStream_t st, int grid_cap, bool pair) {
    if (!m.tmap256 || !m.d_l0 || (f8 && (!m.d_wfp8 || !m.d_fold8))) return TANG_EUNSUPPORTED;
    const Tc256Maps &maps = static_cast<const Tc256Maps *>(m.tmap256)[(pair ? 2 : 0) + (f8 ? 1 : 0)];
    uint32_t grid = uint32_t(grid_cap > 0 ? grid_cap : ctx->sm_count);
    grid = std::min<uint32_t>(prm.n_tiles, std::min<uint32_t>(grid, uint32_t(ctx->sm_count)));
    TcParams prm_t = prm;
#ifdef TANG_TC_TRACE
    static unsigned long long *d_trace = nullptr;
    if (!d_trace) cudaMalloc(&d_trace, sizeof(unsigned long long) * trace::kTotal);
    cudaMemsetAsync(d_trace, 0, sizeof(unsigned long long) * trace::kTotal, st);
    prm_t.trace = d_trace;
#endif
    int rc;
    if (pair)
        rc = m.N == 512 ? (f8 ? tc256_launch_t<true, 512, true>(ctx, maps, prm_t, st, grid)
                              : tc256_launch_t<false, 512, true>(ctx, maps, prm_t, st, grid))
                        : (f8 ? tc256_launch_t<true, 256, true>(ctx, maps, prm_t, st, grid)
                              : tc256_launch_t<false, 256, true>(ctx, maps, prm_t, st, grid));
    else
        rc = m.N == 512 ? (f8 ? tc256_launch_t<true, 512, false>(ctx, maps, prm_t, st, grid)
                              : tc256_launch_t<false, 512, false>(ctx, maps, prm_t, st, grid))
                        : (f8 ? tc256_launch_t<true, 256, false>(ctx, maps, prm_t, st, grid)
                              : tc256_launch_t<false, 256, false>(ctx, maps, prm_t, st, grid));
    if (rc) return rc;
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
