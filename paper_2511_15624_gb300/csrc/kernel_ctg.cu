// The contingency-flow interval kernel: for every contingency k and line l,
//   c_kl = c_l + L[l,k] c_k,       r_kl = sum_b |Phi[l,b] + L[l,k] Phi[k,b]| r_b
// (Sec. II-C eq. (ctg flow simplified) with H_k = Phi + L[:,k] Phi[k,:], under
// the centre/radius rule of eq. (IBP)), fused with the violation interval of
// eq. (slack-Sc) and the per-warp partial sums of eq. (slack-sagg).
//
// |H_k| is never stored: each CTA owns a tile of BL lines x BK contingencies
// and streams bus chunks of the two PTDF row blocks through shared memory with
// TMA (SWIZZLE_128B, a ring of ST stages guarded by mbarriers), while its warps
// hold the tile's LODF entries and radius accumulators in registers.
// Persistent launch: as many CTAs as fit on the SMs walk the tile list with a
// static stride (deterministic output).
//
// One-box variant: the rows are pre-scaled by the bus radius,
//   hat[x,b] = RN(Phi~[x,b] r_b),   h' = RN(hat[l,b] + L~ hat[k,b]),
// so each (pair, bus) term costs one FMA and one round-up add of |h'|:
//   acc <- RU(acc + |h'|).
// Error analysis (u = 2^-24, Phi~ = RN32(Phi), L~ = RN32(L), R~_x = the base
// radius sum of row x rounded up):
//   |H_b r_b - h'_b| <= u |h'_b| + 2.0001u |Phi_lb| r_b + 3.0001u |L| |Phi_kb| r_b
// so  r_kl <= (1 + u) sum|h'| + 4u (R~_l + |L~| R~_k)  (+ eta for underflow),
// and sum|h'| <= A (the round-up sum), giving the certified radius
//   rbar = RU((1 + u) A + 4u (R~_l + |L~| R~_k) + eta).
// The round-up sum is hierarchical (one chunk of CH buses, 256 / CH chunks per
// level-2 sum, the rest in level 3, which S3 keeps in shared memory) to keep
// its excess small; gamma bounds it.  The default one-box shape runs two CTAs
// of 8 warps per SM at 128 registers per thread; a thread owns 4 x 4 pairs and
// sums each pair in two packed lanes (BODY 2).
//
// Multi-box variant: h = RN(Phi~[l,b] + L~ Phi~[k,b]) once per (pair, bus),
// then acc_j <- RU(acc_j + |h| r_jb) for the thread's boxes; the same bound
// holds with R~ the per-box base radius sums.
#include "common.cuh"
#include "ctg_epilogue.cuh"
#include "internal.h"

#include <algorithm>
#include <cstdio>

namespace ibp {

// Tile order: bands of kBand line tiles; inside a band the contingency tiles
// run slowest, so the tiles in flight at one time (one per SM) touch about
// kBand line-row blocks and 152/kBand contingency-row blocks, which stay in L2.
constexpr int kBand = 8;

__device__ __forceinline__ void tile_origin(int tile, int tiles_l, int tiles_k, int BL, int BK,
                                            int &l0, int &k0) {
    const int per_band = kBand * tiles_k;
    const int band = tile / per_band, r = tile % per_band;
    const int g = min(kBand, tiles_l - band * kBand);
    l0 = (band * kBand + r % g) * BL;
    k0 = (r / g) * BK;
}

template <int WL, int WK, int ML, int MK, int ST, bool S3 = false, int CH_ = 32>
struct Shape {
    static constexpr int kWarps = WL * WK;
    static constexpr int kThreads = kWarps * 32;
    static constexpr int TL = WL * 4, TK = WK * 8;  // threads along lines / contingencies
    static constexpr int BL = TL * ML, BK = TK * MK;
    static constexpr int CH = CH_;                  // buses per chunk
    static constexpr int NSUB = CH / 32;            // 128-byte swizzled sub-blocks per row
    static constexpr int kStageFloats = (BL + BK) * CH;
    static constexpr size_t kRing = (size_t)ST * kStageFloats * sizeof(float);
    // level-3 radius sums in shared memory when S3: [slot][thread]
    static constexpr size_t kAcc3 = S3 ? (size_t)ML * MK * kThreads * sizeof(float) : 0;
    // full[ST] mbarriers, arrival counters[ST], last issued chunk[ST], abort flag
    static constexpr size_t kCtl = ST * sizeof(uint64_t) + 2 * ST * sizeof(int) + 16;
    // per-warp queues of the pairs for the FP64 refinement (16-byte aligned)
    static constexpr size_t kQueueOff = kRing + kAcc3 + (kCtl + 15) / 16 * 16;
    static constexpr size_t kBytes = kQueueOff + ref_queue_bytes(kWarps) + 1024;
    static_assert(TL % 8 == 0 && TK % 8 == 0, "swizzle phase must be per-thread constant");
    static_assert(CH == 32 || CH == 64, "chunk of one or two 128-byte rows");
    static_assert(BL <= 256 && BK <= 256, "TMA box rows");
};

// Issue the TMA copies of chunk c (global index within this CTA's tile list),
// chunk ch of the tile at (l0, k0).
template <class S, int ST>
__device__ __forceinline__ void issue_chunk_at(const CUtensorMap *mL, const CUtensorMap *mK, float *ring,
                                               uint64_t *full, int *last_issued, uint32_t c, int l0, int k0,
                                               int ch) {
    constexpr uint32_t kBytes = (uint32_t)S::kStageFloats * sizeof(float);
    const int s = (int)(c % ST);
    // stage layout: [sub][BL rows][32] line block, then [sub][BK rows][32]
    float *sL = ring + (size_t)s * S::kStageFloats;
    float *sK = sL + S::BL * S::CH;
    last_issued[s] = (int)c;
    mbar_arrive_expect_tx(smem_addr(&full[s]), kBytes);
#pragma unroll
    for (int sub = 0; sub < S::NSUB; ++sub) {
        tma_load_2d(smem_addr(sL + sub * S::BL * 32), mL, smem_addr(&full[s]), ch * S::CH + 32 * sub, l0);
        tma_load_2d(smem_addr(sK + sub * S::BK * 32), mK, smem_addr(&full[s]), ch * S::CH + 32 * sub, k0);
    }
}

// The same, locating chunk c from its index (divisions: used for the first
// ST chunks only).
template <class S, int ST>
__device__ __forceinline__ void issue_chunk(const CUtensorMap *mL, const CUtensorMap *mK,
                                            const CtgArgs &a, float *ring, uint64_t *full,
                                            int *last_issued, uint32_t c, int tiles_l, int tiles_k) {
    const int ti = (int)(c / (uint32_t)a.n_chunks), ch = (int)(c % (uint32_t)a.n_chunks);
    const int tile = blockIdx.x + ti * gridDim.x;
    int l0, k0;
    tile_origin(tile, tiles_l, tiles_k, S::BL, S::BK, l0, k0);
    issue_chunk_at<S, ST>(mL, mK, ring, full, last_issued, c, l0, k0, ch);
}

// ---------------------------------------------------------------------------
// One-box kernel (scaled rows).  WL x WK warps; a warp is 4 line-lanes x 8
// contingency-lanes; thread (tl, tk) owns lines tl + TL i (i < ML) and
// contingencies tk + TK j (j < MK).  No dedicated producer warp: the warp
// that releases a stage last (cumulative shared counter) refills it with the
// chunk ST ahead, so no warp waits for "stage empty".
// ---------------------------------------------------------------------------
template <int WL, int WK, int ML, int MK, int ST, bool S3, int CH_, int BODY, int MINB>
__global__ void __launch_bounds__(WL * WK * 32, MINB)
    k_ctg_one(const __grid_constant__ CUtensorMap mL, const __grid_constant__ CUtensorMap mK,
              const CtgArgs a) {
    using S = Shape<WL, WK, ML, MK, ST, S3, CH_>;
    constexpr int CH = S::CH, TL = S::TL, TK = S::TK, BL = S::BL;
    extern __shared__ unsigned char smem_raw[];
    float *ring = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                            ~uintptr_t(1023));
    float *acc3s = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(ring) + S::kRing) +
                   threadIdx.x;  // slot (i, j) at acc3s[(i * MK + j) * kThreads]
    uint64_t *full = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(ring) + S::kRing +
                                                  S::kAcc3);
    int *arrivals = reinterpret_cast<int *>(full + ST);
    int *last_issued = arrivals + ST;
    volatile int *abort_flag = last_issued + ST;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the warp's refinement queue (rebuilt where used: nothing of it stays live
    // through the tile loop)
    auto rq_of = [&]() {
        return ref_queue_of(reinterpret_cast<unsigned char *>(ring) + S::kQueueOff, warp, a.refq,
                            a.refq_cap, S::kWarps);
    };
    ref_queue_init(rq_of());
    // level-2 sums are folded into level 3 every kFold3 chunks (256 buses)
    constexpr int kFold3 = 256 / CH;
    const int tiles_k = (a.n_c + S::BK - 1) / S::BK;
    // screened calls walk the compacted line list live[0 .. n_ll)
    const int n_ll = a.n_live ? *a.n_live : a.n_l;
    const int tiles_l = (n_ll + BL - 1) / BL;
    const int n_tiles = a.n_live ? tiles_l * tiles_k : a.n_tiles;
    const int my_tiles = max(0, (n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x);
    const uint32_t total = (uint32_t)my_tiles * (uint32_t)a.n_chunks;
    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(smem_addr(&full[s]), 1);
            arrivals[s] = 0;
            last_issued[s] = -1;
        }
        *abort_flag = 0;
        fence_mbar_init();
        prefetch_tensormap(&mL);
        prefetch_tensormap(&mK);
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (uint32_t c = 0; c < total && c < (uint32_t)ST; ++c)
            issue_chunk<S, ST>(&mL, &mK, a, ring, full, last_issued, c, tiles_l, tiles_k);

    const int tl = (warp / WK) * 4 + (lane >> 3);
    const int tk = (warp % WK) * 8 + (lane & 7);
    const int xl = tl & 7, xk = tk & 7;  // SWIZZLE_128B: chunk q of row r sits at q ^ (r & 7)
    uint32_t it = 0;
    bool stop = false;
    for (int tile = blockIdx.x; tile < n_tiles && !stop; tile += gridDim.x) {
        int l0, k0;
        tile_origin(tile, tiles_l, tiles_k, S::BL, S::BK, l0, k0);
        float Lr[ML][MK];
#pragma unroll
        for (int i = 0; i < ML; ++i) {
            const int lq = l0 + tl + TL * i;
            int l = lq < n_ll ? (a.live ? __ldg(&a.live[lq]) : lq) : -1;
            if (l >= 0 && !IBP_IDX_OK(l < a.n_l, a.err)) l = -1;
#pragma unroll
            for (int j = 0; j < MK; ++j) {
                const int k = k0 + tk + TK * j;
                Lr[i][j] = (l >= 0 && k < a.n_c) ? __ldg(&a.lodf[(size_t)k * a.n_l + l]) : 0.0f;
            }
        }
        float acc1[ML][MK], acc2[ML][MK], acc3[S3 ? 1 : ML][S3 ? 1 : MK];
        // BODY 2: level-1 sums in two lanes (even / odd buses), packed adds
        float2 acc1p[BODY == 2 ? ML : 1][BODY == 2 ? MK : 1];
#pragma unroll
        for (int i = 0; i < ML; ++i)
#pragma unroll
            for (int j = 0; j < MK; ++j) {
                acc1[i][j] = acc2[i][j] = 0.0f;
                if constexpr (BODY == 2) acc1p[i][j] = make_float2(0.0f, 0.0f);
                if constexpr (S3) acc3s[(i * MK + j) * S::kThreads] = 0.0f;
                else acc3[i][j] = 0.0f;
            }

        for (int ch = 0; ch < a.n_chunks; ++ch, ++it) {
            const int s = (int)(it % ST);
            const uint32_t par = (it / ST) & 1u;
            bool ok = mbar_wait(smem_addr(&full[s]), par, a.wait_ns);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok || *abort_flag) {
                if (!ok && lane == 0) {
                    atomicOr(a.err, kErrTimeout);
                    *abort_flag = 1;
                }
                stop = true;
                break;
            }
            const float *sL = ring + (size_t)s * S::kStageFloats;
            const float *sK = sL + BL * CH;
#pragma unroll (BODY == 2 ? 8 : CH / 4)
            for (int q = 0; q < CH / 4; ++q) {
                // 16-byte group q of the chunk: sub-block q / 8, swizzled slot (q % 8) ^ (row & 7)
                const int sub = q >> 3, qq = q & 7;
                const float *bL = sL + sub * BL * 32, *bK = sK + sub * S::BK * 32;
                float4 fk[MK];
                const int ok4 = (qq ^ xk) << 2, ol4 = (qq ^ xl) << 2;
#pragma unroll
                for (int j = 0; j < MK; ++j)
                    fk[j] = *reinterpret_cast<const float4 *>(bK + (tk + TK * j) * 32 + ok4);
#pragma unroll
                for (int i = 0; i < ML; ++i) {
                    const float4 fl = *reinterpret_cast<const float4 *>(bL + (tl + TL * i) * 32 + ol4);
#pragma unroll
                    for (int j = 0; j < MK; ++j) {
                        const float L = Lr[i][j];
                        if constexpr (BODY == 0) {
                            float h;
                            h = __fmaf_rn(L, fk[j].x, fl.x);
                            acc1[i][j] = __fadd_ru(acc1[i][j], fabsf(h));
                            h = __fmaf_rn(L, fk[j].y, fl.y);
                            acc1[i][j] = __fadd_ru(acc1[i][j], fabsf(h));
                            h = __fmaf_rn(L, fk[j].z, fl.z);
                            acc1[i][j] = __fadd_ru(acc1[i][j], fabsf(h));
                            h = __fmaf_rn(L, fk[j].w, fl.w);
                            acc1[i][j] = __fadd_ru(acc1[i][j], fabsf(h));
                        } else if constexpr (BODY == 2) {
                            // two buses per packed FMA / add: h = RN(L hat_k + hat_l)
                            // per lane, |h| of buses (0,2) and (1,3) summed RU per
                            // lane, then accumulated per lane
                            const float2 L2 = make_float2(L, L);
                            float2 h01 = __ffma2_rn(L2, make_float2(fk[j].x, fk[j].y), make_float2(fl.x, fl.y));
                            float2 h23 = __ffma2_rn(L2, make_float2(fk[j].z, fk[j].w), make_float2(fl.z, fl.w));
                            h01 = make_float2(fabsf(h01.x), fabsf(h01.y));
                            h23 = make_float2(fabsf(h23.x), fabsf(h23.y));
                            acc1p[i][j] = __fadd2_ru(acc1p[i][j], __fadd2_ru(h01, h23));
                        } else {
                            // four buses summed as a round-up tree, then accumulated
                            const float h0 = __fmaf_rn(L, fk[j].x, fl.x);
                            const float h1 = __fmaf_rn(L, fk[j].y, fl.y);
                            const float h2 = __fmaf_rn(L, fk[j].z, fl.z);
                            const float h3 = __fmaf_rn(L, fk[j].w, fl.w);
                            const float s01 = __fadd_ru(fabsf(h0), fabsf(h1));
                            const float s23 = __fadd_ru(fabsf(h2), fabsf(h3));
                            acc1[i][j] = __fadd_ru(acc1[i][j], __fadd_ru(s01, s23));
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) {
                // release the stage; the last of the warps refills it
                __threadfence_block();
                const int old = atomicAdd(&arrivals[s], 1);
                if (old == (int)(it / ST) * S::kWarps + S::kWarps - 1) {
                    const uint32_t nxt = it + ST;
                    if (nxt < total && !*abort_flag) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        // chunk ch + ST of this tile, or (rarely) of a later one:
                        // the refilling warp is on the critical path of the
                        // whole CTA, so it locates the chunk without divisions
                        int nch = ch + ST, nl0 = l0, nk0 = k0;
                        if (nch >= a.n_chunks) {
                            const int ahead = nch / a.n_chunks;
                            nch -= ahead * a.n_chunks;
                            tile_origin(tile + ahead * (int)gridDim.x, tiles_l, tiles_k, S::BL, S::BK, nl0, nk0);
                        }
                        issue_chunk_at<S, ST>(&mL, &mK, ring, full, last_issued, nxt, nl0, nk0, nch);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < ML; ++i)
#pragma unroll
                for (int j = 0; j < MK; ++j) {
                    if constexpr (BODY == 2) {
                        acc2[i][j] = __fadd_ru(acc2[i][j], __fadd_ru(acc1p[i][j].x, acc1p[i][j].y));
                        acc1p[i][j] = make_float2(0.0f, 0.0f);
                    } else {
                        acc2[i][j] = __fadd_ru(acc2[i][j], acc1[i][j]);
                        acc1[i][j] = 0.0f;
                    }
                }
            if ((ch & (kFold3 - 1)) == kFold3 - 1) {
#pragma unroll
                for (int i = 0; i < ML; ++i)
#pragma unroll
                    for (int j = 0; j < MK; ++j) {
                        if constexpr (S3) {
                            float &a3 = acc3s[(i * MK + j) * S::kThreads];
                            a3 = __fadd_ru(a3, acc2[i][j]);
                        } else {
                            acc3[i][j] = __fadd_ru(acc3[i][j], acc2[i][j]);
                        }
                        acc2[i][j] = 0.0f;
                    }
            }
        }
        if (stop) break;
        float slo = 0.0f, shi = 0.0f, whi = 0.0f, wlo = 0.0f, cslo = 0.0f, cwhi = 0.0f;
        uint64_t rmask = 0;
        // the inputs of the thread's pairs, loaded together (two rounds of
        // independent loads per tile rather than dependent loads per pair)
        int ls[ML];
        LineIn lin[ML];
        CtgIn cin[MK];
#pragma unroll
        for (int i = 0; i < ML; ++i) {
            const int lq = l0 + tl + TL * i;
            ls[i] = lq < n_ll ? (a.live ? __ldg(&a.live[lq]) : lq) : -1;
            if (ls[i] >= 0 && !IBP_IDX_OK(ls[i] < a.n_l, a.err)) ls[i] = -1;
        }
#pragma unroll
        for (int j = 0; j < MK; ++j) {
            const int k = k0 + tk + TK * j;
            cin[j] = k < a.n_c ? load_ctg_in(a, 0, k) : CtgIn{-1, 0.0f, 0.0f, 0.0f};
        }
#pragma unroll
        for (int i = 0; i < ML; ++i)
            lin[i] = ls[i] >= 0 ? load_line_in(a, 0, ls[i]) : LineIn{0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        const float eta_r = __ldg(&a.box_consts[0]), eta_c = __ldg(&a.box_consts[1]);
#pragma unroll
        for (int i = 0; i < ML; ++i)
#pragma unroll
            for (int j = 0; j < MK; ++j) {
                if (ls[i] >= 0 && cin[j].kl >= 0) {
                    float a3;
                    if constexpr (S3) a3 = acc3s[(i * MK + j) * S::kThreads];
                    else a3 = acc3[i][j];
                    if (pair_epilogue_call(a, 0, ls[i], k0 + tk + TK * j, Lr[i][j], __fadd_ru(a3, acc2[i][j]),
                                           lin[i], cin[j], eta_r, eta_c, slo, shi, whi, wlo, cslo, cwhi))
                        rmask |= 1ull << (i * MK + j);
                }
            }
        // candidates of the FP64 refinement: queued, or (queue full) the FP32 terms
        const bool queued =
            a.ref.phi64 &&
            ref_enqueue<ML * MK>(
                rq_of(), rmask,
                [&](int q, int &l, int &k) {
                    const int lq = l0 + tl + TL * (q / MK);
                    l = a.live ? __ldg(&a.live[lq]) : lq;
                    k = k0 + tk + TK * (q % MK);
                },
                0, tile * a.warps_per_tile + warp);
        if (!queued) {
            slo = __fadd_rd(slo, cslo);
            whi = __fadd_ru(whi, cwhi);
        }
        write_warp_partials(a, tile, warp, 0, slo, shi, whi, wlo, ML * MK + 1);
    }
    // the queued refinements: published for k_refine_queue, or refined here
    if (a.ref.phi64) ref_finish(rq_of(), a.refq_cnt, S::kWarps, [&](int) -> const CtgArgs & { return a; });
    // Every warp gets here (all waits are bounded).  After an abort, copies
    // may still be in flight: wait (bounded) for the last one of each stage.
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) {
        for (int s = 0; s < ST; ++s) {
            const int c = last_issued[s];
            if (c >= 0) mbar_wait(smem_addr(&full[s]), ((uint32_t)c / ST) & 1u, a.wait_ns);
        }
    }
}

// ---------------------------------------------------------------------------
// Multi-box kernel.  Work item = (line tile of 64, contingency tile of 16,
// box tile of 16).  A warp is 4 line-lanes x 8 contingency-lanes.  With one
// contingency per thread (MK = 1), 8 warps = 4 line groups x 2 contingency
// groups and thread (tl, tk) owns lines tl + 16 i (i < 4), contingency tk and
// all 16 boxes (BH = 1); per (pair, bus)
//   h = RN(L~ Phi~[k,b] + Phi~[l,b]),  acc_j <- RU(|h| r_jb + acc_j)  (j < 16).
// The default (MK = 2, BH = 2) gives a thread contingencies tk and tk + 8 and
// one half of the boxes, so each radius it loads serves 8 pairs instead of 4;
// both halves form h.  Stage = unscaled PTDF rows of the line and contingency
// tiles (SWIZZLE_128B) and the radius tile [32 buses][16 boxes] (bus-major,
// broadcast reads).  Level-3 radius sums live in shared memory.
// ---------------------------------------------------------------------------
constexpr int kMB = 16;  // boxes per work item

// BH = box halves: 1 -> each thread 16 boxes; 2 -> the second set of warps
// takes boxes 8..15 of the item (h is formed by both halves).  ML = lines per
// thread: 4 -> 8 warps per half, 2 -> 16 warps per half (64 lines per item).
// MK = contingencies per thread: 2 halves the warps per half, and each radius
// a thread loads serves twice the pairs.
template <int ST, int BH = 1, int ML_ = 4, int MK_ = 1>
struct MultiShape {
    static constexpr int ML = ML_, MK = MK_;
    static constexpr int TL = 64 / ML, TK = 16 / MK;  // line / contingency lanes
    static_assert(TK % 8 == 0, "a warp spans 8 contingency lanes");
    static constexpr int kWarpsHalf = TL / 4 * (TK / 8);  // warps of one box half
    static constexpr int kWarps = kWarpsHalf * BH, kThreads = 32 * kWarps;
    static constexpr int kMBT = kMB / BH;  // boxes per thread
    static constexpr int BL = TL * ML, BK = TK * MK;
    static constexpr int CH = 32;
    static constexpr int kStageFloats = (BL + BK) * CH + CH * kMB;
    static constexpr size_t kRing = (size_t)ST * kStageFloats * sizeof(float);
    static constexpr size_t kAcc3 = (size_t)ML * MK * kMBT * kThreads * sizeof(float);
    static constexpr size_t kCtl = ST * sizeof(uint64_t) + 2 * ST * sizeof(int) + 16;
    // per-warp copy of the current item's kernel arguments
    static constexpr size_t kArgs = (size_t)kWarps * ((sizeof(CtgArgs) + 15) / 16 * 16);
    // per-warp queues of the pairs for the FP64 refinement (16-byte aligned)
    static constexpr size_t kQueueOff = kRing + kAcc3 + kArgs + (kCtl + 15) / 16 * 16;
    static constexpr size_t kBytes = kQueueOff + ref_queue_bytes(kWarps) + 1024;
    static_assert((BL + BK) * CH * sizeof(float) % 1024 == 0, "radius tile alignment");
    static_assert(kStageFloats * sizeof(float) % 1024 == 0, "stage alignment");
};

__device__ __forceinline__ void multi_origin(int item, int tiles_l, int tiles_k, int box_tiles,
                                             int BL, int BK, int &l0, int &k0, int &b0,
                                             int &tile_lk) {
    // box tiles innermost (concurrent CTAs share rows), then banded (line, ctg)
    tile_lk = item / box_tiles;
    b0 = (item % box_tiles) * kMB;
    tile_origin(tile_lk, tiles_l, tiles_k, BL, BK, l0, k0);
}

// One work item of the multi-box kernel: the case's arguments and TMA maps and
// the tile origin.
struct MultiItemView {
    const CtgArgs *a;
    const CUtensorMap *mL, *mK, *mR;
    int l0, k0, b0, tlk, n_chunks, cid;  // cid: the case's index in the plan
};

// Work plan of one case: item i of this CTA is blockIdx.x + i * gridDim.x.
struct SinglePlan {
    const CtgArgs *a;
    const CUtensorMap *mL, *mK, *mR;
    int tiles_l, tiles_k, box_tiles, BL, BK, n_tiles;
    __device__ int n_items() const {
        return max(0, (n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x);
    }
    __device__ MultiItemView item(int i) const {
        MultiItemView v{a, mL, mK, mR, 0, 0, 0, 0, a->n_chunks, 0};
        multi_origin((int)blockIdx.x + i * (int)gridDim.x, tiles_l, tiles_k, box_tiles, BL, BK,
                     v.l0, v.k0, v.b0, v.tlk);
        return v;
    }
    __device__ const CtgArgs &case_args(int) const { return *a; }
};

// Work plan of many cases: a host-built table, sliced per CTA.
struct CasesPlan {
    const MultiItem *items;       // this CTA's items
    const uint32_t *prefix;       // [count + 1] chunk prefix of this CTA's items
    int count;
    const CtgArgs *args;          // per case
    const CUtensorMap *maps;      // per case: L rows, contingency rows, radius
    __device__ int n_items() const { return count; }
    __device__ MultiItemView item(int i) const {
        const MultiItem m = items[i];
        MultiItemView v{args + m.case_id, maps + 3 * m.case_id, maps + 3 * m.case_id + 1,
                        maps + 3 * m.case_id + 2, m.l0, m.k0, m.b0, m.tile_lk, m.n_chunks, m.case_id};
        return v;
    }
    __device__ const CtgArgs &case_args(int cid) const { return args[cid]; }
};

template <int ST, int BH, int ML, int MK>
__device__ __forceinline__ void issue_multi_at(const MultiItemView &v, float *ring, uint64_t *full,
                                               int *last_issued, uint32_t c, int ch) {
    using S = MultiShape<ST, BH, ML, MK>;
    constexpr uint32_t kBytes = (uint32_t)S::kStageFloats * sizeof(float);
    const int s = (int)(c % ST);
    float *sL = ring + (size_t)s * S::kStageFloats;
    float *sK = sL + S::BL * S::CH;
    float *sR = sK + S::BK * S::CH;
    last_issued[s] = (int)c;
    mbar_arrive_expect_tx(smem_addr(&full[s]), kBytes);
    tma_load_2d(smem_addr(sL), v.mL, smem_addr(&full[s]), ch * S::CH, v.l0);
    tma_load_2d(smem_addr(sK), v.mK, smem_addr(&full[s]), ch * S::CH, v.k0);
    tma_load_2d(smem_addr(sR), v.mR, smem_addr(&full[s]), v.b0, ch * S::CH);
}

template <int ST, int BH, int ML, int MK, class Plan>
__device__ __forceinline__ void issue_multi(const Plan &P, float *ring, uint64_t *full,
                                            int *last_issued, uint32_t c, int i, int ch) {
    issue_multi_at<ST, BH, ML, MK>(P.item(i), ring, full, last_issued, c, ch);
}

// PK: accumulate box pairs with the packed two-lane FMA (same rounding per lane)
// GRP: wait for and release the stages of two chunks of an item together
template <int ST, int BH, int ML_, class Plan, bool PK = false, int MK_ = 1, bool GRP = false>
__device__ __forceinline__ void multi_body(const Plan &P, unsigned long long wait_ns, int *err) {
    using S = MultiShape<ST, BH, ML_, MK_>;
    constexpr int CH = S::CH, ML = S::ML, MK = S::MK, TL = S::TL, TK = S::TK, BL = S::BL,
                  kMBT = S::kMBT;
    extern __shared__ unsigned char smem_raw[];
    float *ring = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                            ~uintptr_t(1023));
    float *acc3 = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(ring) + S::kRing) +
                  threadIdx.x;  // slot (i, c, j) at acc3[((i * MK + c) * kMBT + j) * kThreads]
    constexpr size_t kArgSlot = (sizeof(CtgArgs) + 15) / 16 * 16;
    unsigned char *arg_base = reinterpret_cast<unsigned char *>(ring) + S::kRing + S::kAcc3;
    uint64_t *full = reinterpret_cast<uint64_t *>(arg_base + S::kArgs);
    int *arrivals = reinterpret_cast<int *>(full + ST);
    int *last_issued = arrivals + ST;
    volatile int *abort_flag = last_issued + ST;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    CtgArgs *my_args = reinterpret_cast<CtgArgs *>(arg_base + warp * kArgSlot);
    const CtgArgs &a0 = P.case_args(0);
    const RefQueue rq = ref_queue_of(reinterpret_cast<unsigned char *>(ring) + S::kQueueOff, warp,
                                     a0.refq, a0.refq_cap, S::kWarps);
    ref_queue_init(rq);
    constexpr int kFold3 = 8;
    const int my_items = P.n_items();
    uint32_t total = 0;
    for (int i = 0; i < my_items; ++i) total += (uint32_t)P.item(i).n_chunks;
    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(smem_addr(&full[s]), 1);
            arrivals[s] = 0;
            last_issued[s] = -1;
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int i = 0, ch = 0;
        for (uint32_t c = 0; c < total && c < (uint32_t)ST; ++c) {
            while (ch >= P.item(i).n_chunks) {
                ch -= P.item(i).n_chunks;
                ++i;
            }
            issue_multi<ST, BH, ML_, MK_>(P, ring, full, last_issued, c, i, ch);
            ++ch;
        }
    }

    // box half of this warp (BH = 2) and its position inside the half
    const int half = warp / S::kWarpsHalf, wq = warp % S::kWarpsHalf;
    constexpr int kGK = TK / 8;  // contingency lane groups (warps) per line group
    const int tl = (wq / kGK) * 4 + (lane >> 3);
    const int tk = (wq % kGK) * 8 + (lane & 7);
    const int xl = tl & 7, xk = tk & 7;  // rows tk + TK c share the swizzle phase of tk
    uint32_t it = 0;
    bool stop = false;
    for (int ii = 0; ii < my_items && !stop; ++ii) {
        const MultiItemView v = P.item(ii);
        {
            // this warp's shared copy of the item's arguments (read by the epilogue)
            const int *src = reinterpret_cast<const int *>(v.a);
            int *dst = reinterpret_cast<int *>(my_args);
            for (int w = lane; w < (int)(sizeof(CtgArgs) / sizeof(int)); w += 32) dst[w] = src[w];
            __syncwarp();
        }
        const CtgArgs &a = *my_args;
        const int l0 = v.l0, b0 = v.b0, tlk = v.tlk;
        const int n_l = a.n_l, n_c = a.n_c, n_box = a.n_box;
        // screened calls walk the compacted line list live[0 .. n_ll)
        const int n_ll = a.n_live ? *a.n_live : n_l;
        float Lr[ML][MK];
#pragma unroll
        for (int i = 0; i < ML; ++i) {
            const int lq = l0 + tl + TL * i;
            int l = lq < n_ll ? (a.live ? __ldg(&a.live[lq]) : lq) : -1;
            if (l >= 0 && !IBP_IDX_OK(l < n_l, a.err)) l = -1;
#pragma unroll
            for (int c = 0; c < MK; ++c) {
                const int k = v.k0 + tk + TK * c;
                Lr[i][c] = (l >= 0 && k < n_c) ? __ldg(&a.lodf[(size_t)k * n_l + l]) : 0.0f;
            }
        }
        float acc1[ML][MK][kMBT], acc2[ML][MK][kMBT];
#pragma unroll
        for (int i = 0; i < ML; ++i)
#pragma unroll
            for (int c = 0; c < MK; ++c)
#pragma unroll
                for (int j = 0; j < kMBT; ++j) {
                    acc1[i][c][j] = acc2[i][c][j] = 0.0f;
                    acc3[((i * MK + c) * kMBT + j) * S::kThreads] = 0.0f;
                }
        for (int ch = 0; ch < v.n_chunks; ++ch, ++it) {
            const int s = (int)(it % ST);
            const uint32_t par = (it / ST) & 1u;
            if (!GRP || (ch & 1) == 0) {
                bool ok = mbar_wait(smem_addr(&full[s]), par, wait_ns);
                if (GRP && ok && ch + 1 < v.n_chunks)
                    ok = mbar_wait(smem_addr(&full[(it + 1) % ST]), ((it + 1) / ST) & 1u, wait_ns);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok || *abort_flag) {
                    if (!ok && lane == 0) {
                        atomicOr(err, kErrTimeout);
                        *abort_flag = 1;
                    }
                    stop = true;
                    break;
                }
            }
            const float *sL = ring + (size_t)s * S::kStageFloats;
            const float *sK = sL + BL * CH;
            const float *sR = sK + S::BK * CH;
#pragma unroll 2
            for (int q = 0; q < CH / 4; ++q) {
                float4 fk[MK];
#pragma unroll
                for (int c = 0; c < MK; ++c)
                    fk[c] = *reinterpret_cast<const float4 *>(sK + (tk + TK * c) * CH + ((q ^ xk) << 2));
                float4 fl[ML];
#pragma unroll
                for (int i = 0; i < ML; ++i)
                    fl[i] = *reinterpret_cast<const float4 *>(sL + (tl + TL * i) * CH + ((q ^ xl) << 2));
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const float *rr = sR + (4 * q + t) * kMB + half * kMBT;
                    float r[kMBT];
#pragma unroll
                    for (int u = 0; u < kMBT / 4; ++u) {
                        const float4 r4 = *reinterpret_cast<const float4 *>(rr + 4 * u);
                        r[4 * u] = r4.x;
                        r[4 * u + 1] = r4.y;
                        r[4 * u + 2] = r4.z;
                        r[4 * u + 3] = r4.w;
                    }
#pragma unroll
                    for (int i = 0; i < ML; ++i) {
                        const float flt = t == 0 ? fl[i].x : t == 1 ? fl[i].y : t == 2 ? fl[i].z : fl[i].w;
#pragma unroll
                        for (int c = 0; c < MK; ++c) {
                            const float fkt = t == 0 ? fk[c].x : t == 1 ? fk[c].y : t == 2 ? fk[c].z : fk[c].w;
                            const float ah = fabsf(__fmaf_rn(Lr[i][c], fkt, flt));
                            float *ac = acc1[i][c];
                            if constexpr (PK) {
                                const float2 ah2 = make_float2(ah, ah);
#pragma unroll
                                for (int j = 0; j < kMBT; j += 2) {
                                    const float2 v = __ffma2_ru(ah2, make_float2(r[j], r[j + 1]),
                                                                make_float2(ac[j], ac[j + 1]));
                                    ac[j] = v.x;
                                    ac[j + 1] = v.y;
                                }
                            } else {
#pragma unroll
                                for (int j = 0; j < kMBT; ++j) ac[j] = __fmaf_ru(ah, r[j], ac[j]);
                            }
                        }
                    }
                }
            }
            __syncwarp();
            // release chunk (itr, chr) of this item; the last of the warps refills it
            auto release = [&](uint32_t itr, int chr) {
                const int old = atomicAdd(&arrivals[itr % ST], 1);
                if (old == (int)(itr / ST) * S::kWarps + S::kWarps - 1) {
                    const uint32_t nxt = itr + ST;
                    if (nxt < total && !*abort_flag) {
                        // advance ST chunks from this warp's own position; the
                        // refilling warp is on the critical path of the whole
                        // CTA, so within the item it reuses its own view (no
                        // table loads or divisions)
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        int ch2 = chr + ST;
                        if (ch2 < v.n_chunks) {
                            issue_multi_at<ST, BH, ML_, MK_>(v, ring, full, last_issued, nxt, ch2);
                        } else {
                            int i2 = ii;
                            ch2 -= v.n_chunks;
                            ++i2;
                            while (ch2 >= P.item(i2).n_chunks) {
                                ch2 -= P.item(i2).n_chunks;
                                ++i2;
                            }
                            issue_multi<ST, BH, ML_, MK_>(P, ring, full, last_issued, nxt, i2, ch2);
                        }
                    }
                }
            };
            if (lane == 0 && (!GRP || (ch & 1) || ch == v.n_chunks - 1)) {
                __threadfence_block();
                if (GRP && (ch & 1)) release(it - 1, ch - 1);
                release(it, ch);
            }
#pragma unroll
            for (int i = 0; i < ML; ++i)
#pragma unroll
                for (int c = 0; c < MK; ++c)
#pragma unroll
                    for (int j = 0; j < kMBT; ++j) {
                        acc2[i][c][j] = __fadd_ru(acc2[i][c][j], acc1[i][c][j]);
                        acc1[i][c][j] = 0.0f;
                    }
            if ((ch & (kFold3 - 1)) == kFold3 - 1) {
#pragma unroll
                for (int i = 0; i < ML; ++i)
#pragma unroll
                    for (int c = 0; c < MK; ++c)
#pragma unroll
                        for (int j = 0; j < kMBT; ++j) {
                            float &a3 = acc3[((i * MK + c) * kMBT + j) * S::kThreads];
                            a3 = __fadd_ru(a3, acc2[i][c][j]);
                            acc2[i][c][j] = 0.0f;
                        }
            }
        }
        if (stop) break;
        // the box-independent inputs of the thread's pairs: lines, outaged
        // lines and ratings, loaded once per item
        int ls[ML], kls[MK];
        float rup[ML], rdn[ML];
#pragma unroll
        for (int i = 0; i < ML; ++i) {
            const int lq = l0 + tl + TL * i;
            ls[i] = lq < n_ll ? (a.live ? __ldg(&a.live[lq]) : lq) : -1;
            if (ls[i] >= 0 && !IBP_IDX_OK(ls[i] < a.n_l, a.err)) ls[i] = -1;
            rup[i] = ls[i] >= 0 ? __ldg(&a.rate_up[ls[i]]) : 0.0f;
            rdn[i] = ls[i] >= 0 ? __ldg(&a.rate_dn[ls[i]]) : 0.0f;
        }
#pragma unroll
        for (int c = 0; c < MK; ++c) {
            const int k = v.k0 + tk + TK * c;
            kls[c] = k < n_c ? __ldg(&a.ctg_line[k]) : -1;
            if (kls[c] >= 0 && !IBP_IDX_OK(kls[c] < a.n_l, a.err)) kls[c] = -1;
        }
#pragma unroll 1
        for (int j = 0; j < kMBT; ++j) {
            const int box = b0 + half * kMBT + j;
            if (box >= n_box) break;
            float slo = 0.0f, shi = 0.0f, whi = 0.0f, wlo = 0.0f, cslo = 0.0f, cwhi = 0.0f;
            uint64_t rmask = 0;
            // this box's inputs, loaded together
            const size_t ob = (size_t)box * a.n_l;
            LineIn lin[ML];
            CtgIn cin[MK];
#pragma unroll
            for (int i = 0; i < ML; ++i)
                lin[i] = ls[i] >= 0 ? LineIn{__ldg(&a.line_c[ob + ls[i]]), __ldg(&a.line_e[ob + ls[i]]),
                                             __ldg(&a.line_R[ob + ls[i]]), rup[i], rdn[i]}
                                    : LineIn{0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int c = 0; c < MK; ++c)
                cin[c] = kls[c] >= 0 ? CtgIn{kls[c], __ldg(&a.line_c[ob + kls[c]]), __ldg(&a.line_e[ob + kls[c]]),
                                             __ldg(&a.line_R[ob + kls[c]])}
                                     : CtgIn{-1, 0.0f, 0.0f, 0.0f};
            const float eta_r = __ldg(&a.box_consts[(size_t)box * 4]);
            const float eta_c = __ldg(&a.box_consts[(size_t)box * 4 + 1]);
#pragma unroll
            for (int i = 0; i < ML; ++i) {
#pragma unroll
                for (int c = 0; c < MK; ++c) {
                    if (ls[i] >= 0 && kls[c] >= 0) {
                        float a2 = 0.0f;
                        // registers cannot be indexed by the runtime j: select it
#pragma unroll
                        for (int jj = 0; jj < kMBT; ++jj)
                            if (jj == j) a2 = acc2[i][c][jj];
                        const float A = __fadd_ru(acc3[((i * MK + c) * kMBT + j) * S::kThreads], a2);
                        if (pair_epilogue_in(a, box, ls[i], v.k0 + tk + TK * c, Lr[i][c], A, lin[i], cin[c],
                                             eta_r, eta_c, slo, shi, whi, wlo, cslo, cwhi))
                            rmask |= 1ull << (i * MK + c);
                    }
                }
            }
            // candidates of the FP64 refinement: queued, or (queue full) the FP32 terms
            const bool queued =
                a.ref.phi64 &&
                ref_enqueue<ML * MK>(
                    rq, rmask,
                    [&](int q, int &l, int &k) {
                        l = ls[q / MK];
                        k = v.k0 + tk + TK * (q % MK);
                    },
                    (v.cid << 16) | box, tlk * a.warps_per_tile + wq);
            if (!queued) {
                slo = __fadd_rd(slo, cslo);
                whi = __fadd_ru(whi, cwhi);
            }
            // partial rows per item: kWarpsHalf (the warp's place in its
            // half; each box belongs to exactly one half)
            write_warp_partials(a, tlk, wq, box, slo, shi, whi, wlo, ML * MK + 1);
        }
    }
    // the queued refinements: published for k_refine_queue, or refined here
    ref_finish(rq, a0.refq_cnt, S::kWarps, [&](int cid) -> const CtgArgs & { return P.case_args(cid); });
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) {
        for (int s = 0; s < ST; ++s) {
            const int c = last_issued[s];
            if (c >= 0) mbar_wait(smem_addr(&full[s]), ((uint32_t)c / ST) & 1u, wait_ns);
        }
    }
}

template <int ST, int BH, int ML, bool PK, int MK, bool GRP>
__global__ void __launch_bounds__(MultiShape<ST, BH, ML, MK>::kThreads, 1)
    k_ctg_multi(const __grid_constant__ CUtensorMap mL, const __grid_constant__ CUtensorMap mK,
                const __grid_constant__ CUtensorMap mR, const CtgArgs a) {
    using S = MultiShape<ST, BH, ML, MK>;
    if (threadIdx.x == 0) {
        prefetch_tensormap(&mL);
        prefetch_tensormap(&mK);
        prefetch_tensormap(&mR);
    }
    const int tiles_k = (a.n_c + S::BK - 1) / S::BK, box_tiles = (a.n_box + kMB - 1) / kMB;
    const int n_ll = a.n_live ? *a.n_live : a.n_l;
    const int tiles_l = a.n_live ? (n_ll + S::BL - 1) / S::BL : a.tiles_l;
    const int n_tiles = a.n_live ? tiles_l * tiles_k * box_tiles : a.n_tiles;
    const SinglePlan P{&a, &mL, &mK, &mR, tiles_l, tiles_k, box_tiles, S::BL, S::BK, n_tiles};
    multi_body<ST, BH, ML, SinglePlan, PK, MK, GRP>(P, a.wait_ns, a.err);
}

// Many cases in one persistent launch: CTA b walks items [start[b], start[b+1])
// of the host-built table (longest items first, dealt round-robin).
template <int ST, int BH, bool PK, int MK>
__global__ void __launch_bounds__(MultiShape<ST, BH, 4, MK>::kThreads, 1)
    k_ctg_cases(const MultiItem *__restrict__ items, const int *__restrict__ cta_start,
                const uint32_t *__restrict__ prefix, const CtgArgs *__restrict__ args,
                const CUtensorMap *__restrict__ maps, unsigned long long wait_ns, int *err) {
    const int s0 = cta_start[blockIdx.x], s1 = cta_start[blockIdx.x + 1];
    const CasesPlan P{items + s0, prefix + s0 + blockIdx.x, s1 - s0, args, maps};
    multi_body<ST, BH, 4, CasesPlan, PK, MK>(P, wait_ns, err);
}

template <int ST, int BH, int ML = 4, bool PK = false, int MK = 1, bool GRP = false>
static cudaError_t launch_multi(const CUtensorMap &mL, const CUtensorMap &mK,
                                const CUtensorMap &mR, const CtgArgs &a, int grid,
                                cudaStream_t s) {
    using S = MultiShape<ST, BH, ML, MK>;
    auto kern = k_ctg_multi<ST, BH, ML, PK, MK, GRP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S::kBytes);
    if (e != cudaSuccess) return e;
    grid = std::min(grid, a.n_tiles);
    kern<<<grid, S::kThreads, S::kBytes, s>>>(mL, mK, mR, a);
    return cudaGetLastError();
}

cudaError_t launch_ctg_multi(const CtgVariant &v, const CUtensorMap &mL, const CUtensorMap &mK,
                             const CUtensorMap &mR, const CtgArgs &a, int grid, cudaStream_t s) {
    if (a.n_tiles <= 0) return cudaSuccess;
    switch (v.id) {
    case 20: return launch_multi<4, 1>(mL, mK, mR, a, grid, s);
    case 21: return launch_multi<6, 1>(mL, mK, mR, a, grid, s);
    case 22: return launch_multi<4, 2>(mL, mK, mR, a, grid, s);
    case 23: return launch_multi<6, 2>(mL, mK, mR, a, grid, s);
    case 24: return launch_multi<4, 1, 2>(mL, mK, mR, a, grid, s);
    case 25: return launch_multi<6, 1, 2>(mL, mK, mR, a, grid, s);
    case 26: return launch_multi<4, 1, 4, true>(mL, mK, mR, a, grid, s);
    case 27: return launch_multi<4, 2, 4, true>(mL, mK, mR, a, grid, s);
    case 28: return launch_multi<4, 2, 4, true, 2>(mL, mK, mR, a, grid, s);
    case 29: return launch_multi<6, 2, 4, true, 2>(mL, mK, mR, a, grid, s);
    case 30: return launch_multi<6, 2, 4, true, 2, true>(mL, mK, mR, a, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int ST, int BH, bool PK, int MK>
static cudaError_t launch_cases(const MultiItem *items, const int *cta_start, const uint32_t *prefix,
                                const CtgArgs *args, const CUtensorMap *maps, int grid,
                                unsigned long long wait_ns, int *err, cudaStream_t s) {
    using S = MultiShape<ST, BH, 4, MK>;
    auto kern = k_ctg_cases<ST, BH, PK, MK>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S::kBytes);
    if (e != cudaSuccess) return e;
    kern<<<grid, S::kThreads, S::kBytes, s>>>(items, cta_start, prefix, args, maps, wait_ns, err);
    return cudaGetLastError();
}

// The many-case launch runs the body of multi-box variant `variant`: 20/21
// (8 warps), 22/23 (box halves), 26 (8 warps, packed FMA), 27 (box halves,
// packed FMA), each with 4 stages, and 28 (4 lines x 2 contingencies x 8 boxes
// per thread); 29 and any other value run the default, 28's body with 6
// stages.  The launch and the partial-row count both dispatch through
// with_cases_body, so they agree.
template <int ST_, int BH_, bool PK_, int MK_>
struct CasesBody {
    static constexpr int ST = ST_, BH = BH_, MK = MK_;
    static constexpr bool PK = PK_;
};

template <class F>
static auto with_cases_body(int variant, F f) {
    switch (variant) {
    case 20: case 21: return f(CasesBody<4, 1, false, 1>{});
    case 22: case 23: return f(CasesBody<4, 2, false, 1>{});
    case 26: return f(CasesBody<4, 1, true, 1>{});
    case 27: return f(CasesBody<4, 2, true, 1>{});
    case 28: return f(CasesBody<4, 2, true, 2>{});
    default: return f(CasesBody<6, 2, true, 2>{});  // 29, and 30 (pairs: single-case calls only)
    }
}

cudaError_t launch_ctg_cases(int variant, const MultiItem *items, const int *cta_start,
                             const uint32_t *prefix, const CtgArgs *args, const CUtensorMap *maps,
                             int grid, unsigned long long wait_ns, int *err, cudaStream_t s) {
    if (grid <= 0) return cudaSuccess;
    return with_cases_body(variant, [&](auto body) {
        using B = decltype(body);
        return launch_cases<B::ST, B::BH, B::PK, B::MK>(items, cta_start, prefix, args, maps, grid,
                                                        wait_ns, err, s);
    });
}

int cases_rows_per_item(int variant) {
    return with_cases_body(variant, [](auto body) {
        using B = decltype(body);
        return MultiShape<B::ST, B::BH, 4, B::MK>::kWarpsHalf;
    });
}

void multi_tile_shape(int *BL, int *BK, int *CH) {
    *BL = MultiShape<4>::BL;
    *BK = MultiShape<4>::BK;
    *CH = MultiShape<4>::CH;
}

// ---------------------------------------------------------------------------
// Variant table and launcher
// ---------------------------------------------------------------------------
// {id, batched, BL, BK, CH, ST, boxes per thread, body, name}; warps and the loop
// body are fixed per id in launch_ctg / ctg_warps.
static const CtgVariant kVariants[] = {
    {1, 0, 128, 64, 32, 4, 1, 0, "8 warps, 8x4/thread, 32-bus chunks, 4 stages, 1 add per bus"},
    {3, 0, 128, 64, 32, 4, 1, 0, "16 warps, 4x4/thread, 32-bus chunks, 4 stages, 1 add per bus"},
    {6, 0, 128, 64, 32, 4, 1, 1, "8 warps, 8x4/thread, 32-bus chunks, 4 stages, 4-bus add tree"},
    {7, 0, 128, 64, 64, 3, 1, 1, "8 warps, 8x4/thread, 64-bus chunks, 3 stages, 4-bus add tree"},
    {8, 0, 128, 64, 32, 4, 1, 1, "16 warps, 4x4/thread, 32-bus chunks, 4 stages, 4-bus add tree"},
    {9, 0, 128, 64, 64, 3, 1, 1, "16 warps, 4x4/thread, 64-bus chunks, 3 stages, 4-bus add tree"},
    {10, 0, 64, 64, 32, 4, 1, 1, "2 CTAs/SM x 8 warps, 4x4/thread, 32-bus chunks, 4 stages, tree"},
    {11, 0, 64, 64, 64, 2, 1, 1, "2 CTAs/SM x 8 warps, 4x4/thread, 64-bus chunks, 2 stages, tree"},
    {12, 0, 128, 64, 64, 3, 1, 2, "16 warps, 4x4/thread, 64-bus chunks, 3 stages, packed two-lane sums"},
    {13, 0, 128, 64, 32, 4, 1, 2, "16 warps, 4x4/thread, 32-bus chunks, 4 stages, packed two-lane sums"},
    {15, 0, 64, 64, 32, 4, 1, 2, "2 CTAs/SM x 8 warps, 4x4/thread, 32-bus chunks, 4 stages, packed"},
    {16, 0, 64, 64, 64, 2, 1, 2, "2 CTAs/SM x 8 warps, 4x4/thread, 64-bus chunks, 2 stages, packed"},
    {20, 1, 64, 16, 32, 4, 16, -1, "multi-box 64x16x16, 8 warps, 4 lines x 16 boxes/thread, 4 stages"},
    {21, 1, 64, 16, 32, 6, 16, -1, "multi-box 64x16x16, 8 warps, 4 lines x 16 boxes/thread, 6 stages"},
    {22, 1, 64, 16, 32, 4, 8, -1, "multi-box 64x16x16, 16 warps, 4 lines x 8 boxes/thread, 4 stages"},
    {23, 1, 64, 16, 32, 6, 8, -1, "multi-box 64x16x16, 16 warps, 4 lines x 8 boxes/thread, 6 stages"},
    {24, 1, 64, 16, 32, 4, 16, -1, "multi-box 64x16x16, 16 warps, 2 lines x 16 boxes/thread, 4 stages"},
    {25, 1, 64, 16, 32, 6, 16, -1, "multi-box 64x16x16, 16 warps, 2 lines x 16 boxes/thread, 6 stages"},
    {26, 1, 64, 16, 32, 4, 16, -1, "multi-box 64x16x16, 8 warps, 4 lines x 16 boxes/thread, packed FMA"},
    {27, 1, 64, 16, 32, 4, 8, -1, "multi-box 64x16x16, 16 warps, 4 lines x 8 boxes/thread, packed FMA"},
    {28, 1, 64, 16, 32, 4, 8, -1, "multi-box 64x16x16, 8 warps, 4 lines x 2 ctgs x 8 boxes/thread, packed FMA"},
    {29, 1, 64, 16, 32, 6, 8, -1, "multi-box 64x16x16, 8 warps, 4 lines x 2 ctgs x 8 boxes/thread, packed FMA, 6 stages"},
    {30, 1, 64, 16, 32, 6, 8, -1, "multi-box as 29, stages waited for and released in pairs"},
};

const CtgVariant *ctg_variants(int *count) {
    *count = (int)(sizeof(kVariants) / sizeof(kVariants[0]));
    return kVariants;
}

const CtgVariant *ctg_variant_by_id(int id) {
    int n;
    const CtgVariant *v = ctg_variants(&n);
    for (int i = 0; i < n; ++i)
        if (v[i].id == id) return &v[i];
    return nullptr;
}

template <int WL, int WK, int ML, int MK, int ST, bool S3, int CH, int BODY, int MINB = 1>
static cudaError_t launch_one(const CUtensorMap &mL, const CUtensorMap &mK, const CtgArgs &a,
                              int grid, cudaStream_t s) {
    using S = Shape<WL, WK, ML, MK, ST, S3, CH>;
    auto kern = k_ctg_one<WL, WK, ML, MK, ST, S3, CH, BODY, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S::kBytes);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    if (fa.maxThreadsPerBlock < S::kThreads) {
        fprintf(stderr, "k_ctg_one: %d registers allow only %d threads per block (need %d)\n",
                fa.numRegs, fa.maxThreadsPerBlock, S::kThreads);
        return cudaErrorLaunchOutOfResources;
    }
    // persistent grid: as many CTAs as fit on the SMs at once
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, S::kThreads, S::kBytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    grid = std::min(grid * per_sm, a.n_tiles);
    kern<<<grid, S::kThreads, S::kBytes, s>>>(mL, mK, a);
    return cudaGetLastError();
}

// partial-sum rows written per tile (per work item for the multi-box kernels)
int ctg_warps(const CtgVariant &v) {
    switch (v.id) {
    case 3: case 8: case 9: case 12: case 13: case 24: case 25: return 16;
    case 28: case 29: case 30: return MultiShape<6, 2, 4, 2>::kWarpsHalf;
    default: return 8;
    }
}


cudaError_t launch_ctg(const CtgVariant &v, const CUtensorMap &mL, const CUtensorMap &mK,
                       const CtgArgs &a, int grid, cudaStream_t s) {
    if (a.n_tiles <= 0) return cudaSuccess;
    grid = std::min(grid, a.n_tiles);
    switch (v.id) {
    case 1: return launch_one<4, 2, 8, 4, 4, false, 32, 0>(mL, mK, a, grid, s);
    case 3: return launch_one<8, 2, 4, 4, 4, true, 32, 0>(mL, mK, a, grid, s);
    case 6: return launch_one<4, 2, 8, 4, 4, false, 32, 1>(mL, mK, a, grid, s);
    case 7: return launch_one<4, 2, 8, 4, 3, false, 64, 1>(mL, mK, a, grid, s);
    case 8: return launch_one<8, 2, 4, 4, 4, true, 32, 1>(mL, mK, a, grid, s);
    case 9: return launch_one<8, 2, 4, 4, 3, true, 64, 1>(mL, mK, a, grid, s);
    case 10: return launch_one<4, 2, 4, 4, 4, true, 32, 1, 2>(mL, mK, a, grid, s);
    case 11: return launch_one<4, 2, 4, 4, 2, true, 64, 1, 2>(mL, mK, a, grid, s);
    case 12: return launch_one<8, 2, 4, 4, 3, true, 64, 2>(mL, mK, a, grid, s);
    case 13: return launch_one<8, 2, 4, 4, 4, true, 32, 2>(mL, mK, a, grid, s);
    case 15: return launch_one<4, 2, 4, 4, 4, true, 32, 2, 2>(mL, mK, a, grid, s);
    case 16: return launch_one<4, 2, 4, 4, 2, true, 64, 2, 2>(mL, mK, a, grid, s);
    default: return cudaErrorInvalidValue;
    }
}


// ---------------------------------------------------------------------------
// The refinement of the queued pairs (see refine.cuh): k_refine_queue refines
// every entry of every region with one warp, k_refine_apply adds each region's
// results to their partial-sum rows in queue order (regions of different warps
// never share a row, so the sums do not depend on timing).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_refine_queue(const RefQueueArgs a) {
    extern __shared__ int soff[];  // [n_regions + 1] exclusive prefix of the counts
    __shared__ int part[256];
    const int n = a.n_regions, t = threadIdx.x;
    const int per = (n + 255) / 256;
    int sum = 0;
    for (int i = t * per; i < min(n, (t + 1) * per); ++i) sum += min(a.cnt[i], a.cap);
    part[t] = sum;
    __syncthreads();
    if (t == 0) {
        int run = 0;
        for (int i = 0; i < 256; ++i) {
            const int v = part[i];
            part[i] = run;
            run += v;
        }
        soff[n] = run;
    }
    __syncthreads();
    int run = part[t];
    for (int i = t * per; i < min(n, (t + 1) * per); ++i) {
        soff[i] = run;
        run += min(a.cnt[i], a.cap);
    }
    __syncthreads();
    const int total = soff[n];
    const int lane = t & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + t) >> 5), nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int e = gw; e < total; e += nw) {
        int lo = 0, hi = n;  // the region g with soff[g] <= e < soff[g + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (soff[mid] <= e) lo = mid;
            else hi = mid;
        }
        const size_t slot = (size_t)lo * a.cap + (e - soff[lo]);
        const int4 q = a.e[slot];
        const CtgArgs &c = a.args ? a.args[q.z >> 16] : a.one;
        const int box = q.z & 0xffff;
        const int kl = __ldg(&c.ctg_line[q.y]);
        const float Lt = __ldg(&c.lodf[(size_t)q.y * c.n_l + q.x]);
        const RefOut o = refine_term(c.ref, box, q.x, kl, q.y, Lt, __ldg(&c.ref.rate_c64[q.x]), kRefPair);
        if (lane == 0) a.res[slot] = make_double2(o.s_lo, o.w);
    }
}

__global__ void k_refine_apply(const RefQueueArgs a) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.n_regions) return;
    const int n = min(a.cnt[g], a.cap);
    for (int i = 0; i < n; ++i) {
        const size_t slot = (size_t)g * a.cap + i;
        const int4 q = a.e[slot];
        const CtgArgs &c = a.args ? a.args[q.z >> 16] : a.one;
        const double2 r = a.res[slot];
        double *p = c.partials + ((size_t)q.w * c.n_box + (q.z & 0xffff)) * kPartVals;
        p[0] = __dadd_rd(p[0], r.x);
        p[2] = __dadd_ru(p[2], r.y);
    }
}

cudaError_t launch_refine_queue(const RefQueueArgs &a, int num_sms, cudaStream_t s) {
    if (a.n_regions <= 0) return cudaSuccess;
    const size_t smem = (size_t)(a.n_regions + 1) * sizeof(int);
    k_refine_queue<<<num_sms * 4, 256, smem, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_refine_apply<<<(a.n_regions + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}
}  // namespace ibp
