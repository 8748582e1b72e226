// The contingency-flow interval kernel: for every contingency k and line l,
//   c_kl = c_l + L[l,k] c_k,       r_kl = sum_b |Phi[l,b] + L[l,k] Phi[k,b]| r_b
// (Sec. II-C eq. (ctg flow simplified) with H_k = Phi + L[:,k] Phi[k,:], under
// the centre/radius rule of eq. (IBP)), fused with the violation interval of
// eq. (slack-Sc) and the per-warp partial sums of eq. (slack-sagg).
//
// |H_k| is never stored: each CTA owns a tile of BL lines x BK contingencies
// and streams bus chunks of the two PTDF row blocks through shared memory with
// TMA (SWIZZLE_128B, a ring of ST stages guarded by mbarriers), while 8 warps
// hold the tile's LODF entries and radius accumulators in registers.  Persistent launch: one CTA per SM walks the tile
// list with a static stride (deterministic output).
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
// The round-up sum is hierarchical (32 buses per chunk, 8 chunks per level-2
// sum, the rest in level 3) to keep its excess
// small; gamma bounds it.  Eight warps (two per SM sub-partition) leave room
// for 255 registers per thread, so all three levels stay in registers.
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

constexpr int kThreads = kConsumerWarps * 32;

template <int BL, int BK, int ST>
struct SmemLayout {
    static constexpr int CH = 32;  // buses per chunk: one 128-byte swizzled row
    static constexpr int kStageFloats = (BL + BK) * CH;
    static constexpr size_t kRing = (size_t)ST * kStageFloats * sizeof(float);
    // full[ST] mbarriers, arrival counters[ST], last issued chunk[ST], abort flag
    static constexpr size_t kCtl = ST * sizeof(uint64_t) + 2 * ST * sizeof(int) + 16;
    static constexpr size_t kBytes = kRing + kCtl + 1024;
};

// Issue the TMA copies of chunk c (global index within this CTA's tile list).
template <int BL, int BK, int ST>
__device__ __forceinline__ void issue_chunk(const CUtensorMap *mL, const CUtensorMap *mK,
                                            const CtgArgs &a, float *ring, uint64_t *full,
                                            int *last_issued, uint32_t c) {
    using S = SmemLayout<BL, BK, ST>;
    constexpr uint32_t kBytes = (uint32_t)S::kStageFloats * sizeof(float);
    const int s = (int)(c % ST);
    const int ti = (int)(c / (uint32_t)a.n_chunks), ch = (int)(c % (uint32_t)a.n_chunks);
    const int tile = blockIdx.x + ti * gridDim.x;
    const int l0 = (tile % a.tiles_l) * BL, k0 = (tile / a.tiles_l) * BK;
    float *sL = ring + (size_t)s * S::kStageFloats;
    float *sK = sL + BL * S::CH;
    last_issued[s] = (int)c;
    mbar_arrive_expect_tx(smem_addr(&full[s]), kBytes);
    tma_load_2d(smem_addr(sL), mL, smem_addr(&full[s]), ch * S::CH, l0);
    tma_load_2d(smem_addr(sK), mK, smem_addr(&full[s]), ch * S::CH, k0);
}

// ---------------------------------------------------------------------------
// One-box kernel (scaled rows).  Tile BL x BK, thread micro-tile ML x MK with
// lines tl + 16 i and contingencies tk + 16 j.  No dedicated producer warp:
// the warp that releases a stage last (cumulative shared counter) refills it
// with the chunk ST ahead, so no warp waits for "stage empty".
// ---------------------------------------------------------------------------
template <int BL, int BK, int ST>
__global__ void __launch_bounds__(kThreads, 1)
    k_ctg_one(const __grid_constant__ CUtensorMap mL, const __grid_constant__ CUtensorMap mK,
              const CtgArgs a) {
    using S = SmemLayout<BL, BK, ST>;
    constexpr int ML = BL / 16, MK = BK / 16;
    constexpr int CH = S::CH;
    extern __shared__ unsigned char smem_raw[];
    float *ring = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                            ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(ring) + S::kRing);
    int *arrivals = reinterpret_cast<int *>(full + ST);
    int *last_issued = arrivals + ST;
    volatile int *abort_flag = last_issued + ST;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int my_tiles = (a.n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
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
            issue_chunk<BL, BK, ST>(&mL, &mK, a, ring, full, last_issued, c);

    const int tl = (warp >> 1) * 4 + (lane >> 3);
    const int tk = (warp & 1) * 8 + (lane & 7);
    const int xl = tl & 7, xk = tk & 7;  // SWIZZLE_128B: chunk q of row r sits at q ^ (r & 7)
    uint32_t it = 0;
    bool stop = false;
    for (int tile = blockIdx.x; tile < a.n_tiles && !stop; tile += gridDim.x) {
        const int l0 = (tile % a.tiles_l) * BL, k0 = (tile / a.tiles_l) * BK;
        float Lr[ML][MK];
#pragma unroll
        for (int i = 0; i < ML; ++i)
#pragma unroll
            for (int j = 0; j < MK; ++j) {
                const int l = l0 + tl + 16 * i, k = k0 + tk + 16 * j;
                Lr[i][j] = (l < a.n_l && k < a.n_c) ? __ldg(&a.lodf[(size_t)k * a.n_l + l]) : 0.0f;
            }
        float acc1[ML][MK], acc2[ML][MK], acc3[ML][MK];
#pragma unroll
        for (int i = 0; i < ML; ++i)
#pragma unroll
            for (int j = 0; j < MK; ++j) acc1[i][j] = acc2[i][j] = acc3[i][j] = 0.0f;

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
#pragma unroll
            for (int q = 0; q < CH / 4; ++q) {
                float4 fk[MK];
                const int ok4 = (q ^ xk) << 2, ol4 = (q ^ xl) << 2;
#pragma unroll
                for (int j = 0; j < MK; ++j)
                    fk[j] = *reinterpret_cast<const float4 *>(sK + (tk + 16 * j) * CH + ok4);
#pragma unroll
                for (int i = 0; i < ML; ++i) {
                    const float4 fl = *reinterpret_cast<const float4 *>(sL + (tl + 16 * i) * CH + ol4);
#pragma unroll
                    for (int j = 0; j < MK; ++j) {
                        const float L = Lr[i][j];
                        float h;
                        h = __fmaf_rn(L, fk[j].x, fl.x);
                        acc1[i][j] = __fadd_ru(acc1[i][j], fabsf(h));
                        h = __fmaf_rn(L, fk[j].y, fl.y);
                        acc1[i][j] = __fadd_ru(acc1[i][j], fabsf(h));
                        h = __fmaf_rn(L, fk[j].z, fl.z);
                        acc1[i][j] = __fadd_ru(acc1[i][j], fabsf(h));
                        h = __fmaf_rn(L, fk[j].w, fl.w);
                        acc1[i][j] = __fadd_ru(acc1[i][j], fabsf(h));
                    }
                }
            }
            __syncwarp();
            if (lane == 0) {
                // release the stage; the last of the 8 warps refills it
                __threadfence_block();
                const int old = atomicAdd(&arrivals[s], 1);
                if (old == (int)(it / ST) * kConsumerWarps + kConsumerWarps - 1) {
                    const uint32_t nxt = it + ST;
                    if (nxt < total && !*abort_flag) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        issue_chunk<BL, BK, ST>(&mL, &mK, a, ring, full, last_issued, nxt);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < ML; ++i)
#pragma unroll
                for (int j = 0; j < MK; ++j) {
                    acc2[i][j] = __fadd_ru(acc2[i][j], acc1[i][j]);
                    acc1[i][j] = 0.0f;
                }
            if ((ch & 7) == 7) {
#pragma unroll
                for (int i = 0; i < ML; ++i)
#pragma unroll
                    for (int j = 0; j < MK; ++j) {
                        acc3[i][j] = __fadd_ru(acc3[i][j], acc2[i][j]);
                        acc2[i][j] = 0.0f;
                    }
            }
        }
        if (stop) break;
        float slo = 0.0f, shi = 0.0f, w = 0.0f;
#pragma unroll
        for (int i = 0; i < ML; ++i)
#pragma unroll
            for (int j = 0; j < MK; ++j) {
                const int l = l0 + tl + 16 * i, k = k0 + tk + 16 * j;
                if (l < a.n_l && k < a.n_c) {
                    const float A = __fadd_ru(acc3[i][j], acc2[i][j]);
                    pair_epilogue(a, 0, l, k, Lr[i][j], A, slo, shi, w);
                }
            }
        write_warp_partials(a, tile, warp, 0, slo, shi, w);
    }
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
// Variant table and launcher
// ---------------------------------------------------------------------------
static const CtgVariant kVariants[] = {
    {1, 0, 128, 64, 32, 4, 1, "one-box 128x64 st4"},
    {2, 0, 128, 64, 32, 6, 1, "one-box 128x64 st6"},
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

template <int BL, int BK, int ST>
static cudaError_t launch_one(const CUtensorMap &mL, const CUtensorMap &mK, const CtgArgs &a,
                              int grid, cudaStream_t s) {
    using S = SmemLayout<BL, BK, ST>;
    auto kern = k_ctg_one<BL, BK, ST>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S::kBytes);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    if (fa.maxThreadsPerBlock < kThreads) {
        fprintf(stderr, "k_ctg_one: %d registers allow only %d threads per block (need %d)\n",
                fa.numRegs, fa.maxThreadsPerBlock, kThreads);
        return cudaErrorLaunchOutOfResources;
    }
    kern<<<grid, kThreads, S::kBytes, s>>>(mL, mK, a);
    return cudaGetLastError();
}

cudaError_t launch_ctg(const CtgVariant &v, const CUtensorMap &mL, const CUtensorMap &mK,
                       const CtgArgs &a, int grid, cudaStream_t s) {
    if (a.n_tiles <= 0) return cudaSuccess;
    grid = std::min(grid, a.n_tiles);
    switch (v.id) {
    case 1: return launch_one<128, 64, 4>(mL, mK, a, grid, s);
    case 2: return launch_one<128, 64, 6>(mL, mK, a, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ibp
