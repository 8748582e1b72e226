// FP64 refinement of the violation terms that can reach obj_hi.
//
// obj_hi takes -z_f s_lo for every pair, s_lo = max(|c| - r - rating, 0)
// (eqs. (slack-sfb), (slack-Sc) under eq. (IBP)).  Only the pairs whose lower
// violation bound can be positive contribute, and on the workloads here they
// are a few per ten thousand.  The FP32 kernels bound each of them with
// allowances of a few tens of u32 of the flow's magnitude: the stored PTDF and
// LODF are FP32, and the radius is a round-up sum.  So the kernels hand those
// pairs to this code instead.  A warp recomputes the pair's flow interval from
// the FP64 sensitivities -- the FP64 PTDF of the active columns, and the LODF
// as its FP32 copy plus the FP32 remainder, L = L~ + L_lo to 2^-48 |L| and
// 2^-150 -- and the FP64 bus intervals, with FP64 sums and an explicit error
// bound E:
//   h_b = Phi_l,b + L Phi_k,b,  r = sum_b |h_b| r_b (round-up),
//   c = sum_b h_b c_b,  rho = RU(r + E),
//   s_lo = max(RD(|[c - rho, c + rho]|_lo - rating), 0),
//   E = u64 r + (n + 2) u64 X + e_L X_k + 2^-119 (1 + |L|)(1 + e_L) (sum r + sum |c|),
// with e_L = 2^-47 |L| + 2^-149 the LODF's bound, X_x = (1 + 2^-20)
// sum_b |Phi~_x,b| (r_b + |c_b|) (FP32 round-up from the FP32 PTDF, whose
// entries exceed |Phi| / (1 + 2^-22) or were flushed below 2^-120: the last
// term), X = X_l + |L| X_k, and n the number of FP64 roundings along one sum.
// The refined s_lo is a lower bound of the exact one (sound for obj_hi), and
// the two differ by at most w = 2E + 4 u64 (r + |c| + rating), which goes into
// obj_err.
//
// The contingency kernels do not refine inside their tile loop, where one warp
// would hold up its CTA's shared TMA ring: each warp queues its tile's
// candidates (all of a tile's or none, so the result does not depend on
// timing; a full queue leaves the tile's terms to the FP32 path, which is
// certified too).  With global queues (the library's bound calls) a separate
// launch refines every queued pair with one warp anywhere on the GPU and then
// adds each warp-queue's results to their partial-sum rows in queue order;
// with a shared-memory queue (the entry point without allocation) the warp
// refines its own queue after its last tile.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace ibp {

constexpr double kU64 = 1.1102230246251565e-16;   // 2^-53
constexpr double kU32d = 5.9604644775390625e-08;  // 2^-24
constexpr double k2m20p = 1.0000009536743164;     // 1 + 2^-20
constexpr double k2m47 = 7.105427357601002e-15;   // 2^-47
constexpr double k2m119 = 1.5046327690525280e-36; // 2^-119
constexpr double k2m149 = 1.4012984643248171e-45; // 2^-149

// kinds of refined terms
constexpr int kRefPair = 0;   // contingency pair, H = Phi_l + L Phi_k (tight rule)
constexpr int kRefLine = 1;   // base line or bridge line, H = Phi_l

struct RefOut {
    double s_lo;  // refined lower violation bound (rounded down)
    double w;     // bound on its distance from the exact value (rounded up)
    double c;     // refined flow centre
};

// The FP64 LODF entry L~[k][l] + L_lo[k][l] and the bound on its distance from
// L (k < 0 or no remainder: the FP32 entry and its rounding bound).
__device__ __forceinline__ double ref_lodf(const RefArgs &r, int k, int l, float Lt, double &eL) {
    if (k >= 0 && r.lodf_lo) {
        const double L = (double)Lt + (double)__ldg(&r.lodf_lo[(size_t)k * r.n_l + l]);
        eL = __fma_ru(k2m47, fabs(L), k2m149);
        return L;
    }
    eL = __fma_ru(1.0001 * kU32d, fabs((double)Lt), k2m119);
    return (double)Lt;
}

// FP64 roundings along one sum of n_a_pad columns spread over a warp (4
// columns per lane step and 5 butterfly levels), plus the product and the
// entry of the sum
__device__ __forceinline__ double ref_nu(int n_a_pad) {
    const int steps = ((n_a_pad >> 2) + 31) >> 5;
    return __dmul_ru((double)(4 * steps + 8), kU64);
}

// The error bound E of the refinement (see the top of the file); S the
// round-up radius sum, Xl, Xk the FP32 sums, aL = |L|, tot = sum r + sum |c|.
__device__ __forceinline__ double ref_bound(int n_a_pad, double S, float Xl, float Xk, double aL,
                                            double eL, double tot) {
    const double X = __dmul_ru(k2m20p, __fma_ru(aL, (double)Xk, (double)Xl));
    double E = __dmul_ru(__dadd_ru(ref_nu(n_a_pad), 2.0 * kU64), X);
    E = __fma_ru(__dmul_ru(eL, k2m20p), (double)Xk, E);
    E = __fma_ru(__dmul_ru(k2m119, __dmul_ru(__dadd_ru(1.0, aL), __dadd_ru(1.0, eL))), tot, E);
    return __fma_ru(kU64, S, E);
}

// Warp-cooperative: every lane of the warp calls it with the same arguments and
// gets the same result.  l: line; kl: the outaged line and k its contingency
// index (ignored for kRefLine); Lt: the FP32 LODF entry L~[k][l]; rating: the
// FP64 rating the term uses.
static __device__ __noinline__ RefOut refine_term(const RefArgs r, int box, int l, int kl, int k,
                                                  float Lt, double rating, int kind) {
    const int lane = threadIdx.x & 31;
    const int nv = r.n_a_pad >> 2;
    const size_t ob = (size_t)box * r.n_a_pad;
    const bool two = kind != kRefLine;
    const int k_row = two ? kl : l;
    const double2 *pl64 = reinterpret_cast<const double2 *>(r.phi64 + (size_t)l * r.n_a_pad);
    const double2 *pk64 = reinterpret_cast<const double2 *>(r.phi64 + (size_t)k_row * r.n_a_pad);
    const float4 *pl32 = reinterpret_cast<const float4 *>(r.phi_hi + (size_t)l * r.n_a_pad);
    const float4 *pk32 = reinterpret_cast<const float4 *>(r.phi_hi + (size_t)k_row * r.n_a_pad);
    const double2 *cb = reinterpret_cast<const double2 *>(r.cbus + ob);
    const double2 *rb = reinterpret_cast<const double2 *>(r.rbus64 + ob);
    const float4 *r32 = reinterpret_cast<const float4 *>(r.rbus + ob);
    const float4 *c32 = reinterpret_cast<const float4 *>(r.cabs + ob);
    double eL = 0.0;
    const double L = two ? ref_lodf(r, k, l, Lt, eL) : 0.0;
    double S = 0.0, C = 0.0;
    float Xl = 0.0f, Xk = 0.0f;
    auto col = [&](double pl, double pk, float al, float ak, double c, double rr, float rc) {
        Xl = __fmaf_ru(al, rc, Xl);
        double h = pl;
        if (two) {
            Xk = __fmaf_ru(ak, rc, Xk);
            h = fma(L, pk, pl);
        }
        S = __fma_ru(fabs(h), rr, S);
        C = fma(h, c, C);
    };
    for (int v = lane; v < nv; v += 32) {
        const double2 l01 = __ldg(&pl64[2 * v]), l23 = __ldg(&pl64[2 * v + 1]);
        const float4 a = __ldg(&pl32[v]);
        double2 k01 = make_double2(0.0, 0.0), k23 = k01;
        float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
        if (two) {
            k01 = __ldg(&pk64[2 * v]);
            k23 = __ldg(&pk64[2 * v + 1]);
            b = __ldg(&pk32[v]);
        }
        const double2 c01 = __ldg(&cb[2 * v]), c23 = __ldg(&cb[2 * v + 1]);
        const double2 r01 = __ldg(&rb[2 * v]), r23 = __ldg(&rb[2 * v + 1]);
        const float4 q = __ldg(&r32[v]), ca = __ldg(&c32[v]);
        col(l01.x, k01.x, fabsf(a.x), fabsf(b.x), c01.x, r01.x, __fadd_ru(q.x, ca.x));
        col(l01.y, k01.y, fabsf(a.y), fabsf(b.y), c01.y, r01.y, __fadd_ru(q.y, ca.y));
        col(l23.x, k23.x, fabsf(a.z), fabsf(b.z), c23.x, r23.x, __fadd_ru(q.z, ca.z));
        col(l23.y, k23.y, fabsf(a.w), fabsf(b.w), c23.y, r23.y, __fadd_ru(q.w, ca.w));
    }
    // butterfly sums: every lane ends with the same value (IEEE addition commutes)
    S = warp_sum_ru(S);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) C += __shfl_xor_sync(0xffffffffu, C, o);
    Xl = warp_sum_ru_f(Xl);
    Xk = warp_sum_ru_f(Xk);
    const float *bc = r.box_consts + (size_t)box * 4;
    const double tot = __dadd_ru((double)__ldg(&bc[2]), (double)__ldg(&bc[3]));
    const double E = ref_bound(r.n_a_pad, S, Xl, Xk, fabs(L), eL, tot);
    const double rho = __dadd_ru(S, E);
    const double lo = __dsub_rd(C, rho), hi = __dadd_ru(C, rho);
    const double alo = lo >= 0.0 ? lo : (hi <= 0.0 ? -hi : 0.0);
    RefOut out;
    out.s_lo = fmax(__dsub_rd(alo, rating), 0.0);
    out.w = __fma_ru(4.0 * kU64, __dadd_ru(__dadd_ru(S, fabs(C)), rating), __dmul_ru(2.0, E));
    out.c = C;
    return out;
}

// ------------------------------------------------------------ candidate queue
constexpr int kRefQueue = 64;  // entries per warp of a shared-memory queue

// Per-warp queue: its count (in shared memory) and its entries (l, k,
// case << 16 | box, partial-sum row), in shared memory (drained by the kernel
// itself) or in the global region of the warp (refined by k_refine_queue).
struct RefQueue {
    int *count;
    int4 *e;
    int cap;
};

// 32 counts (16 bytes apart) at `base`; entries after them (shared queue) or
// in the call's global regions (g_e: region (blockIdx.x, warp) of a launch
// with `warps` warps per CTA).
__device__ __forceinline__ RefQueue ref_queue_of(void *base, int warp, int4 *g_e = nullptr,
                                                 int g_cap = 0, int warps = 0) {
    RefQueue q;
    q.count = reinterpret_cast<int *>(base) + 4 * warp;
    if (g_e) {
        q.e = g_e + ((size_t)blockIdx.x * warps + warp) * g_cap;
        q.cap = g_cap;
    } else {
        q.e = reinterpret_cast<int4 *>(base) + 32 + (size_t)warp * kRefQueue;
        q.cap = kRefQueue;
    }
    return q;
}
// shared bytes of the queues of n_warps warps (n_warps <= 32): the counts,
// and the entries unless the queues are global
constexpr size_t ref_queue_bytes(int n_warps) { return 16 * 32 + (size_t)n_warps * kRefQueue * 16; }

__device__ __forceinline__ void ref_queue_init(RefQueue q) {
    if ((threadIdx.x & 31) == 0) *q.count = 0;
    __syncwarp();
}

// Queues every candidate of the warp's tile (bit q of a lane: its q-th pair,
// get(q, l, k) its line and contingency index), in the order q ascending, then
// lane ascending -- or none of them when they do not all fit.  Returns whether
// they were queued (the same in every lane).
template <int NQ, class Get>
__device__ __forceinline__ bool ref_enqueue(RefQueue q, uint64_t mask, Get get, int case_box, int row) {
    const int lane = threadIdx.x & 31;
    const int tot = __reduce_add_sync(0xffffffffu, (unsigned)__popcll(mask));
    if (tot == 0) return true;
    __syncwarp();
    int pos = *q.count;
    if (pos + tot > q.cap) return false;
#pragma unroll 1
    for (int qq = 0; qq < NQ; ++qq) {
        const uint32_t m = __ballot_sync(0xffffffffu, (unsigned)((mask >> qq) & 1u));
        if (!m) continue;
        if ((mask >> qq) & 1u) {
            int l = 0, k = 0;
            get(qq, l, k);
            q.e[pos + __popc(m & ((1u << lane) - 1u))] = make_int4(l, k, case_box, row);
        }
        pos += __popc(m);
    }
    __syncwarp();
    if (lane == 0) *q.count = pos;
    __syncwarp();
    return true;
}

// End of a contingency kernel: a global queue publishes its count for
// k_refine_queue; a shared queue is refined here, in queue order, and each
// refined s_lo (rounded down) and allowance (rounded up) is added to its
// partial-sum row, which the same lane wrote before.  args_of(case) gives the
// pair's case arguments.
template <class ArgsOf>
__device__ __forceinline__ void ref_finish(RefQueue q, int *g_cnt, int warps, ArgsOf args_of) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    const int n = *q.count;
    if (g_cnt) {
        if (lane == 0) g_cnt[(size_t)blockIdx.x * warps + (threadIdx.x >> 5)] = n;
        return;
    }
#pragma unroll 1
    for (int i = 0; i < n; ++i) {
        const int4 t = q.e[i];
        const CtgArgs &a = args_of(t.z >> 16);
        const int box = t.z & 0xffff;
        const int kl = __ldg(&a.ctg_line[t.y]);
        const float Lt = __ldg(&a.lodf[(size_t)t.y * a.n_l + t.x]);
        const RefOut o =
            refine_term(a.ref, box, t.x, kl, t.y, Lt, __ldg(&a.ref.rate_c64[t.x]), kRefPair);
        if (lane == 0) {
            double *p = a.partials + ((size_t)t.w * a.n_box + box) * kPartVals;
            p[0] = __dadd_rd(p[0], o.s_lo);
            p[2] = __dadd_ru(p[2], o.w);
        }
    }
}

}  // namespace ibp
