// Per-pair epilogue of the contingency kernels: the certified flow interval
// of one (k, l) pair from its round-up radius sum, the violation interval of
// eq. (slack-Sc), and the per-warp FP64 partial sums of eq. (slack-sagg).
#pragma once

#include "common.cuh"
#include "internal.h"
#include "refine.cuh"

namespace ibp {

constexpr int kConsumerWarps = 8;

// Centre of the post-contingency flow in FP32 and a bound on its distance from
// the exact centre c_l + L[l,k] c_k of the FP64 data:
//   e_c = e_l + |L|(e_k (1 + 3u) + 2u|c_k|) + 2u|c| + eta_c (1 + |L|).
__device__ __forceinline__ void pair_centre(float Lt, float cl, float ck, float el, float ek,
                                            float eta_c, float one_l, float &c, float &ec) {
    c = __fmaf_rn(Lt, ck, cl);
    ec = __fmaf_ru(2.0f * kU, fabsf(ck), __fmul_ru(ek, 1.0000002f));
    ec = __fmaf_ru(fabsf(Lt), ec, el);
    ec = __fmaf_ru(2.0f * kU, fabsf(c), ec);
    ec = __fmaf_ru(eta_c, one_l, ec);
}

// The per-line inputs of a pair's epilogue (line l, box): base centre, its
// error bound, base radius sum, contingency ratings rounded up and down.
struct LineIn {
    float c, e, R, rup, rdn;
};
// ... and of its contingency k: the outaged line kl and its c, e, R.
struct CtgIn {
    int kl;
    float c, e, R;
};

__device__ __forceinline__ LineIn load_line_in(const CtgArgs &a, int box, int l) {
    const size_t o = (size_t)box * a.n_l + l;
    return LineIn{__ldg(&a.line_c[o]), __ldg(&a.line_e[o]), __ldg(&a.line_R[o]), __ldg(&a.rate_up[l]),
                  __ldg(&a.rate_dn[l])};
}
__device__ __forceinline__ CtgIn load_ctg_in(const CtgArgs &a, int box, int k) {
    const int kl = __ldg(&a.ctg_line[k]);
    if (!IBP_IDX_OK(kl >= 0 && kl < a.n_l && box < a.n_box, a.err)) return CtgIn{-1, 0.0f, 0.0f, 0.0f};
    const size_t o = (size_t)box * a.n_l + kl;
    return CtgIn{kl, __ldg(&a.line_c[o]), __ldg(&a.line_e[o]), __ldg(&a.line_R[o])};
}

// Epilogue for one (k, l) pair from its loaded inputs: flow interval,
// violation interval, error term.  Returns true when the pair's lower
// violation bound can be positive and the FP64 refinement is on
// (a.ref.phi64): its obj_hi terms (s_lo and the allowance) then go to
// cslo_acc / cwhi_acc, which the caller adds only when the pair is not queued
// for the refinement; its obj_lo terms are added here.
__device__ __forceinline__ bool pair_epilogue_in(const CtgArgs &a, int box, int l, int k, float Lt,
                                                 float A, const LineIn &li, const CtgIn &ci,
                                                 float eta_r, float eta_c, float &slo_acc,
                                                 float &shi_acc, float &whi_acc, float &wlo_acc,
                                                 float &cslo_acc, float &cwhi_acc) {
    const int kl = ci.kl;
    if (!IBP_IDX_OK(kl >= 0 && kl < a.n_l && l >= 0 && l < a.n_l && box < a.n_box, a.err)) return false;
    bool refine = false;
    const float cl = li.c, ck = ci.c, el = li.e, ek = ci.e, Rl = li.R, Rk = ci.R;
    const float aL = fabsf(Lt);
    float flo, fhi, slo, shi, whi, wlo;
    if (l == kl) {
        // the outaged line carries exactly nothing (L[k,k] = -1, like M_k)
        flo = fhi = 0.0f;
        slo = shi = whi = wlo = 0.0f;
    } else {
        const float one_l = __fadd_ru(1.0f, aL);
        const float eta = __fmul_ru(eta_r, one_l);
        const float m = __fmaf_ru(aL, Rk, Rl);
        float rbar = __fmaf_ru(A, kU, A);
        rbar = __fmaf_ru(4.0f * kU, m, rbar);
        rbar = __fadd_ru(rbar, eta);
        float c, ec;
        pair_centre(Lt, cl, ck, el, ek, eta_c, one_l, c, ec);
        const float rho = __fadd_ru(rbar, ec);
        flo = __fsub_rd(c, rho);
        fhi = __fadd_ru(c, rho);
        float alo, ahi;
        abs_interval(flo, fhi, alo, ahi);
        const float rup = li.rup, rdn = li.rdn;
        slo = fmax0(__fsub_rd(alo, rup));
        shi = fmax0(__fsub_ru(ahi, rdn));
        whi = wlo = 0.0f;
        if (shi > 0.0f) {
            // |s - s_exact| <= w = (rbar - r_exact) + 2 ec + u rating for both
            // ends; s_hi is exact where it is 0, s_lo where alo - rating + w <= 0
            float w = __fmaf_ru(a.gamma + 3.0f * kU, A, __fmaf_ru(8.0f * kU, m, 0.0f));
            w = __fmaf_ru(2.0f, ec, w);
            w = __fmaf_ru(kU, rup, w);
            w = __fmaf_ru(2.0f, eta, w);
            wlo = w;
            if (__fadd_ru(__fsub_ru(alo, rdn), w) > 0.0f) {
                whi = w;
                refine = a.ref.phi64 != nullptr;
            }
        }
        if (a.act_list_lo && shi > 0.0f) {
            // upper violation bound positive: obj_lo's active set
            const int idx = atomicAdd(&a.act_count_lo[box], 1);
            if (idx < a.act_cap_lo)
                a.act_list_lo[(size_t)box * a.act_cap_lo + idx] =
                    make_int4(l, kl, __float_as_int(Lt), __float_as_int(c > 0.0f ? 1.0f : -1.0f));
            else
                atomicOr(a.err, kErrOverflow);
        }
        if (a.act_list && slo > 0.0f) {
            // certified active: record for the adjoint
            const int idx = atomicAdd(&a.act_count[box], 1);
            if (idx < a.act_cap)
                a.act_list[(size_t)box * a.act_cap + idx] =
                    make_int4(l, kl, __float_as_int(Lt), __float_as_int(c > 0.0f ? 1.0f : -1.0f));
            else
                atomicOr(a.err, kErrOverflow);
        }
    }
    if (a.flow_lo) {
        const size_t o = ((size_t)box * a.n_c + k) * a.n_l + l;
        a.flow_lo[o] = flo;
        a.flow_hi[o] = fhi;
    }
    if (refine) {
        cslo_acc = __fadd_rd(cslo_acc, slo);
        cwhi_acc = __fadd_ru(cwhi_acc, whi);
    } else {
        slo_acc = __fadd_rd(slo_acc, slo);
        whi_acc = __fadd_ru(whi_acc, whi);
    }
    shi_acc = __fadd_ru(shi_acc, shi);
    wlo_acc = __fadd_ru(wlo_acc, wlo);
    return refine;
}

// The same with its inputs loaded here.
__device__ __forceinline__ bool pair_epilogue(const CtgArgs &a, int box, int l, int k, float Lt,
                                              float A, float &slo_acc, float &shi_acc,
                                              float &whi_acc, float &wlo_acc, float &cslo_acc,
                                              float &cwhi_acc) {
    const float *bc = a.box_consts + (size_t)box * 4;
    const CtgIn ci = load_ctg_in(a, box, k);
    if (ci.kl < 0 || !IBP_IDX_OK(l >= 0 && l < a.n_l, a.err)) return false;
    return pair_epilogue_in(a, box, l, k, Lt, A, load_line_in(a, box, l), ci, __ldg(&bc[0]), __ldg(&bc[1]),
                            slo_acc, shi_acc, whi_acc, wlo_acc, cslo_acc, cwhi_acc);
}

// The one-box kernel calls the epilogue out of line: its 16 pairs per thread
// inlined raise the kernel's register pressure in the main loop (measured: the
// contingency kernel takes 0.9% less time this way on mesh8316, while the
// many-box kernel, at 255 registers, is 3.4% slower with the call).  The
// caller loads every pair's inputs first: two rounds of independent loads per
// tile instead of two dependent loads in each call.
static __device__ __noinline__ bool pair_epilogue_call(const CtgArgs &a, int box, int l, int k, float Lt,
                                                       float A, LineIn li, CtgIn ci,
                                                       float eta_r, float eta_c, float &slo_acc,
                                                       float &shi_acc, float &whi_acc, float &wlo_acc,
                                                       float &cslo_acc, float &cwhi_acc) {
    return pair_epilogue_in(a, box, l, k, Lt, A, li, ci, eta_r, eta_c, slo_acc, shi_acc, whi_acc, wlo_acc,
                            cslo_acc, cwhi_acc);
}

// Per-warp FP64 partial sums (deterministic order, directed rounding):
// {sum s_lo (down), sum s_hi (up), error allowance of obj_hi, of obj_lo}.
// partial-sum rows per tile: at most the largest warp count of any kernel
constexpr int kPartRowsPerTile = 16;

// n_terms: violations the thread summed into slo / shi in FP32 (directed);
// those sums are within 2u n_terms of the exact sums, which the error
// allowances take on here.
__device__ __forceinline__ void write_warp_partials(const CtgArgs &a, int tile, int warp, int box,
                                                    float slo, float shi, float whi, float wlo,
                                                    int n_terms) {
    const int lane = threadIdx.x & 31;
    const float g = 2.02f * kU * (float)n_terms;
    whi = __fmaf_ru(g, slo, whi);  // obj_hi takes sum s_lo
    wlo = __fmaf_ru(g, shi, wlo);  // obj_lo takes sum s_hi
    // sum s_lo rounded down as minus the round-up sum of -s_lo
    const double d = warp_sum4_ru(-(double)slo, (double)shi, (double)whi, (double)wlo);
    const int q = (lane >> 3) & 3;  // the value this lane holds the total of
    if ((lane & 7) == 0 &&
        IBP_IDX_OK(a.part_rows_cap <= 0 || tile * a.warps_per_tile + warp < a.part_rows_cap, a.err)) {
        double *p = a.partials + (((size_t)tile * a.warps_per_tile + warp) * a.n_box + box) * kPartVals;
        p[q] = q == 0 ? -d : d;
    }
}

}  // namespace ibp
