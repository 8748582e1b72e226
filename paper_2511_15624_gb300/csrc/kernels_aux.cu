// Box-to-bus, base-flow, objective-assembly and case-build kernels.
//
// Rounding: every quantity that enters a certified bound is computed with
// directed rounding (round-up for upper bounds, round-down for lower bounds)
// or carries an explicit error term; see the comment of each kernel.
#include "common.cuh"
#include "internal.h"
#include "refine.cuh"

#include <cfloat>

namespace ibp {

// ---------------------------------------------------------------------------
// Box -> bus injection intervals.  IBP of p_inj = N_g p_g - N_d p_d
// (Sec. II-A under eq. (IBP)): bus b lies in [P_lo, P_hi] with
//   P_lo = sum_{g@b} lo_g - sum_{d@b} hi_d,  P_hi = sum_{g@b} hi_g - sum_{d@b} lo_d
// (rounded down / up).  The centre c = (P_lo + P_hi)/2 may round; the radius
// r = max(P_hi - c, c - P_lo) is rounded up, so [c - r, c + r] contains the
// interval whatever c is.  Block (b, j) takes the columns b*256 + t +
// k*(gridDim.x*256) of box j; the per-box sums of r and |c| are round-up sums
// in a fixed order (blocks, then k_bus_consts over the blocks when there are
// several).
// ---------------------------------------------------------------------------
// round-up sums of r and |c| and the bad-box flag -> the box constants
__device__ __forceinline__ void write_box_consts(const BusArgs &a, int j, float R, float C, int B) {
    // Absolute error allowances for FP32 underflow (entries of Phi and L
    // below 2^-120 are stored as 0; products may be subnormal):
    //   eta_r covers sum_b |dPhi| r_b and per-term subnormal rounding,
    //   eta_c covers sum_b |dPhi| |c_b|.
    const float t120 = 7.52316384526264e-37f;   // 2^-120
    const float t99 = 1.5777218104420236e-30f;  // 2^-99
    float *bc = a.box_consts + (size_t)j * 4;
    bc[0] = __fadd_ru(__fmul_ru(t99, R), __fmul_ru(t120, (float)a.n_a));
    bc[1] = __fmul_ru(t99, C);
    bc[2] = R;
    bc[3] = C;
    if (B) atomicOr(a.err, kErrBadBox);
}

__global__ void __launch_bounds__(256) k_bus(BusArgs a) {
    const int j = blockIdx.y;
    const int first = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    const double *lo = a.box_lo + (size_t)j * a.n_dev;
    const double *hi = a.box_hi + (size_t)j * a.n_dev;
    float rsum = 0.0f, csum = 0.0f;
    int bad = 0;
    for (int d = first; d < a.n_dev; d += stride) {
        const double x = lo[d], y = hi[d];
        if (!(x <= y) || !isfinite(x) || !isfinite(y)) bad = 1;
    }
    for (int col = first; col < a.n_a_pad; col += stride) {
        double c = 0.0, rd64 = 0.0;
        float r32 = 0.0f, ca = 0.0f;
        if (col < a.n_a) {
            double plo = 0.0, phi = 0.0;
            for (int p = a.act_ptr[col]; p < a.act_ptr[col + 1]; ++p) {
                const int d = a.act_dev[p];
                if (d < a.n_gen) {
                    plo = __dadd_rd(plo, lo[d]);
                    phi = __dadd_ru(phi, hi[d]);
                } else {
                    plo = __dadd_rd(plo, -hi[d]);
                    phi = __dadd_ru(phi, -lo[d]);
                }
            }
            c = 0.5 * (plo + phi);
            const double r = fmax(__dadd_ru(phi, -c), __dadd_ru(c, -plo));
            rd64 = fmax(r, 0.0);
            r32 = __double2float_ru(rd64);
            ca = __double2float_ru(fabs(c));
        }
        a.cbus[(size_t)j * a.n_a_pad + col] = c;
        if (a.cbus2) {
            const float ch = __double2float_rn(c);
            a.cbus2[(size_t)j * a.n_a_pad + col] = make_float2(ch, __double2float_rn(c - (double)ch));
        }
        a.rbus[(size_t)j * a.n_a_pad + col] = r32;
        if (a.rbus64) a.rbus64[(size_t)j * a.n_a_pad + col] = rd64;
        a.cabs[(size_t)j * a.n_a_pad + col] = ca;
        if (a.rbus_t) a.rbus_t[(size_t)col * a.n_box_pad + j] = r32;
        rsum = __fadd_ru(rsum, r32);
        csum = __fadd_ru(csum, ca);
    }
    __shared__ float sr[8], sc[8];
    __shared__ int sbad[8];
    rsum = warp_sum_ru_f(rsum);
    csum = warp_sum_ru_f(csum);
    bad = __any_sync(0xffffffffu, bad);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sr[w] = rsum;
        sc[w] = csum;
        sbad[w] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float R = 0.0f, C = 0.0f;
        int B = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            R = __fadd_ru(R, sr[i]);
            C = __fadd_ru(C, sc[i]);
            B |= sbad[i];
        }
        if (gridDim.x == 1) {
            write_box_consts(a, j, R, C, B);
        } else {
            float *q = a.bus_part + ((size_t)j * gridDim.x + blockIdx.x) * 4;
            q[0] = R;
            q[1] = C;
            q[2] = B ? 1.0f : 0.0f;
        }
    }
}

// the blocks' sums of box j, in block order
__global__ void k_bus_consts(BusArgs a, int n_blocks) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.n_box) return;
    float R = 0.0f, C = 0.0f;
    int B = 0;
    for (int b = 0; b < n_blocks; ++b) {
        const float *q = a.bus_part + ((size_t)j * n_blocks + b) * 4;
        R = __fadd_ru(R, q[0]);
        C = __fadd_ru(C, q[1]);
        B |= q[2] != 0.0f;
    }
    write_box_consts(a, j, R, C, B);
}

cudaError_t launch_bus(const BusArgs &a, cudaStream_t s) {
    const int nb = a.bus_part ? bus_blocks(a.n_a_pad) : 1;
    k_bus<<<dim3(nb, a.n_box), 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || nb == 1) return e;
    k_bus_consts<<<(a.n_box + 127) / 128, 128, 0, s>>>(a, nb);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Base-case flows, one warp per line (eq. (line flow ptdf) under eq. (IBP)).
// For line l and box j:
//   centre   c_l = sum_b Phi~[l,b] c_b       FP64 accumulation (or the
//                                            compensated FP32 sums of
//                                            k_base_ff), then FP32 RN
//   C_l          = sum_b |Phi~[l,b]| |c_b|   FP32 round-up
//   R_l          = sum_b |Phi~[l,b]| r_b     FP32 round-up
// Phi~ is the FP32 copy of the FP64 PTDF (|Phi - Phi~| <= u |Phi~| + 2^-120),
// so the exact centre from the FP64 data is within
//   e_l = 2.1 u C_l + eta_c
// of the FP32 centre (storage u(1+u) C_l, FP64 sum <= 1e-12 C_l, final RN
// u |c_l|), and the exact radius is at most (1 + u) R_l + eta_r.
// The violation interval of eq. (slack-sfb) follows; its lower/upper ends
// and an error allowance are summed per warp into partials (FP64 directed).
// Rows n_l .. n_l + n_c - 1 (one-box mode only) write the scaled rows
// hat_k[k] = RN(Phi~[ctg_line[k], b] r_b) used by the contingency kernel;
// line rows write hat_l[l] likewise when hat_l is given (unscreened calls; the
// line screen writes the rows of the lines it keeps).
// ---------------------------------------------------------------------------
constexpr int kBaseWarps = 8;

int base_partials_count(int num_sms) { return num_sms * 2 * kBaseWarps; }

// Per (line, box) epilogue of the base flows: certified interval, violation
// interval of eq. (slack-sfb), error allowance, active-set recording and, for
// bridge lines, their n_c contingency pairs in closed form.  c = FP32 centre,
// C, R = round-up sums of |Phi~||c_b| and |Phi~| r_b.  Every lane of the warp
// calls it with the same values; `writer` (one lane) stores the results.  With
// the FP64 refinement on (a.ref.phi64), a base term whose lower violation
// bound can be positive is left out of the partial sums and bit 0 of the
// result is set; bit 1 likewise for the bridge's contingency pairs.
__device__ __forceinline__ int base_epilogue(const BaseArgs &a, int l, int j, float c, float C,
                                             float R, double *part, bool writer) {
    const bool refine = a.ref.phi64 != nullptr;
    int flags = 0;
    const float *bc = a.box_consts + (size_t)j * 4;
    const float eta_r = bc[0], eta_c = bc[1];
    const float e = __fadd_ru(__fmul_ru(2.1f * kU, C), eta_c);
    const float rbar = __fadd_ru(__fmaf_ru(R, kU, R), eta_r);
    const float rho = __fadd_ru(rbar, e);
    const float flo = __fsub_rd(c, rho), fhi = __fadd_ru(c, rho);
    float alo, ahi;
    abs_interval(flo, fhi, alo, ahi);
    const float slo_f = fmax0(__fsub_rd(alo, a.rate_up[l]));
    float slo = slo_f;
    const float shi = fmax0(__fsub_ru(ahi, a.rate_dn[l]));
    float whi = 0.0f, wlo = 0.0f;
    if (shi > 0.0f) {
        // |s - s_exact| <= w = (rbar - R_exact) + 2 e + u rating; s_lo is
        // exact where alo - rating + w <= 0
        const float w = __fmaf_ru(a.gamma_base + 3.0f * kU, R,
                                  __fmaf_ru(2.0f, e, __fmaf_ru(kU, a.rate_up[l], 2.0f * eta_r)));
        wlo = w;
        if (__fadd_ru(__fsub_ru(alo, a.rate_dn[l]), w) > 0.0f) {
            whi = w;
            if (refine) {
                flags |= 1;
                slo = whi = 0.0f;  // base_refine adds the FP64 term
            }
        }
    }
    if (writer) {
        a.line_c[(size_t)j * a.n_l + l] = c;
        a.line_e[(size_t)j * a.n_l + l] = e;
        a.line_R[(size_t)j * a.n_l + l] = R;
    }
    // obj_lo's active set (upper violation bound positive)
    if (writer && a.act_list_lo && shi > 0.0f) {
        const int idx = atomicAdd(&a.act_count_lo[j], 1);
        if (idx < a.act_cap_lo)
            a.act_list_lo[(size_t)j * a.act_cap_lo + idx] =
                make_int4(l, l, __float_as_int(0.0f), __float_as_int(c > 0.0f ? 1.0f : -1.0f));
        else
            atomicOr(a.err, kErrOverflow);
    }
    // the adjoint's active set: certified by the FP32 bound
    if (writer && a.act_list && slo_f > 0.0f) {
        const int idx = atomicAdd(&a.act_count[j], 1);
        if (idx < a.act_cap)
            a.act_list[(size_t)j * a.act_cap + idx] =
                make_int4(l, l, __float_as_int(0.0f), __float_as_int(c > 0.0f ? 1.0f : -1.0f));
        else
            atomicOr(a.err, kErrOverflow);
    }
    double *q = part + j * kPartVals;
    if (writer) {
        q[0] = __dadd_rd(q[0], (double)slo);
        q[1] = __dadd_ru(q[1], (double)shi);
        q[2] = __dadd_ru(q[2], (double)whi);
        q[3] = __dadd_ru(q[3], (double)wlo);
    }
    if (a.is_bridge && a.is_bridge[l] && a.n_c > 0) {
        // A bridge carries the net injection of the side away from
        // the slack; no non-islanding outage changes that, so
        // L[l,k] = 0 and every contingency pair of the line has the
        // base interval [c - rho, c + rho] (eq. (slack-Sc) with the
        // contingency rating), n_c times.
        const float rcu = a.rate_c_up[l], rcd = a.rate_c_dn[l];
        const float clo_f = fmax0(__fsub_rd(alo, rcu));
        float clo = clo_f;
        const float chi = fmax0(__fsub_ru(ahi, rcd));
        float cwh = 0.0f, cwl = 0.0f;
        if (chi > 0.0f) {
            const float w = __fmaf_ru(a.gamma_base + 3.0f * kU, R,
                                      __fmaf_ru(2.0f, e, __fmaf_ru(kU, rcu, 2.0f * eta_r)));
            cwl = w;
            if (__fadd_ru(__fsub_ru(alo, rcd), w) > 0.0f) {
                cwh = w;
                if (refine) {
                    flags |= 2;
                    clo = cwh = 0.0f;
                }
            }
        }
        const double nc = (double)a.n_c;
        if (writer) {
            q[0] = __dadd_rd(q[0], __dmul_rd(nc, (double)clo));
            q[1] = __dadd_ru(q[1], __dmul_ru(nc, (double)chi));
            q[2] = __dadd_ru(q[2], __dmul_ru(nc, (double)cwh));
            q[3] = __dadd_ru(q[3], __dmul_ru(nc, (double)cwl));
        }
        if (writer && a.act_list_lo && chi > 0.0f) {
            const int idx = atomicAdd(&a.act_count_lo[j], 1);
            if (idx < a.act_cap_lo)
                a.act_list_lo[(size_t)j * a.act_cap_lo + idx] =
                    make_int4(l, -1, __float_as_int((float)a.n_c),
                              __float_as_int(c > 0.0f ? 1.0f : -1.0f));
            else
                atomicOr(a.err, kErrOverflow);
        }
        if (writer && a.act_list && clo_f > 0.0f) {
            const int idx = atomicAdd(&a.act_count[j], 1);
            if (idx < a.act_cap)
                a.act_list[(size_t)j * a.act_cap + idx] =
                    make_int4(l, -1, __float_as_int((float)a.n_c),
                              __float_as_int(c > 0.0f ? 1.0f : -1.0f));
            else
                atomicOr(a.err, kErrOverflow);
        }
    }
    return flags;
}

// The FP64 refinement of the terms base_epilogue left out (flags): the base
// violation of line l (base rating) and, for a bridge, its n_c contingency
// pairs (contingency rating).  Warp-cooperative; lane 0 writes.
static __device__ __noinline__ void base_refine(const BaseArgs &a, int l, int j, int flags, double *part) {
    const int lane = threadIdx.x & 31;
    double *q = part + j * kPartVals;
    for (int t = 0; t < 2; ++t) {
        if (!((flags >> t) & 1)) continue;
        const double rating = t == 0 ? a.ref.rate64[l] : a.ref.rate_c64[l];
        const RefOut o = refine_term(a.ref, j, l, l, -1, 0.0f, rating, kRefLine);
        const double m = t == 0 ? 1.0 : (double)a.n_c;
        if (lane == 0) {
            q[0] = __dadd_rd(q[0], __dmul_rd(m, o.s_lo));
            q[2] = __dadd_ru(q[2], __dmul_ru(m, o.w));
        }
    }
}

// Compensated FP32 accumulation of sum_b Phi~[l,b] c_b with c_b = hi + lo:
// each product Phi~ hi is split exactly (FMA remainder), the running sum uses
// TwoSum (Knuth, The Art of Computer Programming vol. 2, Sec. 4.2.2; the
// summation is the compensated dot product of Ogita, Rump and Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 26(6), 2005), and
// Phi~ lo goes to the compensation term.  The error is below
// n u^2 sum_b |Phi~[l,b] c_b| plus the representation of c_b (u^2 |c_b|), far
// inside the 0.1 u C_l left in e_l = 2.1 u C_l for the summation.
struct FF {
    float s, e;
};
// (intrinsics throughout: a contracted multiply-add would break TwoSum)
__device__ __forceinline__ void ff_add_prod(FF &acc, float p, float2 c) {
    const float m = __fmul_rn(p, c.x);
    const float me = __fmaf_rn(p, c.x, -m);
    const float t = __fadd_rn(acc.s, m);
    const float z = __fsub_rn(t, acc.s);
    const float err = __fadd_rn(__fsub_rn(acc.s, __fsub_rn(t, z)), __fsub_rn(m, z));
    acc.s = t;
    acc.e = __fmaf_rn(p, c.y, __fadd_rn(acc.e, __fadd_rn(err, me)));
}

// Box-grouped base flows: a warp takes one line and up to G boxes, reads the
// PTDF row once and keeps the sums of every box of the group.  One-box calls
// use G = 1, whose few registers leave room to unroll the row loop (more
// loads in flight per warp).
constexpr int kBaseGroup = 8;

template <int G>
__global__ void __launch_bounds__(kBaseWarps * 32) k_base_ff(BaseArgs a) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kBaseWarps + warp;
    const int nw = gridDim.x * kBaseWarps;
    const int n_groups = (a.n_box + G - 1) / G;
    const int n_items = a.n_l * n_groups + (a.hat_k ? a.n_c : 0);
    const int nv = a.n_a_pad >> 2;  // float4 per row
    double *part = a.partials + (size_t)gw * a.n_box * kPartVals;
    for (int j = 0; j < a.n_box; ++j)
        if (lane == 0)
            for (int v = 0; v < kPartVals; ++v) part[j * kPartVals + v] = 0.0;
    for (int item = gw; item < n_items; item += nw) {
        if (item >= a.n_l * n_groups) {
            // scaled copy of a contingency line's row (one-box mode)
            const int k = item - a.n_l * n_groups;
            const float4 *src = reinterpret_cast<const float4 *>(a.phi + (size_t)a.ctg_line[k] * a.n_a_pad);
            const float4 *rr = reinterpret_cast<const float4 *>(a.rbus);
            float4 *dst = reinterpret_cast<float4 *>(a.hat_k + (size_t)k * a.n_a_pad);
            for (int v = lane; v < nv; v += 32) {
                const float4 p = src[v], r = rr[v];
                dst[v] = make_float4(__fmul_rn(p.x, r.x), __fmul_rn(p.y, r.y), __fmul_rn(p.z, r.z),
                                     __fmul_rn(p.w, r.w));
            }
            continue;
        }
        const int l = item / n_groups, j0 = (item % n_groups) * G;
        const int bg = min(G, a.n_box - j0);
        const float4 *prow = reinterpret_cast<const float4 *>(a.phi + (size_t)l * a.n_a_pad);
        float4 *hl = a.hat_l ? reinterpret_cast<float4 *>(a.hat_l + (size_t)l * a.n_a_pad) : nullptr;
        // C and R keep one round-up sum per bus of the float4 (the same
        // summation tree as the FP64 kernel, so gamma_base holds for both)
        FF cs[G];
        float4 C[G], R[G];
#pragma unroll
        for (int jj = 0; jj < G; ++jj) {
            cs[jj] = FF{0.0f, 0.0f};
            C[jj] = R[jj] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
        // one float4 of the row (4 buses) into the sums of the group's boxes
        auto step = [&](const float4 p, int v) {
            const float4 ap = make_float4(fabsf(p.x), fabsf(p.y), fabsf(p.z), fabsf(p.w));
#pragma unroll
            for (int jj = 0; jj < G; ++jj) {
                if (jj >= bg) break;
                const size_t o = (size_t)(j0 + jj) * a.n_a_pad;
                const float4 *c2 = reinterpret_cast<const float4 *>(a.cbus2 + o) + 2 * v;
                const float4 c01 = c2[0], c23 = c2[1];
                const float4 r = reinterpret_cast<const float4 *>(a.rbus + o)[v];
                const float4 ca = reinterpret_cast<const float4 *>(a.cabs + o)[v];
                ff_add_prod(cs[jj], p.x, make_float2(c01.x, c01.y));
                ff_add_prod(cs[jj], p.y, make_float2(c01.z, c01.w));
                ff_add_prod(cs[jj], p.z, make_float2(c23.x, c23.y));
                ff_add_prod(cs[jj], p.w, make_float2(c23.z, c23.w));
                C[jj].x = __fmaf_ru(ap.x, ca.x, C[jj].x);
                C[jj].y = __fmaf_ru(ap.y, ca.y, C[jj].y);
                C[jj].z = __fmaf_ru(ap.z, ca.z, C[jj].z);
                C[jj].w = __fmaf_ru(ap.w, ca.w, C[jj].w);
                R[jj].x = __fmaf_ru(ap.x, r.x, R[jj].x);
                R[jj].y = __fmaf_ru(ap.y, r.y, R[jj].y);
                R[jj].z = __fmaf_ru(ap.z, r.z, R[jj].z);
                R[jj].w = __fmaf_ru(ap.w, r.w, R[jj].w);
                if (hl && jj == 0)
                    hl[v] = make_float4(__fmul_rn(p.x, r.x), __fmul_rn(p.y, r.y), __fmul_rn(p.z, r.z),
                                        __fmul_rn(p.w, r.w));
            }
        };
        if constexpr (G == 1) {
            // the lane's row entries v = lane + 32 i in ascending i, as below;
            // the next kPf row loads are in flight while the current ones are used
            constexpr int kPf = 8;
            float4 nxt[kPf];
#pragma unroll
            for (int u = 0; u < kPf; ++u) {
                const int v = lane + 32 * u;
                nxt[u] = v < nv ? prow[v] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
            for (int v0 = lane; v0 < nv; v0 += 32 * kPf) {
                float4 cur[kPf];
#pragma unroll
                for (int u = 0; u < kPf; ++u) {
                    cur[u] = nxt[u];
                    const int v = v0 + 32 * (kPf + u);
                    nxt[u] = v < nv ? prow[v] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                }
#pragma unroll
                for (int u = 0; u < kPf; ++u)
                    if (v0 + 32 * u < nv) step(cur[u], v0 + 32 * u);
            }
        } else {
            for (int v = lane; v < nv; v += 32) step(prow[v], v);
        }
#pragma unroll
        for (int jj = 0; jj < G; ++jj) {
            if (jj >= bg) break;
            // lanes' compensated sums are exact in FP64; the 5-level FP64 tree
            // adds about 5 * 2^-53 relative
            double d = (double)cs[jj].s + (double)cs[jj].e;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            const float Cs = warp_sum_ru_f(
                __fadd_ru(__fadd_ru(C[jj].x, C[jj].y), __fadd_ru(C[jj].z, C[jj].w)));
            const float Rs = warp_sum_ru_f(
                __fadd_ru(__fadd_ru(R[jj].x, R[jj].y), __fadd_ru(R[jj].z, R[jj].w)));
            const int f = base_epilogue(a, l, j0 + jj, __double2float_rn(d), Cs, Rs, part, lane == 0);
            if (f) base_refine(a, l, j0 + jj, f, part);
        }
    }
}

__global__ void __launch_bounds__(kBaseWarps * 32) k_base(BaseArgs a) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kBaseWarps + warp;
    const int nw = gridDim.x * kBaseWarps;
    const int n_rows = a.n_l + (a.hat_k ? a.n_c : 0);
    const int nv = a.n_a_pad >> 2;  // float4 per row
    double *part = a.partials + (size_t)gw * a.n_box * kPartVals;
    for (int j = 0; j < a.n_box; ++j)
        if (lane == 0)
            for (int v = 0; v < kPartVals; ++v) part[j * kPartVals + v] = 0.0;
    for (int row = gw; row < n_rows; row += nw) {
        if (row >= a.n_l) {
            // scaled copy of a contingency line's row (one-box mode)
            const int k = row - a.n_l;
            const float4 *src = reinterpret_cast<const float4 *>(a.phi + (size_t)a.ctg_line[k] * a.n_a_pad);
            const float4 *rr = reinterpret_cast<const float4 *>(a.rbus);
            float4 *dst = reinterpret_cast<float4 *>(a.hat_k + (size_t)k * a.n_a_pad);
            for (int v = lane; v < nv; v += 32) {
                const float4 p = src[v], r = rr[v];
                dst[v] = make_float4(__fmul_rn(p.x, r.x), __fmul_rn(p.y, r.y), __fmul_rn(p.z, r.z),
                                     __fmul_rn(p.w, r.w));
            }
            continue;
        }
        const int l = row;
        const float4 *prow = reinterpret_cast<const float4 *>(a.phi + (size_t)l * a.n_a_pad);
        for (int j = 0; j < a.n_box; ++j) {
            const double2 *cb = reinterpret_cast<const double2 *>(a.cbus + (size_t)j * a.n_a_pad);
            const float4 *rb = reinterpret_cast<const float4 *>(a.rbus + (size_t)j * a.n_a_pad);
            const float4 *ab = reinterpret_cast<const float4 *>(a.cabs + (size_t)j * a.n_a_pad);
            double cs = 0.0;
            float C0 = 0.f, C1 = 0.f, C2 = 0.f, C3 = 0.f;
            float R0 = 0.f, R1 = 0.f, R2 = 0.f, R3 = 0.f;
            float4 *hl = a.hat_l ? reinterpret_cast<float4 *>(a.hat_l + (size_t)l * a.n_a_pad) : nullptr;
            for (int v = lane; v < nv; v += 32) {
                const float4 p = prow[v];
                const double2 c01 = cb[2 * v], c23 = cb[2 * v + 1];
                const float4 r = rb[v], ca = ab[v];
                cs = fma((double)p.x, c01.x, cs);
                cs = fma((double)p.y, c01.y, cs);
                cs = fma((double)p.z, c23.x, cs);
                cs = fma((double)p.w, c23.y, cs);
                C0 = __fmaf_ru(fabsf(p.x), ca.x, C0);
                C1 = __fmaf_ru(fabsf(p.y), ca.y, C1);
                C2 = __fmaf_ru(fabsf(p.z), ca.z, C2);
                C3 = __fmaf_ru(fabsf(p.w), ca.w, C3);
                R0 = __fmaf_ru(fabsf(p.x), r.x, R0);
                R1 = __fmaf_ru(fabsf(p.y), r.y, R1);
                R2 = __fmaf_ru(fabsf(p.z), r.z, R2);
                R3 = __fmaf_ru(fabsf(p.w), r.w, R3);
                if (hl)
                    hl[v] = make_float4(__fmul_rn(p.x, r.x), __fmul_rn(p.y, r.y), __fmul_rn(p.z, r.z),
                                        __fmul_rn(p.w, r.w));
            }
            float C = __fadd_ru(__fadd_ru(C0, C1), __fadd_ru(C2, C3));
            float R = __fadd_ru(__fadd_ru(R0, R1), __fadd_ru(R2, R3));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
            C = warp_sum_ru_f(C);
            R = warp_sum_ru_f(R);
            const int f = base_epilogue(a, l, j, __double2float_rn(cs), C, R, part, lane == 0);
            if (f) base_refine(a, l, j, f, part);
            hl = nullptr;
        }
    }
}

cudaError_t launch_base(const BaseArgs &a, int n_part, cudaStream_t s) {
    const int grid = n_part / kBaseWarps;
    if (a.cbus2 && a.n_box == 1) k_base_ff<1><<<grid, kBaseWarps * 32, 0, s>>>(a);
    else if (a.cbus2) k_base_ff<kBaseGroup><<<grid, kBaseWarps * 32, 0, s>>>(a);
    else k_base<<<grid, kBaseWarps * 32, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Objective assembly, in two stages: k_partials (64 blocks per box) sums
// slices of the rows and devices, k_assemble (one block per box) adds them and
// forms the objective (eq. (penalized-objective), appendix
// eq. (ibp_f) under eq. (IBP)):
//   hi = C(pd_hi) - G(pg_lo) - z_inj s_inj,lo - z_f (S_fb,lo + S_fc,lo)
//   lo = C(pd_lo) - G(pg_hi) - z_inj s_inj,hi - z_f (S_fb,hi + S_fc,hi)
// The PWL curves are monotone, so their IBP is the value at the endpoints,
// evaluated through the ReLU chain of eqs. (single ReLU), (combined ReLUs) in
// round-up and round-down arithmetic.  The imbalance uses the closed form
// (E^T Phi - I) p = -(1^T p) e_slack (the explicit matrix has zero rows away
// from the slack), so 1^T s_inj is |.| of the interval of the total
// injection.  All sums are FP64 with directed rounding.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double pwl_eval(const double *a, const double *b, int n, double x,
                                           bool up) {
    double F = 0.0, U = 0.0;
    for (int m = 0; m < n; ++m) {
        double t;
        if (up) {
            t = __dmul_ru(a[m], fmax(__dsub_ru(x, b[m]), 0.0));
            F = __dadd_ru(F, t);
        } else {
            t = __dmul_rd(a[m], fmax(__dsub_rd(x, b[m]), 0.0));
            F = __dadd_rd(F, t);
        }
        if (m + 1 < n) {
            const double seg = up ? __dmul_ru(a[m], __dsub_ru(b[m + 1], b[m]))
                                  : __dmul_rd(a[m], __dsub_rd(b[m + 1], b[m]));
            U = up ? __dadd_ru(U, seg) : __dadd_rd(U, seg);
            F = fmin(F, U);
        }
    }
    return F;
}

__device__ __forceinline__ void block_sum(double *v, int n, bool *up, double *sh) {
    // v[0..n) per thread -> thread 0 holds totals; sh has room for 8 * n doubles
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int i = 0; i < n; ++i) v[i] = up[i] ? warp_sum_ru(v[i]) : warp_sum_rd(v[i]);
    if (l == 0)
        for (int i = 0; i < n; ++i) sh[w * n + i] = v[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k)
                s = up[i] ? __dadd_ru(s, sh[k * n + i]) : __dadd_rd(s, sh[k * n + i]);
            v[i] = s;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ int ctg_partial_rows(const AsmArgs &a) {
    if (a.n_live)
        return (*a.n_live + a.live_BL - 1) / a.live_BL * a.live_tiles_k * a.live_rows_per_tile;
    return a.n_part_ctg;
}

// The sums of the objective assembly (directed FP64; kAsmUp: rounded up):
//   0 Sfc_lo(rd) 1 Sfc_hi(ru) 2 Wfc_hi(ru) 3 Wfc_lo(ru)   contingency partial rows
//   4 Sfb_lo 5 Sfb_hi 6 Wfb_hi 7 Wfb_lo                   base partial rows
//   8 Clo_dn 9 Chi_up 10 Glo_dn 11 Ghi_up 12 cost_err_hi(ru) 13 cost_err_lo(ru)
//   14 Plo_dn 15 Plo_up 16 Phi_dn 17 Phi_up               devices
__device__ __forceinline__ bool asm_up(int i) {
    return !(i == 0 || i == 4 || i == 8 || i == 10 || i == 14 || i == 16);
}

__device__ __forceinline__ void add_rows(double *v, const double *q) {
    const double4 r = *reinterpret_cast<const double4 *>(q);
    v[0] = __dadd_rd(v[0], r.x);
    v[1] = __dadd_ru(v[1], r.y);
    v[2] = __dadd_ru(v[2], r.z);
    v[3] = __dadd_ru(v[3], r.w);
}

// cost, value and injection terms of device d of box j (eq. (penalized-objective))
__device__ __forceinline__ void add_device(const AsmArgs &a, int j, int d, double *v) {
    const double x = a.box_lo[(size_t)j * a.n_dev + d], y = a.box_hi[(size_t)j * a.n_dev + d];
    const int s0 = a.seg_ptr[d], ns = a.seg_ptr[d + 1] - s0;
    const double *sl = a.slope + s0, *bk = a.bkpt + s0;
    const double vlo_dn = pwl_eval(sl, bk, ns, x, false);
    const double vlo_up = pwl_eval(sl, bk, ns, x, true);
    const double vhi_dn = pwl_eval(sl, bk, ns, y, false);
    const double vhi_up = pwl_eval(sl, bk, ns, y, true);
    if (d >= a.n_gen) {  // load value c_j: C(hi) enters obj_hi, C(lo) enters obj_lo
        v[8] = __dadd_rd(v[8], vlo_dn);
        v[9] = __dadd_ru(v[9], vhi_up);
        v[12] = __dadd_ru(v[12], __dsub_ru(vhi_up, vhi_dn));
        v[13] = __dadd_ru(v[13], __dsub_ru(vlo_up, vlo_dn));
        v[14] = __dadd_rd(v[14], -y);
        v[15] = __dadd_ru(v[15], -y);
        v[16] = __dadd_rd(v[16], -x);
        v[17] = __dadd_ru(v[17], -x);
    } else {  // generator cost g_i: G(lo) enters obj_hi, G(hi) enters obj_lo
        v[10] = __dadd_rd(v[10], vlo_dn);
        v[11] = __dadd_ru(v[11], vhi_up);
        v[12] = __dadd_ru(v[12], __dsub_ru(vlo_up, vlo_dn));
        v[13] = __dadd_ru(v[13], __dsub_ru(vhi_up, vhi_dn));
        v[14] = __dadd_rd(v[14], x);
        v[15] = __dadd_ru(v[15], x);
        v[16] = __dadd_rd(v[16], y);
        v[17] = __dadd_ru(v[17], y);
    }
}

// Stage 1 of the assembly: block (g, box) sums its slice -- items g*128 + t +
// k*(n_stage*128) -- of the contingency partial rows, the base partial rows and
// the devices (directed FP64), then reduces its 128 threads in a fixed tree
// and writes the kAsmVals sums; the result does not depend on timing.
__global__ void __launch_bounds__(128) k_partials(AsmArgs a) {
    const int g = blockIdx.x, j = blockIdx.y;
    const int n = ctg_partial_rows(a), first = g * 128 + (int)threadIdx.x, stride = a.n_stage * 128;
    double v[kAsmVals];
    bool up[kAsmVals];
#pragma unroll
    for (int i = 0; i < kAsmVals; ++i) {
        v[i] = 0.0;
        up[i] = asm_up(i);
    }
    for (int p = first; p < n; p += stride)
        add_rows(v, a.part_ctg + ((size_t)p * a.n_box + j) * kPartVals);
    for (int p = first; p < a.n_part_base; p += stride)
        add_rows(v + 4, a.part_base + ((size_t)p * a.n_box + j) * kPartVals);
    for (int d = first; d < a.n_dev; d += stride) add_device(a, j, d, v);
    __shared__ double sh[4 * kAsmVals];
    block_sum(v, kAsmVals, up, sh);
    if (threadIdx.x == 0) {
        double *o = a.part_stage + ((size_t)j * a.n_stage + g) * kAsmVals;
#pragma unroll
        for (int i = 0; i < kAsmVals; ++i) o[i] = v[i];
    }
}

__global__ void __launch_bounds__(256) k_assemble(AsmArgs a) {
    const int j = blockIdx.x;
    constexpr int N = kAsmVals;
    double v[N];
    bool up[N];
    for (int i = 0; i < N; ++i) {
        v[i] = 0.0;
        up[i] = asm_up(i);
    }
    if (a.part_stage) {
        // stage 1 (k_partials) summed the rows and devices: combine its blocks
        for (int p = threadIdx.x; p < a.n_stage; p += blockDim.x) {
            const double *q = a.part_stage + ((size_t)j * a.n_stage + p) * N;
            for (int i = 0; i < N; ++i) v[i] = up[i] ? __dadd_ru(v[i], q[i]) : __dadd_rd(v[i], q[i]);
        }
    } else {
        const int n_part_ctg = ctg_partial_rows(a);
        for (int p = threadIdx.x; p < n_part_ctg; p += blockDim.x)
            add_rows(v, a.part_ctg + ((size_t)p * a.n_box + j) * kPartVals);
        for (int p = threadIdx.x; p < a.n_part_base; p += blockDim.x)
            add_rows(v + 4, a.part_base + ((size_t)p * a.n_box + j) * kPartVals);
        for (int d = threadIdx.x; d < a.n_dev; d += blockDim.x) add_device(a, j, d, v);
    }
    __shared__ double sh[8 * N];
    block_sum(v, N, up, sh);
    if (threadIdx.x == 0) {
        // total injection interval [Plo, Phi] enclosed by [Plo_dn, Phi_up]
        const double plo = v[14], phi = v[17];
        double ilo, ihi;
        if (plo >= 0.0) {
            ilo = plo;
            ihi = phi;
        } else if (phi <= 0.0) {
            ilo = -phi;
            ihi = -plo;
        } else {
            ilo = 0.0;
            ihi = fmax(-plo, phi);
        }
        const double w_inj = fmax(__dsub_ru(v[15], v[14]), __dsub_ru(v[17], v[16]));
        const double pen_dn = __dadd_rd(__dmul_rd(a.zeta_inj, ilo),
                                        __dmul_rd(a.zeta_f, __dadd_rd(v[4], v[0])));
        const double pen_up = __dadd_ru(__dmul_ru(a.zeta_inj, ihi),
                                        __dmul_ru(a.zeta_f, __dadd_ru(v[5], v[1])));
        double ohi = __dsub_ru(__dsub_ru(v[9], v[10]), pen_dn);
        double olo = __dsub_rd(__dsub_rd(v[8], v[11]), pen_up);
        // error bounds: FP32 allowances of the flow terms, the imbalance
        // enclosure, the cost enclosures, plus FP64 summation of the partial sums
        double ehi = __dmul_ru(a.zeta_f, __dadd_ru(v[2], v[6]));
        ehi = __dadd_ru(ehi, __dmul_ru(a.zeta_inj, w_inj));
        ehi = __dadd_ru(ehi, v[12]);
        ehi = __dadd_ru(ehi, __dmul_ru(1e-12, __dadd_ru(__dadd_ru(fabs(v[9]), fabs(v[10])), pen_dn)));
        double elo = __dmul_ru(a.zeta_f, __dadd_ru(v[3], v[7]));
        elo = __dadd_ru(elo, __dmul_ru(a.zeta_inj, w_inj));
        elo = __dadd_ru(elo, v[13]);
        elo = __dadd_ru(elo, __dmul_ru(1e-12, __dadd_ru(__dadd_ru(fabs(v[8]), fabs(v[11])), pen_up)));
        if (*a.err) {
            ohi = olo = ehi = elo = __longlong_as_double(0x7ff8000000000000ll);
        }
        a.obj_hi[j] = ohi;
        a.obj_lo[j] = olo;
        a.obj_err[2 * j] = ehi;
        a.obj_err[2 * j + 1] = elo;
    }
}

cudaError_t launch_assemble(const AsmArgs &a, cudaStream_t s) {
    if (a.part_stage) {
        k_partials<<<dim3(a.n_stage, a.n_box), 128, 0, s>>>(a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_assemble<<<a.n_box, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// error word of a shared launch -> each case's error word
__global__ void k_or_err(int *dst, const int *src) {
    if (threadIdx.x == 0 && *src) atomicOr(dst, *src);
}

cudaError_t launch_or_err(int *dst, const int *src, cudaStream_t s) {
    k_or_err<<<1, 32, 0, s>>>(dst, src);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Bounded-wait self test: one thread waits on an mbarrier whose phase never
// completes (nobody arrives), gives up after limit_ns and reports it.
// ---------------------------------------------------------------------------
__global__ void k_wait_selftest(int *flag, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_addr(&bar), 1);
        fence_mbar_init();
        const bool ok = mbar_wait(smem_addr(&bar), 0, limit_ns);
        *flag = ok ? 0 : kErrTimeout;
    }
}

cudaError_t launch_wait_selftest(int *flag, unsigned long long limit_ns, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(flag, limit_ns);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Case-build kernels (FP64, once per case).
// ---------------------------------------------------------------------------
__global__ void k_scatter_dense(double *dst, int64_t ld, const int *rows, const int *cols,
                                const double *vals, int nnz) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nnz) dst[(int64_t)cols[i] * ld + rows[i]] = vals[i];
}

cudaError_t launch_scatter_dense(double *dst, int64_t ld, const int *rows, const int *cols,
                                 const double *vals, int nnz, cudaStream_t s) {
    if (nnz <= 0) return cudaSuccess;
    k_scatter_dense<<<(nnz + 255) / 256, 256, 0, s>>>(dst, ld, rows, cols, vals, nnz);
    return cudaGetLastError();
}

__device__ __forceinline__ float to_f32_flushed(double x) {
    // values below 2^-120 in magnitude are stored as 0 (accounted for by eta)
    return fabs(x) < 7.52316384526264e-37 ? 0.0f : __double2float_rn(x);
}

// Z is column-major (nb_r x n_l): column l holds Phi_r[l, :] (reduced buses).
// phi_a = the FP32 PTDF of the active columns; phi64 (optional) = the same
// columns in FP64, as built.
__global__ void k_extract_phi(const double *Z, int nb_r, int n_l, const int *act_red, int n_a,
                              int n_a_pad, float *phi_a, double *phi64) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)n_l * n_a_pad;
    if (i >= tot) return;
    const int l = (int)(i / n_a_pad), a = (int)(i % n_a_pad);
    double x = 0.0;
    if (a < n_a) x = Z[(int64_t)l * nb_r + act_red[a]];
    phi_a[i] = a < n_a ? to_f32_flushed(x) : 0.0f;
    if (phi64) phi64[i] = x;
}

cudaError_t launch_extract_phi(const double *Z, int nb_r, int n_l, const int *act_red, int n_a,
                               int n_a_pad, float *phi_a, double *phi64, cudaStream_t s) {
    const int64_t tot = (int64_t)n_l * n_a_pad;
    k_extract_phi<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Z, nb_r, n_l, act_red, n_a, n_a_pad,
                                                                phi_a, phi64);
    return cudaGetLastError();
}

// L[k][l] = PTDF_line[l,k] / (1 - PTDF_line[kline,k]),  L[k][kline] = -1,
// PTDF_line[l,k] = Phi[l, from_k] - Phi[l, to_k] (slack entries are 0).
// One block per contingency.
__global__ void k_lodf(const double *Z, int nb_r, int n_l, int n_c, const int *fr, const int *to,
                       const int *ctg_line, float *lodf, float *lodf_lo, double *den_out,
                       float *maxabs) {
    const int k = blockIdx.x;
    const int f = fr[k], t = to[k], kl = ctg_line[k];
    auto ptl = [&](int l) -> double {
        const double *col = Z + (int64_t)l * nb_r;
        const double a = f >= 0 ? col[f] : 0.0;
        const double b = t >= 0 ? col[t] : 0.0;
        return a - b;
    };
    const double den = 1.0 - ptl(kl);
    if (threadIdx.x == 0) den_out[k] = den;
    float mx = 0.0f;
    for (int l = threadIdx.x; l < n_l; l += blockDim.x) {
        float v, w = 0.0f;
        if (l == kl) {
            v = -1.0f;
        } else {
            const double x = ptl(l) / den;
            v = to_f32_flushed(x);
            w = __double2float_rn(x - (double)v);  // the FP64 remainder (optional copy)
        }
        lodf[(int64_t)k * n_l + l] = v;
        if (lodf_lo) lodf_lo[(int64_t)k * n_l + l] = w;
        mx = fmaxf(mx, fabsf(v));
    }
    mx = warp_max_f(mx);
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(maxabs), __float_as_int(mx));
}

cudaError_t launch_lodf(const double *Z, int nb_r, int n_l, int n_c, const int *ctg_from_red,
                        const int *ctg_to_red, const int *ctg_line, float *lodf, float *lodf_lo,
                        double *den_out, float *maxabs_out, cudaStream_t s) {
    if (n_c <= 0) return cudaSuccess;
    k_lodf<<<n_c, 256, 0, s>>>(Z, nb_r, n_l, n_c, ctg_from_red, ctg_to_red, ctg_line, lodf, lodf_lo,
                               den_out, maxabs_out);
    return cudaGetLastError();
}

__global__ void k_gather_rows(const float *src, int ld, const int *rows, int n_rows, float *dst) {
    const int r = blockIdx.x;
    if (r >= n_rows) return;
    const float *s = src + (int64_t)rows[r] * ld;
    float *d = dst + (int64_t)r * ld;
    for (int i = threadIdx.x; i < ld; i += blockDim.x) d[i] = s[i];
}

cudaError_t launch_gather_rows(const float *src, int ld, const int *rows, int n_rows, float *dst,
                               cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    k_gather_rows<<<n_rows, 256, 0, s>>>(src, ld, rows, n_rows, dst);
    return cudaGetLastError();
}

// dst[r][j] = src[r][cols[j]] for j < n_cols, 0 for n_cols <= j < ld_dst
__global__ void k_gather_cols(const float *src, int ld_src, const int *cols, int n_cols, float *dst,
                              int ld_dst) {
    const int r = blockIdx.x;
    const float *s = src + (int64_t)r * ld_src;
    float *d = dst + (int64_t)r * ld_dst;
    for (int j = threadIdx.x; j < ld_dst; j += blockDim.x) d[j] = j < n_cols ? s[cols[j]] : 0.0f;
}

cudaError_t launch_gather_cols(const float *src, int ld_src, int n_rows, const int *cols, int n_cols,
                               float *dst, int ld_dst, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    k_gather_cols<<<n_rows, 256, 0, s>>>(src, ld_src, cols, n_cols, dst, ld_dst);
    return cudaGetLastError();
}

}  // namespace ibp
