// Paper-mode line screen ahead of the contingency kernel.
//
// The paper propagates the contingency flow of eq. (ctg flow matrix form) as
// two intervals, [Phi p] and [U p], combined with the LODF column; for a pair
// (k, l) that gives the radius R_l + |L[l,k]| R_k, which is never smaller
// than the tight radius sum_b |Phi[l,b] + L[l,k] Phi[k,b]| r_b (triangle
// inequality).  A line whose upper flow bound in that two-part interval stays
// within its contingency rating for every contingency and every box has a
// violation interval of exactly [0, 0] in the tight interval as well, so it
// adds nothing to eq. (slack-Sc) and its tight radii need not be computed.
//
// Certified test (u = 2^-24; R~, c~, e as written by the base-flow kernel):
// the exact radius of line x is at most (1 + u) R~_x + eta_r and
// |L - L~| <= u |L~| + 2^-120, so
//   R_l + |L| R_k <= (1 + 4u)(R~_l + |L~| R~_k) + 2 eta_r (1 + |L~|),
// the exact centre is within e_c of the FP32 centre (pair_centre), and the
// line is dead when  RU(|c~| + e_c + that radius) <= rating rounded down.
//
// Bridge lines never reach the contingency kernel when the network reduction
// is on: no non-islanding outage moves their flow, and the base-flow kernel
// adds their contingency terms in closed form.
//
// Kernels: screen (one thread per line and block of contingencies), compact
// (one block: ascending list of live lines and its length), gather (one warp
// per row: the kept lines' PTDF rows and, in one-box mode, the contingency
// rows, scaled by the radius of each column), and the bus-class radii.
#include "common.cuh"
#include "ctg_epilogue.cuh"
#include "internal.h"

namespace ibp {

constexpr int kScreenThreads = 256;
constexpr int kScreenK = 64;  // contingencies per thread

__global__ void __launch_bounds__(kScreenThreads) k_screen(const ScreenArgs a) {
    const int l = blockIdx.x * kScreenThreads + threadIdx.x;
    if (l >= a.n_l) return;
    if (a.is_bridge && a.is_bridge[l]) return;
    if (!a.paper_test) {
        if (blockIdx.y == 0) a.live_flag[l] = 1;
        return;
    }
    const int k0 = blockIdx.y * kScreenK, k1 = min(k0 + kScreenK, a.n_c);
    const float rdn = __ldg(&a.rate_dn[l]);
    bool live = false;
    for (int j = 0; j < a.n_box && !live; ++j) {
        const size_t ob = (size_t)j * a.n_l;
        const float cl = __ldg(&a.line_c[ob + l]), el = __ldg(&a.line_e[ob + l]);
        const float Rl = __ldg(&a.line_R[ob + l]);
        const float eta_r = __ldg(&a.box_consts[(size_t)j * 4]);
        const float eta_c = __ldg(&a.box_consts[(size_t)j * 4 + 1]);
        for (int k = k0; k < k1; ++k) {
            const int kl = __ldg(&a.ctg_line[k]);
            if (kl == l) continue;  // the outaged line carries exactly nothing
            if (!IBP_IDX_OK(kl >= 0 && kl < a.n_l, a.err)) continue;
            const float Lt = __ldg(&a.lodf[(size_t)k * a.n_l + l]);
            const float ck = __ldg(&a.line_c[ob + kl]), ek = __ldg(&a.line_e[ob + kl]);
            const float Rk = __ldg(&a.line_R[ob + kl]);
            const float aL = fabsf(Lt);
            const float one_l = __fadd_ru(1.0f, aL);
            float c, ec;
            pair_centre(Lt, cl, ck, el, ek, eta_c, one_l, c, ec);
            const float m = __fmaf_ru(aL, Rk, Rl);
            float rp = __fmaf_ru(4.0f * kU, m, m);
            rp = __fmaf_ru(2.0f, __fmul_ru(eta_r, one_l), rp);
            const float U = __fadd_ru(__fadd_ru(fabsf(c), ec), rp);
            if (!(U <= rdn)) {  // NaN counts as live
                live = true;
                break;
            }
        }
    }
    if (live) a.live_flag[l] = 1;
}

// One block of 1024 threads: live[0 .. n_live) = ascending indices of the
// flagged lines.
__global__ void __launch_bounds__(1024) k_compact_live(const ScreenArgs a) {
    __shared__ int warp_off[32];
    __shared__ int chunk_total;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int base = 0;
    for (int l0 = 0; l0 < a.n_l; l0 += 1024) {
        const int l = l0 + (int)threadIdx.x;
        const bool f = l < a.n_l && a.live_flag[l] != 0;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        const int pre = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) warp_off[w] = __popc(bal);
        __syncthreads();
        if (w == 0) {
            const int t = warp_off[lane];
            int incl = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            warp_off[lane] = incl - t;
            if (lane == 31) chunk_total = incl;
        }
        __syncthreads();
        if (f) a.live[base + warp_off[w] + pre] = l;
        base += chunk_total;
        __syncthreads();
    }
    if (threadIdx.x == 0) *a.n_live = base;
}

// rows[i] = src[live[i]] and, with hat_k, hat_k[k] = src[ctg_line[k]]
// (times the column radius when given), one warp per row
__global__ void __launch_bounds__(256) k_gather_live_rows(const ScreenArgs a) {
    const int n = *a.n_live;
    const int n_rows = n + (a.hat_k ? a.n_c : 0);
    const int nv = a.n_w >> 2;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const float4 *rr = reinterpret_cast<const float4 *>(a.radius);
    for (int i = gw; i < n_rows; i += nw) {
        const int row = i < n ? a.live[i] : a.ctg_line[i - n];
        if (!IBP_IDX_OK(row >= 0 && row < a.n_l, a.err)) continue;
        const float4 *src = reinterpret_cast<const float4 *>(a.src + (size_t)row * a.n_w);
        float *d = i < n ? a.rows + (size_t)i * a.n_w : a.hat_k + (size_t)(i - n) * a.n_w;
        float4 *dst = reinterpret_cast<float4 *>(d);
        for (int v = lane; v < nv; v += 32) {
            const float4 p = src[v];
            if (rr) {
                const float4 r = rr[v];
                dst[v] = make_float4(__fmul_rn(p.x, r.x), __fmul_rn(p.y, r.y), __fmul_rn(p.z, r.z),
                                     __fmul_rn(p.w, r.w));
            } else {
                dst[v] = p;
            }
        }
    }
}

// rcls[box][j] = RU(sum over the members b of class j of rbus[box][b]); the
// classes partition a subset of the active columns (padding columns get 0)
__global__ void __launch_bounds__(256) k_class_radius(const ClsArgs a) {
    const int box = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.n_r_pad) return;
    float r = 0.0f;
    if (j < a.n_r) {
        const float *rb = a.rbus + (size_t)box * a.n_a_pad;
        for (int m = a.cls_ptr[j]; m < a.cls_ptr[j + 1]; ++m) r = __fadd_ru(r, rb[a.cls_col[m]]);
    }
    a.rcls[(size_t)box * a.n_r_pad + j] = r;
    if (a.rcls_t) a.rcls_t[(size_t)j * a.n_box_pad + box] = r;
}

cudaError_t launch_class_radius(const ClsArgs &a, cudaStream_t s) {
    if (a.n_box <= 0 || a.n_r_pad <= 0) return cudaSuccess;
    const dim3 g((a.n_r_pad + 255) / 256, a.n_box);
    k_class_radius<<<g, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// Paper-mode objective terms.  Per pair, the certified enclosure of the
// two-part interval is [c~ - rho, c~ + rho] with rho = RU(e_c + rp) and
// rp = RU((1 + 4u) m + 2 eta_r (1 + |L~|)), m = RU(R~_l + |L~| R~_k), as in the
// screen above.  Each violation is within
//   w = (gamma_base + 10u) m + 2 e_c + u rating + 4 eta_r (1 + |L~|)
// of its exact paper-mode value (R~ exceeds the exact radius sum by at most
// (gamma_base + 2.01u) of it plus eta, L~ is within u of L).  One thread per
// line and block of kScreenK contingencies; FP32 directed per thread, FP64
// directed per block.
// FP64 paper-mode interval of pair (k, l): centre c_l + L c_k, radius
// R_l + |L| R_k from the per-line FP64 values, with the bound
//   E = (n + 2) u64 X + e_L (|c_k| + R_k + n u64 X_k) + u64 (|c| + rad)
//       + 2^-118 (1 + |L|)(1 + e_L) (sum r + sum |c|)
// on its distance from the exact paper-mode interval (X, X_k, e_L as in the
// tight pairs' refinement); s_lo and w as there.
struct PaperRef {
    double s_lo, w;
};
__device__ __forceinline__ PaperRef paper_refine(const PaperArgs &a, int j, int l, int kl, int k, float Lt) {
    double eL;
    const double L = ref_lodf(a.ref, k, l, Lt, eL), aL = fabs(L);
    const size_t ob = (size_t)j * a.n_l;
    const double cl = a.lc64[ob + l], ck = a.lc64[ob + kl];
    const double Rl = a.lR64[ob + l], Rk = a.lR64[ob + kl];
    const double Xl = (double)a.lX[ob + l], Xk = (double)a.lX[ob + kl];
    const double c = fma(L, ck, cl);
    const double rad = __fma_ru(aL, Rk, Rl);
    const float *bc = a.ref.box_consts + (size_t)j * 4;
    const double tot = __dadd_ru((double)bc[2], (double)bc[3]);
    const double nu = ref_nu(a.ref.n_a_pad);
    double E = __dmul_ru(__dadd_ru(nu, 2.0 * kU64), __dmul_ru(k2m20p, __fma_ru(aL, Xk, Xl)));
    E = __fma_ru(eL, __fma_ru(nu, Xk, __dadd_ru(fabs(ck), Rk)), E);
    E = __fma_ru(kU64, __dadd_ru(fabs(c), rad), E);
    E = __fma_ru(__dmul_ru(2.0 * k2m119, __dmul_ru(__dadd_ru(1.0, aL), __dadd_ru(1.0, eL))), tot, E);
    const double rho = __dadd_ru(rad, E);
    const double lo = __dsub_rd(c, rho), hi = __dadd_ru(c, rho);
    const double alo = lo >= 0.0 ? lo : (hi <= 0.0 ? -hi : 0.0);
    const double rating = a.ref.rate_c64[l];
    PaperRef o;
    o.s_lo = fmax(__dsub_rd(alo, rating), 0.0);
    o.w = __fma_ru(4.0 * kU64, __dadd_ru(__dadd_ru(rad, fabs(c)), rating), __dmul_ru(2.0, E));
    return o;
}

// One warp per (line, box): the FP64 base-flow values of the paper mode's
// refinement (LineExactArgs).
__global__ void __launch_bounds__(256) k_line_exact(const LineExactArgs a) {
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    const int nv = a.ref.n_a_pad >> 2;
    for (int item = gw; item < a.n_l * a.n_box; item += nw) {
        const int l = item % a.n_l, j = item / a.n_l;
        const size_t ob = (size_t)j * a.ref.n_a_pad;
        const float4 *ph = reinterpret_cast<const float4 *>(a.ref.phi_hi + (size_t)l * a.ref.n_a_pad);
        const double2 *pl = reinterpret_cast<const double2 *>(a.ref.phi64 + (size_t)l * a.ref.n_a_pad);
        const double2 *cb = reinterpret_cast<const double2 *>(a.ref.cbus + ob);
        const double2 *rb = reinterpret_cast<const double2 *>(a.ref.rbus64 + ob);
        const float4 *r32 = reinterpret_cast<const float4 *>(a.ref.rbus + ob);
        const float4 *c32 = reinterpret_cast<const float4 *>(a.ref.cabs + ob);
        double S = 0.0, C = 0.0;
        float X = 0.0f;
        auto col = [&](float h, double p, double c, double r, float rc) {
            S = __fma_ru(fabs(p), r, S);
            C = fma(p, c, C);
            X = __fmaf_ru(fabsf(h), rc, X);
        };
        for (int v = lane; v < nv; v += 32) {
            const float4 h = __ldg(&ph[v]);
            const double2 p01 = __ldg(&pl[2 * v]), p23 = __ldg(&pl[2 * v + 1]);
            const double2 c01 = __ldg(&cb[2 * v]), c23 = __ldg(&cb[2 * v + 1]);
            const double2 r01 = __ldg(&rb[2 * v]), r23 = __ldg(&rb[2 * v + 1]);
            const float4 q = __ldg(&r32[v]), ca = __ldg(&c32[v]);
            col(h.x, p01.x, c01.x, r01.x, __fadd_ru(q.x, ca.x));
            col(h.y, p01.y, c01.y, r01.y, __fadd_ru(q.y, ca.y));
            col(h.z, p23.x, c23.x, r23.x, __fadd_ru(q.z, ca.z));
            col(h.w, p23.y, c23.y, r23.y, __fadd_ru(q.w, ca.w));
        }
        S = warp_sum_ru(S);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) C += __shfl_xor_sync(0xffffffffu, C, o);
        X = warp_sum_ru_f(X);
        if (lane == 0) {
            const size_t o = (size_t)j * a.n_l + l;
            a.c64[o] = C;
            a.R64[o] = S;
            a.X[o] = X;
        }
    }
}

cudaError_t launch_line_exact(const LineExactArgs &a, int num_sms, cudaStream_t s) {
    if (a.n_l <= 0 || a.n_box <= 0) return cudaSuccess;
    k_line_exact<<<num_sms * 8, 256, 0, s>>>(a);
    return cudaGetLastError();
}

int paper_partials_count(int n_l, int n_c) {
    return ((n_l + kScreenThreads - 1) / kScreenThreads) * ((n_c + kScreenK - 1) / kScreenK);
}

__global__ void __launch_bounds__(kScreenThreads) k_paper(const PaperArgs a) {
    const int l = blockIdx.x * kScreenThreads + threadIdx.x;
    const int j = blockIdx.z;
    const int k0 = blockIdx.y * kScreenK, k1 = min(k0 + kScreenK, a.n_c);
    float slo = 0.0f, shi = 0.0f, whi = 0.0f, wlo = 0.0f;
    double rs = 0.0, rw = 0.0;  // refined obj_hi terms of this thread (FP64)
    if (l < a.n_l) {
        const size_t ob = (size_t)j * a.n_l;
        const float cl = __ldg(&a.line_c[ob + l]), el = __ldg(&a.line_e[ob + l]);
        const float Rl = __ldg(&a.line_R[ob + l]);
        const float eta_r = __ldg(&a.box_consts[(size_t)j * 4]);
        const float eta_c = __ldg(&a.box_consts[(size_t)j * 4 + 1]);
        const float rup = __ldg(&a.rate_up[l]), rdn = __ldg(&a.rate_dn[l]);
        for (int k = k0; k < k1; ++k) {
            const int kl = __ldg(&a.ctg_line[k]);
            if (kl == l) continue;  // the outaged line carries exactly nothing
            if (!IBP_IDX_OK(kl >= 0 && kl < a.n_l, a.err)) continue;
            const float Lt = __ldg(&a.lodf[(size_t)k * a.n_l + l]);
            const float ck = __ldg(&a.line_c[ob + kl]), ek = __ldg(&a.line_e[ob + kl]);
            const float Rk = __ldg(&a.line_R[ob + kl]);
            const float aL = fabsf(Lt);
            const float one_l = __fadd_ru(1.0f, aL);
            const float eta = __fmul_ru(eta_r, one_l);
            float c, ec;
            pair_centre(Lt, cl, ck, el, ek, eta_c, one_l, c, ec);
            const float m = __fmaf_ru(aL, Rk, Rl);
            float rp = __fmaf_ru(4.0f * kU, m, m);
            rp = __fmaf_ru(2.0f, eta, rp);
            const float rho = __fadd_ru(rp, ec);
            float alo, ahi;
            abs_interval(__fsub_rd(c, rho), __fadd_ru(c, rho), alo, ahi);
            float vlo = fmax0(__fsub_rd(alo, rup));
            const float vhi = fmax0(__fsub_ru(ahi, rdn));
            shi = __fadd_ru(shi, vhi);
            if (vhi > 0.0f) {
                float w = __fmaf_ru(a.gamma_base + 10.0f * kU, m, __fmul_ru(2.0f, ec));
                w = __fmaf_ru(kU, rup, w);
                w = __fmaf_ru(4.0f, eta, w);
                wlo = __fadd_ru(wlo, w);
                if (__fadd_ru(__fsub_ru(alo, rdn), w) > 0.0f) {
                    if (a.ref.phi64) {
                        // the FP64 paper-mode interval from the per-line FP64 values
                        const PaperRef pr = paper_refine(a, j, l, kl, k, Lt);
                        rs = __dadd_rd(rs, pr.s_lo);
                        rw = __dadd_ru(rw, pr.w);
                        vlo = 0.0f;
                    } else {
                        whi = __fadd_ru(whi, w);
                    }
                }
            }
            slo = __fadd_rd(slo, vlo);
        }
    }
    // the FP32 directed sums of up to kScreenK terms are within 2u kScreenK
    // of the exact sums
    const float g = 2.02f * kU * (float)kScreenK;
    whi = __fmaf_ru(g, slo, whi);
    wlo = __fmaf_ru(g, shi, wlo);
    double d0 = warp_sum_rd(__dadd_rd((double)slo, rs)), d1 = warp_sum_ru((double)shi);
    double d2 = warp_sum_ru(__dadd_ru((double)whi, rw)), d3 = warp_sum_ru((double)wlo);
    __shared__ double sh[kScreenThreads / 32][4];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sh[w][0] = d0;
        sh[w][1] = d1;
        sh[w][2] = d2;
        sh[w][3] = d3;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0;
        for (int i = 0; i < kScreenThreads / 32; ++i) {
            r0 = __dadd_rd(r0, sh[i][0]);
            r1 = __dadd_ru(r1, sh[i][1]);
            r2 = __dadd_ru(r2, sh[i][2]);
            r3 = __dadd_ru(r3, sh[i][3]);
        }
        const size_t row = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        double *p = a.partials + (row * a.n_box + j) * kPartVals;
        p[0] = r0;
        p[1] = r1;
        p[2] = r2;
        p[3] = r3;
    }
}

cudaError_t launch_paper(const PaperArgs &a, cudaStream_t s) {
    if (a.n_l <= 0 || a.n_c <= 0 || a.n_box <= 0) return cudaSuccess;
    const dim3 g((a.n_l + kScreenThreads - 1) / kScreenThreads, (a.n_c + kScreenK - 1) / kScreenK,
                 a.n_box);
    k_paper<<<g, kScreenThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_screen(const ScreenArgs &a, int num_sms, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a.live_flag, 0, (size_t)a.n_l * sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (a.n_l > 0 && a.n_c > 0) {
        const dim3 g((a.n_l + kScreenThreads - 1) / kScreenThreads, (a.n_c + kScreenK - 1) / kScreenK);
        k_screen<<<g, kScreenThreads, 0, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_compact_live<<<1, 1024, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_gather_live_rows<<<num_sms * 4, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ibp
