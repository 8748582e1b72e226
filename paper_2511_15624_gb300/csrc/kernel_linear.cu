// Linear (CROWN-style) relaxation bound of the objective and the
// primal-dual iteration that optimises its slopes (ibp_bound_linear).
//
// f(x) = C(p_d) - G(p_g) - z_inj |sum_b p_b| - z_f (sum_l s_l + sum_{k,l} s_kl),
// s = max(|y| - R, 0) for the base flows y = f_l and the post-contingency
// flows y = f_kl = f_l + L[l,k] f_k (eq. (penalized-objective), eqs.
// (slack-sinj), (slack-sfb), (slack-Sc)).  For slopes a in [-1, 1],
//   max(|y| - R, 0) >= a y - |a| R,   |y| >= a0 y,
// so f(x) <= l_a(x) = C - G - z_inj a0 sum p - z_f sum_t (a_t y_t - |a_t| R_t)
// on the whole box, and max f <= U(a) = max_x l_a(x).  l_a is affine in the bus
// injections, sum_t a_t y_t = sum_b (Phi^T W)_b p_b with line weights
// W_l = a_l + sum_k a_kl and W_{line of k} += sum_l a_kl L[l,k], so
//   U(a) = z_f sum_t |a_t| R_t + sum_i max_{x_i in [lo_i, hi_i]} [phi_i(x_i) + c_i x_i],
//   c_i = -s_i (z_f (Phi^T W)_b(i) + z_inj a0)   (s_i = +1 generator, -1 load),
// exact per device (phi_i: the load's value or minus the generator's cost).
// U is the Lagrangian dual function of the LP whose optimum is max f; any
// slopes give a certified bound, and minimising U over them reaches that LP
// optimum.  The slopes are driven by a primal-dual hybrid gradient iteration
// (Chambolle and Pock, J. Math. Imaging Vision 40, 2011) on max_x min_a l_a(x)
// with the operator D K (K: x -> the flows and the total injection, D: their
// z_f / z_inj weights) and diagonal step sizes (Pock and Chambolle, ICCV
// 2011, alpha = 1: the inverse row and column sums of |D K|, here bounded
// from above by the triangle inequality) split by a primal weight, which
// every 1000 iterations moves halfway (in log) to the ratio of the dual and
// primal moves in the step-weighted norms (PDLP's primal weight update,
// Applegate et al., NeurIPS 2021).  The iterate is kept at these adaptations
// (no restart to averages of the slopes, so the slope step moves 12 bytes per
// pair, not 20); the primal point averaged over each window is the candidate
// maximiser.
// The iterations run in FP32/FP64 without rounding control; the certified
// value U(a) at the final slopes is computed in FP64 with an explicit error
// bound (lin_certify).
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace ibp {

constexpr double kU64Lin = 1.1102230246251565e-16;  // 2^-53

// slope of a device's PWL curve at x (right segment at a breakpoint)
__device__ __forceinline__ double lin_pwl_slope(const double *s, const double *b, int n, double x) {
    if (x < b[0]) return 0.0;
    int i = 0;
    while (i + 1 < n && b[i + 1] <= x) ++i;
    return s[i];
}

// value of the ReLU chain of eqs. (single ReLU), (combined ReLUs) at x,
// rounded up (up) or down
__device__ __forceinline__ double lin_pwl_value(const double *a, const double *b, int n, double x, bool up) {
    double F = 0.0, U = 0.0;
    for (int m = 0; m < n; ++m) {
        if (up) F = __dadd_ru(F, __dmul_ru(a[m], fmax(__dsub_ru(x, b[m]), 0.0)));
        else F = __dadd_rd(F, __dmul_rd(a[m], fmax(__dsub_rd(x, b[m]), 0.0)));
        if (m + 1 < n) {
            U = up ? __dadd_ru(U, __dmul_ru(a[m], __dsub_ru(b[m + 1], b[m])))
                   : __dadd_rd(U, __dmul_rd(a[m], __dsub_rd(b[m + 1], b[m])));
            F = fmin(F, U);
        }
    }
    return F;
}

template <bool UP>
__device__ __forceinline__ double block_sum_d(double v, double *sh) {
    v = UP ? warp_sum_ru(v) : warp_sum_rd(v);
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = UP ? __dadd_ru(t, sh[i]) : __dadd_rd(t, sh[i]);
    return t;  // in thread 0
}

// ------------------------------------------------------------------ x step
// Thread per (device, box): projected gradient ascent on x and the
// extrapolated point xb = 2 x_new - x.
__global__ void __launch_bounds__(128) k_lin_x(const LinArgs a) {
    const int j = blockIdx.y, d = blockIdx.x * blockDim.x + threadIdx.x;
    double part = 0.0;  // this block's share of the total injection of xb
    if (d < a.n_dev) {
        const size_t o = (size_t)j * a.n_dev + d;
        const bool gen = d < a.n_gen;
        const double sg = gen ? 1.0 : -1.0;
        const double xo = a.x[o];
        const int col = a.dev_col[d];
        const double gb = col >= 0 ? (double)a.g[(size_t)j * a.n_a_pad + col] : 0.0;
        const int s0 = a.seg_ptr[d], ns = a.seg_ptr[d + 1] - s0;
        const double sl = lin_pwl_slope(a.slope + s0, a.bkpt + s0, ns, xo);
        const double grad = (gen ? -sl : sl) - sg * (gb + a.zeta_inj * a.a0[j]);
        const double xn = fmin(fmax(xo + (a.pc_tau[d] / a.w[j]) * grad, a.box_lo[o]), a.box_hi[o]);
        const double xbn = 2.0 * xn - xo;
        a.xb[o] = xbn;
        a.x[o] = xn;
        a.sx[o] += xn;
        part = sg * xbn;
    }
    __shared__ double sh[4];
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0)
        a.stot_part[(size_t)j * gridDim.x + blockIdx.x] = sh[0] + sh[1] + sh[2] + sh[3];
}

// Thread per (active column, box): the bus injection of xb; block 0 of each
// box also adds k_lin_x's per-block partials of the total injection, in
// block order
__global__ void __launch_bounds__(128) k_lin_p(const LinArgs a) {
    const int j = blockIdx.y, col = blockIdx.x * blockDim.x + threadIdx.x;
    const double *xb = a.xb + (size_t)j * a.n_dev;
    if (col < a.n_a_pad) {
        double v = 0.0;
        if (col < a.n_a)
            for (int q = a.act_ptr[col]; q < a.act_ptr[col + 1]; ++q) {
                const int d = a.act_dev[q];
                v += (d < a.n_gen ? 1.0 : -1.0) * xb[d];
            }
        a.p[(size_t)j * a.n_a_pad + col] = (float)v;
    }
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int nb = (a.n_dev + 127) / 128;
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += a.stot_part[(size_t)j * nb + b];
    a.stot[j] = t;
}

// base flows f = Phi p of xb: one warp per (line, box)
__global__ void __launch_bounds__(256) k_lin_flows(const LinArgs a) {
    const int j = blockIdx.y;
    const int l = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (l >= a.n_l) return;
    const float4 *row = reinterpret_cast<const float4 *>(a.phi + (size_t)l * a.n_a_pad);
    const float4 *p = reinterpret_cast<const float4 *>(a.p + (size_t)j * a.n_a_pad);
    float s = 0.0f;
    for (int v = lane; v < (a.n_a_pad >> 2); v += 32) {
        const float4 r = __ldg(&row[v]), q = p[v];
        s = fmaf(r.x, q.x, fmaf(r.y, q.y, fmaf(r.z, q.z, fmaf(r.w, q.w, s))));
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) a.f[(size_t)j * a.n_l + l] = s;
}

__device__ __forceinline__ float lin_prox(float v, float thr) {
    // soft threshold by thr (the prox of thr |.|), then the projection on [-1, 1]
    const float t = fminf(fmaxf(fabsf(v) - thr, 0.0f), 1.0f);
    return copysignf(t, v);
}

// V consecutive floats (V = 1, 2, 4): one aligned vector load or store
template <int V>
struct VecF {
    float v[V];
    __device__ __forceinline__ void load(const float *p) {
        if constexpr (V == 4) {
            const float4 t = *reinterpret_cast<const float4 *>(p);
            v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
        } else if constexpr (V == 2) {
            const float2 t = *reinterpret_cast<const float2 *>(p);
            v[0] = t.x; v[1] = t.y;
        } else {
            v[0] = *p;
        }
    }
    __device__ __forceinline__ void load_ro(const float *p) {
        if constexpr (V == 4) {
            const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
            v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
        } else if constexpr (V == 2) {
            const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
            v[0] = t.x; v[1] = t.y;
        } else {
            v[0] = __ldg(p);
        }
    }
    __device__ __forceinline__ void store(float *p) const {
        if constexpr (V == 4) *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
        else if constexpr (V == 2) *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
        else *p = v[0];
    }
};

// Dual step on the slopes: block (x: 256 threads of V adjacent lines each,
// y: 32 / V contingencies, z: box), so a thread takes 32 pairs whatever V;
// n_l is a multiple of V, so every row of L and of the slopes starts
// V-aligned.  Blocks with y == 0 also take the base flows, block (0, 0) the
// imbalance.  Accumulates the line weights' column sums and the rows' dot
// products with L.  The block's outaged-line flows and S values are staged in
// shared memory, and each group of G contingencies
// loads its L and slopes before storing any.  A pair's step (z_f times its
// dual step size times the primal weight) is w / (S_l + |L_lk| S_k).
template <int V>
__global__ void __launch_bounds__(256, 3) k_lin_pairs(const LinArgs a) {
    constexpr int KB = 32 / V;  // contingencies per block
    constexpr int G = 8 / V;    // contingencies per load group (8 / V vectors of V lines)
    const int j = blockIdx.z;
    const int l0 = (blockIdx.x * 256 + threadIdx.x) * V;
    const int k0 = blockIdx.y * KB;
    const float w = (float)a.w[j];
    const float *f = a.f + (size_t)j * a.n_l;
    __shared__ float fk_s[KB], sk_s[KB];
    if (threadIdx.x < KB) {
        const int k = k0 + threadIdx.x;
        const int kl = k < a.n_c ? __ldg(&a.ctg_line[k]) : 0;
        fk_s[threadIdx.x] = k < a.n_c ? f[kl] : 0.0f;
        sk_s[threadIdx.x] = k < a.n_c ? a.pc_S[kl] : 0.0f;
    }
    __syncthreads();
    const bool lv = l0 < a.n_l;
    float fl[V], Sl[V], Rc[V], col[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        fl[v] = lv ? f[l0 + v] : 0.0f;
        Sl[v] = lv ? a.pc_S[l0 + v] : 1.0f;
        Rc[v] = lv ? (float)a.rate_c64[l0 + v] : 0.0f;
        col[v] = 0.0f;
    }
    __shared__ float sh[8][33];
    const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int g = 0; g < KB / G; ++g) {
        VecF<V> Lt[G], av[G];
        float rowv[G];
#pragma unroll
        for (int u = 0; u < G; ++u) {
            const int k = k0 + g * G + u;
            if (lv && k < a.n_c) {
                Lt[u].load_ro(a.lodf + (size_t)k * a.n_l + l0);
                av[u].load(a.a_c + ((size_t)j * a.n_c + k) * a.n_l + l0);
            }
        }
#pragma unroll
        for (int u = 0; u < G; ++u) {
            const int kk = g * G + u, k = k0 + kk;
            float r = 0.0f;
            if (lv && k < a.n_c) {
                VecF<V> an;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const float L = Lt[u].v[v];
                    const float fc = fmaf(L, fk_s[kk], fl[v]);
                    const float gain = __fdividef(w, fmaf(fabsf(L), sk_s[kk], Sl[v]));
                    an.v[v] = lin_prox(fmaf(gain, fc, av[u].v[v]), gain * Rc[v]);
                    col[v] += an.v[v];
                    r = fmaf(an.v[v], L, r);
                }
                an.store(a.a_c + ((size_t)j * a.n_c + k) * a.n_l + l0);
            }
            rowv[u] = r;
        }
        // the warp's share of the G rows' dot products with L
#pragma unroll
        for (int u = 0; u < G; ++u) {
            float r = rowv[u];
            for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
            if (lane == 0) sh[wp][g * G + u] = r;
        }
    }
    __syncthreads();
    if (threadIdx.x < KB && k0 + threadIdx.x < a.n_c) {
        float t = 0.0f;
        for (int i = 0; i < 8; ++i) t += sh[i][threadIdx.x];
        atomicAdd(&a.rowdot[(size_t)j * a.n_c + k0 + threadIdx.x], t);
    }
    if (!lv) return;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int l = l0 + v;
        if (blockIdx.y == 0) {
            const size_t o = (size_t)j * a.n_l + l;
            const float gain = __fdividef(w, Sl[v]);
            const float an = lin_prox(fmaf(gain, fl[v], a.a_b[o]), gain * (float)a.rate64[l]);
            a.a_b[o] = an;
            col[v] += an;
        }
        atomicAdd(&a.colsum[(size_t)j * a.n_l + l], col[v]);
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        // z_inj times the imbalance's step 1 / (z_inj n_dev) times w
        a.a0[j] = fmin(fmax(a.a0[j] + a.w[j] * a.stot[j] / (double)a.n_dev, -1.0), 1.0);
    }
}

// g_b = z_f sum_l W_l Phi[l][b]: a thread takes 4 adjacent columns (one
// 16-byte load per line) and a block row 32 lines, whose weights W_l =
// colsum_l + the row dots of the contingencies of line l it forms first in
// shared memory; atomics into g
constexpr int kLinGLines = 32;
__global__ void __launch_bounds__(128) k_lin_g(const LinArgs a) {
    const int j = blockIdx.z, c4 = blockIdx.x * blockDim.x + threadIdx.x;
    const int l0 = blockIdx.y * kLinGLines, l1 = min(l0 + kLinGLines, a.n_l);
    __shared__ float W[kLinGLines];
    if (threadIdx.x < kLinGLines) {
        const int l = l0 + threadIdx.x;
        float t = 0.0f;
        if (l < a.n_l) {
            t = a.colsum[(size_t)j * a.n_l + l];
            for (int q = a.cl_ptr[l]; q < a.cl_ptr[l + 1]; ++q) t += a.rowdot[(size_t)j * a.n_c + a.cl_ctg[q]];
        }
        W[threadIdx.x] = t;
    }
    __syncthreads();
    if (4 * c4 >= a.n_a_pad) return;
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll 8
    for (int l = l0; l < l1; ++l) {
        const float w = W[l - l0];
        const float4 ph = __ldg(reinterpret_cast<const float4 *>(a.phi + (size_t)l * a.n_a_pad) + c4);
        acc.x = fmaf(w, ph.x, acc.x);
        acc.y = fmaf(w, ph.y, acc.y);
        acc.z = fmaf(w, ph.z, acc.z);
        acc.w = fmaf(w, ph.w, acc.w);
    }
    float *g = a.g + (size_t)j * a.n_a_pad + 4 * c4;
    const float zf = (float)a.zeta_f;
    if (acc.x != 0.0f) atomicAdd(g, zf * acc.x);
    if (acc.y != 0.0f) atomicAdd(g + 1, zf * acc.y);
    if (acc.z != 0.0f) atomicAdd(g + 2, zf * acc.z);
    if (acc.w != 0.0f) atomicAdd(g + 3, zf * acc.w);
}

cudaError_t lin_iteration(const LinArgs &a, int num_sms, cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(a.colsum, 0, (size_t)a.n_box * a.n_l * sizeof(float), s)) != cudaSuccess) return e;
    if (a.n_c > 0 &&
        (e = cudaMemsetAsync(a.rowdot, 0, (size_t)a.n_box * a.n_c * sizeof(float), s)) != cudaSuccess)
        return e;
    k_lin_x<<<dim3((a.n_dev + 127) / 128, a.n_box), 128, 0, s>>>(a);
    k_lin_p<<<dim3((a.n_a_pad + 127) / 128, a.n_box), 128, 0, s>>>(a);
    k_lin_flows<<<dim3((a.n_l + 7) / 8, a.n_box), 256, 0, s>>>(a);
    const dim3 gp4((a.n_l / 4 + 255) / 256, std::max((a.n_c + 7) / 8, 1), a.n_box);
    const dim3 gp2((a.n_l / 2 + 255) / 256, std::max((a.n_c + 15) / 16, 1), a.n_box);
    const dim3 gp1((a.n_l + 255) / 256, std::max((a.n_c + 31) / 32, 1), a.n_box);
    if (a.n_l % 4 == 0) k_lin_pairs<4><<<gp4, 256, 0, s>>>(a);
    else if (a.n_l % 2 == 0) k_lin_pairs<2><<<gp2, 256, 0, s>>>(a);
    else k_lin_pairs<1><<<gp1, 256, 0, s>>>(a);
    if ((e = cudaMemsetAsync(a.g, 0, (size_t)a.n_box * a.n_a_pad * sizeof(float), s)) != cudaSuccess) return e;
    k_lin_g<<<dim3((a.n_a_pad / 4 + 127) / 128, (a.n_l + kLinGLines - 1) / kLinGLines, a.n_box), 128, 0, s>>>(a);
    return cudaGetLastError();
}

// the dual gradient g = z_f Phi^T W of the current slopes (no step)
__global__ void k_lin_colsum_state(const LinArgs a) {
    const int j = blockIdx.y, l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= a.n_l) return;
    float t = a.a_b[(size_t)j * a.n_l + l];
    for (int k = 0; k < a.n_c; ++k) t += a.a_c[((size_t)j * a.n_c + k) * a.n_l + l];
    a.colsum[(size_t)j * a.n_l + l] = t;
}
__global__ void __launch_bounds__(256) k_lin_rowdot_state(const LinArgs a) {
    const int j = blockIdx.y, k = blockIdx.x;
    float t = 0.0f;
    for (int l = threadIdx.x; l < a.n_l; l += blockDim.x)
        t = fmaf(a.a_c[((size_t)j * a.n_c + k) * a.n_l + l], __ldg(&a.lodf[(size_t)k * a.n_l + l]), t);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    __shared__ float sh[8];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
        a.rowdot[(size_t)j * a.n_c + k] = s;
    }
}

cudaError_t lin_gradient(const LinArgs &a, int num_sms, cudaStream_t s) {
    k_lin_colsum_state<<<dim3((a.n_l + 255) / 256, a.n_box), 256, 0, s>>>(a);
    if (a.n_c > 0) k_lin_rowdot_state<<<dim3(a.n_c, a.n_box), 256, 0, s>>>(a);
    cudaError_t e = cudaMemsetAsync(a.g, 0, (size_t)a.n_box * a.n_a_pad * sizeof(float), s);
    if (e != cudaSuccess) return e;
    k_lin_g<<<dim3((a.n_a_pad / 4 + 127) / 128, (a.n_l + kLinGLines - 1) / kLinGLines, a.n_box), 128, 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ restarts
// The averaged point of the window (x_avg), and the step-weighted squared
// moves of x and of the slopes since the last restart (red[j][0], red[j][1]);
// the references move to the current iterate and the running sum restarts.
__global__ void k_lin_avg(const LinArgs a) {
    const int j = blockIdx.y;
    const double inv = 1.0 / (double)a.n_avg;
    const size_t npair = (size_t)a.n_c * a.n_l;
    const size_t tot = (size_t)a.n_dev + a.n_l + npair + 1;
    double dx = 0.0, da = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
        if (i < (size_t)a.n_dev) {
            const size_t o = (size_t)j * a.n_dev + i;
            const double v = a.x[o];
            dx += (v - a.x_last[o]) * (v - a.x_last[o]) / a.pc_tau[i];
            a.x_last[o] = v;
            a.x_avg[o] = a.sx[o] * inv;
            a.sx[o] = 0.0;
        } else if (i < (size_t)a.n_dev + a.n_l) {
            const int l = (int)(i - a.n_dev);
            const size_t o = (size_t)j * a.n_l + l;
            const float v = a.a_b[o];
            da += (double)(v - a.b_last[o]) * (double)(v - a.b_last[o]) * a.zeta_f * (double)a.pc_S[l];
            a.b_last[o] = v;
        } else if (i < (size_t)a.n_dev + a.n_l + npair) {
            const size_t q = i - a.n_dev - a.n_l;
            const size_t o = (size_t)j * npair + q;
            const int k = (int)(q / a.n_l), l = (int)(q % a.n_l);
            const double wgt = a.zeta_f * ((double)a.pc_S[l] +
                                           fabs((double)a.lodf[q]) * (double)a.pc_S[a.ctg_line[k]]);
            const float v = a.a_c[o];
            da += (double)(v - a.c_last[o]) * (double)(v - a.c_last[o]) * wgt;
            a.c_last[o] = v;
        } else {
            const double v = a.a0[j];
            da += (v - a.a0_last[j]) * (v - a.a0_last[j]) * a.zeta_inj * (double)a.n_dev;
            a.a0_last[j] = v;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        dx += __shfl_xor_sync(0xffffffffu, dx, o);
        da += __shfl_xor_sync(0xffffffffu, da, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&a.red[(size_t)j * 4], dx);
        atomicAdd(&a.red[(size_t)j * 4 + 1], da);
    }
}

// primal weight <- exp(0.5 log(|Delta a| / |Delta x|) + 0.5 log w)
__global__ void k_lin_weight(const LinArgs a) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.n_box) return;
    const double dx = sqrt(a.red[(size_t)j * 4]), da = sqrt(a.red[(size_t)j * 4 + 1]);
    if (dx > 1e-12 && da > 1e-12) a.w[j] = exp(0.5 * log(da / dx) + 0.5 * log(a.w[j]));
    a.red[(size_t)j * 4] = 0.0;
    a.red[(size_t)j * 4 + 1] = 0.0;
}

cudaError_t lin_restart(const LinArgs &a, int num_sms, cudaStream_t s) {
    if (a.n_avg <= 0) return cudaSuccess;
    k_lin_avg<<<dim3(num_sms * 4, a.n_box), 256, 0, s>>>(a);
    k_lin_weight<<<(a.n_box + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ certified value
// Column pass (thread per line): W_l = a_l + sum_k a_kl (round to nearest),
// Wabs_l = |a_l| + sum_k |a_kl| (round up), constl_l = |a_l| R_l + Rc_l sum_k |a_kl|
// (round up).
__global__ void k_cert_col(const LinArgs a) {
    const int j = blockIdx.y, l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= a.n_l) return;
    double cs = 0.0, ca = 0.0;
    for (int k = 0; k < a.n_c; ++k) {
        const double v = (double)a.a_c[((size_t)j * a.n_c + k) * a.n_l + l];
        cs += v;
        ca = __dadd_ru(ca, fabs(v));
    }
    const double ab = (double)a.a_b[(size_t)j * a.n_l + l];
    const size_t o = (size_t)j * a.n_l + l;
    a.W64[o] = ab + cs;
    a.Wabs[o] = __dadd_ru(fabs(ab), ca);
    a.constl[o] = __dadd_ru(__dmul_ru(fabs(ab), a.rate64[l]), __dmul_ru(ca, a.rate_c64[l]));
}

// Row pass (block per contingency): rd_k = sum_l a_kl L[l,k], rda_k = sum_l |a_kl| |L[l,k]|
// with the FP64 LODF L~ + L_lo
__global__ void __launch_bounds__(256) k_cert_row(const LinArgs a) {
    const int j = blockIdx.y, k = blockIdx.x;
    double rd = 0.0, rda = 0.0;
    for (int l = threadIdx.x; l < a.n_l; l += blockDim.x) {
        const size_t q = (size_t)k * a.n_l + l;
        const double L = (double)a.lodf[q] + (a.lodf_lo ? (double)a.lodf_lo[q] : 0.0);
        const double v = (double)a.a_c[((size_t)j * a.n_c + k) * a.n_l + l];
        rd = fma(v, L, rd);
        rda = __fma_ru(fabs(v), fabs(L), rda);
    }
    __shared__ double sh[8];
    double t = rd;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
        a.rd64[(size_t)j * a.n_c + k] = s;
    }
    const double ra = block_sum_d<true>(rda, sh);
    if (threadIdx.x == 0) a.rda[(size_t)j * a.n_c + k] = ra;
}

__global__ void k_cert_W(const LinArgs a) {
    const int j = blockIdx.y, l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= a.n_l) return;
    const size_t o = (size_t)j * a.n_l + l;
    double w = a.W64[o], wa = a.Wabs[o];
    for (int q = a.cl_ptr[l]; q < a.cl_ptr[l + 1]; ++q) {
        const int k = a.cl_ctg[q];
        w += a.rd64[(size_t)j * a.n_c + k];
        wa = __dadd_ru(wa, a.rda[(size_t)j * a.n_c + k]);
    }
    a.W64[o] = w;
    a.Wabs[o] = wa;
}

// column b: g64_b = sum_l W_l Phi[l][b] (FP64 PTDF), G64_b = sum_l Wabs_l |Phi[l][b]| (round up)
__global__ void k_cert_g(const LinArgs a) {
    const int j = blockIdx.y, col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= a.n_a_pad) return;
    double g = 0.0, G = 0.0;
    for (int l = 0; l < a.n_l; ++l) {
        const double ph = a.phi64[(size_t)l * a.n_a_pad + col];
        g = fma(a.W64[(size_t)j * a.n_l + l], ph, g);
        G = __fma_ru(a.Wabs[(size_t)j * a.n_l + l], fabs(ph), G);
    }
    a.g64[(size_t)j * a.n_a_pad + col] = g;
    a.G64[(size_t)j * a.n_a_pad + col] = G;
}

// one block per box: U(a) = z_f sum |a| R + sum_i max_x [phi_i(x) + c_i x], with the
// error of c_i (from W and g64) taken at |x|, all rounded up
__global__ void __launch_bounds__(256) k_cert_ub(const LinArgs a) {
    const int j = blockIdx.x;
    __shared__ double sh[8];
    // relative error of g64 against the exact Phi^T W: the column sums (n_c terms),
    // the row dots (n_l terms), the GEMV (n_l terms), the FP64 LODF (2^-47)
    const double gam = __fma_ru((double)(2 * a.n_l + a.n_c + 64), 1.01 * kU64Lin, 2.842170943040401e-14);
    double cst = 0.0;
    for (int l = threadIdx.x; l < a.n_l; l += blockDim.x) cst = __dadd_ru(cst, a.constl[(size_t)j * a.n_l + l]);
    cst = block_sum_d<true>(cst, sh);
    __shared__ double cst_s;
    if (threadIdx.x == 0) cst_s = __dmul_ru(a.zeta_f, cst);
    __syncthreads();
    const double a0 = a.a0[j];
    double sum = 0.0, err = 0.0, mag = 0.0;
    for (int d = threadIdx.x; d < a.n_dev; d += blockDim.x) {
        const bool gen = d < a.n_gen;
        const int col = a.dev_col[d];
        const double g = col >= 0 ? a.g64[(size_t)j * a.n_a_pad + col] : 0.0;
        const double G = col >= 0 ? a.G64[(size_t)j * a.n_a_pad + col] : 0.0;
        // c_i = -s_i (z_f g + z_inj a0), and a bound on its error
        const double lin = (gen ? -1.0 : 1.0) * fma(a.zeta_f, g, a.zeta_inj * a0);
        const double e = __fma_ru(__dmul_ru(a.zeta_f, gam), G,
                                  __dmul_ru(4.0 * kU64Lin, __dadd_ru(fabs(a.zeta_f * g), fabs(a.zeta_inj * a0))));
        const double lo = a.box_lo[(size_t)j * a.n_dev + d], hi = a.box_hi[(size_t)j * a.n_dev + d];
        const int s0 = a.seg_ptr[d], ns = a.seg_ptr[d + 1] - s0;
        const double *sl = a.slope + s0, *bk = a.bkpt + s0;
        // candidates: the endpoints and the breakpoints inside the interval
        double best = -INFINITY;
        for (int c = -2; c < ns; ++c) {
            const double xv = c == -2 ? lo : (c == -1 ? hi : bk[c]);
            if (xv < lo || xv > hi) continue;
            // phi_i rounded up: the load value up, minus the generator cost rounded down
            const double ph = gen ? -lin_pwl_value(sl, bk, ns, xv, false) : lin_pwl_value(sl, bk, ns, xv, true);
            const double v = __dadd_ru(__dadd_ru(ph, __dmul_ru(lin, xv)), __dmul_ru(e, fabs(xv)));
            best = fmax(best, v);
        }
        sum = __dadd_ru(sum, best);
        err = __dadd_ru(err, __dmul_ru(e, fmax(fabs(lo), fabs(hi))));
        mag = __dadd_ru(mag, fabs(best));
    }
    sum = block_sum_d<true>(sum, sh);
    const double es = block_sum_d<true>(err, sh);
    const double ms = block_sum_d<true>(mag, sh);
    if (threadIdx.x == 0) {
        const double u = __dadd_ru(cst_s, sum);
        a.ub[j] = u;
        a.ub_err[j] = __fma_ru(1e-12, __dadd_ru(fabs(cst_s), ms), __dmul_ru(2.0, es));
    }
}

cudaError_t lin_certify(const LinArgs &a, int num_sms, cudaStream_t s) {
    k_cert_col<<<dim3((a.n_l + 255) / 256, a.n_box), 256, 0, s>>>(a);
    if (a.n_c > 0) k_cert_row<<<dim3(a.n_c, a.n_box), 256, 0, s>>>(a);
    k_cert_W<<<dim3((a.n_l + 255) / 256, a.n_box), 256, 0, s>>>(a);
    k_cert_g<<<dim3((a.n_a_pad + 127) / 128, a.n_box), 128, 0, s>>>(a);
    k_cert_ub<<<a.n_box, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ preconditioner
// S_l = sum over active columns of |Phi[l,col]| times the column's device
// count (one warp per line); a row no active bus reaches keeps S = 1
__global__ void k_pc_rows(const LinArgs a, float *S) {
    const int l = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (l >= a.n_l) return;
    double t = 0.0;
    for (int col = lane; col < a.n_a; col += 32)
        t += fabs((double)a.phi[(size_t)l * a.n_a_pad + col]) * (double)(a.act_ptr[col + 1] - a.act_ptr[col]);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) S[l] = t > 0.0 ? (float)t : 1.0f;
}
// Lsum_k = sum_l |L[l,k]| (one warp per contingency)
__global__ void k_pc_lsum(const LinArgs a, double *Lsum) {
    const int k = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (k >= a.n_c) return;
    double t = 0.0;
    for (int l = lane; l < a.n_l; l += 32) t += fabs((double)a.lodf[(size_t)k * a.n_l + l]);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) Lsum[k] = t;
}
// column col: A = sum_l |Phi[l,col]|, B = sum_k |Phi[line of k, col]| Lsum_k
__global__ void k_pc_cols(const LinArgs a, const double *Lsum, double *A, double *B) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= a.n_a_pad) return;
    double sa = 0.0, sb = 0.0;
    for (int l = 0; l < a.n_l; ++l) sa += fabs((double)a.phi[(size_t)l * a.n_a_pad + col]);
    for (int k = 0; k < a.n_c; ++k)
        sb += fabs((double)a.phi[(size_t)a.ctg_line[k] * a.n_a_pad + col]) * Lsum[k];
    A[col] = sa;
    B[col] = sb;
}
// tau[d] = 1 / (z_f (A (1 + n_c) + B) + z_inj): the inverse of the bound on
// the column sum of |D K| (the sum over pairs of |H_k[l,b]| is at most
// n_c A + B)
__global__ void k_pc_tau(const LinArgs a, const double *A, const double *B, double *tau) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= a.n_dev) return;
    const int col = a.dev_col[d];
    const double cs = col >= 0 ? a.zeta_f * (A[col] * (1.0 + a.n_c) + B[col]) : 0.0;
    tau[d] = 1.0 / (cs + a.zeta_inj);
}

cudaError_t lin_precondition(const LinArgs &a, float *S, double *tau, double *A, double *B, double *Lsum,
                             cudaStream_t s) {
    k_pc_rows<<<(a.n_l + 7) / 8, 256, 0, s>>>(a, S);
    if (a.n_c > 0) k_pc_lsum<<<(a.n_c + 7) / 8, 256, 0, s>>>(a, Lsum);
    k_pc_cols<<<(a.n_a_pad + 127) / 128, 128, 0, s>>>(a, Lsum, A, B);
    k_pc_tau<<<(a.n_dev + 127) / 128, 128, 0, s>>>(a, A, B, tau);
    return cudaGetLastError();
}

}  // namespace ibp
