// Adjoints of the certified bounds obj_hi and obj_lo with respect to the box
// endpoints and the line ratings (not certified: FP32 products, FP64 sums).
//
// obj_hi = C(pd_hi) - G(pg_lo) - z_inj s_inj,lo - z_f (sum_l s_fb,lo + sum_{k,l} s_fc,lo)
// (eq. (penalized-objective) under eq. (IBP)).  With A the set of certified
// active pairs, s_lo = |c_kl| - r_kl - rating_l > 0 (base lines included with
// H = Phi), the derivative is
//   d obj_hi / d c_b = -z_f sum_A sgn(c_kl) H_k[l,b],
//   d obj_hi / d r_b = +z_f sum_A |H_k[l,b]|,
//   d obj_hi / d rating_l = +z_f #{pairs of A on line l},
// and sum_A sgn H_k[l,b] = sum_x W_x Phi[x,b] with line weights
//   W_l += sgn, W_{line of k} += sgn L[l,k]  (H_k = Phi + L[:,k] Phi[k,:]).
// An entry (l, -1, m, sgn) stands for m pairs of a bridge line, whose
// contingency flows all equal its base flow (H_k[l,:] = Phi[l,:]).
//
// obj_lo = C(pd_lo) - G(pg_hi) - z_inj s_inj,hi - z_f (sum s_fb,hi + sum s_fc,hi)
// takes the upper violation bounds s_hi = |c| + r - rating > 0 (its active
// set A', recorded by the same forward kernels); the same kernels give
//   d obj_lo / d c_b = -z_f sum_A' sgn(c_kl) H_k[l,b],
//   d obj_lo / d r_b = -z_f sum_A' |H_k[l,b]|,
//   d obj_lo / d rating_l = +z_f #{pairs of A' on line l},
// and s_inj,hi = max(-P_lo, P_hi) with the device endpoints of the total
// injection.  A' holds most pairs of a wide box, so its radius pass sums each
// chunk of entries in FP32 before the FP64 sum (the order of a chunk's
// entries, and so the last bits, then follow the forward kernel's atomics).
// The imbalance term and the monotone cost curves act on the device
// endpoints directly.  Kernels, in order: weights, centre GEMV, radius pass,
// chain rule to the box endpoints.
#include "common.cuh"
#include "internal.h"

namespace ibp {

constexpr int kEntryChunk = 128;
constexpr int kEntryBlocks = 64;

// Each pass is a body over (box, block coordinates), run by a one-case kernel
// (the box from the grid) and by a many-case kernel whose grid rows walk a
// table of (case, box) items with the cases' arguments in device memory.
__device__ __forceinline__ void bwd_weights_body(const BwdArgs &a, int box, int bx, int nbx) {
    const int n = min(a.act_count[box], a.act_cap);
    const int4 *list = a.act_list + (size_t)box * a.act_cap;
    double *W = a.W + (size_t)box * a.n_l;
    int *cnt = a.cnt + (size_t)box * a.n_l;
    for (int i = bx * blockDim.x + threadIdx.x; i < n; i += nbx * blockDim.x) {
        const int4 e = list[i];
        const float sg = __int_as_float(e.w);
        if (e.y < 0) {  // a bridge line, m contingency pairs at once
            const float m = __int_as_float(e.z);
            atomicAdd(&W[e.x], (double)sg * (double)m);
            atomicAdd(&cnt[e.x], (int)m);
            continue;
        }
        const float L = __int_as_float(e.z);
        atomicAdd(&W[e.x], (double)sg);
        if (L != 0.0f) atomicAdd(&W[e.y], (double)sg * (double)L);
        atomicAdd(&cnt[e.x], 1);
    }
}

__global__ void k_bwd_weights(BwdArgs a) { bwd_weights_body(a, blockIdx.y, blockIdx.x, gridDim.x); }

__global__ void k_bwd_weights_cases(const BwdArgs *__restrict__ args, const int2 *__restrict__ items) {
    const int2 it = items[blockIdx.y];
    bwd_weights_body(args[it.x], it.y, blockIdx.x, gridDim.x);
}

// dc[box][col] = sum_l W[box][l] Phi[l][col]  (lines with W = 0 are skipped);
// block row y takes lines [y n_l / kCenterSplit, (y + 1) n_l / kCenterSplit)
// and adds its sum into dc (zeroed by the caller)
constexpr int kCenterSplit = 32;

__device__ __forceinline__ void bwd_center_body(const BwdArgs &a, int box, int bx, int by) {
    const int col = bx * blockDim.x + threadIdx.x;
    const double *W = a.W + (size_t)box * a.n_l;
    const int l0 = (int)((long long)by * a.n_l / kCenterSplit);
    const int l1 = (int)((long long)(by + 1) * a.n_l / kCenterSplit);
    double acc = 0.0;
    if (col < a.n_a_pad) {
        for (int l = l0; l < l1; ++l) {
            const double w = W[l];
            if (w != 0.0) acc = fma(w, (double)__ldg(&a.phi[(size_t)l * a.n_a_pad + col]), acc);
        }
        if (acc != 0.0) atomicAdd(&a.dc[(size_t)box * a.n_a_pad + col], acc);
    }
}

__global__ void k_bwd_center(BwdArgs a) { bwd_center_body(a, blockIdx.z, blockIdx.x, blockIdx.y); }

__global__ void k_bwd_center_cases(const BwdArgs *__restrict__ args, const int2 *__restrict__ items) {
    const int2 it = items[blockIdx.z];
    const BwdArgs &a = args[it.x];
    if ((int)(blockIdx.x * blockDim.x) >= a.n_a_pad) return;  // columns of a wider case
    bwd_center_body(a, it.y, blockIdx.x, blockIdx.y);
}

// dr[box][col] += sum over a chunk of entries of |Phi[l][col] + L Phi[kline][col]|
__device__ __forceinline__ void bwd_radius_body(const BwdArgs &a, int box, int bx, int by, int nby) {
    const int col = bx * blockDim.x + threadIdx.x;
    const int n = min(a.act_count[box], a.act_cap);
    const int4 *list = a.act_list + (size_t)box * a.act_cap;
    if (col >= a.n_a_pad) return;
    // obj_hi's sparse set: FP64 sums, since the list order depends on the
    // forward pass's atomics and the result should not depend on how the
    // entries are grouped
    double tot = 0.0;
    for (int c0 = by * kEntryChunk; c0 < n; c0 += nby * kEntryChunk) {
        const int c1 = min(c0 + kEntryChunk, n);
        float part = 0.0f;  // obj_lo's dense set: FP32 within a chunk
        for (int i = c0; i < c1; ++i) {
            const int4 e = list[i];
            float v;
            if (e.y < 0) {  // a bridge line, m contingency pairs at once
                const double m = (double)__int_as_float(e.z) *
                                 (double)fabsf(__ldg(&a.phi[(size_t)e.x * a.n_a_pad + col]));
                tot += m;
                continue;
            }
            const float L = __int_as_float(e.z);
            const float h = __fmaf_rn(L, __ldg(&a.phi[(size_t)e.y * a.n_a_pad + col]),
                                      __ldg(&a.phi[(size_t)e.x * a.n_a_pad + col]));
            v = fabsf(h);
            if (a.side) part += v;
            else tot += (double)v;
        }
        tot += (double)part;
    }
    if (tot != 0.0) atomicAdd(&a.dr[(size_t)box * a.n_a_pad + col], tot);
}

__global__ void k_bwd_radius(BwdArgs a) { bwd_radius_body(a, blockIdx.z, blockIdx.x, blockIdx.y, gridDim.y); }

__global__ void k_bwd_radius_cases(const BwdArgs *__restrict__ args, const int2 *__restrict__ items) {
    const int2 it = items[blockIdx.z];
    const BwdArgs &a = args[it.x];
    if ((int)(blockIdx.x * blockDim.x) >= a.n_a_pad) return;
    bwd_radius_body(a, it.y, blockIdx.x, blockIdx.y, gridDim.y);
}

// zero the per-box accumulators of every item (and, before the forward
// pass, the active-pair counts of its side)
__global__ void k_bwd_zero_cases(const BwdArgs *__restrict__ args, const int2 *__restrict__ items,
                                 int counts) {
    const int2 it = items[blockIdx.y];
    const BwdArgs &a = args[it.x];
    const int t = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    const size_t ol = (size_t)it.y * a.n_l, oa = (size_t)it.y * a.n_a_pad;
    for (int i = t; i < a.n_l; i += nt) {
        a.W[ol + i] = 0.0;
        a.cnt[ol + i] = 0;
    }
    for (int i = t; i < a.n_a_pad; i += nt) {
        a.dc[oa + i] = 0.0;
        a.dr[oa + i] = 0.0;
    }
    if (counts && t == 0) const_cast<int *>(a.act_count)[it.y] = 0;
}

__device__ __forceinline__ double pwl_slope(const double *s, const double *b, int n, double x) {
    // slope of the segment that contains x (the right one at a breakpoint)
    if (x < b[0]) return 0.0;
    int i = 0;
    while (i + 1 < n && b[i + 1] <= x) ++i;
    return s[i];
}

// one block per box: chain rule to the device endpoints, costs, imbalance
__global__ void __launch_bounds__(256) k_bwd_chain(BwdArgs a) {
    const int box = blockIdx.x;
    const double *lo = a.box_lo + (size_t)box * a.n_dev;
    const double *hi = a.box_hi + (size_t)box * a.n_dev;
    // an active-pair list that overflowed its capacity holds only part of the
    // pairs: the box's gradients are then NaN unless its incoming gradient is
    // 0 (the error word says IBP_ENOMEM either way)
    const double g0 = a.grad_obj_hi[box];
    const double g = (a.act_count[box] > a.act_cap && g0 != 0.0) ? __longlong_as_double(0x7ff8000000000000ll)
                                                                  : g0;
    const bool lo_side = a.side != 0;
    // total injection interval [plo, phi] (imbalance at the slack)
    double plo = 0.0, phi = 0.0;
    for (int d = threadIdx.x; d < a.n_dev; d += blockDim.x) {
        if (d < a.n_gen) {
            plo += lo[d];
            phi += hi[d];
        } else {
            plo -= hi[d];
            phi -= lo[d];
        }
    }
    __shared__ double sp[2][8];
    for (int o = 16; o > 0; o >>= 1) {
        plo += __shfl_xor_sync(0xffffffffu, plo, o);
        phi += __shfl_xor_sync(0xffffffffu, phi, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sp[0][threadIdx.x >> 5] = plo;
        sp[1][threadIdx.x >> 5] = phi;
    }
    __syncthreads();
    plo = phi = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        plo += sp[0][w];
        phi += sp[1][w];
    }
    const int inj = plo > 0.0 ? 1 : (phi < 0.0 ? -1 : 0);
    // obj_lo: s_inj,hi = max(-plo, phi), phi when phi >= -plo
    const bool up_hi = phi >= -plo;
    for (int d = threadIdx.x; d < a.n_dev; d += blockDim.x) {
        const bool gen = d < a.n_gen;
        const double sgn = gen ? 1.0 : -1.0;
        const int col = a.dev_col[d];
        double gc = 0.0, gr = 0.0;
        if (col >= 0) {
            gc = -a.zeta_f * a.dc[(size_t)box * a.n_a_pad + col];
            // obj_hi grows with the radius (s_lo falls), obj_lo falls (s_hi grows)
            gr = (lo_side ? -a.zeta_f : a.zeta_f) * a.dr[(size_t)box * a.n_a_pad + col];
        }
        double glo = 0.5 * sgn * gc - 0.5 * gr;
        double ghi = 0.5 * sgn * gc + 0.5 * gr;
        const int s0 = a.seg_ptr[d], ns = a.seg_ptr[d + 1] - s0;
        if (!lo_side) {
            if (gen) glo -= pwl_slope(a.slope + s0, a.bkpt + s0, ns, lo[d]);
            else ghi += pwl_slope(a.slope + s0, a.bkpt + s0, ns, hi[d]);
            if (inj > 0) {  // s_inj,lo = plo = sum lo_g - sum hi_d
                if (gen) glo -= a.zeta_inj;
                else ghi += a.zeta_inj;
            } else if (inj < 0) {  // s_inj,lo = -phi = sum lo_d - sum hi_g
                if (gen) ghi += a.zeta_inj;
                else glo -= a.zeta_inj;
            }
        } else {
            // obj_lo takes the load values at lo and the generator costs at hi
            if (gen) ghi -= pwl_slope(a.slope + s0, a.bkpt + s0, ns, hi[d]);
            else glo += pwl_slope(a.slope + s0, a.bkpt + s0, ns, lo[d]);
            if (up_hi) {  // s_inj,hi = phi = sum hi_g - sum lo_d
                if (gen) ghi -= a.zeta_inj;
                else glo += a.zeta_inj;
            } else {      // s_inj,hi = -plo = sum hi_d - sum lo_g
                if (gen) glo += a.zeta_inj;
                else ghi -= a.zeta_inj;
            }
        }
        a.grad_lo[(size_t)box * a.n_dev + d] = g * glo;
        a.grad_hi[(size_t)box * a.n_dev + d] = g * ghi;
    }
    if (a.grad_rating)
        for (int l = threadIdx.x; l < a.n_l; l += blockDim.x)
            a.grad_rating[(size_t)box * a.n_l + l] = g * a.zeta_f * (double)a.cnt[(size_t)box * a.n_l + l];
}

cudaError_t launch_backward(const BwdArgs &a, cudaStream_t s) {
    const dim3 gw(kEntryBlocks, a.n_box);
    k_bwd_weights<<<gw, 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const dim3 gc((a.n_a_pad + 127) / 128, kCenterSplit, a.n_box);
    k_bwd_center<<<gc, 128, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const dim3 gr((a.n_a_pad + 127) / 128, kEntryBlocks / 4, a.n_box);
    k_bwd_radius<<<gr, 128, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_bwd_chain<<<a.n_box, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bwd_zero_cases(const BwdArgs *args, const int2 *items, int n_items, bool counts,
                                  cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    k_bwd_zero_cases<<<dim3(8, n_items), 256, 0, s>>>(args, items, counts ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_backward_cases(const BwdArgs *args, const int2 *items, int n_items, int max_n_a_pad,
                                  cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    k_bwd_weights_cases<<<dim3(kEntryBlocks, n_items), 256, 0, s>>>(args, items);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int cb = (max_n_a_pad + 127) / 128;
    k_bwd_center_cases<<<dim3(cb, kCenterSplit, n_items), 128, 0, s>>>(args, items);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_bwd_radius_cases<<<dim3(cb, kEntryBlocks / 4, n_items), 128, 0, s>>>(args, items);
    return cudaGetLastError();
}

cudaError_t launch_bwd_chain(const BwdArgs &a, cudaStream_t s) {
    k_bwd_chain<<<a.n_box, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ibp
