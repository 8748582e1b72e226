// Device helpers shared by the library's kernels: directed-rounding arithmetic,
// bounded mbarrier waits and TMA copies (inline PTX for sm_103a).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "internal.h"

namespace ibp {

// Index guards.  In a checked build (-DIBP_CHECK) a failed guard records
// kErrBounds in the call's error word and the caller skips the access; other
// builds compile the guards to `true`.
__device__ __forceinline__ bool idx_ok(bool cond, int *err) {
    if (!cond) atomicOr(err, kErrBounds);
    return cond;
}
#ifdef IBP_CHECK
#define IBP_IDX_OK(cond, err) ::ibp::idx_ok((cond), (err))
#else
#define IBP_IDX_OK(cond, err) true
#endif

// unit roundoff of FP32 round-to-nearest, 2^-24
constexpr float kU = 5.9604644775390625e-08f;


__device__ __forceinline__ float fmax0(float a) { return a > 0.0f ? a : 0.0f; }

// |x| over [lo, hi] (exact: negation and comparisons do not round)
__device__ __forceinline__ void abs_interval(float lo, float hi, float &alo, float &ahi) {
    alo = lo >= 0.0f ? lo : (hi <= 0.0f ? -hi : 0.0f);
    ahi = fmaxf(-lo, hi);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of the given parity to complete, giving up after
// limit_ns nanoseconds of global time.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0u && globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// 2-D tiled TMA load into shared memory, completion counted on an mbarrier.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                            int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// FP64 directed-rounding warp reductions (deterministic tree order).
__device__ __forceinline__ double warp_sum_rd(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rd(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_sum_ru(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __dadd_ru(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// Four FP64 sums over the warp, each rounded up, by recursive halving: the
// lanes split the four values between them (xor 16, then xor 8) before the
// butterfly over the low three lane bits, so a lane does 6 adds instead of 20.
// Lane L returns the total of value (L >> 3) & 3.  The order is fixed, so the
// result does not depend on timing.
__device__ __forceinline__ double warp_sum4_ru(double v0, double v1, double v2, double v3) {
    const int lane = threadIdx.x & 31;
    const bool b16 = (lane & 16) != 0, b8 = (lane & 8) != 0;
    double k0 = b16 ? v2 : v0, k1 = b16 ? v3 : v1;
    const double s0 = b16 ? v0 : v2, s1 = b16 ? v1 : v3;
    k0 = __dadd_ru(k0, __shfl_xor_sync(0xffffffffu, s0, 16));
    k1 = __dadd_ru(k1, __shfl_xor_sync(0xffffffffu, s1, 16));
    double k = b8 ? k1 : k0;
    k = __dadd_ru(k, __shfl_xor_sync(0xffffffffu, b8 ? k0 : k1, 8));
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) k = __dadd_ru(k, __shfl_xor_sync(0xffffffffu, k, o));
    return k;
}

__device__ __forceinline__ float warp_sum_ru_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __fadd_ru(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

}  // namespace ibp
