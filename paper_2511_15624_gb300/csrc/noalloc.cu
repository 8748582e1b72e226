// ibp_bound_noalloc: a one-box bound that allocates no device memory.
//
// Some callers cannot call cudaMalloc at bound time: code running while a CUDA
// stream is being captured into a graph, host threads with latency limits
// (cudaMalloc and cudaFree can synchronise the whole device), and programs that
// hand all device memory to their own allocator and forbid any other
// allocation.  For them this entry point keeps every per-call buffer (bus
// intervals, base-flow vectors, partial sums, the error word) in one
// file-scope __device__ array of kNoAllocBytes bytes, which every GPU that
// loads the library holds until the process exits.  The case itself (built
// once by ibp_case_create) supplies the sensitivities.
//
// Its contingency kernel is a variant of the library's one-box kernel that
// reads the unscaled FP32 PTDF rows with plain loads and multiplies by the bus
// radius in the accumulation (acc <- RU(acc + |h| r_b)), so it needs no
// per-call copy of the scaled rows; the certified arithmetic and the epilogue
// are the same.
#include <mutex>

#include "common.cuh"
#include "ctg_epilogue.cuh"
#include "internal.h"

namespace ibp {

// Maximum scratch: 8 MiB covers, e.g., 10500 lines x 5000 contingencies.
constexpr size_t kNoAllocBytes = size_t(8) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Host-side device addresses of g_noalloc_scratch, one per device ordinal,
// filled on the first call on that device, together with the CUDA context
// they belong to: after the context is destroyed and created again (e.g. by
// cudaDeviceReset) the module is loaded anew, and the next call looks the
// address up again instead of using the stale one.
constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static unsigned char *g_noalloc_base[kMaxDevices] = {};
static void *g_noalloc_ctx[kMaxDevices] = {};

// The current driver context (CUcontext) of the calling thread, through the
// runtime's driver entry point (the library does not link libcuda directly).
static bool current_context(void **ctx) {
    typedef int (*GetCtx)(void **);
    static GetCtx fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p)
            return false;
        fn = reinterpret_cast<GetCtx>(p);
    }
    return fn(ctx) == 0 && *ctx != nullptr;
}

constexpr int kPlainBL = 128, kPlainBK = 64, kPlainCH = 32;

// One-box contingency kernel, unscaled rows: persistent CTAs over tiles of
// BL lines x BK contingencies; each 32-bus chunk of the two PTDF row blocks
// and of the radius is staged through shared memory with plain loads.
template <int BL, int BK>
__global__ void __launch_bounds__(256, 1)
    k_ctg_plain(const CtgArgs a, const float *__restrict__ phi, int n_a_pad,
                const float *__restrict__ rb) {
    constexpr int ML = BL / 16, MK = BK / 16, CH = kPlainCH, PAD = CH + 4;
    __shared__ __align__(16) float sL[BL * PAD];
    __shared__ __align__(16) float sK[BK * PAD];
    __shared__ __align__(16) float sR[CH];
    __shared__ __align__(16) unsigned char squeue[ref_queue_bytes(8)];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const RefQueue rq = ref_queue_of(squeue, warp);
    ref_queue_init(rq);
    const int tl = (warp >> 1) * 4 + (lane >> 3);
    const int tk = (warp & 1) * 8 + (lane & 7);
    for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
        const int l0 = (tile % a.tiles_l) * BL, k0 = (tile / a.tiles_l) * BK;
        float Lr[ML][MK], acc1[ML][MK], acc2[ML][MK], acc3[ML][MK];
#pragma unroll
        for (int i = 0; i < ML; ++i)
#pragma unroll
            for (int j = 0; j < MK; ++j) {
                const int l = l0 + tl + 16 * i, k = k0 + tk + 16 * j;
                Lr[i][j] = (l < a.n_l && k < a.n_c) ? __ldg(&a.lodf[(size_t)k * a.n_l + l]) : 0.0f;
                acc1[i][j] = acc2[i][j] = acc3[i][j] = 0.0f;
            }
        for (int ch = 0; ch < a.n_chunks; ++ch) {
            __syncthreads();
            const int col = ch * CH;
            for (int idx = threadIdx.x; idx < (BL + BK) * (CH / 4); idx += blockDim.x) {
                const int row = idx / (CH / 4), q = idx % (CH / 4);
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (row < BL) {
                    const int l = l0 + row;
                    if (l < a.n_l)
                        v = __ldg(reinterpret_cast<const float4 *>(phi + (size_t)l * n_a_pad + col) + q);
                    *reinterpret_cast<float4 *>(&sL[row * PAD + 4 * q]) = v;
                } else {
                    const int k = k0 + row - BL;
                    if (k < a.n_c) {
                        const int kl = __ldg(&a.ctg_line[k]);
                        v = __ldg(reinterpret_cast<const float4 *>(phi + (size_t)kl * n_a_pad + col) + q);
                    }
                    *reinterpret_cast<float4 *>(&sK[(row - BL) * PAD + 4 * q]) = v;
                }
            }
            if (threadIdx.x < CH / 4)
                *reinterpret_cast<float4 *>(&sR[4 * threadIdx.x]) =
                    __ldg(reinterpret_cast<const float4 *>(rb + col) + threadIdx.x);
            __syncthreads();
#pragma unroll 2
            for (int q = 0; q < CH / 4; ++q) {
                float4 fk[MK];
#pragma unroll
                for (int j = 0; j < MK; ++j)
                    fk[j] = *reinterpret_cast<const float4 *>(&sK[(tk + 16 * j) * PAD + 4 * q]);
                const float4 r = *reinterpret_cast<const float4 *>(&sR[4 * q]);
#pragma unroll
                for (int i = 0; i < ML; ++i) {
                    const float4 fl = *reinterpret_cast<const float4 *>(&sL[(tl + 16 * i) * PAD + 4 * q]);
#pragma unroll
                    for (int j = 0; j < MK; ++j) {
                        const float L = Lr[i][j];
                        acc1[i][j] = __fmaf_ru(fabsf(__fmaf_rn(L, fk[j].x, fl.x)), r.x, acc1[i][j]);
                        acc1[i][j] = __fmaf_ru(fabsf(__fmaf_rn(L, fk[j].y, fl.y)), r.y, acc1[i][j]);
                        acc1[i][j] = __fmaf_ru(fabsf(__fmaf_rn(L, fk[j].z, fl.z)), r.z, acc1[i][j]);
                        acc1[i][j] = __fmaf_ru(fabsf(__fmaf_rn(L, fk[j].w, fl.w)), r.w, acc1[i][j]);
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
        float slo = 0.0f, shi = 0.0f, whi = 0.0f, wlo = 0.0f, cslo = 0.0f, cwhi = 0.0f;
        uint64_t rmask = 0;
#pragma unroll
        for (int i = 0; i < ML; ++i)
#pragma unroll
            for (int j = 0; j < MK; ++j) {
                const int l = l0 + tl + 16 * i, k = k0 + tk + 16 * j;
                if (l < a.n_l && k < a.n_c &&
                    pair_epilogue(a, 0, l, k, Lr[i][j], __fadd_ru(acc3[i][j], acc2[i][j]), slo, shi, whi,
                                  wlo, cslo, cwhi))
                    rmask |= 1ull << (i * MK + j);
            }
        // candidates of the FP64 refinement: queued, or (queue full) the FP32 terms
        const bool queued =
            a.ref.phi64 &&
            ref_enqueue<ML * MK>(
                rq, rmask,
                [&](int q, int &l, int &k) {
                    l = l0 + tl + 16 * (q / MK);
                    k = k0 + tk + 16 * (q % MK);
                },
                0, tile * a.warps_per_tile + warp);
        if (!queued) {
            slo = __fadd_rd(slo, cslo);
            whi = __fadd_ru(whi, cwhi);
        }
        write_warp_partials(a, tile, warp, 0, slo, shi, whi, wlo, ML * MK + 1);
    }
    // the queued refinements, after the last tile
    if (a.ref.phi64) ref_finish(rq, nullptr, 8, [&](int) -> const CtgArgs & { return a; });
}

static float noalloc_gamma(long n1, long n2, long n3) {
    const double u = std::ldexp(1.0, -24);
    return (float)(std::expm1((double)(n1 + n2 + n3 + 2) * std::log1p(2 * u)) * 1.01);
}

struct NoAllocLayout {
    size_t err, consts, cbus, rbus, rbus64, cabs, line_c, line_e, line_R, part_base, part_ctg, total;
};

static NoAllocLayout noalloc_layout(const CaseView &v, int n_tiles) {
    NoAllocLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~size_t(255);
        return o;
    };
    L.err = take(sizeof(int));
    L.consts = take(4 * sizeof(float));
    L.cbus = take((size_t)v.n_a_pad * sizeof(double));
    L.rbus = take((size_t)v.n_a_pad * sizeof(float));
    L.rbus64 = take((size_t)v.n_a_pad * sizeof(double));
    L.cabs = take((size_t)v.n_a_pad * sizeof(float));
    L.line_c = take((size_t)v.n_line * sizeof(float));
    L.line_e = take((size_t)v.n_line * sizeof(float));
    L.line_R = take((size_t)v.n_line * sizeof(float));
    L.part_base = take((size_t)v.n_part_base * kPartVals * sizeof(double));
    L.part_ctg = take((size_t)std::max(n_tiles, 1) * kConsumerWarps * kPartVals * sizeof(double));
    L.total = off;
    return L;
}

}  // namespace ibp

using namespace ibp;

extern "C" ibp_status ibp_bound_noalloc(ibp_case *c, const double *box_lo, const double *box_hi,
                                        double *obj_lo, double *obj_hi, double *obj_err,
                                        void *cuda_stream) {
    CaseView v;
    if (!case_view(c, &v)) return set_error(IBP_EINVAL, "case is NULL or was created without a device");
    if (!box_lo || !box_hi || !obj_lo || !obj_hi || !obj_err)
        return set_error(IBP_EINVAL, "box and objective pointers must not be NULL");
    const int tiles_l = (v.n_line + kPlainBL - 1) / kPlainBL;
    const int tiles_k = (v.n_ctg + kPlainBK - 1) / kPlainBK;
    const int n_tiles = tiles_l * tiles_k;
    const NoAllocLayout lay = noalloc_layout(v, n_tiles);
    if (lay.total > kNoAllocBytes) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "case needs %zu bytes of scratch; the static buffer of ibp_bound_noalloc holds %zu",
                 lay.total, kNoAllocBytes);
        return set_error(IBP_EINVAL, msg);
    }
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(v.device) != cudaSuccess)
        return set_error(IBP_ECUDA, "cannot select the case's device");
    struct Restore {
        int d;
        ~Restore() {
            if (d >= 0) cudaSetDevice(d);
        }
    } restore{prev};
    if (v.device >= kMaxDevices) return set_error(IBP_EINVAL, "device ordinal too large");
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        void *ctx = nullptr;
        if (!current_context(&ctx)) return set_error(IBP_ECUDA, "no current CUDA context on the case's device");
        if (g_noalloc_ctx[v.device] != ctx) {
            g_noalloc_base[v.device] = nullptr;
            g_noalloc_ctx[v.device] = ctx;
        }
        if (!g_noalloc_base[v.device]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                char msg[256];
                snprintf(msg, sizeof msg, "cudaGetSymbolAddress of the scratch array failed: %s",
                         cudaGetErrorString(e));
                return set_error(IBP_ECUDA, msg);
            }
            g_noalloc_base[v.device] = static_cast<unsigned char *>(p);
        }
        base = g_noalloc_base[v.device];
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int *err = reinterpret_cast<int *>(base + lay.err);
    float *consts = reinterpret_cast<float *>(base + lay.consts);
    double *cbus = reinterpret_cast<double *>(base + lay.cbus);
    float *rbus = reinterpret_cast<float *>(base + lay.rbus);
    double *rbus64 = reinterpret_cast<double *>(base + lay.rbus64);
    float *cabs = reinterpret_cast<float *>(base + lay.cabs);
    float *line_c = reinterpret_cast<float *>(base + lay.line_c);
    float *line_e = reinterpret_cast<float *>(base + lay.line_e);
    float *line_R = reinterpret_cast<float *>(base + lay.line_R);
    double *part_base = reinterpret_cast<double *>(base + lay.part_base);
    double *part_ctg = reinterpret_cast<double *>(base + lay.part_ctg);

    // the error word must start at zero; every other buffer is overwritten
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);

    BusArgs ba{};
    ba.n_a = v.n_a; ba.n_a_pad = v.n_a_pad; ba.n_dev = v.n_dev; ba.n_gen = v.n_gen; ba.n_box = 1;
    ba.act_ptr = v.act_ptr; ba.act_dev = v.act_dev; ba.box_lo = box_lo; ba.box_hi = box_hi;
    ba.cbus = cbus; ba.rbus = rbus; ba.rbus64 = rbus64; ba.rbus_t = nullptr; ba.n_box_pad = 0; ba.cabs = cabs;
    ba.box_consts = consts; ba.err = err;
    if (e == cudaSuccess) e = launch_bus(ba, s);

    BaseArgs bb{};
    bb.n_l = v.n_line; bb.n_c = v.n_ctg; bb.n_a = v.n_a; bb.n_a_pad = v.n_a_pad; bb.n_box = 1;
    bb.phi = v.phi_a; bb.ctg_line = v.ctg_line; bb.cbus = cbus; bb.rbus = rbus; bb.cabs = cabs;
    bb.rate_up = v.rate_up; bb.rate_dn = v.rate_dn; bb.box_consts = consts;
    bb.gamma_base = noalloc_gamma((v.n_a_pad / 4 + 31) / 32, 2, 5);
    bb.line_c = line_c; bb.line_e = line_e; bb.line_R = line_R;
    bb.hat_l = nullptr; bb.hat_k = nullptr; bb.partials = part_base; bb.err = err;
    // FP64 refinement of the terms that can reach obj_hi (as in ibp_bound)
    RefArgs ref{};
    if (v.phi64) {
        ref.phi_hi = v.phi_a; ref.phi64 = v.phi64; ref.cbus = cbus; ref.rbus64 = rbus64;
        ref.rbus = rbus; ref.cabs = cabs; ref.box_consts = consts;
        ref.rate64 = v.rate64; ref.rate_c64 = v.rate_c64; ref.n_a_pad = v.n_a_pad;
        ref.lodf = v.lodf; ref.lodf_lo = v.lodf_lo; ref.n_l = v.n_line;
    }
    bb.ref = ref;
    if (e == cudaSuccess) e = launch_base(bb, v.n_part_base, s);

    const int n_chunks = (v.n_a + kPlainCH - 1) / kPlainCH;
    CtgArgs ca{};
    ca.n_l = v.n_line; ca.n_c = v.n_ctg; ca.n_a = v.n_a; ca.n_chunks = n_chunks; ca.n_box = 1;
    ca.tiles_l = tiles_l; ca.n_tiles = n_tiles; ca.lodf = v.lodf; ca.ctg_line = v.ctg_line;
    ca.line_c = line_c; ca.line_e = line_e; ca.line_R = line_R; ca.rate_up = v.rate_c_up;
    ca.rate_dn = v.rate_c_dn; ca.box_consts = consts; ca.rbus_t = nullptr; ca.n_box_pad = 0;
    ca.gamma = noalloc_gamma(kPlainCH, 8, (n_chunks + 7) / 8);
    ca.flow_lo = nullptr; ca.flow_hi = nullptr; ca.partials = part_ctg; ca.err = err;
    ca.wait_ns = 0;
    ca.warps_per_tile = kConsumerWarps;
    ca.ref = ref;
    if (e == cudaSuccess && n_tiles > 0) {
        const int grid = std::min(v.num_sms, n_tiles);
        k_ctg_plain<kPlainBL, kPlainBK><<<grid, 256, 0, s>>>(ca, v.phi_a, v.n_a_pad, rbus);
        e = cudaGetLastError();
    }

    AsmArgs aa{};
    aa.n_box = 1; aa.n_dev = v.n_dev; aa.n_gen = v.n_gen;
    aa.n_part_ctg = n_tiles * kConsumerWarps; aa.n_part_base = v.n_part_base;
    aa.part_ctg = part_ctg; aa.part_base = part_base; aa.box_lo = box_lo; aa.box_hi = box_hi;
    aa.seg_ptr = v.seg_ptr; aa.slope = v.slope; aa.bkpt = v.bkpt;
    aa.zeta_inj = v.zeta_inj; aa.zeta_f = v.zeta_f;
    aa.obj_lo = obj_lo; aa.obj_hi = obj_hi; aa.obj_err = obj_err; aa.err = err;
    if (e == cudaSuccess) e = launch_assemble(aa, s);
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof msg, "launch failed: %s", cudaGetErrorString(e));
        return set_error(IBP_ECUDA, msg);
    }
    return set_error(IBP_OK, "");
}
