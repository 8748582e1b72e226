// Host side of the C ABI, shared by the files that implement its entry points:
// ibp_abi.cu (case build, bound, adjoints, settings), abi_linear.cu (the linear
// relaxation bound) and abi_multi.cu (many cases in one launch).  It holds the
// case object, the error and device helpers, and the workspace and launch
// helpers more than one of those files calls.
#pragma once

#include "internal.h"

#include <cudaTypedefs.h>
#include <cusolverDn.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <memory>
#include <numeric>
#include <string>
#include <vector>

using namespace ibp;

// ----------------------------------------------------------------- errors
// Set the thread's last-error message and return the status (ibp_last_error).
ibp_status fail(ibp_status s, const char *fmt, ...);
// Clear the thread's last-error message and return IBP_OK.
ibp_status ok();

#define CUDA_TRY(expr)                                                                      \
    do {                                                                                    \
        cudaError_t _e = (expr);                                                            \
        if (_e != cudaSuccess)                                                              \
            return fail(_e == cudaErrorMemoryAllocation ? IBP_ENOMEM : IBP_ECUDA,           \
                        "%s failed: %s", #expr, cudaGetErrorString(_e));                    \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Test hook: device allocations larger than this many bytes fail as if the
// device were out of memory (0: no limit).  See ibp_set_alloc_limit.
extern std::atomic<long long> g_alloc_limit;

template <class T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    cudaError_t alloc(size_t count) {
        free();
        if (count == 0) count = 1;
        const long long lim = g_alloc_limit.load();
        if (lim > 0 && (long long)(count * sizeof(T)) > lim) return cudaErrorMemoryAllocation;
        cudaError_t e = cudaMalloc(&p, count * sizeof(T));
        if (e == cudaSuccess) n = count;
        else p = nullptr;
        return e;
    }
    void free() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    ~DevBuf() { free(); }
};

// ----------------------------------------------------------------- the case
struct ibp_case {
    int device = -1;
    int n_bus = 0, slack = 0, n_line = 0, n_gen = 0, n_load = 0, n_dev = 0, n_ctg = 0;
    int n_a = 0, n_a_pad = 0;
    double zeta_inj = 0, zeta_f = 0;
    double build_seconds = 0, max_abs_lodf = 0;
    int num_sms = 0;
    int variant = 0;
    bool screen = true;      // paper-mode line screen ahead of the contingency kernel
    bool reduce = true;      // exact network reduction (bridges, bus classes)
    bool refine = true;      // FP64 refinement of the terms that can reach obj_hi
    bool has_reduction = false;
    int n_r = 0, n_r_pad = 0, n_bridges = 0;  // bus classes, bridge lines
    std::vector<int> cls_ptr_h, cls_col_h, is_bridge_h;
    int last_screened = 0;   // whether the last bound call ran the screen
    std::vector<int> ctg_line_h;

    // persistent device data
    DevBuf<float> phi_a, lodf, rate_up, rate_dn, rate_c_up, rate_c_dn;
    DevBuf<double> phi64;             // the FP64 PTDF of the active columns
    DevBuf<float> lodf_lo;             // RN32(L - L~) of the contingency list
    DevBuf<double> rate64, rate_c64;   // ratings as given (FP64)
    DevBuf<int> ctg_line, act_ptr, act_dev, seg_ptr, dev_col;
    DevBuf<double> slope, bkpt;
    DevBuf<float> hat_l, hat_k;  // one-box scaled rows (lazily allocated)
    DevBuf<float> phi_k;         // unscaled PTDF rows of the contingency lines
    // network reduction: bridge flags, bus classes (CSR over active columns)
    // and the PTDF columns of one member per class, [n_l][n_r_pad] and the
    // contingency rows [n_c][n_r_pad]
    DevBuf<int> is_bridge, cls_ptr, cls_col;
    DevBuf<float> phi_r, phi_kr;
    // many-case launch: the non-bridge lines (list, count on the device) and
    // their reduced rows [n_nb][n_r_pad], built on first use
    int n_nb = -1;
    DevBuf<int> nb_list, nb_count;
    DevBuf<float> phi_nb;

    // per-call workspace (ws_gen changes whenever its buffers move)
    int cap_box = 0, ws_gen = 0;
    DevBuf<double> box_lo, box_hi, obj;
    DevBuf<double> cbus;
    DevBuf<float2> cbus2;
    DevBuf<float> rbus, cabs, box_consts, line_c, line_e, line_R, rbus_t, bus_part;
    DevBuf<double> rbus64;
    DevBuf<double> lc64, lR64;  // paper-mode refinement: per-line FP64 centre and radius
    DevBuf<float> lX;
    // linear (CROWN-style) relaxation bound: iteration state and certified value
    int lin_cap_box = 0, lin_state_box = 0;  // boxes the workspace holds / the state describes
    bool lin_pc_ready = false;             // the diagonal step sizes are computed (once per case)
    DevBuf<float> lpcS;                    // [n_line] row sums S_l of the step sizes
    DevBuf<double> lpctau, lpcA, lpcB, lpcL;  // [n_dev] primal steps; scratch of their build
    DevBuf<int> cl_ptr, cl_ctg;            // contingencies per outaged line
    DevBuf<double> lw, lx, lsx, lxb, lx_last, lxavg, la0, la0_last, lstot, lstotp, lred, lub, lub_err, lbest;
    DevBuf<float> lac, lc_last, lab, lb_last, lp, lf, lcol, lrow, lg;
    DevBuf<double> lW64, lWabs, lconst, lrd64, lrda, lg64, lG64;
    cudaGraphExec_t lin_graph = nullptr;   // a chunk of iterations
    // refinement queues of the contingency launch (regions per CTA and warp)
    DevBuf<int4> refq;
    DevBuf<int> refq_cnt;
    DevBuf<double2> refq_res;
    DevBuf<double> part_base, part_ctg, part_stage;
    DevBuf<float> flows;
    DevBuf<int> err;
    DevBuf<int> rating_flag;  // sticky: the last ibp_case_set_ratings found a bad entry
    DevBuf<int> live_flag, live, n_live;  // line screen
    DevBuf<float> rcls, rcls_t;           // class radii [box][n_r_pad], [n_r_pad][box_pad]
    // adjoint workspace (obj_hi's active pairs; obj_lo's in the _lo buffers)
    int bwd_cap_box = 0, act_cap = 0;
    DevBuf<int> act_count, cnt;
    DevBuf<int4> act_list;
    int bwd_lo_cap_box = 0, act_cap_lo = 0;
    DevBuf<int> act_count_lo;
    DevBuf<int4> act_list_lo;
    DevBuf<double> W, dc, dr, grads;
    int n_part_base = 0;

    // timing
    bool timing = false;
    static constexpr int kEvents = 7;
    cudaEvent_t ev[kEvents] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    // completion of the case's last enqueued call (recorded on that call's
    // stream), and a private non-blocking stream for reading the error word:
    // ibp_case_sync waits for this case's work only, not the whole device.
    // A call enqueued while its stream was being captured cannot be waited
    // for through the event; the next sync then waits for the device.
    cudaEvent_t done = nullptr;
    cudaStream_t side = nullptr;
    bool captured = false;

    ~ibp_case() {
        if (device >= 0) {
            DeviceGuard g(device);
            for (auto &e : ev)
                if (e) cudaEventDestroy(e);
            if (done) cudaEventDestroy(done);
            if (lin_graph) cudaGraphExecDestroy(lin_graph);
            if (side) cudaStreamDestroy(side);
            phi_a.free(); lodf.free(); rate_up.free(); rate_dn.free(); rate_c_up.free();
            phi64.free(); lodf_lo.free(); rate64.free(); rate_c64.free(); rbus64.free();
            lc64.free(); lR64.free(); lX.free(); refq.free(); refq_cnt.free(); refq_res.free();
            rate_c_dn.free(); ctg_line.free(); act_ptr.free(); act_dev.free(); seg_ptr.free();
            slope.free(); bkpt.free(); hat_l.free(); hat_k.free(); phi_k.free(); rbus_t.free();
            box_lo.free(); box_hi.free();
            obj.free(); cbus.free(); cbus2.free(); rbus.free(); cabs.free(); box_consts.free(); bus_part.free(); line_c.free();
            line_e.free(); line_R.free(); part_base.free(); part_ctg.free(); part_stage.free(); flows.free(); err.free();
            live_flag.free(); live.free(); n_live.free(); is_bridge.free(); cls_ptr.free(); rating_flag.free();
            cls_col.free(); phi_r.free(); phi_kr.free(); rcls.free(); rcls_t.free(); nb_list.free();
            nb_count.free(); phi_nb.free();
            dev_col.free(); act_count.free(); cnt.free(); act_list.free(); W.free(); dc.free(); dr.free();
            act_count_lo.free(); act_list_lo.free();
            grads.free();
        }
    }
};


// ----------------------------------------------------------------- shared helpers
constexpr int32_t kMaxBoxesPerCall = 65535;  // boxes per call (a grid's y dimension)
constexpr int kPartStages = 64;              // blocks of stage 1 of the objective assembly

bool is_fin(double x);
float rup_gamma(long n1, long n2, long n3);
size_t max_part_rows(const ibp_case *c);
ibp_status ensure_workspace(ibp_case *c, int n_box);
ibp_status ensure_class_ws(ibp_case *c);
int ref_regions(int num_sms);
RefArgs ref_args(const ibp_case *c);
ibp_status mark_done(ibp_case *c, cudaStream_t s);
ibp_status wait_case(ibp_case *c);
ibp_status read_err_word(ibp_case *c);
ibp_status check_boxes_host(const ibp_case *c, int n_box, const double *lo, const double *hi);
ibp_status ensure_bwd_workspace(ibp_case *c, int n_box);
ibp_status ensure_bwd_lo_workspace(ibp_case *c, int n_box);
void drop_plans_of(const ibp_case *c);  // abi_multi.cu: forget the plans that name the case

// FP64 refinement queues (per-SM regions) of a case or of a many-case plan,
// grown to their full size on first use
template <class Q>
ibp_status ensure_ref_queue(Q *q, int num_sms) {
    const size_t n = (size_t)ref_regions(num_sms);
    if (q->refq.n >= n * kRefQCap && q->refq_cnt.n >= n && q->refq_res.n >= n * kRefQCap) return IBP_OK;
    CUDA_TRY(q->refq.alloc(n * kRefQCap));
    CUDA_TRY(q->refq_cnt.alloc(n));
    CUDA_TRY(q->refq_res.alloc(n * kRefQCap));
    return IBP_OK;
}
