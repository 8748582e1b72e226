// C ABI of the linear (CROWN-style) relaxation bound: the iteration's
// workspace and state, the chunked CUDA-graph launch of the primal-dual
// iteration, warm starts and state inheritance, and the read-back of the slopes.
#include "abi_case.h"

// ---------------------------------------------------------------- linear bound
static ibp_status ensure_lin_workspace(ibp_case *c, int n_box) {
    if (n_box <= c->lin_cap_box) return IBP_OK;
    const int cap = std::max(n_box, 1);
    c->lin_cap_box = 0;
    const size_t nd = (size_t)cap * c->n_dev, nl = (size_t)cap * c->n_line;
    const size_t np = (size_t)cap * std::max(c->n_ctg, 1) * c->n_line, na = (size_t)cap * c->n_a_pad;
    const size_t nc = (size_t)cap * std::max(c->n_ctg, 1);
    CUDA_TRY(c->lw.alloc(cap)); CUDA_TRY(c->la0.alloc(cap));
    CUDA_TRY(c->la0_last.alloc(cap)); CUDA_TRY(c->lstot.alloc(cap)); CUDA_TRY(c->lred.alloc((size_t)cap * 4));
    CUDA_TRY(c->lstotp.alloc((size_t)cap * ((c->n_dev + 127) / 128)));
    CUDA_TRY(c->lub.alloc(cap)); CUDA_TRY(c->lub_err.alloc(cap)); CUDA_TRY(c->lbest.alloc((size_t)cap * 2));
    CUDA_TRY(c->lx.alloc(nd)); CUDA_TRY(c->lsx.alloc(nd)); CUDA_TRY(c->lxb.alloc(nd)); CUDA_TRY(c->lx_last.alloc(nd));
    CUDA_TRY(c->lac.alloc(np)); CUDA_TRY(c->lc_last.alloc(np)); CUDA_TRY(c->lxavg.alloc(nd));
    CUDA_TRY(c->lab.alloc(nl)); CUDA_TRY(c->lb_last.alloc(nl));
    CUDA_TRY(c->lp.alloc(na)); CUDA_TRY(c->lf.alloc(nl)); CUDA_TRY(c->lcol.alloc(nl));
    CUDA_TRY(c->lrow.alloc(nc)); CUDA_TRY(c->lg.alloc(na));
    CUDA_TRY(c->lW64.alloc(nl)); CUDA_TRY(c->lWabs.alloc(nl)); CUDA_TRY(c->lconst.alloc(nl));
    CUDA_TRY(c->lrd64.alloc(nc)); CUDA_TRY(c->lrda.alloc(nc)); CUDA_TRY(c->lg64.alloc(na));
    CUDA_TRY(c->lG64.alloc(na));
    if (!c->cl_ptr.p) {
        std::vector<int> ptr(c->n_line + 1, 0), ctg;
        for (int k = 0; k < c->n_ctg; ++k) ++ptr[c->ctg_line_h[k] + 1];
        for (int l = 0; l < c->n_line; ++l) ptr[l + 1] += ptr[l];
        ctg.resize(std::max(c->n_ctg, 1));
        std::vector<int> fill(ptr.begin(), ptr.end() - 1);
        for (int k = 0; k < c->n_ctg; ++k) ctg[fill[c->ctg_line_h[k]]++] = k;
        CUDA_TRY(c->cl_ptr.alloc(ptr.size()));
        CUDA_TRY(c->cl_ctg.alloc(ctg.size()));
        CUDA_TRY(cudaMemcpy(c->cl_ptr.p, ptr.data(), ptr.size() * sizeof(int), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(c->cl_ctg.p, ctg.data(), ctg.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    c->lin_cap_box = cap;
    ++c->ws_gen;
    return IBP_OK;
}

// first: the held box whose state the call's box 0 uses (the iteration state
// is box-major; the scratch buffers always start at box 0)
static LinArgs lin_args(const ibp_case *c, int n_box, const double *lo, const double *hi, int first = 0) {
    LinArgs a{};
    a.n_l = c->n_line; a.n_c = c->n_ctg; a.n_a = c->n_a; a.n_a_pad = c->n_a_pad; a.n_dev = c->n_dev;
    a.n_gen = c->n_gen; a.n_box = n_box;
    a.phi = c->phi_a.p; a.phi64 = c->phi64.p; a.lodf = c->lodf.p; a.lodf_lo = c->lodf_lo.p;
    a.ctg_line = c->ctg_line.p; a.cl_ptr = c->cl_ptr.p; a.cl_ctg = c->cl_ctg.p;
    a.act_ptr = c->act_ptr.p; a.act_dev = c->act_dev.p; a.dev_col = c->dev_col.p;
    a.rate64 = c->rate64.p; a.rate_c64 = c->rate_c64.p; a.box_lo = lo; a.box_hi = hi;
    a.seg_ptr = c->seg_ptr.p; a.slope = c->slope.p; a.bkpt = c->bkpt.p;
    a.zeta_inj = c->zeta_inj; a.zeta_f = c->zeta_f;
    a.pc_S = c->lpcS.p; a.pc_tau = c->lpctau.p;
    a.w = c->lw.p; a.x = c->lx.p; a.sx = c->lsx.p; a.xb = c->lxb.p; a.x_last = c->lx_last.p;
    a.a_c = c->lac.p; a.c_last = c->lc_last.p;
    a.a_b = c->lab.p; a.b_last = c->lb_last.p;
    a.a0 = c->la0.p; a.a0_last = c->la0_last.p;
    a.x_avg = c->lxavg.p;
    a.p = c->lp.p; a.stot = c->lstot.p; a.stot_part = c->lstotp.p; a.f = c->lf.p; a.colsum = c->lcol.p; a.rowdot = c->lrow.p;
    a.g = c->lg.p; a.red = c->lred.p;
    a.W64 = c->lW64.p; a.Wabs = c->lWabs.p; a.constl = c->lconst.p; a.rd64 = c->lrd64.p;
    a.rda = c->lrda.p; a.g64 = c->lg64.p; a.G64 = c->lG64.p; a.ub = c->lub.p; a.ub_err = c->lub_err.p;
    if (first > 0) {
        const size_t f = (size_t)first, fd = f * c->n_dev, fl = f * c->n_line;
        const size_t fc = f * std::max(c->n_ctg, 1) * c->n_line;
        a.w += f; a.x += fd; a.sx += fd; a.x_last += fd; a.x_avg += fd;
        a.a_c += fc; a.c_last += fc;
        a.a_b += fl; a.b_last += fl;
        a.a0 += f; a.a0_last += f;
    }
    return a;
}

// x <- the box midpoints (and x_last); primal weight w0; best bound +inf
__global__ void k_lin_init(int n, const double *lo, const double *hi, double *x, double *x_last,
                           int n_box, double *w, double w0, double *best) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        x[i] = 0.5 * (lo[i] + hi[i]);
        x_last[i] = x[i];
    }
    if (i < n_box) {
        w[i] = w0;
        best[2 * i] = INFINITY;
        best[2 * i + 1] = 0.0;
    }
}

// warm start: points clipped into their boxes and taken as the reference of
// the next adaptation; best bound +inf (the slopes, the slope references and
// the primal weight stay; the running sum of the points is 0 after the
// previous call's last adaptation)
__global__ void k_lin_warm(int n, const double *lo, const double *hi, double *x, double *x_last,
                           int n_box, double *best) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        x[i] = fmin(fmax(x[i], lo[i]), hi[i]);
        x_last[i] = x[i];
    }
    if (i < n_box) {
        best[2 * i] = INFINITY;
        best[2 * i + 1] = 0.0;
    }
}

// keep the smaller certified bound of each box (and its error bound)
__global__ void k_lin_best(int n_box, const double *ub, const double *err, double *best) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n_box && ub[j] < best[2 * j]) {
        best[2 * j] = ub[j];
        best[2 * j + 1] = err[j];
    }
}

__global__ void k_lin_out(int n_box, const double *best, double *obj_hi, double *obj_err) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n_box) {
        obj_hi[j] = best[2 * j];
        obj_err[j] = best[2 * j + 1];
    }
}

constexpr int kLinRestart = 1000;   // iterations between adaptations of the primal weight (and certified values)
constexpr int kLinChunk = 50;       // iterations per CUDA graph launch

static ibp_status lin_run(ibp_case *c, int n_box, const double *lo, const double *hi, int n_iter,
                          double w0, double *obj_hi, double *obj_err, double *x_point, cudaStream_t s,
                          bool warm = false, int first = 0) {
    if (warm && (first < 0 || n_box > c->lin_state_box - first))
        return fail(IBP_EINVAL, "no linear state for boxes [%d, %d) to continue from (%d held)", first,
                    first + n_box, c->lin_state_box);
    ibp_status st = ensure_lin_workspace(c, n_box);
    if (st != IBP_OK) return st;
    const size_t nd = (size_t)n_box * c->n_dev, np = (size_t)n_box * std::max(c->n_ctg, 1) * c->n_line;
    const size_t nl = (size_t)n_box * c->n_line;
    auto zero = [&](void *p, size_t bytes) { return cudaMemsetAsync(p, 0, bytes, s); };
    if (!c->lin_pc_ready) {
        // the diagonal step sizes, once per case (they depend on the network only)
        if (!c->lpcS.p) {
            CUDA_TRY(c->lpcS.alloc(c->n_line)); CUDA_TRY(c->lpctau.alloc(c->n_dev));
            CUDA_TRY(c->lpcA.alloc(c->n_a_pad)); CUDA_TRY(c->lpcB.alloc(c->n_a_pad));
            CUDA_TRY(c->lpcL.alloc(std::max(c->n_ctg, 1)));
        }
        LinArgs a = lin_args(c, 1, lo, hi);
        CUDA_TRY(lin_precondition(a, c->lpcS.p, c->lpctau.p, c->lpcA.p, c->lpcB.p, c->lpcL.p, s));
        c->lin_pc_ready = true;
    }
    if (warm) {
        // continue from the state held for these boxes: the points are moved
        // into their (possibly smaller) boxes; the best bound restarts
        const size_t fd = (size_t)first * c->n_dev;
        k_lin_warm<<<(unsigned)((std::max(nd, (size_t)n_box) + 255) / 256), 256, 0, s>>>(
            (int)nd, lo, hi, c->lx.p + fd, c->lx_last.p + fd, n_box, c->lbest.p);
        CUDA_TRY(cudaGetLastError());
    } else {
    k_lin_init<<<(unsigned)((std::max(nd, (size_t)n_box) + 255) / 256), 256, 0, s>>>(
        (int)nd, lo, hi, c->lx.p, c->lx_last.p, n_box, c->lw.p, w0, c->lbest.p);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(zero(c->lsx.p, nd * sizeof(double)));
    CUDA_TRY(zero(c->lac.p, np * sizeof(float)));
    CUDA_TRY(zero(c->lc_last.p, np * sizeof(float)));
    CUDA_TRY(zero(c->lab.p, nl * sizeof(float)));
    CUDA_TRY(zero(c->lb_last.p, nl * sizeof(float)));
    CUDA_TRY(zero(c->la0.p, n_box * sizeof(double)));
    CUDA_TRY(zero(c->la0_last.p, n_box * sizeof(double)));
    CUDA_TRY(zero(c->lred.p, (size_t)n_box * 4 * sizeof(double)));
    CUDA_TRY(zero(c->lg.p, (size_t)n_box * c->n_a_pad * sizeof(float)));
    }
    // the state is box-major: a warm call on held boxes [first, first + n_box)
    // leaves the rest of the held state as it was
    if (!warm) c->lin_state_box = n_box;
    LinArgs a = lin_args(c, n_box, lo, hi, warm ? first : 0);
    if (warm) {
        // the dual gradient g of the inherited slopes (the iteration's first x
        // step uses it), and the certified value at those slopes: on a sub-box
        // it is at most the parent's, so a continued bound never rises
        CUDA_TRY(lin_gradient(a, c->num_sms, s));
        CUDA_TRY(lin_certify(a, c->num_sms, s));
        k_lin_best<<<(n_box + 127) / 128, 128, 0, s>>>(n_box, c->lub.p, c->lub_err.p, c->lbest.p);
        CUDA_TRY(cudaGetLastError());
    }
    // a chunk of iterations as one CUDA graph, captured on a private stream
    // (the arguments hold this call's box pointers, so each call captures anew)
    const int chunk = std::min(kLinChunk, kLinRestart);
    {
        if (c->lin_graph) {
            cudaGraphExecDestroy(c->lin_graph);
            c->lin_graph = nullptr;
        }
        cudaStream_t cs = nullptr;
        CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        for (int i = 0; e == cudaSuccess && i < chunk; ++i) e = lin_iteration(a, c->num_sms, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->lin_graph, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        CUDA_TRY(e);
    }
    int done = 0, since = 0;
    while (done < n_iter) {
        const int m = std::min(chunk, n_iter - done);
        if (m == chunk) {
            CUDA_TRY(cudaGraphLaunch(c->lin_graph, s));
        } else {
            for (int i = 0; i < m; ++i) CUDA_TRY(lin_iteration(a, c->num_sms, s));
        }
        done += m;
        since += m;
        if (since >= kLinRestart || done == n_iter) {
            a.n_avg = since;
            CUDA_TRY(lin_restart(a, c->num_sms, s));
            since = 0;
            CUDA_TRY(lin_certify(a, c->num_sms, s));
            k_lin_best<<<(n_box + 127) / 128, 128, 0, s>>>(n_box, c->lub.p, c->lub_err.p, c->lbest.p);
            CUDA_TRY(cudaGetLastError());
        }
    }
    if (n_iter == 0 && !warm) {
        CUDA_TRY(lin_certify(a, c->num_sms, s));
        k_lin_best<<<(n_box + 127) / 128, 128, 0, s>>>(n_box, c->lub.p, c->lub_err.p, c->lbest.p);
    }
    k_lin_out<<<(n_box + 127) / 128, 128, 0, s>>>(n_box, c->lbest.p, obj_hi, obj_err);
    CUDA_TRY(cudaGetLastError());
    if (x_point) CUDA_TRY(cudaMemcpyAsync(x_point, a.x_avg, nd * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return mark_done(c, s);
}

extern "C" ibp_status ibp_bound_linear(ibp_case *c, int32_t n_box, const double *box_lo,
                                       const double *box_hi, int32_t n_iter, double primal_weight,
                                       int32_t warm, double *obj_hi, double *obj_err,
                                       double *x_point, int32_t ptr_mode, void *cuda_stream) {
    if (!c) return fail(IBP_EINVAL, "case is NULL");
    if (n_box < 0 || n_box > kMaxBoxesPerCall) return fail(IBP_EINVAL, "n_box must be in [0, %d]", kMaxBoxesPerCall);
    if (n_iter < 0) return fail(IBP_EINVAL, "n_iter must be >= 0");
    if (warm < 0) return fail(IBP_EINVAL, "warm must be >= 0");
    if (!(primal_weight > 0.0) || !std::isfinite(primal_weight))
        return fail(IBP_EINVAL, "primal_weight must be finite and > 0");
    if (ptr_mode != 0 && ptr_mode != 1) return fail(IBP_EINVAL, "ptr_mode must be 0 or 1");
    if (n_box == 0) return ok();
    if (!box_lo || !box_hi || !obj_hi || !obj_err) return fail(IBP_EINVAL, "box and output pointers must not be NULL");
    if (ptr_mode == 0) {
        ibp_status st = check_boxes_host(c, n_box, box_lo, box_hi);
        if (st != IBP_OK) return st;
    }
    if (c->device < 0) return fail(IBP_ENOTSUP, "case was created without a device (dry run)");
    if (!c->phi64.p) return fail(IBP_ENOTSUP, "the case holds no FP64 PTDF");
    DeviceGuard guard(c->device);
    if (!guard.ok) return fail(IBP_ECUDA, "cannot select device %d", c->device);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    ibp_status st = ensure_workspace(c, n_box);
    if (st != IBP_OK) return st;
    if (ptr_mode == 1)
        return lin_run(c, n_box, box_lo, box_hi, n_iter, primal_weight, obj_hi, obj_err, x_point, s, warm != 0,
                       warm - 1);
    const size_t nd = (size_t)n_box * c->n_dev;
    CUDA_TRY(cudaMemcpyAsync(c->box_lo.p, box_lo, nd * sizeof(double), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->box_hi.p, box_hi, nd * sizeof(double), cudaMemcpyHostToDevice, s));
    double *dobj = c->obj.p;  // [n_box] bound, [n_box] error
    DevBuf<double> dx;
    if (x_point) CUDA_TRY(dx.alloc(nd));
    st = lin_run(c, n_box, c->box_lo.p, c->box_hi.p, n_iter, primal_weight, dobj, dobj + n_box,
                 x_point ? dx.p : nullptr, s, warm != 0, warm - 1);
    if (st != IBP_OK) return st;
    CUDA_TRY(cudaMemcpyAsync(obj_hi, dobj, n_box * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(obj_err, dobj + n_box, n_box * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (x_point) CUDA_TRY(cudaMemcpyAsync(x_point, dx.p, nd * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return ok();
}

// Rearranges the linear state for a new list of boxes: box j takes the state
// (slopes, running sums, point, primal weight) of box parent[j] (host array).
__global__ void k_lin_gather_f(const float *src, float *dst, const int *parent, int n_new, size_t per) {
    const size_t tot = (size_t)n_new * per;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[(size_t)parent[i / per] * per + i % per];
}
__global__ void k_lin_gather_d(const double *src, double *dst, const int *parent, int n_new, size_t per) {
    const size_t tot = (size_t)n_new * per;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[(size_t)parent[i / per] * per + i % per];
}

extern "C" ibp_status ibp_case_linear_inherit(ibp_case *c, int32_t n_new, const int32_t *parent) {
    if (!c || !parent) return fail(IBP_EINVAL, "NULL argument");
    if (c->device < 0) return fail(IBP_ENOTSUP, "dry-run case");
    if (n_new < 1 || n_new > kMaxBoxesPerCall) return fail(IBP_EINVAL, "n_new must be in [1, %d]", kMaxBoxesPerCall);
    for (int j = 0; j < n_new; ++j)
        if (parent[j] < 0 || parent[j] >= c->lin_state_box)
            return fail(IBP_EINVAL, "parent[%d] = %d is not a box of the linear state (%d boxes)", j, parent[j],
                        c->lin_state_box);
    DeviceGuard guard(c->device);
    if (!guard.ok) return fail(IBP_ECUDA, "cannot select device %d", c->device);
    ibp_status st = wait_case(c);
    if (st != IBP_OK) return st;
    const int old_cap = c->lin_cap_box;
    DevBuf<int> dpar;
    CUDA_TRY(dpar.alloc(n_new));
    CUDA_TRY(cudaMemcpy(dpar.p, parent, n_new * sizeof(int), cudaMemcpyHostToDevice));
    const size_t pc = (size_t)std::max(c->n_ctg, 1) * c->n_line;
    // gather into fresh buffers, then replace the old ones
    auto gf = [&](DevBuf<float> &b, size_t per) -> ibp_status {
        DevBuf<float> t;
        CUDA_TRY(t.alloc((size_t)std::max(n_new, old_cap) * per));
        k_lin_gather_f<<<c->num_sms * 8, 256>>>(b.p, t.p, dpar.p, n_new, per);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaDeviceSynchronize());
        std::swap(b.p, t.p);
        std::swap(b.n, t.n);
        return IBP_OK;
    };
    auto gd = [&](DevBuf<double> &b, size_t per) -> ibp_status {
        DevBuf<double> t;
        CUDA_TRY(t.alloc((size_t)std::max(n_new, old_cap) * per));
        k_lin_gather_d<<<c->num_sms * 8, 256>>>(b.p, t.p, dpar.p, n_new, per);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaDeviceSynchronize());
        std::swap(b.p, t.p);
        std::swap(b.n, t.n);
        return IBP_OK;
    };
    if ((st = gf(c->lac, pc)) || (st = gf(c->lc_last, pc)) ||
        (st = gf(c->lab, c->n_line)) || (st = gf(c->lb_last, c->n_line)) ||
        (st = gd(c->la0, 1)) || (st = gd(c->la0_last, 1)) || (st = gd(c->lw, 1)) ||
        (st = gd(c->lx, c->n_dev)) || (st = gd(c->lsx, c->n_dev)) || (st = gd(c->lxavg, c->n_dev)))
        return st;
    CUDA_TRY(cudaDeviceSynchronize());
    // the other per-box buffers only need the room
    if (n_new > old_cap) {
        c->lin_cap_box = old_cap;  // ensure_lin_workspace grows the rest (its state buffers are resized above)
        const size_t nd = (size_t)n_new * c->n_dev, nl = (size_t)n_new * c->n_line;
        const size_t na = (size_t)n_new * c->n_a_pad, nc = (size_t)n_new * std::max(c->n_ctg, 1);
        CUDA_TRY(c->lx_last.alloc(nd)); CUDA_TRY(c->lxb.alloc(nd));
        CUDA_TRY(c->lstot.alloc(n_new)); CUDA_TRY(c->lred.alloc((size_t)n_new * 4));
        CUDA_TRY(c->lstotp.alloc((size_t)n_new * ((c->n_dev + 127) / 128)));
        CUDA_TRY(c->lub.alloc(n_new)); CUDA_TRY(c->lub_err.alloc(n_new)); CUDA_TRY(c->lbest.alloc((size_t)n_new * 2));
        CUDA_TRY(c->lp.alloc(na)); CUDA_TRY(c->lf.alloc(nl)); CUDA_TRY(c->lcol.alloc(nl));
        CUDA_TRY(c->lrow.alloc(nc)); CUDA_TRY(c->lg.alloc(na));
        CUDA_TRY(c->lW64.alloc(nl)); CUDA_TRY(c->lWabs.alloc(nl)); CUDA_TRY(c->lconst.alloc(nl));
        CUDA_TRY(c->lrd64.alloc(nc)); CUDA_TRY(c->lrda.alloc(nc)); CUDA_TRY(c->lg64.alloc(na));
        CUDA_TRY(c->lG64.alloc(na));
        c->lin_cap_box = n_new;
        ++c->ws_gen;
    }
    CUDA_TRY(cudaMemset(c->lred.p, 0, (size_t)c->lin_cap_box * 4 * sizeof(double)));
    c->lin_state_box = n_new;
    return ok();
}

// The slopes of the last ibp_bound_linear call (host copies, for checking the
// certified value against an independent evaluation): a_ctg [n_box][n_ctg][n_line],
// a_base [n_box][n_line], a_inj [n_box].
extern "C" ibp_status ibp_case_linear_slopes(ibp_case *c, int32_t n_box, float *a_ctg, float *a_base,
                                             double *a_inj) {
    if (!c || !a_ctg || !a_base || !a_inj) return fail(IBP_EINVAL, "NULL argument");
    if (c->device < 0) return fail(IBP_ENOTSUP, "dry-run case");
    if (n_box < 1 || n_box > c->lin_cap_box) return fail(IBP_EINVAL, "no linear bound of that many boxes");
    DeviceGuard guard(c->device);
    ibp_status st = wait_case(c);
    if (st != IBP_OK) return st;
    const size_t np = (size_t)n_box * c->n_ctg * c->n_line;
    if (np) CUDA_TRY(cudaMemcpy(a_ctg, c->lac.p, np * sizeof(float), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(a_base, c->lab.p, (size_t)n_box * c->n_line * sizeof(float), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(a_inj, c->la0.p, n_box * sizeof(double), cudaMemcpyDeviceToHost));
    return ok();
}

