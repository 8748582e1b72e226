// C ABI of the library: argument validation, host-side graph checks, the FP64
// sensitivity build, per-call workspace, the launch sequence of a bound and of
// its adjoints, and the case settings.  The linear relaxation bound is in
// abi_linear.cu, many cases in one launch in abi_multi.cu.
#include "abi_case.h"

// ----------------------------------------------------------------- errors
static thread_local std::string g_last_error;

ibp_status fail(ibp_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

ibp_status ok() {
    g_last_error.clear();
    return IBP_OK;
}

// Test hook: device allocations larger than this many bytes fail as if the
// device were out of memory (0: no limit).  See ibp_set_alloc_limit.
std::atomic<long long> g_alloc_limit{0};

// ----------------------------------------------------------------- helpers
bool is_fin(double x) { return std::isfinite(x); }

static ibp_status check_pwl(const char *what, int n, const int32_t *nseg, const double *slope,
                            const double *bkpt, std::vector<int> &ptr) {
    ptr.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        if (nseg[i] < 1 || nseg[i] > 1024)
            return fail(IBP_EINVAL, "%s_nseg[%d] = %d out of [1, 1024]", what, i, nseg[i]);
        ptr[i + 1] = ptr[i] + nseg[i];
    }
    for (int i = 0; i < n; ++i) {
        for (int m = ptr[i]; m < ptr[i + 1]; ++m) {
            if (!is_fin(slope[m]) || slope[m] < 0)
                return fail(IBP_EINVAL, "%s_slope[%d] must be finite and >= 0", what, m);
            if (!is_fin(bkpt[m])) return fail(IBP_EINVAL, "%s_bkpt[%d] is not finite", what, m);
            if (m > ptr[i] && !(bkpt[m] > bkpt[m - 1]))
                return fail(IBP_EINVAL, "%s_bkpt of device %d must increase", what, i);
        }
    }
    return IBP_OK;
}

// connectivity (BFS) and bridges (iterative Tarjan low-link) on the host
static bool connected(int n, const std::vector<std::vector<std::pair<int, int>>> &adj) {
    std::vector<char> seen(n, 0);
    std::vector<int> st{0};
    seen[0] = 1;
    int cnt = 1;
    while (!st.empty()) {
        int v = st.back();
        st.pop_back();
        for (auto &e : adj[v])
            if (!seen[e.first]) {
                seen[e.first] = 1;
                ++cnt;
                st.push_back(e.first);
            }
    }
    return cnt == n;
}

static std::vector<char> bridges(int n, int m, const std::vector<std::vector<std::pair<int, int>>> &adj) {
    std::vector<char> is_bridge(m, 0);
    std::vector<int> disc(n, -1), low(n, 0);
    int t = 0;
    struct Frame { int v, pe; size_t i; };
    for (int root = 0; root < n; ++root) {
        if (disc[root] >= 0) continue;
        std::vector<Frame> st{{root, -1, 0}};
        disc[root] = low[root] = t++;
        while (!st.empty()) {
            Frame &f = st.back();
            if (f.i < adj[f.v].size()) {
                auto [w, e] = adj[f.v][f.i++];
                if (e == f.pe) continue;
                if (disc[w] < 0) {
                    disc[w] = low[w] = t++;
                    st.push_back({w, e, 0});
                } else {
                    low[f.v] = std::min(low[f.v], disc[w]);
                }
            } else {
                int v = f.v, pe = f.pe;
                st.pop_back();
                if (!st.empty()) {
                    int u = st.back().v;
                    low[u] = std::min(low[u], low[v]);
                    if (low[v] > disc[u]) is_bridge[pe] = 1;
                }
            }
        }
    }
    return is_bridge;
}

static int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Bus classes of the exact network reduction.  Removing the bridges leaves the
// 2-edge-connected components; an injection at bus b, withdrawn at the slack,
// enters a component C through one vertex e_C(b) (b itself when b is in C) and
// leaves it through e_C(slack), so on a line inside C its flow depends on b
// only through e_C(b).  Buses with the same e_C for every component that has
// a line inside it therefore have equal PTDF columns on every non-bridge line,
// and buses with e_C(b) = e_C(slack) for all those components have a zero
// column there.  Returns the classes as CSR over active column indices
// (ascending within a class, classes ordered by their first member) without
// the slack's class.
static void bus_classes(int n, const std::vector<std::vector<std::pair<int, int>>> &adj,
                        const std::vector<char> &br, const std::vector<int> &active, int slack,
                        std::vector<int> &cls_ptr, std::vector<int> &cls_col) {
    std::vector<int> comp(n, -1), size;
    for (int r = 0; r < n; ++r) {
        if (comp[r] >= 0) continue;
        const int id = (int)size.size();
        size.push_back(0);
        std::vector<int> st{r};
        comp[r] = id;
        while (!st.empty()) {
            const int v = st.back();
            st.pop_back();
            ++size[id];
            for (auto [w, e] : adj[v])
                if (!br[e] && comp[w] < 0) {
                    comp[w] = id;
                    st.push_back(w);
                }
        }
    }
    std::vector<int> key(n, 0), label(n);
    for (int C = 0; C < (int)size.size(); ++C) {
        if (size[C] < 2) continue;  // no line inside
        // multi-source search from the vertices of C that avoids C's own lines
        std::fill(label.begin(), label.end(), -1);
        std::vector<int> st;
        for (int v = 0; v < n; ++v)
            if (comp[v] == C) {
                label[v] = v;
                st.push_back(v);
            }
        while (!st.empty()) {
            const int v = st.back();
            st.pop_back();
            for (auto [w, e] : adj[v]) {
                if (comp[v] == C && comp[w] == C) continue;
                if (label[w] < 0) {
                    label[w] = label[v];
                    st.push_back(w);
                }
            }
        }
        // refine the partition by the entry vertex
        std::map<std::pair<int, int>, int> ids;
        for (int v = 0; v < n; ++v) {
            auto it = ids.emplace(std::make_pair(key[v], label[v]), (int)ids.size()).first;
            key[v] = it->second;
        }
    }
    std::map<int, int> cls_of_key;
    std::vector<std::vector<int>> members;
    for (size_t i = 0; i < active.size(); ++i) {
        const int k = key[active[i]];
        if (k == key[slack]) continue;
        auto it = cls_of_key.emplace(k, (int)members.size()).first;
        if (it->second == (int)members.size()) members.emplace_back();
        members[it->second].push_back((int)i);
    }
    cls_ptr.assign(1, 0);
    cls_col.clear();
    for (auto &m : members) {
        cls_col.insert(cls_col.end(), m.begin(), m.end());
        cls_ptr.push_back((int)cls_col.size());
    }
}

// worst-case relative excess of a round-up sum accumulated in levels of
// n1, n2, n3 terms: (1 + 2u)^(n1 + n2 + n3) - 1, with slack
float rup_gamma(long n1, long n2, long n3) {
    const double u = std::ldexp(1.0, -24);
    const double n = (double)(n1 + n2 + n3 + 2);
    return (float)(std::expm1(n * std::log1p(2 * u)) * 1.01);
}

// ----------------------------------------------------------------- tensor maps
namespace ibp {
bool encode_map_2d(CUtensorMap *map, const float *base, int64_t inner, int64_t outer,
                   int64_t row_stride_elems, int box_inner, int box_outer, std::string *err,
                   bool swizzle) {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p) {
            *err = "cuTensorMapEncodeTiled is not available";
            return false;
        }
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)(row_stride_elems * sizeof(float))};
    cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides,
                    box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        *err = "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r);
        return false;
    }
    return true;
}
}  // namespace ibp

// ----------------------------------------------------------------- the build
static ibp_status build_sensitivities(ibp_case *c, const std::vector<int> &from,
                                      const std::vector<int> &to, const double *x,
                                      const std::vector<int> &active) {
    const int nb_r = c->n_bus - 1;
    const int n_l = c->n_line, n_c = c->n_ctg;
    std::vector<int> red(c->n_bus, -1);
    for (int b = 0, r = 0; b < c->n_bus; ++b)
        if (b != c->slack) red[b] = r++;

    // reduced admittance Y_B,r = E_r^T Y_D E_r (eq. (line flow ptdf)), as COO
    std::map<std::pair<int, int>, double> Y;
    for (int l = 0; l < n_l; ++l) {
        const double b = 1.0 / x[l];
        const int i = red[from[l]], j = red[to[l]];
        if (i >= 0) Y[{i, i}] += b;
        if (j >= 0) Y[{j, j}] += b;
        if (i >= 0 && j >= 0) {
            Y[{i, j}] -= b;
            Y[{j, i}] -= b;
        }
    }
    std::vector<int> yr, yc;
    std::vector<double> yv;
    for (auto &kv : Y) {
        yr.push_back(kv.first.first);
        yc.push_back(kv.first.second);
        yv.push_back(kv.second);
    }
    // right-hand sides E_r^T Y_D: column l has b_l at from, -b_l at to
    std::vector<int> rr, rc;
    std::vector<double> rv;
    for (int l = 0; l < n_l; ++l) {
        const double b = 1.0 / x[l];
        if (red[from[l]] >= 0) { rr.push_back(red[from[l]]); rc.push_back(l); rv.push_back(b); }
        if (red[to[l]] >= 0) { rr.push_back(red[to[l]]); rc.push_back(l); rv.push_back(-b); }
    }

    cudaStream_t s = nullptr;
    DevBuf<double> dY, dZ, dV1, dV2;
    DevBuf<int> dI1, dI2, dI3, dI4, dinfo;
    CUDA_TRY(dY.alloc((size_t)nb_r * nb_r));
    CUDA_TRY(dZ.alloc((size_t)nb_r * n_l));
    CUDA_TRY(cudaMemsetAsync(dY.p, 0, (size_t)nb_r * nb_r * sizeof(double), s));
    CUDA_TRY(cudaMemsetAsync(dZ.p, 0, (size_t)nb_r * n_l * sizeof(double), s));
    CUDA_TRY(dV1.alloc(yv.size()));
    CUDA_TRY(dI1.alloc(yv.size()));
    CUDA_TRY(dI2.alloc(yv.size()));
    CUDA_TRY(cudaMemcpy(dV1.p, yv.data(), yv.size() * sizeof(double), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(dI1.p, yr.data(), yr.size() * sizeof(int), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(dI2.p, yc.data(), yc.size() * sizeof(int), cudaMemcpyHostToDevice));
    CUDA_TRY(launch_scatter_dense(dY.p, nb_r, dI1.p, dI2.p, dV1.p, (int)yv.size(), s));
    CUDA_TRY(dV2.alloc(rv.size()));
    CUDA_TRY(dI3.alloc(rv.size()));
    CUDA_TRY(dI4.alloc(rv.size()));
    CUDA_TRY(cudaMemcpy(dV2.p, rv.data(), rv.size() * sizeof(double), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(dI3.p, rr.data(), rr.size() * sizeof(int), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(dI4.p, rc.data(), rc.size() * sizeof(int), cudaMemcpyHostToDevice));
    CUDA_TRY(launch_scatter_dense(dZ.p, nb_r, dI3.p, dI4.p, dV2.p, (int)rv.size(), s));

    // Cholesky of the SPD reduced Laplacian, then Z = Y^-1 E_r^T Y_D = Phi_r^T
    cusolverDnHandle_t h = nullptr;
    if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS) return fail(IBP_ECUDA, "cusolverDnCreate failed");
    std::unique_ptr<cusolverDnContext, decltype(&cusolverDnDestroy)> hg(h, cusolverDnDestroy);
    int lwork = 0;
    if (cusolverDnDpotrf_bufferSize(h, CUBLAS_FILL_MODE_LOWER, nb_r, dY.p, nb_r, &lwork) !=
        CUSOLVER_STATUS_SUCCESS)
        return fail(IBP_ECUDA, "cusolverDnDpotrf_bufferSize failed");
    DevBuf<double> work;
    CUDA_TRY(work.alloc((size_t)std::max(lwork, 1)));
    CUDA_TRY(dinfo.alloc(1));
    if (cusolverDnDpotrf(h, CUBLAS_FILL_MODE_LOWER, nb_r, dY.p, nb_r, work.p, lwork, dinfo.p) !=
        CUSOLVER_STATUS_SUCCESS)
        return fail(IBP_ECUDA, "cusolverDnDpotrf failed");
    int info = 0;
    CUDA_TRY(cudaMemcpy(&info, dinfo.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (info != 0)
        return fail(IBP_ESINGULAR, "Cholesky of the reduced admittance failed (info=%d)", info);
    if (cusolverDnDpotrs(h, CUBLAS_FILL_MODE_LOWER, nb_r, n_l, dY.p, nb_r, dZ.p, nb_r, dinfo.p) !=
        CUSOLVER_STATUS_SUCCESS)
        return fail(IBP_ECUDA, "cusolverDnDpotrs failed");
    CUDA_TRY(cudaMemcpy(&info, dinfo.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (info != 0) return fail(IBP_ESINGULAR, "Cholesky solve failed (info=%d)", info);
    work.free();
    dY.free();

    // FP32 PTDF of the active buses
    std::vector<int> act_red(active.size());
    for (size_t i = 0; i < active.size(); ++i) act_red[i] = red[active[i]];
    DevBuf<int> dact;
    CUDA_TRY(dact.alloc(act_red.size()));
    if (!act_red.empty())
        CUDA_TRY(cudaMemcpy(dact.p, act_red.data(), act_red.size() * sizeof(int), cudaMemcpyHostToDevice));
    CUDA_TRY(c->phi_a.alloc((size_t)n_l * c->n_a_pad));
    CUDA_TRY(c->phi64.alloc((size_t)n_l * c->n_a_pad));
    CUDA_TRY(launch_extract_phi(dZ.p, nb_r, n_l, dact.p, c->n_a, c->n_a_pad, c->phi_a.p, c->phi64.p, s));
    CUDA_TRY(c->phi_k.alloc((size_t)std::max(n_c, 1) * c->n_a_pad));
    CUDA_TRY(launch_gather_rows(c->phi_a.p, c->n_a_pad, c->ctg_line.p, n_c, c->phi_k.p, s));

    // LODF of the contingency list
    CUDA_TRY(c->lodf.alloc((size_t)std::max(n_c, 1) * n_l));
    if (n_c > 0) {
        std::vector<int> cf(n_c), ct(n_c);
        for (int k = 0; k < n_c; ++k) {
            cf[k] = red[from[c->ctg_line_h[k]]];
            ct[k] = red[to[c->ctg_line_h[k]]];
        }
        DevBuf<int> dcf, dct;
        DevBuf<double> dden;
        DevBuf<float> dmax;
        CUDA_TRY(dcf.alloc(n_c));
        CUDA_TRY(dct.alloc(n_c));
        CUDA_TRY(dden.alloc(n_c));
        CUDA_TRY(dmax.alloc(1));
        CUDA_TRY(cudaMemcpy(dcf.p, cf.data(), n_c * sizeof(int), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(dct.p, ct.data(), n_c * sizeof(int), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemset(dmax.p, 0, sizeof(float)));
        CUDA_TRY(c->lodf_lo.alloc((size_t)n_c * n_l));
        CUDA_TRY(launch_lodf(dZ.p, nb_r, n_l, n_c, dcf.p, dct.p, c->ctg_line.p, c->lodf.p, c->lodf_lo.p,
                             dden.p, dmax.p, s));
        std::vector<double> den(n_c);
        float mx = 0;
        CUDA_TRY(cudaMemcpy(den.data(), dden.p, n_c * sizeof(double), cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemcpy(&mx, dmax.p, sizeof(float), cudaMemcpyDeviceToHost));
        for (int k = 0; k < n_c; ++k)
            if (!(std::fabs(den[k]) > 1e-9))
                return fail(IBP_EISLAND, "contingency %d (line %d) islands the network", k,
                            c->ctg_line_h[k]);
        c->max_abs_lodf = mx;
    }
    CUDA_TRY(cudaDeviceSynchronize());
    return IBP_OK;
}

// ----------------------------------------------------------------- create
extern "C" ibp_status ibp_case_create(int32_t n_bus, int32_t slack_bus, int32_t n_line,
                                      const int32_t *line_from, const int32_t *line_to,
                                      const double *reactance, const double *rating,
                                      const double *rating_ctg, int32_t n_gen,
                                      const int32_t *gen_bus, const int32_t *gen_nseg,
                                      const double *gen_slope, const double *gen_bkpt,
                                      int32_t n_load, const int32_t *load_bus,
                                      const int32_t *load_nseg, const double *load_slope,
                                      const double *load_bkpt, double zeta_inj, double zeta_f,
                                      int32_t n_ctg, const int32_t *ctg_line, int32_t device,
                                      ibp_case **out) {
    if (!out) return fail(IBP_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_bus < 2) return fail(IBP_EINVAL, "n_bus must be >= 2");
    if (slack_bus < 0 || slack_bus >= n_bus) return fail(IBP_EINVAL, "slack_bus out of range");
    if (n_line < 1) return fail(IBP_EINVAL, "n_line must be >= 1");
    if (n_gen < 0 || n_load < 0 || n_gen + n_load < 1)
        return fail(IBP_EINVAL, "need n_gen, n_load >= 0 and at least one device");
    if (n_ctg < 0) return fail(IBP_EINVAL, "n_ctg must be >= 0");
    if (!line_from || !line_to || !reactance || !rating)
        return fail(IBP_EINVAL, "line arrays must not be NULL");
    if ((n_gen > 0 && (!gen_bus || !gen_nseg || !gen_slope || !gen_bkpt)) ||
        (n_load > 0 && (!load_bus || !load_nseg || !load_slope || !load_bkpt)))
        return fail(IBP_EINVAL, "device arrays must not be NULL");
    if (n_ctg > 0 && !ctg_line) return fail(IBP_EINVAL, "ctg_line is NULL");
    if (!is_fin(zeta_inj) || !is_fin(zeta_f) || zeta_inj < 0 || zeta_f < 0)
        return fail(IBP_EINVAL, "penalty prices must be finite and >= 0");
    for (int l = 0; l < n_line; ++l) {
        if (line_from[l] < 0 || line_from[l] >= n_bus || line_to[l] < 0 || line_to[l] >= n_bus)
            return fail(IBP_EINVAL, "line %d has a bus index out of range", l);
        if (line_from[l] == line_to[l]) return fail(IBP_EINVAL, "line %d is a self loop", l);
        if (!is_fin(reactance[l]) || !(reactance[l] > 0))
            return fail(IBP_EINVAL, "reactance[%d] must be finite and > 0", l);
        if (!is_fin(rating[l]) || rating[l] < 0)
            return fail(IBP_EINVAL, "rating[%d] must be finite and >= 0", l);
        if (rating_ctg && (!is_fin(rating_ctg[l]) || rating_ctg[l] < 0))
            return fail(IBP_EINVAL, "rating_ctg[%d] must be finite and >= 0", l);
    }
    for (int i = 0; i < n_gen; ++i)
        if (gen_bus[i] < 0 || gen_bus[i] >= n_bus) return fail(IBP_EINVAL, "gen_bus[%d] out of range", i);
    for (int i = 0; i < n_load; ++i)
        if (load_bus[i] < 0 || load_bus[i] >= n_bus) return fail(IBP_EINVAL, "load_bus[%d] out of range", i);
    for (int k = 0; k < n_ctg; ++k)
        if (ctg_line[k] < 0 || ctg_line[k] >= n_line) return fail(IBP_EINVAL, "ctg_line[%d] out of range", k);
    std::vector<int> gptr, lptr;
    ibp_status st;
    if ((st = check_pwl("gen", n_gen, gen_nseg, gen_slope, gen_bkpt, gptr)) != IBP_OK) return st;
    if ((st = check_pwl("load", n_load, load_nseg, load_slope, load_bkpt, lptr)) != IBP_OK) return st;

    // graph checks on the host, before any device work
    std::vector<std::vector<std::pair<int, int>>> adj(n_bus);
    for (int l = 0; l < n_line; ++l) {
        adj[line_from[l]].push_back({line_to[l], l});
        adj[line_to[l]].push_back({line_from[l], l});
    }
    if (!connected(n_bus, adj)) return fail(IBP_EISLAND, "the network is not connected");
    const std::vector<char> br = bridges(n_bus, n_line, adj);
    for (int k = 0; k < n_ctg; ++k)
        if (br[ctg_line[k]])
            return fail(IBP_EISLAND, "contingency %d outages bridge line %d (islanding)", k, ctg_line[k]);

    std::unique_ptr<ibp_case> c(new ibp_case());
    c->n_bus = n_bus;
    c->slack = slack_bus;
    c->n_line = n_line;
    c->n_gen = n_gen;
    c->n_load = n_load;
    c->n_dev = n_gen + n_load;
    c->n_ctg = n_ctg;
    c->zeta_inj = zeta_inj;
    c->zeta_f = zeta_f;
    c->ctg_line_h.assign(ctg_line, ctg_line + n_ctg);

    // active bus columns: buses with a device, slack excluded, in bus order
    std::vector<std::vector<int>> devs_at(n_bus);
    for (int i = 0; i < n_gen; ++i) devs_at[gen_bus[i]].push_back(i);
    for (int i = 0; i < n_load; ++i) devs_at[load_bus[i]].push_back(n_gen + i);
    std::vector<int> active, aptr{0}, adev;
    for (int b = 0; b < n_bus; ++b) {
        if (b == slack_bus || devs_at[b].empty()) continue;
        active.push_back(b);
        for (int d : devs_at[b]) adev.push_back(d);
        aptr.push_back((int)adev.size());
    }
    c->n_a = (int)active.size();
    c->n_a_pad = round_up(std::max(c->n_a, 1), 32);
    // exact network reduction for the contingency kernel (host part)
    bus_classes(n_bus, adj, br, active, slack_bus, c->cls_ptr_h, c->cls_col_h);
    c->is_bridge_h.resize(n_line);
    for (int l = 0; l < n_line; ++l) c->is_bridge_h[l] = br[l] ? 1 : 0;
    c->n_bridges = (int)std::count(c->is_bridge_h.begin(), c->is_bridge_h.end(), 1);
    c->n_r = (int)c->cls_ptr_h.size() - 1;
    c->n_r_pad = round_up(std::max(c->n_r, 1), 32);
    c->has_reduction = c->n_bridges > 0 || c->n_r < c->n_a;

    if (device < 0) {  // dry run: validation only
        c->device = -1;
        *out = c.release();
        return ok();
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return fail(IBP_ECUDA, "no CUDA device is available");
    if (device >= ndev) return fail(IBP_EINVAL, "device %d out of range (%d devices)", device, ndev);
    DeviceGuard guard(device);
    if (!guard.ok) return fail(IBP_ECUDA, "cannot select device %d", device);
    c->device = device;
    CUDA_TRY(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));

    const auto t0 = std::chrono::steady_clock::now();
    // small persistent arrays
    auto up32 = [](double v) {
        float f = (float)v;
        return (double)f < v ? std::nextafter(f, INFINITY) : f;
    };
    auto dn32 = [](double v) {
        float f = (float)v;
        return (double)f > v ? std::nextafter(f, -INFINITY) : f;
    };
    std::vector<float> ru(n_line), rd(n_line), rcu(n_line), rcd(n_line);
    for (int l = 0; l < n_line; ++l) {
        ru[l] = up32(rating[l]);
        rd[l] = dn32(rating[l]);
        const double rc = rating_ctg ? rating_ctg[l] : rating[l];
        rcu[l] = up32(rc);
        rcd[l] = dn32(rc);
    }
    {
        std::vector<double> r64(rating, rating + n_line), rc64(n_line);
        for (int l = 0; l < n_line; ++l) rc64[l] = rating_ctg ? rating_ctg[l] : rating[l];
        CUDA_TRY(c->rate64.alloc(n_line));
        CUDA_TRY(c->rate_c64.alloc(n_line));
        CUDA_TRY(cudaMemcpy(c->rate64.p, r64.data(), n_line * sizeof(double), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(c->rate_c64.p, rc64.data(), n_line * sizeof(double), cudaMemcpyHostToDevice));
    }
    CUDA_TRY(c->rate_up.alloc(n_line));
    CUDA_TRY(c->rate_dn.alloc(n_line));
    CUDA_TRY(c->rate_c_up.alloc(n_line));
    CUDA_TRY(c->rate_c_dn.alloc(n_line));
    CUDA_TRY(cudaMemcpy(c->rate_up.p, ru.data(), n_line * sizeof(float), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c->rate_dn.p, rd.data(), n_line * sizeof(float), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c->rate_c_up.p, rcu.data(), n_line * sizeof(float), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c->rate_c_dn.p, rcd.data(), n_line * sizeof(float), cudaMemcpyHostToDevice));
    CUDA_TRY(c->ctg_line.alloc(std::max(n_ctg, 1)));
    if (n_ctg > 0)
        CUDA_TRY(cudaMemcpy(c->ctg_line.p, ctg_line, n_ctg * sizeof(int), cudaMemcpyHostToDevice));
    CUDA_TRY(c->act_ptr.alloc(aptr.size()));
    CUDA_TRY(cudaMemcpy(c->act_ptr.p, aptr.data(), aptr.size() * sizeof(int), cudaMemcpyHostToDevice));
    CUDA_TRY(c->act_dev.alloc(std::max<size_t>(adev.size(), 1)));
    if (!adev.empty())
        CUDA_TRY(cudaMemcpy(c->act_dev.p, adev.data(), adev.size() * sizeof(int), cudaMemcpyHostToDevice));
    std::vector<int> sp(c->n_dev + 1, 0);
    std::vector<double> sl, bk;
    for (int i = 0; i < n_gen; ++i) {
        for (int m = gptr[i]; m < gptr[i + 1]; ++m) { sl.push_back(gen_slope[m]); bk.push_back(gen_bkpt[m]); }
        sp[i + 1] = (int)sl.size();
    }
    for (int i = 0; i < n_load; ++i) {
        for (int m = lptr[i]; m < lptr[i + 1]; ++m) { sl.push_back(load_slope[m]); bk.push_back(load_bkpt[m]); }
        sp[n_gen + i + 1] = (int)sl.size();
    }
    CUDA_TRY(c->seg_ptr.alloc(sp.size()));
    CUDA_TRY(c->slope.alloc(sl.size()));
    CUDA_TRY(c->bkpt.alloc(bk.size()));
    CUDA_TRY(cudaMemcpy(c->seg_ptr.p, sp.data(), sp.size() * sizeof(int), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c->slope.p, sl.data(), sl.size() * sizeof(double), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c->bkpt.p, bk.data(), bk.size() * sizeof(double), cudaMemcpyHostToDevice));
    CUDA_TRY(c->err.alloc(1));
    {
        std::vector<int> col_of_bus(n_bus, -1), dcol(c->n_dev);
        for (size_t i = 0; i < active.size(); ++i) col_of_bus[active[i]] = (int)i;
        for (int i = 0; i < n_gen; ++i) dcol[i] = col_of_bus[gen_bus[i]];
        for (int i = 0; i < n_load; ++i) dcol[n_gen + i] = col_of_bus[load_bus[i]];
        CUDA_TRY(c->dev_col.alloc(c->n_dev));
        CUDA_TRY(cudaMemcpy(c->dev_col.p, dcol.data(), c->n_dev * sizeof(int), cudaMemcpyHostToDevice));
    }

    std::vector<int> from(line_from, line_from + n_line), to(line_to, line_to + n_line);
    if ((st = build_sensitivities(c.get(), from, to, reactance, active)) != IBP_OK) return st;
    {
        // exact network reduction for the contingency kernel (device part)
        const std::vector<int> &cptr = c->cls_ptr_h, &ccol = c->cls_col_h, &isb = c->is_bridge_h;
        if (c->has_reduction) {
            std::vector<int> rep_col(std::max(c->n_r, 1), 0);
            for (int j = 0; j < c->n_r; ++j) rep_col[j] = ccol[cptr[j]];
            DevBuf<int> drep;
            CUDA_TRY(drep.alloc(rep_col.size()));
            CUDA_TRY(cudaMemcpy(drep.p, rep_col.data(), rep_col.size() * sizeof(int), cudaMemcpyHostToDevice));
            CUDA_TRY(c->is_bridge.alloc(n_line));
            CUDA_TRY(cudaMemcpy(c->is_bridge.p, isb.data(), n_line * sizeof(int), cudaMemcpyHostToDevice));
            CUDA_TRY(c->cls_ptr.alloc(cptr.size()));
            CUDA_TRY(cudaMemcpy(c->cls_ptr.p, cptr.data(), cptr.size() * sizeof(int), cudaMemcpyHostToDevice));
            CUDA_TRY(c->cls_col.alloc(std::max<size_t>(ccol.size(), 1)));
            if (!ccol.empty())
                CUDA_TRY(cudaMemcpy(c->cls_col.p, ccol.data(), ccol.size() * sizeof(int), cudaMemcpyHostToDevice));
            CUDA_TRY(c->phi_r.alloc((size_t)n_line * c->n_r_pad));
            CUDA_TRY(launch_gather_cols(c->phi_a.p, c->n_a_pad, n_line, drep.p, c->n_r, c->phi_r.p,
                                        c->n_r_pad, nullptr));
            CUDA_TRY(c->phi_kr.alloc((size_t)std::max(n_ctg, 1) * c->n_r_pad));
            CUDA_TRY(launch_gather_rows(c->phi_r.p, c->n_r_pad, c->ctg_line.p, n_ctg, c->phi_kr.p, nullptr));
            CUDA_TRY(cudaDeviceSynchronize());
        }
    }
    c->build_seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (auto &e : c->ev) CUDA_TRY(cudaEventCreate(&e));
    CUDA_TRY(cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming));
    CUDA_TRY(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    c->n_part_base = base_partials_count(c->num_sms);
    *out = c.release();
    return ok();
}

extern "C" void ibp_case_destroy(ibp_case *c) {
    if (!c) return;
    drop_plans_of(c);
    delete c;
}

namespace ibp {
bool case_view(const ibp_case *c, CaseView *v) {
    if (!c || !v || c->device < 0) return false;
    v->device = c->device; v->n_line = c->n_line; v->n_ctg = c->n_ctg; v->n_gen = c->n_gen;
    v->n_dev = c->n_dev; v->n_a = c->n_a; v->n_a_pad = c->n_a_pad; v->num_sms = c->num_sms;
    v->zeta_inj = c->zeta_inj; v->zeta_f = c->zeta_f;
    v->phi_a = c->phi_a.p; v->lodf = c->lodf.p; v->rate_up = c->rate_up.p; v->rate_dn = c->rate_dn.p;
    v->rate_c_up = c->rate_c_up.p; v->rate_c_dn = c->rate_c_dn.p; v->ctg_line = c->ctg_line.p;
    v->act_ptr = c->act_ptr.p; v->act_dev = c->act_dev.p; v->seg_ptr = c->seg_ptr.p;
    v->slope = c->slope.p; v->bkpt = c->bkpt.p; v->n_part_base = c->n_part_base;
    v->phi64 = c->refine ? c->phi64.p : nullptr;
    v->lodf_lo = c->lodf_lo.p;
    v->rate64 = c->rate64.p; v->rate_c64 = c->rate_c64.p;
    return true;
}

ibp_status set_error(ibp_status s, const char *msg) {
    if (s == IBP_OK) return ok();
    return fail(s, "%s", msg);
}
}  // namespace ibp

// ----------------------------------------------------------------- workspace
// fastest shapes measured on GB300: one box, 2 CTAs per SM of 8 warps, 4x4
// pairs per thread, 64-bus chunks in 2 stages, packed two-lane sums; many
// boxes, 8 warps in two box halves, 4 lines x 2 contingencies x 8 boxes per
// thread, packed FMA, 6 stages
constexpr int kDefaultOneBoxVariant = 16;
constexpr int kDefaultMultiBoxVariant = 30;

static const CtgVariant *pick_variant(const ibp_case *c, int n_box) {
    if (c->variant > 0) {
        const CtgVariant *v = ctg_variant_by_id(c->variant);
        if (v && (v->batched != 0) == (n_box > 1)) return v;
    }
    return ctg_variant_by_id(n_box > 1 ? kDefaultMultiBoxVariant : kDefaultOneBoxVariant);
}

// partial-sum rows of the contingency kernels: (line, contingency) tiles x warps
size_t max_part_rows(const ibp_case *c) {
    int n;
    size_t best = 1;
    const CtgVariant *v = ctg_variants(&n);
    for (int i = 0; i < n; ++i) {
        const size_t t = (size_t)((c->n_line + v[i].BL - 1) / v[i].BL) *
                         ((std::max(c->n_ctg, 1) + v[i].BK - 1) / v[i].BK) * ctg_warps(v[i]);
        best = std::max(best, t);
    }
    return best;
}

// blocks per box of the first stage of the contingency partial sums

ibp_status ensure_workspace(ibp_case *c, int n_box) {
    if (n_box <= c->cap_box) return IBP_OK;
    const int cap = std::max(n_box, 1);
    const size_t na = c->n_a_pad;
    // buffers move from here on: a failure part-way leaves cap_box = 0, so the
    // next call allocates every buffer again
    c->cap_box = 0;
    ++c->ws_gen;
    CUDA_TRY(c->box_lo.alloc((size_t)cap * c->n_dev));
    CUDA_TRY(c->box_hi.alloc((size_t)cap * c->n_dev));
    CUDA_TRY(c->obj.alloc((size_t)cap * 4));
    CUDA_TRY(c->cbus.alloc(cap * na));
    CUDA_TRY(c->cbus2.alloc(cap * na));
    CUDA_TRY(c->rbus.alloc(cap * na));
    CUDA_TRY(c->rbus64.alloc(cap * na));
    CUDA_TRY(c->cabs.alloc(cap * na));
    CUDA_TRY(c->box_consts.alloc((size_t)cap * 4));
    CUDA_TRY(c->bus_part.alloc((size_t)cap * bus_blocks(c->n_a_pad) * 4));
    CUDA_TRY(c->line_c.alloc((size_t)cap * c->n_line));
    CUDA_TRY(c->line_e.alloc((size_t)cap * c->n_line));
    CUDA_TRY(c->line_R.alloc((size_t)cap * c->n_line));
    CUDA_TRY(c->part_base.alloc((size_t)c->n_part_base * cap * kPartVals));
    CUDA_TRY(c->part_ctg.alloc(max_part_rows(c) * cap * kPartVals));
    CUDA_TRY(c->part_stage.alloc((size_t)kPartStages * cap * kAsmVals));
    const int cap_pad = (cap + kBoxTile - 1) / kBoxTile * kBoxTile;
    CUDA_TRY(c->rbus_t.alloc(na * cap_pad));
    if (!c->live.p || !c->live_flag.p || !c->n_live.p) {
        CUDA_TRY(c->live_flag.alloc(std::max(c->n_line, 1)));
        CUDA_TRY(c->live.alloc(std::max(c->n_line, 1)));
        CUDA_TRY(c->n_live.alloc(1));
    }
    c->cap_box = cap;
    ++c->ws_gen;
    return IBP_OK;
}

// class radii of the reduction, sized like the other per-box buffers
ibp_status ensure_class_ws(ibp_case *c) {
    const size_t cap_pad = (size_t)(c->cap_box + kBoxTile - 1) / kBoxTile * kBoxTile;
    if (c->rcls.n >= (size_t)c->cap_box * c->n_r_pad && c->rcls_t.n >= cap_pad * c->n_r_pad)
        return IBP_OK;
    CUDA_TRY(c->rcls.alloc((size_t)c->cap_box * c->n_r_pad));
    CUDA_TRY(c->rcls_t.alloc(cap_pad * c->n_r_pad));
    ++c->ws_gen;
    return IBP_OK;
}

// Arguments of the FP64 refinement of the terms that can reach obj_hi (all
// null when the case does not refine).
RefArgs ref_args(const ibp_case *c) {
    RefArgs r{};
    if (!c->refine || !c->phi64.p) return r;
    r.phi_hi = c->phi_a.p; r.phi64 = c->phi64.p; r.cbus = c->cbus.p; r.rbus64 = c->rbus64.p;
    r.rbus = c->rbus.p; r.cabs = c->cabs.p; r.box_consts = c->box_consts.p;
    r.rate64 = c->rate64.p; r.rate_c64 = c->rate_c64.p; r.n_a_pad = c->n_a_pad;
    r.lodf = c->lodf.p; r.lodf_lo = c->lodf_lo.p; r.n_l = c->n_line;
    return r;
}

// The global refinement queues of a contingency launch: kRefQCap entries per
// (CTA, warp) region, for up to kRefRegionsPerSm regions per SM.
int ref_regions(int num_sms) { return num_sms * kRefRegionsPerSm; }


// Record the completion of the work just enqueued on s for ibp_case_sync.
ibp_status mark_done(ibp_case *c, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) {
        c->captured = true;
        return IBP_OK;
    }
    CUDA_TRY(cudaEventRecord(c->done, s));
    return IBP_OK;
}

// Wait for the case's last call: its completion event, or the device when a
// call was captured into a graph since the last wait.
ibp_status wait_case(ibp_case *c) {
    if (c->captured) {
        CUDA_TRY(cudaDeviceSynchronize());
        c->captured = false;
    } else {
        CUDA_TRY(cudaEventSynchronize(c->done));
    }
    return IBP_OK;
}

// ----------------------------------------------------------------- bound
static ibp_status enqueue_bound(ibp_case *c, int n_box, const double *lo, const double *hi,
                                double *olo, double *ohi, double *oerr, float *flo, float *fhi,
                                cudaStream_t s, bool record = false, bool paper = false,
                                bool record_lo = false) {
    ibp_status st = ensure_workspace(c, n_box);
    if (st != IBP_OK) return st;
    const CtgVariant *v = pick_variant(c, n_box);
    if (!v) return fail(IBP_EINVAL, "no kernel variant");
    const bool multi = n_box > 1;
    // the screen and the reduction leave the flows of the lines they drop unwritten
    // paper mode: the two-part contingency intervals, no tight kernel
    const bool reduced = !paper && c->reduce && c->has_reduction && !flo && c->n_ctg > 0;
    const bool screened = !paper && (c->screen || reduced) && !flo && c->n_ctg > 0;
    c->last_screened = screened;
    // columns of the rows the contingency kernel streams
    const int n_w = reduced ? c->n_r_pad : c->n_a_pad;
    const int n_box_pad = (n_box + kBoxTile - 1) / kBoxTile * kBoxTile;
    if (!paper && (!multi || screened) && !c->hat_l.p)
        CUDA_TRY(c->hat_l.alloc((size_t)c->n_line * c->n_a_pad));
    if (!paper && !multi && !c->hat_k.p)
        CUDA_TRY(c->hat_k.alloc((size_t)std::max(c->n_ctg, 1) * c->n_a_pad));
    if (reduced && (st = ensure_class_ws(c)) != IBP_OK) return st;
    CUDA_TRY(cudaMemsetAsync(c->err.p, 0, sizeof(int), s));
    if (multi) {
        CUDA_TRY(cudaMemsetAsync(c->rbus_t.p, 0, (size_t)c->n_a_pad * n_box_pad * sizeof(float), s));
        if (reduced)
            CUDA_TRY(cudaMemsetAsync(c->rcls_t.p, 0, (size_t)c->n_r_pad * n_box_pad * sizeof(float), s));
    }
    if (c->timing) CUDA_TRY(cudaEventRecord(c->ev[0], s));

    BusArgs ba{};
    ba.n_a = c->n_a; ba.n_a_pad = c->n_a_pad; ba.n_dev = c->n_dev; ba.n_gen = c->n_gen; ba.n_box = n_box;
    ba.act_ptr = c->act_ptr.p; ba.act_dev = c->act_dev.p; ba.box_lo = lo; ba.box_hi = hi;
    ba.cbus = c->cbus.p; ba.cbus2 = c->cbus2.p; ba.rbus = c->rbus.p; ba.rbus_t = multi ? c->rbus_t.p : nullptr;
    ba.rbus64 = c->rbus64.p;
    ba.n_box_pad = n_box_pad;
    ba.cabs = c->cabs.p; ba.box_consts = c->box_consts.p; ba.err = c->err.p;
    ba.bus_part = c->bus_part.p;
    CUDA_TRY(launch_bus(ba, s));
    if (reduced) {
        ClsArgs ra{};
        ra.n_box = n_box; ra.n_r = c->n_r; ra.n_r_pad = c->n_r_pad; ra.n_a_pad = c->n_a_pad;
        ra.n_box_pad = n_box_pad; ra.cls_ptr = c->cls_ptr.p; ra.cls_col = c->cls_col.p;
        ra.rbus = c->rbus.p; ra.rcls = c->rcls.p; ra.rcls_t = multi ? c->rcls_t.p : nullptr;
        CUDA_TRY(launch_class_radius(ra, s));
    }
    if (c->timing) CUDA_TRY(cudaEventRecord(c->ev[1], s));

    BaseArgs bb{};
    bb.n_l = c->n_line; bb.n_c = c->n_ctg; bb.n_a = c->n_a; bb.n_a_pad = c->n_a_pad; bb.n_box = n_box;
    bb.phi = c->phi_a.p; bb.ctg_line = c->ctg_line.p; bb.cbus = c->cbus.p; bb.cbus2 = c->cbus2.p; bb.rbus = c->rbus.p;
    bb.cabs = c->cabs.p; bb.rate_up = c->rate_up.p; bb.rate_dn = c->rate_dn.p;
    bb.box_consts = c->box_consts.p;
    bb.gamma_base = rup_gamma((c->n_a_pad / 4 + 31) / 32, 2, 5);
    bb.line_c = c->line_c.p; bb.line_e = c->line_e.p; bb.line_R = c->line_R.p;
    bb.hat_l = (multi || screened || paper) ? nullptr : c->hat_l.p;
    bb.hat_k = (multi || screened || paper) ? nullptr : c->hat_k.p;
    bb.partials = c->part_base.p;
    bb.err = c->err.p;
    if (reduced) {
        bb.is_bridge = c->is_bridge.p;
        bb.rate_c_up = c->rate_c_up.p;
        bb.rate_c_dn = c->rate_c_dn.p;
    }
    if (record) {
        bb.act_count = c->act_count.p;
        bb.act_list = c->act_list.p;
        bb.act_cap = c->act_cap;
    }
    if (record_lo) {
        bb.act_count_lo = c->act_count_lo.p;
        bb.act_list_lo = c->act_list_lo.p;
        bb.act_cap_lo = c->act_cap_lo;
    }
    bb.ref = ref_args(c);
    CUDA_TRY(launch_base(bb, c->n_part_base, s));
    if (c->timing) CUDA_TRY(cudaEventRecord(c->ev[2], s));

    if (screened) {
        ScreenArgs sa{};
        sa.n_l = c->n_line; sa.n_c = c->n_ctg; sa.n_box = n_box;
        sa.lodf = c->lodf.p; sa.ctg_line = c->ctg_line.p;
        sa.line_c = c->line_c.p; sa.line_e = c->line_e.p; sa.line_R = c->line_R.p;
        sa.box_consts = c->box_consts.p; sa.rate_dn = c->rate_c_dn.p;
        sa.live_flag = c->live_flag.p; sa.live = c->live.p; sa.n_live = c->n_live.p;
        sa.is_bridge = reduced ? c->is_bridge.p : nullptr;
        sa.paper_test = c->screen ? 1 : 0;
        sa.src = reduced ? c->phi_r.p : c->phi_a.p;
        sa.radius = multi ? nullptr : (reduced ? c->rcls.p : c->rbus.p);
        sa.rows = c->hat_l.p;
        sa.hat_k = multi ? nullptr : c->hat_k.p;
        sa.n_w = n_w;
        sa.err = c->err.p;
        CUDA_TRY(launch_screen(sa, c->num_sms, s));
    }
    if (c->timing) CUDA_TRY(cudaEventRecord(c->ev[3], s));

    const int tiles_l = (c->n_line + v->BL - 1) / v->BL;
    const int tiles_k = (c->n_ctg + v->BK - 1) / v->BK;
    const int n_chunks = (n_w + v->CH - 1) / v->CH;
    CtgArgs ca{};
    ca.n_l = c->n_line; ca.n_c = c->n_ctg; ca.n_a = c->n_a; ca.n_chunks = n_chunks; ca.n_box = n_box;
    ca.tiles_l = tiles_l;
    ca.n_tiles = tiles_l * tiles_k * (multi ? n_box_pad / kBoxTile : 1);
    ca.lodf = c->lodf.p; ca.ctg_line = c->ctg_line.p;
    ca.line_c = c->line_c.p; ca.line_e = c->line_e.p; ca.line_R = c->line_R.p;
    ca.rate_up = c->rate_c_up.p; ca.rate_dn = c->rate_c_dn.p; ca.box_consts = c->box_consts.p;
    ca.rbus_t = multi ? (reduced ? c->rcls_t.p : c->rbus_t.p) : nullptr; ca.n_box_pad = n_box_pad;
    // round-up adds per radius sum: level 1 within a chunk (one per bus, or a
    // depth-2 tree per 4 buses plus one add), level 2 over 256/CH chunks, level 3
    {
        const bool tree = !multi && v->body >= 1;
        // two level-1 sums per pair (packed body): one more add to join them
        const bool two_sums = !multi && v->body >= 2;
        const long n1 = tree ? v->CH / 4 + 2 + (two_sums ? 1 : 0) : v->CH;
        const long n2 = 256 / v->CH;
        ca.gamma = rup_gamma(n1, n2, (n_chunks + n2 - 1) / n2);
    }
    ca.flow_lo = flo; ca.flow_hi = fhi; ca.partials = c->part_ctg.p; ca.err = c->err.p;
    ca.wait_ns = 2000000000ull;
    ca.warps_per_tile = ctg_warps(*v);
    ca.ref = ref_args(c);
    const bool queue = !paper && ca.ref.phi64 && ca.n_tiles > 0;
    if (queue) {
        if ((st = ensure_ref_queue(c, c->num_sms)) != IBP_OK) return st;
        ca.refq = c->refq.p; ca.refq_cnt = c->refq_cnt.p; ca.refq_cap = kRefQCap;
        CUDA_TRY(cudaMemsetAsync(c->refq_cnt.p, 0, (size_t)ref_regions(c->num_sms) * sizeof(int), s));
    }
    ca.part_rows_cap = (int)max_part_rows(c);
    if (record) {
        ca.act_count = c->act_count.p;
        ca.act_list = c->act_list.p;
        ca.act_cap = c->act_cap;
    }
    if (record_lo) {
        ca.act_count_lo = c->act_count_lo.p;
        ca.act_list_lo = c->act_list_lo.p;
        ca.act_cap_lo = c->act_cap_lo;
    }
    if (screened) {
        ca.live = c->live.p;
        ca.n_live = c->n_live.p;
    }
    if (paper) {
        PaperArgs pa{};
        pa.n_l = c->n_line; pa.n_c = c->n_ctg; pa.n_box = n_box;
        pa.lodf = c->lodf.p; pa.ctg_line = c->ctg_line.p;
        pa.line_c = c->line_c.p; pa.line_e = c->line_e.p; pa.line_R = c->line_R.p;
        pa.box_consts = c->box_consts.p; pa.rate_up = c->rate_c_up.p; pa.rate_dn = c->rate_c_dn.p;
        pa.gamma_base = bb.gamma_base; pa.partials = c->part_ctg.p; pa.err = c->err.p;
        pa.ref = ref_args(c);
        if (pa.ref.phi64) {
            // FP64 base-flow values of every line for the refinement
            const size_t nl = (size_t)c->cap_box * c->n_line;
            if (c->lc64.n < nl || c->lR64.n < nl || c->lX.n < nl) {
                CUDA_TRY(c->lc64.alloc(nl));
                CUDA_TRY(c->lR64.alloc(nl));
                CUDA_TRY(c->lX.alloc(nl));
            }
            LineExactArgs la{};
            la.ref = pa.ref; la.n_l = c->n_line; la.n_box = n_box;
            la.c64 = c->lc64.p; la.R64 = c->lR64.p; la.X = c->lX.p;
            CUDA_TRY(launch_line_exact(la, c->num_sms, s));
            pa.lc64 = c->lc64.p; pa.lR64 = c->lR64.p; pa.lX = c->lX.p;
        }
        CUDA_TRY(launch_paper(pa, s));
    } else if (ca.n_tiles > 0) {
        CUtensorMap mL, mK, mR;
        std::string err;
        // rows of n_w columns: bus classes (reduced) or active buses
        if (multi) {
            const float *rows = screened ? c->hat_l.p : c->phi_a.p;
            const float *krows = reduced ? c->phi_kr.p : c->phi_k.p;
            const float *rt = reduced ? c->rcls_t.p : c->rbus_t.p;
            if (!encode_map_2d(&mL, rows, n_w, c->n_line, n_w, 32, v->BL, &err) ||
                !encode_map_2d(&mK, krows, n_w, c->n_ctg, n_w, 32, v->BK, &err) ||
                !encode_map_2d(&mR, rt, n_box_pad, n_w, n_box_pad, kBoxTile, 32, &err, false))
                return fail(IBP_ECUDA, "%s", err.c_str());
            CUDA_TRY(launch_ctg_multi(*v, mL, mK, mR, ca, c->num_sms, s));
        } else {
            if (!encode_map_2d(&mL, c->hat_l.p, n_w, c->n_line, n_w, 32, v->BL, &err) ||
                !encode_map_2d(&mK, c->hat_k.p, n_w, c->n_ctg, n_w, 32, v->BK, &err))
                return fail(IBP_ECUDA, "%s", err.c_str());
            CUDA_TRY(launch_ctg(*v, mL, mK, ca, c->num_sms, s));
        }
        if (c->timing) CUDA_TRY(cudaEventRecord(c->ev[4], s));
        if (queue) {
            RefQueueArgs qa{};
            qa.args = nullptr; qa.one = ca; qa.n_regions = ref_regions(c->num_sms); qa.cap = kRefQCap;
            qa.e = c->refq.p; qa.cnt = c->refq_cnt.p; qa.res = c->refq_res.p;
            CUDA_TRY(launch_refine_queue(qa, c->num_sms, s));
        }
    } else if (c->timing) {
        CUDA_TRY(cudaEventRecord(c->ev[4], s));
    }
    if (c->timing) CUDA_TRY(cudaEventRecord(c->ev[5], s));

    AsmArgs aa{};
    aa.n_box = n_box; aa.n_dev = c->n_dev; aa.n_gen = c->n_gen;
    aa.n_part_ctg = paper ? paper_partials_count(c->n_line, c->n_ctg) : tiles_l * tiles_k * ca.warps_per_tile;
    aa.n_part_base = c->n_part_base;
    aa.part_stage = c->part_stage.p; aa.n_stage = kPartStages;
    aa.part_ctg = c->part_ctg.p; aa.part_base = c->part_base.p; aa.box_lo = lo; aa.box_hi = hi;
    aa.seg_ptr = c->seg_ptr.p; aa.slope = c->slope.p; aa.bkpt = c->bkpt.p;
    aa.zeta_inj = c->zeta_inj; aa.zeta_f = c->zeta_f;
    aa.obj_lo = olo; aa.obj_hi = ohi; aa.obj_err = oerr; aa.err = c->err.p;
    if (screened) {
        aa.n_live = c->n_live.p;
        aa.live_BL = v->BL;
        aa.live_tiles_k = tiles_k;
        aa.live_rows_per_tile = ca.warps_per_tile;
    }
    CUDA_TRY(launch_assemble(aa, s));
    if (c->timing) CUDA_TRY(cudaEventRecord(c->ev[6], s));
    return mark_done(c, s);
}

// Reads the error word through the case's private stream (no wait on other
// streams); the caller has waited for the work that writes it.
ibp_status read_err_word(ibp_case *c) {
    int e = 0, rf = 0;
    CUDA_TRY(cudaMemcpyAsync(&e, c->err.p, sizeof(int), cudaMemcpyDeviceToHost, c->side));
    if (c->rating_flag.p)
        CUDA_TRY(cudaMemcpyAsync(&rf, c->rating_flag.p, sizeof(int), cudaMemcpyDeviceToHost, c->side));
    CUDA_TRY(cudaStreamSynchronize(c->side));
    if (rf) return fail(IBP_EINVAL, "ibp_case_set_ratings was given a negative or non-finite rating "
                                    "(the ratings were left unchanged)");
    if (e & kErrTimeout) return fail(IBP_ETIMEOUT, "a bounded device wait ran out");
    if (e & kErrBadBox) return fail(IBP_EINVAL, "a box has lo > hi or a non-finite entry");
    if (e & kErrOverflow)
        return fail(IBP_ENOMEM, "too many active pairs for the adjoint's list; call with fewer boxes");
    if (e & kErrBounds) return fail(IBP_EUNSOUND, "an index guard of the checked build failed");
    return IBP_OK;
}

ibp_status check_boxes_host(const ibp_case *c, int n_box, const double *lo, const double *hi) {
    const size_t n = (size_t)n_box * c->n_dev;
    for (size_t i = 0; i < n; ++i) {
        if (!is_fin(lo[i]) || !is_fin(hi[i]))
            return fail(IBP_EINVAL, "box entry %zu (box %zu, device %zu) is not finite", i, i / c->n_dev,
                        i % c->n_dev);
        if (lo[i] > hi[i])
            return fail(IBP_EINVAL, "box %zu device %zu has lo > hi", i / c->n_dev, i % c->n_dev);
    }
    return IBP_OK;
}

// boxes per call: several kernels put the box index on a grid's y dimension

static ibp_status bound_entry(ibp_case *c, int32_t n_box, const double *box_lo,
                              const double *box_hi, double *obj_lo, double *obj_hi, double *obj_err,
                              float *flow_lo, float *flow_hi, int32_t ptr_mode, void *cuda_stream,
                              bool paper) {
    if (!c) return fail(IBP_EINVAL, "case is NULL");
    if (n_box < 0) return fail(IBP_EINVAL, "n_box must be >= 0");
    if (n_box > kMaxBoxesPerCall) return fail(IBP_EINVAL, "n_box must be <= %d", kMaxBoxesPerCall);
    if (ptr_mode != 0 && ptr_mode != 1) return fail(IBP_EINVAL, "ptr_mode must be 0 or 1");
    if (n_box == 0) return ok();
    if (!box_lo || !box_hi || !obj_lo || !obj_hi || !obj_err)
        return fail(IBP_EINVAL, "box and objective pointers must not be NULL");
    if ((flow_lo == nullptr) != (flow_hi == nullptr))
        return fail(IBP_EINVAL, "flow_lo and flow_hi must both be NULL or both be set");
    if (ptr_mode == 0) {
        ibp_status st = check_boxes_host(c, n_box, box_lo, box_hi);
        if (st != IBP_OK) return st;
    }
    if (c->device < 0) return fail(IBP_ENOTSUP, "case was created without a device (dry run)");
    DeviceGuard guard(c->device);
    if (!guard.ok) return fail(IBP_ECUDA, "cannot select device %d", c->device);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (ptr_mode == 1)
        return enqueue_bound(c, n_box, box_lo, box_hi, obj_lo, obj_hi, obj_err, flow_lo, flow_hi, s,
                             false, paper);

    ibp_status st = ensure_workspace(c, n_box);
    if (st != IBP_OK) return st;
    const size_t nd = (size_t)n_box * c->n_dev;
    CUDA_TRY(cudaMemcpyAsync(c->box_lo.p, box_lo, nd * sizeof(double), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->box_hi.p, box_hi, nd * sizeof(double), cudaMemcpyHostToDevice, s));
    float *dflo = nullptr, *dfhi = nullptr;
    const size_t nf = (size_t)n_box * c->n_ctg * c->n_line;
    if (flow_lo && nf > 0) {
        if (c->flows.n < 2 * nf) CUDA_TRY(c->flows.alloc(2 * nf));
        dflo = c->flows.p;
        dfhi = c->flows.p + nf;
    }
    double *dobj = c->obj.p;
    st = enqueue_bound(c, n_box, c->box_lo.p, c->box_hi.p, dobj, dobj + n_box, dobj + 2 * n_box,
                       dflo, dfhi, s, false, paper);
    if (st != IBP_OK) return st;
    CUDA_TRY(cudaMemcpyAsync(obj_lo, dobj, n_box * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(obj_hi, dobj + n_box, n_box * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(obj_err, dobj + 2 * n_box, 2 * n_box * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (dflo) {
        CUDA_TRY(cudaMemcpyAsync(flow_lo, dflo, nf * sizeof(float), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaMemcpyAsync(flow_hi, dfhi, nf * sizeof(float), cudaMemcpyDeviceToHost, s));
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    st = read_err_word(c);
    if (st != IBP_OK) return st;
    return ok();
}

extern "C" ibp_status ibp_bound(ibp_case *c, int32_t n_box, const double *box_lo,
                                const double *box_hi, double *obj_lo, double *obj_hi,
                                double *obj_err, float *flow_lo, float *flow_hi, int32_t ptr_mode,
                                void *cuda_stream) {
    return bound_entry(c, n_box, box_lo, box_hi, obj_lo, obj_hi, obj_err, flow_lo, flow_hi, ptr_mode,
                       cuda_stream, false);
}

extern "C" ibp_status ibp_bound_paper(ibp_case *c, int32_t n_box, const double *box_lo,
                                      const double *box_hi, double *obj_lo, double *obj_hi,
                                      double *obj_err, int32_t ptr_mode, void *cuda_stream) {
    return bound_entry(c, n_box, box_lo, box_hi, obj_lo, obj_hi, obj_err, nullptr, nullptr, ptr_mode,
                       cuda_stream, true);
}

ibp_status ensure_bwd_workspace(ibp_case *c, int n_box) {
    if (n_box <= c->bwd_cap_box) return IBP_OK;
    const int cap = std::max(n_box, 1);
    c->bwd_cap_box = 0;  // a failure part-way makes the next call start over
    // active-pair list: about 16M entries (256 MB) shared by the boxes
    const long long pairs = (long long)c->n_ctg * c->n_line + c->n_line;
    c->act_cap = (int)std::max<long long>(4096, std::min<long long>(pairs, (16ll << 20) / cap));
    CUDA_TRY(c->act_count.alloc(cap));
    CUDA_TRY(c->act_list.alloc((size_t)cap * c->act_cap));
    CUDA_TRY(c->W.alloc((size_t)cap * c->n_line));
    CUDA_TRY(c->cnt.alloc((size_t)cap * c->n_line));
    CUDA_TRY(c->dc.alloc((size_t)cap * c->n_a_pad));
    CUDA_TRY(c->dr.alloc((size_t)cap * c->n_a_pad));
    CUDA_TRY(c->grads.alloc((size_t)cap * (2 * c->n_dev + c->n_line + 1)));
    c->bwd_cap_box = cap;
    ++c->ws_gen;  // cached many-case plans hold these pointers
    return IBP_OK;
}

// obj_lo's active set holds most pairs of a wide box: its list takes up to
// 64M entries (1 GiB) shared by the boxes of a call
ibp_status ensure_bwd_lo_workspace(ibp_case *c, int n_box) {
    if (n_box <= c->bwd_lo_cap_box) return IBP_OK;
    const int cap = std::max(n_box, 1);
    c->bwd_lo_cap_box = 0;
    const long long pairs = (long long)c->n_ctg * c->n_line + c->n_line;
    c->act_cap_lo = (int)std::max<long long>(4096, std::min<long long>(pairs, (64ll << 20) / cap));
    CUDA_TRY(c->act_count_lo.alloc(cap));
    CUDA_TRY(c->act_list_lo.alloc((size_t)cap * c->act_cap_lo));
    c->bwd_lo_cap_box = cap;
    ++c->ws_gen;
    return IBP_OK;
}

// side 0: adjoint of obj_hi; side 1: of obj_lo.  gobj = d loss / d obj.
static ibp_status enqueue_backward(ibp_case *c, int n_box, const double *lo, const double *hi,
                                   const double *gobj, double *glo, double *ghi, double *grat,
                                   cudaStream_t s, int side = 0) {
    ibp_status st = ensure_bwd_workspace(c, n_box);
    if (st != IBP_OK) return st;
    if (side && (st = ensure_bwd_lo_workspace(c, n_box)) != IBP_OK) return st;
    int *count = side ? c->act_count_lo.p : c->act_count.p;
    CUDA_TRY(cudaMemsetAsync(count, 0, n_box * sizeof(int), s));
    // forward pass with recording of the active pairs of the side
    double *dobj = c->obj.p;
    if ((st = enqueue_bound(c, n_box, lo, hi, dobj, dobj + n_box, dobj + 2 * n_box, nullptr,
                            nullptr, s, side == 0, false, side == 1)) != IBP_OK)
        return st;
    CUDA_TRY(cudaMemsetAsync(c->W.p, 0, (size_t)n_box * c->n_line * sizeof(double), s));
    CUDA_TRY(cudaMemsetAsync(c->cnt.p, 0, (size_t)n_box * c->n_line * sizeof(int), s));
    CUDA_TRY(cudaMemsetAsync(c->dr.p, 0, (size_t)n_box * c->n_a_pad * sizeof(double), s));
    CUDA_TRY(cudaMemsetAsync(c->dc.p, 0, (size_t)n_box * c->n_a_pad * sizeof(double), s));
    BwdArgs b{};
    b.n_l = c->n_line; b.n_a = c->n_a; b.n_a_pad = c->n_a_pad; b.n_dev = c->n_dev; b.n_gen = c->n_gen;
    b.n_box = n_box; b.side = side;
    b.act_cap = side ? c->act_cap_lo : c->act_cap; b.phi = c->phi_a.p; b.act_count = count;
    b.act_list = side ? c->act_list_lo.p : c->act_list.p;
    b.W = c->W.p; b.cnt = c->cnt.p; b.dc = c->dc.p; b.dr = c->dr.p;
    b.dev_col = c->dev_col.p; b.box_lo = lo; b.box_hi = hi; b.seg_ptr = c->seg_ptr.p;
    b.slope = c->slope.p; b.bkpt = c->bkpt.p; b.zeta_inj = c->zeta_inj; b.zeta_f = c->zeta_f;
    b.grad_obj_hi = gobj; b.grad_lo = glo; b.grad_hi = ghi; b.grad_rating = grat;
    CUDA_TRY(launch_backward(b, s));
    return mark_done(c, s);
}

static ibp_status backward_entry(ibp_case *c, int32_t n_box, const double *box_lo,
                                 const double *box_hi, const double *grad_obj_hi, double *grad_lo,
                                 double *grad_hi, double *grad_rating, int32_t ptr_mode,
                                 void *cuda_stream, int side) {
    if (!c) return fail(IBP_EINVAL, "case is NULL");
    if (n_box < 0) return fail(IBP_EINVAL, "n_box must be >= 0");
    if (n_box > kMaxBoxesPerCall) return fail(IBP_EINVAL, "n_box must be <= %d", kMaxBoxesPerCall);
    if (ptr_mode != 0 && ptr_mode != 1) return fail(IBP_EINVAL, "ptr_mode must be 0 or 1");
    if (n_box == 0) return ok();
    if (!box_lo || !box_hi || !grad_obj_hi || !grad_lo || !grad_hi)
        return fail(IBP_EINVAL, "box and gradient pointers must not be NULL");
    if (ptr_mode == 0) {
        ibp_status st = check_boxes_host(c, n_box, box_lo, box_hi);
        if (st != IBP_OK) return st;
        for (int j = 0; j < n_box; ++j)
            if (!is_fin(grad_obj_hi[j])) return fail(IBP_EINVAL, "grad_obj[%d] is not finite", j);
    }
    if (c->device < 0) return fail(IBP_ENOTSUP, "case was created without a device (dry run)");
    DeviceGuard guard(c->device);
    if (!guard.ok) return fail(IBP_ECUDA, "cannot select device %d", c->device);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    ibp_status st = ensure_workspace(c, n_box);
    if (st != IBP_OK) return st;
    if (ptr_mode == 1)
        return enqueue_backward(c, n_box, box_lo, box_hi, grad_obj_hi, grad_lo, grad_hi, grad_rating, s,
                                side);
    if ((st = ensure_bwd_workspace(c, n_box)) != IBP_OK) return st;
    const size_t nd = (size_t)n_box * c->n_dev;
    CUDA_TRY(cudaMemcpyAsync(c->box_lo.p, box_lo, nd * sizeof(double), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->box_hi.p, box_hi, nd * sizeof(double), cudaMemcpyHostToDevice, s));
    double *dg = c->grads.p;                 // [n_box] grad_obj_hi
    double *dglo = dg + n_box;               // [n_box][n_dev]
    double *dghi = dglo + nd;                // [n_box][n_dev]
    double *dgr = dghi + nd;                 // [n_box][n_line]
    CUDA_TRY(cudaMemcpyAsync(dg, grad_obj_hi, n_box * sizeof(double), cudaMemcpyHostToDevice, s));
    st = enqueue_backward(c, n_box, c->box_lo.p, c->box_hi.p, dg, dglo, dghi,
                          grad_rating ? dgr : nullptr, s, side);
    if (st != IBP_OK) return st;
    CUDA_TRY(cudaMemcpyAsync(grad_lo, dglo, nd * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(grad_hi, dghi, nd * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (grad_rating)
        CUDA_TRY(cudaMemcpyAsync(grad_rating, dgr, (size_t)n_box * c->n_line * sizeof(double),
                                 cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return read_err_word(c);
}

extern "C" ibp_status ibp_bound_backward(ibp_case *c, int32_t n_box, const double *box_lo,
                                         const double *box_hi, const double *grad_obj_hi,
                                         double *grad_lo, double *grad_hi, double *grad_rating,
                                         int32_t ptr_mode, void *cuda_stream) {
    return backward_entry(c, n_box, box_lo, box_hi, grad_obj_hi, grad_lo, grad_hi, grad_rating,
                          ptr_mode, cuda_stream, 0);
}

extern "C" ibp_status ibp_bound_backward_lo(ibp_case *c, int32_t n_box, const double *box_lo,
                                            const double *box_hi, const double *grad_obj_lo,
                                            double *grad_lo, double *grad_hi, double *grad_rating,
                                            int32_t ptr_mode, void *cuda_stream) {
    return backward_entry(c, n_box, box_lo, box_hi, grad_obj_lo, grad_lo, grad_hi, grad_rating,
                          ptr_mode, cuda_stream, 1);
}

// ---------------------------------------------------------------- ratings
// New ratings: a check of every entry into a sticky flag, then (only when no
// entry failed) their directed FP32 copies and FP64 values.
__global__ void k_check_ratings(int n_l, const double *rating, const double *rating_ctg, int *flag) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_l) return;
    const double r = rating[l], rc = rating_ctg ? rating_ctg[l] : r;
    if (!(r >= 0.0) || !(rc >= 0.0) || !isfinite(r) || !isfinite(rc)) atomicOr(flag, kErrBadRating);
}

__global__ void k_apply_ratings(int n_l, const double *rating, const double *rating_ctg, float *ru,
                                float *rd, float *rcu, float *rcd, double *r64, double *rc64,
                                const int *flag) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_l || *flag) return;
    const double r = rating[l], rc = rating_ctg ? rating_ctg[l] : r;
    ru[l] = __double2float_ru(r);
    rd[l] = __double2float_rd(r);
    rcu[l] = __double2float_ru(rc);
    rcd[l] = __double2float_rd(rc);
    r64[l] = r;
    rc64[l] = rc;
}

extern "C" ibp_status ibp_case_set_ratings(ibp_case *c, const double *rating,
                                           const double *rating_ctg, int32_t ptr_mode,
                                           void *cuda_stream) {
    if (!c) return fail(IBP_EINVAL, "case is NULL");
    if (!rating) return fail(IBP_EINVAL, "rating must not be NULL");
    if (ptr_mode != 0 && ptr_mode != 1) return fail(IBP_EINVAL, "ptr_mode must be 0 or 1");
    if (ptr_mode == 0)
        for (int l = 0; l < c->n_line; ++l) {
            if (!is_fin(rating[l]) || rating[l] < 0)
                return fail(IBP_EINVAL, "rating[%d] must be finite and >= 0", l);
            if (rating_ctg && (!is_fin(rating_ctg[l]) || rating_ctg[l] < 0))
                return fail(IBP_EINVAL, "rating_ctg[%d] must be finite and >= 0", l);
        }
    if (c->device < 0) return fail(IBP_ENOTSUP, "case was created without a device (dry run)");
    DeviceGuard guard(c->device);
    if (!guard.ok) return fail(IBP_ECUDA, "cannot select device %d", c->device);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const double *r = rating, *rc = rating_ctg;
    DevBuf<double> tmp;
    if (ptr_mode == 0) {
        CUDA_TRY(tmp.alloc((size_t)2 * c->n_line));
        CUDA_TRY(cudaMemcpyAsync(tmp.p, rating, c->n_line * sizeof(double), cudaMemcpyHostToDevice, s));
        if (rating_ctg)
            CUDA_TRY(cudaMemcpyAsync(tmp.p + c->n_line, rating_ctg, c->n_line * sizeof(double),
                                     cudaMemcpyHostToDevice, s));
        r = tmp.p;
        rc = rating_ctg ? tmp.p + c->n_line : nullptr;
    }
    if (!c->rating_flag.p) CUDA_TRY(c->rating_flag.alloc(1));
    CUDA_TRY(cudaMemsetAsync(c->rating_flag.p, 0, sizeof(int), s));
    const int blocks = (c->n_line + 255) / 256;
    k_check_ratings<<<blocks, 256, 0, s>>>(c->n_line, r, rc, c->rating_flag.p);
    CUDA_TRY(cudaGetLastError());
    k_apply_ratings<<<blocks, 256, 0, s>>>(c->n_line, r, rc, c->rate_up.p, c->rate_dn.p, c->rate_c_up.p,
                                           c->rate_c_dn.p, c->rate64.p, c->rate_c64.p, c->rating_flag.p);
    CUDA_TRY(cudaGetLastError());
    if (ptr_mode == 0) {
        CUDA_TRY(cudaStreamSynchronize(s));
        return ok();
    }
    return mark_done(c, s);
}

extern "C" ibp_status ibp_case_sync(ibp_case *c) {
    if (!c) return fail(IBP_EINVAL, "case is NULL");
    if (c->device < 0) return fail(IBP_ENOTSUP, "case was created without a device (dry run)");
    DeviceGuard guard(c->device);
    ibp_status st = wait_case(c);
    if (st != IBP_OK) return st;
    st = read_err_word(c);
    if (st != IBP_OK) return st;
    return ok();
}

extern "C" ibp_status ibp_case_info(const ibp_case *c, ibp_case_info_t *o) {
    if (!c || !o) return fail(IBP_EINVAL, "NULL argument");
    o->n_bus = c->n_bus; o->n_line = c->n_line; o->n_ctg = c->n_ctg; o->n_gen = c->n_gen;
    o->n_load = c->n_load; o->n_active = c->n_a; o->n_active_pad = c->n_a_pad; o->device = c->device;
    int64_t bytes = 0;
    bytes += (int64_t)c->phi_a.n * 4 + (int64_t)c->lodf.n * 4 + (int64_t)c->hat_l.n * 4 + (int64_t)c->hat_k.n * 4;
    bytes += (int64_t)c->phi64.n * 8 + (int64_t)c->lodf_lo.n * 4;
    bytes += (int64_t)(c->cbus.n + c->part_base.n + c->part_ctg.n + c->box_lo.n + c->box_hi.n) * 8;
    bytes += (int64_t)(c->rbus.n + c->cabs.n + c->line_c.n + c->line_e.n + c->line_R.n + c->flows.n) * 4;
    o->device_bytes = bytes;
    o->build_seconds = c->build_seconds;
    o->max_abs_lodf = c->max_abs_lodf;
    o->n_bus_classes = c->n_r;
    o->n_bridges = c->n_bridges;
    return ok();
}

extern "C" ibp_status ibp_case_reduction(const ibp_case *c, int32_t *class_of_active, int32_t *is_bridge) {
    if (!c) return fail(IBP_EINVAL, "case is NULL");
    if (class_of_active) {
        for (int i = 0; i < c->n_a; ++i) class_of_active[i] = -1;
        for (int j = 0; j < c->n_r; ++j)
            for (int m = c->cls_ptr_h[j]; m < c->cls_ptr_h[j + 1]; ++m) class_of_active[c->cls_col_h[m]] = j;
    }
    if (is_bridge)
        for (int l = 0; l < c->n_line; ++l) is_bridge[l] = c->is_bridge_h[l];
    return ok();
}

extern "C" ibp_status ibp_case_set_variant(ibp_case *c, int32_t variant) {
    if (!c) return fail(IBP_EINVAL, "case is NULL");
    if (variant != 0 && !ctg_variant_by_id(variant)) return fail(IBP_EINVAL, "unknown variant %d", variant);
    c->variant = variant;
    return ok();
}

extern "C" ibp_status ibp_set_alloc_limit(int64_t bytes) {
    if (bytes < 0) return fail(IBP_EINVAL, "bytes must be >= 0");
    g_alloc_limit.store(bytes);
    return ok();
}

extern "C" ibp_status ibp_case_set_screen(ibp_case *c, int32_t enable) {
    if (!c) return fail(IBP_EINVAL, "case is NULL");
    c->screen = enable != 0;
    return ok();
}

extern "C" ibp_status ibp_case_set_refine(ibp_case *c, int32_t enable) {
    if (!c) return fail(IBP_EINVAL, "case is NULL");
    c->refine = enable != 0;
    ++c->ws_gen;  // cached many-case plans carry the refinement arguments
    return ok();
}

extern "C" ibp_status ibp_case_set_reduction(ibp_case *c, int32_t enable) {
    if (!c) return fail(IBP_EINVAL, "case is NULL");
    c->reduce = enable != 0;
    return ok();
}

extern "C" ibp_status ibp_case_last_live(ibp_case *c, int32_t *n_live, int32_t *lines) {
    if (!c || !n_live) return fail(IBP_EINVAL, "NULL argument");
    if (c->device < 0) return fail(IBP_ENOTSUP, "dry-run case");
    if (!c->last_screened || !c->n_live.p) {
        *n_live = -1;
        return ok();
    }
    DeviceGuard guard(c->device);
    ibp_status st = wait_case(c);
    if (st != IBP_OK) return st;
    CUDA_TRY(cudaMemcpyAsync(n_live, c->n_live.p, sizeof(int32_t), cudaMemcpyDeviceToHost, c->side));
    CUDA_TRY(cudaStreamSynchronize(c->side));
    if (*n_live < 0 || *n_live > c->n_line) return fail(IBP_ECUDA, "corrupt live-line count");
    if (lines && *n_live > 0) {
        CUDA_TRY(cudaMemcpyAsync(lines, c->live.p, (size_t)*n_live * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                 c->side));
        CUDA_TRY(cudaStreamSynchronize(c->side));
    }
    return ok();
}

extern "C" int32_t ibp_kernel_variants(int32_t *ids, int32_t cap, int32_t batched) {
    int n;
    const CtgVariant *v = ctg_variants(&n);
    int32_t k = 0;
    for (int i = 0; i < n; ++i) {
        if ((v[i].batched != 0) != (batched != 0)) continue;
        if (ids && k < cap) ids[k] = v[i].id;
        ++k;
    }
    return k;
}

extern "C" ibp_status ibp_case_set_timing(ibp_case *c, int32_t enable) {
    if (!c) return fail(IBP_EINVAL, "case is NULL");
    if (c->device < 0) return fail(IBP_ENOTSUP, "dry-run case");
    c->timing = enable != 0;
    return ok();
}

extern "C" ibp_status ibp_case_last_timing(ibp_case *c, float *ms, int32_t n) {
    if (!c || !ms) return fail(IBP_EINVAL, "NULL argument");
    if (!c->timing) return fail(IBP_EINVAL, "timing is not enabled");
    DeviceGuard guard(c->device);
    CUDA_TRY(cudaEventSynchronize(c->ev[ibp_case::kEvents - 1]));
    for (int i = 0; i < std::min<int>(n, ibp_case::kEvents - 1); ++i)
        CUDA_TRY(cudaEventElapsedTime(&ms[i], c->ev[i], c->ev[i + 1]));
    return ok();
}

extern "C" ibp_status ibp_selftest_wait_timeout(int32_t device, int32_t limit_us) {
    if (limit_us <= 0 || limit_us > 2000000) return fail(IBP_EINVAL, "limit_us out of (0, 2e6]");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(IBP_ECUDA, "no such CUDA device");
    DeviceGuard guard(device);
    DevBuf<int> flag;
    CUDA_TRY(flag.alloc(1));
    CUDA_TRY(cudaMemset(flag.p, 0xff, sizeof(int)));
    CUDA_TRY(launch_wait_selftest(flag.p, (unsigned long long)limit_us * 1000ull, nullptr));
    CUDA_TRY(cudaDeviceSynchronize());
    int f = 0;
    CUDA_TRY(cudaMemcpy(&f, flag.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (f == kErrTimeout) return fail(IBP_ETIMEOUT, "wait ran out after %d us (expected)", limit_us);
    if (f == 0) return ok();
    return fail(IBP_ECUDA, "self-test kernel did not report");
}

extern "C" const char *ibp_last_error(void) { return g_last_error.c_str(); }

extern "C" const char *ibp_status_string(ibp_status s) {
    switch (s) {
    case IBP_OK: return "IBP_OK";
    case IBP_EINVAL: return "IBP_EINVAL";
    case IBP_EISLAND: return "IBP_EISLAND";
    case IBP_ESINGULAR: return "IBP_ESINGULAR";
    case IBP_ENOMEM: return "IBP_ENOMEM";
    case IBP_ECUDA: return "IBP_ECUDA";
    case IBP_ETIMEOUT: return "IBP_ETIMEOUT";
    case IBP_EUNSOUND: return "IBP_EUNSOUND";
    case IBP_ENOTSUP: return "IBP_ENOTSUP";
    }
    return "unknown";
}
