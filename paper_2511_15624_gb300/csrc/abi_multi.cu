// C ABI of many cases of uneven size in one persistent launch: the cached
// work plan (items, per-case arguments, TMA descriptors), the forward pass
// and the batched adjoint.
#include "abi_case.h"

// ---------------------------------------------------------------- many cases
// Work plan of one ibp_bound_multi configuration (cases, box counts and their
// workspace generations), built and uploaded once, then reused.
struct MultiPlan {
    std::vector<const ibp_case *> cases;
    std::vector<int> n_box, gens, reduced;
    int device = -1, grid = 0;
    int variant = 0, rows_per_item = 0;  // kernel body (the first case's variant) and its partial rows
    DevBuf<MultiItem> items;
    DevBuf<int> cta_start, err;
    DevBuf<uint32_t> prefix;
    DevBuf<CtgArgs> args;
    DevBuf<CUtensorMap> maps;
    // refinement queues of the launch (shared by the cases), when a case refines
    bool refine = false;
    DevBuf<int4> refq;
    DevBuf<int> refq_cnt;
    DevBuf<double2> refq_res;
    // 0: plain bound; 1 + side: the forward pass of a backward, recording the
    // side's active pairs, with the backward's (case, box) items and arguments
    int record = 0;
    int n_items = 0, max_n_a_pad = 0;
    DevBuf<BwdArgs> bargs;
    DevBuf<int2> bitems;
    ~MultiPlan() {
        if (device >= 0) {
            DeviceGuard g(device);
            items.free(); cta_start.free(); err.free(); prefix.free(); args.free(); maps.free();
            refq.free(); refq_cnt.free(); refq_res.free(); bargs.free(); bitems.free();
        }
    }
};
static std::mutex g_plan_mu;
static std::vector<std::unique_ptr<MultiPlan>> g_plans;

void drop_plans_of(const ibp_case *c) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_plans.erase(std::remove_if(g_plans.begin(), g_plans.end(),
                                 [c](const std::unique_ptr<MultiPlan> &p) {
                                     return std::find(p->cases.begin(), p->cases.end(), c) !=
                                            p->cases.end();
                                 }),
                  g_plans.end());
}

static CtgArgs multi_args(const ibp_case *c, int n_box, int BL, int BK, int CH, bool reduced,
                          int rows_per_item, int record) {
    const int n_box_pad = (n_box + kBoxTile - 1) / kBoxTile * kBoxTile;
    const int n_rows = reduced ? c->n_nb : c->n_line;
    const int tiles_l = (n_rows + BL - 1) / BL, tiles_k = (c->n_ctg + BK - 1) / BK;
    const int n_chunks = ((reduced ? c->n_r_pad : c->n_a_pad) + CH - 1) / CH;
    CtgArgs ca{};
    ca.n_l = c->n_line; ca.n_c = c->n_ctg; ca.n_a = c->n_a; ca.n_chunks = n_chunks; ca.n_box = n_box;
    ca.tiles_l = tiles_l; ca.n_tiles = tiles_l * tiles_k * (n_box_pad / kBoxTile);
    ca.lodf = c->lodf.p; ca.ctg_line = c->ctg_line.p;
    ca.line_c = c->line_c.p; ca.line_e = c->line_e.p; ca.line_R = c->line_R.p;
    ca.rate_up = c->rate_c_up.p; ca.rate_dn = c->rate_c_dn.p; ca.box_consts = c->box_consts.p;
    ca.rbus_t = reduced ? c->rcls_t.p : c->rbus_t.p; ca.n_box_pad = n_box_pad;
    ca.gamma = rup_gamma(CH, 256 / CH, (n_chunks + 256 / CH - 1) / (256 / CH));
    ca.flow_lo = nullptr; ca.flow_hi = nullptr; ca.partials = c->part_ctg.p; ca.err = c->err.p;
    ca.wait_ns = 2000000000ull;
    ca.warps_per_tile = rows_per_item;
    ca.part_rows_cap = (int)max_part_rows(c);
    ca.ref = ref_args(c);
    if (reduced) {
        ca.live = c->nb_list.p;
        ca.n_live = c->nb_count.p;
    }
    if (record == 1) {
        ca.act_count = c->act_count.p;
        ca.act_list = c->act_list.p;
        ca.act_cap = c->act_cap;
    } else if (record == 2) {
        ca.act_count_lo = c->act_count_lo.p;
        ca.act_list_lo = c->act_list_lo.p;
        ca.act_cap_lo = c->act_cap_lo;
    }
    return ca;
}

// the backward's arguments of one case without the per-call pointers
static BwdArgs bwd_args(const ibp_case *c, int n_box, int side) {
    BwdArgs b{};
    b.n_l = c->n_line; b.n_a = c->n_a; b.n_a_pad = c->n_a_pad; b.n_dev = c->n_dev; b.n_gen = c->n_gen;
    b.n_box = n_box; b.side = side;
    b.act_cap = side ? c->act_cap_lo : c->act_cap; b.phi = c->phi_a.p;
    b.act_count = side ? c->act_count_lo.p : c->act_count.p;
    b.act_list = side ? c->act_list_lo.p : c->act_list.p;
    b.W = c->W.p; b.cnt = c->cnt.p; b.dc = c->dc.p; b.dr = c->dr.p;
    b.dev_col = c->dev_col.p; b.seg_ptr = c->seg_ptr.p;
    b.slope = c->slope.p; b.bkpt = c->bkpt.p; b.zeta_inj = c->zeta_inj; b.zeta_f = c->zeta_f;
    return b;
}

// the many-case launch uses the static part of the network reduction: every
// non-bridge line, with its reduced row
static bool multi_reduced(const ibp_case *c) { return c->reduce && c->has_reduction && c->n_ctg > 0; }

static ibp_status ensure_nonbridge_rows(ibp_case *c) {
    if (c->n_nb >= 0) return IBP_OK;
    std::vector<int> nb;
    for (int l = 0; l < c->n_line; ++l)
        if (!c->is_bridge_h[l]) nb.push_back(l);
    const int n = (int)nb.size();
    CUDA_TRY(c->nb_list.alloc(std::max(n, 1)));
    CUDA_TRY(c->nb_count.alloc(1));
    CUDA_TRY(c->phi_nb.alloc((size_t)std::max(n, 1) * c->n_r_pad));
    if (n > 0) {
        CUDA_TRY(cudaMemcpy(c->nb_list.p, nb.data(), n * sizeof(int), cudaMemcpyHostToDevice));
        CUDA_TRY(launch_gather_rows(c->phi_r.p, c->n_r_pad, c->nb_list.p, n, c->phi_nb.p, nullptr));
    }
    CUDA_TRY(cudaMemcpy(c->nb_count.p, &n, sizeof(int), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaDeviceSynchronize());
    c->n_nb = n;
    return IBP_OK;
}

static ibp_status build_plan(ibp_case *const *cases, const int32_t *n_box, int n_case, int num_sms,
                             int record, MultiPlan **out) {
    int BL, BK, CH;
    multi_tile_shape(&BL, &BK, &CH);
    std::unique_ptr<MultiPlan> P(new MultiPlan());
    P->device = cases[0]->device;
    P->variant = cases[0]->variant;
    P->rows_per_item = cases_rows_per_item(P->variant);
    std::vector<CtgArgs> args(n_case);
    std::vector<CUtensorMap> maps(3 * (size_t)n_case);
    struct Item { MultiItem m; long long cost; int order; };
    std::vector<Item> all;
    for (int i = 0; i < n_case; ++i) {
        const ibp_case *c = cases[i];
        P->cases.push_back(c);
        P->n_box.push_back(n_box[i]);
        P->gens.push_back(c->ws_gen);
        const bool red = multi_reduced(c);
        P->reduced.push_back(red ? 1 : 0);
        args[i] = multi_args(c, n_box[i], BL, BK, CH, red, P->rows_per_item, record);
        const int n_box_pad = args[i].n_box_pad;
        const int w = red ? c->n_r_pad : c->n_a_pad;
        const float *rows = red ? c->phi_nb.p : c->phi_a.p;
        const int n_rows = std::max(red ? c->n_nb : c->n_line, 1);
        std::string err;
        if (!encode_map_2d(&maps[3 * i], rows, w, n_rows, w, 32, BL, &err) ||
            !encode_map_2d(&maps[3 * i + 1], red ? c->phi_kr.p : c->phi_k.p, w, std::max(c->n_ctg, 1), w,
                           32, BK, &err) ||
            !encode_map_2d(&maps[3 * i + 2], red ? c->rcls_t.p : c->rbus_t.p, n_box_pad, w, n_box_pad,
                           kBoxTile, 32, &err, false))
            return fail(IBP_ECUDA, "%s", err.c_str());
        if (c->n_ctg == 0) continue;
        const int tiles_l = args[i].tiles_l, tiles_k = (c->n_ctg + BK - 1) / BK;
        const long long cost = (long long)args[i].n_chunks * BL * BK * kBoxTile;
        for (int tl = 0; tl < tiles_l; ++tl)
            for (int tk = 0; tk < tiles_k; ++tk)
                for (int bt = 0; bt < n_box_pad / kBoxTile; ++bt) {
                    Item it;
                    it.m = MultiItem{i, tl * BL, tk * BK, bt * kBoxTile, tl * tiles_k + tk, args[i].n_chunks};
                    it.cost = cost;
                    it.order = (int)all.size();
                    all.push_back(it);
                }
    }
    // longest items first, dealt round-robin to the persistent CTAs
    std::stable_sort(all.begin(), all.end(), [](const Item &a, const Item &b) { return a.cost > b.cost; });
    const int G = std::max(1, std::min<int>(num_sms, (int)all.size()));
    std::vector<std::vector<MultiItem>> per(G);
    for (size_t k = 0; k < all.size(); ++k) per[k % G].push_back(all[k].m);
    std::vector<MultiItem> items;
    std::vector<int> start(G + 1, 0);
    std::vector<uint32_t> prefix;
    for (int b = 0; b < G; ++b) {
        start[b] = (int)items.size();
        uint32_t acc = 0;
        for (const MultiItem &m : per[b]) {
            items.push_back(m);
            prefix.push_back(acc);
            acc += (uint32_t)m.n_chunks;
        }
        prefix.push_back(acc);
    }
    start[G] = (int)items.size();
    P->grid = all.empty() ? 0 : G;
    // one set of refinement queues for the launch, when any case refines
    for (int i = 0; i < n_case; ++i) P->refine = P->refine || args[i].ref.phi64 != nullptr;
    if (P->refine) {
        ibp_status st = ensure_ref_queue(P.get(), num_sms);
        if (st != IBP_OK) return st;
        for (int i = 0; i < n_case; ++i) {
            args[i].refq = P->refq.p; args[i].refq_cnt = P->refq_cnt.p; args[i].refq_cap = kRefQCap;
        }
    }
    CUDA_TRY(P->items.alloc(std::max<size_t>(items.size(), 1)));
    CUDA_TRY(P->cta_start.alloc(start.size()));
    CUDA_TRY(P->prefix.alloc(prefix.size() + 1));
    CUDA_TRY(P->args.alloc(args.size()));
    CUDA_TRY(P->maps.alloc(maps.size()));
    CUDA_TRY(P->err.alloc(1));
    if (!items.empty())
        CUDA_TRY(cudaMemcpy(P->items.p, items.data(), items.size() * sizeof(MultiItem), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(P->cta_start.p, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(P->prefix.p, prefix.data(), prefix.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(P->args.p, args.data(), args.size() * sizeof(CtgArgs), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(P->maps.p, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    P->record = record;
    if (record) {
        std::vector<BwdArgs> bargs(n_case);
        std::vector<int2> bitems;
        for (int i = 0; i < n_case; ++i) {
            bargs[i] = bwd_args(cases[i], n_box[i], record - 1);
            P->max_n_a_pad = std::max(P->max_n_a_pad, cases[i]->n_a_pad);
            for (int j = 0; j < n_box[i]; ++j) bitems.push_back(make_int2(i, j));
        }
        P->n_items = (int)bitems.size();
        CUDA_TRY(P->bargs.alloc(bargs.size()));
        CUDA_TRY(P->bitems.alloc(bitems.size()));
        CUDA_TRY(cudaMemcpy(P->bargs.p, bargs.data(), bargs.size() * sizeof(BwdArgs), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(P->bitems.p, bitems.data(), bitems.size() * sizeof(int2), cudaMemcpyHostToDevice));
    }
    *out = P.release();
    return IBP_OK;
}

static MultiPlan *find_plan(ibp_case *const *cases, const int32_t *n_box, int n_case, int record) {
    for (auto &p : g_plans) {
        if ((int)p->cases.size() != n_case || p->variant != cases[0]->variant || p->record != record) continue;
        bool same = true;
        for (int i = 0; i < n_case && same; ++i)
            same = p->cases[i] == cases[i] && p->n_box[i] == n_box[i] && p->gens[i] == cases[i]->ws_gen &&
                   p->reduced[i] == (int)multi_reduced(cases[i]);
        if (same) return p.get();
    }
    return nullptr;
}

static ibp_status check_multi_args(int32_t n_case, ibp_case *const *cases, const int32_t *n_box,
                                   const double *const *box_lo, const double *const *box_hi) {
    if (n_case < 0) return fail(IBP_EINVAL, "n_case must be >= 0");
    if (n_case == 0) return IBP_OK;
    if (!cases || !n_box || !box_lo || !box_hi) return fail(IBP_EINVAL, "array arguments must not be NULL");
    for (int i = 0; i < n_case; ++i) {
        if (!cases[i]) return fail(IBP_EINVAL, "case %d is NULL", i);
        if (cases[i]->device < 0) return fail(IBP_ENOTSUP, "case %d was created without a device", i);
        if (cases[i]->device != cases[0]->device) return fail(IBP_EINVAL, "cases live on different devices");
        if (n_box[i] < 1 || n_box[i] > kMaxBoxesPerCall)
            return fail(IBP_EINVAL, "n_box[%d] must be in [1, %d]", i, kMaxBoxesPerCall);
        if (!box_lo[i] || !box_hi[i]) return fail(IBP_EINVAL, "box pointers of case %d must not be NULL", i);
        for (int j = 0; j < i; ++j)
            if (cases[j] == cases[i]) return fail(IBP_EINVAL, "case %d appears twice", i);
    }
    return IBP_OK;
}

// the many-case forward pass (record: 0 plain, 1 + side: record the side's
// active pairs for a backward); returns the plan it ran
static ibp_status enqueue_multi(int32_t n_case, ibp_case *const *cases, const int32_t *n_box,
                                const double *const *box_lo, const double *const *box_hi,
                                double *const *obj_lo, double *const *obj_hi, double *const *obj_err,
                                cudaStream_t s, int record, MultiPlan **plan_out) {
    ibp_status st;
    for (int i = 0; i < n_case; ++i) {
        if ((st = ensure_workspace(cases[i], n_box[i])) != IBP_OK) return st;
        if (multi_reduced(cases[i]) &&
            ((st = ensure_class_ws(cases[i])) != IBP_OK || (st = ensure_nonbridge_rows(cases[i])) != IBP_OK))
            return st;
        if (record && (st = ensure_bwd_workspace(cases[i], n_box[i])) != IBP_OK) return st;
        if (record == 2 && (st = ensure_bwd_lo_workspace(cases[i], n_box[i])) != IBP_OK) return st;
    }
    MultiPlan *P = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        P = find_plan(cases, n_box, n_case, record);
        if (!P) {
            if ((st = build_plan(cases, n_box, n_case, cases[0]->num_sms, record, &P)) != IBP_OK) return st;
            g_plans.emplace_back(P);
        }
    }
    if (plan_out) *plan_out = P;
    if (record) CUDA_TRY(launch_bwd_zero_cases(P->bargs.p, P->bitems.p, P->n_items, true, s));
    CUDA_TRY(cudaMemsetAsync(P->err.p, 0, sizeof(int), s));
    // per-case box intervals and base flows
    for (int i = 0; i < n_case; ++i) {
        ibp_case *c = cases[i];
        const int nb = n_box[i];
        const int n_box_pad = (nb + kBoxTile - 1) / kBoxTile * kBoxTile;
        CUDA_TRY(cudaMemsetAsync(c->err.p, 0, sizeof(int), s));
        CUDA_TRY(cudaMemsetAsync(c->rbus_t.p, 0, (size_t)c->n_a_pad * n_box_pad * sizeof(float), s));
        const bool red = P->reduced[i] != 0;
        if (red)
            CUDA_TRY(cudaMemsetAsync(c->rcls_t.p, 0, (size_t)c->n_r_pad * n_box_pad * sizeof(float), s));
        BusArgs ba{};
        ba.n_a = c->n_a; ba.n_a_pad = c->n_a_pad; ba.n_dev = c->n_dev; ba.n_gen = c->n_gen; ba.n_box = nb;
        ba.act_ptr = c->act_ptr.p; ba.act_dev = c->act_dev.p; ba.box_lo = box_lo[i]; ba.box_hi = box_hi[i];
        ba.cbus = c->cbus.p; ba.cbus2 = c->cbus2.p; ba.rbus = c->rbus.p; ba.rbus_t = c->rbus_t.p;
        ba.rbus64 = c->rbus64.p;
        ba.n_box_pad = n_box_pad;
        ba.cabs = c->cabs.p; ba.box_consts = c->box_consts.p; ba.err = c->err.p;
        ba.bus_part = c->bus_part.p;
        CUDA_TRY(launch_bus(ba, s));
        if (red) {
            ClsArgs ra{};
            ra.n_box = nb; ra.n_r = c->n_r; ra.n_r_pad = c->n_r_pad; ra.n_a_pad = c->n_a_pad;
            ra.n_box_pad = n_box_pad; ra.cls_ptr = c->cls_ptr.p; ra.cls_col = c->cls_col.p;
            ra.rbus = c->rbus.p; ra.rcls = c->rcls.p; ra.rcls_t = c->rcls_t.p;
            CUDA_TRY(launch_class_radius(ra, s));
        }
        BaseArgs bb{};
        bb.n_l = c->n_line; bb.n_c = c->n_ctg; bb.n_a = c->n_a; bb.n_a_pad = c->n_a_pad; bb.n_box = nb;
        bb.phi = c->phi_a.p; bb.ctg_line = c->ctg_line.p; bb.cbus = c->cbus.p; bb.cbus2 = c->cbus2.p; bb.rbus = c->rbus.p;
        bb.cabs = c->cabs.p; bb.rate_up = c->rate_up.p; bb.rate_dn = c->rate_dn.p;
        bb.box_consts = c->box_consts.p;
        bb.gamma_base = rup_gamma((c->n_a_pad / 4 + 31) / 32, 2, 5);
        bb.line_c = c->line_c.p; bb.line_e = c->line_e.p; bb.line_R = c->line_R.p;
        bb.partials = c->part_base.p; bb.err = c->err.p;
        if (red) {
            bb.is_bridge = c->is_bridge.p;
            bb.rate_c_up = c->rate_c_up.p;
            bb.rate_c_dn = c->rate_c_dn.p;
        }
        bb.ref = ref_args(c);
        if (record == 1) {
            bb.act_count = c->act_count.p;
            bb.act_list = c->act_list.p;
            bb.act_cap = c->act_cap;
        } else if (record == 2) {
            bb.act_count_lo = c->act_count_lo.p;
            bb.act_list_lo = c->act_list_lo.p;
            bb.act_cap_lo = c->act_cap_lo;
        }
        CUDA_TRY(launch_base(bb, c->n_part_base, s));
    }
    // one persistent launch over the contingency tiles of every case
    const int num_sms = cases[0]->num_sms;
    if (P->refine)
        CUDA_TRY(cudaMemsetAsync(P->refq_cnt.p, 0, (size_t)ref_regions(num_sms) * sizeof(int), s));
    CUDA_TRY(launch_ctg_cases(P->variant, P->items.p, P->cta_start.p, P->prefix.p, P->args.p,
                              P->maps.p, P->grid, 2000000000ull, P->err.p, s));
    if (P->refine) {
        RefQueueArgs qa{};
        qa.args = P->args.p; qa.n_regions = ref_regions(num_sms); qa.cap = kRefQCap;
        qa.e = P->refq.p; qa.cnt = P->refq_cnt.p; qa.res = P->refq_res.p;
        CUDA_TRY(launch_refine_queue(qa, num_sms, s));
    }
    int BL, BK, CH;
    multi_tile_shape(&BL, &BK, &CH);
    for (int i = 0; i < n_case; ++i) {
        ibp_case *c = cases[i];
        CUDA_TRY(launch_or_err(c->err.p, P->err.p, s));
        AsmArgs aa{};
        aa.n_box = n_box[i]; aa.n_dev = c->n_dev; aa.n_gen = c->n_gen;
        const int rows = P->reduced[i] ? c->n_nb : c->n_line;
        aa.n_part_ctg = ((rows + BL - 1) / BL) * ((c->n_ctg + BK - 1) / BK) * P->rows_per_item;
        aa.part_stage = c->part_stage.p; aa.n_stage = kPartStages;
        aa.n_part_base = c->n_part_base;
        aa.part_ctg = c->part_ctg.p; aa.part_base = c->part_base.p; aa.box_lo = box_lo[i]; aa.box_hi = box_hi[i];
        aa.seg_ptr = c->seg_ptr.p; aa.slope = c->slope.p; aa.bkpt = c->bkpt.p;
        aa.zeta_inj = c->zeta_inj; aa.zeta_f = c->zeta_f;
        aa.obj_lo = obj_lo[i]; aa.obj_hi = obj_hi[i]; aa.obj_err = obj_err[i]; aa.err = c->err.p;
        CUDA_TRY(launch_assemble(aa, s));
        if ((st = mark_done(c, s)) != IBP_OK) return st;
    }
    return IBP_OK;
}

extern "C" ibp_status ibp_bound_multi(int32_t n_case, ibp_case *const *cases, const int32_t *n_box,
                                      const double *const *box_lo, const double *const *box_hi,
                                      double *const *obj_lo, double *const *obj_hi,
                                      double *const *obj_err, void *cuda_stream) {
    ibp_status st = check_multi_args(n_case, cases, n_box, box_lo, box_hi);
    if (st != IBP_OK) return st;
    if (n_case == 0) return ok();
    if (!obj_lo || !obj_hi || !obj_err) return fail(IBP_EINVAL, "array arguments must not be NULL");
    for (int i = 0; i < n_case; ++i)
        if (!obj_lo[i] || !obj_hi[i] || !obj_err[i])
            return fail(IBP_EINVAL, "pointers of case %d must not be NULL", i);
    DeviceGuard guard(cases[0]->device);
    if (!guard.ok) return fail(IBP_ECUDA, "cannot select device %d", cases[0]->device);
    st = enqueue_multi(n_case, cases, n_box, box_lo, box_hi, obj_lo, obj_hi, obj_err,
                       static_cast<cudaStream_t>(cuda_stream), 0, nullptr);
    if (st != IBP_OK) return st;
    return ok();
}

extern "C" ibp_status ibp_bound_multi_backward(int32_t n_case, ibp_case *const *cases, const int32_t *n_box,
                                               const double *const *box_lo, const double *const *box_hi,
                                               const double *const *grad_obj, double *const *grad_lo,
                                               double *const *grad_hi, double *const *grad_rating,
                                               int32_t side, void *cuda_stream) {
    if (side != 0 && side != 1) return fail(IBP_EINVAL, "side must be 0 (obj_hi) or 1 (obj_lo)");
    ibp_status st = check_multi_args(n_case, cases, n_box, box_lo, box_hi);
    if (st != IBP_OK) return st;
    if (n_case == 0) return ok();
    if (!grad_obj || !grad_lo || !grad_hi) return fail(IBP_EINVAL, "array arguments must not be NULL");
    long long n_items = 0;
    for (int i = 0; i < n_case; ++i) {
        if (!grad_obj[i] || !grad_lo[i] || !grad_hi[i])
            return fail(IBP_EINVAL, "gradient pointers of case %d must not be NULL", i);
        n_items += n_box[i];
    }
    if (n_items > 65535) return fail(IBP_EINVAL, "at most 65535 boxes over all cases (%lld given)", n_items);
    DeviceGuard guard(cases[0]->device);
    if (!guard.ok) return fail(IBP_ECUDA, "cannot select device %d", cases[0]->device);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the forward pass, recording the side's active pairs; its objective goes
    // to each case's scratch
    std::vector<double *> olo(n_case), ohi(n_case), oerr(n_case);
    for (int i = 0; i < n_case; ++i) {
        if ((st = ensure_workspace(cases[i], n_box[i])) != IBP_OK) return st;
        double *d = cases[i]->obj.p;
        olo[i] = d;
        ohi[i] = d + n_box[i];
        oerr[i] = d + 2 * n_box[i];
    }
    MultiPlan *P = nullptr;
    st = enqueue_multi(n_case, cases, n_box, box_lo, box_hi, olo.data(), ohi.data(), oerr.data(), s, 1 + side, &P);
    if (st != IBP_OK) return st;
    // weights, centre and radius passes of every (case, box) in one launch each
    CUDA_TRY(launch_backward_cases(P->bargs.p, P->bitems.p, P->n_items, P->max_n_a_pad, s));
    // the chain rule to each case's box endpoints
    for (int i = 0; i < n_case; ++i) {
        ibp_case *c = cases[i];
        BwdArgs b = bwd_args(c, n_box[i], side);
        b.box_lo = box_lo[i]; b.box_hi = box_hi[i];
        b.grad_obj_hi = grad_obj[i]; b.grad_lo = grad_lo[i]; b.grad_hi = grad_hi[i];
        b.grad_rating = grad_rating ? grad_rating[i] : nullptr;
        CUDA_TRY(launch_bwd_chain(b, s));
        if ((st = mark_done(c, s)) != IBP_OK) return st;
    }
    return ok();
}

