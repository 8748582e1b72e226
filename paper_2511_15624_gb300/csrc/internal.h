// Internal declarations shared by the ABI implementation and the kernel launchers.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/ibp.h"

namespace ibp {

// error word bits (device -> host)
constexpr int kErrTimeout = 1;
constexpr int kErrBadBox = 2;
constexpr int kErrOverflow = 4;  // active-pair list of the adjoint ran out of room
constexpr int kErrBounds = 8;    // an index guard of a checked build (-DIBP_CHECK) failed
constexpr int kErrBadRating = 16;  // a rating given on the device was negative or not finite
// values per partial-sum row: sum s_lo, sum s_hi, error of obj_hi, error of obj_lo
constexpr int kPartVals = 4;
// sums of the objective assembly per (box, stage-1 block)
constexpr int kAsmVals = 18;

// ---------------------------------------------------------------- kernel args
// FP64 refinement of the pairs that can reach obj_hi (null phi64: off).
struct RefArgs {
    const float *phi_hi;     // [n_l][n_a_pad] Phi~ = RN32(Phi) (the FP32 PTDF)
    const double *phi64;     // [n_l][n_a_pad] Phi, the FP64 PTDF of the active columns, or null
    const double *cbus;      // [n_box][n_a_pad] bus centres (FP64)
    const double *rbus64;    // [n_box][n_a_pad] bus radii (FP64, rounded up)
    const float *rbus;       // [n_box][n_a_pad] bus radii (FP32, rounded up)
    const float *cabs;       // [n_box][n_a_pad] |centre| (FP32, rounded up)
    const float *box_consts; // [n_box][4]: ..., sum r, sum |c|
    const double *rate64;    // [n_l] base ratings (FP64, as given)
    const double *rate_c64;  // [n_l] contingency ratings (FP64, as given)
    const float *lodf;       // [n_c][n_l] L~ = RN32(L)
    const float *lodf_lo;    // [n_c][n_l] RN32(L - L~)
    int n_a_pad, n_l;
};

struct BusArgs {
    int n_a, n_a_pad, n_dev, n_gen, n_box;
    const int *act_ptr;     // [n_a + 1] CSR over active bus columns
    const int *act_dev;     // device indices (gens < n_gen are +, loads are -)
    const double *box_lo;   // [n_box][n_dev]
    const double *box_hi;
    double *cbus;           // [n_box][n_a_pad] bus injection centre (FP64)
    float2 *cbus2;          // [n_box][n_a_pad] the same as hi + lo FP32 pair, or null
    float *rbus;            // [n_box][n_a_pad] radius, rounded up
    double *rbus64;         // [n_box][n_a_pad] the FP64 radius, rounded up (or null)
    float *rbus_t;          // [n_a_pad][n_box_pad] transposed radius (or null)
    int n_box_pad;
    float *cabs;            // [n_box][n_a_pad] |centre| rounded up
    float *box_consts;      // [n_box][4] eta_r, eta_c, sum r, sum |c|
    int *err;
    // [n_box][bus_blocks(n_a_pad)][4] per-block sums (sum r, sum |c|, bad box);
    // null: one block per box writes box_consts itself
    float *bus_part;
};

// column blocks per box of the box -> bus kernel when it has bus_part
inline int bus_blocks(int n_a_pad) { return (n_a_pad + 255) / 256; }

struct BaseArgs {
    int n_l, n_c, n_a, n_a_pad, n_box;
    const float *phi;        // [n_l][n_a_pad]
    const int *ctg_line;     // [n_c]
    const double *cbus;
    const float2 *cbus2;     // hi + lo split of cbus; given -> compensated FP32 centre sums
    const float *rbus;
    const float *cabs;
    const float *rate_up;    // base ratings rounded up / down
    const float *rate_dn;
    const float *box_consts;
    float gamma_base;        // worst-case relative excess of the RU radius sums
    float *line_c;           // [n_box][n_l] FP32 centre of the base flow
    float *line_e;           // [n_box][n_l] bound on the centre's error
    float *line_R;           // [n_box][n_l] radius sum, rounded up
    float *hat_l;            // [n_l][n_a_pad] Phi * r (one-box mode) or null
    float *hat_k;            // [n_c][n_a_pad] Phi[ctg line] * r or null
    double *partials;        // [n_part][n_box][kPartVals]
    // adjoint support (null when not recording): active base lines are
    // appended to act_list[box][act_cap] as (l, l, 0, sign); active bridge
    // lines under every contingency as (l, -1, multiplicity bits, sign)
    int *act_count;
    int4 *act_list;
    int act_cap;
    // the same for the adjoint of obj_lo: lines whose upper violation bound
    // s_hi is > 0 (null when not recording)
    int *act_count_lo;
    int4 *act_list_lo;
    int act_cap_lo;
    int *err;
    // bridge lines in closed form (null: off): no contingency of the list
    // moves the flow of a bridge, so its n_c contingency pairs share its base
    // interval, judged against the contingency ratings
    const int *is_bridge;    // [n_l]
    const float *rate_c_up, *rate_c_dn;
    RefArgs ref;             // FP64 refinement of base lines and bridges that can reach obj_hi
};

struct CtgArgs {
    int n_l, n_c, n_a, n_chunks, n_box;
    int tiles_l, n_tiles;
    const float *lodf;       // [n_c][n_l]
    const int *ctg_line;     // [n_c]
    const float *line_c, *line_e, *line_R;  // [n_box][n_l]
    const float *rate_up, *rate_dn;         // contingency ratings
    const float *box_consts;                // [n_box][4]
    const float *rbus_t;     // [n_a_pad][n_box_pad] (batched kernel)
    int n_box_pad;
    float gamma;             // worst-case relative excess of the RU radius sums
    float *flow_lo, *flow_hi;  // [n_box][n_c][n_l] or null
    double *partials;        // [n_tiles * warps_per_tile][n_box][kPartVals]
    int warps_per_tile;      // partial-sum rows written per tile
    int *err;
    unsigned long long wait_ns;
    // adjoint support (null when not recording): pairs whose certified lower
    // violation bound is > 0 are appended as (l, ctg line, L bits, sign bits)
    int *act_count;
    int4 *act_list;
    int act_cap;
    // the same for the adjoint of obj_lo: pairs whose upper violation bound
    // s_hi is > 0 (null when not recording)
    int *act_count_lo;
    int4 *act_list_lo;
    int act_cap_lo;
    int part_rows_cap;       // rows the partials buffer holds (index guard of checked builds)
    // line screen (null: all n_l lines): line tile rows index the compacted
    // list live[0 .. *n_live) of lines that can carry a violation
    const int *live;
    const int *n_live;
    RefArgs ref;             // FP64 refinement of the pairs that can reach obj_hi
    // global queues of the refinement, one region of refq_cap entries per
    // (CTA, warp) of the launch; null: queue in shared memory and refine in
    // the kernel
    int4 *refq;
    int *refq_cnt;
    int refq_cap;
};

// The refinement of the queued pairs, after a contingency launch: every queue
// entry (l, k, case << 16 | box, row) is refined by one warp anywhere on the
// GPU (k_refine_queue), then each region's results are added to their
// partial-sum rows in queue order (k_refine_apply).
struct RefQueueArgs {
    const CtgArgs *args;     // per case (device array), or null: `one`
    CtgArgs one;
    int n_regions, cap;
    const int4 *e;           // [n_regions][cap]
    const int *cnt;          // [n_regions]
    double2 *res;            // [n_regions][cap]: refined s_lo, allowance
};
cudaError_t launch_refine_queue(const RefQueueArgs &a, int num_sms, cudaStream_t s);
constexpr int kRefRegionsPerSm = 32;  // queue regions the workspace holds per SM
constexpr int kRefQCap = 128;         // entries per region

// Paper-mode line screen (Sec. II-C, the interval of eq. (ctg flow matrix
// form) propagated in two parts): line l needs the tight radius only if, for
// some contingency and box, |c_kl| + R_l + |L[l,k]| R_k can exceed its rating.
struct ScreenArgs {
    int n_l, n_c, n_box;
    const float *lodf;       // [n_c][n_l]
    const int *ctg_line;     // [n_c]
    const float *line_c, *line_e, *line_R;  // [n_box][n_l]
    const float *box_consts;                // [n_box][4]
    const float *rate_dn;    // contingency ratings rounded down
    int *live_flag;          // [n_l], zeroed before the launch
    int *live;               // [n_l] compacted list (ascending)
    int *n_live;             // [1]
    // bridge lines never reach the contingency kernel (null: none); with
    // paper_test == 0 every other line is kept
    const int *is_bridge;
    int paper_test;
    // rows of the compacted list: rows[i] = src[live[i]] (* radius when
    // scaled); one-box calls also write hat_k[k] = src[ctg_line[k]] * radius
    const float *src;        // [n_l][n_w]: PTDF columns of the active buses or bus classes
    const float *radius;     // [n_w] (one-box) or null (copy)
    float *rows;             // [n_l][n_w]
    float *hat_k;            // [n_c][n_w] or null
    int n_w;                 // row width (a multiple of 32)
    int *err;
};

// Paper-mode objective: every contingency flow takes the two-part interval
// c_kl +- (R_l + |L[l,k]| R_k) (eq. (ctg flow matrix form) propagated as the
// paper does), and the violation sums of eq. (slack-Sc) go to partial rows
// [gridDim.x * gridDim.y][n_box][kPartVals].
struct PaperArgs {
    int n_l, n_c, n_box;
    const float *lodf;       // [n_c][n_l]
    const int *ctg_line;     // [n_c]
    const float *line_c, *line_e, *line_R;  // [n_box][n_l]
    const float *box_consts;                // [n_box][4]
    const float *rate_up, *rate_dn;         // contingency ratings
    float gamma_base;        // relative excess of the base radius sums R~
    double *partials;
    int *err;
    // FP64 refinement of the pairs that can reach obj_hi (ref.phi64 null:
    // off), from the per-line FP64 values of k_line_exact: centre c64, radius
    // R64 and X = sum_b |Phi~_l,b| (r_b + |c_b|), each [n_box][n_l]
    RefArgs ref;
    const double *lc64, *lR64;
    const float *lX;
};

// Per (box, line) FP64 values of the base flow from the FP64 PTDF (the paper
// mode's refinement): c64 = sum_b Phi_l,b c_b, R64 = sum_b |Phi_l,b| r_b
// (round-up), X = sum_b |Phi~_l,b| (r_b + |c_b|) (FP32 round-up).
struct LineExactArgs {
    RefArgs ref;
    int n_l, n_box;
    double *c64, *R64;       // [n_box][n_l]
    float *X;                // [n_box][n_l]
};
cudaError_t launch_line_exact(const LineExactArgs &a, int num_sms, cudaStream_t s);

// Linear (CROWN-style) relaxation of the penalty terms and its optimised
// slopes (ibp_bound_linear).  Every penalty term t -- a base line, a
// contingency pair, the imbalance -- is bounded below by a line with slope
// a_t in [-1, 1]: max(|y| - R, 0) >= a y - |a| R and |y| >= a y, so for every
// choice of slopes f(x) <= l_a(x) on the box and max f <= max_x l_a(x), whose
// maximum over the box is exact because l_a is separable per device.  The
// slopes are optimised by a primal-dual hybrid gradient iteration on
// max_x min_a l_a(x); any slopes give a certified bound.
struct LinArgs {
    int n_l, n_c, n_a, n_a_pad, n_dev, n_gen, n_box;
    const float *phi;          // [n_l][n_a_pad] FP32 PTDF (iterations)
    const double *phi64;       // [n_l][n_a_pad] FP64 PTDF (certified value)
    const float *lodf, *lodf_lo;  // [n_c][n_l]
    const int *ctg_line;       // [n_c]
    const int *cl_ptr, *cl_ctg;   // CSR: contingencies whose outaged line is l
    const int *act_ptr, *act_dev, *dev_col;
    const double *rate64, *rate_c64;
    const double *box_lo, *box_hi;  // [n_box][n_dev]
    const int *seg_ptr;
    const double *slope, *bkpt;
    double zeta_inj, zeta_f;
    // diagonal step sizes (Pock-Chambolle, alpha = 1, with row and column sums
    // of |D K| bounded by the triangle inequality): a pair's dual step is
    // 1 / (z_f (S_l + |L_lk| S_k)), a base line's 1 / (z_f S_l), the
    // imbalance's 1 / (z_inj n_dev); a device's primal step is tau[d]
    const float *pc_S;         // [n_l] S_l = sum_b |Phi[l,b]| (devices at b)
    const double *pc_tau;      // [n_dev]
    // iteration state
    double *w;                 // [n_box] primal weight
    double *x, *sx, *xb, *x_last, *x_avg;  // [n_box][n_dev]
    float *a_c, *c_last;                   // [n_box][n_c][n_l]
    float *a_b, *b_last;                   // [n_box][n_l]
    double *a0, *a0_last;                  // [n_box]
    float *p;                  // [n_box][n_a_pad] bus injections of xb
    double *stot;              // [n_box] total injection of xb
    double *stot_part;         // [n_box][ceil(n_dev / 128)] per-block partial sums of it
    float *f;                  // [n_box][n_l] base flows of xb
    float *colsum;             // [n_box][n_l]
    float *rowdot;             // [n_box][n_c]
    float *g;                  // [n_box][n_a_pad] zeta_f (Phi^T W)_b
    double *red;               // [n_box][4] restart reductions
    int n_avg;                 // iterations in the running sum of x
    // certified value of the dual function at the slopes (a_c, a_b, a0)
    double *W64, *Wabs, *constl;           // [n_box][n_l]
    double *rd64, *rda;                    // [n_box][n_c]
    double *g64, *G64;                     // [n_box][n_a_pad]
    double *ub, *ub_err;                   // [n_box]
};
cudaError_t lin_iteration(const LinArgs &a, int num_sms, cudaStream_t s);
cudaError_t lin_restart(const LinArgs &a, int num_sms, cudaStream_t s);
cudaError_t lin_certify(const LinArgs &a, int num_sms, cudaStream_t s);
// the preconditioner of a case (once): S, tau; A, B [n_a_pad] and Lsum [n_c] scratch
cudaError_t lin_precondition(const LinArgs &a, float *S, double *tau, double *A, double *B, double *Lsum,
                             cudaStream_t s);
cudaError_t lin_gradient(const LinArgs &a, int num_sms, cudaStream_t s);

// Radius of each bus class (the active buses whose PTDF columns coincide on
// every non-bridge line): rcls[j] = RU(sum of rbus over the class members).
struct ClsArgs {
    int n_box, n_r, n_r_pad, n_a_pad, n_box_pad;
    const int *cls_ptr;      // [n_r + 1] CSR over active columns
    const int *cls_col;
    const float *rbus;       // [n_box][n_a_pad]
    float *rcls;             // [n_box][n_r_pad]
    float *rcls_t;           // [n_r_pad][n_box_pad] or null
};

struct BwdArgs {
    int n_l, n_a, n_a_pad, n_dev, n_gen, n_box, act_cap;
    // 0: adjoint of obj_hi (its active set: s_lo > 0); 1: of obj_lo (s_hi > 0)
    int side;
    const float *phi;          // [n_l][n_a_pad]
    const int *act_count;      // [n_box]
    const int4 *act_list;      // [n_box][act_cap]
    double *W;                 // [n_box][n_l] line weights of the centre gradient
    int *cnt;                  // [n_box][n_l] active count per line (rating gradient)
    double *dc, *dr;           // [n_box][n_a_pad] d(sum s_lo)/dc, d(sum s_lo)/dr (sign: see kernels)
    const int *dev_col;        // [n_dev] active column of the device's bus or -1
    const double *box_lo, *box_hi;
    const int *seg_ptr;
    const double *slope, *bkpt;
    double zeta_inj, zeta_f;
    const double *grad_obj_hi; // [n_box]: d loss / d obj (obj_hi or obj_lo, by side)
    double *grad_lo, *grad_hi; // [n_box][n_dev]
    double *grad_rating;       // [n_box][n_l] or null
};

struct AsmArgs {
    int n_box, n_dev, n_gen;
    int n_part_ctg, n_part_base;
    // screened calls: the contingency partials cover ceil(*n_live / BL) line
    // tiles x tiles_k x rows_per_tile rows (n_part_ctg is ignored)
    const int *n_live;
    int live_BL, live_tiles_k, live_rows_per_tile;
    // two-stage assembly (null: one block per box reads every row and device):
    // stage 1 writes [n_box][n_stage][kAsmVals]
    double *part_stage;
    int n_stage;
    const double *part_ctg;   // [n_part_ctg][n_box][kPartVals]
    const double *part_base;  // [n_part_base][n_box][kPartVals]
    const double *box_lo, *box_hi;
    const int *seg_ptr;       // [n_dev + 1]
    const double *slope, *bkpt;
    double zeta_inj, zeta_f;
    double *obj_lo, *obj_hi, *obj_err;  // obj_err [n_box][2]: error of hi, of lo
    const int *err;
};

// ----------------------------------------------------------- kernel variants
struct CtgVariant {
    int id;
    int batched;     // 0: one-box scaled kernel, 1: multi-box kernel
    int BL, BK, CH, ST;
    int boxes_per_thread;
    // one-box inner sum: 0 one round-up add per bus, 1 a 4-bus add tree,
    // 2 packed two-lane sums (-1: multi-box)
    int body;
    const char *name;
};

const CtgVariant *ctg_variants(int *count);
const CtgVariant *ctg_variant_by_id(int id);
int ctg_warps(const CtgVariant &v);

// launchers (return cudaError_t of the launch)
cudaError_t launch_bus(const BusArgs &a, cudaStream_t s);
cudaError_t launch_base(const BaseArgs &a, int n_part, cudaStream_t s);
int base_partials_count(int num_sms);
cudaError_t launch_ctg(const CtgVariant &v, const CUtensorMap &mL, const CUtensorMap &mK,
                       const CtgArgs &a, int grid, cudaStream_t s);
cudaError_t launch_ctg_multi(const CtgVariant &v, const CUtensorMap &mL, const CUtensorMap &mK,
                             const CUtensorMap &mR, const CtgArgs &a, int grid, cudaStream_t s);
constexpr int kBoxTile = 16;  // boxes per work item of the multi-box kernel

// one work item of the many-case launch
struct MultiItem {
    int case_id, l0, k0, b0, tile_lk, n_chunks;
};
cudaError_t launch_ctg_cases(int variant, const MultiItem *items, const int *cta_start,
                             const uint32_t *prefix, const CtgArgs *args, const CUtensorMap *maps,
                             int grid, unsigned long long wait_ns, int *err, cudaStream_t s);
void multi_tile_shape(int *BL, int *BK, int *CH);
// partial rows per work item of the body launch_ctg_cases runs for `variant`
int cases_rows_per_item(int variant);
cudaError_t launch_assemble(const AsmArgs &a, cudaStream_t s);
cudaError_t launch_screen(const ScreenArgs &a, int num_sms, cudaStream_t s);
cudaError_t launch_class_radius(const ClsArgs &a, cudaStream_t s);
int paper_partials_count(int n_l, int n_c);
cudaError_t launch_paper(const PaperArgs &a, cudaStream_t s);
cudaError_t launch_backward(const BwdArgs &a, cudaStream_t s);
// many cases: items = (case, box) pairs, args = the cases' BwdArgs in device
// memory (per-call pointers unused); the chain rule runs per case
cudaError_t launch_bwd_zero_cases(const BwdArgs *args, const int2 *items, int n_items, bool counts,
                                  cudaStream_t s);
cudaError_t launch_backward_cases(const BwdArgs *args, const int2 *items, int n_items, int max_n_a_pad,
                                  cudaStream_t s);
cudaError_t launch_bwd_chain(const BwdArgs &a, cudaStream_t s);
cudaError_t launch_wait_selftest(int *flag, unsigned long long limit_ns, cudaStream_t s);
cudaError_t launch_or_err(int *dst, const int *src, cudaStream_t s);

// case-build kernels
cudaError_t launch_scatter_dense(double *dst, int64_t ld, const int *rows, const int *cols,
                                 const double *vals, int nnz, cudaStream_t s);
cudaError_t launch_extract_phi(const double *Z, int nb_r, int n_l, const int *act_red, int n_a,
                               int n_a_pad, float *phi_a, double *phi64, cudaStream_t s);
cudaError_t launch_lodf(const double *Z, int nb_r, int n_l, int n_c, const int *ctg_from_red,
                        const int *ctg_to_red, const int *ctg_line, float *lodf, float *lodf_lo,
                        double *den_out, float *maxabs_out, cudaStream_t s);
cudaError_t launch_gather_rows(const float *src, int ld, const int *rows, int n_rows,
                               float *dst, cudaStream_t s);
cudaError_t launch_gather_cols(const float *src, int ld_src, int n_rows, const int *cols, int n_cols,
                               float *dst, int ld_dst, cudaStream_t s);

// read-only view of a case's device data and sizes (for entry points that
// live in other translation units)
struct CaseView {
    int device, n_line, n_ctg, n_gen, n_dev, n_a, n_a_pad, num_sms;
    double zeta_inj, zeta_f;
    const float *phi_a, *lodf, *rate_up, *rate_dn, *rate_c_up, *rate_c_dn;
    const int *ctg_line, *act_ptr, *act_dev, *seg_ptr;
    const double *slope, *bkpt;
    int n_part_base;
    const double *phi64;                // null when the case does not refine
    const float *lodf_lo;
    const double *rate64, *rate_c64;
};
bool case_view(const ibp_case *c, CaseView *v);
ibp_status set_error(ibp_status s, const char *msg);

// tensor maps
bool encode_map_2d(CUtensorMap *map, const float *base, int64_t inner, int64_t outer,
                   int64_t row_stride_elems, int box_inner, int box_outer, std::string *err,
                   bool swizzle = true);

}  // namespace ibp
