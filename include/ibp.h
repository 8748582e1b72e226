/*
 * ibp.h -- C ABI of the GB300 interval-bound-propagation library for the
 * soft-constrained security-constrained DCOPF market-clearing objective.
 *
 * What it computes (arXiv 2511.15624):
 *   f_ibp(p_d, p_g) = sum_j c_j(p_d,j) - sum_i g_i(p_g,i)
 *                     - zeta_inj 1^T s_inj - zeta_f (1^T s_fb + s_fc^agg)
 *   (appendix eq. (ibp_f), eq. (penalized-objective)), with
 *     s_inj  = |(E^T Phi - I) p_inj|                      eq. (slack-sinj)
 *     s_fb   = max(|Phi p_inj| - p_fb^max, 0)             eq. (slack-sfb)
 *     S_fc   = max(|P_fc| - 1 (p_fc^max)^T, 0), s_fc^agg = 1^T S_fc 1
 *                                                         eqs. (slack-Sc), (slack-sagg)
 *     P_fc[k,:] = H_k p_inj,  H_k = Phi + L[:,k] Phi[k,:] (Sec. II-C,
 *       eq. (ctg flow simplified); L = line outage distribution factors)
 *     p_inj = N_g p_g - N_d p_d                           (Sec. II-A)
 *   and bounds it over the input box [box_lo, box_hi] by interval bound
 *   propagation, eq. (IBP): an affine map W over a box with centre x_mu and
 *   radius x_sigma lands in [W x_mu - |W| x_sigma, W x_mu + |W| x_sigma].
 *   The contingency flows use the tight per-row rule (|H_k| r), which gives
 *   the exact range of every post-contingency flow.
 *
 * Certification: every reported interval contains the exact IBP interval
 * computed in real arithmetic from the FP64 sensitivities the library built
 * (outward rounding throughout).  obj_err bounds the distance between each
 * reported and exact IBP objective bound.
 *
 * Conventions
 *   - Units: MW, $/MWh, reactance in p.u.; a single slack bus absorbs any
 *     mismatch; flows are positive from line_from to line_to.
 *   - Devices: boxes hold generators first, then loads: [n_gen + n_load].
 *   - Piecewise-linear cost/value curves (Sec. III-B, eqs. (single ReLU),
 *     (combined ReLUs)): device i owns n_seg[i] consecutive entries of the
 *     flattened slope[] (a_m >= 0) and bkpt[] (segment starts, strictly
 *     increasing); the curve is 0 before bkpt[0] and continues with the last
 *     slope beyond the last breakpoint.
 *   - Ownership: every input array is copied during the call; outputs are
 *     written to caller-owned memory.  A case owns its device memory until
 *     ibp_case_destroy.
 *   - Pointers: ptr_mode 0 = host pointers, the call is synchronous (it copies
 *     inputs to the device, runs, copies results back and synchronises the
 *     stream).  ptr_mode 1 = device pointers, the call only enqueues work on
 *     cuda_stream (NULL = legacy default stream) and returns; numerical errors
 *     found on the device are reported by the next ibp_case_sync().
 *   - Errors: no exception crosses the ABI.  Every call returns ibp_status and
 *     leaves a message in a thread-local buffer read by ibp_last_error().
 *     A device-side failure (an input box with lo > hi or a non-finite entry
 *     seen only on the device, or a bounded wait that ran out) writes NaN into
 *     obj_lo/obj_hi/obj_err of the call and makes ibp_case_sync() return
 *     IBP_EINVAL or IBP_ETIMEOUT.  Nothing traps or hangs on the device.
 *   - Threads: calls on one case must not overlap; distinct cases may be used
 *     from distinct host threads.
 */
#ifndef IBP_GB300_H
#define IBP_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ibp_case ibp_case; /* opaque; owns device buffers */

typedef enum {
    IBP_OK = 0,
    IBP_EINVAL = 1,    /* bad argument (index, size, NaN, lo > hi, ...) */
    IBP_EISLAND = 2,   /* network not connected, or a contingency islands it */
    IBP_ESINGULAR = 3, /* FP64 factorisation failed for another reason */
    IBP_ENOMEM = 4,    /* host or device allocation failed */
    IBP_ECUDA = 5,     /* a CUDA runtime / library call failed, or no device */
    IBP_ETIMEOUT = 6,  /* a bounded device-side wait ran out */
    IBP_EUNSOUND = 7,  /* an internal consistency check on the bound failed */
    IBP_ENOTSUP = 8    /* the case was created without a device (dry run) */
} ibp_status;

/*
 * Build a case: validate the network, build the FP64 PTDF (Sec. II-A, eq. (line
 * flow ptdf), slack column zero) and the line outage distribution factors of
 * every listed contingency (Sec. II-C, eq. (ctg flow simplified): the
 * Sherman-Morrison rank-1 update written as L[l,k] = PTDF_line[l,k] /
 * (1 - PTDF_line[k,k]), L[k,k] = -1), keep the columns of buses that carry a
 * device (slack excluded) in FP32 on the device, and allocate the per-call
 * working buffers.  Runs once per case, outside any timed bound.
 *
 *   n_bus >= 2, 0 <= slack_bus < n_bus
 *   n_line >= 1, line_from/line_to in [0, n_bus), from != to
 *   reactance[n_line] > 0 (p.u.), rating[n_line] >= 0 (MW, base case),
 *   rating_ctg[n_line] >= 0 or NULL (then = rating), eq. (slack-Sc)
 *   n_gen, n_load >= 0 with n_gen + n_load >= 1; *_bus in [0, n_bus);
 *   *_nseg[i] >= 1; *_slope >= 0; *_bkpt strictly increasing per device
 *   zeta_inj, zeta_f >= 0 ($/MW), eq. (penalized-objective)
 *   n_ctg >= 0, ctg_line[n_ctg] in [0, n_line) (duplicates are allowed and
 *     counted twice, as in eq. (slack-sagg))
 *   device: CUDA device ordinal; -1 = dry run (validation and host-side graph
 *     checks only, no device work; the case then only validates arguments)
 * Errors: IBP_EINVAL, IBP_EISLAND (disconnected network or a bridge
 * contingency, checked on the host before any device work), IBP_ESINGULAR,
 * IBP_ENOMEM, IBP_ECUDA.
 */
ibp_status ibp_case_create(int32_t n_bus, int32_t slack_bus, int32_t n_line,
                           const int32_t *line_from, const int32_t *line_to,
                           const double *reactance, const double *rating,
                           const double *rating_ctg, int32_t n_gen,
                           const int32_t *gen_bus, const int32_t *gen_nseg,
                           const double *gen_slope, const double *gen_bkpt,
                           int32_t n_load, const int32_t *load_bus,
                           const int32_t *load_nseg, const double *load_slope,
                           const double *load_bkpt, double zeta_inj, double zeta_f,
                           int32_t n_ctg, const int32_t *ctg_line, int32_t device,
                           ibp_case **out);

void ibp_case_destroy(ibp_case *c);

/*
 * Certified IBP bound of f_ibp over each of n_box boxes (appendix eq. (f-ibp)
 * bounds max f over the box from above by obj_hi).
 *   box_lo, box_hi [n_box][n_gen + n_load] (FP64, MW), lo <= hi, finite
 *   obj_lo, obj_hi [n_box] (FP64): obj_hi >= the exact IBP upper bound >=
 *     max f over the box; obj_lo <= the exact IBP lower bound.
 *   obj_err [n_box][2] (FP64): {e_hi, e_lo} with |obj_hi - exact IBP upper
 *     bound| <= e_hi and |obj_lo - exact IBP lower bound| <= e_lo (a-priori
 *     bounds of the FP32 outward rounding, stated per result).
 *     obj_hi < 0 certifies that the box is welfare-negative, eq. (inf-or-wn).
 *   flow_lo, flow_hi [n_box][n_ctg][n_line] (FP32) or NULL: outward-rounded
 *     post-contingency flow intervals (the outaged line is exactly [0, 0]).
 * 1 <= n_box <= 65535 (n_box == 0 is a no-op returning IBP_OK; more than
 * 65535 boxes return IBP_EINVAL: split them over several calls).  The same
 * limit holds for ibp_bound_paper, ibp_bound_backward and each case of
 * ibp_bound_multi.
 */
ibp_status ibp_bound(ibp_case *c, int32_t n_box, const double *box_lo,
                     const double *box_hi, double *obj_lo, double *obj_hi,
                     double *obj_err, float *flow_lo, float *flow_hi,
                     int32_t ptr_mode, void *cuda_stream);

/*
 * Adjoint of obj_hi (not certified; FP32 kernels with FP64 accumulation).
 * Given grad_obj_hi [n_box] (d loss / d obj_hi), writes
 *   grad_lo, grad_hi [n_box][n_gen + n_load]: d loss / d box_lo, d box_hi
 *   grad_rating [n_box][n_line] or NULL: d loss / d rating[l] when the base
 *     rating and the contingency rating of line l move together (the shared
 *     rating of a case created with rating_ctg = NULL):
 *     zeta_f * grad_obj_hi * (the line's active base flow, 0 or 1, plus its
 *     active contingency pairs), eqs. (slack-sfb), (slack-Sc).  With separate
 *     contingency ratings, the base part alone is the derivative in rating
 *     and the pair count alone the one in rating_ctg.
 * The derivative is taken with the active set of the forward pass (pairs whose
 * certified lower violation bound is > 0); it is valid away from kinks.  The
 * forward pass records that set in a list of up to 16M entries per call,
 * shared by the boxes (IBP_ENOMEM beyond it, as for any device-side error, and
 * the gradients of a box whose share overflowed are NaN).
 */
ibp_status ibp_bound_backward(ibp_case *c, int32_t n_box, const double *box_lo,
                              const double *box_hi, const double *grad_obj_hi,
                              double *grad_lo, double *grad_hi, double *grad_rating,
                              int32_t ptr_mode, void *cuda_stream);

/*
 * Adjoint of obj_lo (not certified), with the arguments and layouts of
 * ibp_bound_backward: grad_obj_lo [n_box] = d loss / d obj_lo.  obj_lo =
 * C(pd_lo) - G(pg_hi) - zeta_inj s_inj,hi - zeta_f (sum s_fb,hi + sum s_fc,hi)
 * (eq. (penalized-objective) under eq. (IBP)) takes the upper violation bounds
 * s_hi = max(|c| + r - rating, 0); the derivative uses the pairs whose s_hi
 * is > 0 in the forward pass:
 *   d obj_lo / d c_b = -zeta_f sum sgn(c_kl) H_k[l,b],
 *   d obj_lo / d r_b = -zeta_f sum |H_k[l,b]|,
 *   grad_rating[l] = zeta_f * grad_obj_lo * (the line's active base flow plus
 *     its active contingency pairs), for base and contingency ratings moving
 *     together,
 * plus the imbalance and cost terms, chained to the box endpoints.  Those
 * pairs are most pairs of a wide box: the forward pass records them in a list
 * of up to 64M entries per call, shared by the boxes (1 GiB; IBP_ENOMEM beyond
 * it, reported by the call in host mode and by ibp_case_sync in device mode,
 * and the gradients of a box whose share overflowed are NaN), and the radius
 * pass costs O(pairs x active buses), like the forward kernel without its
 * tiling.
 * Valid away from kinks.
 */
ibp_status ibp_bound_backward_lo(ibp_case *c, int32_t n_box, const double *box_lo,
                                 const double *box_hi, const double *grad_obj_lo,
                                 double *grad_lo, double *grad_hi, double *grad_rating,
                                 int32_t ptr_mode, void *cuda_stream);

/*
 * Linear (CROWN-style) relaxation bound of max f over each box, the dual of
 * the LP whose optimum is max f (the paper bounds f by IBP and names linear
 * relaxations of the CROWN family as related work, Sec. I).  Every penalty
 * term is bounded below by a line with slope a in [-1, 1] --
 * max(|y| - R, 0) >= a y - |a| R for the base and contingency flows of
 * eqs. (slack-sfb), (slack-Sc), |y| >= a y for the total injection of
 * eq. (slack-sinj) -- so f <= l_a on the box for every choice of slopes, and
 * max over the box of l_a, which is separable per device, is exact.  The
 * slopes are optimised by n_iter primal-dual hybrid gradient iterations
 * with diagonal step sizes (the inverse row and column sums of the operator,
 * bounded by the triangle inequality) and a primal weight starting at
 * primal_weight (a scale of the dual steps against the primal ones; the
 * binding starts at 0.01), adapted every 1000 iterations and at the end of a
 * call, when the dual function is also certified at the current slopes; any
 * slopes give a certified bound, and the iteration approaches the LP
 * optimum.  Warm calls of any length follow one long call closely (calls of
 * 500 iterations were measured to end within 1e-5 of it).
 *   box_lo, box_hi [n_box][n_gen + n_load]; obj_hi [n_box]: the smallest
 *     certified value of the dual function met at an adaptation (or, warm,
 *     at the start of the call), computed from the FP64 sensitivities with
 *     outward rounding: obj_hi >= max f;
 *   obj_err [n_box]: a bound on its rounding error;
 *   x_point [n_box][n_gen + n_load] or NULL: the primal point averaged over
 *     the last adaptation window, a candidate maximiser (f there, e.g. from
 *     ibp_bound on the zero-width box at it, is a certified lower bound of
 *     max f);
 *   warm: 0 starts from zero slopes and the box midpoints (the case then
 *     holds state for these n_box boxes); warm = 1 + f (f >= 0) continues
 *     the iteration from the state the case holds for its boxes
 *     [f, f + n_box) (see ibp_case_linear_inherit), the points moved into the
 *     boxes, keeping the state of the other held boxes (IBP_EINVAL when those
 *     boxes are not held); obj_hi is then also at most the certified value at
 *     the held slopes, so a sub-box continued from its parent never gets a
 *     larger bound than the parent's last one.
 * The first call on a case computes the diagonal step sizes of the
 * iteration (row and column sums of the operator, O(n_line n_active +
 * n_ctg n_active), no synchronisation).  Each call captures its chunk of 50
 * iterations into a CUDA graph on a private stream, so the call itself must
 * not be made while the caller's stream is being captured.  Memory: 8 bytes
 * per (box, contingency, line).  ptr_mode and stream as in ibp_bound.
 */
ibp_status ibp_bound_linear(ibp_case *c, int32_t n_box, const double *box_lo,
                            const double *box_hi, int32_t n_iter, double primal_weight,
                            int32_t warm, double *obj_hi, double *obj_err, double *x_point,
                            int32_t ptr_mode, void *cuda_stream);

/* Keep optimising from the state a case holds (warm != 0 in ibp_bound_linear,
 * primal_weight then ignored): box j of the next call continues from the
 * slopes, their last adaptation's reference, the point, its running sum and
 * the primal weight of box parent[j] of the last
 * call or inheritance (host array [n_new]).  A sub-box can start from its
 * parent's slopes: any slopes give a certified bound, and the parent's bound
 * already holds for the sub-box.  Synchronises the device.  No counterpart in
 * the paper. */
ibp_status ibp_case_linear_inherit(ibp_case *c, int32_t n_new, const int32_t *parent);

/* The slopes of the last ibp_bound_linear call of the case (host arrays):
 * a_ctg [n_box][n_ctg][n_line], a_base [n_box][n_line], a_inj [n_box].  For an
 * independent evaluation of the certified value.  Synchronises the case's
 * last call.  No counterpart in the paper. */
ibp_status ibp_case_linear_slopes(ibp_case *c, int32_t n_box, float *a_ctg, float *a_base,
                                  double *a_inj);

/*
 * Replace the case's line ratings (eqs. (slack-sfb), (slack-Sc)): rating
 * [n_line] (base, MW) and rating_ctg [n_line] or NULL (then the contingency
 * ratings equal the new base ratings).  ptr_mode 0: host pointers, validated
 * on the host (finite, >= 0; IBP_EINVAL leaves the ratings unchanged), the
 * call returns when the device copies are updated.  ptr_mode 1: device
 * pointers, enqueued on cuda_stream; a bad entry leaves every rating
 * unchanged and makes the next ibp_case_sync return IBP_EINVAL.  Later calls
 * on the same stream use the new ratings; the sensitivities are unchanged.
 * The paper treats ratings as data; this lets a caller differentiate through
 * them (torch.autograd.Function of the binding).
 */
ibp_status ibp_case_set_ratings(ibp_case *c, const double *rating, const double *rating_ctg,
                                int32_t ptr_mode, void *cuda_stream);

/*
 * Bounds of many cases of uneven size in one persistent launch of the
 * contingency kernel (device pointers only).  For case i:
 *   box_lo[i], box_hi[i] [n_box[i]][n_dev_i], obj_lo[i], obj_hi[i], obj_err[i]
 *   [n_box[i]].  Flow intervals are not written.
 */
ibp_status ibp_bound_multi(int32_t n_case, ibp_case *const *cases,
                           const int32_t *n_box, const double *const *box_lo,
                           const double *const *box_hi, double *const *obj_lo,
                           double *const *obj_hi, double *const *obj_err,
                           void *cuda_stream);

/*
 * Adjoint of many cases' bounds (ibp_bound_backward for side 0: obj_hi;
 * ibp_bound_backward_lo for side 1: obj_lo), device pointers only.  The
 * forward pass runs as in ibp_bound_multi, one persistent launch over every
 * case's contingency tiles, recording the side's active pairs; the weights,
 * centre and radius passes then run once each over all (case, box) items,
 * and the chain rule to the box endpoints once per case.  For case i:
 *   box_lo[i], box_hi[i] [n_box[i]][n_dev_i]; grad_obj[i] [n_box[i]]:
 *   d loss / d obj; grad_lo[i], grad_hi[i] [n_box[i]][n_dev_i] (written);
 *   grad_rating NULL, or grad_rating[i] NULL or [n_box[i]][n_line_i]
 *   (written, as in ibp_bound_backward).
 * At most 65535 boxes over all cases (IBP_EINVAL).  The work plan is cached
 * per set of cases and box counts (separately from ibp_bound_multi's), so
 * later calls only enqueue kernels and can be captured in a CUDA graph.
 * Device-side errors (a box with lo > hi, an active-pair list that
 * overflows) are reported by ibp_case_sync of the case concerned, as for
 * the other device-pointer calls.  The paper differentiates nothing; this is
 * the batched form of the adjoint.
 */
ibp_status ibp_bound_multi_backward(int32_t n_case, ibp_case *const *cases,
                                    const int32_t *n_box, const double *const *box_lo,
                                    const double *const *box_hi,
                                    const double *const *grad_obj, double *const *grad_lo,
                                    double *const *grad_hi, double *const *grad_rating,
                                    int32_t side, void *cuda_stream);

/*
 * One-box bound that allocates no device memory (the paper has no counterpart:
 * this is a deployment aid).  Some callers cannot call cudaMalloc while they
 * compute a bound: code that runs while a CUDA stream is being captured into a
 * graph, host threads with latency limits (cudaMalloc/cudaFree may synchronise
 * the whole device), and programs whose own allocator owns all device memory.
 * ibp_bound may allocate its per-call workspace on first use; this entry point
 * never does.  Its per-call buffers live in one file-scope __device__ array of
 * 8 MiB that every GPU which loads the library holds until the process exits.
 *
 *   c: a case from ibp_case_create (its sensitivities were allocated there)
 *   box_lo, box_hi [n_gen + n_load], obj_lo, obj_hi [1], obj_err [2]: DEVICE
 *     pointers; the work is only enqueued on cuda_stream (NULL = legacy
 *     default stream).  Same results as ibp_bound up to FP32 rounding order
 *     (same certified arithmetic, unscaled PTDF rows, the same FP64
 *     refinement of the obj_hi terms, queued per warp in shared memory);
 *     flows are not written.
 * Limits and behaviour:
 *   - returns IBP_EINVAL, touching nothing, when the case needs more scratch
 *     than the array holds.  The scratch is 24 bytes per active bus, 12 per
 *     line, 256 per tile of 128 lines x 64 contingencies and 512 per SM, each
 *     part rounded up to 256 bytes: 2,015,744 bytes (1.9 MiB) for 8316 buses
 *     (5474 with a device), 10500 lines and 5000 contingencies on a 152-SM GPU;
 *   - the first call on a device (in a CUDA context) looks up the array's
 *     device address (cudaGetSymbolAddress), so make that first call before
 *     any stream capture; after the context is created again (e.g. after
 *     cudaDeviceReset) the next call looks the address up again, and must
 *     likewise come before any capture;
 *   - every call, on every case, shares the one array (it keeps the last
 *     call's contents; the error word is cleared at the start of each call):
 *     calls whose work overlaps on the GPU race and must be serialised by the
 *     caller, e.g. by issuing them on one stream;
 *   - a device-side error (a box with lo > hi, a non-finite entry) writes NaN
 *     into obj_lo, obj_hi and obj_err.
 */
ibp_status ibp_bound_noalloc(ibp_case *c, const double *box_lo, const double *box_hi,
                             double *obj_lo, double *obj_hi, double *obj_err, void *cuda_stream);

/* Wait for the case's stream work and report device-side errors of the last
 * asynchronous call (IBP_EINVAL for a bad box, IBP_ETIMEOUT for a wait). */
ibp_status ibp_case_sync(ibp_case *c);

typedef struct {
    int32_t n_bus, n_line, n_ctg, n_gen, n_load;
    int32_t n_active;      /* buses with a device, slack excluded */
    int32_t n_active_pad;  /* row stride of the FP32 PTDF on the device */
    int32_t device;        /* -1 for a dry-run case */
    int64_t device_bytes;  /* device memory held by the case */
    double build_seconds;  /* wall time of the FP64 sensitivity build */
    double max_abs_lodf;   /* max |L| over the contingency list */
    int32_t n_bus_classes; /* columns of the reduced rows (see ibp_case_reduction) */
    int32_t n_bridges;     /* bridge lines (never contingencies) */
} ibp_case_info_t;

ibp_status ibp_case_info(const ibp_case *c, ibp_case_info_t *out);

/*
 * Kernel-shape selection for the contingency kernel (used by the autotuner).
 * variant: 0 = library default for the box count; other values select one of
 * the compiled tile shapes listed by ibp_kernel_variants().  Returns
 * IBP_EINVAL for an unknown variant.  A one-box variant applies to calls with
 * one box and a multi-box variant to calls with more (the other calls keep
 * the default).  ibp_bound_multi runs the multi-box body of the first case's
 * variant, or variant 29's body for 0 or an id without a many-case form: the
 * default multi-box variant of single-case calls, 30, is variant 29 with the
 * ring's stages waited for and released in pairs, which the many-case launch
 * does not use.
 */
ibp_status ibp_case_set_variant(ibp_case *c, int32_t variant);
int32_t ibp_kernel_variants(int32_t *ids, int32_t cap, int32_t batched);

/*
 * The objective interval with the paper's own contingency intervals (Sec.
 * II-C, eq. (ctg flow matrix form): [Phi p] and [U p] propagated separately,
 * so every contingency flow takes the radius R_l + |L[l,k]| R_k) in place of
 * the tight per-row radius of ibp_bound.  The result encloses ibp_bound's (it
 * is the bound of the paper's graph), costs O(n_ctg * n_line) instead of
 * O(n_ctg * n_line * n_active), and is certified the same way (outward FP32,
 * FP64 sums, obj_err as in ibp_bound).  A box whose paper-mode obj_hi is
 * already negative is certified welfare-negative without the tight pass.
 * Arguments, layouts, ptr_mode, stream and errors as in ibp_bound (no flows).
 */
ibp_status ibp_bound_paper(ibp_case *c, int32_t n_box, const double *box_lo,
                           const double *box_hi, double *obj_lo, double *obj_hi,
                           double *obj_err, int32_t ptr_mode, void *cuda_stream);

/*
 * Paper-mode line screen (Sec. II-C: the contingency flow of eq. (ctg flow
 * matrix form) propagated as the two intervals [Phi p] and [U p], radius
 * R_l + |L[l,k]| R_k, an upper bound of the tight radius).  When enabled (the
 * default), ibp_bound and ibp_bound_backward first drop every line whose
 * certified upper flow bound in that interval stays within its contingency
 * rating for all contingencies and boxes of the call: those pairs have a
 * violation interval of exactly [0, 0], so the result is unchanged up to the
 * rounding order of the sums (and stays certified); only the remaining lines
 * reach the contingency kernel.  Calls that ask for flow_lo/flow_hi and
 * ibp_bound_multi never screen.  enable: 0 disables, other values enable.
 *
 * ibp_case_last_live: *n_live = number of lines the last ibp_bound /
 * ibp_bound_backward call of this case kept, or -1 when that call did not
 * screen; lines (nullable, host, room for n_line) receives their indices in
 * ascending order.  Synchronises the device.  No counterpart in the paper
 * beyond the interval it uses.
 */
ibp_status ibp_case_set_screen(ibp_case *c, int32_t enable);
ibp_status ibp_case_last_live(ibp_case *c, int32_t *n_live, int32_t *lines);

/*
 * Exact network reduction of the contingency pass (enabled by default;
 * enable = 0 disables).  Two identities of the DC network, both exact in
 * exact arithmetic, shrink the n_c x n_l x n_a contraction behind
 * eq. (ctg flow simplified):
 *  - a bridge line carries the net injection of the side away from the slack,
 *    which no non-islanding outage changes (L[l,k] = 0), so all n_c pairs of a
 *    bridge share its base interval and are added in closed form;
 *  - removing the bridges leaves 2-edge-connected components; an injection
 *    enters each component through one vertex, so active buses that enter
 *    every component with inner lines through the same vertices have equal
 *    PTDF columns on every non-bridge line.  Such a class streams as one
 *    column whose radius is the rounded-up sum of its members' radii; the
 *    class of the slack has a zero column there and is dropped.
 * The result stays certified against the FP64 data (the column equalities
 * hold to the accuracy of the FP64 build); only the rounding of the sums
 * moves.  Calls that ask for flow_lo/flow_hi and ibp_bound_multi do not use
 * it.  ibp_case_reduction reports the partition: class_of_active[i] (host,
 * [n_active], nullable) is the class of active column i or -1 for the
 * slack's class; is_bridge[l] (host, [n_line], nullable) is 1 for bridges.
 * Works on dry-run cases.  No counterpart in the paper.
 */
ibp_status ibp_case_set_reduction(ibp_case *c, int32_t enable);

/*
 * FP64 refinement of the terms that can reach obj_hi (enabled by default;
 * enable = 0 disables).  obj_hi takes -zeta_f s_lo for every base line and
 * contingency pair, s_lo = max(|c| - r - rating, 0) (eqs. (slack-sfb),
 * (slack-Sc) under eq. (IBP)), and only the few terms whose lower violation
 * bound can be positive contribute.  With the refinement on, the FP32 kernels
 * leave those terms to one warp each, which recomputes the flow interval from
 * the FP64 PTDF (kept on the device as the FP32 copy plus its FP32 remainder,
 * about 4 bytes per line and active bus more) and the FP64 bus intervals with
 * FP64 sums and an explicit error bound.  The term keeps its certification
 * (a lower bound of the exact s_lo), and its share of obj_err falls from tens
 * of FP32 units of the flow's magnitude to FP64 rounding.  All bound entry
 * points (ibp_bound, ibp_bound_paper, ibp_bound_backward, ibp_bound_multi and
 * ibp_bound_noalloc) use it.  obj_lo is unaffected.  No counterpart in the
 * paper.
 */
ibp_status ibp_case_set_refine(ibp_case *c, int32_t enable);
ibp_status ibp_case_reduction(const ibp_case *c, int32_t *class_of_active, int32_t *is_bridge);

/*
 * Optional per-kernel timing of the last ibp_bound call, recorded with CUDA
 * events on the call's stream when enabled (0 disables).  ms[0..n) receives
 * {box_to_bus, base_flow, screen, contingency, refine, assemble} durations in
 * milliseconds (screen is the paper-mode line screen and the gather of the
 * kept rows, about 0 when the call does not screen; refine is the FP64
 * refinement of the queued pairs, see ibp_case_set_refine); the call
 * synchronises the stream.
 */
ibp_status ibp_case_set_timing(ibp_case *c, int32_t enable);
ibp_status ibp_case_last_timing(ibp_case *c, float *ms, int32_t n);

/* Allocation-failure hook for tests: from this call on, every device buffer
 * the library allocates that is larger than `bytes` fails as if the device
 * were out of memory (the call returns IBP_ENOMEM and leaves the case as it
 * was); 0 removes the limit.  Process-wide.  No counterpart in the paper. */
ibp_status ibp_set_alloc_limit(int64_t bytes);

/* Bounded-wait self test: launches one kernel that waits on an mbarrier that
 * no thread arrives at, with a limit of limit_us microseconds; returns
 * IBP_ETIMEOUT when the wait ran out and the kernel returned (expected), or
 * IBP_OK / IBP_ECUDA otherwise. */
ibp_status ibp_selftest_wait_timeout(int32_t device, int32_t limit_us);

const char *ibp_last_error(void);
const char *ibp_status_string(ibp_status s);

#ifdef __cplusplus
}
#endif

#endif /* IBP_GB300_H */
