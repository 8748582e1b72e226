/*
 * Plain FP64 oracle for the contingency terms of the IBP objective bound.
 *
 * TEST INFRASTRUCTURE ONLY: this file, and everything under oracle/, may be
 * loaded by the tests, by the smoke check and by the CPU-baseline leg of the
 * benchmark, never by the library's product path.  It shares no code with the
 * CUDA library.
 *
 * What it computes, straight from the definitions, with no blocking, fusion
 * or factorisation:
 *   - the contingency flow of line l after the outage of line k is
 *       p_{f,c}^k[l] = sum_b H_k[l,b] p_inj[b],   H_k = Phi + L[:,k] Phi[k,:]
 *     (Sec. II-C, eq. (ctg flow simplified); L is the line outage
 *     distribution factor matrix, L[k,k] = -1 zeroes the outaged line like M_k);
 *   - IBP of that affine map over the bus-injection box, eq. (IBP):
 *       centre c_kl = sum_b H_k[l,b] c_b,  radius r_kl = sum_b |H_k[l,b]| r_b,
 *     summed over every bus b;
 *   - the violation interval of eq. (slack-Sc): |x| on [c-r, c+r], then
 *     max(. - rating_l, 0), and its sum over all (k,l), eq. (slack-sagg);
 *   - the hand-derived adjoint of sum_{k,l} s_lo[k,l] with respect to the bus
 *     centre c_b and radius r_b (the lower violation bound enters the upper
 *     objective bound).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no fused multiply-add
 * so that x86 and Arm hosts give the same bits).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Interval of |x| for x in [lo, hi], then max(. - rating, 0): eq. (slack-sfb)
 * and eq. (slack-Sc) under the monotone-activation rule of eq. (IBP). */
static void viol_interval(double lo, double hi, double rating, double *s_lo, double *s_hi)
{
    double alo, ahi;
    if (lo >= 0.0) {
        alo = lo;
        ahi = hi;
    } else if (hi <= 0.0) {
        alo = -hi;
        ahi = -lo;
    } else {
        alo = 0.0;
        ahi = (-lo > hi) ? -lo : hi;
    }
    double a = alo - rating, b = ahi - rating;
    *s_lo = a > 0.0 ? a : 0.0;
    *s_hi = b > 0.0 ? b : 0.0;
}

void orc_viol_interval(double lo, double hi, double rating, double *s_lo, double *s_hi)
{
    viol_interval(lo, hi, rating, s_lo, s_hi);
}

/* Centre and radius of H_k[l,:] p over the box, by the plain sum over buses. */
static void flow_interval(int nb, const double *phi_l, const double *phi_k, double lkl,
                          const double *c, const double *r, double *cent, double *rad)
{
    double sc = 0.0, sr = 0.0;
    for (int b = 0; b < nb; ++b) {
        double h = phi_l[b] + lkl * phi_k[b];
        sc += h * c[b];
        sr += fabs(h) * r[b];
    }
    *cent = sc;
    *rad = sr;
}

/*
 * Sum over all contingencies k and lines l of the violation interval bounds.
 *   phi      [nl][nb]  PTDF with a zero slack column
 *   lodf     [nl][nc]  L[l][k]
 *   ctg_line [nc]      outaged line of contingency k
 *   rating   [nl]      contingency rating p^max_{f,c}
 *   cbus, rbus [nbox][nb]  bus injection centre and radius
 * Outputs per box: s_lo_sum, s_hi_sum; optionally g_c, g_r [nbox][nb] =
 * d(sum s_lo)/dc_b and d(sum s_lo)/dr_b, and n_active = #{(k,l): s_lo > 0}.
 */
int orc_ctg_terms(int nb, int nl, int nc, const double *phi, const double *lodf,
                  const int32_t *ctg_line, const double *rating, int nbox,
                  const double *cbus, const double *rbus, double *s_lo_sum,
                  double *s_hi_sum, double *g_c, double *g_r, int64_t *n_active,
                  int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#endif
    for (int j = 0; j < nbox; ++j) {
        const double *c = cbus + (size_t)j * nb;
        const double *r = rbus + (size_t)j * nb;
        double tot_lo = 0.0, tot_hi = 0.0;
        int64_t act = 0;
        int want_grad = (g_c != NULL && g_r != NULL);
        if (want_grad) {
            memset(g_c + (size_t)j * nb, 0, sizeof(double) * nb);
            memset(g_r + (size_t)j * nb, 0, sizeof(double) * nb);
        }
#pragma omp parallel reduction(+ : tot_lo, tot_hi, act)
        {
            double *lgc = NULL, *lgr = NULL;
            if (want_grad) {
                lgc = (double *)calloc((size_t)nb, sizeof(double));
                lgr = (double *)calloc((size_t)nb, sizeof(double));
            }
#pragma omp for schedule(dynamic, 4)
            for (int k = 0; k < nc; ++k) {
                const double *phi_k = phi + (size_t)ctg_line[k] * nb;
                for (int l = 0; l < nl; ++l) {
                    const double *phi_l = phi + (size_t)l * nb;
                    double lkl = lodf[(size_t)l * nc + k];
                    double cent, rad, slo, shi;
                    flow_interval(nb, phi_l, phi_k, lkl, c, r, &cent, &rad);
                    viol_interval(cent - rad, cent + rad, rating[l], &slo, &shi);
                    tot_lo += slo;
                    tot_hi += shi;
                    if (slo > 0.0) {
                        act += 1;
                        if (want_grad) {
                            double sg = cent > 0.0 ? 1.0 : -1.0;
                            for (int b = 0; b < nb; ++b) {
                                double h = phi_l[b] + lkl * phi_k[b];
                                lgc[b] += sg * h;
                                lgr[b] -= fabs(h);
                            }
                        }
                    }
                }
            }
            if (want_grad) {
#pragma omp critical
                {
                    for (int b = 0; b < nb; ++b) {
                        g_c[(size_t)j * nb + b] += lgc[b];
                        g_r[(size_t)j * nb + b] += lgr[b];
                    }
                }
                free(lgc);
                free(lgr);
            }
        }
        s_lo_sum[j] = tot_lo;
        s_hi_sum[j] = tot_hi;
        if (n_active)
            n_active[j] = act;
    }
    return 0;
}

/* Flow intervals (centre, radius) of sampled (k,l) pairs, per box:
 * cent/rad [nbox][npair]. */
int orc_ctg_flows(int nb, int nl, int nc, const double *phi, const double *lodf,
                  const int32_t *ctg_line, int nbox, const double *cbus,
                  const double *rbus, int64_t npair, const int32_t *pk,
                  const int32_t *pl, double *cent, double *rad, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#endif
    (void)nl;
    for (int j = 0; j < nbox; ++j) {
        const double *c = cbus + (size_t)j * nb;
        const double *r = rbus + (size_t)j * nb;
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < npair; ++p) {
            int k = pk[p], l = pl[p];
            const double *phi_k = phi + (size_t)ctg_line[k] * nb;
            const double *phi_l = phi + (size_t)l * nb;
            flow_interval(nb, phi_l, phi_k, lodf[(size_t)l * nc + k], c, r,
                          &cent[(size_t)j * npair + p], &rad[(size_t)j * npair + p]);
        }
    }
    return 0;
}
