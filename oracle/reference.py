"""Plain FP64 CPU oracle of the IBP bound on the soft-constrained SC-DCOPF objective.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
leg of the benchmark import this module; the library's product path never does.
It shares no code with the CUDA library: it builds its own PTDF (LU with
partial pivoting through ``numpy.linalg.solve``; the library uses its own
Cholesky), its own LODF, and sums every contingency flow over every bus by the
plain definition (``libibp_oracle.so``).

Every function names the passage of the paper it follows:

* ``ptdf``                Sec. II-A, eq. (line flow ptdf): Phi = [0  Y_D E_r (E_r^T Y_D E_r)^-1]
* ``lodf``                Sec. II-C, eq. (ctg flow simplified) rewritten with line outage
                          distribution factors; ``paper_ctg_matrices`` builds the
                          literal u_i, g_i, B, U, M of Sec. II-C / eq. (ctg flow matrix form)
* ``bus_box``             p_inj = N_g p_g - N_d p_d (Sec. II-A) under eq. (IBP)
* ``cost_interval``       Sec. III-B, eqs. (single ReLU), (combined ReLUs) under eq. (IBP)
* ``imbalance_interval``  eq. (slack-sinj) through the explicit matrix E^T Phi - I
* ``base_terms``          eq. (slack-sfb)
* ``ctg_terms``           eqs. (slack-Sc), (slack-sagg)
* ``bound``               eq. (penalized-objective) / appendix eq. (ibp_f) under eq. (IBP)
* ``grad_hi``             hand-derived adjoint of the upper bound (the paper has none)
* ``grad_hi_ratings``     its rating part, split into base and contingency ratings
* ``grad_lo``             hand-derived adjoint of the lower bound (the paper has none)
* ``linear_bound``        the linear (CROWN-style) relaxation bound at given slopes (the paper has none)
* ``paper_mode_flows``    IBP applied literally to eq. (ctg flow matrix form)
* ``screen_lines``        lines whose paper-mode contingency interval can exceed the rating
* ``paper_ctg_terms``     eq. (slack-Sc) sums over the paper-mode intervals (``bound(mode="paper")``)
* ``objective_point``     f_ibp at a point, appendix eq. (ibp_f)

Parity pins: every function above is checked in ``tests/test_oracle_*.py``
against something other than itself (Kirchhoff's laws, re-solving the outaged
network, vertex enumeration, an LP solver, finite differences).  The paper's
reported optimality gaps on the GO3 instances are not reproducible without
that data: that comparison is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional

import numpy as np

from .build import build_oracle

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = build_oracle()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        lib.orc_ctg_terms.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P, P,
                                      ctypes.c_int, P, P, P, P, P, P, P, ctypes.c_int]
        lib.orc_ctg_terms.restype = ctypes.c_int
        lib.orc_ctg_flows.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P,
                                      ctypes.c_int, P, P, ctypes.c_int64, P, P, P, P,
                                      ctypes.c_int]
        lib.orc_ctg_flows.restype = ctypes.c_int
        lib.orc_viol_interval.argtypes = [ctypes.c_double] * 3 + [P, P]
        lib.orc_viol_interval.restype = None
        _LIB = lib
    return _LIB


def _p(a: Optional[np.ndarray]):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _nthreads(n):
    if n is not None:
        return int(n)
    return int(os.environ.get("IBP_ORACLE_THREADS", "0"))


# ----------------------------------------------------------------------------
# Sensitivities (Sec. II-A, II-C)
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Sensitivities:
    phi: np.ndarray        # [n_line, n_bus], zero slack column
    lodf: np.ndarray       # [n_line, n_ctg], L[l, k]
    ptdf_kk: np.ndarray    # [n_ctg], PTDF of each outaged line w.r.t. its own transfer


def incidence(case) -> np.ndarray:
    """E in R^{n_l x n_b}: +1 at the from bus, -1 at the to bus (reading C1)."""
    E = np.zeros((case.n_line, case.n_bus))
    idx = np.arange(case.n_line)
    E[idx, case.line_from] = 1.0
    E[idx, case.line_to] = -1.0
    return E


def reduced_admittance(case) -> np.ndarray:
    """Y_B,r = E_r^T Y_D E_r with the slack row/column removed, Y_D = diag(1/x)."""
    b = 1.0 / case.reactance
    Y = np.zeros((case.n_bus, case.n_bus))
    fr, to = case.line_from, case.line_to
    np.add.at(Y, (fr, fr), b)
    np.add.at(Y, (to, to), b)
    np.add.at(Y, (fr, to), -b)
    np.add.at(Y, (to, fr), -b)
    keep = np.array([i for i in range(case.n_bus) if i != case.slack])
    return Y[np.ix_(keep, keep)], keep


def ptdf(case) -> np.ndarray:
    """Eq. (line flow ptdf): Phi_r = Y_D E_r (E_r^T Y_D E_r)^-1, zero slack column.

    Phi_r^T = Y_B,r^-1 (E_r^T Y_D) because Y_B,r is symmetric; one dense LU
    solve (partial pivoting) with n_l right-hand sides.
    """
    Yr, keep = reduced_admittance(case)
    b = 1.0 / case.reactance
    rhs = np.zeros((keep.size, case.n_line))
    pos = -np.ones(case.n_bus, dtype=np.int64)
    pos[keep] = np.arange(keep.size)
    for l in range(case.n_line):
        i, j = pos[case.line_from[l]], pos[case.line_to[l]]
        if i >= 0:
            rhs[i, l] += b[l]
        if j >= 0:
            rhs[j, l] -= b[l]
    Z = np.linalg.solve(Yr, rhs)
    phi = np.zeros((case.n_line, case.n_bus))
    phi[:, keep] = Z.T
    return phi


class IslandingContingency(ValueError):
    pass


def lodf(case, phi: np.ndarray, tol: float = 1e-9):
    """Line outage distribution factors of the contingency list.

    PTDF_line[l,k] = Phi[l, from_k] - Phi[l, to_k] is the flow on l per unit
    transfer from the from-bus to the to-bus of outaged line k; the post-outage
    flow is f_l + L[l,k] f_k with L[l,k] = PTDF_line[l,k] / (1 - PTDF_line[k,k])
    and L[k,k] = -1 (the outaged line carries nothing, like M_k in Sec. II-C).
    A contingency with 1 - PTDF_line[k,k] ~ 0 islands the network (the
    Sherman-Morrison denominator 1 + e_i^T u_i y_i vanishes) and is rejected.
    """
    ks = case.ctg_line
    ptl = phi[:, case.line_from[ks]] - phi[:, case.line_to[ks]]  # [n_l, n_c]
    kk = ptl[ks, np.arange(ks.size)]
    den = 1.0 - kk
    if np.any(np.abs(den) < tol):
        raise IslandingContingency("contingency islands the network")
    L = np.ascontiguousarray(ptl / den[None, :])
    L[ks, np.arange(ks.size)] = -1.0
    return L, kk


def sensitivities(case) -> Sensitivities:
    phi = np.ascontiguousarray(ptdf(case))
    L, kk = lodf(case, phi)
    return Sensitivities(phi=phi, lodf=L, ptdf_kk=kk)


def paper_ctg_matrices(case):
    """The literal pre-processing of Sec. II-C and eq. (ctg flow matrix form).

    u_i = Y_B,r^-1 e_i (e_i: i-th row of E_r), y_i = -(Y_D)_ii,
    g_i = y_i / (1 + e_i^T u_i y_i), b_i = M_i Y_D E_r u_i g_i,
    U rows u'_i = u_i padded with the slack entry, M rows all ones but the
    outaged line.  Returns (M, B, U).
    """
    Yr, keep = reduced_admittance(case)
    E = incidence(case)
    Er = E[:, keep]
    Yd = 1.0 / case.reactance
    ks = case.ctg_line
    nc = ks.size
    ei = Er[ks, :].T                    # [n_b-1, n_c]
    u = np.linalg.solve(Yr, ei)         # u_i columns
    y = -Yd[ks]
    g = y / (1.0 + np.einsum("ij,ij->j", ei, u) * y)
    M = np.ones((nc, case.n_line))
    M[np.arange(nc), ks] = 0.0
    Bm = (Yd[:, None] * (Er @ u)) * g[None, :]   # [n_l, n_c] = Y_D E_r u_i g_i
    Bm = Bm.T * M                                 # rows b_i^T with M_i applied
    U = np.zeros((nc, case.n_bus))
    U[:, keep] = u.T
    return M, Bm, U


def outage_ptdf(case, k_line: int) -> np.ndarray:
    """PTDF of the network with line ``k_line`` removed, re-solved from scratch
    (the brute-force definition of eq. (ctg flow computation)); row k_line = 0."""
    keep_lines = np.array([l for l in range(case.n_line) if l != k_line])
    sub = dataclasses.replace(case, line_from=case.line_from[keep_lines],
                              line_to=case.line_to[keep_lines],
                              reactance=case.reactance[keep_lines],
                              rating=case.rating[keep_lines],
                              ctg_line=np.zeros(0, np.int32))
    p = ptdf(sub)
    out = np.zeros((case.n_line, case.n_bus))
    out[keep_lines] = p
    return out


# ----------------------------------------------------------------------------
# IBP of the objective (Sec. III, appendix)
# ----------------------------------------------------------------------------

def bus_box(case, lo: np.ndarray, hi: np.ndarray):
    """IBP of p_inj = N_g p_g - N_d p_d, eq. (IBP) with W = [N_g, -N_d]:
    c = W x_mu, r = |W| x_sigma (each device sits on one bus)."""
    lo = np.atleast_2d(lo)
    hi = np.atleast_2d(hi)
    mu = 0.5 * (lo + hi)
    sg = 0.5 * (hi - lo)
    nb = lo.shape[0]
    ng = case.n_gen
    W = np.zeros((case.n_bus, case.n_dev))
    W[case.gen_bus, np.arange(ng)] = 1.0
    W[case.load_bus, ng + np.arange(case.n_load)] = -1.0
    c = mu @ W.T
    r = sg @ np.abs(W).T
    assert c.shape == (nb, case.n_bus)
    return c, r


def _segments(nseg, slope, bkpt):
    ptr = np.concatenate([[0], np.cumsum(nseg)])
    return [(slope[ptr[i]:ptr[i + 1]], bkpt[ptr[i]:ptr[i + 1]]) for i in range(len(nseg))]


def relu_chain_interval(a, b, x_lo, x_hi):
    """IBP through F_i(x) = a_i ReLU(x - b_i), F*_i = min(F*_{i-1} + F_i, U_i),
    eqs. (single ReLU), (combined ReLUs), with U_i the cumulative value at the
    end of segment i (last U = +inf), reading C7.  Each step is monotone
    non-decreasing for a_i >= 0, so eq. (IBP) maps lower to lower and upper to upper.
    """
    n = len(a)
    U = np.empty(n)
    acc = 0.0
    for i in range(n):
        if i + 1 < n:
            acc += a[i] * (b[i + 1] - b[i])
            U[i] = acc
        else:
            U[i] = np.inf
    f_lo, f_hi = 0.0, 0.0
    for i in range(n):
        fl = a[i] * max(x_lo - b[i], 0.0)
        fh = a[i] * max(x_hi - b[i], 0.0)
        f_lo = min(f_lo + fl, U[i])
        f_hi = min(f_hi + fh, U[i])
    return f_lo, f_hi


def cost_interval(case, lo: np.ndarray, hi: np.ndarray):
    """[sum_j c_j(p_d)] and [sum_i g_i(p_g)] intervals over one box."""
    ng = case.n_gen
    G_lo = G_hi = 0.0
    for i, (a, b) in enumerate(_segments(case.gen_nseg, case.gen_slope, case.gen_bkpt)):
        fl, fh = relu_chain_interval(a, b, lo[i], hi[i])
        G_lo += fl
        G_hi += fh
    C_lo = C_hi = 0.0
    for j, (a, b) in enumerate(_segments(case.load_nseg, case.load_slope, case.load_bkpt)):
        fl, fh = relu_chain_interval(a, b, lo[ng + j], hi[ng + j])
        C_lo += fl
        C_hi += fh
    return C_lo, C_hi, G_lo, G_hi


def viol_interval(lo, hi, rating):
    """|x| over [lo, hi] then max(. - rating, 0), vectorised (eq. (slack-sfb))."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    alo = np.where(lo >= 0, lo, np.where(hi <= 0, -hi, 0.0))
    ahi = np.maximum(np.abs(lo), np.abs(hi))
    return np.maximum(alo - rating, 0.0), np.maximum(ahi - rating, 0.0)


def imbalance_matrix(case, phi) -> np.ndarray:
    """W = E^T Phi - I of eq. (slack-sinj), built row by row from the lines."""
    try:
        import scipy.sparse as sp
        rows = np.concatenate([case.line_from, case.line_to])
        cols = np.concatenate([np.arange(case.n_line), np.arange(case.n_line)])
        vals = np.concatenate([np.ones(case.n_line), -np.ones(case.n_line)])
        Et = sp.csr_matrix((vals, (rows, cols)), shape=(case.n_bus, case.n_line))
        W = np.asarray(Et @ phi)
    except ImportError:
        W = incidence(case).T @ phi
    W[np.arange(case.n_bus), np.arange(case.n_bus)] -= 1.0
    return W


def imbalance_interval(case, phi, c, r, W=None):
    """IBP of 1^T |W p_inj| (eq. (slack-sinj)); returns (sum lo, sum hi) per box."""
    if W is None:
        W = imbalance_matrix(case, phi)
    cc = c @ W.T
    rr = r @ np.abs(W).T
    s_lo, s_hi = viol_interval(cc - rr, cc + rr, 0.0)
    return s_lo.sum(axis=1), s_hi.sum(axis=1)


def base_terms(case, phi, c, r):
    """Base flows Phi p_inj under eq. (IBP), then eq. (slack-sfb), summed."""
    fc = c @ phi.T
    fr = r @ np.abs(phi).T
    s_lo, s_hi = viol_interval(fc - fr, fc + fr, case.rating[None, :])
    return s_lo.sum(axis=1), s_hi.sum(axis=1), fc, fr


def ctg_terms(case, sens: Sensitivities, c, r, grad=False, nthreads=None):
    rating_c = case.rating if case.rating_ctg is None else case.rating_ctg
    nbox = c.shape[0]
    c = np.ascontiguousarray(c, np.float64)
    r = np.ascontiguousarray(r, np.float64)
    phi = np.ascontiguousarray(sens.phi)
    L = np.ascontiguousarray(sens.lodf)
    ctg = np.ascontiguousarray(case.ctg_line, np.int32)
    rc = np.ascontiguousarray(rating_c, np.float64)
    s_lo = np.zeros(nbox)
    s_hi = np.zeros(nbox)
    act = np.zeros(nbox, np.int64)
    gc = np.zeros((nbox, case.n_bus)) if grad else None
    gr = np.zeros((nbox, case.n_bus)) if grad else None
    _lib().orc_ctg_terms(case.n_bus, case.n_line, case.n_ctg, _p(phi), _p(L), _p(ctg),
                         _p(rc), nbox, _p(c), _p(r), _p(s_lo), _p(s_hi), _p(gc), _p(gr),
                         _p(act), _nthreads(nthreads))
    return s_lo, s_hi, act, gc, gr


def ctg_flows(case, sens: Sensitivities, c, r, pk, pl, nthreads=None):
    """Centre and radius of sampled contingency flows (k = pk[i], l = pl[i])."""
    nbox = c.shape[0]
    # every array handed to C is bound to a local name so that it outlives the call
    pk = np.ascontiguousarray(pk, np.int32)
    pl = np.ascontiguousarray(pl, np.int32)
    phi = np.ascontiguousarray(sens.phi, np.float64)
    L = np.ascontiguousarray(sens.lodf, np.float64)
    ctg = np.ascontiguousarray(case.ctg_line, np.int32)
    c = np.ascontiguousarray(c, np.float64)
    r = np.ascontiguousarray(r, np.float64)
    if pk.size and (pk.min() < 0 or pk.max() >= case.n_ctg or pl.min() < 0 or pl.max() >= case.n_line):
        raise IndexError("pair index out of range")
    cent = np.zeros((nbox, pk.size))
    rad = np.zeros((nbox, pk.size))
    _lib().orc_ctg_flows(case.n_bus, case.n_line, case.n_ctg, _p(phi), _p(L), _p(ctg), nbox,
                         _p(c), _p(r), pk.size, _p(pk), _p(pl), _p(cent), _p(rad),
                         _nthreads(nthreads))
    return cent, rad


def all_ctg_flows(case, sens, c, r, nthreads=None):
    """Every contingency flow interval, [nbox, n_ctg, n_line] (small cases)."""
    kk, ll = np.meshgrid(np.arange(case.n_ctg), np.arange(case.n_line), indexing="ij")
    cent, rad = ctg_flows(case, sens, c, r, kk.ravel(), ll.ravel(), nthreads)
    shp = (c.shape[0], case.n_ctg, case.n_line)
    return cent.reshape(shp), rad.reshape(shp)


@dataclasses.dataclass
class Bound:
    lo: np.ndarray
    hi: np.ndarray
    terms: dict


def paper_ctg_terms(case, sens: Sensitivities, c, r):
    """Sums of the contingency violation intervals of eq. (slack-Sc) when the
    contingency flows take the paper-mode interval (``paper_mode_flows``)."""
    rating = case.rating if case.rating_ctg is None else case.rating_ctg
    cent, rad = paper_mode_flows(case, sens, c, r)
    v_lo, v_hi = viol_interval(cent - rad, cent + rad, rating[None, None, :])
    return v_lo.sum(axis=(1, 2)), v_hi.sum(axis=(1, 2))


def bound(case, sens: Optional[Sensitivities] = None, lo=None, hi=None, nthreads=None,
          W=None, mode: str = "tight") -> Bound:
    """IBP bound of f_ibp over each box (appendix eq. (ibp_f), eq. (penalized-objective)).

    hi = C_hi - G_lo - z_inj S_inj,lo - z_f (S_fb,lo + S_fc,lo)
    lo = C_lo - G_hi - z_inj S_inj,hi - z_f (S_fb,hi + S_fc,hi)

    mode "tight": every contingency flow by the per-row rule (reading C9);
    mode "paper": the paper's two-part interval of eq. (ctg flow matrix form).
    """
    if sens is None:
        sens = sensitivities(case)
    lo = case.box_lo if lo is None else np.atleast_2d(lo)
    hi = case.box_hi if hi is None else np.atleast_2d(hi)
    c, r = bus_box(case, lo, hi)
    inj_lo, inj_hi = imbalance_interval(case, sens.phi, c, r, W)
    fb_lo, fb_hi, _, _ = base_terms(case, sens.phi, c, r)
    if mode == "paper":
        fc_lo, fc_hi = paper_ctg_terms(case, sens, c, r)
    else:
        fc_lo, fc_hi, _, _, _ = ctg_terms(case, sens, c, r, nthreads=nthreads)
    nbox = lo.shape[0]
    out_lo = np.empty(nbox)
    out_hi = np.empty(nbox)
    costs = []
    for j in range(nbox):
        C_lo, C_hi, G_lo, G_hi = cost_interval(case, lo[j], hi[j])
        costs.append((C_lo, C_hi, G_lo, G_hi))
        out_hi[j] = C_hi - G_lo - case.zeta_inj * inj_lo[j] - case.zeta_f * (fb_lo[j] + fc_lo[j])
        out_lo[j] = C_lo - G_hi - case.zeta_inj * inj_hi[j] - case.zeta_f * (fb_hi[j] + fc_hi[j])
    return Bound(lo=out_lo, hi=out_hi,
                 terms=dict(costs=np.array(costs), inj=(inj_lo, inj_hi), fb=(fb_lo, fb_hi),
                            fc=(fc_lo, fc_hi), zeta=(case.zeta_inj, case.zeta_f)))


# ----------------------------------------------------------------------------
# Point evaluation and the hand adjoint
# ----------------------------------------------------------------------------

def pwl_value(a, b, x):
    """Value of the ReLU-chain PWL at a point (lower = upper endpoint)."""
    return relu_chain_interval(a, b, x, x)[0]


def objective_point(case, sens: Sensitivities, x: np.ndarray) -> float:
    """f_ibp(p_d, p_g) of appendix eq. (ibp_f) at one point x = [p_g, p_d]."""
    x = np.asarray(x, np.float64)
    ng = case.n_gen
    c, _ = bus_box(case, x[None, :], x[None, :])
    p = c[0]
    f = sens.phi @ p
    s_inj = np.abs(imbalance_matrix(case, sens.phi) @ p).sum()
    s_fb = np.maximum(np.abs(f) - case.rating, 0.0).sum()
    rating_c = case.rating if case.rating_ctg is None else case.rating_ctg
    P = f[None, :] + sens.lodf.T * f[case.ctg_line][:, None]      # [n_c, n_l]
    s_fc = np.maximum(np.abs(P) - rating_c[None, :], 0.0).sum()
    C = sum(pwl_value(a, b, x[ng + j]) for j, (a, b) in
            enumerate(_segments(case.load_nseg, case.load_slope, case.load_bkpt)))
    G = sum(pwl_value(a, b, x[i]) for i, (a, b) in
            enumerate(_segments(case.gen_nseg, case.gen_slope, case.gen_bkpt)))
    return C - G - case.zeta_inj * s_inj - case.zeta_f * (s_fb + s_fc)


def _pwl_slope(a, b, x):
    """Slope of the PWL at x (segment containing x; right segment at a breakpoint)."""
    i = int(np.searchsorted(b, x, side="right")) - 1
    return float(a[max(i, 0)]) if x >= b[0] else 0.0


def grad_hi(case, sens: Sensitivities, lo=None, hi=None, nthreads=None):
    """Hand adjoint of the upper bound: d hi / d box_lo, d hi / d box_hi, d hi / d rating.

    With A = {(k,l): |c_kl| - r_kl > rating_l} (and the same test on the base
    flows), d hi/dc_b = -z_f sum_A sgn(c_kl) H_k[l,b] - z_inj sgn(sum c)[s_inj active],
    d hi/dr_b = +z_f sum_A |H_k[l,b]| + z_inj [s_inj active], then the chain
    rule through c = N mu, r = |N| sigma and the cost slopes at the endpoints.
    Valid away from kinks (no tie in any max or |.|).
    """
    lo = case.box_lo if lo is None else np.atleast_2d(lo)
    hi = case.box_hi if hi is None else np.atleast_2d(hi)
    c, r = bus_box(case, lo, hi)
    nbox = lo.shape[0]
    phi = sens.phi
    # contingency part
    _, _, _, gc_c, gr_c = ctg_terms(case, sens, c, r, grad=True, nthreads=nthreads)
    # base part
    fc = c @ phi.T
    fr = r @ np.abs(phi).T
    act_b = (np.abs(fc) - fr - case.rating[None, :]) > 0
    sg_b = np.sign(fc) * act_b
    gc_b = sg_b @ phi
    gr_b = -(act_b.astype(float) @ np.abs(phi))
    # imbalance part (closed form of the explicit matrix: the slack row is -1^T)
    tot_c = c.sum(axis=1)
    tot_r = r.sum(axis=1)
    act_i = (np.abs(tot_c) - tot_r) > 0
    gc_i = (np.sign(tot_c) * act_i)[:, None] * np.ones((1, case.n_bus))
    gr_i = -(act_i.astype(float))[:, None] * np.ones((1, case.n_bus))
    # d hi / d c, d hi / d r
    dc = -case.zeta_f * (gc_c + gc_b) - case.zeta_inj * gc_i
    dr = -case.zeta_f * (gr_c + gr_b) - case.zeta_inj * gr_i
    # rating gradient for base and contingency ratings moving together
    g_rating = None
    if case.n_ctg * case.n_line <= 4_000_000:
        g_base, g_ctg = grad_hi_ratings(case, sens, lo, hi, nthreads)
        g_rating = g_base + g_ctg
    # chain to device endpoints
    ng = case.n_gen
    bus = np.concatenate([case.gen_bus, case.load_bus])
    sgn = np.concatenate([np.ones(ng), -np.ones(case.n_load)])
    g_lo = 0.5 * sgn[None, :] * dc[:, bus] - 0.5 * dr[:, bus]
    g_hi = 0.5 * sgn[None, :] * dc[:, bus] + 0.5 * dr[:, bus]
    for j in range(nbox):
        for i, (a, b) in enumerate(_segments(case.gen_nseg, case.gen_slope, case.gen_bkpt)):
            g_lo[j, i] -= _pwl_slope(a, b, lo[j, i])
        for d, (a, b) in enumerate(_segments(case.load_nseg, case.load_slope, case.load_bkpt)):
            g_hi[j, ng + d] += _pwl_slope(a, b, hi[j, ng + d])
    return g_lo, g_hi, g_rating


def grad_lo(case, sens: Sensitivities, lo=None, hi=None, nthreads=None):
    """Hand adjoint of the lower bound: d lo / d box_lo, d lo / d box_hi, d lo / d rating.

    lo = C_lo - G_hi - z_inj S_inj,hi - z_f (S_fb,hi + S_fc,hi) with
    s_hi = max(|c| + r - rating, 0) for every base line and (k, l) pair (the
    upper end of |x| over [c - r, c + r], eqs. (slack-sfb), (slack-Sc) under
    eq. (IBP)) and S_inj,hi = |sum c| + sum r (eq. (slack-sinj), reading C5).
    With A = {pairs: |c| + r - rating > 0}:
      d lo/dc_b = -z_f sum_A sgn(c) H[b] - z_inj sgn(sum c),
      d lo/dr_b = -z_f sum_A |H[b]| - z_inj,
      d lo/d rating_l = +z_f #{pairs of A on line l} (shared base and
        contingency rating; None for cases too large to form every flow),
    then the chain rule through c = N mu, r = |N| sigma; the load values enter
    at box_lo, the generator costs at box_hi.  Valid away from kinks.
    """
    lo = case.box_lo if lo is None else np.atleast_2d(lo)
    hi = case.box_hi if hi is None else np.atleast_2d(hi)
    c, r = bus_box(case, lo, hi)
    nbox = lo.shape[0]
    phi = sens.phi
    rating_c = case.rating if case.rating_ctg is None else case.rating_ctg
    cent, rad = all_ctg_flows(case, sens, c, r, nthreads)          # [nbox, n_c, n_l]
    act_c = (np.abs(cent) + rad - rating_c[None, None, :]) > 0
    H_sum_c = np.zeros((nbox, case.n_bus))
    H_sum_r = np.zeros((nbox, case.n_bus))
    for k in range(case.n_ctg):
        kl = case.ctg_line[k]
        Hk = phi + np.outer(sens.lodf[:, k], phi[kl])               # [n_l, n_b]
        for j in range(nbox):
            a = act_c[j, k]
            H_sum_c[j] += (np.sign(cent[j, k]) * a) @ Hk
            H_sum_r[j] += a.astype(float) @ np.abs(Hk)
    fc = c @ phi.T
    fr = r @ np.abs(phi).T
    act_b = (np.abs(fc) + fr - case.rating[None, :]) > 0
    gc_b = (np.sign(fc) * act_b) @ phi
    gr_b = act_b.astype(float) @ np.abs(phi)
    tot_c = c.sum(axis=1)
    dc = -case.zeta_f * (H_sum_c + gc_b) - case.zeta_inj * np.sign(tot_c)[:, None]
    dr = -case.zeta_f * (H_sum_r + gr_b) - case.zeta_inj
    g_rating = case.zeta_f * (act_c.sum(axis=1) + act_b)
    ng = case.n_gen
    bus = np.concatenate([case.gen_bus, case.load_bus])
    sgn = np.concatenate([np.ones(ng), -np.ones(case.n_load)])
    g_lo = 0.5 * sgn[None, :] * dc[:, bus] - 0.5 * dr[:, bus]
    g_hi = 0.5 * sgn[None, :] * dc[:, bus] + 0.5 * dr[:, bus]
    for j in range(nbox):
        for i, (a, b) in enumerate(_segments(case.gen_nseg, case.gen_slope, case.gen_bkpt)):
            g_hi[j, i] -= _pwl_slope(a, b, hi[j, i])
        for d, (a, b) in enumerate(_segments(case.load_nseg, case.load_slope, case.load_bkpt)):
            g_lo[j, ng + d] += _pwl_slope(a, b, lo[j, ng + d])
    return g_lo, g_hi, g_rating


def linear_bound(case, sens: Sensitivities, lo, hi, a_base, a_ctg, a_inj, factored: bool = False):
    """The linear relaxation bound U(a) = max over the box of l_a (the dual
    function of the LP whose optimum is max f).

    For slopes a in [-1, 1] every penalty term has a linear lower bound,
    max(|y| - R, 0) >= a y - |a| R (base flows y = f_l with the base rating,
    contingency flows y = f_kl with the contingency rating, eqs. (slack-sfb),
    (slack-Sc)) and |1^T p| >= a_inj 1^T p (eq. (slack-sinj), reading C5), so
      f(x) <= l_a(x) = C(p_d) - G(p_g) - z_inj a_inj 1^T p
                       - z_f (sum_t a_t y_t(x) - |a_t| R_t)
    on the box (appendix eq. (ibp_f)).  l_a is a sum of one-device functions,
    so its maximum is taken device by device over the endpoints and the
    breakpoints of the device's PWL curve inside its interval.
    a_base [n_line], a_ctg [n_ctg, n_line], a_inj a scalar; lo, hi one box.
    The slope of x_i in sum_t a_t y_t is s_i sum_t a_t H_t[b(i)] with H_t the
    flow's row (Phi_l, or Phi_l + L[l,k] Phi_k); factored=False forms every
    H_k, factored=True uses sum_t a_t H_t = Phi^T w with w_l = a_l + sum_k a_kl,
    w_{line of k} += sum_l a_kl L[l,k] (the same sum regrouped).
    """
    lo = np.asarray(lo, np.float64).ravel()
    hi = np.asarray(hi, np.float64).ravel()
    a_base = np.asarray(a_base, np.float64)
    a_ctg = np.asarray(a_ctg, np.float64).reshape(case.n_ctg, case.n_line)
    phi, L = sens.phi, sens.lodf
    rating_c = case.rating if case.rating_ctg is None else case.rating_ctg
    if factored:
        w = a_base + a_ctg.sum(axis=0)
        np.add.at(w, case.ctg_line, (a_ctg * L.T).sum(axis=1))
        row = w @ phi
    else:
        row = a_base @ phi
        for k in range(case.n_ctg):
            Hk = phi + np.outer(L[:, k], phi[case.ctg_line[k]])
            row = row + a_ctg[k] @ Hk
    const = case.zeta_f * (np.abs(a_base) @ case.rating + (np.abs(a_ctg) * rating_c[None, :]).sum())
    ng = case.n_gen
    bus = np.concatenate([case.gen_bus, case.load_bus])
    sgn = np.concatenate([np.ones(ng), -np.ones(case.n_load)])
    coef = -sgn * (case.zeta_f * row[bus] + case.zeta_inj * float(a_inj))
    total = const
    segs = _segments(case.gen_nseg, case.gen_slope, case.gen_bkpt) + \
        _segments(case.load_nseg, case.load_slope, case.load_bkpt)
    for i in range(case.n_dev):
        a, b = segs[i]
        pts = [lo[i], hi[i]] + [v for v in b if lo[i] < v < hi[i]]
        vals = []
        for xv in pts:
            v = pwl_value(a, b, xv)
            vals.append((-v if i < ng else v) + coef[i] * xv)
        total += max(vals)
    return total


def grad_hi_ratings(case, sens: Sensitivities, lo=None, hi=None, nthreads=None):
    """d hi / d rating (base ratings, eq. (slack-sfb)) and d hi / d rating_ctg
    (contingency ratings, eq. (slack-Sc)), per box and line.

    hi takes -z_f s_lo with s_lo = max(|c| - r - rating, 0) for every base line
    and every (k, l) pair, so each pair whose lower violation bound is positive
    adds +z_f to the derivative in its own rating: the base part counts the
    active base lines, the contingency part the active pairs of each line.
    When the case has no separate contingency ratings both parts belong to the
    one rating vector, whose derivative is their sum.  Every contingency flow
    is formed, so this is for small cases.
    """
    lo = case.box_lo if lo is None else np.atleast_2d(lo)
    hi = case.box_hi if hi is None else np.atleast_2d(hi)
    c, r = bus_box(case, lo, hi)
    fc = c @ sens.phi.T
    fr = r @ np.abs(sens.phi).T
    act_b = (np.abs(fc) - fr - case.rating[None, :]) > 0
    rating_c = case.rating if case.rating_ctg is None else case.rating_ctg
    cent, rad = all_ctg_flows(case, sens, c, r, nthreads)
    act_c = (np.abs(cent) - rad - rating_c[None, None, :]) > 0
    return case.zeta_f * act_b.astype(float), case.zeta_f * act_c.sum(axis=1).astype(float)


def paper_mode_flows(case, sens: Sensitivities, c, r):
    """IBP applied literally to eq. (ctg flow matrix form).

    P = M (x) (1 (Phi p)^T) - B (x) ((U p) 1^T): the intervals of Phi p and U p
    are propagated separately and then combined (reading C9), so
    centre = M c_l - B_kl (U c)_k,  radius = M R_l + |B_kl| (|U| r)_k.
    Returns (centre, radius) of shape [nbox, n_ctg, n_line].
    """
    M, Bm, U = paper_ctg_matrices(case)
    fc = c @ sens.phi.T
    fr = r @ np.abs(sens.phi).T
    uc = c @ U.T
    ur = r @ np.abs(U).T
    cent = M[None] * fc[:, None, :] - Bm[None] * uc[:, :, None]
    rad = M[None] * fr[:, None, :] + np.abs(Bm)[None] * ur[:, :, None]
    return cent, rad


def screen_lines(case, sens: Sensitivities, c, r, rel: float = 0.0):
    """Lines that the paper-mode interval (``paper_mode_flows``, eq. (ctg flow
    matrix form)) cannot clear: True where |centre| + radius > rating * (1 - rel)
    for some contingency and box.  The paper-mode radius bounds the tight one
    from above, so every other line has the violation interval [0, 0] of
    eq. (slack-Sc) for every contingency.  Returns a bool array [n_line]."""
    cent, rad = paper_mode_flows(case, sens, c, r)
    rating = case.rating if getattr(case, "rating_ctg", None) is None else case.rating_ctg
    up = np.abs(cent) + rad
    return np.any(up > rating[None, None, :] * (1.0 - rel), axis=(0, 1))
