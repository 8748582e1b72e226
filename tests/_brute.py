"""Brute-force DC power flow for pinning the oracle (test helper).

Solves the bus angles of the (outaged) network directly for a given injection
vector; no sensitivity matrix is formed.  Used only to check the oracle.
"""
import numpy as np


def dc_flows(n_bus, slack, fr, to, x, inj, drop_line=None):
    """Line flows for nodal injections ``inj`` with the slack absorbing the
    mismatch; ``drop_line`` removes one line (its flow is reported as 0)."""
    lines = [l for l in range(len(fr)) if l != drop_line]
    Y = np.zeros((n_bus, n_bus))
    for l in lines:
        i, j, b = fr[l], to[l], 1.0 / x[l]
        Y[i, i] += b
        Y[j, j] += b
        Y[i, j] -= b
        Y[j, i] -= b
    keep = [i for i in range(n_bus) if i != slack]
    th = np.zeros(n_bus)
    th[keep] = np.linalg.solve(Y[np.ix_(keep, keep)], inj[keep])
    f = np.zeros(len(fr))
    for l in lines:
        f[l] = (th[fr[l]] - th[to[l]]) / x[l]
    return f


def pwl_direct(a, b, x):
    """PWL value as the integral of its piecewise-constant slope from b[0]."""
    v = 0.0
    n = len(a)
    for i in range(n):
        start = b[i]
        end = b[i + 1] if i + 1 < n else np.inf
        if x > start:
            v += a[i] * (min(x, end) - start)
    return v


def objective_brute(case, x):
    """f_ibp at a point from re-solved base and outaged networks."""
    x = np.asarray(x, np.float64)
    ng = case.n_gen
    inj = np.zeros(case.n_bus)
    np.add.at(inj, case.gen_bus, x[:ng])
    np.add.at(inj, case.load_bus, -x[ng:])
    f = dc_flows(case.n_bus, case.slack, case.line_from, case.line_to, case.reactance, inj)
    # nodal imbalance: net outflow of the solved flows minus the injection
    out = np.zeros(case.n_bus)
    np.add.at(out, case.line_from, f)
    np.add.at(out, case.line_to, -f)
    s_inj = np.abs(out - inj).sum()
    s_fb = np.maximum(np.abs(f) - case.rating, 0.0).sum()
    s_fc = 0.0
    for k in case.ctg_line:
        fk = dc_flows(case.n_bus, case.slack, case.line_from, case.line_to, case.reactance,
                      inj, drop_line=int(k))
        s_fc += np.maximum(np.abs(fk) - case.rating, 0.0).sum()
    ptr_g = np.concatenate([[0], np.cumsum(case.gen_nseg)])
    ptr_d = np.concatenate([[0], np.cumsum(case.load_nseg)])
    G = sum(pwl_direct(case.gen_slope[ptr_g[i]:ptr_g[i + 1]], case.gen_bkpt[ptr_g[i]:ptr_g[i + 1]], x[i])
            for i in range(ng))
    C = sum(pwl_direct(case.load_slope[ptr_d[j]:ptr_d[j + 1]], case.load_bkpt[ptr_d[j]:ptr_d[j + 1]], x[ng + j])
            for j in range(case.n_load))
    return C - G - case.zeta_inj * s_inj - case.zeta_f * (s_fb + s_fc)


def read_golden(path):
    out = {}
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = [float(v) for v in vals]
    return out
