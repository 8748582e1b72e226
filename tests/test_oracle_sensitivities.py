"""Pins for the oracle's PTDF and LODF (Sec. II-A and II-C) against Kirchhoff's
laws, a textbook closed form, full re-solves of outaged networks and the
paper's own Sherman-Morrison construction."""
import dataclasses
import os
from collections import deque

import numpy as np
import pytest

import oracle as O
from gen import make_network_case
from tests._brute import dc_flows, read_golden

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _three_bus():
    g = read_golden(os.path.join(GOLD, "ptdf_3bus.txt"))
    c = make_network_case("tri", 3, 3, 1, 1, seed=1, ring5=False)
    c = dataclasses.replace(c, line_from=np.array(g["from"], np.int32),
                            line_to=np.array(g["to"], np.int32),
                            reactance=np.array(g["x"]), rating=np.ones(3) * 100,
                            ctg_line=np.array([int(g["ctg"][0])], np.int32))
    return c, g


def test_ptdf_three_bus_closed_form():
    c, g = _three_bus()
    phi = O.ptdf(c)
    want = np.array([g["phi_row0"], g["phi_row1"], g["phi_row2"]])
    np.testing.assert_allclose(phi, want, rtol=0, atol=1e-14)
    L, _ = O.lodf(c, phi)
    np.testing.assert_allclose(L[:, 0], g["lodf_col"], rtol=0, atol=1e-14)


@pytest.mark.parametrize("cfg", [0, 1])
def test_ptdf_kcl_and_zero_slack(cases, cfg):
    c = cases(cfg)
    phi = O.ptdf(c)
    assert np.all(phi[:, c.slack] == 0.0)
    rng = np.random.default_rng(7)
    p = rng.normal(size=(c.n_bus, 5)) * 100
    f = phi @ p
    out = np.zeros((c.n_bus, 5))
    np.add.at(out, c.line_from, f)
    np.add.at(out, c.line_to, -f)
    nonslack = [b for b in range(c.n_bus) if b != c.slack]
    np.testing.assert_allclose(out[nonslack], p[nonslack], atol=1e-9 * np.abs(p).max())
    # the slack absorbs the whole mismatch
    np.testing.assert_allclose(out[c.slack], -p[nonslack].sum(axis=0), atol=1e-9 * np.abs(p).sum())


@pytest.mark.parametrize("cfg", [0, 1])
def test_ptdf_kvl_angles_exist(cases, cfg):
    """Flows from Phi admit bus angles theta with f_l = (theta_from - theta_to)/x_l:
    propagate angles along a BFS spanning tree from the slack, then every other
    line must agree (Kirchhoff's voltage law)."""
    c = cases(cfg)
    phi = O.ptdf(c)
    rng = np.random.default_rng(3)
    p = rng.normal(size=c.n_bus) * 50
    f = phi @ p
    adj = [[] for _ in range(c.n_bus)]
    for l in range(c.n_line):
        adj[c.line_from[l]].append(l)
        adj[c.line_to[l]].append(l)
    th = np.full(c.n_bus, np.nan)
    th[c.slack] = 0.0
    q = deque([c.slack])
    used = set()
    while q:
        v = q.popleft()
        for l in adj[v]:
            a, b = c.line_from[l], c.line_to[l]
            w = b if a == v else a
            if np.isnan(th[w]):
                # f_l = (th_a - th_b)/x
                th[w] = th[v] - f[l] * c.reactance[l] if a == v else th[v] + f[l] * c.reactance[l]
                used.add(l)
                q.append(w)
    resid = f - (th[c.line_from] - th[c.line_to]) / c.reactance
    assert np.abs(resid).max() < 1e-9 * np.abs(f).max()


@pytest.mark.parametrize("cfg", [0, 1])
def test_lodf_matches_outaged_resolve(cases, cfg):
    c = cases(cfg)
    s = O.sensitivities(c)
    assert np.all(s.lodf[c.ctg_line, np.arange(c.n_ctg)] == -1.0)
    for k in range(c.n_ctg):
        kl = int(c.ctg_line[k])
        Hk = s.phi + np.outer(s.lodf[:, k], s.phi[kl, :])
        assert np.all(Hk[kl] == 0.0)  # the outaged line carries exactly nothing
        ref = O.outage_ptdf(c, kl)
        np.testing.assert_allclose(Hk, ref, rtol=0, atol=1e-10 * max(1.0, np.abs(ref).max()))


@pytest.mark.parametrize("cfg", [0, 1])
def test_lodf_matches_angle_resolve(cases, cfg):
    """Contingency flows H_k p equal the angle solve of the outaged network."""
    c = cases(cfg)
    s = O.sensitivities(c)
    rng = np.random.default_rng(11)
    p = rng.normal(size=c.n_bus) * 80
    for k in range(0, c.n_ctg, max(1, c.n_ctg // 12)):
        kl = int(c.ctg_line[k])
        fk = (s.phi + np.outer(s.lodf[:, k], s.phi[kl, :])) @ p
        ref = dc_flows(c.n_bus, c.slack, c.line_from, c.line_to, c.reactance, p, drop_line=kl)
        np.testing.assert_allclose(fk, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("cfg", [0, 1])
def test_paper_sherman_morrison_form(cases, cfg):
    """Eq. (ctg flow matrix form) with the literal u_i, g_i, B, U, M reproduces H_k p."""
    c = cases(cfg)
    s = O.sensitivities(c)
    M, Bm, U = O.paper_ctg_matrices(c)
    rng = np.random.default_rng(5)
    p = rng.normal(size=c.n_bus) * 60
    P = M * (s.phi @ p)[None, :] - Bm * (U @ p)[:, None]
    H = (s.phi @ p)[None, :] + s.lodf.T * (s.phi @ p)[c.ctg_line][:, None]
    np.testing.assert_allclose(P, H, rtol=0, atol=1e-9 * np.abs(H).max())


def test_bridge_contingency_rejected():
    c = make_network_case("t", 6, 6, 2, 2, seed=3)
    bridges = __import__("gen").find_bridges(c.n_bus, c.line_from, c.line_to)
    assert bridges.any()
    bad = dataclasses.replace(c, ctg_line=np.flatnonzero(bridges)[:1].astype(np.int32))
    phi = O.ptdf(bad)
    with pytest.raises(O.IslandingContingency):
        O.lodf(bad, phi)


def test_find_bridges_brute_force():
    """Tarjan bridges agree with 'removal disconnects' on small random graphs."""
    from gen import find_bridges
    rng = np.random.default_rng(0)
    for trial in range(30):
        n = int(rng.integers(3, 12))
        m = int(rng.integers(n - 1, min(n * (n - 1) // 2, 2 * n) + 1))
        c = make_network_case("g", n, m, 1, 1, seed=int(rng.integers(1 << 20)))
        got = find_bridges(n, c.line_from, c.line_to)
        for l in range(m):
            seen = {0}
            stack = [0]
            while stack:
                v = stack.pop()
                for e in range(m):
                    if e == l:
                        continue
                    a, b = c.line_from[e], c.line_to[e]
                    for (u, w) in ((a, b), (b, a)):
                        if u == v and w not in seen:
                            seen.add(w)
                            stack.append(w)
            assert got[l] == (len(seen) < n)
