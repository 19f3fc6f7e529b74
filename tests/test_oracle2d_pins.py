"""Pins of the FP64 2D oracle (5-point DF on wall sections) against what the mathematics fixes.

* interior nodes, constant coefficients: the 2D form of [eq:dufort],
  (1 + 2 lam) u^{n+1} = (1 - 2 lam) u^{n-1} + lam (sum of the 4 neighbours), lam = 2 nu dt / h^2;
* edge and corner nodes: the DF update with the ghost nodes of [eq:ghost_node_v0] /
  [eq:ghost_node_u0] on the Robin faces and mirror ghosts on the adiabatic faces, solved for u^{n+1}
  (coupled Pv / T with the kTM cross flux and the cTM storage) -- this fixes the half-cell weights;
* the separable exact solution of linear diffusion with Robin faces at x = 0, y = 0 and adiabatic
  faces at x = L, y = L: the error falls ~4x per halving of h (dt ~ h^2);
* transposition symmetry and uniform invariance.
"""
import dataclasses
import math

import numpy as np
import pytest
from scipy.optimize import brentq

from paper_1703_10119_gb300 import workloads as wk


def section(nx, ny, layer, bc, dt, n_steps=10, region=None, kinds=(0, 1, 0, 1), Lv=wk.LV, T0=293.0, P0=1000.0,
            h=1e-3):
    layers = layer if isinstance(layer, list) else [layer]
    par = np.array([[[lay.get(k, 0.0) for k in wk.LAYER_FIELDS] for lay in layers]], np.float64)
    reg = np.zeros((1, ny, nx), np.uint8) if region is None else region[None].astype(np.uint8)
    bc_par = np.zeros((1, 4, len(wk.BC_FIELDS)))
    for f in range(4):
        b = bc if isinstance(bc, dict) else bc[f]
        bc_par[0, f] = [b.get("hT", 0.0), b.get("hM", 0.0), b.get("q_inf", 0.0), b.get("g_inf", 0.0),
                        b.get("T_mean", T0), b.get("T_amp", 0.0), b.get("P_mean", P0), b.get("P_amp", 0.0),
                        b.get("period", 86400.0), b.get("phase_T", 0.0), b.get("phase_P", 0.0), 3600.0,
                        b.get("period_P", 0.0)]
    return wk.Section2D(name="test", h=h, region=reg, region_par=par, bc_kind=np.array([kinds], np.int32),
                        bc_par=bc_par, noise=[None] * 4, T_init=np.array([T0]), P_init=np.array([P0]),
                        dt=dt, t0=0.0, n_steps=n_steps, Lv=Lv)


def one_step(oracle_mod, sec, lv):
    o = oracle_mod.Oracle2D(sec, 1)
    o.set_levels(*[x[None] for x in lv])
    o.run(1)
    return o.T_cur[0], o.P_cur[0]


def rand_levels(rng, ny, nx):
    return (293 + rng.uniform(-5, 5, (ny, nx)), 293 + rng.uniform(-5, 5, (ny, nx)),
            1000 + rng.uniform(-200, 200, (ny, nx)), 1000 + rng.uniform(-200, 200, (ny, nx)))


def test_interior_closed_form(oracle_mod):
    rng = np.random.default_rng(31)
    nx, ny, dt, h = 9, 7, 60.0, 1e-3
    lay = dict(kM0=4e-11, cM0=3e-2, kTT0=0.9, cTT0=1.1e6)
    sec = section(nx, ny, lay, dict(hT=10.0, hM=1e-8), dt, Lv=0.0)
    Tp, Tc, Pp, Pc = rand_levels(rng, ny, nx)
    T1, P1 = one_step(oracle_mod, sec, (Tp, Tc, Pp, Pc))
    for up, uc, nu, got in ((Pp, Pc, 4e-11 / 3e-2, P1), (Tp, Tc, 0.9 / 1.1e6, T1)):
        lam = 2 * nu * dt / h ** 2
        i = np.s_[1:-1, 1:-1]
        nb = uc[:-2, 1:-1] + uc[2:, 1:-1] + uc[1:-1, :-2] + uc[1:-1, 2:]
        want = ((1 - 2 * lam) * up[i] + lam * nb) / (1 + 2 * lam)
        np.testing.assert_allclose(got[i], want, rtol=1e-13)


def _solve_linear(f):
    f0, f1 = f(0.0), f(1.0)
    return -f0 / (f1 - f0)


@pytest.mark.parametrize("node", ["west_edge", "south_edge", "corner", "east_edge"])
def test_boundary_nodes_ghost_form(oracle_mod, node):
    """Edge and corner nodes equal DF with ghost nodes (Robin at x = 0 and y = 0, mirror at x = L, y = L)."""
    rng = np.random.default_rng(32)
    nx, ny, dt, h = 7, 6, 90.0, 1e-3
    Lv, chi = 2.5e6, 5e4
    kM, cM, kT, cT = 6e-11, 3e-2, 0.9, 1.1e6
    hT, hM, Tinf, Pinf = 17.0, 2.5e-8, 301.0, 1350.0
    air = dict(hT=hT, hM=hM, T_mean=Tinf, P_mean=Pinf)
    sec = section(nx, ny, dict(kM0=kM, cM0=cM, kTT0=kT, cTT0=cT, chi=chi), [air, {}, air, {}], dt, Lv=Lv)
    Tp, Tc, Pp, Pc = rand_levels(rng, ny, nx)
    T1, P1 = one_step(oracle_mod, sec, (Tp, Tc, Pp, Pc))
    i, j = {"west_edge": (0, 3), "south_edge": (3, 0), "corner": (0, 0), "east_edge": (nx - 1, 2)}[node]
    r = 2 * dt / h ** 2
    lam, mu = r * kM / cM, r * kT / cT
    beta, gamma = r * Lv * kM / cT, chi * cM / cT

    def ghost_P(d, Pn):
        """Value of the neighbour in direction d = (di, dj), ghost across a domain face."""
        ii, jj = i + d[0], j + d[1]
        if 0 <= ii < nx and 0 <= jj < ny:
            return Pc[jj, ii]
        mi, mj = i - d[0], j - d[1]                     # mirror node
        robin = (ii < 0) or (jj < 0)
        g = Pc[mj, mi]
        if robin:
            g -= 2 * (hM / kM) * h * (0.5 * (Pn + Pp[j, i]) - Pinf)
        return g

    dirs = [(1, 0), (-1, 0), (0, 1), (0, -1)]
    P_new = _solve_linear(lambda x: x - ((1 - 2 * lam) * Pp[j, i] + lam * sum(ghost_P(d, x) for d in dirs)) /
                          (1 + 2 * lam))
    assert abs(P1[j, i] - P_new) <= 1e-12 * abs(P_new)
    Pg = {d: ghost_P(d, P_new) for d in dirs}

    def ghost_T(d, Tn):
        ii, jj = i + d[0], j + d[1]
        if 0 <= ii < nx and 0 <= jj < ny:
            return Tc[jj, ii]
        mi, mj = i - d[0], j - d[1]
        robin = (ii < 0) or (jj < 0)
        g = Tc[mj, mi]
        if robin:
            g += (Lv * kM / kT) * (Pc[mj, mi] - Pg[d]) - 2 * (hT / kT) * h * (0.5 * (Tn + Tp[j, i]) - Tinf) \
                 - 2 * (Lv * hM / kT) * h * (0.5 * (P_new + Pp[j, i]) - Pinf)
        return g

    # 2D [eq:DF_eq2b]: (1 + 2 mu) u+ = (1 - 2 mu) u- + mu sum u_nb + (gamma - 2 beta) v- + beta sum v_nb - (gamma + 2 beta) v+
    T_new = _solve_linear(lambda x: x - ((1 - 2 * mu) * Tp[j, i] + mu * sum(ghost_T(d, x) for d in dirs)
                                         + (gamma - 2 * beta) * Pp[j, i] + beta * sum(Pg[d] for d in dirs)
                                         - (gamma + 2 * beta) * P_new) / (1 + 2 * mu))
    assert abs(T1[j, i] - T_new) <= 1e-12 * abs(T_new)


def _series_1d(x, t, L, alpha, H0, n_terms=200):
    """theta(x, t) / theta0 for theta_t = alpha theta_xx, theta_x = H0 theta at 0, theta_x = 0 at L."""
    f = lambda b: b * math.sin(b * L) - H0 * math.cos(b * L)
    grid = np.linspace(1e-9, (n_terms + 2) * math.pi / L, 40 * (n_terms + 2))
    vals = np.array([f(b) for b in grid])
    roots = [brentq(f, grid[k], grid[k + 1], xtol=1e-14)
             for k in range(len(grid) - 1) if vals[k] * vals[k + 1] < 0][:n_terms]
    xg, wg = np.polynomial.legendre.leggauss(300)
    xq, wq = 0.5 * L * (xg + 1), 0.5 * L * wg
    out = np.zeros_like(x)
    for b in roots:
        X = lambda y: b * np.cos(b * y) + H0 * np.sin(b * y)
        c = np.sum(wq * X(xq)) / np.sum(wq * X(xq) ** 2)
        out += c * X(x) * math.exp(-alpha * b * b * t)
    return out


def test_separable_exact_solution_convergence(oracle_mod):
    L, k, c, hcoef, Ti, Tinf = 0.04, 1.0, 1e6, 20.0, 293.0, 303.0
    alpha = k / c
    t_end = 0.1 * L * L / alpha
    errs = []
    for n_int, steps in ((8, 40), (16, 160), (32, 640)):
        n = n_int + 1
        h = L / n_int
        air = dict(hT=hcoef, T_mean=Tinf)
        sec = section(n, n, dict(kM0=1e-12, cM0=5e-2, kTT0=k, cTT0=c), [air, {}, air, {}], t_end / steps,
                      Lv=0.0, h=h, T0=Ti)
        o = oracle_mod.Oracle2D(sec, 1)
        o.run(steps)
        x = np.linspace(0, L, n)
        X = _series_1d(x, t_end, L, alpha, hcoef / k)
        exact = Tinf + (Ti - Tinf) * np.outer(X, X)          # [y, x]
        errs.append(np.abs(o.T_cur[0] - exact).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.0 < r1 < 5.5 and 3.0 < r2 < 5.5, errs


def test_transposition_symmetry(oracle_mod):
    rng = np.random.default_rng(33)
    nx, ny = 12, 9
    region = (rng.uniform(size=(ny, nx)) < 0.3).astype(np.uint8)
    layers = [dict(kM0=3e-11, a=0.9, cM0=4e-2, b=0.4, kTT0=0.8, cTT0=1.2e6, chi=8.36e4),
              dict(kM0=1e-11, a=0.3, cM0=7e-2, b=1.1, kTT0=0.2, cTT0=9e5, chi=8.36e4)]
    air0 = dict(hT=12.0, hM=2e-8, T_mean=300.0, T_amp=8.0, P_mean=1300.0, P_amp=300.0, phase_P=0.7)
    air2 = dict(hT=7.0, hM=1e-8, T_mean=290.0, T_amp=3.0, P_mean=900.0, P_amp=100.0, phase_T=0.3)
    a = section(nx, ny, layers, [air0, {}, air2, {}], 300.0, region=region)
    b = section(ny, nx, layers, [air2, {}, air0, {}], 300.0, region=region.T.copy())
    oa, ob = oracle_mod.Oracle2D(a, 1), oracle_mod.Oracle2D(b, 1)
    oa.run(200)
    ob.run(200)
    np.testing.assert_allclose(oa.T_cur[0], ob.T_cur[0].T, rtol=1e-13)
    np.testing.assert_allclose(oa.P_cur[0], ob.P_cur[0].T, rtol=1e-13)


def test_uniform_invariance(oracle_mod):
    rng = np.random.default_rng(34)
    region = (rng.uniform(size=(10, 11)) < 0.4).astype(np.uint8)
    layers = [dict(kM0=3e-11, a=1.7, cM0=4e-2, b=1.2, kTT0=0.8, cTT0=1.2e6, chi=8.36e4, aT=0.3, bT=0.2),
              dict(kM0=1e-12, a=0.2, cM0=9e-2, b=0.1, kTT0=0.05, cTT0=2e5)]
    air = dict(hT=12.0, hM=2e-8, T_mean=293.0, P_mean=1000.0)
    sec = section(11, 10, layers, [air, air, air, {}], 600.0, region=region, kinds=(0, 0, 0, 1))
    o = oracle_mod.Oracle2D(sec, 1)
    o.run(500)
    assert np.abs(o.T_cur - 293.0).max() <= 1e-12 * 293.0
    assert np.abs(o.P_cur - 1000.0).max() <= 1e-12 * 1000.0


@pytest.mark.parametrize("axis", ["x", "y"])
def test_steady_series_resistance_across_regions(oracle_mod, axis):
    """Three regions in series along one axis (Robin faces at both ends of it, adiabatic faces along it):
    the discrete steady state is uniform across the other axis and every node lies on the exact
    series-resistance profile, with each region interface at the mid-face between its two nodes
    (harmonic face means) -- the 1D steady state of the paper's scheme, reached in 2D."""
    counts, L = [7, 9, 6], 0.1
    ks, cs = [0.05, 1.5, 0.3], [1e6, 1.5e6, 8e5]
    layers = [dict(kM0=1e-11, cM0=5e-2, kTT0=k, cTT0=c) for k, c in zip(ks, cs)]
    N, M = sum(counts), 5
    h = L / (N - 1)
    dt = 0.5 * h ** 2 / max(k / c for k, c in zip(ks, cs))
    h0, h1, T0, T1 = 25.0, 8.0, 303.0, 283.0
    line = np.repeat(np.arange(3), counts).astype(np.uint8)
    amb0, amb1, adi = dict(hT=h0, T_mean=T0), dict(hT=h1, T_mean=T1), dict()
    if axis == "x":
        region, nx, ny, bc, kinds = np.tile(line, (M, 1)), N, M, [amb0, amb1, adi, adi], (0, 0, 1, 1)
    else:
        region, nx, ny, bc, kinds = np.tile(line[:, None], (1, M)), M, N, [adi, adi, amb0, amb1], (1, 1, 0, 0)
    sec = section(nx, ny, layers, bc, dt, region=region, kinds=kinds, Lv=0.0, h=h)
    o = oracle_mod.Oracle2D(sec, 1)
    for _ in range(100):
        o.run(20000)
        if np.abs(o.T_cur - o.T_prev).max() / np.abs(o.T_cur).max() < 1e-13:
            break
    else:
        raise AssertionError("no steady state reached")
    Ls = [(counts[0] - 0.5) * h, counts[1] * h, (counts[2] - 0.5) * h]
    q = (T0 - T1) / (1 / h0 + sum(l / k for l, k in zip(Ls, ks)) + 1 / h1)
    s = np.arange(N) * h
    edges = np.cumsum([0.0] + Ls)
    want = np.empty(N)
    Ts = T0 - q / h0
    for l in range(3):
        m = (s >= edges[l] - 1e-12) & (s <= edges[l + 1] + 1e-12)
        want[m] = Ts - q * (s[m] - edges[l]) / ks[l]
        Ts = Ts - q * Ls[l] / ks[l]
    got = o.T_cur[0] if axis == "x" else o.T_cur[0].T
    for row in got:
        np.testing.assert_allclose(row, want, rtol=0, atol=1e-9 * (T0 - T1))
    np.testing.assert_allclose(o.P_cur[0], 1000.0, rtol=0, atol=1e-9)
