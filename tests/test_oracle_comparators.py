"""Pins of the paper's comparison schemes (oracle/hygro_comparators.c: Euler implicit with the fixed-point
sub-iterations of Alg. 1, Euler explicit within its stability bound), which the benchmark times next to the
DF oracle.

* both converge at first order in the time step to the exact solution of the semi-discrete linear system
  (matrix exponential of a two-layer wall with latent cross flux and cTM storage), the implicit scheme as dt
  halves, the explicit one as its substep halves;
* the implicit scheme's fixed point is the exact steady state of the discrete problem (series resistance of
  a layered wall with Robin films);
* on the paper's one-zone building (Sec. 5.2, linear walls coupled to the zone air) with the paper's
  tolerance 0.01 dt* (dt* = dt / 1 h) on the Euclidean norm of the relative changes, the fixed-point
  iteration takes two sub-iterations per step (the paper reports "almost three" and names no norm; a
  count that includes the initial iterate gives three);
* on the Table-1 material the implicit, explicit and DF schemes approach one another as dt falls.
"""
import dataclasses

import numpy as np
import pytest
from scipy.linalg import expm

from paper_1703_10119_gb300 import workloads as wk


def _linear_wall():
    counts, L = [3, 3], 0.1
    lays = [dict(kM0=2e-11, cM0=5e-2, kTT0=0.8, cTT0=1.0e6, chi=8.0e4),
            dict(kM0=6e-11, cM0=3e-2, kTT0=0.3, cTT0=1.6e6, chi=5.0e4)]
    b0 = dict(hT=10.0, hM=2e-8, T_mean=300.0, P_mean=1400.0, q_inf=15.0, g_inf=3e-8)
    b1 = dict(hT=6.0, hM=3e-8, T_mean=288.0, P_mean=800.0)
    return counts, L, lays, b0, b1


def _exact(t, Lv=wk.LV, T0=293.0, P0=1000.0):
    """Semi-discrete solution of _linear_wall at time t: dy/dt = J y + c, y = (P, T), y(0) uniform."""
    counts, L, lays, b0, b1 = _linear_wall()
    N = sum(counts)
    dx = L / (N - 1)
    lay_of = np.repeat([0, 1], counts)
    w = np.ones(N)
    w[0] = w[-1] = 0.5

    def faces(key):
        k = np.array([lays[l][key] for l in lay_of])
        K = np.zeros((N, N))
        for j in range(N - 1):
            kf = 0.5 * (k[j] + k[j + 1]) if lay_of[j] == lay_of[j + 1] else 2 * k[j] * k[j + 1] / (k[j] + k[j + 1])
            K[[j, j + 1], [j, j + 1]] += kf / dx
            K[j, j + 1] -= kf / dx
            K[j + 1, j] -= kf / dx
        return K

    KP, KT = faces("kM0"), faces("kTT0")
    KP[0, 0] += b0["hM"]
    KP[-1, -1] += b1["hM"]
    KT[0, 0] += b0["hT"]
    KT[-1, -1] += b1["hT"]
    MP = w * dx * np.array([lays[l]["cM0"] for l in lay_of])
    MT = w * dx * np.array([lays[l]["cTT0"] for l in lay_of])
    CTM = w * dx * np.array([lays[l]["chi"] * lays[l]["cM0"] for l in lay_of])
    bPh = np.zeros(N)
    bPh[0], bPh[-1] = b0["hM"] * b0["P_mean"], b1["hM"] * b1["P_mean"]
    bP = bPh.copy()
    bP[0] += b0["g_inf"]
    bT = np.zeros(N)
    bT[0], bT[-1] = b0["hT"] * b0["T_mean"] + b0["q_inf"], b1["hT"] * b1["T_mean"]
    JPP = -KP / MP[:, None]
    J = np.zeros((2 * N, 2 * N))
    J[:N, :N] = JPP
    J[N:, :N] = (-Lv * KP - CTM[:, None] * JPP) / MT[:, None]
    J[N:, N:] = -KT / MT[:, None]
    c = np.concatenate([bP / MP, (bT + Lv * bPh - CTM * bP / MP) / MT])
    y0 = np.concatenate([np.full(N, P0), np.full(N, T0)])
    ys = -np.linalg.solve(J, c)
    return ys + expm(J * t) @ (y0 - ys), y0


def test_implicit_euler_converges_at_first_order(oracle_mod):
    counts, L, lays, b0, b1 = _linear_wall()
    t_end = 4 * 3600.0
    exact, y0 = _exact(t_end)
    errs = []
    for n in (8, 16, 32, 64):
        wl = wk.layered_wall(counts, L, lays, dt=t_end / n, T0=293.0, P0=1000.0, bc0=b0, bc1=b1)
        o = oracle_mod.Oracle(wl, n_threads=1)
        it = o.run_implicit(n, eta=1e-14)
        assert it == 2 * n      # linear walls without rooms: the second sub-iteration confirms the first
        got = np.concatenate([o.wall(0, "P"), o.wall(0, "T")])
        errs.append(np.max(np.abs(got - exact) / np.abs(exact - y0).max()))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(1.8 < r < 2.2 for r in ratios), (errs, ratios)


def test_explicit_euler_converges_at_first_order(oracle_mod):
    counts, L, lays, b0, b1 = _linear_wall()
    dt, n = 600.0, 24
    exact, y0 = _exact(dt * n)
    errs, subs = [], []
    for refine in (2.0, 4.0, 8.0, 16.0):
        wl = wk.layered_wall(counts, L, lays, dt=dt, T0=293.0, P0=1000.0, bc0=b0, bc1=b1)
        o = oracle_mod.Oracle(wl, n_threads=1)
        subs.append(o.run_explicit(n, refine))
        got = np.concatenate([o.wall(0, "P"), o.wall(0, "T")])
        errs.append(np.max(np.abs(got - exact) / np.abs(exact - y0).max()))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(1.8 < r < 2.2 for r in ratios), (errs, ratios, subs)
    assert subs[-1] > subs[0]


def test_implicit_steady_state_is_the_series_resistance(oracle_mod):
    counts, L = [7, 9, 6], 0.1
    ks, cs = [0.05, 1.5, 0.3], [1e6, 1.5e6, 8e5]
    layers = [dict(kM0=1e-11, cM0=5e-2, kTT0=k, cTT0=c) for k, c in zip(ks, cs)]
    N = sum(counts)
    dx = L / (N - 1)
    h0, h1, T0, T1 = 25.0, 8.0, 303.0, 283.0
    wl = wk.layered_wall(counts, L, layers, Lv=0.0, dt=1e6, T0=293.0, P0=1000.0,
                         bc0=dict(hT=h0, T_mean=T0, P_mean=1000.0), bc1=dict(hT=h1, T_mean=T1, P_mean=1000.0))
    o = oracle_mod.Oracle(wl, n_threads=1)
    o.run_implicit(60, eta=1e-15, max_iter=10)
    Ls = [(counts[0] - 0.5) * dx, counts[1] * dx, (counts[2] - 0.5) * dx]
    q = (T0 - T1) / (1 / h0 + sum(l / k for l, k in zip(Ls, ks)) + 1 / h1)
    T = o.wall(0, "T")
    assert abs(h0 * (T0 - T[0]) - q) <= 1e-9 * q
    assert abs(h1 * (T[-1] - T1) - q) <= 1e-9 * q


def test_one_zone_subiterations(oracle_mod):
    """Sec. 5.2 reports almost three fixed-point sub-iterations per step for the one-zone case (linear walls
    coupled to the zone air) at the tolerance 0.01 dt*, dt* = dt / 1 h (Appendix B's reference time). With
    the Euclidean norm the walls' resolvent runs twice per step (the second run confirms the first within the
    tolerance); with the largest-change norm many 3.6 s steps stop after one."""
    wl = wk.one_zone()
    n = 2000
    eta = 0.01 * wl.dt / 3600.0
    o = oracle_mod.Oracle(wl)
    assert 2.0 <= o.run_implicit(n, eta=eta, norm="l2") / n <= 3.0
    o = oracle_mod.Oracle(wl)
    assert 1.0 <= o.run_implicit(n, eta=eta, norm="max") / n < 2.0


@pytest.mark.parametrize("law", [wk.LAW_TABLE1, wk.LAW_TABLE1_C])
def test_schemes_agree_on_the_table1_material(oracle_mod, law):
    """The Table-1 wall over 20 min: the implicit and explicit Euler schemes and DF (all on the same spatial
    operator) approach one another as dt falls (Euler first order, DF second)."""
    wl0 = wk.table1_walls(seed=9, n_walls=1, N=41, hours=1.0, law=law)
    diffs = []
    for dt in (12.0, 6.0, 3.0):
        n = int(round(1200.0 / dt))
        wl = dataclasses.replace(wl0, dt=dt)
        o_df, o_im, o_ex = (oracle_mod.Oracle(wl, n_threads=1) for _ in range(3))
        o_df.run(n)
        o_im.run_implicit(n, eta=1e-12)
        o_ex.run_explicit(n, 1.0)
        dT = max(np.abs(o_im.T_cur - o_df.T_cur).max(), np.abs(o_ex.T_cur - o_df.T_cur).max())
        dP = max(np.abs(o_im.P_cur - o_df.P_cur).max(), np.abs(o_ex.P_cur - o_df.P_cur).max())
        diffs.append((dT, dP))
    for i in range(2):
        assert diffs[i + 1][0] < 0.7 * diffs[i][0] and diffs[i + 1][1] < 0.7 * diffs[i][1], diffs
