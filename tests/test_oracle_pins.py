"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the
closed forms the paper prints for special cases (linear DF [eq:dufort], the
nonlinear DF with lambda_0..lambda_3 [eq:DF_NL], the coupled update
[eq:DF_eq2b], the ghost-node surface update [eq:ghost_node_v0],
[eq:ghost_node_u0]), exact steady states (series resistance, Kirchhoff
transform), the Fourier series of linear diffusion with Robin ends, the
exact solution of the semi-discrete system (matrix exponential, tiny grid),
the discrete balance identity, symmetry / invariance properties, the
dimensionless numbers of Appendix B, and a closed-form room steady state.
"""
import dataclasses
import math

import numpy as np
import pytest
from scipy.linalg import expm
from scipy.optimize import brentq

from paper_1703_10119_gb300 import workloads as wk

import golden_data

PS = wk.PSAT_REF


def _one_step(oracle_mod, wl, Tp, Tc, Pp, Pc):
    o = oracle_mod.Oracle(wl, n_threads=1)
    o.set_levels(Tp, Tc, Pp, Pc)
    r = o.run(1)
    return o.wall(0, "T"), o.wall(0, "P"), r


def _rand_levels(rng, N):
    Tp = 293.0 + rng.uniform(-5, 5, N)
    Tc = 293.0 + rng.uniform(-5, 5, N)
    Pp = 1000.0 + rng.uniform(-300, 300, N)
    Pc = 1000.0 + rng.uniform(-300, 300, N)
    return Tp, Tc, Pp, Pc


def test_linear_df_closed_form(oracle_mod):
    """Constant coefficients, interior nodes: [eq:dufort] with lambda = 2 nu dt / dx^2."""
    rng = np.random.default_rng(11)
    N, L, dt = 12, 0.011, 600.0
    lay = dict(kM0=3e-11, cM0=2e-2, kTT0=1.1, cTT0=1.4e6)
    wl = wk.uniform_wall(N, L, lay, Lv=0.0, dt=dt, bc0=dict(hT=10, hM=1e-8), bc1=dict(hT=5, hM=2e-8))
    Tp, Tc, Pp, Pc = _rand_levels(rng, N)
    T1, P1, _ = _one_step(oracle_mod, wl, Tp, Tc, Pp, Pc)
    dx = L / (N - 1)
    for u_prev, u_cur, nu, got in ((Pp, Pc, 3e-11 / 2e-2, P1), (Tp, Tc, 1.1 / 1.4e6, T1)):
        lam = 2.0 * nu * dt / dx ** 2
        j = np.arange(1, N - 1)
        want = (1 - lam) / (1 + lam) * u_prev[j] + lam / (1 + lam) * (u_cur[j + 1] + u_cur[j - 1])
        np.testing.assert_allclose(got[j], want, rtol=1e-13)


def test_nonlinear_df_lambda_form(oracle_mod):
    """Nonlinear kM(Pv), cM(Pv): [eq:DF_NL] solved with lambda_0..lambda_3, nu at the face-mean Pv."""
    rng = np.random.default_rng(12)
    N, L, dt = 15, 0.014, 300.0
    kM0, a, cM0, b = 4e-11, 1.3, 3e-2, 0.8
    lay = dict(kM0=kM0, a=a, cM0=cM0, b=b, kTT0=1.0, cTT0=1e6)
    wl = wk.uniform_wall(N, L, lay, Lv=0.0, dt=dt)
    Tp, Tc, Pp, Pc = _rand_levels(rng, N)
    _, P1, _ = _one_step(oracle_mod, wl, Tp, Tc, Pp, Pc)
    dx = L / (N - 1)
    for j in range(1, N - 1):
        c_j = cM0 * (1 + b * Pc[j] / PS)                     # storage at level n, node j
        nu_p = kM0 * (1 + a * 0.5 * (Pc[j] + Pc[j + 1]) / PS) / c_j
        nu_m = kM0 * (1 + a * 0.5 * (Pc[j] + Pc[j - 1]) / PS) / c_j
        l0, l1, l2 = 1.0, 2 * dt / dx ** 2 * nu_p, 2 * dt / dx ** 2 * nu_m
        l3 = dt / dx ** 2 * (nu_p + nu_m)
        want = (l1 * Pc[j + 1] + l2 * Pc[j - 1] + (l0 - l3) * Pp[j]) / (l0 + l3)
        assert abs(P1[j] - want) <= 1e-13 * abs(want), j


def test_coupled_df_eq2b(oracle_mod):
    """Coupled T update with kTM cross flux and cTM storage: [eq:DF_eq1] then [eq:DF_eq2b]."""
    rng = np.random.default_rng(13)
    N, L, dt, Lv, chi = 10, 0.009, 120.0, 2.5e6, 8.36e4
    kM0, cM0, kTT, cTT = 5e-11, 4e-2, 0.7, 9e5
    lay = dict(kM0=kM0, cM0=cM0, kTT0=kTT, cTT0=cTT, chi=chi)
    wl = wk.uniform_wall(N, L, lay, Lv=Lv, dt=dt)
    Tp, Tc, Pp, Pc = _rand_levels(rng, N)
    T1, P1, _ = _one_step(oracle_mod, wl, Tp, Tc, Pp, Pc)
    dx = L / (N - 1)
    r = 2 * dt / dx ** 2
    lam = r * kM0 / cM0
    mu = r * kTT / cTT
    beta = r * Lv * kM0 / cTT
    gamma = chi * cM0 / cTT
    j = np.arange(1, N - 1)
    v1 = (1 - lam) / (1 + lam) * Pp[j] + lam / (1 + lam) * (Pc[j + 1] + Pc[j - 1])
    np.testing.assert_allclose(P1[j], v1, rtol=1e-13)
    u1 = ((1 - mu) / (1 + mu) * Tp[j] + mu / (1 + mu) * (Tc[j + 1] + Tc[j - 1])
          + (gamma - beta) / (1 + mu) * Pp[j] + beta / (1 + mu) * (Pc[j + 1] + Pc[j - 1])
          - (gamma + beta) / (1 + mu) * v1)
    np.testing.assert_allclose(T1[j], u1, rtol=1e-12)


def _solve_linear(f):
    f0, f1 = f(0.0), f(1.0)
    return -f0 / (f1 - f0)


@pytest.mark.parametrize("face", [0, 1])
def test_ghost_node_surface(oracle_mod, face):
    """Surface node = DF with the ghost node of [eq:ghost_node_v0] and [eq:ghost_node_u0]."""
    rng = np.random.default_rng(14 + face)
    N, L, dt, Lv, chi = 9, 0.008, 90.0, 2.5e6, 5e4
    kM, cM, kTT, cTT = 6e-11, 3e-2, 0.9, 1.1e6
    hT, hM, Tinf, Pinf = (17.0, 2.5e-8, 301.0, 1350.0) if face == 0 else (6.0, 3.5e-8, 287.0, 780.0)
    bcs = [dict(hT=3.0, hM=1e-8, T_mean=295.0, P_mean=1100.0)] * 2
    bcs[face] = dict(hT=hT, hM=hM, T_mean=Tinf, P_mean=Pinf)
    wl = wk.uniform_wall(N, L, dict(kM0=kM, cM0=cM, kTT0=kTT, cTT0=cTT, chi=chi), Lv=Lv, dt=dt,
                         bc0=bcs[0], bc1=bcs[1])
    Tp, Tc, Pp, Pc = _rand_levels(rng, N)
    T1, P1, _ = _one_step(oracle_mod, wl, Tp, Tc, Pp, Pc)
    dx = L / (N - 1)
    s, i = (0, 1) if face == 0 else (N - 1, N - 2)        # surface node, first interior node
    r = 2 * dt / dx ** 2
    lam, mu = r * kM / cM, r * kTT / cTT
    beta, gamma = r * Lv * kM / cTT, chi * cM / cTT
    BiM, BiTT, BiTM = hM / kM, hT / kTT, Lv * hM / kTT   # Bi per unit length (h / k)

    def v_ghost(vn):
        return Pc[i] - 2 * BiM * dx * (0.5 * (vn + Pp[s]) - Pinf)

    v1 = _solve_linear(lambda x: x - ((1 - lam) / (1 + lam) * Pp[s] + lam / (1 + lam) * (Pc[i] + v_ghost(x))))
    assert abs(P1[s] - v1) <= 1e-12 * abs(v1)
    v0 = v_ghost(v1)

    def u_ghost(un):
        return (Tc[i] + (Lv * kM / kTT) * (Pc[i] - v0) - 2 * BiTT * dx * (0.5 * (un + Tp[s]) - Tinf)
                - 2 * BiTM * dx * (0.5 * (v1 + Pp[s]) - Pinf))

    u1 = _solve_linear(lambda x: x - ((1 - mu) / (1 + mu) * Tp[s] + mu / (1 + mu) * (Tc[i] + u_ghost(x))
                                      + (gamma - beta) / (1 + mu) * Pp[s] + beta / (1 + mu) * (Pc[i] + v0)
                                      - (gamma + beta) / (1 + mu) * v1))
    assert abs(T1[s] - u1) <= 1e-12 * abs(u1)


def _run_to_steady(oracle_mod, wl, chunk=20000, max_chunks=100, tol=1e-13):
    o = oracle_mod.Oracle(wl, n_threads=1)
    for _ in range(max_chunks):
        r = o.run(chunk)
        dT = np.abs(o.T_cur - o.T_prev).max() / np.abs(o.T_cur).max()
        dP = np.abs(o.P_cur - o.P_prev).max() / np.abs(o.P_cur).max()
        if dT < tol and dP < tol:
            return o, r
    raise AssertionError("no steady state reached")


def test_steady_series_resistance(oracle_mod):
    """Linear multilayer heat: the steady flux is the series-resistance value, nodes on the exact profile."""
    counts, L = [7, 9, 6], 0.1
    ks, cs = [0.05, 1.5, 0.3], [1e6, 1.5e6, 8e5]
    layers = [dict(kM0=1e-11, cM0=5e-2, kTT0=k, cTT0=c) for k, c in zip(ks, cs)]
    N = sum(counts)
    dx = L / (N - 1)
    dt = 0.5 * dx ** 2 / max(k / c for k, c in zip(ks, cs))
    h0, h1, T0, T1 = 25.0, 8.0, 303.0, 283.0
    wl = wk.layered_wall(counts, L, layers, Lv=0.0, dt=dt, T0=293.0, P0=1000.0,
                         bc0=dict(hT=h0, T_mean=T0, P_mean=1000.0), bc1=dict(hT=h1, T_mean=T1, P_mean=1000.0))
    o, r = _run_to_steady(oracle_mod, wl)
    Ls = [(counts[0] - 0.5) * dx, counts[1] * dx, (counts[2] - 0.5) * dx]
    R = 1 / h0 + sum(l / k for l, k in zip(Ls, ks)) + 1 / h1
    q = (T0 - T1) / R
    assert abs(r["flux"][0, 0, 0] - q) <= 1e-9 * q
    assert abs(r["flux"][0, 1, 0] + q) <= 1e-9 * q
    x = np.arange(N) * dx
    edges = np.cumsum([0.0] + Ls)
    T = np.empty(N)
    Ts = T0 - q / h0
    for l in range(3):
        m = (x >= edges[l] - 1e-12) & (x <= edges[l + 1] + 1e-12)
        T[m] = Ts - q * (x[m] - edges[l]) / ks[l]
        Ts = Ts - q * Ls[l] / ks[l]
    np.testing.assert_allclose(o.wall(0, "T"), T, rtol=0, atol=1e-9 * (T0 - T1))


def test_steady_kirchhoff_moisture(oracle_mod):
    """Nonlinear kM = kM0 (1 + a Pv/Ps): the face-mean flux is the Kirchhoff difference, so the
    discrete steady state is the exact continuous solution at the nodes."""
    N, L, kM0, a = 26, 0.05, 2e-11, 1.5
    hM0, hM1, Pi0, Pi1 = 2e-8, 3e-8, 1600.0, 800.0
    cM0 = 5e-2
    dx = L / (N - 1)
    nu = kM0 * (1 + a * Pi0 / PS) / cM0
    dt = 0.5 * dx ** 2 / nu
    wl = wk.uniform_wall(N, L, dict(kM0=kM0, a=a, cM0=cM0, b=0.7, kTT0=1.0, cTT0=1e6), Lv=0.0, dt=dt,
                         P0=1200.0, bc0=dict(hM=hM0, P_mean=Pi0), bc1=dict(hM=hM1, P_mean=Pi1))
    o, r = _run_to_steady(oracle_mod, wl, chunk=50000, max_chunks=200)

    def Phi(P):
        return P + a * P ** 2 / (2 * PS)

    def Pinv(F):
        c = a / PS
        return (-1 + np.sqrt(1 + 2 * c * F)) / c

    def resid(P0):
        g = hM0 * (Pi0 - P0)
        PL = Pi1 + g / hM1
        return kM0 * (Phi(P0) - Phi(PL)) / L - g

    P0 = brentq(resid, Pi1, Pi0, xtol=1e-14, rtol=1e-15)
    g = hM0 * (Pi0 - P0)
    PL = Pi1 + g / hM1
    want = Pinv(Phi(P0) - np.arange(N) / (N - 1) * (Phi(P0) - Phi(PL)))
    np.testing.assert_allclose(o.wall(0, "P"), want, rtol=1e-10)
    assert abs(r["flux"][0, 0, 1] - g) <= 1e-8 * g


def _fourier_robin(x, t, L, alpha, H0, H1, theta0, n_terms=300):
    """Series solution of theta_t = alpha theta_xx, theta_x = H0 theta (x=0), theta_x = -H1 theta (x=L)."""
    f = lambda b: (b * b - H0 * H1) * math.sin(b * L) - b * (H0 + H1) * math.cos(b * L)
    grid = np.linspace(1e-9, (n_terms + 2) * math.pi / L, 40 * (n_terms + 2))
    vals = np.array([f(b) for b in grid])
    roots = [brentq(f, grid[k], grid[k + 1], xtol=1e-14)
             for k in range(len(grid) - 1) if vals[k] * vals[k + 1] < 0][:n_terms]
    xg, wg = np.polynomial.legendre.leggauss(400)
    xq = 0.5 * L * (xg + 1)
    wq = 0.5 * L * wg
    out = np.zeros_like(x)
    for b in roots:
        X = lambda y: b * np.cos(b * y) + H0 * np.sin(b * y)
        c = theta0 * np.sum(wq * X(xq)) / np.sum(wq * X(xq) ** 2)
        out += c * X(x) * math.exp(-alpha * b * b * t)
    return out


def test_fourier_series_convergence(oracle_mod):
    """Linear diffusion with Robin ends: DF error vs the Fourier series falls ~4x per halving of dx
    with dt proportional to dx^2 (second order in space, Sec. 3.1)."""
    L, k, c, h0, h1 = 0.1, 1.0, 1e6, 10.0, 5.0
    Ti, Tinf = 293.0, 303.0
    alpha = k / c
    t_end = 0.1 * L * L / alpha
    errs = []
    for n_int, steps in ((10, 50), (20, 200), (40, 800)):
        N = n_int + 1
        dt = t_end / steps
        wl = wk.uniform_wall(N, L, dict(kM0=1e-12, cM0=5e-2, kTT0=k, cTT0=c), Lv=0.0, dt=dt, T0=Ti,
                             bc0=dict(hT=h0, T_mean=Tinf, P_mean=1000.0), bc1=dict(hT=h1, T_mean=Tinf, P_mean=1000.0))
        o = oracle_mod.Oracle(wl, n_threads=1)
        o.run(steps)
        x = np.linspace(0, L, N)
        exact = Tinf + _fourier_robin(x, t_end, L, alpha, h0 / k, h1 / k, Ti - Tinf)
        errs.append(np.abs(o.wall(0, "T") - exact).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.0 < r1 < 5.5 and 3.0 < r2 < 5.5, errs
    assert errs[2] < 2e-3 * abs(Ti - Tinf)


def test_second_order_in_time_semidiscrete(oracle_mod):
    """Tiny two-layer wall: DF against the exact solution of the semi-discrete system (matrix
    exponential), started from exact levels; the error falls ~4x per halving of dt (Sec. 3.1)."""
    counts, L = [3, 3], 0.1
    ks, cs = [0.5, 1.2], [1e6, 2e6]
    h0, h1, Tinf0, Tinf1 = 10.0, 4.0, 300.0, 285.0
    N = 6
    dx = L / (N - 1)
    w = np.ones(N)
    w[0] = w[-1] = 0.5
    lay_of = np.repeat([0, 1], counts)
    kn = np.array([ks[l] for l in lay_of])
    M = np.diag(w * dx * np.array([cs[l] for l in lay_of]))
    K = np.zeros((N, N))
    for j in range(N - 1):
        kf = 0.5 * (kn[j] + kn[j + 1]) if lay_of[j] == lay_of[j + 1] else 2 * kn[j] * kn[j + 1] / (kn[j] + kn[j + 1])
        g = kf / dx
        K[j, j] += g
        K[j + 1, j + 1] += g
        K[j, j + 1] -= g
        K[j + 1, j] -= g
    K[0, 0] += h0
    K[-1, -1] += h1
    bvec = np.zeros(N)
    bvec[0], bvec[-1] = h0 * Tinf0, h1 * Tinf1
    A = -np.linalg.solve(M, K)
    Ts = np.linalg.solve(K, bvec)
    T0 = np.full(N, 293.0)

    def exact(t):
        return Ts + expm(A * t) @ (T0 - Ts)

    t_start, t_end = 500.0, 2500.0
    errs = []
    for dt in (40.0, 20.0, 10.0):
        layers = [dict(kM0=1e-12, cM0=5e-2, kTT0=k, cTT0=c) for k, c in zip(ks, cs)]
        wl = wk.layered_wall(counts, L, layers, Lv=0.0, dt=dt, bc0=dict(hT=h0, T_mean=Tinf0, P_mean=1000.0),
                             bc1=dict(hT=h1, T_mean=Tinf1, P_mean=1000.0))
        o = oracle_mod.Oracle(wl, n_threads=1)
        P = np.full(N, 1000.0)
        o.set_levels(exact(t_start - dt), exact(t_start), P, P)
        o.run(int(round((t_end - t_start) / dt)))
        errs.append(np.abs(o.wall(0, "T") - exact(t_end)).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4, errs


def _rich_batch(n_walls=24, steps=200, seed=5):
    wl = wk.wall_batch(seed=seed, n_walls=n_walls, n_steps=steps, n_min=5, n_max=60)
    lp = wl.layer_par.copy()
    rng = np.random.default_rng(seed)
    lp[:, 5] = rng.uniform(0, 0.5, len(lp))          # aT
    lp[:, 7] = rng.uniform(0, 0.5, len(lp))          # bT
    lp[:, 8] = 8.36e4                                # chi = cw * 20
    bp = wl.bc_par.copy()
    bp[:, :, 2] = rng.uniform(-20, 20, (n_walls, 2))     # q_inf
    bp[:, :, 3] = rng.uniform(-1e-6, 1e-6, (n_walls, 2))  # g_inf
    return dataclasses.replace(wl, layer_par=lp, bc_par=bp)


def test_balance_identity(oracle_mod):
    """Summed over the nodes, the DF balance gives S = B + D exactly (storage = surface flux + DF defect)."""
    wl = _rich_batch()
    o = oracle_mod.Oracle(wl, n_threads=4)
    o.run(37)
    r = o.run(1, want_balance=True)
    bal = r["balance"]
    S, B, D, M = bal[..., 0], bal[..., 1], bal[..., 2], bal[..., 3]
    assert np.all(np.abs(S - B - D) <= 1e-12 * M)
    assert np.all(np.abs(D) > 0)                      # the defect is real, not identically zero


def test_mirror_symmetry(oracle_mod):
    counts = [8, 10, 8]
    outer = dict(kM0=3e-11, a=0.9, cM0=4e-2, b=0.4, kTT0=0.8, cTT0=1.2e6, chi=8.36e4)
    inner = dict(kM0=1e-11, a=0.3, cM0=7e-2, b=1.1, kTT0=0.2, cTT0=9e5, chi=8.36e4)
    bc = dict(hT=12.0, hM=2e-8, T_mean=300.0, T_amp=8.0, P_mean=1300.0, P_amp=300.0, phase_P=0.7)
    wl = wk.layered_wall(counts, 0.12, [outer, inner, outer], dt=300.0, bc0=bc, bc1=bc)
    o = oracle_mod.Oracle(wl, n_threads=1)
    o.run(400)
    for f in "TP":
        u = o.wall(0, f)
        np.testing.assert_allclose(u, u[::-1], rtol=1e-13)


def test_uniform_invariance(oracle_mod):
    lay = [dict(kM0=3e-11, a=1.7, cM0=4e-2, b=1.2, kTT0=0.8, cTT0=1.2e6, chi=8.36e4, aT=0.3, bT=0.2),
           dict(kM0=1e-12, a=0.2, cM0=9e-2, b=0.1, kTT0=0.05, cTT0=2e5, chi=8.36e4)]
    bc = dict(hT=12.0, hM=2e-8, T_mean=293.0, P_mean=1000.0)
    wl = wk.layered_wall([20, 13], 0.1, lay, dt=600.0, bc0=bc, bc1=bc)
    o = oracle_mod.Oracle(wl, n_threads=1)
    o.run(2000)
    assert np.abs(o.wall(0, "T") - 293.0).max() <= 1e-12 * 293.0
    assert np.abs(o.wall(0, "P") - 1000.0).max() <= 1e-12 * 1000.0


def test_appendix_b_dimensionless_numbers():
    """Table 2 (one-zone walls) with t0 = 1 h, L = 0.1 m, Ti = 293.15 K and Pvi = Psat/2 reproduce
    the Fourier, gamma and Biot numbers printed in Appendix B (within their 2-3 printed digits); both
    tables as printed in tests/golden/one_zone_table2_appendix_b.txt."""
    g = golden_data.load("one_zone_table2_appendix_b.txt")
    z = g["zone"]["zone"]
    t0, L, Ti, Lv = 3600.0, z["L"], 273.15 + z["Ti_C"], 2.5e6
    Pvi = z["phi_i"] * PS
    hT_in, hM_in = z["hT_in"], z["hM_in"]
    cols = ("FoM", "FoTT", "FoTM", "gamma", "BiM_0", "BiTT_0", "BiTM_0", "BiM_1", "BiTT_1", "BiTM_1")
    for name, w in g["table2"].items():
        cM, kM, cTT, kTT, cTM, kTM, hT, hM = (w[k] for k in ("cM", "kM", "cTT", "kTT", "cTM", "kTM", "hT", "hM"))
        got = (t0 * kM / (L * L * cM), t0 * kTT / (L * L * cTT), t0 * kTM / (L * L * cTM), cTM * Pvi / (cTT * Ti),
               hM * L / kM, hT * L / kTT, Lv * hM * L * Pvi / (kTT * Ti),
               hM_in * L / kM, hT_in * L / kTT, Lv * hM_in * L * Pvi / (kTT * Ti))
        printed = g["appendix_b"][name]
        for c, v in zip(cols, got):
            p = printed[c]
            assert abs(v - p) <= 0.012 * abs(p), (name, c, v, p)
    # cTM / cM = cw * 20 (the coupling storage with T in Celsius), for every wall of Table 2
    for w in g["table2"].values():
        assert abs(w["cTM"] / w["cM"] / (4180.0 * 20.0) - 1.0) < 0.01


def test_dimensionless_similarity(oracle_mod):
    """Two dimensional problems with the same Fourier and Biot numbers (L -> 2L, t -> 4t, h -> h/2)
    give the same discrete solution (Sec. 2: one dimensionless problem for a class of problems)."""
    lay = dict(kM0=5.89e-9, cM0=1.82e-2, kTT0=0.294, cTT0=7.7e5, chi=8.36e4)
    runs = []
    for s in (1.0, 2.0):
        bc0 = dict(hT=5.0 / s, hM=2e-7 / s, T_mean=293.0, T_amp=4.0, P_mean=1200.0, P_amp=200.0,
                   period=86400.0 * s * s, phase_P=0.3)
        bc1 = dict(hT=8.0 / s, hM=3e-8 / s, T_mean=295.0, P_mean=1100.0)
        wl = wk.uniform_wall(21, 0.1 * s, lay, dt=36.0 * s * s, bc0=bc0, bc1=bc1, P0=1168.5, T0=293.15)
        o = oracle_mod.Oracle(wl, n_threads=1)
        o.run(500)
        runs.append((o.wall(0, "T").copy(), o.wall(0, "P").copy()))
    np.testing.assert_allclose(runs[0][0], runs[1][0], rtol=1e-12)
    np.testing.assert_allclose(runs[0][1], runs[1][1], rtol=1e-11)


def test_ambient_forcing(oracle_mod):
    """Face air state: daily sinusoid plus a linearly interpolated noise table held at its ends."""
    wl = wk.wall_batch(seed=3, n_walls=2, n_steps=100)
    o = oracle_mod.Oracle(wl, n_threads=1)
    nz = wl.noise[0][1].astype(np.float64)
    bp = wl.bc_par[1, 0]
    T, P = o.ambient(1, 0, 0.0)
    assert abs(T - (293.0 + 10 * math.sin(bp[9]) + nz[0, 0])) < 1e-9
    assert abs(P - (1200.0 + 400 * math.sin(bp[10]) + nz[0, 1])) < 1e-9
    t = 3600.0 * 7 + 1800.0
    T, P = o.ambient(1, 0, t)
    ph = 2 * math.pi * t / 86400.0
    assert abs(T - (293.0 + 10 * math.sin(ph + bp[9]) + 0.5 * (nz[7, 0] + nz[8, 0]))) < 1e-9
    T, P = o.ambient(1, 0, 1e9)
    assert abs(P - (1200.0 + 400 * math.sin(2 * math.pi * 1e9 / 86400.0 + bp[10]) + nz[-1, 1])) < 1e-6
    T, P = o.ambient(1, 1, 12345.0)                   # face 1: constant 293 K / 1000 Pa
    assert (T, P) == (293.0, 1000.0)


@pytest.mark.parametrize("scheme", [0, 1])
def test_room_steady_state(oracle_mod, scheme):
    """One room, two walls, constant gains, Lv = 0: the steady room air state is the closed form
    Ta = To + Q / (gv cpa + sum A / R), Pva = Po + g / (gv / Pref + sum A / R_M) -- for the room as a DF
    node (scheme 0) and for the explicit Euler room update of Sec. 5.2 (scheme 1, stable at this dt): both
    have the steady balance as their fixed point."""
    To, Po, Q, g, V, ach = 275.0, 600.0, 400.0, 1.5e-4, 30.0, 1.0
    rho, cpa, cpv, Pref = 1.2, 1006.0, 1860.0, 1.61e5
    walls = []
    specs = [([6, 8], [dict(kM0=1e-9, cM0=5e-2, kTT0=0.9, cTT0=1.8e6), dict(kM0=3e-9, cM0=3e-2, kTT0=0.1, cTT0=4e5)],
              0.08, 12.0, 18.0, 2e-8, 3e-8),
             ([10], [dict(kM0=2e-9, cM0=4e-2, kTT0=0.6, cTT0=1.2e6)], 0.05, 8.0, 25.0, 1e-8, 2e-8)]
    Rs, RMs = [], []
    for counts, layers, L, A, h_out, hM_out, hM_in in specs:
        h_in = 7.0
        w = wk.layered_wall(counts, L, layers, dt=60.0, T0=290.0, P0=900.0, Lv=0.0,
                            bc0=dict(hT=h_out, hM=hM_out, T_mean=To, P_mean=Po),
                            bc1=dict(hT=h_in, hM=hM_in), kinds=(wk.BC_AMBIENT, wk.BC_ROOM))
        w.bc_room = np.array([[-1, 0]], np.int32)
        walls.append(w)
        N = sum(counts)
        dx = L / (N - 1)
        Ls = [(counts[0] - 0.5) * dx] + [c * dx for c in counts[1:-1]] + ([(counts[-1] - 0.5) * dx] if len(counts) > 1 else [])
        if len(counts) == 1:
            Ls = [L]
        Rs.append((A, 1 / h_out + sum(l / lay["kTT0"] for l, lay in zip(Ls, layers)) + 1 / h_in))
        RMs.append((A, 1 / hM_out + sum(l / lay["kM0"] for l, lay in zip(Ls, layers)) + 1 / hM_in))
    wl = wk.concat(walls)
    wl.Lv = 0.0
    par = np.zeros((1, len(wk.ROOM_FIELDS)))
    par[0, :15] = [V, ach, Q, g, To, 0.0, Po, 0.0, 86400.0, 0.0, 0.0, rho, cpa, cpv, Pref]
    par[0, 15] = scheme
    wl.rooms = dict(par=par, wall_area=np.array([s[3] for s in specs]), Ta0=np.array([291.0]), Pa0=np.array([950.0]))
    o, _ = _run_to_steady(oracle_mod, wl, chunk=20000, max_chunks=200, tol=1e-14)
    gv = rho * V * ach / 3600.0
    Ta = To + Q / (gv * cpa + sum(A / R for A, R in Rs))
    Pa = Po + g / (gv / Pref + sum(A / R for A, R in RMs))
    assert abs(o.room[0, 1] - Ta) <= 1e-9 * Ta
    assert abs(o.room[0, 3] - Pa) <= 1e-9 * Pa


def test_room_euler_is_unstable_at_the_building_time_step(oracle_mod):
    """Reading R26: with the whole-building workload's dt = 300 s, a small room's time constant (heat
    capacity over exchange conductance) is below dt / 2, so the explicit Euler room update of Sec. 5.2
    grows without bound, while the room as a DF node stays at physical values."""
    wl = wk.building(seed=3, n_rooms=2, walls_per_room=6, n_steps=400)
    rooms = dict(wl.rooms)
    par = np.array(rooms["par"], np.float64).copy()
    par[:, 0] = 30.0          # 30 m^3 rooms
    wl.rooms = dict(rooms, par=par)
    rho_V_cp = par[:, 11] * par[:, 0] * par[:, 12]
    tau = rho_V_cp / (np.bincount(np.where(wl.bc_room[:, 1] >= 0, wl.bc_room[:, 1], 0),
                                  weights=wl.rooms["wall_area"] * wl.bc_par[:, 1, 0], minlength=2))
    assert np.all(tau < wl.dt / 2)
    o = oracle_mod.Oracle(wl, n_threads=1)
    o.run(400)
    assert np.all(np.abs(o.room[:, 1] - 293.0) < 60.0)
    par_e = par.copy()
    par_e[:, 15] = 1.0
    wl.rooms = dict(rooms, par=par_e)
    oe = oracle_mod.Oracle(wl, n_threads=1)
    with np.errstate(all="ignore"):
        oe.run(400)
    Ta = oe.room[:, 1]
    assert np.any(~np.isfinite(Ta)) or np.max(np.abs(Ta - 293.0)) > 1e3


def test_euler_start_converges_to_the_semidiscrete_solution(oracle_mod):
    """The start by explicit Euler substeps: level 1 tends to the exact solution at t = dt of the coupled
    linear semi-discrete system (two layers, constant coefficients, latent cross flux, cTM storage, Robin
    faces with sources), written as dy/dt = J y + c and solved by the matrix exponential. The error is first
    order in the substep: it halves when the substep count doubles."""
    counts, L = [3, 3], 0.1
    lays = [dict(kM0=2e-11, cM0=5e-2, kTT0=0.8, cTT0=1.0e6, chi=8.0e4),
            dict(kM0=6e-11, cM0=3e-2, kTT0=0.3, cTT0=1.6e6, chi=5.0e4)]
    Lv, dt = wk.LV, 600.0
    b0 = dict(hT=10.0, hM=2e-8, T_mean=300.0, P_mean=1400.0, q_inf=15.0, g_inf=3e-8)
    b1 = dict(hT=6.0, hM=3e-8, T_mean=288.0, P_mean=800.0)
    T0, P0 = 293.0, 1000.0
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
    # dP/dt = MP^-1 (-KP P + bP); MT dT/dt + CTM dP/dt = -KT T + bT + Lv (-KP P + bPh)
    JPP = -KP / MP[:, None]
    J = np.zeros((2 * N, 2 * N))
    J[:N, :N] = JPP
    J[N:, :N] = (-Lv * KP - CTM[:, None] * JPP) / MT[:, None]
    J[N:, N:] = -KT / MT[:, None]
    c = np.concatenate([bP / MP, (bT + Lv * bPh - CTM * bP / MP) / MT])
    y0 = np.concatenate([np.full(N, P0), np.full(N, T0)])
    ys = -np.linalg.solve(J, c)
    exact = ys + expm(J * dt) @ (y0 - ys)
    errs = []
    for refine in (2.0, 4.0, 8.0, 16.0):
        wl = wk.layered_wall(counts, L, lays, dt=dt, T0=T0, P0=P0, bc0=b0, bc1=b1, Lv=Lv)
        o = oracle_mod.Oracle(wl, n_threads=1)
        o.euler_start(refine)
        assert o.step == 1
        assert np.array_equal(o.wall(0, "T", 1), np.full(N, T0))
        got = np.concatenate([o.wall(0, "P"), o.wall(0, "T")])
        errs.append(np.max(np.abs(got - exact) / np.abs(exact - y0).max()))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(1.8 < r < 2.2 for r in ratios), (errs, ratios)
    assert errs[-1] < 0.05
