"""Pins of the oracle's room air node (Sec. 5.1, [eq:LAV_equation], [eq:LAV_couplage]; the room advanced
with the wall surface values of level n as in [eq:wbse_tn_exp]) with the latent terms and the vapour part
of the air's heat capacity switched on.

Three checks, each against something the room update itself does not compute:

* the closed system of the walls and the room air over one step: the energy (and the vapour mass) stored
  in the walls and in the air equals what enters through the outdoor faces, the ventilation and the
  internal gains, plus the walls' DF defects and the coupling defect of the room faces (the room sees
  the walls at level n, the walls see the room at level n; each side takes its own time-averaged value).
  The walls' storage, flux and defect terms come from the wall update, whose own balance identity is
  pinned elsewhere; the room's terms are written here from the physics;
* a room without walls is a linear scalar problem: vapour mass rho V dw/dt = g + gv (w_out - w) and,
  with the vapour at its steady state, heat rho V (cpa + cpv w) dTa/dt = Q + gv cpa (T_out - Ta) (the
  latent gain Lv g and the latent ventilation Lv gv (w_out - w) then cancel). The DF node's three-level
  recurrence for such a problem has the closed-form solution e^{n+1} = rho e^{n-1} around the fixed
  point; the explicit Euler update has e^{n+1} = (1 - k dt / C) e^n;
* with the vapour away from its steady state the latent ventilation drives the heat balance; the DF
  room node started from exact levels converges to the solution of the two ODEs at second order in dt.

Interzone airflow (Sec. 5.1, Q_inz and G_inz) and long-wave radiation among a room's surfaces (Sec. 2,
q_rw, taken in the DF step as faces to the room's other surfaces: T'^4 - Ts^4 = h' (T' - Ts), the
conductance h' = s eps sigma (T'^2 + Ts^2)(T' + Ts) and T' of level n, Ts averaged over levels n+1 and n-1):
two zones exchanging air
converge at second order to the solution of their four ODEs (latent terms on); the radiative flux between
two faces matches the linearised exchange 4 s eps sigma T^3 dT, is reciprocal for equal emissivities and
areas, and takes each face's own emissivity; radiation alone equalises two walls' surfaces over a long run
(a level-n own value would be a leapfrog term, and a level-n Ts^4 with only Ts^3 averaged leaves the
explicit coupling four times the damping: both unstable in DF); and the
closed-system balance of two linked rooms with radiating walls holds to 1e-12 with the interzone coupling
defect and the radiation deposited in the walls.
"""
import dataclasses
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

from paper_1703_10119_gb300 import workloads as wk

RHO, CPA, CPV, PREF = 1.2, 1006.0, 1860.0, 1.61e5


def _room_row(V, ach, Q, g, T_out, P_out, scheme=0, T_amp=0.0, P_amp=0.0, period=86400.0, phase_T=0.0,
              phase_P=0.0):
    row = dict(volume=V, ach=ach, Q_gain=Q, g_vap=g, T_out_mean=T_out, T_out_amp=T_amp, P_out_mean=P_out,
               P_out_amp=P_amp, period=period, phase_T=phase_T, phase_P=phase_P, rho_a=RHO, cp_a=CPA, cp_v=CPV,
               Pv_ref=PREF, scheme=scheme)
    return np.array([row.get(k, 0.0) for k in wk.ROOM_FIELDS], np.float64)


def _lonely_room(V, ach, Q, g, T_out, P_out, Ta0, Pa0, dt, scheme=0):
    """One room that no wall faces (a dummy wall with two ambient faces keeps the workload valid)."""
    w = wk.uniform_wall(5, 0.05, dict(kM0=1e-11, cM0=5e-2, kTT0=0.5, cTT0=1e6), dt=dt,
                        bc0=dict(hT=5.0, hM=1e-8), bc1=dict(hT=5.0, hM=1e-8))
    w.rooms = dict(par=_room_row(V, ach, Q, g, T_out, P_out, scheme)[None], wall_area=np.array([1.0]),
                   Ta0=np.array([Ta0]), Pa0=np.array([Pa0]))
    return w


# --------------------------------------------------------------------------------------------------
# closed system: walls + room air, one step


def _building(Lv, scheme):
    """Three layered walls (one with cTM storage, one with face sources) around one ventilated room
    with heat and vapour gains; outdoor air on face 0, the room on face 1."""
    specs = [
        ([6, 7], [dict(kM0=2e-9, a=0.6, cM0=5e-2, b=0.4, kTT0=0.9, cTT0=1.8e6, chi=8.0e4),
                  dict(kM0=4e-9, a=0.2, cM0=3e-2, b=0.9, kTT0=0.2, cTT0=6e5, chi=2.0e4)], 0.08, 11.0),
        ([9], [dict(kM0=1e-9, a=1.1, cM0=4e-2, b=0.3, kTT0=0.6, aT=0.3, cTT0=1.2e6, bT=0.2)], 0.05, 7.5),
        ([4, 5, 4], [dict(kM0=3e-9, cM0=2e-2, kTT0=1.4, cTT0=2.0e6), dict(kM0=8e-10, a=0.5, cM0=6e-2, kTT0=0.05,
                                                                          cTT0=1.0e5),
                     dict(kM0=2e-9, b=0.7, cM0=4e-2, kTT0=0.7, cTT0=1.5e6)], 0.12, 14.0),
    ]
    walls, area = [], []
    for i, (counts, layers, L, A) in enumerate(specs):
        bc0 = dict(hT=18.0 + i, hM=2e-8 + 1e-9 * i, T_mean=278.0, T_amp=6.0, P_mean=800.0, P_amp=250.0,
                   period=86400.0, phase_T=0.4 + i, phase_P=1.3, q_inf=12.0 if i == 1 else 0.0,
                   g_inf=4e-8 if i == 1 else 0.0)
        bc1 = dict(hT=7.0 + 0.5 * i, hM=3e-8 - 2e-9 * i)
        w = wk.layered_wall(counts, L, layers, dt=300.0, T0=291.0 + i, P0=950.0 + 40 * i, Lv=Lv,
                            bc0=bc0, bc1=bc1, kinds=(wk.BC_AMBIENT, wk.BC_ROOM))
        w.bc_room = np.array([[-1, 0]], np.int32)
        walls.append(w)
        area.append(A)
    wl = wk.concat(walls)
    wl.Lv = Lv
    par = _room_row(45.0, 1.3, 350.0, 2.2e-4, 279.0, 820.0, scheme, T_amp=5.0, P_amp=200.0, phase_T=0.7,
                    phase_P=2.1)
    wl.rooms = dict(par=par[None], wall_area=np.array(area), Ta0=np.array([292.0]), Pa0=np.array([1400.0]))
    return wl


def _closed_system_terms(oracle_mod, wl, n_before):
    """Every term of the walls + room balance of the step n -> n+1 after n_before steps."""
    o = oracle_mod.Oracle(wl, n_threads=1)
    o.run(n_before)
    n = o.step
    room0 = o.room[0].copy()            # Ta^{n-1}, Ta^n, Pa^{n-1}, Pa^n
    surf_prev = [(o.wall(w, "T", 1)[-1], o.wall(w, "P", 1)[-1]) for w in range(wl.n_walls)]   # level n-1
    surf_n = [(o.wall(w, "T", 0)[-1], o.wall(w, "P", 0)[-1]) for w in range(wl.n_walls)]      # level n
    r = o.run(1, want_balance=True)
    room1 = o.room[0].copy()            # Ta^n, Ta^{n+1}, Pa^n, Pa^{n+1}
    surf_next = [(o.wall(w, "T", 0)[-1], o.wall(w, "P", 0)[-1]) for w in range(wl.n_walls)]   # level n+1
    assert room1[0] == room0[1] and room1[2] == room0[3]

    q = wl.rooms["par"][0]
    f = dict(zip(wk.ROOM_FIELDS, q))
    dt, Lv = wl.dt, wl.Lv
    t = wl.t0 + n * dt
    V, rho = f["volume"], f["rho_a"]
    gv = rho * V * f["ach"] / 3600.0                       # kg/s of exchanged air
    T_out = f["T_out_mean"] + f["T_out_amp"] * math.sin(2 * math.pi * t / f["period"] + f["phase_T"])
    P_out = f["P_out_mean"] + f["P_out_amp"] * math.sin(2 * math.pi * t / f["period"] + f["phase_P"])
    w_out = P_out / f["Pv_ref"]
    Ta_m, Ta_n, Ta_p = room0[0], room0[1], room1[1]
    Pa_m, Pa_n, Pa_p = room0[2], room0[3], room1[3]
    euler = f["scheme"] == 1.0
    if euler:   # every room term at level n, forward difference
        Ta_s, Pa_s = Ta_n, Pa_n
        dTa, dPa = (Ta_p - Ta_n) / dt, (Pa_p - Pa_n) / dt
    else:       # the room node's own value is the mean of levels n+1 and n-1, centred difference
        Ta_s, Pa_s = 0.5 * (Ta_p + Ta_m), 0.5 * (Pa_p + Pa_m)
        dTa, dPa = (Ta_p - Ta_m) / (2 * dt), (Pa_p - Pa_m) / (2 * dt)
    # air: vapour mass rho V w and enthalpy with the heat capacity rho V (cpa + cpv w^n)
    C_heat = rho * V * (f["cp_a"] + f["cp_v"] * Pa_n / f["Pv_ref"])
    store_air = {"T": C_heat * dTa, "P": rho * V / f["Pv_ref"] * dPa}
    w_s = Pa_s / f["Pv_ref"]
    sources = {"T": [f["Q_gain"], Lv * f["g_vap"], gv * f["cp_a"] * (T_out - Ta_s), Lv * gv * (w_out - w_s)],
               "P": [f["g_vap"], gv * (w_out - w_s)]}
    A = wl.rooms["wall_area"]
    bal = r["balance"]       # [wall][T, Pv][S, B, D, M] per unit area
    flux = r["flux"]         # [wall][face][heat, moisture], positive into the wall
    terms = {}
    for k, fld in enumerate(("T", "P")):
        store_walls = float(np.sum(A * bal[:, k, 0]))
        outdoor = float(np.sum(A * flux[:, 0, k]))
        defect_walls = float(np.sum(A * bal[:, k, 2]))
        # coupling defect of the room faces: the wall takes (air^n - its surface mean), the room takes
        # (surface^n - its own value); their sum is what the pair does not conserve
        coup = 0.0
        for w in range(wl.n_walls):
            hT, hM = wl.bc_par[w, 1, 0], wl.bc_par[w, 1, 1]
            sT_bar = 0.5 * (surf_next[w][0] + surf_prev[w][0])
            sP_bar = 0.5 * (surf_next[w][1] + surf_prev[w][1])
            dP_pair = (Pa_n - sP_bar) + (surf_n[w][1] - Pa_s)
            if fld == "T":
                coup += A[w] * (hT * ((Ta_n - sT_bar) + (surf_n[w][0] - Ta_s)) + Lv * hM * dP_pair)
            else:
                coup += A[w] * hM * dP_pair
        terms[fld] = dict(store_walls=store_walls, store_air=store_air[fld], outdoor=outdoor,
                          defect_walls=defect_walls, coupling=coup, sources=sources[fld],
                          scale=float(np.sum(A * bal[:, k, 3])))
    return terms


@pytest.mark.parametrize("scheme", [0, 1])
def test_closed_system_balance_walls_and_room(oracle_mod, scheme):
    """Storage in walls + air = outdoor-face fluxes + ventilation + gains + the walls' DF defects +
    the room faces' coupling defect, for heat (latent terms, vapour heat capacity and cTM on) and vapour,
    to 1e-12 of the sum of the magnitudes of the terms, at several steps of a forced run."""
    wl = _building(Lv=2.5e6, scheme=scheme)
    for n_before in (1, 7, 40):
        terms = _closed_system_terms(oracle_mod, wl, n_before)
        for fld in ("T", "P"):
            t = terms[fld]
            lhs = t["store_walls"] + t["store_air"]
            rhs = t["outdoor"] + sum(t["sources"]) + t["defect_walls"] + t["coupling"]
            mag = (abs(t["store_walls"]) + abs(t["store_air"]) + abs(t["outdoor"]) + sum(map(abs, t["sources"]))
                   + abs(t["defect_walls"]) + abs(t["coupling"]) + t["scale"])
            assert abs(lhs - rhs) <= 1e-12 * mag, (fld, n_before, lhs, rhs, mag)


def test_closed_system_balance_has_teeth(oracle_mod):
    """Each room term a plausible mistake would drop or flip (the latent gain, the latent ventilation, the
    latent part of the wall exchange, the vapour part of the heat capacity) is many orders of magnitude
    above the 1e-12 tolerance of the balance, so the balance cannot hold without it."""
    wl = _building(Lv=2.5e6, scheme=0)
    t = _closed_system_terms(oracle_mod, wl, 40)["T"]
    mag = (abs(t["store_walls"]) + abs(t["store_air"]) + abs(t["outdoor"]) + sum(map(abs, t["sources"]))
           + abs(t["defect_walls"]) + abs(t["coupling"]) + t["scale"])
    f = dict(zip(wk.ROOM_FIELDS, wl.rooms["par"][0]))
    o = oracle_mod.Oracle(wl, n_threads=1)
    o.run(41)
    Pa = o.room[0, 2]
    # latent gain, latent ventilation
    assert abs(t["sources"][1]) > 1e-6 * mag and abs(t["sources"][3]) > 1e-6 * mag
    # latent part of the wall exchange seen by the room: Lv sum A hM (Ps - Pa), Ps the surface values
    A = wl.rooms["wall_area"]
    lat_walls = sum(A[w] * wl.Lv * wl.bc_par[w, 1, 1] * (o.wall(w, "P", 1)[-1] - Pa) for w in range(wl.n_walls))
    assert abs(lat_walls) > 1e-6 * mag
    # vapour part of the heat capacity: rho V cpv w times the air's temperature rate
    cpv_part = t["store_air"] * (f["cp_v"] * Pa / f["Pv_ref"]) / (f["cp_a"] + f["cp_v"] * Pa / f["Pv_ref"])
    assert abs(cpv_part) > 1e-9 * mag


# --------------------------------------------------------------------------------------------------
# a room without walls: closed-form recurrences


def test_lonely_room_vapour_recurrence(oracle_mod):
    """Vapour mass balance rho V dw/dt = g + gv (w_out - w), w = Pa / Pv_ref: fixed point
    w* = w_out + g / gv, and the DF node gives e^{n+1} = (1 - r dt) / (1 + r dt) e^{n-1} exactly, with
    r = gv / (rho V) = ach / 3600 (level -1 := level 0, so e^n = rho^ceil(n/2) e^0); explicit Euler gives
    e^{n+1} = (1 - r dt) e^n."""
    V, ach, g, P_out, dt = 50.0, 1.0, 2.0e-4, 900.0, 300.0
    gv = RHO * V * ach / 3600.0
    P_star = PREF * (P_out / PREF + g / gv)
    r = ach / 3600.0
    for scheme in (0, 1):
        wl = _lonely_room(V, ach, 500.0, g, 280.0, P_out, 295.0, 1100.0, dt, scheme)
        o = oracle_mod.Oracle(wl, n_threads=1)
        e0 = 1100.0 - P_star
        for n in range(1, 41):
            o.run(1)
            if scheme == 0:
                want = ((1 - r * dt) / (1 + r * dt)) ** ((n + 1) // 2) * e0
            else:
                want = (1 - r * dt) ** n * e0
            assert abs((o.room[0, 3] - P_star) - want) <= 1e-12 * abs(e0), (scheme, n)


def test_lonely_room_heat_recurrence_with_latent_terms(oracle_mod):
    """With the vapour at its steady state w* the latent gain Lv g and the latent ventilation
    Lv gv (w_out - w*) cancel, so the heat balance is rho V (cpa + cpv w*) dTa/dt = Q + gv cpa (T_out - Ta):
    fixed point T_out + Q / (gv cpa), and the DF node's recurrence e^{n+1} = (C - k dt) / (C + k dt) e^{n-1}
    with C = rho V (cpa + cpv w*), k = gv cpa; explicit Euler e^{n+1} = (1 - k dt / C) e^n. Lv = 2.5e6 and
    a vapour gain of 0.2 g/s: a dropped or flipped latent term moves the fixed point by tens of kelvin."""
    V, ach, Q, g, T_out, P_out, dt = 50.0, 1.0, 500.0, 2.0e-4, 280.0, 900.0, 300.0
    gv = RHO * V * ach / 3600.0
    w_star = P_out / PREF + g / gv
    P_star = PREF * w_star
    T_star = T_out + Q / (gv * CPA)
    C = RHO * V * (CPA + CPV * w_star)
    k = gv * CPA
    assert wk.LV * g / k > 20.0        # the latent gain alone would shift the fixed point by > 20 K
    for scheme in (0, 1):
        wl = _lonely_room(V, ach, Q, g, T_out, P_out, 295.0, P_star, dt, scheme)
        assert wl.Lv == wk.LV
        o = oracle_mod.Oracle(wl, n_threads=1)
        e0 = 295.0 - T_star
        for n in range(1, 41):
            o.run(1)
            if scheme == 0:
                want = ((C - k * dt) / (C + k * dt)) ** ((n + 1) // 2) * e0
            else:
                want = (1 - k * dt / C) ** n * e0
            assert abs((o.room[0, 1] - T_star) - want) <= 1e-11 * abs(e0), (scheme, n, o.room[0, 1])
            assert abs(o.room[0, 3] - P_star) <= 1e-12 * P_star


def test_lonely_room_transient_converges_at_second_order(oracle_mod):
    """Vapour away from its steady state: w(t) = w* + (w0 - w*) exp(-r t), and the heat balance
    rho V (cpa + cpv w(t)) dTa/dt = Q + Lv g + gv cpa (T_out - Ta) + Lv gv (w_out - w(t)) carries a latent
    ventilation term of about 300 W and a heat capacity that changes with w. The DF room node started from
    the exact levels at t = -dt and t = 0 converges to the solution of these ODEs (integrated to 1e-12)
    at second order: the error falls about 4x per halving of dt."""
    V, ach, Q, g, T_out, P_out = 50.0, 1.0, 500.0, 2.0e-4, 280.0, 900.0
    gv = RHO * V * ach / 3600.0
    r = ach / 3600.0
    w_out = P_out / PREF
    w_star = w_out + g / gv
    w0 = w_star - 0.007
    Ta0 = 300.0
    Lv = wk.LV

    def w_of(t):
        return w_star + (w0 - w_star) * np.exp(-r * t)

    def rhs(t, y):
        w = w_of(t)
        return [(Q + Lv * g + gv * CPA * (T_out - y[0]) + Lv * gv * (w_out - w)) / (RHO * V * (CPA + CPV * w))]

    assert Lv * gv * abs(w0 - w_star) > 250.0
    t_end = 6 * 3600.0
    exact_end = solve_ivp(rhs, (0.0, t_end), [Ta0], method="DOP853", rtol=1e-13, atol=1e-11).y[0, -1]
    errs = []
    for dt in (600.0, 300.0, 150.0, 75.0):
        Ta_m = solve_ivp(rhs, (0.0, -dt), [Ta0], method="DOP853", rtol=1e-13, atol=1e-11).y[0, -1]
        wl = _lonely_room(V, ach, Q, g, T_out, P_out, Ta0, PREF * w0, dt)
        o = oracle_mod.Oracle(wl, n_threads=1)
        o.room[0] = [Ta_m, Ta0, PREF * w_of(-dt), PREF * w0]
        o.run(int(round(t_end / dt)))
        errs.append((abs(o.room[0, 1] - exact_end), abs(o.room[0, 3] - PREF * w_of(t_end))))
    for i in range(3):
        for fld in range(2):
            ratio = errs[i][fld] / errs[i + 1][fld]
            assert 3.6 < ratio < 4.4, (errs, i, fld)
    assert errs[-1][0] < 1e-3


# --------------------------------------------------------------------------------------------------
# interzone airflow and long-wave radiation among room surfaces (Sec. 5.1 Q_inz, G_inz; Sec. 2 q_rw)


def _two_zones(V1, V2, g, dt, T0=(300.0, 290.0), P0=(1500.0, 900.0)):
    """Two rooms without walls, no ventilation or gains, exchanging g kg/s of air (a dummy wall with two
    ambient faces keeps the workload valid)."""
    w = wk.uniform_wall(5, 0.05, dict(kM0=1e-11, cM0=5e-2, kTT0=0.5, cTT0=1e6), dt=dt,
                        bc0=dict(hT=5.0, hM=1e-8), bc1=dict(hT=5.0, hM=1e-8))
    par = np.stack([_room_row(V1, 0.0, 0.0, 0.0, 280.0, 900.0), _room_row(V2, 0.0, 0.0, 0.0, 280.0, 900.0)])
    w.rooms = dict(par=par, wall_area=np.array([1.0]), Ta0=np.array(T0), Pa0=np.array(P0), links=[(0, 1, g)])
    return w


def test_interzone_transient_converges_at_second_order(oracle_mod):
    """Two zones exchanging air: rho V_i dw_i/dt = g (w_j - w_i) and rho V_i (cpa + cpv w_i) dT_i/dt =
    g cpa (T_j - T_i) + Lv g (w_j - w_i). From exact starting levels the DF zone nodes (each zone's own value
    averaged over levels n+1 and n-1, the other zone's of level n) converge to the ODE solution at second
    order, both fields."""
    V1, V2, g, Lv = 40.0, 90.0, 0.02, wk.LV

    def rhs(t, y):
        T1, T2, w1, w2 = y
        return [(g * CPA * (T2 - T1) + Lv * g * (w2 - w1)) / (RHO * V1 * (CPA + CPV * w1)),
                (g * CPA * (T1 - T2) + Lv * g * (w1 - w2)) / (RHO * V2 * (CPA + CPV * w2)),
                g * (w2 - w1) / (RHO * V1), g * (w1 - w2) / (RHO * V2)]

    y0 = [300.0, 290.0, 1500.0 / PREF, 900.0 / PREF]
    t_end = 4 * 3600.0
    ex = solve_ivp(rhs, (0.0, t_end), y0, method="DOP853", rtol=1e-13, atol=1e-14).y[:, -1]
    errs = []
    for dt in (200.0, 100.0, 50.0, 25.0):
        ym = solve_ivp(rhs, (0.0, -dt), y0, method="DOP853", rtol=1e-13, atol=1e-14).y[:, -1]
        wl = _two_zones(V1, V2, g, dt)
        o = oracle_mod.Oracle(wl, n_threads=1)
        o.room[0] = [ym[0], y0[0], ym[2] * PREF, y0[2] * PREF]
        o.room[1] = [ym[1], y0[1], ym[3] * PREF, y0[3] * PREF]
        o.run(int(round(t_end / dt)))
        errs.append((max(abs(o.room[0, 1] - ex[0]), abs(o.room[1, 1] - ex[1])),
                     max(abs(o.room[0, 3] - ex[2] * PREF), abs(o.room[1, 3] - ex[3] * PREF))))
    for i in range(3):
        for f in range(2):
            assert 3.6 < errs[i][f] / errs[i + 1][f] < 4.4, (errs, i, f)


def _radiating_pair(eps, area, T0=(295.0, 285.0), hT_in=0.0):
    """Two single-layer walls, outer faces adiabatic, inner faces on one room; the room faces exchange heat
    with each other by long-wave radiation (view factor 0.2) and with the air through hT_in only."""
    walls = []
    for i in range(2):
        w = wk.uniform_wall(11, 0.05, dict(kM0=1e-11, cM0=5e-2, kTT0=0.8, cTT0=1.2e6), T0=T0[i], P0=1000.0,
                            dt=60.0, Lv=0.0, bc0=dict(hT=0.0, hM=0.0), bc1=dict(hT=hT_in, hM=0.0),
                            kinds=(wk.BC_ADIABATIC, wk.BC_ROOM))
        w.bc_room = np.array([[-1, 0]], np.int32)
        walls.append(w)
    wl = wk.concat(walls)
    wl.Lv = 0.0
    wl.rooms = dict(par=_room_row(30.0, 0.0, 0.0, 0.0, 290.0, 1000.0)[None], wall_area=np.array(area),
                    Ta0=np.array([290.0]), Pa0=np.array([1000.0]),
                    emissivity=np.array([[0.0, eps[0]], [0.0, eps[1]]]), view=np.array([0.2]))
    return wl


def test_radiation_linearised_conductance_and_reciprocity(oracle_mod):
    """For a small temperature difference the radiative flux between two surfaces is the linearised
    exchange 4 s eps sigma T^3 dT (the Stefan-Boltzmann law, sigma = 5.670374419e-8 W/m2/K4), flowing from the
    warmer to the cooler face; with equal areas and emissivities the two faces' fluxes cancel (the radiation
    moves energy between the walls and creates none)."""
    T1, dT = 293.15, 1e-3
    wl = dataclasses.replace(_radiating_pair((0.5, 0.5), (12.0, 12.0), T0=(T1, T1 + dT)), dt=1.0)
    o = oracle_mod.Oracle(wl, n_threads=1)
    r = o.run(1)
    q0, q1 = r["flux"][0, 1, 0], r["flux"][1, 1, 0]   # heat into each wall at its room face over one 1 s step
    h_r = 4 * 0.2 * 0.5 * 5.670374419e-8 * T1 ** 3
    assert abs(q0 - h_r * dT) <= 1e-3 * h_r * dT and q0 > 0       # the cooler wall gains
    assert abs(q0 + q1) <= 1e-3 * abs(q0)
    # unequal emissivities: each face takes its own emissivity
    wl = dataclasses.replace(_radiating_pair((0.5, 0.9), (12.0, 12.0), T0=(T1, T1 + dT)), dt=1.0)
    r = oracle_mod.Oracle(wl, n_threads=1).run(1)
    assert abs(r["flux"][1, 1, 0] / r["flux"][0, 1, 0] + 0.9 / 0.5) <= 1e-3


def test_radiation_equalises_the_surfaces(oracle_mod):
    """Two walls exchanging heat by radiation only (adiabatic outer faces, no air exchange): the surfaces
    converge to one temperature, between the initial ones, and the radiative fluxes vanish. Without any
    exchange to damp it, DF keeps its neutral odd-even mode ((-1)^j (-1)^n, amplification -1), so the check
    is on the mean of the two newest levels, which cancels it; the mode itself stays bounded."""
    wl = _radiating_pair((0.7, 0.7), (10.0, 10.0))
    o = oracle_mod.Oracle(wl, n_threads=1)
    for _ in range(100):
        r = o.run(2000)
    mean = [0.5 * (o.wall(w, "T", 0) + o.wall(w, "T", 1)) for w in range(2)]
    assert np.ptp(np.concatenate(mean)) < 1e-6
    assert 285.0 < mean[0][0] < 295.0
    assert np.abs(np.concatenate([o.wall(0, "T"), o.wall(1, "T")]) - mean[0][0]).max() < 0.05
    assert abs(r["flux"][0, 1, 0]) < 1e-2


def test_closed_system_balance_two_linked_rooms_with_radiation(oracle_mod):
    """Two rooms, each with its layered walls, linked by interzone airflow, their surfaces exchanging
    long-wave radiation: over one step the stored heat and vapour of all walls and both airs equal the
    outdoor fluxes + ventilation + gains + DF defects + the coupling defects of the room faces and of the
    interzone link + the radiation deposited in the walls, to 1e-12 of the term magnitudes."""
    wl = _building(Lv=2.5e6, scheme=0)
    W = wl.n_walls
    wl.bc_room = np.array([[-1, 0], [-1, 1], [-1, 1]], np.int32)
    par0 = wl.rooms["par"][0]
    par1 = _room_row(70.0, 0.8, 150.0, 1.2e-4, 279.0, 820.0, 0, T_amp=5.0, P_amp=200.0, phase_T=0.7, phase_P=2.1)
    emis = np.array([[0.0, 0.9], [0.0, 0.5], [0.0, 0.6]])
    g = 0.015
    wl.rooms = dict(par=np.stack([par0, par1]), wall_area=wl.rooms["wall_area"], Ta0=np.array([292.0, 289.0]),
                    Pa0=np.array([1400.0, 1100.0]), emissivity=emis, view=np.array([0.2, 0.3]),
                    links=[(0, 1, g)])
    o = oracle_mod.Oracle(wl, n_threads=1)
    o.run(25)
    n = o.step
    room0 = o.room[:2].copy()
    surf_prev = [(o.wall(w, "T", 1)[-1], o.wall(w, "P", 1)[-1]) for w in range(W)]
    surf_n = [(o.wall(w, "T", 0)[-1], o.wall(w, "P", 0)[-1]) for w in range(W)]
    r = o.run(1, want_balance=True)
    room1 = o.room[:2].copy()
    surf_next = [(o.wall(w, "T", 0)[-1], o.wall(w, "P", 0)[-1]) for w in range(W)]
    Lv, dt = wl.Lv, wl.dt
    t = wl.t0 + n * dt
    A = wl.rooms["wall_area"]
    sig = 5.670374419e-8
    lhs = {"T": 0.0, "P": 0.0}
    rhs = {"T": 0.0, "P": 0.0}
    mag = {"T": 0.0, "P": 0.0}
    bal, flux = r["balance"], r["flux"]
    for k, fld in enumerate(("T", "P")):
        lhs[fld] += float(np.sum(A * bal[:, k, 0]))
        for term in (np.sum(A * flux[:, 0, k]), np.sum(A * bal[:, k, 2])):
            rhs[fld] += float(term)
            mag[fld] += abs(float(term))
        mag[fld] += float(np.sum(A * bal[:, k, 3]))
    zone_of = wl.bc_room[:, 1]
    for z in range(2):
        f = dict(zip(wk.ROOM_FIELDS, wl.rooms["par"][z]))
        V, rho, Pref = f["volume"], f["rho_a"], f["Pv_ref"]
        gv = rho * V * f["ach"] / 3600.0
        T_out = f["T_out_mean"] + f["T_out_amp"] * np.sin(2 * np.pi * t / f["period"] + f["phase_T"])
        P_out = f["P_out_mean"] + f["P_out_amp"] * np.sin(2 * np.pi * t / f["period"] + f["phase_P"])
        Ta_m, Ta_n, Ta_p = room0[z, 0], room0[z, 1], room1[z, 1]
        Pa_m, Pa_n, Pa_p = room0[z, 2], room0[z, 3], room1[z, 3]
        Ta_s, Pa_s = 0.5 * (Ta_p + Ta_m), 0.5 * (Pa_p + Pa_m)
        o_z = 1 - z
        To_n, wo_n = room0[o_z, 1], room0[o_z, 3] / Pref
        store = {"T": rho * V * (f["cp_a"] + f["cp_v"] * Pa_n / Pref) * (Ta_p - Ta_m) / (2 * dt),
                 "P": rho * V / Pref * (Pa_p - Pa_m) / (2 * dt)}
        src = {"T": [f["Q_gain"], Lv * f["g_vap"], gv * f["cp_a"] * (T_out - Ta_s), Lv * gv * (P_out / Pref - Pa_s / Pref),
                     g * f["cp_a"] * (To_n - Ta_s), Lv * g * (wo_n - Pa_s / Pref)],
               "P": [f["g_vap"], gv * (P_out / Pref - Pa_s / Pref), g * (wo_n - Pa_s / Pref)]}
        for fld in ("T", "P"):
            lhs[fld] += store[fld]
            mag[fld] += abs(store[fld])
            for x in src[fld]:
                rhs[fld] += x
                mag[fld] += abs(x)
        # room-face coupling defects of this zone's walls
        for w in np.where(zone_of == z)[0]:
            hT, hM = wl.bc_par[w, 1, 0], wl.bc_par[w, 1, 1]
            sT_bar = 0.5 * (surf_next[w][0] + surf_prev[w][0])
            sP_bar = 0.5 * (surf_next[w][1] + surf_prev[w][1])
            dPp = (Pa_n - sP_bar) + (surf_n[w][1] - Pa_s)
            cT = A[w] * (hT * ((Ta_n - sT_bar) + (surf_n[w][0] - Ta_s)) + Lv * hM * dPp)
            cP = A[w] * hM * dPp
            # radiation deposited in the wall: T'^4 - Ts^4 = (T'^2 + Ts^2)(T' + Ts)(T' - Ts), conductance and
            # the other faces' values of level n, the face's own value averaged over the step
            others = [u for u in np.where(zone_of == z)[0] if u != w]
            c = wl.rooms["view"][z] * emis[w, 1] * sig
            Ts = surf_n[w][0]
            qr = c * sum((surf_n[u][0] ** 2 + Ts ** 2) * (surf_n[u][0] + Ts) * (surf_n[u][0] - sT_bar) for u in others)
            rhs["T"] += cT + A[w] * qr
            rhs["P"] += cP
            mag["T"] += abs(cT) + abs(A[w] * qr)
            mag["P"] += abs(cP)
    for fld in ("T", "P"):
        assert abs(lhs[fld] - rhs[fld]) <= 1e-12 * mag[fld], (fld, lhs[fld], rhs[fld], mag[fld])
