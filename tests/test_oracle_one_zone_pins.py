"""Oracle pins of the one-zone extensions (paper Sec. 5.2 and Appendix B): the vapour fraction of the
cross conductivity (kTM = nu Lv kM inside the wall, Lv hM at the surface), a Pv sinusoid with its own
period, and the zone's daily vapour pulse.

* a single linear wall at steady state is the exact linear solution of the coupled equations with
  Robin faces (for constant coefficients the DF fixed point is the continuous solution at the nodes);
* shifting t0 by one Pv period, with the T phase moved back by the same time, gives the same run;
* with no vapour exchange and no ventilation, the zone's vapour pressure follows the rectangle sum of
  the production (the DF node: mean of the two newest levels = start + dt / C_P * sum of g(t_k))."""
import math

import numpy as np
import pytest

from paper_1703_10119_gb300 import workloads as wk
from test_oracle_pins import _run_to_steady

import golden_data


@pytest.mark.parametrize("nu", [0.3, 1.0, 1.7])
def test_vapour_fraction_steady_state_is_exact(oracle_mod, nu):
    N, L = 11, 0.05
    kM, cM, kTT, cTT, chi, Lv = 1e-10, 1e-4, 1.0, 1e6, 8.36e4, 2.5e6
    hT0, hM0, hT1, hM1 = 20.0, 3e-8, 8.0, 2e-8
    Ta0, Pa0, Ta1, Pa1 = 300.0, 1500.0, 290.0, 900.0
    q0, g0, q1, g1 = 15.0, 2e-7, -5.0, -1e-7
    dx = L / (N - 1)
    dt = 0.4 * dx * dx * min(cTT / kTT, cM / kM)
    wl = wk.uniform_wall(N, L, dict(kM0=kM, cM0=cM, kTT0=kTT, cTT0=cTT, chi=chi), T0=295.0, P0=1200.0,
                         bc0=dict(hT=hT0, hM=hM0, T_mean=Ta0, P_mean=Pa0, period=0.0, q_inf=q0, g_inf=g0),
                         bc1=dict(hT=hT1, hM=hM1, T_mean=Ta1, P_mean=Pa1, period=0.0, q_inf=q1, g_inf=g1),
                         dt=dt, Lv=Lv)
    wl.vapour_frac = np.array([nu])
    o, r = _run_to_steady(oracle_mod, wl, chunk=20000, max_chunks=200)
    # moisture: J (in +x) = hM0 (Pa0 - P0) + g0 = kM (P0 - PL) / L = -(hM1 (Pa1 - PL) + g1)
    A = np.array([[1.0, hM0, 0.0], [1.0, -kM / L, kM / L], [-1.0, 0.0, hM1]])
    J, P0, PL = np.linalg.solve(A, [hM0 * Pa0 + g0, 0.0, hM1 * Pa1 + g1])
    # heat: Q = hT0 (Ta0 - T0) + Lv hM0 (Pa0 - P0) + q0 = kTT (T0 - TL) / L + nu Lv J
    #         = -(hT1 (Ta1 - TL) + Lv hM1 (Pa1 - PL) + q1)
    B = np.array([[1.0, hT0, 0.0], [1.0, -kTT / L, kTT / L], [-1.0, 0.0, hT1]])
    Q, T0, TL = np.linalg.solve(B, [hT0 * Ta0 + Lv * hM0 * (Pa0 - P0) + q0, nu * Lv * J,
                                    hT1 * Ta1 + Lv * hM1 * (Pa1 - PL) + q1])
    x = np.arange(N) * dx / L
    np.testing.assert_allclose(o.wall(0, "P"), P0 + (PL - P0) * x, rtol=0, atol=1e-9 * abs(Pa0 - Pa1))
    np.testing.assert_allclose(o.wall(0, "T"), T0 + (TL - T0) * x, rtol=0, atol=1e-9 * abs(Ta0 - Ta1))
    assert abs(r["flux"][0, 0, 0] - Q) <= 1e-9 * abs(Q)
    assert abs(r["flux"][0, 0, 1] - J) <= 1e-9 * abs(J)


def test_pv_period_is_its_own(oracle_mod):
    """T period 10 h, Pv period 24 h: starting one Pv period later with the T phase moved back by the
    same time replays the run."""
    pT, pP = 36000.0, 86400.0

    def case(t0, phase_T):
        layers = [dict(kM0=2e-11, a=0.5, cM0=5e-2, b=0.3, kTT0=0.8, aT=0.1, cTT0=1.2e6, chi=8.36e4)]
        bc0 = dict(hT=25.0, hM=2e-8, T_mean=285.0, T_amp=8.0, P_mean=1100.0, P_amp=300.0, period=pT,
                   phase_T=phase_T, period_P=pP, phase_P=0.4)
        bc1 = dict(hT=8.0, hM=3e-8, T_mean=293.0, T_amp=2.0, P_mean=1000.0, P_amp=100.0, period=pT,
                   phase_T=phase_T + 1.0, period_P=pP, phase_P=2.0)
        return wk.layered_wall([21], 0.1, layers, bc0=bc0, bc1=bc1, dt=300.0, t0=t0)

    a = oracle_mod.Oracle(case(0.0, 0.7), n_threads=1)
    b = oracle_mod.Oracle(case(pP, 0.7 - 2 * math.pi * pP / pT), n_threads=1)
    ra, rb = a.run(400, 10), b.run(400, 10)
    np.testing.assert_allclose(rb["samples"], ra["samples"], rtol=1e-11)
    # and the Pv period matters: the same start with the Pv period taken as the T period differs
    c = case(0.0, 0.7)
    c.bc_par[:, :, 12] = pT
    rc = oracle_mod.Oracle(c, n_threads=1).run(400, 10)
    assert np.max(np.abs(rc["samples"][..., 1] - ra["samples"][..., 1])) > 1.0


def test_zone_vapour_pulse_sum(oracle_mod):
    dt, n = 60.0, 1500
    g0, g1, on, off, per = 7e-6, 1.1e-4, 6 * 3600.0, 9 * 3600.0, 86400.0
    rho, V, Pref, P0 = 1.2, 54.0, 1.61e5, 1168.5
    wl = wk.uniform_wall(21, 0.1, dict(kM0=5e-9, cM0=6e-2, kTT0=0.4, cTT0=8.6e5), T0=293.15, P0=P0,
                         bc0=dict(hT=12.0, hM=4e-7, T_mean=290.0, P_mean=1100.0),
                         bc1=dict(hT=8.0, hM=0.0), dt=dt, t0=5 * 3600.0, kinds=(wk.BC_AMBIENT, wk.BC_ROOM))
    par = np.zeros((1, len(wk.ROOM_FIELDS)))
    row = dict(volume=V, ach=0.0, g_vap=g0, T_out_mean=290.0, P_out_mean=1100.0, rho_a=rho, cp_a=1006.0,
               cp_v=1860.0, Pv_ref=Pref, g_pulse=g1, pulse_on=on, pulse_off=off, pulse_period=per)
    par[0] = [row.get(k, 0.0) for k in wk.ROOM_FIELDS]
    wl.bc_room = np.array([[-1, 0]], np.int32)
    wl.rooms = dict(par=par, wall_area=np.array([20.0]), Ta0=np.array([293.15]), Pa0=np.array([P0]))
    o = oracle_mod.Oracle(wl, n_threads=1)
    o.run(n)
    t = wl.t0 + dt * np.arange(n)
    g = g0 + g1 * ((np.mod(t, per) >= on) & (np.mod(t, per) < off))
    expect = P0 + dt * Pref / (rho * V) * g.sum()
    mean = 0.5 * (o.room[0, 2] + o.room[0, 3])
    assert abs(mean - expect) <= 1e-12 * expect
    assert 100 < np.count_nonzero(g > g0) < n   # the window opened and closed inside the run


def test_one_zone_workload_takes_the_printed_set_up():
    """The one-zone inputs carry the printed values of tests/golden/one_zone_table2_appendix_b.txt (Sec. 5.2
    and its Table 2): per wall the linear coefficients (cTM as chi cM, kTM as the vapour fraction
    nu = kTM / (Lv kM)), area and outdoor exchange; the zone's volume, exchange, load and ventilation."""
    g = golden_data.load("one_zone_table2_appendix_b.txt")
    z = g["zone"]["zone"]
    wl = wk.one_zone()
    Lv = wl.Lv
    table = [g["table2"][n] for n in ("north", "south", "east", "east")]   # west = east (one column)
    lp = wl.layer_par                                                      # one layer per wall
    col = {k: i for i, k in enumerate(wk.LAYER_FIELDS)}
    bcol = {k: i for i, k in enumerate(wk.BC_FIELDS)}
    rcol = {k: i for i, k in enumerate(wk.ROOM_FIELDS)}
    assert wl.n_walls == 4 and lp.shape[0] == 4
    for w, t in enumerate(table):
        assert lp[w, col["cM0"]] == t["cM"] and lp[w, col["kM0"]] == t["kM"]
        assert lp[w, col["cTT0"]] == t["cTT"] and lp[w, col["kTT0"]] == t["kTT"]
        assert lp[w, col["a"]] == lp[w, col["b"]] == lp[w, col["aT"]] == lp[w, col["bT"]] == 0.0
        assert abs(lp[w, col["chi"]] * t["cM"] - t["cTM"]) <= 1e-12 * t["cTM"]
        assert abs(wl.vapour_frac[w] * Lv * t["kM"] - t["kTM"]) <= 1e-12 * t["kTM"]
        assert wl.rooms["wall_area"][w] == t["A"]
        assert wl.bc_par[w, 0, bcol["hT"]] == t["hT"] and wl.bc_par[w, 0, bcol["hM"]] == t["hM"]
        assert wl.bc_par[w, 1, bcol["hT"]] == z["hT_in"] and wl.bc_par[w, 1, bcol["hM"]] == z["hM_in"]
        assert wl.bc_kind[w, 0] == wk.BC_AMBIENT and wl.bc_kind[w, 1] == wk.BC_ROOM
        assert abs(wl.thickness[w] - z["L"]) < 1e-15
    r = wl.rooms["par"][0]
    assert r[rcol["volume"]] == z["volume"] and r[rcol["ach"]] == z["ach"]
    assert abs(r[rcol["g_vap"]] * 3.6e6 - z["g_base"]) < 1e-9            # kg/s -> g/h
    assert abs(r[rcol["g_pulse"]] * 3.6e6 - z["g_extra"]) < 1e-9
    assert r[rcol["pulse_on"]] == 3600.0 * z["extra_on"] and r[rcol["pulse_off"]] == 3600.0 * z["extra_off"]
    assert r[rcol["pulse_period"]] == 86400.0
    Ti = 273.15 + z["Ti_C"]
    assert np.all(wl.T_init == Ti) and abs(wl.rooms["Ta0"][0] - Ti) < 1e-12
    assert np.allclose(wl.P_init, z["phi_i"] * wk.PSAT_REF, rtol=1e-15)
