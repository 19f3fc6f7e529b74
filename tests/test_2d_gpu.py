"""GPU parity of the 2D sections: the temporally blocked TMA kernel against the FP64 2D oracle.

Tolerances (relative L-infinity per field, max |x - x_ref| / max |x_ref| over every node of every
section, both stored levels): FP64 1e-12, FP32 1e-4. Fused steps per launch change only where the
work is done, not the arithmetic of a node, so every blocking depth gives the same bits.
"""
import dataclasses

import numpy as np
import pytest

from paper_1703_10119_gb300 import workloads as wk

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-4}


@pytest.fixture(scope="module")
def H():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_10119_gb300 import build, hygro

    build.build()
    return hygro


def relinf(x, ref):
    return float(np.max(np.abs(np.asarray(x, np.float64) - ref)) / np.max(np.abs(ref)))


def mixed_sections(G, nx, ny, n_steps, seed=5, n_regions=4, dt=60.0, h=1e-3):
    """Sections with every term switched on: random rectangular regions (interfaces in both
    directions, some one node wide), Pv-dependent kTT and cTT, cTM storage, q_inf and g_inf, noisy
    ambient air on faces 0 and 2, sinusoidal air or no flux on faces 1 and 3, per-grid initial states."""
    rng = np.random.default_rng(seed)
    region = np.zeros((G, ny, nx), np.uint8)
    for g in range(G):
        for r in range(1, n_regions):
            for _ in range(2):
                x0, y0 = rng.integers(0, nx), rng.integers(0, ny)
                region[g, y0:y0 + rng.integers(1, max(2, ny // 2)), x0:x0 + rng.integers(1, max(2, nx // 2))] = r
    par = np.zeros((G, n_regions, 9))
    for g in range(G):
        for r in range(n_regions):
            par[g, r] = [10 ** rng.uniform(-12, -10), rng.uniform(0, 2), 10 ** rng.uniform(*wk.CM0_LOG10_RANGE),
                         rng.uniform(0, 2), rng.uniform(0.04, 2), rng.uniform(0, 0.3), rng.uniform(1e5, 2e6),
                         rng.uniform(0, 0.3), 8.36e4]
    kinds = np.zeros((G, 4), np.int32)
    bc = np.zeros((G, 4, len(wk.BC_FIELDS)))
    for g in range(G):
        for f in range(4):
            kinds[g, f] = wk.BC_AMBIENT if f in (0, 2) or (g + f) % 3 == 0 else wk.BC_ADIABATIC
            bc[g, f] = [rng.uniform(5, 25), rng.uniform(1e-8, 3e-8), rng.uniform(-20, 20), rng.uniform(-1e-7, 1e-7),
                        rng.uniform(285, 300), rng.uniform(2, 10), rng.uniform(900, 1300), rng.uniform(100, 400),
                        rng.choice([86400.0, 3600.0 * 7]), rng.uniform(0, 6.28), rng.uniform(0, 6.28), 1800.0,
                        rng.choice([0.0, 3600.0 * 5])]
    nl = int(np.ceil(n_steps * dt / 1800.0)) + 2
    nz0 = np.stack([rng.normal(0, 1.0, (G, nl)), rng.normal(0, 50.0, (G, nl))], -1).astype(np.float32)
    nz2 = np.stack([rng.normal(0, 1.0, (G, nl)), rng.normal(0, 50.0, (G, nl))], -1).astype(np.float32)
    return wk.Section2D(name="mixed 2D test sections", h=h, region=region, region_par=par, bc_kind=kinds,
                        bc_par=bc, noise=[nz0, None, nz2, None], T_init=rng.uniform(285, 300, G),
                        P_init=rng.uniform(800, 1300, G), dt=dt, t0=0.0, n_steps=n_steps)


def run_gpu(H, sec, precision, n_steps, k=0, pieces=None):
    with H.Hygro2D(sec, precision=precision, steps_per_launch=k) as g:
        for n in (pieces or [n_steps]):
            g.run(n)
        g.sync()
        assert g.step == n_steps
        return g.fields(0), g.fields(1)


def run_oracle(oracle_mod, sec, n_steps):
    o = oracle_mod.Oracle2D(sec)
    o.run(n_steps)
    return (o.T_cur, o.P_cur), (o.T_prev, o.P_prev)


def check(got, ref, tol, what):
    for lev in range(2):
        for f, name in ((0, "T"), (1, "P")):
            e = relinf(got[lev][f], ref[lev][f])
            assert e <= tol, f"{what}: level {lev} {name} rel Linf {e:.3e} > {tol:g}"


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mixed_sections_match_oracle(H, oracle_mod, precision):
    # 150 x 130: several 64-wide (32-wide in FP64) tiles in each direction and ragged last tiles;
    # 37 steps: full launches and a shorter last one
    sec = mixed_sections(3, 150, 130, 37)
    got = run_gpu(H, sec, precision, 37)
    ref = run_oracle(oracle_mod, sec, 37)
    check(got, ref, TOL[precision], f"mixed {precision}")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_blocking_depth_does_not_change_the_bits(H, precision):
    sec = mixed_sections(2, 97, 70, 24, seed=9)
    base = run_gpu(H, sec, precision, 24, k=1)
    for k in (2, 3, 4):
        got = run_gpu(H, sec, precision, 24, k=k)
        for lev in range(2):
            for f in range(2):
                assert np.array_equal(got[lev][f], base[lev][f]), f"k={k} level {lev} field {f}"
    # calls of uneven length continue the same sequence
    got = run_gpu(H, sec, precision, 24, pieces=[5, 1, 11, 7])
    for lev in range(2):
        for f in range(2):
            assert np.array_equal(got[lev][f], base[lev][f])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_intervals_give_the_same_bits(H, precision):
    """Runs whose whole intervals are replayed from CUDA graphs (2 and 6 launches per interval) against
    single launches: the same bits and the same step, over calls that start on either buffer set (an odd
    call in between flips the sets), with the step index of each replay read from the device."""
    sec = mixed_sections(2, 97, 70, 80, seed=13)
    pieces = [17, 3, 26, 34]   # 4-step launches: intervals of 8 and 24 steps, remainders, an odd launch count
    ref = run_gpu(H, sec, precision, 80, k=4, pieces=pieces)
    with H.Hygro2D(sec, precision=precision, steps_per_launch=4) as g0:
        g0.set_option(H.HYGRO2D_OPT_GRAPH_LAUNCHES, 0)
        for n in pieces:
            g0.run(n)
        g0.sync()
        plain = g0.fields(0), g0.fields(1)
    for launches in (2, 6):
        with H.Hygro2D(sec, precision=precision, steps_per_launch=4) as g:
            g.set_option(H.HYGRO2D_OPT_GRAPH_LAUNCHES, launches)
            assert g.option(H.HYGRO2D_OPT_GRAPH_LAUNCHES) == launches
            for n in pieces:
                g.run(n)
            g.sync()
            assert g.step == 80
            got = g.fields(0), g.fields(1)
        for lev in range(2):
            for f in range(2):
                assert np.array_equal(got[lev][f], plain[lev][f]), (launches, lev, f)
                assert np.array_equal(got[lev][f], ref[lev][f]), (launches, lev, f)


def test_graph_option_validation(H):
    sec = mixed_sections(1, 40, 30, 4, seed=3)
    with H.Hygro2D(sec, precision="fp32") as g:
        for opt, bad in ((H.HYGRO2D_OPT_GRAPH_LAUNCHES, 3), (H.HYGRO2D_OPT_GRAPH_LAUNCHES, -2),
                         (H.HYGRO2D_OPT_GRAPH_LAUNCHES, 4098), (H.HYGRO2D_OPT_STEPS_PER_LAUNCH, 0),
                         (H.HYGRO2D_OPT_STEPS_PER_LAUNCH, 5), (99, 1)):
            with pytest.raises(H.HygroError) as e:
                g.set_option(opt, bad)
            assert e.value.status == H.HYGRO_E_INVALID
        assert g.option(H.HYGRO2D_OPT_GRAPH_LAUNCHES) == 64
        assert g.option(H.HYGRO2D_OPT_STEPS_PER_LAUNCH) == 4


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_autotune_keeps_state_and_bits(H, precision):
    """The depth autotuner times every depth from the current state and restores it: afterwards the stored
    levels and the step are as before, and the run that follows gives the bits of a run at any depth."""
    sec = mixed_sections(2, 150, 130, 40, seed=17)
    ref = run_gpu(H, sec, precision, 40, k=1, pieces=[9, 31])
    with H.Hygro2D(sec, precision=precision, steps_per_launch=1) as g:
        g.run(9)
        g.sync()
        before = g.fields(0), g.fields(1)
        k, ms = g.autotune(6)
        assert 1 <= k <= 4 and g.option(H.HYGRO2D_OPT_STEPS_PER_LAUNCH) == k
        assert np.all(ms > 0) and ms[k - 1] == ms.min()
        assert g.step == 9
        after = g.fields(0), g.fields(1)
        for lev in range(2):
            for f in range(2):
                assert np.array_equal(after[lev][f], before[lev][f])
        g.run(31)
        g.sync()
        got = g.fields(0), g.fields(1)
    for lev in range(2):
        for f in range(2):
            assert np.array_equal(got[lev][f], ref[lev][f])


@pytest.mark.parametrize("shape", [(2, 2), (3, 2), (64, 64), (65, 63), (8, 200), (200, 5)])
def test_edge_shapes(H, oracle_mod, shape):
    nx, ny = shape
    sec = mixed_sections(2, nx, ny, 19, seed=nx * 1000 + ny, n_regions=2)
    ref = run_oracle(oracle_mod, sec, 19)
    for precision in ("fp64", "fp32"):
        check(run_gpu(H, sec, precision, 19), ref, TOL[precision], f"{shape} {precision}")


def test_corner_workload_reduced_matches_oracle(H, oracle_mod):
    # the thermal-bridge generator at 4 sections of 192 x 160 (ragged tiles), 64 steps
    sec = wk.sections_2d(n_grids=4, nx=192, ny=160, n_steps=64)
    ref = run_oracle(oracle_mod, sec, 64)
    for precision in ("fp64", "fp32"):
        check(run_gpu(H, sec, precision, 64), ref, TOL[precision], f"corner {precision}")


def test_full_size_corner_batch_on_sampled_sections(H, oracle_mod):
    """All 64 sections of 512 x 512 on the GPU in the benchmark's launch configuration (4 fused
    steps, FP32); the oracle advances three of them (the first, a middle and the last)."""
    n = 48
    sec = wk.sections_2d(n_steps=n)
    got = run_gpu(H, sec, "fp32", n)
    pick = [0, 31, 63]
    ref = run_oracle(oracle_mod, sec.subset(pick), n)
    for lev in range(2):
        for f, name in ((0, "T"), (1, "P")):
            e = relinf(got[lev][f][pick], ref[lev][f])
            assert e <= TOL["fp32"], f"level {lev} {name}: {e:.3e}"


def test_fields_round_trip_and_restart(H, oracle_mod):
    """Levels read after 12 steps and written into a fresh context whose clock starts at t0 + 12 dt
    continue the run: 18 more steps match the oracle's 30."""
    sec = mixed_sections(2, 70, 66, 30, seed=21)
    ref = run_oracle(oracle_mod, sec, 30)
    with H.Hygro2D(sec, precision="fp64") as g:
        g.run(12)
        (T0, P0), (T1, P1) = g.fields(0), g.fields(1)
    with H.Hygro2D(dataclasses.replace(sec, t0=sec.t0 + 12 * sec.dt), precision="fp64") as g2:
        g2.set_fields(0, T0, P0)
        g2.set_fields(1, T1, P1)
        assert np.array_equal(g2.fields(0)[0], T0) and np.array_equal(g2.fields(1)[1], P1)
        g2.run(18)
        got = g2.fields(0), g2.fields(1)
    check(got, ref, TOL["fp64"], "restart")


def test_invalid_calls_change_nothing(H):
    sec = mixed_sections(1, 20, 20, 4, seed=3, n_regions=2)
    with H.Hygro2D(sec, precision="fp32") as g:
        g.run(4)
        before = g.fields(0)
        bad = sec.region.copy()
        bad[0, 3, 3] = 7
        lay = (H.hygro_layer * 2)()
        for i in range(2):
            lay[i] = H.hygro_layer(*[float(x) for x in sec.region_par[0, i]])
        with pytest.raises(H.HygroError) as e:
            H.hygro2d_set_materials(g.ctx, 2, bad, lay, np.array([293.0]), np.array([1000.0]))
        assert e.value.status == H.HYGRO_E_INVALID
        room = H._bc_array(1, [wk.BC_ROOM], sec.bc_par[:, 0], None)
        with pytest.raises(H.HygroError) as e:
            H.hygro2d_set_bc(g.ctx, 0, room)
        assert e.value.status == H.HYGRO_E_INVALID
        with pytest.raises(H.HygroError):
            H.hygro2d_set_bc(g.ctx, 4, room)
        with pytest.raises(H.HygroError):
            H.hygro2d_run(g.ctx, -1)
        after = g.fields(0)
        assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
        assert g.step == 4


def test_nonfinite_is_reported(H):
    sec = mixed_sections(1, 20, 20, 4, seed=4, n_regions=2)
    sec.bc_par[0, 0, 2] = 1e39   # q_inf beyond the FP32 range: the FP32 path turns it into infinity
    with H.Hygro2D(sec, precision="fp32") as g:
        g.run(2)
        with pytest.raises(H.HygroError) as e:
            g.sync()
        assert e.value.status == H.HYGRO_E_NONFINITE
        g.sync()   # the flag is cleared once reported
