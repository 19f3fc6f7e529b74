"""GPU parity: the CUDA library against the FP64 oracle on the same seeded inputs.

Tolerances (relative L-infinity per field, max |x - x_ref| / max |x_ref| over
all nodes of all walls, and over all samples):
  * FP64 kernels: 1e-12;
  * FP32 kernel: 1e-4 (fields and samples) after the whole horizon.
Fluxes are compared relative to the largest flux of the batch, their running sums relative to the
largest sum: FP64 1e-9; FP32 5e-5 (last step's fluxes, largest measured 8.7e-6) and 1e-3 (running sums,
largest measured 2.1e-4, on the single wall whose day-long net sums are small against the gross flux).
"""
import dataclasses

import numpy as np
import pytest

from paper_1703_10119_gb300 import workloads as wk

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-4}
COMBOS = [("fp64", "plain"), ("fp64", "persistent"), ("fp32", "persistent"), ("fp32", "plain")]


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


def ragged_batch(Ns, n_steps, seed=7, dt=600.0, simple_heat=False):
    """Walls with the given node counts, 1-3 layers (some a single node thick),
    noisy sinusoidal face 0, sinusoidal face 1, a few adiabatic faces, and all
    coefficient terms switched on (Pv slopes of kTT, cTT, cTM storage, q_inf, g_inf);
    with simple_heat, kTT and cTT are constant and cTM = 0 (the benchmark's materials)."""
    rng = np.random.default_rng(seed)
    walls = []
    for i, N in enumerate(Ns):
        nl = 1 + i % 3 if N >= 3 else 1
        cuts = np.sort(rng.choice(np.arange(1, N), size=nl - 1, replace=False)) if nl > 1 else np.array([], int)
        counts = np.diff(np.concatenate([[0], cuts, [N]])).astype(int).tolist()
        layers = []
        for _ in counts:
            layers.append(dict(kM0=10 ** rng.uniform(-12, -10), a=rng.uniform(0, 2),
                               cM0=10 ** rng.uniform(*wk.CM0_LOG10_RANGE), b=rng.uniform(0, 2),
                               kTT0=rng.uniform(0.04, 2), aT=rng.uniform(0, 0.3), cTT0=rng.uniform(1e5, 2e6),
                               bT=rng.uniform(0, 0.3), chi=8.36e4))
            if simple_heat:
                layers[-1].update(aT=0.0, bT=0.0, chi=0.0)
        bc0 = dict(hT=25.0, hM=2e-8, T_mean=293.0, T_amp=10.0, P_mean=1200.0, P_amp=400.0,
                   phase_T=rng.uniform(0, 6.28), phase_P=rng.uniform(0, 6.28), q_inf=rng.uniform(-30, 30),
                   g_inf=rng.uniform(-2e-7, 2e-7))
        bc1 = dict(hT=8.0, hM=3e-8, T_mean=295.0, T_amp=3.0, P_mean=1000.0, P_amp=150.0, period=3600.0 * 7,
                   phase_P=rng.uniform(0, 6.28))
        kinds = [wk.BC_AMBIENT, wk.BC_AMBIENT]
        if i % 7 == 3:
            kinds[1] = wk.BC_ADIABATIC
        if i % 11 == 5:
            kinds[0] = wk.BC_ADIABATIC
        w = wk.layered_wall(counts, rng.uniform(0.05, 0.4), layers, dt=dt, n_steps=n_steps,
                            T0=rng.uniform(285, 300), P0=rng.uniform(800, 1300), bc0=bc0, bc1=bc1, kinds=kinds)
        nz = np.stack([rng.normal(0, 1.0, 80), rng.normal(0, 50.0, 80)], -1).astype(np.float32)
        w.noise = [nz[None], None]
        walls.append(w)
    return wk.concat(walls, name="ragged test batch")


EDGE_NS = [3, 4, 5, 17, 31, 32, 33, 47, 64, 65, 96, 97, 100, 129, 160, 200, 255, 256, 257, 300, 383, 384, 385,
           400, 416, 450, 480, 481, 500, 511, 512]


def _compare(H, oracle_mod, wl, precision, kernel, n_steps, sample_every, splits=None):
    g = H.Hygro(wl, precision=precision, kernel=kernel)
    splits = splits or [n_steps]
    samples = []
    for s in splits:
        samples.append(g.run_sampled(s, sample_every))
    samples = np.concatenate(samples)
    T0, P0 = g.fields(0)
    T1, P1 = g.fields(1)
    flux, cum = g.fluxes()
    assert g.step == n_steps
    g.close()
    o = oracle_mod.Oracle(wl)
    rs = [o.run(s, sample_every) for s in splits]
    ref_samples = np.concatenate([r["samples"] for r in rs])
    tol = TOL[precision]
    errs = dict(T=relinf(T0, o.T_cur), P=relinf(P0, o.P_cur), Tm1=relinf(T1, o.T_prev), Pm1=relinf(P1, o.P_prev),
                sT=relinf(samples[..., 0], ref_samples[..., 0]), sP=relinf(samples[..., 1], ref_samples[..., 1]))
    errs.update(flux=relinf(flux, rs[-1]["flux"]), cum=relinf(cum, o.cumul))
    print(f"measured-error {wl.name} {precision} {kernel} " + " ".join(f"{k}={v:.3e}" for k, v in errs.items()))
    for k in ("T", "P", "Tm1", "Pm1", "sT", "sP"):
        assert errs[k] <= tol, (precision, kernel, k, errs[k], errs)
    ftol, ctol = (1e-9, 1e-9) if precision == "fp64" else (5e-5, 1e-3)
    assert errs["flux"] <= ftol, errs["flux"]
    assert errs["cum"] <= ctol, errs["cum"]
    return errs


@pytest.mark.parametrize("precision,kernel", COMBOS)
def test_single_wall(H, oracle_mod, precision, kernel):
    wl = wk.single_wall()
    _compare(H, oracle_mod, wl, precision, kernel, 1440, 60)


@pytest.mark.parametrize("simple_heat", [False, True])
@pytest.mark.parametrize("precision,kernel", COMBOS)
def test_ragged_batch_all_lane_layouts(H, oracle_mod, precision, kernel, simple_heat):
    """Walls of 3..512 nodes: every nodes-per-lane count 1..16, short lanes, unused lanes,
    interfaces inside lanes and on lane boundaries, adiabatic faces; an odd split of the run.
    Both the general and the simple-heat (constant kTT, cTT, no cTM) persistent variants."""
    wl = ragged_batch(EDGE_NS, 401, simple_heat=simple_heat)
    _compare(H, oracle_mod, wl, precision, kernel, 401, 7, splits=[200, 201])


def test_wall_batch_full_size_sampled(H, oracle_mod):
    """Full configuration (4096 walls, 52560 steps, FP32 persistent, the benchmark launch) against
    the oracle on a sample of walls (walls are independent, so the subset is exact)."""
    wl = wk.wall_batch()
    g = H.Hygro(wl, precision="fp32", kernel="persistent")
    samples = g.run_sampled(wl.n_steps, 1440)
    T, P = g.fields(0)
    g.close()
    order = np.argsort(wl.n_nodes)
    pick = np.unique(np.concatenate([order[:3], order[-3:], np.where(wl.n_layers == 3)[0][:3],
                                     np.arange(0, wl.n_walls, 683)]))
    sub = wl.subset(pick)
    o = oracle_mod.Oracle(sub)
    r = o.run(wl.n_steps, 1440)
    off = np.concatenate([[0], np.cumsum(wl.n_nodes)])
    Tg = np.concatenate([T[off[w]:off[w + 1]] for w in pick])
    Pg = np.concatenate([P[off[w]:off[w + 1]] for w in pick])
    assert relinf(Tg, o.T_cur) <= 1e-4
    assert relinf(Pg, o.P_cur) <= 1e-4
    assert relinf(samples[:, pick], r["samples"]) <= 1e-4


@pytest.mark.parametrize("kernel", ["plain", "persistent"])
def test_wall_batch_full_size_fp64_sampled(H, oracle_mod, kernel):
    """The FP64 kernels at full size against the oracle on a sample of walls, to 1e-12."""
    wl = wk.wall_batch()
    g = H.Hygro(wl, precision="fp64", kernel=kernel)
    g.run(wl.n_steps)
    T, P = g.fields(0)
    g.close()
    pick = np.array([0, 1, 2, 1000, 2047, 4095])
    o = oracle_mod.Oracle(wl.subset(pick))
    o.run(wl.n_steps)
    off = np.concatenate([[0], np.cumsum(wl.n_nodes)])
    Tg = np.concatenate([T[off[w]:off[w + 1]] for w in pick])
    Pg = np.concatenate([P[off[w]:off[w + 1]] for w in pick])
    assert relinf(Tg, o.T_cur) <= 1e-12
    assert relinf(Pg, o.P_cur) <= 1e-12


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_checkpoint_resume_bit_exact(H, precision):
    wl = ragged_batch(EDGE_NS[::3], 300, seed=3)
    g = H.Hygro(wl, precision=precision)
    g.run(100)
    img = g.get_state()
    g.run(57)
    Ta, Pa = g.fields(0)
    Tb_, Pb_ = g.fields(1)
    g.set_state(img)
    assert g.step == 100
    g.run(57)
    Tb, Pb = g.fields(0)
    assert np.array_equal(Ta, Tb) and np.array_equal(Pa, Pb)
    h = H.Hygro(wl, precision=precision)
    h.run(157)
    Tc, Pc = h.fields(0)
    Tc1, Pc1 = h.fields(1)
    assert np.array_equal(Ta, Tc) and np.array_equal(Pa, Pc)
    assert np.array_equal(Tb_, Tc1) and np.array_equal(Pb_, Pc1)
    g.close()
    h.close()


def test_zero_steps_and_invalid_calls_leave_state(H):
    wl = ragged_batch(EDGE_NS[:6], 10)
    g = H.Hygro(wl, precision="fp64")
    g.run(5)
    T0, P0 = g.fields(0)
    g.run(0)
    with pytest.raises(H.HygroError) as e:
        g.run(10, 3, np.zeros(4, np.float64))          # samples buffer too small
    assert e.value.status == H.HYGRO_E_INVALID
    with pytest.raises(H.HygroError):
        g.run(-1)
    assert g.step == 5
    T1, P1 = g.fields(0)
    assert np.array_equal(T0, T1) and np.array_equal(P0, P1)
    g.close()


def test_set_fields_one_step_matches_oracle(H, oracle_mod):
    wl = ragged_batch(EDGE_NS[::2], 1, seed=9)
    rng = np.random.default_rng(1)
    n = wl.total_nodes
    lv = [293 + rng.uniform(-5, 5, n), 293 + rng.uniform(-5, 5, n), 1000 + rng.uniform(-200, 200, n),
          1000 + rng.uniform(-200, 200, n)]
    for precision, kernel in COMBOS:
        g = H.Hygro(wl, precision=precision, kernel=kernel)
        g.set_fields(1, lv[0], lv[2])
        g.set_fields(0, lv[1], lv[3])
        g.run(1)
        T, P = g.fields(0)
        g.close()
        o = oracle_mod.Oracle(wl)
        o.set_levels(lv[0], lv[1], lv[2], lv[3])
        o.run(1)
        tol = 1e-13 if precision == "fp64" else 1e-5
        assert relinf(T, o.T_cur) <= tol and relinf(P, o.P_cur) <= tol, (precision, kernel)


def test_nonfinite_is_reported(H):
    """cM0 = 1e-4 with strongly nonlinear kM at dt = 600 s: the DF moisture update diverges."""
    wl = wk.uniform_wall(101, 0.1, dict(kM0=2e-10, a=2.0, cM0=1e-4, b=0.0, kTT0=1.0, cTT0=1e6), dt=600.0,
                         bc0=dict(hT=25, hM=2e-8, P_mean=1900.0), bc1=dict(hT=8, hM=3e-8))
    g = H.Hygro(wl, precision="fp32")
    g.run(3000)
    with pytest.raises(H.HygroError) as e:
        g.sync()
    assert e.value.status == H.HYGRO_E_NONFINITE
    g.sync()   # the flag is cleared once reported
    g.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_balance_of_the_next_step(H, oracle_mod, precision, tol):
    """hygro_balance: storage, boundary flux and DF defect of the step n -> n+1 per wall, against the oracle's
    balance of the same step (FP64), and the identity S = B + D on the GPU's own terms; the call changes
    nothing."""
    wl = ragged_batch([3, 5, 17, 33, 64, 100, 257, 400, 512], 40, dt=600.0)
    with H.Hygro(wl, precision=precision, kernel="persistent") as g:
        g.run(37)
        before = g.fields(0), g.fields(1), g.fluxes()
        bal = g.balance()
        after = g.fields(0), g.fields(1), g.fluxes()
        assert g.step == 37
        for x, y in zip(before, after):
            assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
    S, B, D, M = bal[..., 0], bal[..., 1], bal[..., 2], bal[..., 3]
    assert np.all(np.abs(S - B - D) <= tol * M)
    if precision == "fp64":
        o = oracle_mod.Oracle(wl, n_threads=1)
        o.run(37)
        ref = o.run(1, want_balance=True)["balance"]
        # the terms are sums of differences of fields that agree to ~1e-12 of their own size, summed in
        # another order: 1e-9 of M separates rounding from a wrong term (which would be off by O(M))
        for k in range(3):
            assert np.all(np.abs(bal[..., k] - ref[..., k]) <= 1e-9 * ref[..., 3]), k


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-4)])
def test_euler_start_matches_oracle(H, oracle_mod, precision, tol):
    """hygro_start_euler (the first step by explicit Euler substeps) then DF steps, against the oracle."""
    wl = ragged_batch([3, 6, 17, 40, 65, 120], 30, dt=60.0)
    with H.Hygro(wl, precision=precision, kernel="persistent") as g:
        g.start_euler()
        assert g.step == 1
        T1, P1 = g.fields(0)
        T0, P0 = g.fields(1)
        s = g.run_sampled(24, 6)
        T, P = g.fields(0)
        _, cum = g.fluxes()
        with pytest.raises(H.HygroError) as e:
            g.start_euler()
        assert e.value.status == H.HYGRO_E_STATE
    o = oracle_mod.Oracle(wl, n_threads=1)
    o.euler_start(1.0)
    assert relinf(T0, o.T_prev) == 0.0 and relinf(P0, o.P_prev) == 0.0
    assert relinf(T1, o.T_cur) <= tol and relinf(P1, o.P_cur) <= tol
    r = o.run(24, 6)
    assert relinf(T, o.T_cur) <= tol and relinf(P, o.P_cur) <= tol
    assert relinf(s, r["samples"]) <= tol
    assert np.max(np.abs(cum - o.cumul)) <= 50 * tol * np.max(np.abs(o.cumul))
