"""GPU parity of the paper's one-zone case (Sec. 5.2, Table 2, Appendix B) and of the features it adds
(the vapour fraction of the cross conductivity, a Pv sinusoid with its own period, the zone's daily
vapour pulse) against the FP64 oracle. Tolerances as the other parity tests: FP64 1e-12, FP32 1e-4
relative L-infinity."""
import numpy as np
import pytest

from paper_1703_10119_gb300 import workloads as wk

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-4)])
def test_one_zone_80_hours(H, oracle_mod, precision, tol):
    """All 80 hours at dt = 3.6 s: hourly surface samples, the final wall fields and zone air, fluxes."""
    wl = wk.one_zone()
    with H.Hygro(wl, precision=precision) as g:
        s = g.run_sampled(wl.n_steps, 1000)
        T, P = g.fields(0)
        Ta, Pa = g.rooms(0)
        Ta1, Pa1 = g.rooms(1)
        _, cum = g.fluxes()
    o = oracle_mod.Oracle(wl)
    r = o.run(wl.n_steps, 1000)
    assert relinf(s, r["samples"]) <= tol
    assert relinf(T, o.T_cur) <= tol and relinf(P, o.P_cur) <= tol
    assert relinf(Ta, o.room[:, 1]) <= tol and relinf(Pa, o.room[:, 3]) <= tol
    assert relinf(Ta1, o.room[:, 0]) <= tol and relinf(Pa1, o.room[:, 2]) <= tol
    assert np.max(np.abs(cum - o.cumul)) <= 50 * tol * np.max(np.abs(o.cumul))
    # the zone's vapour pressure rises while the load pulse is on (6 h to 9 h of each day)
    ref = r["room_samples"][:, 0, 1]
    assert ref[8] > ref[5] + 20.0


@pytest.mark.parametrize("kernel", ["persistent", "plain"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-4)])
def test_vapour_fraction_ragged_walls(H, oracle_mod, kernel, precision, tol):
    """Walls of 3..512 nodes (1-3 layers, cTM on) with vapour fractions 0..1.6 and Pv periods of their own."""
    import test_parity_gpu as par

    wl = par.ragged_batch([3, 5, 17, 33, 64, 100, 257, 400, 512], 60, dt=600.0)
    wl.vapour_frac = np.linspace(0.0, 1.6, wl.n_walls)
    wl.bc_par[:, 0, 12] = 3600.0 * 17
    with H.Hygro(wl, precision=precision, kernel=kernel) as g:
        s = g.run_sampled(60, 6)
        T, P = g.fields(0)
        _, cum = g.fluxes()
    o = oracle_mod.Oracle(wl, n_threads=1)
    r = o.run(60, 6)
    assert relinf(s, r["samples"]) <= tol
    assert relinf(T, o.T_cur) <= tol and relinf(P, o.P_cur) <= tol
    assert np.max(np.abs(cum - o.cumul)) <= 50 * tol * np.max(np.abs(o.cumul))


def test_vapour_fraction_balance_and_start(H, oracle_mod):
    """The balance of the next step and the Euler-substep start with vapour fractions != 1 (FP64)."""
    import test_parity_gpu as par

    wl = par.ragged_batch([3, 6, 17, 40, 65, 120], 30, dt=60.0)
    wl.vapour_frac = np.array([0.2, 0.5, 0.9, 1.0, 1.3, 0.05])
    with H.Hygro(wl, precision="fp64") as g:
        g.start_euler()
        T1, P1 = g.fields(0)
        g.run(20)
        bal = g.balance()
    o = oracle_mod.Oracle(wl, n_threads=1)
    o.euler_start(1.0)
    assert relinf(T1, o.T_cur) <= 1e-12 and relinf(P1, o.P_cur) <= 1e-12
    o.run(20)
    ref = o.run(1, want_balance=True)["balance"]
    S, B, D, M = bal[..., 0], bal[..., 1], bal[..., 2], bal[..., 3]
    assert np.all(np.abs(S - B - D) <= 1e-12 * M)
    for k in range(3):
        assert np.all(np.abs(bal[..., k] - ref[..., k]) <= 1e-9 * ref[..., 3]), k


def test_vapour_fraction_validation_and_adjoint(H):
    wl = wk.single_wall()
    with H.Hygro(wl, precision="fp64") as g:
        for bad in (np.array([-0.1]), np.array([np.nan])):
            with pytest.raises(H.HygroError) as e:
                H.hygro_set_vapour_fraction(g.ctx, bad)
            assert e.value.status == H.HYGRO_E_INVALID
        H.hygro_set_vapour_fraction(g.ctx, np.array([0.5]))
        obs = np.zeros((2, 1, 2, 2), np.float32)
        with pytest.raises(H.HygroError) as e:
            g.loss_grad(20, 10, obs, 1.0, 1e-4)
        assert e.value.status == H.HYGRO_E_UNSUPPORTED
