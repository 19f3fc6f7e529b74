"""Pins of the FP64 adjoint oracle (sensor-misfit loss and its gradient with respect to the layer
parameters, by the reverse-time sweep of the DF step).

What fixes the gradient independently of the adjoint code:
* the loss itself equals the misfit of the samples of the forward oracle (pinned in
  test_oracle_pins.py), so the adjoint differentiates the scheme the oracle runs;
* the directional derivatives of a second implementation, the forward run in dual numbers
  (value, derivative), agree with central finite differences of the loss;
* the adjoint gradient projected on any direction equals the dual-number derivative along it, and each
  component equals a central finite difference of the forward oracle's loss.
"""
import numpy as np
import pytest

from paper_1703_10119_gb300 import workloads as wk

N_STEPS, EVERY, WT, WP = 120, 10, 1.0, 1e-4


def small_batch(seed=3):
    """Three walls, every coefficient term on: two layers (Pv-dependent kTT, cTT, cTM storage), one
    layer with an adiabatic face, three layers; noisy ambient air, q_inf and g_inf."""
    rng = np.random.default_rng(seed)
    walls = []
    for i, counts in enumerate(([4, 5], [7], [3, 5, 4])):
        layers = [dict(kM0=10 ** rng.uniform(-11.5, -10.5), a=rng.uniform(0.2, 1.5),
                       cM0=10 ** rng.uniform(*wk.CM0_LOG10_RANGE), b=rng.uniform(0.2, 1.5),
                       kTT0=rng.uniform(0.3, 1.5), aT=rng.uniform(0.05, 0.3), cTT0=rng.uniform(8e5, 2e6),
                       bT=rng.uniform(0.05, 0.3), chi=8.36e4) for _ in counts]
        bc0 = dict(hT=20.0, hM=2e-8, T_mean=298.0, T_amp=6.0, P_mean=1300.0, P_amp=300.0,
                   phase_T=rng.uniform(0, 6.28), phase_P=rng.uniform(0, 6.28), q_inf=rng.uniform(-20, 20),
                   g_inf=rng.uniform(-1e-7, 1e-7), period=3600.0)
        bc1 = dict(hT=8.0, hM=3e-8, T_mean=291.0, T_amp=2.0, P_mean=900.0, P_amp=100.0, period=5400.0)
        kinds = [wk.BC_AMBIENT, wk.BC_ADIABATIC if i == 1 else wk.BC_AMBIENT]
        w = wk.layered_wall(counts, rng.uniform(0.03, 0.06), layers, dt=60.0, n_steps=N_STEPS,
                            T0=rng.uniform(288, 296), P0=rng.uniform(900, 1200), bc0=bc0, bc1=bc1, kinds=kinds)
        nz = np.stack([rng.normal(0, 1.0, 20), rng.normal(0, 50.0, 20)], -1).astype(np.float32)
        w.noise = [nz[None], None]
        w.bc_par[:, 0, 11] = 600.0
        walls.append(w)
    wl = wk.concat(walls, name="adjoint pin batch")
    K = N_STEPS // EVERY
    obs = np.stack([293 + rng.normal(0, 3, (K, wl.n_walls, 2)), 1000 + rng.normal(0, 200, (K, wl.n_walls, 2))], -1)
    return wl, obs


def with_par(wl, par):
    import dataclasses

    return dataclasses.replace(wl, layer_par=np.asarray(par, np.float64).copy())


def forward_loss(oracle_mod, wl, obs):
    """The misfit computed from the samples of the (pinned) forward oracle."""
    o = oracle_mod.Oracle(wl, n_threads=1)
    s = o.run(N_STEPS, EVERY)["samples"]
    e = s - obs
    return float(WT * np.sum(e[..., 0] ** 2) + WP * np.sum(e[..., 1] ** 2))


def scales(par):
    """A magnitude per parameter (the value, or a typical size where the value is 0)."""
    typ = np.array([1e-11, 1.0, 5e-2, 1.0, 1.0, 0.1, 1e6, 0.1, 8e4])
    return np.maximum(np.abs(par), typ * 1e-3)


def test_adjoint_loss_is_the_forward_oracles_misfit(oracle_mod):
    wl, obs = small_batch()
    L, g = oracle_mod.loss_and_gradient(wl, N_STEPS, obs, EVERY, WT, WP)
    Lf = forward_loss(oracle_mod, wl, obs)
    assert abs(L - Lf) <= 1e-13 * Lf
    assert g.shape == (len(wl.layer_par), 9) and np.all(np.isfinite(g))


def test_dual_numbers_match_central_differences(oracle_mod):
    wl, obs = small_batch()
    rng = np.random.default_rng(5)
    sc = scales(wl.layer_par)
    for _ in range(3):
        d = rng.normal(size=wl.layer_par.shape) * sc
        L0, dL = oracle_mod.loss_tangent(wl, N_STEPS, obs, EVERY, WT, WP, d)
        assert abs(L0 - forward_loss(oracle_mod, wl, obs)) <= 1e-13 * L0
        def central(eps):
            Lp = forward_loss(oracle_mod, with_par(wl, wl.layer_par + eps * d), obs)
            Lm = forward_loss(oracle_mod, with_par(wl, wl.layer_par - eps * d), obs)
            return (Lp - Lm) / (2 * eps)

        fd = (4 * central(5e-4) - central(1e-3)) / 3   # Richardson: truncation O(eps^4)
        assert abs(fd - dL) <= 1e-6 * abs(dL), (fd, dL)


def test_adjoint_gradient_equals_dual_number_derivatives(oracle_mod):
    wl, obs = small_batch()
    _, g = oracle_mod.loss_and_gradient(wl, N_STEPS, obs, EVERY, WT, WP)
    rng = np.random.default_rng(7)
    sc = scales(wl.layer_par)
    for _ in range(4):
        d = rng.normal(size=wl.layer_par.shape) * sc
        _, dL = oracle_mod.loss_tangent(wl, N_STEPS, obs, EVERY, WT, WP, d)
        assert abs(np.sum(g * d) - dL) <= 1e-10 * np.sum(np.abs(g * d)), (np.sum(g * d), dL)
    # every parameter of two layers on its own (errors relative to the largest scaled component: a
    # small component carries the rounding of the large terms it is the difference of)
    big = np.max(np.abs(g * sc))
    for layer in (0, 4):
        for k in range(9):
            d = np.zeros_like(wl.layer_par)
            d[layer, k] = sc[layer, k]
            _, dL = oracle_mod.loss_tangent(wl, N_STEPS, obs, EVERY, WT, WP, d)
            assert abs(g[layer, k] * d[layer, k] - dL) <= 1e-11 * big, (layer, k)
            assert abs(g[layer, k] * d[layer, k] - dL) <= 1e-6 * abs(dL), (layer, k)


def test_adjoint_gradient_central_differences_per_parameter(oracle_mod):
    """The six parameters of the gradient workload (kM0, a, cM0, b, kTT0, cTT0) of every layer."""
    wl, obs = small_batch()
    _, g = oracle_mod.loss_and_gradient(wl, N_STEPS, obs, EVERY, WT, WP)
    def central(layer, k, h):
        par = wl.layer_par.copy()
        par[layer, k] += h
        Lp = forward_loss(oracle_mod, with_par(wl, par), obs)
        par[layer, k] -= 2 * h
        Lm = forward_loss(oracle_mod, with_par(wl, par), obs)
        return (Lp - Lm) / (2 * h)

    # components compared in the scaled form g_k theta_k: a component far below the largest one (a
    # deep layer the moisture hardly reaches in a short run) is a difference drowned in rounding
    big = np.max(np.abs(g * wl.layer_par)[:, [0, 1, 2, 3, 4, 6]])
    for layer in range(len(wl.layer_par)):
        for k in (0, 1, 2, 3, 4, 6):
            # Richardson extrapolation of central differences: truncation O(h^4) at h = 1e-3 relative
            th = abs(wl.layer_par[layer, k])
            fd = (4 * central(layer, k, 5e-4 * th) - central(layer, k, 1e-3 * th)) / 3
            assert abs(fd - g[layer, k]) * th <= 1e-6 * abs(g[layer, k]) * th + 1e-9 * big, (layer, k, fd, g[layer, k])


def test_zero_misfit_gives_zero_gradient(oracle_mod):
    """Observations equal to the run's own samples: the loss and every gradient component vanish."""
    wl, _ = small_batch()
    o = oracle_mod.Oracle(wl, n_threads=1)
    obs = o.run(N_STEPS, EVERY)["samples"]
    L, g = oracle_mod.loss_and_gradient(wl, N_STEPS, obs, EVERY, WT, WP)
    assert L == 0.0 and np.all(g == 0.0)
