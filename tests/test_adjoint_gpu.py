"""GPU reverse-time adjoint (hygro_loss_grad) against the FP64 adjoint oracle.

Gradients are compared in the scaled form g_k theta_k (the loss change per relative change of a
parameter), relative to the largest scaled component of the batch, because a component far below the
largest one is a difference of larger terms:
  * FP64 path: loss 1e-12 relative, scaled gradient 1e-10;
  * FP32 path: loss 1e-5 relative, scaled gradient 2e-5 (the FP32 trajectory and adjoint carry the
    single-precision rounding of every step; measured at most 8.7e-7 (loss) and 4.2e-6 (gradient, the
    full 30-day workload); the bounds keep a margin of about 5);
  * FP32 gradient against central differences of the FP64 oracle's loss: 1e-5 (measured 9.3e-7).
"""
import dataclasses

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


def small_batch(seed=3):
    """The adjoint pins' batch: three walls, every coefficient term on, noisy ambient air."""
    import test_oracle_adjoint_pins as pins

    return pins.small_batch(seed)


def scaled_err(g, ref, par):
    big = np.max(np.abs(ref * par))
    return float(np.max(np.abs((g - ref) * par)) / big)


def gpu_loss_grad(H, wl, n_steps, obs, every, wT, wP, precision="fp64", ck=0):
    with H.Hygro(wl, precision=precision, kernel="persistent") as g:
        L, grad = g.loss_grad(n_steps, every, obs, wT, wP, ck)
        g.sync()
    return L, grad


@pytest.mark.parametrize("precision,tol_loss,tol_grad", [("fp64", 1e-12, 1e-10), ("fp32", 1e-5, 2e-5)])
def test_matches_oracle_adjoint(H, oracle_mod, precision, tol_loss, tol_grad):
    wl, obs = small_batch()
    L, g = gpu_loss_grad(H, wl, 120, obs.astype(np.float32), 10, 1.0, 1e-4, precision)
    # the GPU reads the observations in FP32: compare against the oracle on the same rounded values
    L0, g0 = oracle_mod.loss_and_gradient(wl, 120, obs.astype(np.float32).astype(np.float64), 10, 1.0, 1e-4)
    print(f"measured-error adjoint-small {precision} loss={abs(L - L0) / L0:.3e} "
          f"grad={scaled_err(g, g0, wl.layer_par):.3e}")
    assert abs(L - L0) <= tol_loss * L0, (L, L0)
    assert scaled_err(g, g0, wl.layer_par) <= tol_grad


def test_checkpoint_stride_does_not_change_the_result(H):
    wl, obs = small_batch()
    obs = obs.astype(np.float32)
    ref = gpu_loss_grad(H, wl, 120, obs, 10, 1.0, 1e-4, "fp64", ck=120)
    for ck in (1, 7, 0, 64):
        L, g = gpu_loss_grad(H, wl, 120, obs, 10, 1.0, 1e-4, "fp64", ck=ck)
        assert L == ref[0]
        assert scaled_err(g, ref[1], wl.layer_par) <= 1e-13


@pytest.mark.parametrize("precision,tol_loss,tol_grad", [("fp64", 1e-12, 1e-10), ("fp32", 1e-5, 2e-5)])
def test_ragged_walls_and_lane_layouts(H, oracle_mod, precision, tol_loss, tol_grad):
    """Walls of 3 to 512 nodes with 1 to 3 layers (some a few nodes thick), adiabatic faces, a run whose
    length is not a multiple of the sampling or the checkpoint stride. The lane runs span 1 to 17 nodes:
    both the register kernel and the shared-memory kernel (runs longer than the register slots) take
    part, in both precisions."""
    import test_parity_gpu as par

    wl = par.ragged_batch([3, 4, 17, 33, 64, 97, 200, 257, 400, 511, 512], 77, dt=60.0)
    rng = np.random.default_rng(2)
    every, n = 5, 77
    K = n // every
    obs = np.stack([293 + rng.normal(0, 3, (K, wl.n_walls, 2)), 1000 + rng.normal(0, 200, (K, wl.n_walls, 2))],
                   -1).astype(np.float32)
    L0, g0 = oracle_mod.loss_and_gradient(wl, n, obs.astype(np.float64), every, 1.0, 1e-4)
    L, g = gpu_loss_grad(H, wl, n, obs, every, 1.0, 1e-4, precision, ck=9)
    print(f"measured-error adjoint-ragged {precision} loss={abs(L - L0) / L0:.3e} "
          f"grad={scaled_err(g, g0, wl.layer_par):.3e}")
    assert abs(L - L0) <= tol_loss * L0
    assert scaled_err(g, g0, wl.layer_par) <= tol_grad


def test_autograd_function(H):
    import torch

    from paper_1703_10119_gb300.autograd import MisfitLoss

    wl, obs = small_batch()
    obs = obs.astype(np.float32)
    with H.Hygro(wl, precision="fp64") as g:
        theta = torch.tensor(wl.layer_par, dtype=torch.float64, requires_grad=True)
        loss = MisfitLoss.apply(theta, g, 120, 10, obs, 1.0, 1e-4)
        loss.backward()
        L, ref = g.loss_grad(120, 10, obs, 1.0, 1e-4)
        assert float(loss) == L
        assert np.array_equal(theta.grad.numpy(), ref)
        # a directional finite difference of the GPU loss along a random scaled direction
        rng = np.random.default_rng(4)
        d = rng.normal(size=wl.layer_par.shape) * np.abs(wl.layer_par)
        d[:, [5, 7, 8]] = 0.0
        vals = []
        for eps in (1e-3, 5e-4):
            lp = float(MisfitLoss.apply(torch.tensor(wl.layer_par + eps * d), g, 120, 10, obs, 1.0, 1e-4))
            lm = float(MisfitLoss.apply(torch.tensor(wl.layer_par - eps * d), g, 120, 10, obs, 1.0, 1e-4))
            vals.append((lp - lm) / (2 * eps))
        fd = (4 * vals[1] - vals[0]) / 3
        assert abs(fd - np.sum(ref * d)) <= 1e-6 * np.sum(np.abs(ref * d))


def test_autograd_function_keeps_the_run_state(H):
    """MisfitLoss sets the context's materials to theta; the run state (levels, step, flux sums) that was
    there before is restored, so a run under way goes on from where it was."""
    import torch

    from paper_1703_10119_gb300.autograd import MisfitLoss

    wl, obs = small_batch()
    obs = obs.astype(np.float32)
    with H.Hygro(wl, precision="fp64") as g:
        g.run(7)
        before = [g.fields(0), g.fields(1), g.fluxes()]
        theta = torch.tensor(wl.layer_par, dtype=torch.float64, requires_grad=True)
        MisfitLoss.apply(theta, g, 120, 10, obs, 1.0, 1e-4).backward()
        after = [g.fields(0), g.fields(1), g.fluxes()]
        assert g.step == 7
        for b, a in zip(before, after):
            assert np.array_equal(b[0], a[0]) and np.array_equal(b[1], a[1])


def test_invalid_calls(H):
    wl, obs = small_batch()
    obs = obs.astype(np.float32)
    with H.Hygro(wl, precision="fp32") as g:
        for args in ((0, 10, obs), (120, 0, obs), (120, 10, None)):
            with pytest.raises(H.HygroError) as e:
                H.hygro_loss_grad(g.ctx, args[0], args[1], args[2], 1.0, 1e-4)
            assert e.value.status == H.HYGRO_E_INVALID
        with pytest.raises(H.HygroError):
            H.hygro_loss_grad(g.ctx, 120, 10, obs, 1.0, 1e-4, -1)
        # the stored state is untouched by the adjoint
        g.run(5)
        before = g.fields(0)
        g.loss_grad(120, 10, obs, 1.0, 1e-4)
        after = g.fields(0)
        assert np.array_equal(before[0], after[0]) and g.step == 5
    wl3 = wk.building(n_rooms=1, walls_per_room=2, n_steps=10)
    with H.Hygro(wl3, precision="fp32") as g:
        with pytest.raises(H.HygroError) as e:
            g.loss_grad(10, 5, np.zeros((2, wl3.n_walls, 2, 2), np.float32), 1.0, 1e-4)
        assert e.value.status == H.HYGRO_E_UNSUPPORTED


def test_gradient_workload_full_size_sampled_walls(H, oracle_mod):
    """All 1024 walls over the 30 days in FP32 with sqrt(T) checkpoints; the oracle adjoint runs two of
    them (their layers' gradient rows depend on those walls alone)."""
    wl, s = wk.gradient_walls()
    with H.Hygro(wl, precision="fp32") as g:
        L, grad = g.loss_grad(wl.n_steps, s.sample_every, s.obs, s.wT, s.wP)
    assert np.isfinite(L) and np.all(np.isfinite(grad))
    pick = [0, 777]
    sub = wl.subset(pick)
    L0, g0 = oracle_mod.loss_and_gradient(sub, wl.n_steps, s.obs[:, pick].astype(np.float64), s.sample_every,
                                          s.wT, s.wP)
    rows = np.concatenate([np.arange(2 * w, 2 * w + 2) for w in pick])
    print(f"measured-error adjoint-full fp32 loss-part grad={scaled_err(grad[rows], g0, sub.layer_par):.3e}")
    assert scaled_err(grad[rows], g0, sub.layer_par) <= 2e-5


def test_fp32_gradient_against_central_differences(H, oracle_mod):
    """The FP32 GPU gradient (FP32 trajectory and adjoint, FP64 loss and parameter sums) against central
    differences of the FP64 oracle's loss, each parameter of each layer moved by 1e-4 of its value
    (the differences' own truncation error is O(1e-8) relative). Compared in the scaled form g_k theta_k
    relative to the largest scaled component."""
    wl, obs = small_batch()
    obs = obs.astype(np.float32)
    L, g = gpu_loss_grad(H, wl, 120, obs, 10, 1.0, 1e-4, "fp32")
    obs64 = obs.astype(np.float64)
    par = wl.layer_par
    fd = np.zeros_like(par)
    h = 1e-4
    for r in range(par.shape[0]):
        for k in range(par.shape[1]):
            if par[r, k] == 0.0:
                continue
            vals = []
            for sgn in (1.0, -1.0):
                p2 = par.copy()
                p2[r, k] *= 1.0 + sgn * h
                w2 = dataclasses.replace(wl, layer_par=p2)
                vals.append(oracle_mod.loss_and_gradient(w2, 120, obs64, 10, 1.0, 1e-4, gradient=False)[0])
            fd[r, k] = (vals[0] - vals[1]) / (2 * h * par[r, k])
    err = scaled_err(g, fd, par)
    print(f"measured-error adjoint-fd fp32 grad-vs-central-differences={err:.3e}")
    assert err <= 1e-5
