"""The wall-schedule autotuner of the persistent kernel (hygro_autotune): it refits the step-time model on a
traced probe of the workload and keeps the faster schedule. Where a wall runs does not change what it
computes, so the run after tuning matches a run without it bit for bit, and the probe leaves the stored state
as it was."""
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


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_autotune_keeps_state_and_results(H, precision):
    import test_parity_gpu as par

    # the benchmark's generator (all four code variants when mixed with the ragged test batch's walls)
    wl = wk.concat([wk.wall_batch(seed=31, n_walls=600, n_steps=300), par.ragged_batch(par.EDGE_NS, 300)])
    ref = H.Hygro(wl, precision=precision)
    ref.run(40)
    ref.run(260)
    Tr, Pr = ref.fields(0)
    Tr1, Pr1 = ref.fields(1)
    fr, cr = ref.fluxes()
    ref.close()
    with H.Hygro(wl, precision=precision) as g:
        g.run(40)
        before = g.fields(0), g.fields(1), g.fluxes()
        a, b, ms = g.autotune(64)
        assert np.all(np.isfinite(a)) and np.all(np.isfinite(b)) and np.all(b >= 0)
        assert ms[0] > 0 and ms[1] > 0
        assert g.step == 40
        after = g.fields(0), g.fields(1), g.fluxes()
        for x, y in zip(before, after):
            assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
        g.run(260)
        T, P = g.fields(0)
        T1, P1 = g.fields(1)
        f, c = g.fluxes()
    assert np.array_equal(T, Tr) and np.array_equal(P, Pr)
    assert np.array_equal(T1, Tr1) and np.array_equal(P1, Pr1)
    assert np.array_equal(f, fr) and np.array_equal(c, cr)


def test_autotune_refusals(H):
    wl = wk.wall_batch(seed=32, n_walls=40, n_steps=50, n_min=3, n_max=100)
    with H.Hygro(wl, precision="fp32") as g:
        for bad in (0, 15, (1 << 20) + 1):
            with pytest.raises(H.HygroError) as e:
                g.autotune(bad)
            assert e.value.status == H.HYGRO_E_INVALID
    with H.Hygro(wl, precision="fp32", kernel="plain") as g:
        with pytest.raises(H.HygroError) as e:
            g.autotune(32)
        assert e.value.status == H.HYGRO_E_UNSUPPORTED
    wb = wk.building(n_rooms=2, walls_per_room=3, n_steps=20)
    with H.Hygro(wb, precision="fp32") as g:
        with pytest.raises(H.HygroError) as e:
            g.autotune(32)
        assert e.value.status == H.HYGRO_E_UNSUPPORTED
