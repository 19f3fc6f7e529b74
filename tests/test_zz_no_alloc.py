"""hygro_run_noalloc: the run entry point for callers that cannot allocate device memory at the call.

Some callers cannot call cudaMalloc when they run a step: their process hands all device memory to
its own pool allocator (as PyTorch's caching allocator does), or they sit in a loop that must not
allocate. hygro_run allocates a staging buffer for samples bound for host memory; hygro_run_noalloc
stages them in a fixed device array that the library carries instead. These checks call it through
the C ABI and compare it with hygro_run on two calls in a row, bit for bit (both calls run the same
kernels on the same inputs; only the staging of the samples differs), with samples bound for host memory
and with samples in device memory (which neither call stages). They also check that repeated calls leave
the device's free memory unchanged, and that an oversized request is refused without changing anything.
This file is collected last so that a stop at the first failure has run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_10119_gb300 import build, hygro

    build.build()
    return hygro


def _same_run(H, a, b, wl, n, every, device_samples):
    """One hygro_run on a and one hygro_run_noalloc on b; samples, both stored levels and the fluxes must
    agree bit for bit."""
    import torch

    shape = (n // every, wl.n_walls, 2, 2)
    if device_samples:
        sa = torch.zeros(shape, dtype=torch.float32, device="cuda")
        sb = torch.zeros_like(sa)
    else:
        sa = np.zeros(shape, np.float32)
        sb = np.zeros_like(sa)
    H.hygro_run(a.ctx, n, every, sa)
    H.hygro_run_noalloc(b.ctx, n, every, sb)
    a.sync()
    b.sync()
    if device_samples:
        sa, sb = sa.cpu().numpy(), sb.cpu().numpy()
    assert np.any(sa != 0.0)
    assert np.array_equal(sa, sb)
    for level in (0, 1):
        Ta, Pa = a.fields(level)
        Tb, Pb = b.fields(level)
        assert np.array_equal(Ta, Tb) and np.array_equal(Pa, Pb), level
    fa, ca = a.fluxes()
    fb, cb = b.fluxes()
    assert np.array_equal(fa, fb) and np.array_equal(ca, cb)
    assert a.step == b.step


@pytest.mark.parametrize("device_samples", [False, True])
@pytest.mark.parametrize("kernel", ["persistent", "plain"])
def test_noalloc_matches_run_two_calls(H, kernel, device_samples):
    import torch

    from paper_1703_10119_gb300 import workloads as wk

    wl = wk.wall_batch(seed=21, n_walls=96, n_steps=300, n_min=3, n_max=512)
    a = H.Hygro(wl, precision="fp32", kernel=kernel)
    b = H.Hygro(wl, precision="fp32", kernel=kernel)
    for call in range(2):
        _same_run(H, a, b, wl, 150 + 7 * call, 10, device_samples)
    # once the first call on this device has looked up the array, further calls allocate nothing
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    sb = np.zeros((5, wl.n_walls, 2, 2), np.float32)
    for _ in range(3):
        H.hygro_run_noalloc(b.ctx, 50, 10, sb)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    a.close()
    b.close()


def test_noalloc_refuses_oversized_samples(H):
    from paper_1703_10119_gb300 import workloads as wk

    wl = wk.wall_batch(seed=22, n_walls=64, n_steps=100, n_min=3, n_max=100)
    g = H.Hygro(wl, precision="fp32")
    g.run(3)
    T0, P0 = g.fields(0)
    per_sample = wl.n_walls * 4 * 4
    n = H.HYGRO_NOALLOC_SCRATCH_BYTES // per_sample + 1
    big = np.zeros((n, wl.n_walls, 2, 2), np.float32)
    with pytest.raises(H.HygroError) as e:
        H.hygro_run_noalloc(g.ctx, n, 1, big)
    assert e.value.status == H.HYGRO_E_UNSUPPORTED
    assert g.step == 3
    T1, P1 = g.fields(0)
    assert np.array_equal(T0, T1) and np.array_equal(P0, P1)
    g.close()
