"""GPU: the noise tables of the ambient faces (hourly Gaussian forcing, linearly interpolated).

Each face's tables live in a region of their own in the context's device array, filled when that face is
set. These tests set them in the other ways the C ABI allows (one table per host allocation, a face set
again with longer tables, which moves the other face's region) and require results identical to those of
the one-array setup, and the two-face-noise workload to match the FP64 oracle.
"""
import dataclasses

import numpy as np
import pytest

from paper_1703_10119_gb300 import workloads as wk

pytestmark = pytest.mark.gpu

N_STEPS = 300


@pytest.fixture(scope="module")
def H():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_10119_gb300 import build, hygro

    build.build()
    return hygro


def two_face_noise_batch():
    """A small ragged batch (64 walls, 50-400 nodes) with noise tables on both faces."""
    wl = wk.wall_batch(seed=11, n_walls=64, n_steps=N_STEPS, noise=True)
    z0 = wl.noise[0]
    key = wk.stream_key(11, np.arange(64) + (1 << 33))
    a, b = wk.normal_pairs(key[:, None], np.arange(z0.shape[1], dtype=np.uint64)[None, :])
    z1 = np.stack([0.5 * a, 20.0 * b], axis=-1).astype(np.float32)
    bc_par = wl.bc_par.copy()
    bc_par[:, 1, wk.BC_FIELDS.index("noise_dt")] = bc_par[:, 0, wk.BC_FIELDS.index("noise_dt")]
    return dataclasses.replace(wl, noise=[z0, z1], bc_par=bc_par)


def _state(g):
    T0, P0 = g.fields(0)
    T1, P1 = g.fields(1)
    f, c = g.fluxes()
    return np.concatenate([T0, P0, T1, P1, f.ravel(), c.ravel()])


def _bc_separate(H, wl, face, tables):
    """hygro_bc array whose tables are separate host arrays (allocated in reverse wall order)."""
    arr = H._bc_array(wl.n_walls, wl.bc_kind[:, face], wl.bc_par[:, face], None)
    for w in range(wl.n_walls):
        arr[w].room = int(wl.bc_room[w, face])
        arr[w].noise = tables[w].ctypes.data
        arr[w].noise_len = tables[w].shape[0]
    return arr


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_separate_and_regrown_tables_give_identical_results(H, precision):
    wl = two_face_noise_batch()
    ref = H.Hygro(wl, precision=precision)
    ref.run(N_STEPS)
    want = _state(ref)
    ref.close()

    g = H.Hygro(wl, precision=precision)
    # face 1 again, one allocation per wall
    t1 = [np.array(wl.noise[1][w]) for w in reversed(range(wl.n_walls))][::-1]
    H.hygro_set_bc(g.ctx, 1, _bc_separate(H, wl, 1, t1))
    # face 0 again with tables 50 entries longer (past the horizon): its region grows, face 1's moves
    pad = np.zeros((wl.n_walls, 50, 2), np.float32) + 7.0
    t0 = [np.ascontiguousarray(np.concatenate([wl.noise[0][w], pad[w]])) for w in range(wl.n_walls)]
    H.hygro_set_bc(g.ctx, 0, _bc_separate(H, wl, 0, t0))
    g.run(N_STEPS)
    got = _state(g)
    g.close()
    assert np.array_equal(got, want)


def test_two_face_noise_matches_oracle_fp64(H, oracle_mod):
    wl = two_face_noise_batch()
    g = H.Hygro(wl, precision="fp64")
    g.run(N_STEPS)
    T, P = g.fields(0)
    flux, cum = g.fluxes()
    g.close()
    o = oracle_mod.Oracle(wl)
    r = o.run(N_STEPS, 0)
    assert np.max(np.abs(T - o.T_cur)) / np.max(np.abs(o.T_cur)) <= 1e-12
    assert np.max(np.abs(P - o.P_cur)) / np.max(np.abs(o.P_cur)) <= 1e-12
    assert np.max(np.abs(cum - o.cumul)) / np.max(np.abs(o.cumul)) <= 1e-9
    assert np.max(np.abs(flux - r["flux"])) / np.max(np.abs(r["flux"])) <= 1e-9


def test_noise_changes_the_result(H):
    """The face-1 tables are read: zeroing them changes the fields."""
    wl = two_face_noise_batch()
    a = H.Hygro(wl, precision="fp64")
    a.run(N_STEPS)
    sa = _state(a)
    a.close()
    quiet = dataclasses.replace(wl, noise=[wl.noise[0], np.zeros_like(wl.noise[1])])
    b = H.Hygro(quiet, precision="fp64")
    b.run(N_STEPS)
    sb = _state(b)
    b.close()
    assert not np.array_equal(sa, sb)


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_nonfinite_table_is_refused_and_leaves_the_face(H, bad):
    wl = two_face_noise_batch()
    ref = H.Hygro(wl, precision="fp64")
    ref.run(N_STEPS)
    want = _state(ref)
    ref.close()

    g = H.Hygro(wl, precision="fp64")
    tabs = [np.array(wl.noise[0][w]) for w in range(wl.n_walls)]
    tabs[37][5, 1] = bad
    with pytest.raises(H.HygroError) as e:
        H.hygro_set_bc(g.ctx, 0, _bc_separate(H, wl, 0, tabs))
    assert e.value.status == H.HYGRO_E_INVALID
    assert "wall 37" in str(e.value) and "non-finite noise" in str(e.value)
    g.run(N_STEPS)
    assert np.array_equal(_state(g), want)
    g.close()


def long_table_batch(n_steps=140000):
    """64 thin walls (50-60 nodes) whose face-0 tables hold one entry per step (noise_dt = dt), so every
    entry enters the cumulative fluxes; 64 x (n_steps + 2) pairs exceed one 2^23-pair upload chunk, the
    chunk boundary falling inside wall 59's table."""
    wl = wk.wall_batch(seed=12, n_walls=64, n_min=50, n_max=60, n_steps=n_steps, dt=600.0, noise=False)
    L = n_steps + 2
    key = wk.stream_key(12, np.arange(64) + (1 << 34))
    a, b = wk.normal_pairs(key[:, None], np.arange(L, dtype=np.uint64)[None, :])
    z0 = np.stack([1.0 * a, 50.0 * b], axis=-1).astype(np.float32)
    bc_par = wl.bc_par.copy()
    bc_par[:, 0, wk.BC_FIELDS.index("noise_dt")] = wl.dt
    return dataclasses.replace(wl, noise=[z0, None], bc_par=bc_par)


def test_tables_across_upload_chunks_match_oracle_fp64(H, oracle_mod):
    wl = long_table_batch()
    assert wl.noise[0].shape[0] * wl.noise[0].shape[1] > (1 << 23)
    g = H.Hygro(wl, precision="fp64")
    g.run(wl.n_steps)
    T, P = g.fields(0)
    flux, cum = g.fluxes()
    g.close()
    o = oracle_mod.Oracle(wl)
    o.run(wl.n_steps, 0)
    assert np.max(np.abs(T - o.T_cur)) / np.max(np.abs(o.T_cur)) <= 1e-12
    assert np.max(np.abs(P - o.P_cur)) / np.max(np.abs(o.P_cur)) <= 1e-12
    # every table entry entered the running flux sums: compare them wall by wall
    err = np.abs(cum - o.cumul).max(axis=(1, 2)) / np.abs(o.cumul).max()
    assert err.max() <= 1e-9, (int(err.argmax()), float(err.max()))


def test_nonfinite_value_in_a_later_chunk_is_refused(H):
    wl = long_table_batch(n_steps=140000)
    g = H.Hygro(wl, precision="fp64")
    z = np.array(wl.noise[0])
    z[62, 1000, 0] = np.nan   # pair 62 * 140002 + 1000, in the second chunk
    arr = H._bc_array(wl.n_walls, wl.bc_kind[:, 0], wl.bc_par[:, 0], z)
    with pytest.raises(H.HygroError) as e:
        H.hygro_set_bc(g.ctx, 0, arr)
    assert "wall 62 face 0: non-finite noise" in str(e.value)
    g.close()


def _pinned(a):
    import torch

    t = torch.empty(a.shape, dtype=torch.float32, pin_memory=True)
    t.numpy()[...] = a
    return t


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_pinned_tables_take_the_direct_copy(H, precision):
    """Tables in page-locked host memory go to the device by DMA, one copy per run of adjacent tables,
    and are checked on the device: one pinned array for all walls, and one pinned array per wall (runs of
    one table) give the results of the pageable upload, bit for bit."""
    wl = two_face_noise_batch()
    ref = H.Hygro(wl, precision=precision)
    ref.run(N_STEPS)
    want = _state(ref)
    ref.close()
    keep = [_pinned(wl.noise[0]), _pinned(wl.noise[1])]
    g = H.Hygro(wl, precision=precision)
    for f in range(2):
        H.hygro_set_bc(g.ctx, f, H._bc_array(wl.n_walls, wl.bc_kind[:, f], wl.bc_par[:, f], keep[f].numpy()))
    g.run(N_STEPS)
    assert np.array_equal(_state(g), want)
    g.close()
    per_wall = [_pinned(np.ascontiguousarray(wl.noise[1][w])) for w in reversed(range(wl.n_walls))][::-1]
    g = H.Hygro(wl, precision=precision)
    H.hygro_set_bc(g.ctx, 1, _bc_separate(H, wl, 1, [t.numpy() for t in per_wall]))
    g.run(N_STEPS)
    assert np.array_equal(_state(g), want)
    g.close()


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_pinned_nonfinite_table_is_refused_and_leaves_the_face(H, bad):
    wl = two_face_noise_batch()
    ref = H.Hygro(wl, precision="fp64")
    ref.run(N_STEPS)
    want = _state(ref)
    ref.close()
    z = np.array(wl.noise[0])
    z[41, 7, 0] = bad
    z[50, 3, 1] = bad   # a later one: the first is reported
    t = _pinned(z)
    g = H.Hygro(wl, precision="fp64")
    with pytest.raises(H.HygroError) as e:
        H.hygro_set_bc(g.ctx, 0, H._bc_array(wl.n_walls, wl.bc_kind[:, 0], wl.bc_par[:, 0], t.numpy()))
    assert e.value.status == H.HYGRO_E_INVALID
    assert "wall 41 face 0: non-finite noise" in str(e.value)
    g.run(N_STEPS)
    assert np.array_equal(_state(g), want)
    g.close()


def test_device_resident_tables(H):
    """Tables already in device memory (a torch CUDA tensor) take the direct path too: a device-to-device
    copy into the staging area. The results equal the host upload's, bit for bit."""
    import torch

    wl = two_face_noise_batch()
    ref = H.Hygro(wl, precision="fp32")
    ref.run(N_STEPS)
    want = _state(ref)
    ref.close()
    dev = [torch.from_numpy(np.ascontiguousarray(z)).cuda() for z in wl.noise]
    torch.cuda.synchronize()
    g = H.Hygro(wl, precision="fp32")
    for f in range(2):
        arr = H._bc_array(wl.n_walls, wl.bc_kind[:, f], wl.bc_par[:, f], None)
        L = dev[f].shape[1]
        for w in range(wl.n_walls):
            arr[w].noise = dev[f].data_ptr() + w * L * 2 * 4
            arr[w].noise_len = L
        H.hygro_set_bc(g.ctx, f, arr)
    g.run(N_STEPS)
    assert np.array_equal(_state(g), want)
    g.close()
