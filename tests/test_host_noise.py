"""CPU tests of the noise-table gather behind the staged upload (csrc/host_noise.h), built with g++.

Per-wall tables of (T, Pv) float pairs, back to back in wall order, are copied into a chunk by several
host threads, each checking the values it copies; the gather returns the first pair that holds a
non-finite value. Required: the chunk equals the concatenation bit for bit (signed zeros, subnormals,
the largest floats included), for any sub-range and thread count, and the first non-finite pair is
found wherever it lies relative to the table and thread boundaries."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    out = str(tmp_path_factory.mktemp("host_noise") / "libhost_logic.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                    "-I", os.path.join(ROOT, "paper_1703_10119_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host_logic_shim.cpp"), "-o", out], check=True)
    lib = C.CDLL(out)
    lib.shim_gather_tables.restype = C.c_int64
    lib.shim_gather_tables.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_int,
                                       C.c_int64]
    return lib


def tables(rng, n, max_len=50):
    lens = rng.integers(1, max_len + 1, n)
    tabs = [rng.normal(0, 100, (int(L), 2)).astype(np.float32) for L in lens]
    # values a copy must keep bit for bit
    special = np.array([0.0, -0.0, 1e-45, -1e-40, 3.4028235e38, -3.4028235e38], np.float32)
    for k in range(0, n, 3):
        tabs[k].ravel()[: len(special)] = special[: tabs[k].size]
    return tabs


def gather(lib, tabs, p0, p1, threads, min_pairs=1):
    ptrs = (C.c_void_p * len(tabs))(*[t.ctypes.data for t in tabs])
    lens = np.array([t.shape[0] for t in tabs], np.int64)
    dst = np.full((max(p1 - p0, 0), 2), 12345.0, np.float32)
    bad = lib.shim_gather_tables(len(tabs), C.cast(ptrs, C.c_void_p), lens.ctypes.data, p0, p1, dst.ctypes.data,
                                 threads, min_pairs)
    return int(bad), dst


@pytest.mark.parametrize("threads", [1, 2, 3, 8])
def test_gather_equals_concatenation_bit_for_bit(shim, threads):
    rng = np.random.default_rng(threads)
    tabs = tables(rng, 40)
    cat = np.concatenate(tabs)
    total = cat.shape[0]
    for p0, p1 in [(0, total), (0, 1), (total - 1, total), (17, 17), (5, total - 9), (31, 32 + 50)]:
        p1 = min(p1, total)
        bad, dst = gather(shim, tabs, p0, p1, threads)
        assert bad == -1
        assert dst.view(np.uint32).tobytes() == cat[p0:p1].view(np.uint32).tobytes(), (p0, p1)


@pytest.mark.parametrize("threads", [1, 4, 8])
@pytest.mark.parametrize("bad_value", [np.nan, np.inf, -np.inf])
def test_first_nonfinite_pair_is_found(shim, threads, bad_value):
    rng = np.random.default_rng(7)
    tabs = tables(rng, 30)
    cat = np.concatenate(tabs)
    total = cat.shape[0]
    starts = np.concatenate([[0], np.cumsum([t.shape[0] for t in tabs])])
    # the first pair of a table, the last pair of a table, a pair in the middle, the very last pair
    for pos in [int(starts[5]), int(starts[6] - 1), total // 2, total - 1]:
        for comp in (0, 1):
            tt = [t.copy() for t in tabs]
            k = int(np.searchsorted(starts, pos, side="right") - 1)
            tt[k][pos - starts[k], comp] = bad_value
            # a second bad value later must not hide the first
            tt[-1][-1, 1 - comp] = bad_value
            bad, _ = gather(shim, tt, 0, total, threads)
            assert bad == pos, (pos, comp, bad)
            # a sub-range that stops before the pair does not see it (unless the later one is inside)
            if pos > 3:
                bad, _ = gather(shim, tt, 0, pos, threads)
                assert bad == -1


def test_default_thread_floor_keeps_small_ranges_on_one_thread(shim):
    rng = np.random.default_rng(3)
    tabs = tables(rng, 10)
    cat = np.concatenate(tabs)
    bad, dst = gather(shim, tabs, 0, cat.shape[0], 8, min_pairs=1 << 18)
    assert bad == -1 and np.array_equal(dst.view(np.uint32), cat.view(np.uint32))
