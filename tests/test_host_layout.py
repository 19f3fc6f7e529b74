"""CPU tests of the persistent kernel's host-side work partition (csrc/host_layout.h), built with g++.

The lane layout puts a wall of N nodes into one warp: K or K-1 consecutive nodes per lane, node 0 in
lane 0 and node N-1 in the last slot of lane Wl-1, layer interfaces on lane boundaries when it can.
The schedule cuts the walls, sorted by size and code variant, into rounds of R walls and deals the
rounds to G persistent blocks, largest estimated cost first, each to the least loaded block (LPT)."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MAX_K = 16


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    out = str(tmp_path_factory.mktemp("host_layout") / "libhost_layout.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC",
                    "-I", os.path.join(ROOT, "paper_1703_10119_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host_logic_shim.cpp"), "-o", out], check=True)
    lib = C.CDLL(out)
    lib.shim_sched_cost.restype = C.c_double
    return lib


def layout(lib, N, first):
    f = np.ascontiguousarray(first, np.int32)
    out = np.zeros(4, np.int64)
    lib.shim_wall_layout(int(N), f.ctypes.data_as(C.c_void_p), len(f), out.ctypes.data_as(C.c_void_p))
    return int(out[0]), int(out[1]), int(out[2]), int(out[3])


def lane_starts(K, Wl, mask):
    sizes = [K - ((mask >> i) & 1) for i in range(Wl)]
    return np.concatenate([[0], np.cumsum(sizes)]).astype(int), sizes


def check_layout(N, first, K, Wl, mask, aligned):
    assert 1 <= K <= MAX_K and K >= -(-N // 32), (N, K)
    assert 1 <= Wl <= 32
    assert mask >> Wl == 0, "short lanes beyond the used lanes"
    assert (mask >> (Wl - 1)) & 1 == 0, "the last lane must be full"
    if K == 1:
        assert mask == 0, "a lane of K - 1 = 0 nodes"
    starts, sizes = lane_starts(K, Wl, mask)
    assert starts[-1] == N, "lanes must hold exactly the wall's nodes"
    on_boundary = all(f in set(starts[:-1].tolist()) for f in first[1:])
    assert bool(aligned) == on_boundary, (N, list(first), K, Wl, bin(mask), aligned)


def test_single_layer_walls_every_size(shim):
    for N in range(1, 32 * MAX_K + 1):
        K, Wl, mask, aligned = layout(shim, N, [0])
        check_layout(N, [0], K, Wl, mask, aligned)
        assert aligned == 1 and K == -(-N // 32), N


def test_layered_walls(shim):
    rng = np.random.default_rng(1703)
    n_aligned = 0
    cases = 0
    for N in list(range(3, 70)) + list(rng.integers(70, 32 * MAX_K + 1, 400)):
        for nl in (2, 3, 5, 8):
            if nl > N:
                continue
            first = np.concatenate([[0], np.sort(rng.choice(np.arange(1, N), nl - 1, replace=False))])
            K, Wl, mask, aligned = layout(shim, N, first)
            check_layout(N, first, K, Wl, mask, aligned)
            n_aligned += aligned
            cases += 1
    assert n_aligned > cases // 2   # most random splits get their interfaces on lane boundaries


def test_layers_of_whole_lanes_stay_at_the_smallest_K(shim):
    # layers of 10, 20 and 30 nodes in a 60-node wall: K = 2 puts every interface on a lane start
    K, Wl, mask, aligned = layout(shim, 60, [0, 10, 30])
    assert (K, Wl, mask, aligned) == (2, 30, 0, 1)
    # an interface at an odd node with K = 2 and no room for short lanes: K grows to 3
    K, Wl, mask, aligned = layout(shim, 64, [0, 33])
    check_layout(64, [0, 33], K, Wl, mask, aligned)
    assert aligned == 1 and K == 3


def test_misaligned_when_no_K_fits(shim):
    # 511 nodes need K = 16 on 32 lanes; an interface at node 1 cannot start a lane of 15 or 16 nodes
    K, Wl, mask, aligned = layout(shim, 511, [0, 1])
    check_layout(511, [0, 1], K, Wl, mask, aligned)
    assert aligned == 0 and K == 16


def lpt(lib, K, kind, N, G, R):
    n = len(K)
    wall = np.arange(n, dtype=np.int32)
    K = np.ascontiguousarray(K, np.int32)
    kind = np.ascontiguousarray(kind, np.int32)
    N = np.ascontiguousarray(N, np.int32)
    cap = (n + R) * 1 + R
    order = np.zeros(max(cap, 1), np.int32)
    boff = np.zeros(G + 1, np.int32)
    load = np.zeros(G)
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    m = lib.shim_lpt_rounds(n, p(wall), p(K), p(kind), p(N), G, R, p(order), len(order), p(boff), p(load))
    assert m >= 0
    return order[:m], boff, load


@pytest.mark.parametrize("n,G,R", [(4096, 152, 16), (4096, 152, 12), (1000, 152, 6), (100, 152, 1), (1, 152, 1),
                                   (0, 152, 1), (333, 7, 16)])
def test_lpt_rounds(shim, n, G, R):
    rng = np.random.default_rng(n + G + R)
    N = rng.integers(50, 401, n)
    K = -(-N // 32)
    kind = rng.choice([0, 0, 0, 1, 2, 3], n)
    order, boff, load = lpt(shim, K, kind, N, G, R)
    n_rounds = -(-n // R)
    assert len(order) == n_rounds * R
    assert boff[0] == 0 and boff[G] == len(order) and np.all(np.diff(boff) >= 0)
    assert np.all(np.diff(boff) % R == 0), "a block holds whole rounds"
    # every wall exactly once; the empty entries are the tail of one round
    assert sorted(order[order >= 0].tolist()) == list(range(n))
    assert np.count_nonzero(order < 0) == n_rounds * R - n
    cost = np.array([shim.shim_sched_cost(int(k), int(t)) for k, t in zip(K, kind)])
    rounds = order.reshape(-1, R) if n else order.reshape(0, R)
    rcost = np.array([cost[r[r >= 0]].max() for r in rounds]) if n else np.zeros(0)
    # a round is a run of the sorted walls: nodes per lane non-increasing, then variant non-decreasing
    for r in rounds:
        w = r[r >= 0]
        key = list(zip(-K[w], kind[w]))
        assert key == sorted(key)
    # block loads: the costs of their rounds; a block runs its rounds largest first; the LPT bound
    for g in range(G):
        rc = rcost[boff[g] // R: boff[g + 1] // R]
        assert abs(rc.sum() - load[g]) <= 1e-9 * max(1.0, load[g])
        assert np.all(np.diff(rc) <= 1e-12)
    assert abs(load.sum() - rcost.sum()) <= 1e-9 * max(1.0, rcost.sum())
    if n_rounds >= G:
        assert load.max() - load.min() <= rcost.max() + 1e-9
    else:
        assert np.count_nonzero(load > 0) == n_rounds   # one round per block while rounds are fewer


def _fit(shim, K, kind, ns, base):
    K = np.ascontiguousarray(K, np.int32)
    kind = np.ascontiguousarray(kind, np.int32)
    ns = np.ascontiguousarray(ns, np.float64)
    base = np.ascontiguousarray(base, np.float64)
    out = np.zeros(8)
    p = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    n = shim.shim_fit_cost_model(len(K), p(K), p(kind), p(ns), p(base), p(out))
    return n, out[:4], out[4:]


def test_cost_model_fit_recovers_exact_lines(shim):
    """The autotuner's fit of the per-variant step time a + b K: exact data give back a and b; a variant
    measured at a single K keeps the base slope and fits the intercept; a variant with no measured wall (or
    only unmeasured ones) keeps the base model."""
    rng = np.random.default_rng(3)
    base = [100.0, 200.0, 150.0, 190.0, 60.0, 70.0, 120.0, 80.0]
    a_true, b_true = [90.0, 250.0, 0, 0], [55.0, 81.0, 0, 0]
    K, kind, ns = [], [], []
    for v in (0, 1):
        for k in rng.integers(2, 14, 40):
            K.append(k)
            kind.append(v)
            ns.append(a_true[v] + b_true[v] * k)
    for _ in range(5):            # variant 2 at one K only: 7 -> 1000 ns
        K.append(7)
        kind.append(2)
        ns.append(1000.0)
    K.append(5)
    kind.append(3)
    ns.append(-1.0)               # not measured
    n, a, b = _fit(shim, K, kind, ns, base)
    assert n == 3
    np.testing.assert_allclose(a[:2], a_true[:2], rtol=1e-12)
    np.testing.assert_allclose(b[:2], b_true[:2], rtol=1e-12)
    assert b[2] == base[6] and abs(a[2] - (1000.0 - base[6] * 7)) < 1e-9
    assert a[3] == base[3] and b[3] == base[7]


def test_cost_model_fit_least_squares_and_nonnegative_slope(shim):
    """Noisy data give the least-squares line (numpy's polyfit); a falling trend is clipped to a flat one."""
    rng = np.random.default_rng(4)
    K = rng.integers(2, 14, 200)
    ns = 120.0 + 66.0 * K + rng.normal(0, 15.0, K.size)
    n, a, b = _fit(shim, K, np.zeros(K.size), ns, [0.0] * 8)
    slope, icpt = np.polyfit(K.astype(float), ns, 1)
    assert n == 1 and abs(b[0] - slope) < 1e-9 * slope and abs(a[0] - icpt) < 1e-6 * abs(icpt)
    n, a, b = _fit(shim, K, np.zeros(K.size), 900.0 - 10.0 * K, [0.0] * 8)
    assert b[0] == 0.0 and abs(a[0] - np.mean(900.0 - 10.0 * K)) < 1e-9
