"""CPU tests of the fixed-point forcing accumulators (csrc/host_forcing.h), built with g++.

The FP32 kernels form the ambient air of step n ([eq:HAM_BC] data at t^n = t0 + n dt) from integers:
the sinusoid's phase in turns as phT0 + n pstep modulo 2^64 (scaled by 2^64), and the noise table
position as npos0 + n nstep (entries scaled by 2^40), held at the last entry from step n_hi on.
Checked against exact rational arithmetic on the same double inputs."""
import ctypes as C
import math
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TWO_PI = 6.283185307179586476925286766559   # the double the library uses
M64 = 1 << 64


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    out = str(tmp_path_factory.mktemp("host_forcing") / "libhost_logic.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                    "-I", os.path.join(ROOT, "paper_1703_10119_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host_logic_shim.cpp"), "-o", out], check=True)
    lib = C.CDLL(out)
    lib.shim_turns_fixed.restype = C.c_uint64
    lib.shim_turns_fixed.argtypes = [C.c_double]
    lib.shim_noise_fixed.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int64, C.c_void_p]
    return lib


def circ(a, b):
    """Distance of two phases on the 2^64 circle."""
    d = (a - b) % M64
    return min(d, M64 - d)


def exact_turns(f: Fraction) -> int:
    return math.floor((f - math.floor(f)) * M64)


def test_turns_fixed_is_the_fraction_of_a_turn(shim):
    rng = np.random.default_rng(1)
    xs = list(rng.uniform(-1e6, 1e6, 300)) + list(rng.uniform(-1, 1, 100)) + [0.0, 1.0, -1.0, 0.5, -0.5, 3.25,
                                                                                 -1e-300, 1e-300, 12345.0]
    for x in xs:
        got = shim.shim_turns_fixed(float(x))
        want = exact_turns(Fraction(float(x)))
        # x - floor(x) is exact for x >= 0; for x < 0 it may round by one unit of the fraction (2^-53)
        tol = 0 if x >= 0 else 1 << 11
        assert circ(got, want) <= tol, (x, got, want)
    assert shim.shim_turns_fixed(0.25) == 1 << 62
    assert shim.shim_turns_fixed(-0.25) == 3 << 62
    assert shim.shim_turns_fixed(7.0) == 0


def test_phase_accumulator_tracks_the_exact_phase_over_a_year(shim):
    rng = np.random.default_rng(2)
    for _ in range(40):
        t0 = float(rng.choice([0.0, rng.uniform(0, 1e7)]))
        dt = float(rng.choice([600.0, 60.0, 3.6, rng.uniform(0.5, 3600)]))
        period = float(rng.choice([86400.0, 43200.0, rng.uniform(3600, 1e6)]))
        phase = float(rng.uniform(-10, 10))
        A, B, s = t0 / period, phase / TWO_PI, dt / period
        ph0 = shim.shim_turns_fixed(A + B)
        pst = shim.shim_turns_fixed(s)
        for n in [0, 1, 2, 17, 1000, 52559, 52560, 400000]:
            got = (ph0 + n * pst) % M64
            want = exact_turns(Fraction(t0) / Fraction(period) + Fraction(phase) / Fraction(TWO_PI)
                               + n * Fraction(dt) / Fraction(period))
            # double rounding of t0 / period, phase / 2 pi, their sum and dt / period, and the truncations
            bound = (abs(A) + abs(B) + abs(A + B)) * 2.0 ** -53 + n * (s * 2.0 ** -53 + 2.0 ** -64) + 3 * 2.0 ** -64
            assert circ(got, want) <= 2 * bound * M64 + 4, (t0, dt, period, phase, n)
            # the kernels take the top 32 bits: the phase is right to well within one of those units
            assert circ(got, want) < 1 << 24


def noise(lib, t0, dt, noise_dt, L):
    out = np.zeros(3, np.int64)
    lib.shim_noise_fixed(t0, dt, noise_dt, L, out.ctypes.data)
    return [int(v) for v in out]


def round_half_away(f: Fraction) -> int:
    return int(math.floor(f + Fraction(1, 2))) if f >= 0 else -int(math.floor(-f + Fraction(1, 2)))


def test_noise_position_and_first_held_step(shim):
    rng = np.random.default_rng(3)
    cases = [(0.0, 600.0, 3600.0, 8762), (0.0, 3600.0, 3600.0, 3), (1e7, 600.0, 3600.0, 10), (-5000.0, 600.0, 3600.0, 20),
             (0.0, 600.0, 600.0, 1), (123.0, 0.37, 7.0, 1 << 22)]
    for _ in range(200):
        nd = float(rng.uniform(1, 7200))
        cases.append((float(rng.uniform(-1e5, 1e7)), float(rng.uniform(0.5, 7200)), nd, int(rng.integers(1, 20000))))
    for t0, dt, nd, L in cases:
        npos0, nstep, n_hi = noise(shim, t0, dt, nd, L)
        assert npos0 == round_half_away(Fraction(t0 / nd) * (1 << 40))
        assert nstep == round_half_away(Fraction(dt / nd) * (1 << 40))
        target = (L - 1) << 40
        assert n_hi >= 0
        assert npos0 + n_hi * nstep >= target, (t0, dt, nd, L)
        if n_hi > 0:
            assert npos0 + (n_hi - 1) * nstep < target, (t0, dt, nd, L)
        # the positions the kernel forms before n_hi stay inside 64 bits
        assert abs(npos0) + n_hi * nstep < 1 << 63
