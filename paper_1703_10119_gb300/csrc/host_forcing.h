// Host side of the FP32 forcing: the fixed-point accumulators that let a kernel form the ambient air of
// step n ([eq:HAM_BC] boundary data at t^n = t0 + n dt) with integer arithmetic only, no FP64 per step.
// Plain C++ without CUDA: the library (hygro_api.cu) includes it, and the CPU tests compile it on their own.
#pragma once

#include <stdint.h>

#include <cmath>

namespace hygro {

// The fraction of x in [0, 1), scaled by 2^64 (a sinusoid's phase in turns, modulo one turn). For
// |x| < 2^52, x - floor(x) is exact; the scaling is exact; the conversion truncates.
inline uint64_t turns_fixed(double x)
{
    const double f = x - std::floor(x);
    const double s = std::ldexp(f, 64);
    if (!(s < 18446744073709551616.0)) return 0;   // f rounded up to one turn
    if (s < 0) return 0;
    return (uint64_t)s;
}

// Position in a noise table (entries, scaled by 2^40) of step n: npos0 + n nstep, held at the last entry
// (len - 1) from step n_hi on, so the kernel never forms a product that could overflow.
struct NoiseFixed {
    int64_t npos0;
    int64_t nstep;
    int64_t n_hi;   // first step n >= 0 with npos0 + n nstep >= (len - 1) 2^40
};

// Needs noise_dt > 0, len >= 1, |t0 / noise_dt| and dt / noise_dt at most a few million (the library
// refuses larger ratios) so that the scaled values fit in 64 bits.
inline NoiseFixed noise_fixed(double t0, double dt, double noise_dt, int64_t len)
{
    NoiseFixed o;
    o.npos0 = (int64_t)std::llround(std::ldexp(t0 / noise_dt, 40));
    o.nstep = (int64_t)std::llround(std::ldexp(dt / noise_dt, 40));
    const __int128 target = (__int128)(len - 1) << 40;
    o.n_hi = 0;
    if ((__int128)o.npos0 < target) {
        const __int128 need = target - o.npos0;
        o.n_hi = o.nstep > 0 ? (int64_t)((need + o.nstep - 1) / o.nstep) : INT64_MAX;
    }
    return o;
}

}  // namespace hygro
