// Device helpers shared by the 1D kernels: layer constants, face means,
// division, and the ambient air state of a face (paper Sec. 2, [eq:HAM_BC]).
#pragma once

#include <math.h>
#include <stdint.h>

#include "hygro_internal.cuh"

namespace hygro {

template <typename real>
struct LayerC {
    real kMa, kMb;  // kM / (2 dx)  = kMa + kMb P'
    real kTa, kTb;  // kTT / (2 dx) = kTa + kTb P'
    real Aa, Ab;    // dx cM / (2 dt)
    real Ba, Bb;    // dx cTT / (2 dt)
    real chi;       // cTM / cM
};

template <typename real>
__device__ __forceinline__ LayerC<real> load_layer(const real *tab, int l)
{
    const real *p = tab + l * kLayerStride;
    LayerC<real> c;
    c.kMa = p[LT_KMA];
    c.kMb = p[LT_KMB];
    c.kTa = p[LT_KTA];
    c.kTb = p[LT_KTB];
    c.Aa = p[LT_AA];
    c.Ab = p[LT_AB];
    c.Ba = p[LT_BA];
    c.Bb = p[LT_BB];
    c.chi = p[LT_CHI];
    return c;
}

// FP32: a times the hardware approximate reciprocal of b (one MUFU op); FP64: IEEE division.
__device__ __forceinline__ float fast_div(float a, float b)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b));
    return a * r;
}
__device__ __forceinline__ double fast_div(double a, double b) { return a / b; }

// Face conductance / dx from the two half values kh = k / (2 dx) of the
// adjacent nodes: arithmetic mean inside a layer (kh_l + kh_r = (k_l + k_r)
// / (2 dx)), harmonic mean across a layer interface (4 kh_l kh_r / (kh_l +
// kh_r) = 2 k_l k_r / ((k_l + k_r) dx)).
template <typename real>
__device__ __forceinline__ real face_harmonic(real a, real b)
{
    return fast_div(real(4) * a * b, a + b);
}

// A (T, Pv) pair with component-wise arithmetic, in the order of the stored pairs (x = T, y = Pv):
// FP32 pairs use the packed f32x2 instructions (one instruction for both components, each rounded as
// the scalar operation), FP64 pairs scalar operations.
template <typename real>
struct P2;
template <>
struct P2<float> {
    uint64_t v;
};
template <>
struct P2<double> {
    double x, y;
};

__device__ __forceinline__ P2<float> p2_make(float t, float p)
{
    P2<float> r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(t), "f"(p));
    return r;
}
__device__ __forceinline__ float p2_t(P2<float> a) { return __uint_as_float((uint32_t)a.v); }
__device__ __forceinline__ float p2_p(P2<float> a) { return __uint_as_float((uint32_t)(a.v >> 32)); }
__device__ __forceinline__ P2<float> p2_add(P2<float> a, P2<float> b)
{
    P2<float> r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ P2<float> p2_sub(P2<float> a, P2<float> b)
{
    P2<float> r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ P2<float> p2_mul(P2<float> a, P2<float> b)
{
    P2<float> r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ P2<float> p2_fma(P2<float> a, P2<float> b, P2<float> c)
{
    P2<float> r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
__device__ __forceinline__ P2<float> p2_load(const float2 *p)
{
    P2<float> r;
    r.v = *reinterpret_cast<const uint64_t *>(p);
    return r;
}
__device__ __forceinline__ void p2_store(float2 *p, P2<float> a) { *reinterpret_cast<uint64_t *>(p) = a.v; }

__device__ __forceinline__ P2<double> p2_make(double t, double p) { return P2<double>{t, p}; }
__device__ __forceinline__ double p2_t(P2<double> a) { return a.x; }
__device__ __forceinline__ double p2_p(P2<double> a) { return a.y; }
__device__ __forceinline__ P2<double> p2_add(P2<double> a, P2<double> b) { return P2<double>{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ P2<double> p2_sub(P2<double> a, P2<double> b) { return P2<double>{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ P2<double> p2_mul(P2<double> a, P2<double> b) { return P2<double>{a.x * b.x, a.y * b.y}; }
__device__ __forceinline__ P2<double> p2_fma(P2<double> a, P2<double> b, P2<double> c)
{
    return P2<double>{fma(a.x, b.x, c.x), fma(a.y, b.y, c.y)};
}
__device__ __forceinline__ P2<double> p2_load(const double2 *p)
{
    const double2 v = *p;
    return P2<double>{v.x, v.y};
}
__device__ __forceinline__ void p2_store(double2 *p, P2<double> a) { *p = make_double2(a.x, a.y); }

// ---- ambient forcing -------------------------------------------------------

// sin(2 pi x) for x = ph / 2^64 (ph: fraction of a turn in 0.64 fixed point).
__device__ __forceinline__ float sin_turns_fx(uint64_t ph)
{
    const int32_t hi = (int32_t)(uint32_t)(ph >> 32);        // signed turn fraction in [-1/2, 1/2)
    const float x = (float)hi * 2.3283064365386963e-10f;     // 2^-32
    return __sinf(6.2831853071795865f * x);
}

// Linear interpolation of a (T, Pv) table at position pos / 2^40, held at
// the end values outside [0, len - 1].
__device__ __forceinline__ float2 noise_fx(const float2 *tab, int32_t len, int64_t pos)
{
    if (len <= 0) return make_float2(0.f, 0.f);
    if (pos <= 0) return tab[0];
    const int64_t i = pos >> 40;
    if (i >= (int64_t)len - 1) return tab[len - 1];
    const float f = (float)((pos >> 16) & 0xFFFFFF) * (1.0f / 16777216.0f);
    const float2 a = tab[i], b = tab[i + 1];
    return make_float2(fmaf(f, b.x - a.x, a.x), fmaf(f, b.y - a.y, a.y));
}

// Ambient air (deviation from the wall reference) of face fi at step n, FP32 path.
__device__ __forceinline__ void ambient_at(const FaceInfo &fi, const float2 *noise, int64_t n, double /*t0*/,
                                           double /*dt*/, float &T, float &P)
{
    T = (float)fi.T_mean_dev;
    P = (float)fi.P_mean_dev;
    const uint64_t un = (uint64_t)n;
    if (fi.period > 0.0) T = fmaf((float)fi.T_amp, sin_turns_fx(fi.phT0 + un * fi.pstep), T);
    if (fi.period_P > 0.0) P = fmaf((float)fi.P_amp, sin_turns_fx(fi.phP0 + un * fi.pstepP), P);
    if (fi.noise_len > 0) {
        // position = npos0 + n * nstep up to the last table entry (from step n_hi on the table is held
        // at its end, and the product is not formed, so it cannot overflow)
        const int64_t pos = n >= fi.n_hi ? ((int64_t)(fi.noise_len - 1) << 40) : fi.npos0 + n * fi.nstep;
        const float2 v = noise_fx(noise + fi.noise_off, fi.noise_len, pos);
        T += v.x;
        P += v.y;
    }
}

// Ambient air of face fi at step n, FP64 path: the same expression as the
// definition, t = t0 + n dt.
__device__ __forceinline__ void ambient_at(const FaceInfo &fi, const float2 *noise, int64_t n, double t0, double dt,
                                           double &T, double &P)
{
    const double t = t0 + (double)n * dt;
    const double two_pi = 6.283185307179586476925286766559;
    T = fi.T_mean_dev;
    P = fi.P_mean_dev;
    if (fi.period > 0.0) T += fi.T_amp * sin(two_pi * t / fi.period + fi.phase_T);
    if (fi.period_P > 0.0) P += fi.P_amp * sin(two_pi * t / fi.period_P + fi.phase_P);
    if (fi.noise_len > 0 && fi.noise_dt > 0.0) {
        const float2 *tab = noise + fi.noise_off;
        const double x = t / fi.noise_dt;
        double nT, nP;
        if (x <= 0.0) {
            nT = tab[0].x;
            nP = tab[0].y;
        } else if (x >= (double)(fi.noise_len - 1)) {
            nT = tab[fi.noise_len - 1].x;
            nP = tab[fi.noise_len - 1].y;
        } else {
            const double i = floor(x);
            const int64_t k = (int64_t)i;
            const double f = x - i;
            nT = (1.0 - f) * (double)tab[k].x + f * (double)tab[k + 1].x;
            nP = (1.0 - f) * (double)tab[k].y + f * (double)tab[k + 1].y;
        }
        T += nT;
        P += nP;
    }
}

}  // namespace hygro
