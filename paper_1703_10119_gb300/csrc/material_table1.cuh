// The load bearing material of Sec. 4 (Table 1) as a coefficient law of the DF update: the six
// coefficients of [eq:HAM_equation2] at a node's absolute (T, Pv) of level n.
//   saturation pressure: Ps = 610.94 exp(17.625 theta / (theta + 243.04)) Pa, theta = T - 273.15 C (the
//     paper gives none; the Magnus form of Alduchov & Eskridge 1996);
//   capillary pressure (Kelvin relation, Sec. 2): Pc = rho_l Rv T ln(Pv / Ps), held at 0 above saturation;
//   sorption isotherm: f = 47.1 (1 + (-c1 Pc)^1.65)^-0.39 + 109.9 (1 + (-c2 Pc)^6)^-0.83 kg/m3;
//   cM = f'(phi) / Ps = (df/dPc) rho_l Rv T / Pv; vapour permeability dv = 1.88e-6 / T * s / (0.503 s^2 +
//   0.497), s = 1 - f / 157; kTT = lambda = 0.2 + 0.0045 f; cTT = rho0 c0 + cw f; kTM = Lv dv;
//   cTM = cw theta cM; kM = 1.97e-10 exp(1.44 - 0.07 log10 x) + 1.77e-7 L(x), x = 2 Pv / Ps, with the
//   liquid term L of Table 1's garbled bracket read as (exp(-8x-2))^2 (HYGRO_LAW_TABLE1), exp((-8x-2)^2)
//   (HYGRO_LAW_TABLE1_A) or exp(-8 (x-2)^2) (HYGRO_LAW_TABLE1_C).
#pragma once

#include <math.h>

#include "../../include/hygro.h"

namespace hygro {

template <typename real>
struct LawCoef {
    real kM, cM, kTT, cTT, kTM, cTM;
};

template <typename real>
__device__ __forceinline__ LawCoef<real> table1_law(int law, real T, real Pv, real Lv)
{
    const real theta = T - real(273.15);
    const real Ps = real(610.94) * exp(real(17.625) * theta / (theta + real(243.04)));
    const real rlRvT = real(1000.0 * 461.5) * T;                 // rho_l Rv T
    const real Pc = fmin(real(0), rlRvT * log(Pv / Ps));
    const real y1 = real(-1.25e-5) * Pc, y2 = real(-1.8e-5) * Pc;  // -c1 Pc, -c2 Pc (>= 0)
    const real p1 = pow(y1, real(0.65)), p2 = pow(y2, real(5));
    const real u1 = real(1) + p1 * y1, u2 = real(1) + p2 * y2;     // 1 + y1^1.65, 1 + y2^6
    const real f = real(47.1) * pow(u1, real(-0.39)) + real(109.9) * pow(u2, real(-0.83));
    // df/dPc of each term a (1 + y^m)^-e, y = -c Pc: a e m c y^(m-1) (1 + y^m)^(-e-1)
    const real dfdPc = real(47.1 * 0.39 * 1.65 * 1.25e-5) * p1 * pow(u1, real(-1.39)) +
                       real(109.9 * 0.83 * 6.0 * 1.8e-5) * p2 * pow(u2, real(-1.83));
    LawCoef<real> k;
    k.cM = dfdPc * rlRvT / Pv;
    const real s = real(1) - f / real(157);
    const real dv = real(1.88e-6) / T * s / (real(0.503) * s * s + real(0.497));
    const real x = real(2) * Pv / Ps;
    real liquid;
    if (law == HYGRO_LAW_TABLE1_A) {
        const real z = real(-8) * x - real(2);
        liquid = exp(z * z);
    } else if (law == HYGRO_LAW_TABLE1_C) {
        const real z = x - real(2);
        liquid = exp(real(-8) * z * z);
    } else {
        const real e = exp(real(-8) * x - real(2));
        liquid = e * e;
    }
    k.kM = real(1.97e-10) * exp(real(1.44) - real(0.07) * log10(x)) + real(1.77e-7) * liquid;
    k.kTT = real(0.2) + real(0.0045) * f;
    k.cTT = real(790.0 * 870.0) + real(4180) * f;
    k.kTM = Lv * dv;
    k.cTM = real(4180) * theta * k.cM;
    return k;
}

}  // namespace hygro
