// Reverse-time adjoint of the DF wall update: the sensor-misfit loss of a run and its gradient with
// respect to every layer's parameters (kM0, a, cM0, b, kTT0, aT, cTT0, bT, chi).
//
// One warp per wall. The wall's levels, adjoint variables and scatter buffers live in the warp's
// shared memory; lane l owns the contiguous nodes [start[l], start[l+1]), all of one layer, so that its
// nine parameter sums stay in registers (compensated sums within a segment, FP64 across segments).
//   1. forward run from the uniform initial state, saving (level n-1, level n) every C steps and
//      accumulating the misfit of the surface values in FP64;
//   2. segments from the last to the first: recompute the segment's levels from its checkpoint into a
//      global buffer, then walk its steps backwards, applying the transposed Jacobian of each step to the
//      adjoint of the level it produced (the reverse of the increment form, operation by operation).
// Per node j (weights w = 1/2 at the surfaces, deviation variables, kh = k / (2 dx)):
//   numP = sum_f FM_f (P_nb - p-) + hM (P_inf - p-),  S = sum_f FM_f + hM,  dP = (numP + g) / (A + S/2)
//   X = numP - S dP / 2
//   numT = sum_f FT_f (T_nb - t-) + hT (T_inf - t-) + q + Lv X - chi A dP,  ST = sum_f FT_f + hT,
//   dT = numT / (B + ST/2);   P+ = p- + dP, T+ = t- + dT
// FM_f = khM_j + khM_nb inside a layer, 4 khM_j khM_nb / (khM_j + khM_nb) across layers (FT likewise),
// A = w dx cM / (2 dt), B = w dx cTT / (2 dt), coefficients at level n ([eq:DF_NL], Pv first, [eq:DF_eq2]).
#pragma once

#include "df1d_common.cuh"

namespace hygro {

constexpr int kAdjAirChunk = 64;   // steps of ambient air computed at a time
constexpr int kAdjWarps = 4;       // warps (walls) per block at most

struct AdjWall {
    int32_t N, node_off, layer_off, n_layers;
    int16_t start[33];   // lane l owns nodes [start[l], start[l+1])
    int8_t layer[32];    // layer of lane l's nodes (-1: no nodes)
    int32_t kt;          // register kernel: slots per lane (>= the longest run); 0: shared-memory kernel
    int32_t dense;       // every run that holds nodes has kt - 1 or kt of them
    double dx;
    int64_t ck_off, seg_off;   // first real of the wall's checkpoints and segment levels
};

template <typename real>
struct AdjDev {
    const AdjWall *walls;
    int32_t W, Nmax;
    const FaceInfo *faces;      // [W][2]
    const real *layer_tab;      // [sum layers][kLayerStride] (deviation form of the context)
    const real *phys;           // [sum layers][9] kM0, a, cM0, b, kTT0, aT, cTT0, bT, chi
    const real *Pref, *Tref;    // [W]
    const float2 *noise;
    const float *obs;           // [K][W][2][2] observed (T, Pv), absolute
    double wT, wP;
    int32_t se, K;              // samples after every se-th step, K of them
    int64_t n_steps;
    int32_t C, n_seg;           // checkpoint stride and count
    const int32_t *list;        // walls of this launch (one warp each)
    int32_t n_list;
    // Per wall, at ckpt + ck_off / seg + seg_off, with Ns = Nmax (shared-memory kernel, node-major) or
    // kt x 32 (register kernel, slot-major: slot i of lane l at i * 32 + l):
    real *ckpt;                 // [n_seg][4][Ns]: T(n-1), T(n), P(n-1), P(n) at n = c C
    real *seg;                  // [C + 2][2][Ns]: T, P of levels c C - 1 .. (c + 1) C
    double *loss;               // [W]
    double *grad;               // [sum layers][9]
    int32_t *nonfinite;
    double dt, t0, Lv, Psat;
};

// Shared-memory arrays of one warp, each Nmax reals: three level slots of T and of Pv, three adjoint
// slots of T and of Pv, the neighbour scatter buffers and the face adjoints; then the air of
// kAdjAirChunk steps.
enum { AS_T0, AS_T1, AS_T2, AS_P0, AS_P1, AS_P2, AS_A0, AS_A1, AS_A2, AS_B0, AS_B1, AS_B2, AS_TTL, AS_TTR, AS_TPL,
       AS_TPR, AS_FML, AS_FMR, AS_FTL, AS_FTR, AS_COUNT };

template <typename real>
__host__ __device__ constexpr size_t adj_smem_per_warp(int Nmax)
{
    return ((size_t)AS_COUNT * Nmax + (size_t)kAdjAirChunk * 4) * sizeof(real);
}

// Constants of a lane's layer.
template <typename real>
struct AdjLayer {
    real kMa, kMb, kTa, kTb, Aa, Ab, Ba, Bb, chi;   // deviation form (kh, storage)
};

template <typename real>
__device__ __forceinline__ void adj_load_layer(AdjLayer<real> &c, const real *q)
{
    c.kMa = q[LT_KMA];
    c.kMb = q[LT_KMB];
    c.kTa = q[LT_KTA];
    c.kTb = q[LT_KTB];
    c.Aa = q[LT_AA];
    c.Ab = q[LT_AB];
    c.Ba = q[LT_BA];
    c.Bb = q[LT_BB];
    c.chi = q[LT_CHI];
}

// Compensated (Neumaier) running sum.
template <typename real>
struct KSum {
    real s, c;
    __device__ __forceinline__ void add(real x)
    {
        const real t = s + x;
        c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
        s = t;
    }
    __device__ __forceinline__ real value() const { return s + c; }
};

// Per-wall state of the warp.
template <typename real>
struct AdjWarp {
    const AdjDev<real> *d;
    int w, lane, N, s0, s1;       // this lane's nodes [s0, s1)
    int lay;                      // this lane's layer (local index), -1 if none
    int layL, layR;               // layer of node s0 - 1 and of node s1 (-1 outside the wall)
    AdjLayer<real> c;             // this lane's layer
    real khMaL, khMbL, khTaL, khTbL, khMaR, khMbR, khTaR, khTbR;   // kh laws of the outer neighbours
    real *sm;                     // this warp's shared arrays
    real *air;                    // [kAdjAirChunk][4]: T_inf', P_inf' of face 0, face 1
    int64_t air_chunk;            // chunk held in air, -1 none
    const FaceInfo *f0, *f1;
    real hT0, hM0, q0, g0, hT1, hM1, q1, g1;
    real Pr;                      // reference Pv of the wall (the deviations are relative to it)
    int lp, lc, ln;               // level slots: n-1, n, n+1 (0..2)
    int al, am, an;               // adjoint slots: complete (n+1), partial (n), fresh (n-1)
    KSum<real> acc[9];            // raw parameter sums of the lane's layer in the current segment
    __device__ __forceinline__ real *arr(int k) const { return sm + (size_t)k * d->Nmax; }
    __device__ __forceinline__ real *T(int slot) const { return arr(AS_T0 + slot); }
    __device__ __forceinline__ real *P(int slot) const { return arr(AS_P0 + slot); }
    __device__ __forceinline__ real *AT(int slot) const { return arr(AS_A0 + slot); }
    __device__ __forceinline__ real *AP(int slot) const { return arr(AS_B0 + slot); }
};

// ambient air of both faces for the chunk of kAdjAirChunk steps holding step n (warp-uniform)
template <typename real>
__device__ __forceinline__ void adj_air(AdjWarp<real> &x, int64_t n)
{
    const int64_t ch = n / kAdjAirChunk;
    if (ch == x.air_chunk) return;
    __syncwarp();
    for (int i = x.lane; i < 2 * kAdjAirChunk; i += 32) {
        const int s = i >> 1, f = i & 1;
        const FaceInfo &fi = f ? *x.f1 : *x.f0;
        real aT = real(0), aP = real(0);
        if (fi.kind == HYGRO_BC_AMBIENT) ambient_at(fi, x.d->noise, ch * kAdjAirChunk + s, x.d->t0, x.d->dt, aT, aP);
        x.air[s * 4 + f * 2] = aT;
        x.air[s * 4 + f * 2 + 1] = aP;
    }
    x.air_chunk = ch;
    __syncwarp();
}

// Forward quantities of node j at step n that both the forward and the reverse need.
template <typename real>
struct AdjNode {
    real w, pc, pp, tp, khM, khT, A, B;
    real pl, pr, tl, tr;          // level-n neighbours (0 where absent)
    real FML, FMR, FTL, FTR;      // face conductances (0 where absent)
    real S, ST, numP, numT0, src; // sums (numT0 without the latent and storage terms)
    bool hl, hr;                  // harmonic left / right faces
};

template <typename real>
__device__ __forceinline__ void adj_node(const AdjWarp<real> &x, int j, const real *air, AdjNode<real> &o)
{
    const real *Tp = x.T(x.lp), *Tc = x.T(x.lc), *Pp = x.P(x.lp), *Pc = x.P(x.lc);
    const real half = real(0.5);
    const int N = x.N;
    o.w = (j == 0 || j == N - 1) ? half : real(1);
    o.pc = Pc[j];
    o.pp = Pp[j];
    o.tp = Tp[j];
    o.khM = fma(x.c.kMb, o.pc, x.c.kMa);
    o.khT = fma(x.c.kTb, o.pc, x.c.kTa);
    o.A = o.w * fma(x.c.Ab, o.pc, x.c.Aa);
    o.B = o.w * fma(x.c.Bb, o.pc, x.c.Ba);
    o.pl = o.pr = o.tl = o.tr = real(0);
    o.FML = o.FMR = o.FTL = o.FTR = real(0);
    o.numP = o.S = o.numT0 = o.ST = o.src = real(0);
    o.hl = o.hr = false;
    if (j > 0) {
        o.hl = j == x.s0 && x.layL != x.lay;
        o.pl = Pc[j - 1];
        o.tl = Tc[j - 1];
        const real kM2 = o.hl ? fma(x.khMbL, o.pl, x.khMaL) : fma(x.c.kMb, o.pl, x.c.kMa);
        const real kT2 = o.hl ? fma(x.khTbL, o.pl, x.khTaL) : fma(x.c.kTb, o.pl, x.c.kTa);
        o.FML = o.hl ? face_harmonic(o.khM, kM2) : o.khM + kM2;
        o.FTL = o.hl ? face_harmonic(o.khT, kT2) : o.khT + kT2;
        o.numP = fma(o.FML, o.pl - o.pp, o.numP);
        o.S += o.FML;
        o.numT0 = fma(o.FTL, o.tl - o.tp, o.numT0);
        o.ST += o.FTL;
    }
    if (j < N - 1) {
        o.hr = j == x.s1 - 1 && x.layR != x.lay;
        o.pr = Pc[j + 1];
        o.tr = Tc[j + 1];
        const real kM2 = o.hr ? fma(x.khMbR, o.pr, x.khMaR) : fma(x.c.kMb, o.pr, x.c.kMa);
        const real kT2 = o.hr ? fma(x.khTbR, o.pr, x.khTaR) : fma(x.c.kTb, o.pr, x.c.kTa);
        o.FMR = o.hr ? face_harmonic(o.khM, kM2) : o.khM + kM2;
        o.FTR = o.hr ? face_harmonic(o.khT, kT2) : o.khT + kT2;
        o.numP = fma(o.FMR, o.pr - o.pp, o.numP);
        o.S += o.FMR;
        o.numT0 = fma(o.FTR, o.tr - o.tp, o.numT0);
        o.ST += o.FTR;
    }
    if (j == 0) {
        o.numP = fma(x.hM0, air[1] - o.pp, o.numP);
        o.S += x.hM0;
        o.src += x.g0;
        o.numT0 = fma(x.hT0, air[0] - o.tp, o.numT0 + x.q0);
        o.ST += x.hT0;
    }
    if (j == N - 1) {
        o.numP = fma(x.hM1, air[3] - o.pp, o.numP);
        o.S += x.hM1;
        o.src += x.g1;
        o.numT0 = fma(x.hT1, air[2] - o.tp, o.numT0 + x.q1);
        o.ST += x.hT1;
    }
}

// Forward DF step of the lane's nodes: slots lp (n-1), lc (n) -> ln (n+1).
template <typename real>
__device__ __forceinline__ void adj_forward(const AdjWarp<real> &x, int64_t n)
{
    real *Tn = x.T(x.ln), *Pn = x.P(x.ln);
    const real *air = x.air + (n % kAdjAirChunk) * 4;
    const real half = real(0.5), Lv = (real)x.d->Lv;
    for (int j = x.s0; j < x.s1; ++j) {
        AdjNode<real> o;
        adj_node(x, j, air, o);
        const real dP = (o.numP + o.src) / fma(half, o.S, o.A);
        const real X = fma(-o.S, half * dP, o.numP);
        real numT = fma(Lv, X, o.numT0);
        numT = fma(-x.c.chi * o.A, dP, numT);
        const real dT = numT / fma(half, o.ST, o.B);
        Pn[j] = o.pp + dP;
        Tn[j] = o.tp + dT;
    }
}

// Reverse of the step n -> n+1, phase A (the lane's own nodes): from the complete adjoint of level n+1
// (slot al), the fresh adjoint of level n-1 (slot an, own nodes), the storage terms' contribution to the
// partial adjoint of level n (slot am), the contributions to the neighbours' level-n adjoints and the
// face adjoints (scatter arrays), and the storage / chi parameter sums.
template <typename real>
__device__ __forceinline__ void adj_reverse_a(AdjWarp<real> &x, int64_t n)
{
    const real *Tn = x.T(x.ln), *Pn = x.P(x.ln), *lT = x.AT(x.al), *lP = x.AP(x.al);
    real *nT = x.AT(x.an), *nP = x.AP(x.an), *mP = x.AP(x.am);
    real *TTL = x.arr(AS_TTL), *TTR = x.arr(AS_TTR), *TPL = x.arr(AS_TPL), *TPR = x.arr(AS_TPR);
    real *FML = x.arr(AS_FML), *FMR = x.arr(AS_FMR), *FTL = x.arr(AS_FTL), *FTR = x.arr(AS_FTR);
    const real *air = x.air + (n % kAdjAirChunk) * 4;
    const real half = real(0.5), Lv = (real)x.d->Lv, Ps = (real)x.d->Psat;
    real sA = real(0), sAr = real(0), sB = real(0), sBr = real(0), schi = real(0);
    for (int j = x.s0; j < x.s1; ++j) {
        AdjNode<real> o;
        adj_node(x, j, air, o);
        const real D = fma(half, o.S, o.A), E = fma(half, o.ST, o.B);
        const real dP = (o.numP + o.src) / D;   // the forward's increments, recomputed
        const real X = fma(-o.S, half * dP, o.numP);
        real numT = fma(Lv, X, o.numT0);
        numT = fma(-x.c.chi * o.A, dP, numT);
        const real dT = numT / E;
        (void)Tn;
        (void)Pn;
        // T update: T+ = t- + numT / E
        const real gdT = lT[j];
        const real gnumT = gdT / E;
        const real gE = -gdT * dT / E;
        real gtp = gdT - gnumT * o.ST;      // t- in every (T_nb - t-) and (T_inf - t-) term
        real gB = gE;
        const real gST = half * gE;
        const real gFTL = gnumT * (o.tl - o.tp) + gST, gFTR = gnumT * (o.tr - o.tp) + gST;
        const real gtl = gnumT * o.FTL, gtr = gnumT * o.FTR;
        const real gX = gnumT * Lv;
        real gA = -gnumT * x.c.chi * dP;
        real gdP = lP[j] - gnumT * x.c.chi * o.A;
        schi -= gnumT * o.A * dP;
        // X = numP - S dP / 2
        real gnumP = gX;
        real gS = -gX * half * dP;
        gdP -= gX * half * o.S;
        // dP = (numP + src) / D, D = A + S / 2
        gnumP += gdP / D;
        const real gD = -gdP * dP / D;
        gA += gD;
        gS += half * gD;
        const real gpp = lP[j] - gnumP * o.S;   // P+ = p- + dP; p- in every (P_nb - p-) and (P_inf - p-)
        const real gFML = gnumP * (o.pl - o.pp) + gS, gFMR = gnumP * (o.pr - o.pp) + gS;
        const real gpl = gnumP * o.FML, gpr = gnumP * o.FMR;
        // storage laws A = w (Aa + Ab P'), B = w (Ba + Bb P') at level n
        const real gLA = gA * o.w, gLB = gB * o.w;
        const real r = (x.Pr + o.pc) / Ps;
        sA += gLA;
        sAr += gLA * r;
        sB += gLB;
        sBr += gLB * r;
        mP[j] += gLA * x.c.Ab + gLB * x.c.Bb;
        nT[j] = gtp;
        nP[j] = gpp;
        TTL[j] = gtl;
        TTR[j] = gtr;
        TPL[j] = gpl;
        TPR[j] = gpr;
        FML[j] = gFML;
        FMR[j] = gFMR;
        FTL[j] = gFTL;
        FTR[j] = gFTR;
    }
    x.acc[2].add(sA);
    x.acc[3].add(sAr);
    x.acc[6].add(sB);
    x.acc[7].add(sBr);
    x.acc[8].add(schi);
}

// Phase B (after a warp sync): the face adjoints of both faces of each node -> half-conductance adjoints
// -> conductivity parameter sums and the node's level-n adjoint; the neighbours' contributions to it.
template <typename real>
__device__ __forceinline__ void adj_reverse_b(AdjWarp<real> &x)
{
    const real *Pc = x.P(x.lc);
    real *mT = x.AT(x.am), *mP = x.AP(x.am);
    const real *TTL = x.arr(AS_TTL), *TTR = x.arr(AS_TTR), *TPL = x.arr(AS_TPL), *TPR = x.arr(AS_TPR);
    const real *FML = x.arr(AS_FML), *FMR = x.arr(AS_FMR), *FTL = x.arr(AS_FTL), *FTR = x.arr(AS_FTR);
    const int N = x.N;
    const real Ps = (real)x.d->Psat;
    real sM = real(0), sMr = real(0), sT = real(0), sTr = real(0);
    for (int j = x.s0; j < x.s1; ++j) {
        const real pc = Pc[j];
        const real khM = fma(x.c.kMb, pc, x.c.kMa), khT = fma(x.c.kTb, pc, x.c.kTa);
        real gkhM = real(0), gkhT = real(0), gT = real(0), gP = real(0);
        if (j > 0) {
            // face (j-1, j): adjoint from node j-1 (its right face) and node j (its left face)
            const real tM = FMR[j - 1] + FML[j], tT = FTR[j - 1] + FTL[j];
            if (j == x.s0 && x.layL != x.lay) {
                const real pl = Pc[j - 1];
                const real kM2 = fma(x.khMbL, pl, x.khMaL), kT2 = fma(x.khTbL, pl, x.khTaL);
                const real uM = khM + kM2, uT = khT + kT2;
                gkhM += tM * real(4) * kM2 * kM2 / (uM * uM);
                gkhT += tT * real(4) * kT2 * kT2 / (uT * uT);
            } else {
                gkhM += tM;
                gkhT += tT;
            }
            gT += TTR[j - 1];   // node j-1's right neighbour is j
            gP += TPR[j - 1];
        }
        if (j < N - 1) {
            const real tM = FMR[j] + FML[j + 1], tT = FTR[j] + FTL[j + 1];
            if (j == x.s1 - 1 && x.layR != x.lay) {
                const real pr = Pc[j + 1];
                const real kM2 = fma(x.khMbR, pr, x.khMaR), kT2 = fma(x.khTbR, pr, x.khTaR);
                const real uM = khM + kM2, uT = khT + kT2;
                gkhM += tM * real(4) * kM2 * kM2 / (uM * uM);
                gkhT += tT * real(4) * kT2 * kT2 / (uT * uT);
            } else {
                gkhM += tM;
                gkhT += tT;
            }
            gT += TTL[j + 1];   // node j+1's left neighbour is j
            gP += TPL[j + 1];
        }
        gP += gkhM * x.c.kMb + gkhT * x.c.kTb;   // kh = ka + kb P' at level n
        const real r = (x.Pr + pc) / Ps;
        sM += gkhM;
        sMr += gkhM * r;
        sT += gkhT;
        sTr += gkhT * r;
        mT[j] += gT;
        mP[j] += gP;
    }
    x.acc[0].add(sM);
    x.acc[1].add(sMr);
    x.acc[4].add(sT);
    x.acc[5].add(sTr);
}

// The lane's raw sums -> parameter gradients of its layer (FP64, added to the wall's layers):
//   kh_M = kM0 (1 + a r) / (2 dx):        dL/dkM0 = (S0 + a S1) / (2 dx),   dL/da = kM0 S1 / (2 dx)
//   A-law = dx cM0 (1 + b r) / (2 dt):   dL/dcM0 = dx (S2 + b S3) / (2 dt), dL/db = dx cM0 S3 / (2 dt)
//   kTT and cTT likewise (S4, S5; S6, S7); chi: S8.
template <typename real>
__device__ __forceinline__ void adj_fold(const AdjDev<real> &d, const AdjWall &aw, int lay, KSum<real> (&acc)[9])
{
    if (lay >= 0) {
        const real *p = d.phys + (size_t)(aw.layer_off + lay) * 9;
        double *g = d.grad + (size_t)(aw.layer_off + lay) * 9;
        const double dx = aw.dx, dt = d.dt;
        double s[9];
        for (int k = 0; k < 9; ++k) s[k] = (double)acc[k].value();
        const double kM0 = p[0], a = p[1], cM0 = p[2], b = p[3], kTT0 = p[4], aT = p[5], cTT0 = p[6], bT = p[7];
        atomicAdd(g + 0, (s[0] + a * s[1]) / (2.0 * dx));
        atomicAdd(g + 1, kM0 * s[1] / (2.0 * dx));
        atomicAdd(g + 2, dx * (s[2] + b * s[3]) / (2.0 * dt));
        atomicAdd(g + 3, dx * cM0 * s[3] / (2.0 * dt));
        atomicAdd(g + 4, (s[4] + aT * s[5]) / (2.0 * dx));
        atomicAdd(g + 5, kTT0 * s[5] / (2.0 * dx));
        atomicAdd(g + 6, dx * (s[6] + bT * s[7]) / (2.0 * dt));
        atomicAdd(g + 7, dx * cTT0 * s[7] / (2.0 * dt));
        atomicAdd(g + 8, s[8]);
    }
    for (int k = 0; k < 9; ++k) acc[k].s = acc[k].c = real(0);
}

template <typename real>
__global__ void __launch_bounds__(32 * kAdjWarps) adjoint_kernel(const AdjDev<real> d)
{
    extern __shared__ __align__(16) unsigned char adj_smem[];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wi = blockIdx.x * (blockDim.x >> 5) + wib;
    if (wi >= d.n_list) return;   // the whole warp
    const int w = d.list[wi];
    const AdjWall &aw = d.walls[w];
    AdjWarp<real> x;
    x.d = &d;
    x.w = w;
    x.lane = lane;
    x.N = aw.N;
    x.s0 = aw.start[lane];
    x.s1 = aw.start[lane + 1];
    x.lay = aw.layer[lane];
    x.layL = -1;
    x.layR = -1;
    for (int l = lane - 1; l >= 0; --l)
        if (aw.start[l] < aw.start[l + 1]) {
            x.layL = aw.layer[l];
            break;
        }
    for (int l = lane + 1; l < 32; ++l)
        if (aw.start[l] < aw.start[l + 1]) {
            x.layR = aw.layer[l];
            break;
        }
    const real *tab = d.layer_tab + (size_t)aw.layer_off * kLayerStride;
    if (x.lay >= 0) adj_load_layer(x.c, tab + x.lay * kLayerStride);
    x.khMaL = x.khMbL = x.khTaL = x.khTbL = x.khMaR = x.khMbR = x.khTaR = x.khTbR = real(0);
    if (x.layL >= 0) {
        const real *q = tab + x.layL * kLayerStride;
        x.khMaL = q[LT_KMA];
        x.khMbL = q[LT_KMB];
        x.khTaL = q[LT_KTA];
        x.khTbL = q[LT_KTB];
    }
    if (x.layR >= 0) {
        const real *q = tab + x.layR * kLayerStride;
        x.khMaR = q[LT_KMA];
        x.khMbR = q[LT_KMB];
        x.khTaR = q[LT_KTA];
        x.khTbR = q[LT_KTB];
    }
    x.sm = reinterpret_cast<real *>(adj_smem + (size_t)wib * adj_smem_per_warp<real>(d.Nmax));
    x.air = x.sm + (size_t)AS_COUNT * d.Nmax;
    x.air_chunk = -1;
    x.f0 = d.faces + (size_t)w * 2;
    x.f1 = x.f0 + 1;
    const bool a0 = x.f0->kind == HYGRO_BC_AMBIENT, a1 = x.f1->kind == HYGRO_BC_AMBIENT;
    x.hT0 = a0 ? (real)x.f0->hT : real(0);
    x.hM0 = a0 ? (real)x.f0->hM : real(0);
    x.q0 = a0 ? (real)x.f0->q_inf : real(0);
    x.g0 = a0 ? (real)x.f0->g_inf : real(0);
    x.hT1 = a1 ? (real)x.f1->hT : real(0);
    x.hM1 = a1 ? (real)x.f1->hM : real(0);
    x.q1 = a1 ? (real)x.f1->q_inf : real(0);
    x.g1 = a1 ? (real)x.f1->g_inf : real(0);
    x.Pr = d.Pref[w];
    const real Tr = d.Tref[w];
    for (int k = 0; k < 9; ++k) x.acc[k].s = x.acc[k].c = real(0);
    const int N = x.N, Nm = d.Nmax;
    real *ck = d.ckpt + aw.ck_off;
    real *sg = d.seg + aw.seg_off;

    // 1. forward from the uniform initial state (zero deviations; level -1 := level 0)
    x.lp = 0;
    x.lc = 1;
    x.ln = 2;
    for (int j = x.s0; j < x.s1; ++j) {
        x.T(0)[j] = x.T(1)[j] = real(0);
        x.P(0)[j] = x.P(1)[j] = real(0);
    }
    __syncwarp();
    double loss = 0.0;
    bool bad = false;
    for (int64_t n = 0; n < d.n_steps; ++n) {
        if (n % d.C == 0) {
            real *c4 = ck + (size_t)(n / d.C) * 4 * Nm;
            for (int j = x.s0; j < x.s1; ++j) {
                c4[j] = x.T(x.lp)[j];
                c4[Nm + j] = x.T(x.lc)[j];
                c4[2 * Nm + j] = x.P(x.lp)[j];
                c4[3 * Nm + j] = x.P(x.lc)[j];
            }
        }
        adj_air(x, n);
        adj_forward(x, n);
        __syncwarp();
        if ((n + 1) % d.se == 0 && (n + 1) / d.se <= d.K) {
            const int64_t k = (n + 1) / d.se - 1;
            for (int f = 0; f < 2; ++f) {
                const int j = f == 0 ? 0 : N - 1;
                if (j >= x.s0 && j < x.s1) {
                    const float *o = d.obs + ((size_t)k * d.W + w) * 4 + f * 2;
                    const double eT = (double)x.T(x.ln)[j] + (double)Tr - (double)o[0];
                    const double eP = (double)x.P(x.ln)[j] + (double)x.Pr - (double)o[1];
                    loss += d.wT * eT * eT + d.wP * eP * eP;
                    bad |= !isfinite(eT) || !isfinite(eP);
                }
            }
        }
        const int t = x.lp;
        x.lp = x.lc;
        x.lc = x.ln;
        x.ln = t;
    }
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if (lane == 0) d.loss[w] = loss;

    // 2. reverse. Adjoint slots: al = complete adjoint of level n+1, am = partial of level n.
    x.al = 0;
    x.am = 1;
    x.an = 2;
    for (int j = x.s0; j < x.s1; ++j) {
        x.AT(0)[j] = x.AP(0)[j] = x.AT(1)[j] = x.AP(1)[j] = real(0);
    }
    // direct term of the last level (slot lc holds level n_steps)
    auto direct = [&](int64_t lev, int slot, int aslot) {
        if (lev >= 1 && lev % d.se == 0 && lev / d.se <= d.K) {
            const int64_t k = lev / d.se - 1;
            for (int f = 0; f < 2; ++f) {
                const int j = f == 0 ? 0 : N - 1;
                if (j >= x.s0 && j < x.s1) {
                    const float *o = d.obs + ((size_t)k * d.W + w) * 4 + f * 2;
                    x.AT(aslot)[j] += (real)(2.0 * d.wT * ((double)x.T(slot)[j] + (double)Tr - (double)o[0]));
                    x.AP(aslot)[j] += (real)(2.0 * d.wP * ((double)x.P(slot)[j] + (double)x.Pr - (double)o[1]));
                }
            }
        }
    };
    direct(d.n_steps, x.lc, x.al);
    __syncwarp();
    for (int c = d.n_seg - 1; c >= 0; --c) {
        const int64_t start = (int64_t)c * d.C;
        const int64_t end = start + d.C < d.n_steps ? start + d.C : d.n_steps;
        // recompute the segment from its checkpoint: slots lp / lc <- levels start - 1, start
        const real *c4 = ck + (size_t)c * 4 * Nm;
        x.lp = 0;
        x.lc = 1;
        x.ln = 2;
        for (int j = x.s0; j < x.s1; ++j) {
            x.T(0)[j] = c4[j];
            x.T(1)[j] = c4[Nm + j];
            x.P(0)[j] = c4[2 * Nm + j];
            x.P(1)[j] = c4[3 * Nm + j];
            sg[j] = c4[j];
            sg[Nm + j] = c4[2 * Nm + j];
            sg[2 * Nm + j] = c4[Nm + j];
            sg[3 * Nm + j] = c4[3 * Nm + j];
        }
        __syncwarp();
        for (int64_t n = start; n < end; ++n) {
            adj_air(x, n);
            adj_forward(x, n);
            __syncwarp();
            real *s2 = sg + (size_t)(n + 1 - start + 1) * 2 * Nm;
            for (int j = x.s0; j < x.s1; ++j) {
                s2[j] = x.T(x.ln)[j];
                s2[Nm + j] = x.P(x.ln)[j];
            }
            const int t = x.lp;
            x.lp = x.lc;
            x.lc = x.ln;
            x.ln = t;
        }
        // slots now: lp = level end - 1, lc = level end; reverse needs (n-1, n, n+1) = (end-2, end-1, end)
        {
            const int t = x.ln;
            x.ln = x.lc;
            x.lc = x.lp;
            x.lp = t;
            if (end - 2 >= start - 1) {
                const real *s2 = sg + (size_t)(end - 2 - start + 1) * 2 * Nm;
                for (int j = x.s0; j < x.s1; ++j) {
                    x.T(x.lp)[j] = s2[j];
                    x.P(x.lp)[j] = s2[Nm + j];
                }
            }
        }
        __syncwarp();
        for (int64_t n = end - 1; n >= start; --n) {
            direct(n, x.lc, x.am);
            adj_air(x, n);
            adj_reverse_a(x, n);
            __syncwarp();
            adj_reverse_b(x);
            __syncwarp();
            // level n is complete: shift the adjoint slots; the levels move down one
            const int ta = x.al;
            x.al = x.am;
            x.am = x.an;
            x.an = ta;
            if (n > start) {
                const int tl = x.ln;
                x.ln = x.lc;
                x.lc = x.lp;
                x.lp = tl;
                const real *s2 = sg + (size_t)(n - 2 - start + 1) * 2 * Nm;
                for (int j = x.s0; j < x.s1; ++j) {
                    x.T(x.lp)[j] = s2[j];
                    x.P(x.lp)[j] = s2[Nm + j];
                }
                __syncwarp();
            }
        }
        adj_fold(d, aw, x.lay, x.acc);
    }
    for (int j = x.s0; j < x.s1; ++j) bad |= !isfinite(x.AT(x.al)[j]) || !isfinite(x.AP(x.al)[j]);
    if (bad) atomicExch(d.nonfinite, 1);
}

}  // namespace hygro
