// Register-resident form of the reverse-time adjoint (the arithmetic of adjoint.cuh, same loss and
// gradient): one warp per wall, lane l owns the run of nodes [start[l], start[l+1]) of one layer, held
// in KT register slots (slot i = node start[l] + i; slots at and beyond the run length nl are idle and
// held at zero). Neighbours across lanes come by shuffles; the three level sets and the two adjoint sets
// rotate by renaming (the time loops advance two steps per iteration); the segment levels of the
// reverse sweep are stored slot-major (slot i of lane l at i * 32 + l), so every global access of a warp
// is one 128-byte line per slot.
//
// Per node (increment form of the DF step, deviation variables, kh = k / (2 dx), Robin faces as faces
// with conductance h towards the ambient air):
//   numP = FML (pl - p-) + FMR (pr - p-),  S = FML + FMR,  D = A + S / 2,  dP = (numP + g) / D
//   X = numP - S dP / 2,  numT = FTL (tl - t-) + FTR (tr - t-) + q + Lv X - chi A dP,  E = B + ST / 2
//   P+ = p- + dP,  T+ = t- + numT / E
// The reverse applies the transposed Jacobian of these operations in the opposite order ([eq:DF_NL],
// [eq:DF_eq2]; coefficients at level n, Pv first).
#pragma once

#include "adjoint.cuh"

namespace hygro {

// longest lane run the register kernel holds, by precision (longer runs take the shared-memory kernel)
template <typename real>
__host__ __device__ constexpr int adj_reg_max_k()
{
    return sizeof(real) == 4 ? 16 : 8;
}

// register slots per lane for a run of k nodes: the instantiated sizes
__host__ __device__ constexpr int adj_reg_slots(int k)
{
    return k <= 2 ? 2 : k <= 8 ? k : k <= 10 ? 10 : k <= 12 ? 12 : k <= 14 ? 14 : k <= 16 ? 16 : 0;
}

template <typename real>
__device__ __forceinline__ real adj_rcp(real x);
template <>
__device__ __forceinline__ float adj_rcp<float>(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <>
__device__ __forceinline__ double adj_rcp<double>(double x)
{
    return 1.0 / x;
}

// Slot predicates. A lane's run holds slots [0, nl). DENSE walls have every run that holds nodes at KT - 1
// or KT nodes, so only the last two slots depend on nl there; lanes without nodes then compute values
// that no other lane reads (the last lane with nodes takes the ambient air on its right).
template <int KT, bool DENSE>
__device__ __forceinline__ bool s_fixed(int i)
{
    return DENSE && i + 2 < KT;
}
template <int KT, bool DENSE>
__device__ __forceinline__ bool s_act(int i, int nl)
{
    return s_fixed<KT, DENSE>(i) || i < nl;
}
template <int KT, bool DENSE>
__device__ __forceinline__ bool s_last(int i, int nl)
{
    return !s_fixed<KT, DENSE>(i) && i == nl - 1;
}
template <int KT, bool DENSE>
__device__ __forceinline__ bool s_inR(int i, int nl)
{
    return s_fixed<KT, DENSE>(i) || i + 1 < nl;
}

// Constants of one lane.
template <typename real>
struct RegLane {
    int lane, nl;                 // lane, nodes of its run (0: idle)
    int lay;                      // its layer (local index), -1 if idle
    bool lsurf, rsurf;            // the run holds node 0 / node N-1
    bool hl, hr;                  // the faces to the neighbour lanes' runs are layer interfaces
    AdjLayer<real> c;
    real kLa, kLb, tLa, tLb, kRa, kRb, tRa, tRb;   // kh laws (kM, kTT) of the neighbour lanes' layers
    real hT0, hM0, q0, g0, hT1, hM1, q1, g1;       // surface faces (0 for adiabatic)
    real Pr, Tr, Lv, rPs;
};

// The lane's edges at level n: neighbour values and face conductances of slot 0 (left) and of the last
// slot nl - 1 (right), the surface sources, and the quantities the reverse needs at the edges.
template <typename real>
struct RegEdge {
    real XLP, XLT, FLM, FLT;      // left neighbour (or ambient air) and the left face of slot 0
    real XRP, XRT, FRM, FRT;      // right neighbour (or ambient air) and the right face of the last slot
    real gf, qf, gl, ql;          // vapour / heat sources of slot 0 and of the last slot
    real kLM, kLT, kRM, kRT;      // kh of the neighbour nodes across the lane edges
    real pcl, khlM, khlT;         // the last slot's Pv and kh
};

template <typename real, int KT, bool DENSE>
__device__ __forceinline__ void reg_edges(const RegLane<real> &L, const real (&tc)[KT], const real (&pc)[KT],
                                          const real (&khM)[KT], const real (&khT)[KT], const real *air,
                                          RegEdge<real> &e)
{
    real pcl = pc[0], tcl = tc[0];
#pragma unroll
    for (int i = 1; i < KT; ++i) {
        pcl = s_last<KT, DENSE>(i, L.nl) ? pc[i] : pcl;
        tcl = s_last<KT, DENSE>(i, L.nl) ? tc[i] : tcl;
    }
    const unsigned full = 0xffffffffu;
    const real pLn = __shfl_up_sync(full, pcl, 1), tLn = __shfl_up_sync(full, tcl, 1);
    const real pRn = __shfl_down_sync(full, pc[0], 1), tRn = __shfl_down_sync(full, tc[0], 1);
    e.pcl = pcl;
    e.khlM = fma(L.c.kMb, pcl, L.c.kMa);
    e.khlT = fma(L.c.kTb, pcl, L.c.kTa);
    e.kLM = fma(L.kLb, pLn, L.kLa);
    e.kLT = fma(L.tLb, pLn, L.tLa);
    e.kRM = fma(L.kRb, pRn, L.kRa);
    e.kRT = fma(L.tRb, pRn, L.tRa);
    const real FLMi = L.hl ? face_harmonic(khM[0], e.kLM) : khM[0] + e.kLM;
    const real FLTi = L.hl ? face_harmonic(khT[0], e.kLT) : khT[0] + e.kLT;
    const real FRMi = L.hr ? face_harmonic(e.khlM, e.kRM) : e.khlM + e.kRM;
    const real FRTi = L.hr ? face_harmonic(e.khlT, e.kRT) : e.khlT + e.kRT;
    e.XLP = L.lsurf ? air[1] : pLn;
    e.XLT = L.lsurf ? air[0] : tLn;
    e.FLM = L.lsurf ? L.hM0 : FLMi;
    e.FLT = L.lsurf ? L.hT0 : FLTi;
    e.XRP = L.rsurf ? air[3] : pRn;
    e.XRT = L.rsurf ? air[2] : tRn;
    e.FRM = L.rsurf ? L.hM1 : FRMi;
    e.FRT = L.rsurf ? L.hT1 : FRTi;
    e.gf = L.lsurf ? L.g0 : real(0);
    e.qf = L.lsurf ? L.q0 : real(0);
    e.gl = L.rsurf ? L.g1 : real(0);
    e.ql = L.rsurf ? L.q1 : real(0);
}

// Forward quantities of slot i that the step and its reverse share.
template <typename real>
struct RegSlot {
    real w, A, S, ST, numP, numT0, src, pl, pr, tl, tr, FML, FMR, FTL, FTR, D, rD, dP, E, rE, dT;
};

template <typename real, int KT, bool DENSE>
__device__ __forceinline__ void reg_slot(const RegLane<real> &L, const RegEdge<real> &e, const real (&tp)[KT],
                                         const real (&pp)[KT], const real (&tc)[KT], const real (&pc)[KT],
                                         const real (&khM)[KT], const real (&khT)[KT], const int i, RegSlot<real> &o)
{
    const real half = real(0.5);
    const bool lastslot = s_last<KT, DENSE>(i, L.nl), inR = s_inR<KT, DENSE>(i, L.nl);
    const int im = i > 0 ? i - 1 : 0, ip = i + 1 < KT ? i + 1 : i;
    if (i == 0) {
        o.pl = e.XLP;
        o.tl = e.XLT;
        o.FML = e.FLM;
        o.FTL = e.FLT;
    } else {
        o.pl = pc[im];
        o.tl = tc[im];
        o.FML = khM[im] + khM[i];
        o.FTL = khT[im] + khT[i];
    }
    o.pr = inR ? pc[ip] : e.XRP;
    o.tr = inR ? tc[ip] : e.XRT;
    o.FMR = inR ? khM[i] + khM[ip] : e.FRM;
    o.FTR = inR ? khT[i] + khT[ip] : e.FRT;
    const bool surf = (i == 0 && L.lsurf) || (lastslot && L.rsurf);
    o.w = surf ? half : real(1);
    o.src = (i == 0 ? e.gf : real(0)) + (lastslot ? e.gl : real(0));
    const real q = (i == 0 ? e.qf : real(0)) + (lastslot ? e.ql : real(0));
    o.A = o.w * fma(L.c.Ab, pc[i], L.c.Aa);
    const real B = o.w * fma(L.c.Bb, pc[i], L.c.Ba);
    o.S = o.FML + o.FMR;
    o.ST = o.FTL + o.FTR;
    o.numP = fma(o.FMR, o.pr - pp[i], o.FML * (o.pl - pp[i]));
    o.numT0 = fma(o.FTR, o.tr - tp[i], fma(o.FTL, o.tl - tp[i], q));
    o.D = fma(half, o.S, o.A);
    o.rD = adj_rcp(o.D);
    o.dP = (o.numP + o.src) * o.rD;
    const real X = fma(-o.S, half * o.dP, o.numP);
    real numT = fma(L.Lv, X, o.numT0);
    numT = fma(-L.c.chi * o.A, o.dP, numT);
    o.E = fma(half, o.ST, B);
    o.rE = adj_rcp(o.E);
    o.dT = numT * o.rE;
}

template <typename real, int KT>
__device__ __forceinline__ void reg_kh(const RegLane<real> &L, const real (&pc)[KT], real (&khM)[KT], real (&khT)[KT])
{
#pragma unroll
    for (int i = 0; i < KT; ++i) {
        khM[i] = fma(L.c.kMb, pc[i], L.c.kMa);
        khT[i] = fma(L.c.kTb, pc[i], L.c.kTa);
    }
}

// One DF step of the lane's slots: (tp, pp) = level n-1 is overwritten with level n+1.
template <typename real, int KT, bool DENSE>
__device__ __forceinline__ void reg_forward(const RegLane<real> &L, real (&tp)[KT], real (&pp)[KT],
                                            const real (&tc)[KT], const real (&pc)[KT], const real *air)
{
    real khM[KT], khT[KT];
    reg_kh(L, pc, khM, khT);
    RegEdge<real> e;
    reg_edges<real, KT, DENSE>(L, tc, pc, khM, khT, air, e);
#pragma unroll
    for (int i = 0; i < KT; ++i) {
        RegSlot<real> o;
        reg_slot<real, KT, DENSE>(L, e, tp, pp, tc, pc, khM, khT, i, o);
        const bool act = s_act<KT, DENSE>(i, L.nl);
        pp[i] = act ? pp[i] + o.dP : real(0);
        tp[i] = act ? tp[i] + o.dT : real(0);
    }
}

// Per-step parameter sums of the lane's layer (raw, before the chain to the layer parameters).
template <typename real>
struct RegSums {
    real s[9];   // kM: S0, S1 (x r); storage A: S2, S3; kTT: S4, S5; storage B: S6, S7; chi: S8
};

// Reverse of the step n -> n+1. In: (tp, pp) level n-1, (tc, pc) level n, (lT, lP) the complete adjoint
// of level n+1, (mT, mP) the partial adjoint of level n. Out: (lT, lP) the partial adjoint of level n-1
// (from this step), (mT, mP) complete.
template <typename real, int KT, bool DENSE>
__device__ __forceinline__ void reg_reverse(const RegLane<real> &L, const real (&tp)[KT], const real (&pp)[KT],
                                            const real (&tc)[KT], const real (&pc)[KT], real (&lT)[KT],
                                            real (&lP)[KT], real (&mT)[KT], real (&mP)[KT], const real *air,
                                            RegSums<real> &g)
{
    const real half = real(0.5);
    real khM[KT], khT[KT];
    reg_kh(L, pc, khM, khT);
    RegEdge<real> e;
    reg_edges<real, KT, DENSE>(L, tc, pc, khM, khT, air, e);
#pragma unroll
    for (int k = 0; k < 9; ++k) g.s[k] = real(0);
    // carried between slots: the previous slot's right-face adjoints and right-neighbour contributions
    real pFM = real(0), pFT = real(0), ptr = real(0), ppr = real(0), pr_i = real(0);
    real l0T = real(0), l0P = real(0), l0FM = real(0), l0FT = real(0);       // slot 0's left side
    real rLT = real(0), rLP = real(0), rLFM = real(0), rLFT = real(0);       // the last slot's right side
#pragma unroll
    for (int i = 0; i < KT; ++i) {
        RegSlot<real> o;
        reg_slot<real, KT, DENSE>(L, e, tp, pp, tc, pc, khM, khT, i, o);
        const bool act = s_act<KT, DENSE>(i, L.nl);
        // T+ = t- + numT / E
        const real gdT = lT[i];
        const real gnumT = gdT * o.rE;
        const real gE = -gnumT * o.dT;
        const real gtp = fma(-gnumT, o.ST, gdT);
        const real gST = half * gE;
        const real gFTL = fma(gnumT, o.tl - tp[i], gST), gFTR = fma(gnumT, o.tr - tp[i], gST);
        const real gtl = gnumT * o.FTL, gtr = gnumT * o.FTR;
        const real gX = gnumT * L.Lv;
        const real cA = gnumT * L.c.chi;
        real gA = -cA * o.dP;
        real gdP = fma(-cA, o.A, lP[i]);
        // X = numP - S dP / 2
        real gS = -gX * half * o.dP;
        gdP = fma(-gX * half, o.S, gdP);
        // dP = (numP + g) / D, D = A + S / 2
        const real gnumP = fma(gdP, o.rD, gX);
        const real gD = -gdP * o.dP * o.rD;
        gA += gD;
        gS = fma(half, gD, gS);
        const real gpp = fma(-gnumP, o.S, lP[i]);
        const real gFML = fma(gnumP, o.pl - pp[i], gS), gFMR = fma(gnumP, o.pr - pp[i], gS);
        const real gpl = gnumP * o.FML, gpr = gnumP * o.FMR;
        // storage laws A = w (Aa + Ab P'), B = w (Ba + Bb P') at level n
        const real gLA = gA * o.w, gLB = gE * o.w;
        const real r = (L.Pr + pc[i]) * L.rPs;
        if (act) {
            g.s[2] += gLA;
            g.s[3] = fma(gLA, r, g.s[3]);
            g.s[6] += gLB;
            g.s[7] = fma(gLB, r, g.s[7]);
            g.s[8] = fma(-gnumT * o.A, o.dP, g.s[8]);
        }
        mP[i] += act ? fma(gLA, L.c.Ab, gLB * L.c.Bb) : real(0);
        lT[i] = act ? gtp : real(0);
        lP[i] = act ? gpp : real(0);
        if (i == 0) {
            l0T = gtl;
            l0P = gpl;
            l0FM = gFML;
            l0FT = gFTL;
        } else {
            // face (i-1, i) inside the run: both sides' face adjoints, arithmetic mean of kh
            const bool in = act;
            const real tM = pFM + gFML, tT = pFT + gFTL;
            const real kk = fma(tM, L.c.kMb, tT * L.c.kTb);
            mP[i - 1] += in ? kk + gpl : real(0);
            mT[i - 1] += in ? gtl : real(0);
            mP[i] += in ? kk + ppr : real(0);
            mT[i] += in ? ptr : real(0);
            if (in) {
                g.s[0] = fma(real(2), tM, g.s[0]);
                g.s[1] = fma(tM, pr_i + r, g.s[1]);
                g.s[4] = fma(real(2), tT, g.s[4]);
                g.s[5] = fma(tT, pr_i + r, g.s[5]);
            }
        }
        if (s_last<KT, DENSE>(i, L.nl)) {
            rLT = gtr;
            rLP = gpr;
            rLFM = gFMR;
            rLFT = gFTR;
        }
        pFM = gFMR;
        pFT = gFTR;
        ptr = gtr;
        ppr = gpr;
        pr_i = r;
    }
    // across the lane edges: slot 0's left side goes to the left lane, the last slot's right side to the
    // right lane
    const unsigned full = 0xffffffffu;
    const real fromR_T = __shfl_down_sync(full, l0T, 1), fromR_P = __shfl_down_sync(full, l0P, 1);
    const real fromR_FM = __shfl_down_sync(full, l0FM, 1), fromR_FT = __shfl_down_sync(full, l0FT, 1);
    const real fromL_T = __shfl_up_sync(full, rLT, 1), fromL_P = __shfl_up_sync(full, rLP, 1);
    const real fromL_FM = __shfl_up_sync(full, rLFM, 1), fromL_FT = __shfl_up_sync(full, rLFT, 1);
    if (L.nl > 0 && !L.lsurf) {
        // face (left lane's last node, slot 0)
        const real tM = fromL_FM + l0FM, tT = fromL_FT + l0FT;
        real eM = tM, eT = tT;
        if (L.hl) {
            const real uM = adj_rcp(khM[0] + e.kLM), uT = adj_rcp(khT[0] + e.kLT);
            const real aM = e.kLM * uM, aT = e.kLT * uT;
            eM = real(4) * tM * aM * aM;
            eT = real(4) * tT * aT * aT;
        }
        const real r0 = (L.Pr + pc[0]) * L.rPs;
        mT[0] += fromL_T;
        mP[0] += fromL_P + fma(eM, L.c.kMb, eT * L.c.kTb);
        g.s[0] += eM;
        g.s[1] = fma(eM, r0, g.s[1]);
        g.s[4] += eT;
        g.s[5] = fma(eT, r0, g.s[5]);
    }
    if (L.nl > 0 && !L.rsurf) {
        // face (last slot, right lane's slot 0)
        const real tM = rLFM + fromR_FM, tT = rLFT + fromR_FT;
        real eM = tM, eT = tT;
        if (L.hr) {
            const real uM = adj_rcp(e.khlM + e.kRM), uT = adj_rcp(e.khlT + e.kRT);
            const real aM = e.kRM * uM, aT = e.kRT * uT;
            eM = real(4) * tM * aM * aM;
            eT = real(4) * tT * aT * aT;
        }
        const real rl = (L.Pr + e.pcl) * L.rPs;
        const real addT = fromR_T, addP = fromR_P + fma(eM, L.c.kMb, eT * L.c.kTb);
#pragma unroll
        for (int i = 0; i < KT; ++i) {
            mT[i] += s_last<KT, DENSE>(i, L.nl) ? addT : real(0);
            mP[i] += s_last<KT, DENSE>(i, L.nl) ? addP : real(0);
        }
        g.s[0] += eM;
        g.s[1] = fma(eM, rl, g.s[1]);
        g.s[4] += eT;
        g.s[5] = fma(eT, rl, g.s[5]);
    }
}

// Ambient air of both faces for the chunk of kAdjAirChunk steps holding step n (warp-uniform).
template <typename real>
__device__ __forceinline__ void reg_air(const AdjDev<real> &d, const FaceInfo &f0, const FaceInfo &f1, real *air,
                                        int64_t &chunk, int64_t n, int lane)
{
    const int64_t ch = n / kAdjAirChunk;
    if (ch == chunk) return;
    __syncwarp();
    for (int i = lane; i < 2 * kAdjAirChunk; i += 32) {
        const int s = i >> 1, f = i & 1;
        const FaceInfo &fi = f ? f1 : f0;
        real aT = real(0), aP = real(0);
        if (fi.kind == HYGRO_BC_AMBIENT) ambient_at(fi, d.noise, ch * kAdjAirChunk + s, d.t0, d.dt, aT, aP);
        air[s * 4 + f * 2] = aT;
        air[s * 4 + f * 2 + 1] = aP;
    }
    chunk = ch;
    __syncwarp();
}

// The value of slot nl - 1 (a run of selects: register arrays take no run-time index).
template <typename real, int KT, bool DENSE>
__device__ __forceinline__ real reg_last(const real (&v)[KT], int nl)
{
    real x = v[0];
#pragma unroll
    for (int i = 1; i < KT; ++i) x = s_last<KT, DENSE>(i, nl) ? v[i] : x;
    return x;
}

template <typename real, int KT, bool DENSE>
__device__ __forceinline__ void reg_add_last(real (&v)[KT], int nl, real a)
{
#pragma unroll
    for (int i = 0; i < KT; ++i) v[i] += s_last<KT, DENSE>(i, nl) ? a : real(0);
}

template <typename real, int KT>
__device__ __forceinline__ void reg_load(real (&v)[KT], const real *src, int lane)
{
#pragma unroll
    for (int i = 0; i < KT; ++i) v[i] = src[i * 32 + lane];
}

template <typename real, int KT>
__device__ __forceinline__ void reg_store(real *dst, const real (&v)[KT], int lane)
{
#pragma unroll
    for (int i = 0; i < KT; ++i) dst[i * 32 + lane] = v[i];
}

template <typename real, int KT>
__device__ __forceinline__ void reg_swap(real (&a)[KT], real (&b)[KT])
{
#pragma unroll
    for (int i = 0; i < KT; ++i) {
        const real t = a[i];
        a[i] = b[i];
        b[i] = t;
    }
}

// Loss and gradient of one wall (the whole warp).
template <typename real, int KT, bool DENSE>
__device__ __noinline__ void adj_reg_wall(const AdjDev<real> &d, const int w, real *air)
{
    const AdjWall &aw = d.walls[w];
    const int lane = threadIdx.x & 31;
    RegLane<real> L;
    L.lane = lane;
    L.nl = aw.start[lane + 1] - aw.start[lane];
    L.lay = aw.layer[lane];
    int last = 0;
    for (int l = 0; l < 32; ++l)
        if (aw.start[l + 1] > aw.start[l]) last = l;
    L.lsurf = lane == 0;
    L.rsurf = lane == last;
    const int layL = lane > 0 ? aw.layer[lane - 1] : -1;
    const int layR = lane < last ? aw.layer[lane + 1] : -1;
    L.hl = L.nl > 0 && layL >= 0 && layL != L.lay;
    L.hr = L.nl > 0 && layR >= 0 && layR != L.lay;
    const real *tab = d.layer_tab + (size_t)aw.layer_off * kLayerStride;
    L.c = AdjLayer<real>{};
    if (L.lay >= 0) adj_load_layer(L.c, tab + L.lay * kLayerStride);
    L.kLa = L.kLb = L.tLa = L.tLb = L.kRa = L.kRb = L.tRa = L.tRb = real(0);
    if (layL >= 0) {
        const real *q = tab + layL * kLayerStride;
        L.kLa = q[LT_KMA];
        L.kLb = q[LT_KMB];
        L.tLa = q[LT_KTA];
        L.tLb = q[LT_KTB];
    }
    if (layR >= 0) {
        const real *q = tab + layR * kLayerStride;
        L.kRa = q[LT_KMA];
        L.kRb = q[LT_KMB];
        L.tRa = q[LT_KTA];
        L.tRb = q[LT_KTB];
    }
    const FaceInfo &f0 = d.faces[(size_t)w * 2], &f1 = d.faces[(size_t)w * 2 + 1];
    const bool a0 = f0.kind == HYGRO_BC_AMBIENT, a1 = f1.kind == HYGRO_BC_AMBIENT;
    L.hT0 = a0 ? (real)f0.hT : real(0);
    L.hM0 = a0 ? (real)f0.hM : real(0);
    L.q0 = a0 ? (real)f0.q_inf : real(0);
    L.g0 = a0 ? (real)f0.g_inf : real(0);
    L.hT1 = a1 ? (real)f1.hT : real(0);
    L.hM1 = a1 ? (real)f1.hM : real(0);
    L.q1 = a1 ? (real)f1.q_inf : real(0);
    L.g1 = a1 ? (real)f1.g_inf : real(0);
    L.Pr = d.Pref[w];
    L.Tr = d.Tref[w];
    L.Lv = (real)d.Lv;
    L.rPs = (real)(1.0 / d.Psat);
    KSum<real> acc[9];
    for (int k = 0; k < 9; ++k) acc[k].s = acc[k].c = real(0);
    int64_t chunk = -1;
    real *ck = d.ckpt + aw.ck_off;
    real *sg = d.seg + aw.seg_off;
    const size_t lev = (size_t)2 * KT * 32;   // reals per stored level (T then Pv)
    const int C = d.C;

    real Tp[KT], Pp[KT], Tc[KT], Pc[KT];
#pragma unroll
    for (int i = 0; i < KT; ++i) Tp[i] = Pp[i] = Tc[i] = Pc[i] = real(0);

    // the misfit of sample k (FP64) from the surface values of its level
    double loss = 0.0;
    bool bad = false;
    const int se = d.se;
    const int64_t Ks = d.K;
    auto misfit = [&](int64_t k, const real (&T)[KT], const real (&P)[KT]) {
        const float *o = d.obs + ((size_t)k * d.W + w) * 4;
        if (L.lsurf && L.nl > 0) {
            const double eT = (double)T[0] + (double)L.Tr - (double)o[0];
            const double eP = (double)P[0] + (double)L.Pr - (double)o[1];
            loss += d.wT * eT * eT + d.wP * eP * eP;
            bad |= !isfinite(eT) || !isfinite(eP);
        }
        const real Tl = reg_last<real, KT, DENSE>(T, L.nl), Plv = reg_last<real, KT, DENSE>(P, L.nl);
        if (L.rsurf && L.nl > 0) {
            const double eT = (double)Tl + (double)L.Tr - (double)o[2];
            const double eP = (double)Plv + (double)L.Pr - (double)o[3];
            loss += d.wT * eT * eT + d.wP * eP * eP;
            bad |= !isfinite(eT) || !isfinite(eP);
        }
    };
    // the misfit's gradient of sample k, added to the adjoint (aT, aP) of its level
    auto direct = [&](int64_t k, const real (&T)[KT], const real (&P)[KT], real (&aT)[KT], real (&aP)[KT]) {
        const float *o = d.obs + ((size_t)k * d.W + w) * 4;
        if (L.lsurf && L.nl > 0) {
            aT[0] += (real)(2.0 * d.wT * ((double)T[0] + (double)L.Tr - (double)o[0]));
            aP[0] += (real)(2.0 * d.wP * ((double)P[0] + (double)L.Pr - (double)o[1]));
        }
        const real Tl = reg_last<real, KT, DENSE>(T, L.nl), Plv = reg_last<real, KT, DENSE>(P, L.nl);
        if (L.rsurf && L.nl > 0) {
            reg_add_last<real, KT, DENSE>(aT, L.nl, (real)(2.0 * d.wT * ((double)Tl + (double)L.Tr - (double)o[2])));
            reg_add_last<real, KT, DENSE>(aP, L.nl, (real)(2.0 * d.wP * ((double)Plv + (double)L.Pr - (double)o[3])));
        }
    };

    // Forward steps [n0, n1) from (Tp, Pp) = level n0-1, (Tc, Pc) = level n0, which end as levels n1-1, n1.
    // first (the first run, n0 = 0): checkpoints every C steps and the misfit; store: each new level goes
    // to the segment buffer (slot s = level start-1+s). Both at once when the run is a single segment:
    // every level is stored by the first run and nothing is recomputed. One rolled loop serves all
    // cases (the kernel's speed follows its code size: the hot loops must stay in the instruction
    // cache); step positions are tracked by counters (no 64-bit division in the loop).
    auto forward = [&](int64_t n0, int64_t n1, bool first, bool store, int64_t start) {
        int cc = 0;            // steps to the next checkpoint (the first run starts on one)
        int64_t ci = 0;        // next checkpoint
        int sc = se;           // steps until the new level is a sample level
        int64_t k = 0;         // next sample
        real *s2 = sg + (size_t)(n0 + 1 - start + 1) * lev;
        for (int64_t n = n0; n < n1; ++n) {
            if (first) {
                if (cc == 0) {
                    real *c4 = ck + (size_t)ci * 2 * lev;
                    reg_store(c4, Tp, lane);
                    reg_store(c4 + KT * 32, Tc, lane);
                    reg_store(c4 + 2 * KT * 32, Pp, lane);
                    reg_store(c4 + 3 * KT * 32, Pc, lane);
                    ++ci;
                    cc = C;
                }
                --cc;
            }
            reg_air(d, f0, f1, air, chunk, n, lane);
            reg_forward<real, KT, DENSE>(L, Tp, Pp, Tc, Pc, air + (int)(n & (kAdjAirChunk - 1)) * 4);
            if (store) {
                reg_store(s2, Tp, lane);
                reg_store(s2 + KT * 32, Pp, lane);
                s2 += lev;
            }
            if (first && --sc == 0) {
                sc = se;
                if (k < Ks) misfit(k, Tp, Pp);
                ++k;
            }
            reg_swap(Tp, Tc);
            reg_swap(Pp, Pc);
        }
    };

    // 1. forward from the uniform initial state (zero deviations; level -1 := level 0)
    const bool single = d.n_seg == 1;
    if (single) {
        reg_store(sg, Tp, lane);
        reg_store(sg + KT * 32, Pp, lane);
        reg_store(sg + lev, Tc, lane);
        reg_store(sg + lev + KT * 32, Pc, lane);
    }
    forward(0, d.n_steps, true, single, 0);
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if (lane == 0) d.loss[w] = loss;

    // 2. reverse, one checkpoint segment at a time from the last
    real LT[KT], LP[KT], MT[KT], MP[KT];
#pragma unroll
    for (int i = 0; i < KT; ++i) LT[i] = LP[i] = MT[i] = MP[i] = real(0);
    for (int c = d.n_seg - 1; c >= 0; --c) {
        const int64_t start = (int64_t)c * C;
        const int64_t end = start + C < d.n_steps ? start + C : d.n_steps;
        // recompute the segment's levels start + 1 .. end into the segment buffer (a single segment was
        // stored by the first run)
        if (!single) {
            const real *c4 = ck + (size_t)c * 2 * lev;
            reg_load(Tp, c4, lane);
            reg_load(Tc, c4 + KT * 32, lane);
            reg_load(Pp, c4 + 2 * KT * 32, lane);
            reg_load(Pc, c4 + 3 * KT * 32, lane);
            reg_store(sg, Tp, lane);
            reg_store(sg + KT * 32, Pp, lane);
            reg_store(sg + lev, Tc, lane);
            reg_store(sg + lev + KT * 32, Pc, lane);
            forward(start, end, false, true, start);
        }
        __syncwarp();
        // sample position of level end: end = kk se + rr
        int64_t kk = end / se;
        int rr = (int)(end - kk * se);
        // the last level's misfit gradient (level n_steps, only in the last segment)
        if (c == d.n_seg - 1) {
            const real *s2 = sg + (size_t)(end - start + 1) * lev;
            reg_load(Tc, s2, lane);
            reg_load(Pc, s2 + KT * 32, lane);
            if (rr == 0 && kk >= 1 && kk <= Ks) direct(kk - 1, Tc, Pc, LT, LP);
        }
        // levels end-2 (slot end-start-1) and end-1 (slot end-start)
        reg_load(Tp, sg + (size_t)(end - start - 1) * lev, lane);
        reg_load(Pp, sg + (size_t)(end - start - 1) * lev + KT * 32, lane);
        reg_load(Tc, sg + (size_t)(end - start) * lev, lane);
        reg_load(Pc, sg + (size_t)(end - start) * lev + KT * 32, lane);
        // reverse step n: (Tp, Pp) = level n-1, (Tc, Pc) = level n, (LT, LP) = complete adjoint of level
        // n+1, (MT, MP) = partial adjoint of level n. The loop is not unrolled; the sets rotate by copies.
        if (rr == 0) {   // position of level end - 1
            rr = se - 1;
            --kk;
        } else {
            --rr;
        }
        for (int64_t n = end - 1; n >= start; --n) {
            // level n-2 (slot n-1-start), loaded ahead; at n = start it is not needed (slot 0 is read)
            real xT[KT], xP[KT];
            {
                const real *sx = sg + (size_t)(n > start ? n - 1 - start : 0) * lev;
                reg_load(xT, sx, lane);
                reg_load(xP, sx + KT * 32, lane);
            }
            if (rr == 0 && kk >= 1 && kk <= Ks) direct(kk - 1, Tc, Pc, MT, MP);
            if (rr == 0) {
                rr = se - 1;
                --kk;
            } else {
                --rr;
            }
            reg_air(d, f0, f1, air, chunk, n, lane);
            RegSums<real> gs;
            reg_reverse<real, KT, DENSE>(L, Tp, Pp, Tc, Pc, LT, LP, MT, MP, air + (int)(n & (kAdjAirChunk - 1)) * 4, gs);
#pragma unroll
            for (int k = 0; k < 9; ++k) acc[k].add(gs.s[k]);
            // levels move down one; the completed adjoint of level n becomes the complete one
#pragma unroll
            for (int i = 0; i < KT; ++i) {
                Tc[i] = Tp[i];
                Pc[i] = Pp[i];
                Tp[i] = xT[i];
                Pp[i] = xP[i];
            }
            reg_swap(LT, MT);
            reg_swap(LP, MP);
        }
        adj_fold(d, aw, L.lay, acc);
        __syncwarp();
    }
#pragma unroll
    for (int i = 0; i < KT; ++i)
        if (i < L.nl) bad |= !isfinite(LT[i]) || !isfinite(LP[i]);
    if (bad) atomicExch(d.nonfinite, 1);
}

template <typename real>
__global__ void __launch_bounds__(32, 8) adjoint_reg_kernel(const __grid_constant__ AdjDev<real> d)
{
    __shared__ __align__(16) real air[kAdjAirChunk * 4];
    if ((int)blockIdx.x >= d.n_list) return;
    const int w = d.list[blockIdx.x];
    const AdjWall &aw = d.walls[w];
    switch (aw.kt * 2 + (aw.dense ? 1 : 0)) {
    case 4: adj_reg_wall<real, 2, false>(d, w, air); break;
    case 5: adj_reg_wall<real, 2, true>(d, w, air); break;
    case 6: adj_reg_wall<real, 3, false>(d, w, air); break;
    case 7: adj_reg_wall<real, 3, true>(d, w, air); break;
    case 8: adj_reg_wall<real, 4, false>(d, w, air); break;
    case 9: adj_reg_wall<real, 4, true>(d, w, air); break;
    case 10: adj_reg_wall<real, 5, false>(d, w, air); break;
    case 11: adj_reg_wall<real, 5, true>(d, w, air); break;
    case 12: adj_reg_wall<real, 6, false>(d, w, air); break;
    case 13: adj_reg_wall<real, 6, true>(d, w, air); break;
    case 14: adj_reg_wall<real, 7, false>(d, w, air); break;
    case 15: adj_reg_wall<real, 7, true>(d, w, air); break;
    case 16: adj_reg_wall<real, 8, false>(d, w, air); break;
    case 17: adj_reg_wall<real, 8, true>(d, w, air); break;
    case 20:
        if constexpr (adj_reg_max_k<real>() >= 10) adj_reg_wall<real, 10, false>(d, w, air);
        break;
    case 21:
        if constexpr (adj_reg_max_k<real>() >= 10) adj_reg_wall<real, 10, true>(d, w, air);
        break;
    case 24:
        if constexpr (adj_reg_max_k<real>() >= 12) adj_reg_wall<real, 12, false>(d, w, air);
        break;
    case 25:
        if constexpr (adj_reg_max_k<real>() >= 12) adj_reg_wall<real, 12, true>(d, w, air);
        break;
    case 28:
        if constexpr (adj_reg_max_k<real>() >= 14) adj_reg_wall<real, 14, false>(d, w, air);
        break;
    case 29:
        if constexpr (adj_reg_max_k<real>() >= 14) adj_reg_wall<real, 14, true>(d, w, air);
        break;
    case 32:
        if constexpr (adj_reg_max_k<real>() >= 16) adj_reg_wall<real, 16, false>(d, w, air);
        break;
    case 33:
        if constexpr (adj_reg_max_k<real>() >= 16) adj_reg_wall<real, 16, true>(d, w, air);
        break;
    default: break;
    }
}

}  // namespace hygro
