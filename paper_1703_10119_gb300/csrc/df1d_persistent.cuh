// Persistent DF kernel for batches of 1D walls: one warp owns one wall and
// advances it through all the steps of a hygro_run call with both time
// levels held in registers.
//
// Lane layout of a wall of N nodes (chosen on the host, WallInfo): K nodes
// per lane, Wl lanes in use, each lane holding K or K-1 consecutive nodes
// (bit i of short_mask: lane i holds K-1, its slot K-1 is a frozen dummy).
// Node 0 sits in lane 0 slot 0 and node N-1 in lane Wl-1 slot K-1 (the last
// lane is always full), so only those two slots carry surface terms. Lanes
// >= Wl hold nothing (all-zero state with zero faces, which stays zero).
// When every layer interface falls on a lane boundary ("aligned" walls,
// the common case) a lane holds one layer and its material constants stay
// in registers; otherwise a variant switches constants inside the lane.
// Neighbour values across lanes move with warp shuffles (4 values each way
// per step); there is no shared-memory traffic and no block barrier in the
// time loop. Per step and node the work is the coefficient evaluation at
// level n (Sec. 2 coefficients, explicit at t^n as in Sec. 3.1), the face
// means, the Pv update and then the T update using Pv^{n+1} (Appendix A
// order), written in increment form:
//   du = [sum_f F_f (u_nb^n - u^{n-1}) + surface terms] / (C + sum_f F_f / 2 + H / 2)
// which is the DF balance of [eq:DF_NL] solved for u^{n+1} - u^{n-1}. The
// latent cross flux of the T equation, sum_f F_f (Pv_nb - Pvbar), reuses the
// Pv numerator: num_P - (S / 2) dPv.
// Surface fluxes are linear in the time-averaged surface values and the air
// values, so a step only adds its surface values to batch sums; the fluxes
// of a batch of 16 steps follow from those sums and the batch's air sums
// ([eq:HAM_BC] summed over the batch), and go to compensated sums that are
// added to FP64 running sums every 16 batches.
#pragma once

#include "df1d_common.cuh"

namespace hygro {

template <typename real>
struct LaneCtx {
    LayerC<real> c0;          // constants of the layer of slot 0
    real clkMa, clkMb;        // kM half-value constants of the last real slot's layer
    real clkTa, clkTb;        // kTT half-value constants of the last real slot's layer
    real w0, w1;              // half-cell weights of slot 0 / slot K-1 (1/2 at a wall surface)
    real hM0, hT0, q0, g0;    // face-0 exchange (lane 0 only, else 0)
    real hM1, hT1, q1, g1;    // face-1 exchange (lane Wl-1 only, else 0)
    real hMs, hTs, qs, gs;    // this lane's face exchange (sum of the two sets above)
    real Lvn;                 // Lv nu: latent heat carried by the moisture flux inside the wall (kTM = nu Lv kM;
                              // simple-heat variants are only used with nu = 1)
    bool nu_corr;             // nu != 1 (warp-uniform)
    uint32_t imask;           // bit k: slot k is the first node of a layer >= 1 (its left face is an interface)
    uint32_t wimask;          // OR of imask bits 1.. over the warp (warp-uniform)
    int l0;                   // layer of slot 0
    bool short_lane;          // lane holds K-1 nodes
    bool face1;               // this lane holds the face-1 surface node (slot K-1)
    bool has_left, has_right; // a face exists between this lane and its neighbour lane
    bool iface_left0;         // the lane-boundary face on the left is an interface
    bool iface_right;         // the lane-boundary face on the right is an interface
    bool any_lb_iface;        // some lane-boundary face of the warp is an interface (warp-uniform)
    // simple-heat walls (kTT, cTT independent of Pv and cTM = 0 in every layer): the thermal faces and the
    // T denominators do not change in time and are set up once per wall
    real FTin;                // in-lane thermal face kTT / dx (one layer per lane)
    real m2FTin;              // -2 FTin
    real FTl0c, FTbc;         // thermal faces at the left / right lane boundary (0 at wall ends)
    real rT0, rTm, rTK2, rTK1; // 1 / T denominator of slot 0, interior slots, slot K-2, slot K-1
};

// One DF step of the lane's K slots: level n+1 is written into Tp / Pp.
// fT, fP: ambient air of this lane's surface face (if any) at level n.
// sT, sP: receive the time-averaged values (u^{n+1} + u^{n-1}) / 2 of this lane's surface node, which
// the Robin exchange of [eq:HAM_BC] uses.
// IFACE: the wall has layer interfaces inside lanes. SIMPLE: simple-heat
// wall (see LaneCtx; only with one layer per lane).
// With IFACE && SIMPLE, sft / srt hold this lane's per-slot right thermal face and reciprocal T
// denominator (stride 32 between slots), set up once per wall.
// VARH (general variants of room walls): the surface thermal conductances of faces 0 and 1 are hT0v, hT1v
// of this step instead of the constant hT0, hT1 (a room face exchanging long-wave radiation).
template <typename real, int K, bool IFACE, bool SIMPLE, bool VARH = false>
__device__ __forceinline__ void df_step(real (&Tp)[K], const real (&Tc)[K], real (&Pp)[K], const real (&Pc)[K],
                                        const LaneCtx<real> &L, const real *tab, const real fT, const real fP,
                                        const real Lv, real &sT, real &sP, const real *sft, const real *srt,
                                        const real hT0v = real(0), const real hT1v = real(0))
{
    constexpr unsigned FULL = 0xffffffffu;
    const real half = real(0.5);

    // the lane's last real node: its values go to the next lane, with the right boundary face
    const real lastT = (K >= 2 && L.short_lane) ? Tc[K >= 2 ? K - 2 : 0] : Tc[K - 1];
    const real lastP = (K >= 2 && L.short_lane) ? Pc[K >= 2 ? K - 2 : 0] : Pc[K - 1];
    const real khM_first = fma(L.c0.kMb, Pc[0], L.c0.kMa);
    const real khM_last = fma(L.clkMb, lastP, L.clkMa);
    // right neighbour of the lane's last node: the next lane's first node, or beyond the face-1 surface
    // the ambient air, entering as a neighbour through a face of conductance hM1 / hT1 (the Robin
    // exchange of [eq:HAM_BC] has the form of a face term)
    real rT = __shfl_down_sync(FULL, Tc[0], 1);
    real rP = __shfl_down_sync(FULL, Pc[0], 1);
    rT = L.has_right ? rT : fT;
    rP = L.has_right ? rP : fP;
    const real rkM = __shfl_down_sync(FULL, khM_first, 1);
    real FMb = khM_last + rkM;
    real FTb;
    if (SIMPLE) {
        FTb = L.FTbc;
    } else {
        const real khT_first = fma(L.c0.kTb, Pc[0], L.c0.kTa);
        const real khT_last = fma(L.clkTb, lastP, L.clkTa);
        const real rkT = __shfl_down_sync(FULL, khT_first, 1);
        FTb = khT_last + rkT;
        if (L.any_lb_iface && L.iface_right) FTb = face_harmonic(khT_last, rkT);
    }
    if (L.any_lb_iface && L.iface_right) FMb = face_harmonic(khM_last, rkM);
    FMb = L.has_right ? FMb : L.hM1;
    if (!SIMPLE) FTb = L.has_right ? FTb : (VARH ? hT1v : L.hT1);
    // left boundary: the previous lane's last node and its right face, or before the face-0 surface
    // the ambient air through hM0 / hT0
    real lT = __shfl_up_sync(FULL, lastT, 1);
    real lP = __shfl_up_sync(FULL, lastP, 1);
    lT = L.has_left ? lT : fT;
    lP = L.has_left ? lP : fP;
    real FMl0 = __shfl_up_sync(FULL, FMb, 1);
    real FTl0;
    if (SIMPLE)
        FTl0 = L.FTl0c;
    else
        FTl0 = __shfl_up_sync(FULL, FTb, 1);
    FMl0 = L.has_left ? FMl0 : L.hM0;
    if (!SIMPLE) FTl0 = L.has_left ? FTl0 : (VARH ? hT0v : L.hT0);

    LayerC<real> c = L.c0;         // constants of the current slot's layer
    int lcur = L.l0;
    real FMl = FMl0, FTl = FTl0;   // left face of the current slot
    real Tl = lT, Pl = lP;         // left neighbour at level n
    real khM = khM_first;
    real khT = SIMPLE ? real(0) : fma(L.c0.kTb, Pc[0], L.c0.kTa);
    real sPbar = real(0), sTbar = real(0);   // time-averaged surface values of this lane's face

#pragma unroll
    for (int k = 0; k < K; ++k) {
        // storage terms of slot k at level n (half-cell weight at the wall surfaces)
        const real Pk = Pc[k];
        real A = fma(c.Ab, Pk, c.Aa);
        real B = SIMPLE ? real(0) : fma(c.Bb, Pk, c.Ba);
        if (k == 0) {
            A *= L.w0;
            if (!SIMPLE) B *= L.w0;
        }
        if (k == K - 1) {
            A *= L.w1;
            if (!SIMPLE) B *= L.w1;
        }
        const real chiA = SIMPLE ? real(0) : c.chi * A;

        // right neighbour and right face
        real FMr, FTr, Tr, Pr, khMn = real(0), khTn = real(0);
        if (k + 1 < K) {
            khMn = fma(c.kMb, Pc[k + 1], c.kMa);
            FMr = khM + khMn;
            if (SIMPLE) {
                FTr = IFACE ? sft[k * 32] : L.FTin;
            } else {
                khTn = fma(c.kTb, Pc[k + 1], c.kTa);
                FTr = khT + khTn;
            }
            if (IFACE) {
                // the next slot may open a new layer (warp-uniform test first)
                if ((L.wimask >> (k + 1)) & 1u) {
                    if ((L.imask >> (k + 1)) & 1u) {
                        ++lcur;
                        c = load_layer(tab, lcur);
                        khMn = fma(c.kMb, Pc[k + 1], c.kMa);
                        FMr = face_harmonic(khM, khMn);
                        if (!SIMPLE) {
                            khTn = fma(c.kTb, Pc[k + 1], c.kTa);
                            FTr = face_harmonic(khT, khTn);
                        }
                    }
                }
            }
            Tr = Tc[k + 1];
            Pr = Pc[k + 1];
            if (k == K - 2) {       // short lanes: slot K-2 is the last real node
                FMr = L.short_lane ? FMb : FMr;
                FTr = L.short_lane ? FTb : FTr;
                Tr = L.short_lane ? rT : Tr;
                Pr = L.short_lane ? rP : Pr;
            }
        } else {
            FMr = FMb;
            FTr = (SIMPLE && IFACE) ? sft[k * 32] : FTb;
            Tr = rT;
            Pr = rP;
            if (K >= 2) {           // short lanes: freeze the dummy slot K-1
                FMl = L.short_lane ? real(0) : FMl;
                FTl = L.short_lane ? real(0) : FTl;
                FMr = L.short_lane ? real(0) : FMr;
                FTr = L.short_lane ? real(0) : FTr;
            }
        }

        // vapour pressure: num = sum_f F (P_nb - P^{n-1}) = sum_f F P_nb - S P^{n-1}, S = sum_f F, the
        // surface faces being the Robin exchanges with the ambient air as neighbour
        const real pp = Pp[k];
        const real S = FMl + FMr;
        const real numP = fma(FMl, Pl, fma(FMr, Pr, -S * pp));
        real numPg = numP;   // + the surface source, on the surface slots only
        if (k == 0) numPg += L.g0;
        if (k == K - 1) numPg += L.g1;
        const real dP = fast_div(numPg, fma(half, S, A));
        // latent cross flux sum_f F (P_nb - Pbar) [+ hM (Pinf - Pbar)] = num - S dP / 2, which the vapour
        // balance of the node, (A + S / 2) dP = num + g, turns into A dP - g
        real X = A * dP;
        if (k == 0) X -= L.g0;
        if (k == K - 1) X -= L.g1;

        // temperature: conduction, Lv x cross flux, cTM storage. Inside a lane of a simple-heat wall
        // without interfaces both thermal faces are FTin: FTin (T_l + T_r) - 2 FTin T^{n-1}.
        const real tp = Tp[k];
        const real ST = SIMPLE ? real(0) : FTl + FTr;
        real numT;
        if (SIMPLE && !IFACE && k >= 1 && k + 2 < K)
            numT = fma(L.m2FTin, tp, L.FTin * (Tl + Tr));
        else if (SIMPLE)
            numT = fma(FTl, Tl - tp, FTr * (Tr - tp));
        else
            numT = fma(FTl, Tl, fma(FTr, Tr, -ST * tp));
        if (k == 0) numT += L.q0;
        if (k == K - 1) numT += L.q1;
        if (SIMPLE) {
            numT = fma(Lv, X, numT);   // simple-heat walls have nu = 1
        } else {
            numT = fma(L.Lvn, X, numT);
            if (L.nu_corr) {
                // X holds the surface exchange too, whose latent heat is Lv hM (Pinf - Pbar) whatever nu
                if (k == 0) numT = fma((Lv - L.Lvn) * L.hM0, fP - fma(half, dP, pp), numT);
                if (k == K - 1) numT = fma((Lv - L.Lvn) * L.hM1, fP - fma(half, dP, pp), numT);
            }
        }
        real dT;
        if (SIMPLE) {
            real r;
            if (IFACE) {
                r = srt[k * 32];
            } else {
                r = L.rTm;
                if (k == K - 2) r = L.rTK2;
                if (k == K - 1) r = L.rTK1;
                if (k == 0) r = L.rT0;
            }
            dT = numT * r;
        } else {
            numT = fma(-chiA, dP, numT);
            dT = fast_div(numT, fma(half, ST, B));
        }
        Pp[k] = pp + dP;
        Tp[k] = tp + dT;

        if (k == 0) {
            sPbar = fma(half, dP, pp);
            sTbar = fma(half, dT, tp);
        }
        if (k == K - 1) {
            sPbar = L.face1 ? fma(half, dP, pp) : sPbar;
            sTbar = L.face1 ? fma(half, dT, tp) : sTbar;
        }

        // advance to the next slot
        Tl = Tc[k];
        Pl = Pk;
        FMl = FMr;
        FTl = FTr;
        khM = khMn;
        khT = khTn;
    }
    sT = sTbar;
    sP = sPbar;
}

constexpr int kRoomAirChunk = 32;   // steps of outdoor air and vapour production computed at a time

// Air state of a room and the level-n surface values of its walls, shared by the room's warps; the
// time-dependent sources of the current chunk of steps.
struct RoomShared {
    double Ta_p, Ta_c, Pa_p, Pa_c;        // levels n-1 and n (the room warp's own history)
    double airT[2], airP[2];              // room air of level n for the walls, slot n & 1
    double surfT[2][HYGRO_MAX_ROOM_WALLS];   // room-side surface T of each wall at level n, slot n & 1
    double surfP[2][HYGRO_MAX_ROOM_WALLS];
    double srcP[kRoomAirChunk];           // g + gv w_out
    double srcT[kRoomAirChunk];           // Q_gain + Lv g + gv cp_a T_out + Lv gv w_out (w_out = Pv_out / Pv_ref)
};

// Time-independent parts of a room's update (FP64).
struct RoomConst {
    double AhT[HYGRO_MAX_ROOM_WALLS], AhM[HYGRO_MAX_ROOM_WALLS];   // A hT, A hM of each wall
    double sAhT, sAhM;        // their sums
    double rhoV, gv, Pref;
    double a_p, k_p;          // vapour node: capacity rho V / Pv_ref / (2 dt), conductance gv / Pv_ref + sum A hM
    double at0, at1;          // heat capacity rho V (cp_a + cp_v Pv / Pv_ref) / (2 dt) = at0 + at1 Pv
    double k_t;               // gv cp_a + sum A hT + G cp_a
    double G;                 // interzone airflow of the room, kg/s (sum over its links)
};

static __device__ __forceinline__ RoomConst room_const(const RoomInfo &ri, const FaceInfo *faces, double dt)
{
    RoomConst k;
    const double *q = ri.par;
    k.sAhT = 0.0;
    k.sAhM = 0.0;
    for (int i = 0; i < ri.n_walls; ++i) {
        const FaceInfo &fc = faces[(size_t)ri.wall[i] * 2 + ri.face[i]];
        k.AhT[i] = ri.area[i] * fc.hT;
        k.AhM[i] = ri.area[i] * fc.hM;
        k.sAhT += k.AhT[i];
        k.sAhM += k.AhM[i];
    }
    k.rhoV = q[RP_RHOA] * q[RP_VOL];
    k.gv = k.rhoV * q[RP_ACH] / 3600.0;
    k.Pref = q[RP_PVREF];
    k.a_p = k.rhoV / k.Pref / (2.0 * dt);
    k.G = 0.0;
    for (int l = 0; l < ri.n_links; ++l) k.G += ri.link_g[l];
    k.k_p = k.gv / k.Pref + k.sAhM + k.G / k.Pref;
    k.at0 = k.rhoV * q[RP_CPA] / (2.0 * dt);
    k.at1 = k.rhoV * q[RP_CPV] / k.Pref / (2.0 * dt);
    k.k_t = k.gv * q[RP_CPA] + k.sAhT + k.G * q[RP_CPA];
    return k;
}

// Outdoor air and vapour production of the steps n_first .. n_first + 31 (lane i: step n_first + i; the
// whole warp), as the time-dependent sources of the room balances.
static __device__ __forceinline__ void room_air_chunk(RoomShared &rs, const RoomInfo &ri, const RoomConst &k,
                                                      int64_t n_first, double t0, double dt, double Lv, int lane)
{
    const double *q = ri.par;
    const double two_pi = 6.283185307179586476925286766559;
    const double t = t0 + (double)(n_first + lane) * dt;
    double T_out = q[RP_TMEAN], P_out = q[RP_PMEAN];
    if (q[RP_PERIOD] > 0.0) T_out += q[RP_TAMP] * sin(two_pi * t / q[RP_PERIOD] + q[RP_PHT]);
    if (q[RP_PERIODP] > 0.0) P_out += q[RP_PAMP] * sin(two_pi * t / q[RP_PERIODP] + q[RP_PHP]);
    // vapour production: the base load plus the daily pulse (occupants' load of Sec. 5.1)
    double g = q[RP_GVAP];
    if (q[RP_PPER] > 0.0) {
        const double ph = fmod(t, q[RP_PPER]);
        if (ph >= q[RP_PON] && ph < q[RP_POFF]) g += q[RP_GPULSE];
    }
    const double w_out = P_out / k.Pref;
    rs.srcP[lane] = g + k.gv * w_out;
    rs.srcT[lane] = q[RP_QGAIN] + Lv * g + k.gv * q[RP_CPA] * T_out + Lv * k.gv * w_out;
}

// Room air node of Sec. 5.1 advanced from level n to n+1 in FP64 with the walls' level-n surface
// values (explicit coupling of [eq:wbse_tn_exp]); the room's own value in its balance is the mean of
// levels n+1 and n-1 (one more DF node), vapour first, heat capacity at level n:
//   a_p (Pa+ - Pa-) = srcP + sum A hM Pvs - k_p Pabar,   k_p = gv / Pv_ref + sum A hM
//   a_t (Ta+ - Ta-) = srcT + sum A hT Ts + Lv sum A hM Pvs - Lv k_p Pabar - k_t Tabar,  k_t = gv cp_a + sum A hT
// i is the step's entry in the chunk, b the buffer of the level-n surface values.
// Interzone airflow (Sec. 5.1, Q_inz and G_inz) enters with the linked rooms' air of level n (all_rs: the
// block's rooms, slot b): the sources sum g cp_a T_o and sum g w_o, the room's own value in k_t and k_p.
static __device__ void room_update(RoomShared &rs, const RoomConst &k, const RoomInfo &ri, int i, int b, double dt,
                                   double Lv, const RoomShared *all_rs)
{
    const double *q = ri.par;
    double AhTTs = 0.0, AhMPs = 0.0;
    for (int w = 0; w < ri.n_walls; ++w) {
        AhTTs = fma(k.AhT[w], rs.surfT[b][w], AhTTs);
        AhMPs = fma(k.AhM[w], rs.surfP[b][w], AhMPs);
    }
    double srcP = rs.srcP[i], srcT = rs.srcT[i];
    if (ri.n_links > 0) {   // a room without links keeps the serial chain of its update short
        double GT = 0.0, Gw = 0.0;
        for (int l = 0; l < ri.n_links; ++l) {
            const RoomShared &o = all_rs[ri.link_slot[l]];
            GT = fma(ri.link_g[l], o.airT[b], GT);
            Gw = fma(ri.link_gw[l], o.airP[b], Gw);
        }
        srcP += Gw;
        srcT += q[RP_CPA] * GT + Lv * Gw;
    }
    if (q[RP_SCHEME] == (double)HYGRO_ROOM_EULER) {
        // explicit Euler of Sec. 5.2: every term at level n
        const double Pa_n = rs.Pa_c + dt * k.Pref / k.rhoV * (srcP + AhMPs - k.k_p * rs.Pa_c);
        const double CT = 2.0 * dt * fma(k.at1, rs.Pa_c, k.at0);
        const double rhs = srcT + AhTTs + Lv * AhMPs - Lv * k.k_p * rs.Pa_c - k.k_t * rs.Ta_c;
        const double Ta_n = rs.Ta_c + dt / CT * rhs;
        rs.Ta_p = rs.Ta_c;
        rs.Ta_c = Ta_n;
        rs.Pa_p = rs.Pa_c;
        rs.Pa_c = Pa_n;
        return;
    }
    const double Pa_n = (fma(k.a_p - 0.5 * k.k_p, rs.Pa_p, srcP) + AhMPs) / (k.a_p + 0.5 * k.k_p);
    const double Pa_bar = 0.5 * (Pa_n + rs.Pa_p);
    const double a_t = fma(k.at1, rs.Pa_c, k.at0);
    const double rhs = srcT + AhTTs + Lv * (AhMPs - k.k_p * Pa_bar);
    const double Ta_n = fma(a_t - 0.5 * k.k_t, rs.Ta_p, rhs) / (a_t + 0.5 * k.k_t);
    rs.Ta_p = rs.Ta_c;
    rs.Ta_c = Ta_n;
    rs.Pa_p = rs.Pa_c;
    rs.Pa_c = Pa_n;
}

// Everything one warp does for one wall over n_steps steps. ROOM: the wall is one of the walls of
// the block's room (rs, its face room_face on the room); every step then ends with the room update
// between two block barriers, which all warps of the block pass once per step.
// Per-lane constants of a wall for the persistent kernel (layout, layer constants, surface exchange,
// and for simple-heat walls the constant thermal faces and T denominators).
template <typename real>
struct WallLane {
    LaneCtx<real> L;
    int first, nreal, my_face;
    const FaceInfo *fw;
    real Tref, Pref;
};

template <typename real, int K, bool IFACE, bool SIMPLE>
__device__ __forceinline__ void lane_setup(const DevCtx<real> &d, const WallInfo &wi, int w, const real *tab,
                                           real *sft, real *srt, WallLane<real> &WLn)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int Wl = wi.Wl;
    const uint32_t smask = (uint32_t)wi.short_mask;
    LaneCtx<real> &L = WLn.L;
    L.short_lane = (K >= 2) && ((smask >> lane) & 1u);
    const int first = lane * K - __popc(smask & ((1u << lane) - 1u));   // wall-local node of slot 0
    const int nreal = lane >= Wl ? 0 : (L.short_lane ? K - 1 : K);
    const int32_t *lf = d.layer_first + wi.layer_off;

    int l0 = 0;
    for (int l = 1; l < wi.n_layers; ++l)
        if (nreal > 0 && first >= lf[l]) l0 = l;
    uint32_t imask = 0;
    bool iface_right = false;
    for (int l = 1; l < wi.n_layers; ++l) {
        const int s = lf[l] - first;
        if (nreal > 0 && s >= 0 && s < nreal) imask |= 1u << s;
        if (nreal > 0 && lf[l] == first + nreal) iface_right = true;
    }
    L.l0 = l0;
    L.imask = imask;
    L.wimask = __reduce_or_sync(FULL, imask) & ~1u;
    L.iface_left0 = (imask & 1u) != 0;
    L.iface_right = iface_right && lane < Wl - 1;
    L.any_lb_iface = __any_sync(FULL, L.iface_left0 || L.iface_right);
    L.has_left = lane >= 1 && lane < Wl;
    L.has_right = lane < Wl - 1;
    L.c0 = load_layer(tab, l0);
    const int llast = l0 + __popc(imask & ~1u);
    const LayerC<real> cl = load_layer(tab, llast);
    L.clkMa = cl.kMa;
    L.clkMb = cl.kMb;
    L.clkTa = cl.kTa;
    L.clkTb = cl.kTb;

    // surface exchange: face 0 on lane 0 slot 0, face 1 on lane Wl-1 slot K-1
    const FaceInfo *fw = d.faces + (size_t)w * 2;
    L.w0 = lane == 0 ? real(0.5) : real(1);
    L.w1 = lane == Wl - 1 ? real(0.5) : real(1);
    L.hM0 = L.hT0 = L.q0 = L.g0 = real(0);
    L.hM1 = L.hT1 = L.q1 = L.g1 = real(0);
    const int my_face = lane == 0 ? 0 : (lane == Wl - 1 ? 1 : -1);
    L.face1 = my_face == 1;
    if (my_face == 0) {
        L.hM0 = (real)fw[0].hM;
        L.hT0 = (real)fw[0].hT;
        L.q0 = (real)fw[0].q_inf;
        L.g0 = (real)fw[0].g_inf;
    } else if (my_face == 1) {
        L.hM1 = (real)fw[1].hM;
        L.hT1 = (real)fw[1].hT;
        L.q1 = (real)fw[1].q_inf;
        L.g1 = (real)fw[1].g_inf;
    }
    L.hMs = L.hM0 + L.hM1;
    L.hTs = L.hT0 + L.hT1;
    L.qs = L.q0 + L.q1;
    L.gs = L.g0 + L.g1;
    const real Lv = (real)d.Lv;
    L.Lvn = (real)(d.Lv * wi.nu);
    L.nu_corr = wi.nu != 1.0;
    const real Tref = d.Tref[w], Pref = d.Pref[w];
    L.FTin = L.m2FTin = L.FTl0c = L.FTbc = real(0);
    L.rT0 = L.rTm = L.rTK2 = L.rTK1 = real(1);
    if (SIMPLE) {
        // constant thermal faces and T denominators B w + (F_left + F_right + hT) / 2
        const real half = real(0.5);
        const real khf = L.c0.kTa;                        // kTT / (2 dx) of slot 0's layer
        const real khl = L.clkTa;                         // of the last real slot's layer
        const real khr = __shfl_down_sync(FULL, khf, 1);  // of the next lane's first slot
        real Fb = L.iface_right ? face_harmonic(khl, khr) : khl + khr;
        Fb = L.has_right ? Fb : real(0);
        real Fl = __shfl_up_sync(FULL, Fb, 1);
        Fl = L.has_left ? Fl : real(0);
        L.FTin = real(2) * khf;
        L.m2FTin = real(-2) * L.FTin;
        L.FTl0c = L.has_left ? Fl : L.hT0;    // the face-0 Robin exchange as the left face of lane 0
        L.FTbc = L.has_right ? Fb : L.hT1;    // the face-1 Robin exchange as the right face of lane Wl-1
        if (!IFACE) {
            const real Bc = L.c0.Ba;
            // slot 0: right face FTin, or the boundary face when slot 0 is the last real slot (K = 1, or
            // K = 2 on a short lane); with K = 1 it is also slot K-1 (both surface sets apply)
            real d0;
            if (K == 1)
                d0 = Bc * L.w0 * L.w1 + half * (Fl + Fb + L.hT0 + L.hT1);
            else
                d0 = Bc * L.w0 + half * (Fl + ((K == 2 && L.short_lane) ? Fb : L.FTin) + L.hT0);
            L.rT0 = real(1) / d0;
            L.rTm = real(1) / (Bc + L.FTin);
            L.rTK2 = real(1) / (Bc + half * (L.FTin + (L.short_lane ? Fb : L.FTin)));
            L.rTK1 = L.short_lane ? real(1) : real(1) / (Bc * L.w1 + half * (L.FTin + Fb + L.hT1));
        } else {
            // per-slot table: layer of each slot, right face (harmonic at an interface, the lane
            // boundary after the last real slot, zero around a short lane's dummy slot) and 1 / denominator
            int l = l0;
            real Fleft = Fl;
            for (int k = 0; k < K; ++k) {
                if (k > 0 && ((imask >> k) & 1u)) ++l;
                const real kh = tab[l * kLayerStride + LT_KTA];
                real Fr;
                if (k + 1 < nreal) {
                    const bool nl = (imask >> (k + 1)) & 1u;
                    const real khn = tab[(l + (nl ? 1 : 0)) * kLayerStride + LT_KTA];
                    Fr = nl ? face_harmonic(kh, khn) : kh + khn;
                } else if (k + 1 == nreal) {
                    Fr = Fb;
                } else {
                    Fr = real(0);
                }
                const bool dummy = k >= nreal;
                const real Fl_k = dummy ? real(0) : Fleft;
                real B = tab[l * kLayerStride + LT_BA];
                real hT = real(0);
                if (k == 0) {
                    B *= L.w0;
                    hT += L.hT0;
                }
                if (k == K - 1) {
                    B *= L.w1;
                    hT += L.hT1;
                }
                // the last real slot of lane Wl-1 faces the ambient air: its right face is hT1
                sft[k * 32] = (k + 1 == nreal && !L.has_right) ? L.hT1 : Fr;
                srt[k * 32] = real(1) / (B + half * (Fl_k + Fr + hT));
                Fleft = Fr;
            }
        }
    }

    WLn.first = first;
    WLn.nreal = nreal;
    WLn.my_face = my_face;
    WLn.fw = fw;
    WLn.Tref = Tref;
    WLn.Pref = Pref;
    (void)Lv;
}

// Room walls (ROOM): rs is the room's shared state, room_face the wall's face on the room, room_slot its
// position among the room's walls, ri the room (long-wave exchange: its view factor and the face's
// emissivity). A radiating room face (RAD, general variants only) receives q_rw = sum over the room's other
// faces of h' (T' - Ts), h' = s eps sigma (T'^2 + Ts^2)(T' + Ts), with h' and T' of level n and Ts averaged
// over levels n+1 and n-1 like the convective exchange: the face's thermal conductance for the step is
// hT + hR (hR = sum h') and its air value (hT Ta + qR) / (hT + hR) (qR = sum h' T').
template <typename real, int K, bool IFACE, bool SIMPLE, bool ROOM = false, bool RAD = false>
__device__ __noinline__ void run_wall(const DevCtx<real> &d, const WallInfo &wi, int w, const real *tab, int64_t n0,
                                      int32_t n_steps, int32_t sample_every, real *samples, real *sft, real *srt,
                                      RoomShared *rs = nullptr, int room_face = -1, int room_slot = 0,
                                      const RoomInfo *ri = nullptr)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int Wl = wi.Wl;
    const uint32_t smask = (uint32_t)wi.short_mask;

    WallLane<real> WLn;
    lane_setup<real, K, IFACE, SIMPLE>(d, wi, w, tab, sft, srt, WLn);
    const LaneCtx<real> &L = WLn.L;
    const int first = WLn.first, nreal = WLn.nreal, my_face = WLn.my_face;
    const FaceInfo *fw = WLn.fw;
    const real Tref = WLn.Tref, Pref = WLn.Pref;
    const real Lv = (real)d.Lv;
    (void)smask;

    // load the two levels
    const int cur = d.cur;
    const size_t base = (size_t)wi.node_off + first;
    real Ta[K], Pa[K], Tb[K], Pb[K];   // a: level n-1 (written with n+1), b: level n
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const bool ok = k < nreal;
        Tb[k] = ok ? d.T[cur][base + k] : real(0);
        Pb[k] = ok ? d.P[cur][base + k] : real(0);
        Ta[k] = ok ? d.T[1 - cur][base + k] : real(0);
        Pa[k] = ok ? d.P[1 - cur][base + k] : real(0);
    }

    double cum_q = 0.0, cum_g = 0.0;
    // surface fluxes: FP32 within a batch of 16 steps, a compensated FP32 sum of 16 batches, then FP64
    real kq = real(0), kq_c = real(0), kg = real(0), kg_c = real(0);
    int kbatches = 0;
    const real dt_r = (real)d.dt;
    if (my_face >= 0) {
        cum_q = d.cumul[(size_t)w * 4 + my_face * 2 + 0];
        cum_g = d.cumul[(size_t)w * 4 + my_face * 2 + 1];
    }
    // values of the last step, for its flux
    real last_sT = real(0), last_sP = real(0), last_fT = real(0), last_fP = real(0);
    int scount = sample_every;
    int64_t sidx = 0;
    const int W = d.W;
    // a sample holds the surface values: lane 0 -> face 0 (slot 0), lane Wl-1 -> face 1 (slot K-1)
    auto sample = [&](const real (&Tn)[K], const real (&Pn)[K]) {
        if (sample_every > 0 && --scount == 0) {
            scount = sample_every;
            if (samples != nullptr && my_face >= 0) {
                real *o = samples + ((size_t)sidx * W + w) * 4 + my_face * 2;
                o[0] = Tref + (my_face == 0 ? Tn[0] : Tn[K - 1]);
                o[1] = Pref + (my_face == 0 ? Pn[0] : Pn[K - 1]);
            }
            ++sidx;
        }
    };

    const int src_base = lane == Wl - 1 ? kForcingBatch : 0;
    const int f_face = lane / kForcingBatch;   // lanes 0..15: face 0, 16..31: face 1
    const FaceInfo &ff = fw[f_face];
    const bool f_ambient = ff.kind == HYGRO_BC_AMBIENT;

    // room coupling: the lane of the room face takes the room air at level n as its ambient air and
    // publishes its surface values for the room update. Step n reads the room air of level n and writes
    // the wall's level-n+1 surface values, while the room warp advances the room from the level-n
    // values (both double-buffered by level parity); one block barrier per step.
    const int room_lane = room_face == 0 ? 0 : Wl - 1;
    const double Tref_d = (double)Tref, Pref_d = (double)Pref;
    // long-wave exchange of the room face (warp-uniform): s eps sigma of this face
    static_assert(!RAD || (ROOM && !SIMPLE), "radiating faces take the general room variants");
    const double rad_c = RAD ? ri->view * ri->emis[room_slot] * 5.670374419e-8 : 0.0;
    const real hT_room = room_face == 0 ? L.hT0 : L.hT1;   // the room face's convective conductance (room lane)
    // sums over the current batch of the lane's time-averaged surface values, and (room walls) of its air
    // and of its radiative exchange
    real acc_sT = real(0), acc_sP = real(0), acc_fT = real(0), acc_fP = real(0), acc_rad = real(0);
    real last_rad = real(0);
    int64_t n_cur = n0;
    auto publish = [&](const real (&T_)[K], const real (&P_)[K], int b) {
        if (lane == room_lane) {
            const int slot = room_face == 0 ? 0 : K - 1;
            real ts = T_[0], ps = P_[0];
#pragma unroll
            for (int k = 1; k < K; ++k) {
                ts = k == slot ? T_[k] : ts;
                ps = k == slot ? P_[k] : ps;
            }
            rs->surfT[b][room_slot] = Tref_d + (double)ts;
            rs->surfP[b][room_slot] = Pref_d + (double)ps;
        }
    };
    auto one_step = [&](auto &Tp_, auto &Tc_, auto &Pp_, auto &Pc_, real bT, real bP, int src) {
        real fT = __shfl_sync(FULL, bT, src);
        real fP = __shfl_sync(FULL, bP, src);
        real fT_step = fT, hT_step = hT_room, hR = real(0), qRd = real(0);
        if (ROOM) {
            if (lane == room_lane) {
                fT = (real)(rs->airT[n_cur & 1] - Tref_d);
                fP = (real)(rs->airP[n_cur & 1] - Pref_d);
                fT_step = fT;
                if (RAD) {
                    // radiative conductances to the room's other faces at level n, in FP64
                    const int b = (int)(n_cur & 1);
                    const double Ts = rs->surfT[b][room_slot];
                    double sh = 0.0, shT = 0.0;
                    for (int u = 0; u < ri->n_walls; ++u) {
                        if (u == room_slot) continue;
                        const double To = rs->surfT[b][u];
                        const double h = rad_c * (To * To + Ts * Ts) * (To + Ts);
                        sh += h;
                        shT = fma(h, To, shT);
                    }
                    hR = (real)sh;
                    qRd = (real)(shT - sh * Tref_d);   // sum h' (T' - T_ref): the deviation form
                    const double hT = (double)hT_room;
                    fT_step = (real)((hT * (double)fT + (shT - sh * Tref_d)) / (hT + sh));
                    hT_step = (real)(hT + sh);
                }
            }
            acc_fT += fT;
            acc_fP += fP;
            last_fT = fT;
            last_fP = fP;
        }
        real sT, sP;
        if constexpr (RAD) {
            const real hT0v = room_face == 0 ? hT_step : L.hT0, hT1v = room_face == 1 ? hT_step : L.hT1;
            df_step<real, K, IFACE, SIMPLE, true>(Tp_, Tc_, Pp_, Pc_, L, tab, fT_step, fP, Lv, sT, sP, sft, srt, hT0v,
                                                  hT1v);
        } else {
            df_step<real, K, IFACE, SIMPLE>(Tp_, Tc_, Pp_, Pc_, L, tab, fT, fP, Lv, sT, sP, sft, srt);
        }
        if (RAD) {
            // radiation received over the step: sum h' (T' - Tbar) = qRd - hR Tbar
            last_rad = fma(-hR, sT, qRd);
            acc_rad += last_rad;
        }
        acc_sT += sT;
        acc_sP += sP;
        last_sT = sT;
        last_sP = sP;
        sample(Tp_, Pp_);
        if (ROOM) {
            publish(Tp_, Pp_, (int)((n_cur + 1) & 1));   // level n+1
            __syncthreads();
        }
        ++n_cur;
    };
    if (ROOM) {
        publish(Tb, Pb, (int)(n0 & 1));   // level n0, before the first step
        __syncthreads();
    }

    int s = 0;
    bool flipped = false;
    real bT = real(0), bP = real(0);
    int last_src = 0;
    while (s < n_steps) {
        const int cnt = min(kForcingBatch, n_steps - s);
        // ambient air for steps n0+s .. n0+s+15: lane i<16 computes face 0 at step i, lane 16+i face 1
        bT = real(0);
        bP = real(0);
        if (f_ambient) ambient_at(ff, d.noise, n0 + s + (lane % kForcingBatch), d.t0, d.dt, bT, bP);
        acc_sT = acc_sP = real(0);
        if (ROOM) acc_fT = acc_fP = real(0);
        if (RAD) acc_rad = real(0);
        int i = 0;
        for (; i + 1 < cnt; i += 2) {
            one_step(Ta, Tb, Pa, Pb, bT, bP, src_base + i);
            one_step(Tb, Ta, Pb, Pa, bT, bP, src_base + i + 1);
        }
        if (i < cnt) {   // odd final step: afterwards level n lives in the "a" arrays
            one_step(Ta, Tb, Pa, Pb, bT, bP, src_base + i);
            flipped = true;
        }
        {
            // the batch's air sums of the lane's face: room walls summed them per step; otherwise lanes
            // 0..cnt-1 (face 0) and 16..15+cnt (face 1) hold the batch's air, summed within each half-warp
            real sfT, sfP;
            if (ROOM) {
                sfT = acc_fT;
                sfP = acc_fP;
            } else {
                real xT = (lane % kForcingBatch) < cnt ? bT : real(0);
                real xP = (lane % kForcingBatch) < cnt ? bP : real(0);
#pragma unroll
                for (int o = kForcingBatch / 2; o >= 1; o >>= 1) {
                    xT += __shfl_xor_sync(FULL, xT, o);
                    xP += __shfl_xor_sync(FULL, xP, o);
                }
                sfT = __shfl_sync(FULL, xT, src_base);
                sfP = __shfl_sync(FULL, xP, src_base);
                last_src = src_base + cnt - 1;
            }
            // [eq:HAM_BC] summed over the batch: q = hT (T_inf - Tbar) + Lv hM (Pv_inf - Pvbar) + q_inf,
            // g = hM (Pv_inf - Pvbar) + g_inf
            const real rc = (real)cnt;
            const real hm = L.hMs * (sfP - acc_sP);
            const real acc_q = fma(L.hTs, sfT - acc_sT, fma(Lv, hm, rc * L.qs)) + (RAD ? acc_rad : real(0));
            const real acc_g = fma(rc, L.gs, hm);
            const real xq = acc_q * dt_r, xg = acc_g * dt_r;
            real t = kq + xq;
            kq_c += fabs(kq) >= fabs(xq) ? (kq - t) + xq : (xq - t) + kq;
            kq = t;
            t = kg + xg;
            kg_c += fabs(kg) >= fabs(xg) ? (kg - t) + xg : (xg - t) + kg;
            kg = t;
        }
        s += cnt;
        if (++kbatches == 16 || s >= n_steps) {
            if (my_face >= 0) {
                cum_q += (double)kq + (double)kq_c;
                cum_g += (double)kg + (double)kg_c;
            }
            kq = kq_c = kg = kg_c = real(0);
            kbatches = 0;
        }
    }

    // write back: level n into T[cur], level n-1 into T[1-cur]
    bool bad = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (k < nreal) {
            const real tn = flipped ? Ta[k] : Tb[k], pn = flipped ? Pa[k] : Pb[k];
            const real to = flipped ? Tb[k] : Ta[k], po = flipped ? Pb[k] : Pa[k];
            d.T[cur][base + k] = tn;
            d.P[cur][base + k] = pn;
            d.T[1 - cur][base + k] = to;
            d.P[1 - cur][base + k] = po;
            bad |= !(isfinite(tn) && isfinite(pn));
        }
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicExch(d.nonfinite, 1);
    // flux of the last step
    if (!ROOM) {
        last_fT = __shfl_sync(FULL, bT, last_src);
        last_fP = __shfl_sync(FULL, bP, last_src);
    }
    const real last_hm = L.hMs * (last_fP - last_sP);
    const real last_q = fma(L.hTs, last_fT - last_sT, fma(Lv, last_hm, L.qs)) + (RAD ? last_rad : real(0));
    const real last_g = last_hm + L.gs;
    if (my_face >= 0 && n_steps > 0) {
        d.cumul[(size_t)w * 4 + my_face * 2 + 0] = cum_q;
        d.cumul[(size_t)w * 4 + my_face * 2 + 1] = cum_g;
        d.flast[(size_t)w * 4 + my_face * 2 + 0] = (double)last_q;
        d.flast[(size_t)w * 4 + my_face * 2 + 1] = (double)last_g;
    }
}

// The simple-heat specialisation is built for FP32 only; FP64 runs those walls through the general code.
template <typename real>
constexpr bool kSimpleVariant = sizeof(real) == 4;

template <typename real>
__global__ void __launch_bounds__(PersistCfg<real>::warps * 32, 1)
    df1d_persistent_kernel(const DevCtx<real> d, int64_t n0, int32_t n_steps, int32_t sample_every, real *samples)
{
    // Each block owns a sequence of rounds of walls (balanced across blocks on the host by estimated
    // cost; a round holds walls of one code variant); warp i takes entry i of each round in turn,
    // without block-wide synchronisation.
    // dynamic shared memory per warp: layer table of the current wall, then (simple-heat walls with
    // interfaces inside lanes) the per-slot thermal face and reciprocal T denominator tables
    extern __shared__ __align__(16) unsigned char s_raw[];
    real *s_all = reinterpret_cast<real *>(s_raw);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int R = d.round_size;
    if (wib >= R) return;
    const int end = d.block_off[blockIdx.x + 1];
    for (int idx = d.block_off[blockIdx.x] + wib; idx < end; idx += R) {
        const int w = d.order[idx];
        if (w < 0) continue;
        const WallInfo wi = d.walls[w];
        real *tabw = s_all + (size_t)wib * kSmemRealsPerWarp;
        for (int i = lane; i < wi.n_layers * kLayerStride; i += 32)
            tabw[i] = d.layer_tab[(size_t)wi.layer_off * kLayerStride + i];
        __syncwarp();
        const real *tab = tabw;
        real *sft = tabw + kMaxLayers * kLayerStride + lane;
        real *srt = sft + kMaxK * 32;
        // variant: 0 = one layer per lane, simple heat; 1 = one layer per lane; 2 = interfaces in lanes;
        // 3 = interfaces in lanes, simple heat
        const bool simple = wi.simple && kSimpleVariant<real>;
        const int kind = wi.aligned ? (simple ? 0 : 1) : (simple ? 3 : 2);
        unsigned long long t_start = 0;
        if (d.trace != nullptr) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));
        switch (wi.K * 4 + kind) {
#define HYGRO_CASE(KK)                                                                                        \
    case 4 * KK:                                                                                              \
        run_wall<real, KK, false, kSimpleVariant<real>>(d, wi, w, tab, n0, n_steps, sample_every, samples, sft,   \
                                                        srt);                                                 \
        break;                                                                                                \
    case 4 * KK + 1:                                                                                          \
        run_wall<real, KK, false, false>(d, wi, w, tab, n0, n_steps, sample_every, samples, sft, srt);         \
        break;                                                                                                \
    case 4 * KK + 2:                                                                                          \
        run_wall<real, KK, true, false>(d, wi, w, tab, n0, n_steps, sample_every, samples, sft, srt);          \
        break;                                                                                                \
    case 4 * KK + 3:                                                                                          \
        run_wall<real, KK, true, kSimpleVariant<real>>(d, wi, w, tab, n0, n_steps, sample_every, samples, sft,    \
                                                       srt);                                                  \
        break;
            HYGRO_CASE(1) HYGRO_CASE(2) HYGRO_CASE(3) HYGRO_CASE(4) HYGRO_CASE(5) HYGRO_CASE(6)
            HYGRO_CASE(7) HYGRO_CASE(8) HYGRO_CASE(9) HYGRO_CASE(10) HYGRO_CASE(11) HYGRO_CASE(12)
            HYGRO_CASE(13) HYGRO_CASE(14) HYGRO_CASE(15) HYGRO_CASE(16)
#undef HYGRO_CASE
            default: break;
        }
        __syncwarp();
        if (d.trace != nullptr && lane == 0) {
            unsigned long long t_end;
            unsigned int smid;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
            asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
            unsigned long long *t = d.trace + (size_t)w * 4;
            t[0] = ((unsigned long long)smid << 32) | ((unsigned long long)blockIdx.x << 8) | (unsigned long long)wib;
            t[1] = t_start;
            t[2] = t_end;
            t[3] = (unsigned long long)n_steps;
        }
    }
}

}  // namespace hygro
