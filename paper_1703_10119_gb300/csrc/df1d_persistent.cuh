// Persistent DF kernel for batches of 1D walls: one warp owns one wall and
// advances it through all the steps of a hygro_run call with both time
// levels held in registers.
//
// Lane layout of a wall of N nodes: K = ceil(N / 32) nodes per lane,
// Wl = ceil(N / K) lanes in use, m = Wl K - N "short" lanes. Lanes 0..m-1
// hold K-1 consecutive nodes (their slot K-1 is a frozen dummy), lanes
// m..Wl-1 hold K; so node 0 sits in lane 0 slot 0 and node N-1 always in
// lane Wl-1 slot K-1, and only those two slots carry surface terms. Lanes
// >= Wl hold nothing (all-zero state with zero faces, which stays zero).
// Neighbour values across lanes move with warp shuffles (4 values each way
// per step); there is no shared-memory traffic and no block barrier in the
// time loop. Per step and node the work is the coefficient evaluation at
// level n (Sec. 2 coefficients, explicit at t^n as in Sec. 3.1), the face
// means, the Pv update and then the T update using Pv^{n+1} (Appendix A
// order), written in increment form:
//   du = [sum_f F_f (u_nb^n - u^{n-1}) + surface terms] / (C + sum_f F_f / 2 + H / 2)
// which is the DF balance of [eq:DF_NL] solved for u^{n+1} - u^{n-1}.
// Surface fluxes are summed in the working precision over batches of 16
// steps and then added to FP64 running sums.
#pragma once

#include "df1d_common.cuh"

namespace hygro {

template <typename real>
struct LaneCtx {
    LayerC<real> c0;          // constants of the layer of slot 0
    real clkMa, clkMb;        // kM half-values constants of the last real slot's layer
    real clkTa, clkTb;
    real w0, w1;              // half-cell weights of slot 0 / slot K-1 (1/2 at a wall surface)
    real hM0, hT0, q0, g0;    // face-0 exchange (lane 0 only, else 0)
    real hM1, hT1, q1, g1;    // face-1 exchange (lane Wl-1 only, else 0)
    uint32_t imask;           // bit k: slot k is the first node of a layer >= 1 (its left face is an interface)
    uint32_t wimask;          // OR of imask over the warp (warp-uniform)
    int l0;                   // layer of slot 0
    bool short_lane;          // lane holds K-1 nodes
    bool has_left, has_right; // a face exists between this lane and its neighbour lane
    bool iface_left0;         // the lane-boundary face on the left is an interface
    bool iface_right;         // the lane-boundary face on the right is an interface
    bool any_lb_iface;        // some lane-boundary face of the warp is an interface (warp-uniform)
};

// One DF step of the lane's K slots: level n+1 is written into Tp / Pp.
// fT, fP: ambient air of this lane's surface face (if any) at level n.
// fq, fg: receive this lane's surface heat / moisture flux of the step.
template <typename real, int K>
__device__ __forceinline__ void df_step(real (&Tp)[K], const real (&Tc)[K], real (&Pp)[K], const real (&Pc)[K],
                                        const LaneCtx<real> &L, const real *tab, const real fT, const real fP,
                                        const real Lv, real &fq, real &fg)
{
    constexpr unsigned FULL = 0xffffffffu;
    const real half = real(0.5);

    // values of the lane's first and last real nodes, exchanged with the neighbour lanes
    const real lastT = (K >= 2 && L.short_lane) ? Tc[K >= 2 ? K - 2 : 0] : Tc[K - 1];
    const real lastP = (K >= 2 && L.short_lane) ? Pc[K >= 2 ? K - 2 : 0] : Pc[K - 1];
    const real khM_first = fma(L.c0.kMb, Pc[0], L.c0.kMa);
    const real khT_first = fma(L.c0.kTb, Pc[0], L.c0.kTa);
    const real khM_last = fma(L.clkMb, lastP, L.clkMa);
    const real khT_last = fma(L.clkTb, lastP, L.clkTa);

    const real lT = __shfl_up_sync(FULL, lastT, 1);
    const real lP = __shfl_up_sync(FULL, lastP, 1);
    const real lkM = __shfl_up_sync(FULL, khM_last, 1);
    const real lkT = __shfl_up_sync(FULL, khT_last, 1);
    const real rT = __shfl_down_sync(FULL, Tc[0], 1);
    const real rP = __shfl_down_sync(FULL, Pc[0], 1);
    const real rkM = __shfl_down_sync(FULL, khM_first, 1);
    const real rkT = __shfl_down_sync(FULL, khT_first, 1);

    // lane-boundary faces (zero at the wall ends and on unused lanes)
    real FMl0 = lkM + khM_first, FTl0 = lkT + khT_first;
    real FMb = khM_last + rkM, FTb = khT_last + rkT;
    if (L.any_lb_iface) {
        if (L.iface_left0) {
            FMl0 = face_harmonic(lkM, khM_first);
            FTl0 = face_harmonic(lkT, khT_first);
        }
        if (L.iface_right) {
            FMb = face_harmonic(khM_last, rkM);
            FTb = face_harmonic(khT_last, rkT);
        }
    }
    FMl0 = L.has_left ? FMl0 : real(0);
    FTl0 = L.has_left ? FTl0 : real(0);
    FMb = L.has_right ? FMb : real(0);
    FTb = L.has_right ? FTb : real(0);

    LayerC<real> c = L.c0;
    int lcur = L.l0;
    real FMl = FMl0, FTl = FTl0;   // left face of the current slot
    real Tl = lT, Pl = lP;         // left neighbour at level n
    real khM = khM_first, khT = khT_first;
    fq = real(0);
    fg = real(0);

#pragma unroll
    for (int k = 0; k < K; ++k) {
        // constants and half-values of the next slot, and the right face of this one
        LayerC<real> cn = c;
        real FMr, FTr, Tr, Pr, khMn = real(0), khTn = real(0);
        if (k + 1 < K) {
            if ((L.wimask >> (k + 1)) & 1u) {
                if ((L.imask >> (k + 1)) & 1u) cn = load_layer(tab, lcur + 1);
            }
            khMn = fma(cn.kMb, Pc[k + 1], cn.kMa);
            khTn = fma(cn.kTb, Pc[k + 1], cn.kTa);
            FMr = khM + khMn;
            FTr = khT + khTn;
            if ((L.wimask >> (k + 1)) & 1u) {
                if ((L.imask >> (k + 1)) & 1u) {
                    FMr = face_harmonic(khM, khMn);
                    FTr = face_harmonic(khT, khTn);
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
            FTr = FTb;
            Tr = rT;
            Pr = rP;
            if (K >= 2) {           // short lanes: freeze the dummy slot K-1
                FMl = L.short_lane ? real(0) : FMl;
                FTl = L.short_lane ? real(0) : FTl;
                FMr = L.short_lane ? real(0) : FMr;
                FTr = L.short_lane ? real(0) : FTr;
            }
        }

        // node coefficients at level n (storage terms), half-cell weight at surfaces
        const real Pk = Pc[k];
        real A = fma(c.Ab, Pk, c.Aa);
        real B = fma(c.Bb, Pk, c.Ba);
        if (k == 0) {
            A *= L.w0;
            B *= L.w0;
        }
        if (k == K - 1) {
            A *= L.w1;
            B *= L.w1;
        }

        // vapour pressure
        const real pp = Pp[k];
        real numP = fma(FMl, Pl - pp, FMr * (Pr - pp));
        real denP = fma(half, FMl + FMr, A);
        if (k == 0) {
            numP = fma(L.hM0, fP - pp, numP + L.g0);
            denP = fma(half, L.hM0, denP);
        }
        if (k == K - 1) {
            numP = fma(L.hM1, fP - pp, numP + L.g1);
            denP = fma(half, L.hM1, denP);
        }
        const real dP = fast_div(numP, denP);
        const real Pbar = fma(half, dP, pp);

        // temperature, with the kTM cross flux (kTM_f = Lv kM_f) and the cTM storage term
        const real tp = Tp[k];
        real numT = fma(FTl, Tl - tp, FTr * (Tr - tp));
        numT = fma(Lv, fma(FMl, Pl - Pbar, FMr * (Pr - Pbar)), numT);
        numT = fma(-c.chi * A, dP, numT);
        real denT = fma(half, FTl + FTr, B);
        real hm0 = real(0), hm1 = real(0);   // hM (Pv_inf - Pbar) at the surfaces
        if (k == 0) {
            hm0 = L.hM0 * (fP - Pbar);
            numT = fma(L.hT0, fT - tp, fma(Lv, hm0, numT + L.q0));
            denT = fma(half, L.hT0, denT);
        }
        if (k == K - 1) {
            hm1 = L.hM1 * (fP - Pbar);
            numT = fma(L.hT1, fT - tp, fma(Lv, hm1, numT + L.q1));
            denT = fma(half, L.hT1, denT);
        }
        const real dT = fast_div(numT, denT);
        Pp[k] = pp + dP;
        Tp[k] = tp + dT;

        if (k == 0 || k == K - 1) {
            // surface fluxes into the wall with the time-averaged surface values
            const real Tbar = fma(half, dT, tp);
            if (k == 0) {
                fq += fma(L.hT0, fT - Tbar, fma(Lv, hm0, L.q0));
                fg += hm0 + L.g0;
            }
            if (k == K - 1) {
                fq += fma(L.hT1, fT - Tbar, fma(Lv, hm1, L.q1));
                fg += hm1 + L.g1;
            }
        }

        // advance to the next slot
        Tl = Tc[k];
        Pl = Pk;
        FMl = FMr;
        FTl = FTr;
        khM = khMn;
        khT = khTn;
        if (k + 1 < K) {
            if ((L.wimask >> (k + 1)) & 1u) {
                if ((L.imask >> (k + 1)) & 1u) ++lcur;
            }
        }
        c = cn;
    }
}

// Everything one warp does for one wall over n_steps steps.
template <typename real, int K>
__device__ __noinline__ void run_wall(const DevCtx<real> &d, const WallInfo &wi, int w, const real *tab, int64_t n0,
                                      int32_t n_steps, int32_t sample_every, real *samples)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int Wl = wi.Wl, m = wi.m;

    LaneCtx<real> L;
    L.short_lane = (K >= 2) && lane < m;
    const int first = L.short_lane ? lane * (K - 1) : lane * K - m;   // wall-local node of slot 0
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
    const real Lv = (real)d.Lv;
    const real Tref = d.Tref[w], Pref = d.Pref[w];

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
    if (my_face >= 0) {
        cum_q = d.cumul[(size_t)w * 4 + my_face * 2 + 0];
        cum_g = d.cumul[(size_t)w * 4 + my_face * 2 + 1];
    }
    real last_q = real(0), last_g = real(0);
    int scount = sample_every;
    int64_t sidx = 0;
    const int W = d.W;
    // surface values written by a sample: lane 0 -> face 0 (slot 0), lane Wl-1 -> face 1 (slot K-1)
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

    int s = 0;
    bool flipped = false;
    while (s < n_steps) {
        const int cnt = min(kForcingBatch, n_steps - s);
        // ambient air for steps n0+s .. n0+s+15: lane i<16 computes face 0 at step i, lane 16+i face 1
        real bT = real(0), bP = real(0);
        if (f_ambient) ambient_at(ff, d.noise, n0 + s + (lane % kForcingBatch), d.t0, d.dt, bT, bP);
        real acc_q = real(0), acc_g = real(0);
        int i = 0;
        for (; i + 1 < cnt; i += 2) {
            real fq, fg;
            real fT = __shfl_sync(FULL, bT, src_base + i);
            real fP = __shfl_sync(FULL, bP, src_base + i);
            df_step<real, K>(Ta, Tb, Pa, Pb, L, tab, fT, fP, Lv, fq, fg);
            acc_q += fq;
            acc_g += fg;
            sample(Ta, Pa);
            fT = __shfl_sync(FULL, bT, src_base + i + 1);
            fP = __shfl_sync(FULL, bP, src_base + i + 1);
            df_step<real, K>(Tb, Ta, Pb, Pa, L, tab, fT, fP, Lv, fq, fg);
            acc_q += fq;
            acc_g += fg;
            sample(Tb, Pb);
            last_q = fq;
            last_g = fg;
        }
        if (i < cnt) {   // odd final step: afterwards level n lives in the "a" arrays
            real fq, fg;
            const real fT = __shfl_sync(FULL, bT, src_base + i);
            const real fP = __shfl_sync(FULL, bP, src_base + i);
            df_step<real, K>(Ta, Tb, Pa, Pb, L, tab, fT, fP, Lv, fq, fg);
            acc_q += fq;
            acc_g += fg;
            sample(Ta, Pa);
            last_q = fq;
            last_g = fg;
            flipped = true;
        }
        cum_q += (double)acc_q * d.dt;
        cum_g += (double)acc_g * d.dt;
        s += cnt;
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
    if (my_face >= 0 && n_steps > 0) {
        d.cumul[(size_t)w * 4 + my_face * 2 + 0] = cum_q;
        d.cumul[(size_t)w * 4 + my_face * 2 + 1] = cum_g;
        d.flast[(size_t)w * 4 + my_face * 2 + 0] = (double)last_q;
        d.flast[(size_t)w * 4 + my_face * 2 + 1] = (double)last_g;
    }
}

template <typename real>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    df1d_persistent_kernel(const DevCtx<real> d, int64_t n0, int32_t n_steps, int32_t sample_every, real *samples,
                           int32_t *queue_counter)
{
    __shared__ real s_tab[kWarpsPerBlock][kMaxLayers * kLayerStride];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(queue_counter, 1);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= d.W) break;
        const int w = d.order[idx];
        const WallInfo wi = d.walls[w];
        for (int i = lane; i < wi.n_layers * kLayerStride; i += 32)
            s_tab[wib][i] = d.layer_tab[(size_t)wi.layer_off * kLayerStride + i];
        __syncwarp();
        const real *tab = s_tab[wib];
        switch (wi.K) {
#define HYGRO_CASE(KK) \
    case KK: run_wall<real, KK>(d, wi, w, tab, n0, n_steps, sample_every, samples); break;
            HYGRO_CASE(1) HYGRO_CASE(2) HYGRO_CASE(3) HYGRO_CASE(4) HYGRO_CASE(5) HYGRO_CASE(6)
            HYGRO_CASE(7) HYGRO_CASE(8) HYGRO_CASE(9) HYGRO_CASE(10) HYGRO_CASE(11) HYGRO_CASE(12)
            HYGRO_CASE(13) HYGRO_CASE(14) HYGRO_CASE(15) HYGRO_CASE(16)
#undef HYGRO_CASE
            default: break;
        }
        __syncwarp();
    }
}

}  // namespace hygro
