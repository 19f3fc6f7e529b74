// Plain DF kernel: one thread per node, one launch per step, both levels in
// global memory. The same scheme as the persistent kernel (coefficients at
// level n, face means, Pv then T, half-cell Robin surfaces; paper Sec. 3.1
// [eq:DF_NL] and Appendix A), in its most direct GPU form.
#include "df1d_common.cuh"
#include "material_table1.cuh"

namespace hygro {

// Coefficients of one node of a wall with Table-1 layers: half-values kh = k / (2 dx) of kM, kTT and kTM,
// and the storage terms dx c / (2 dt) of cM, cTT and cTM (before the surface half weight). Affine layers
// give the values of their affine laws (kTM = nu Lv kM).
template <typename real>
struct NodeCoef {
    real khM, khT, khX, A, B, C;
    bool law;
};

template <typename real>
__device__ __forceinline__ NodeCoef<real> node_coef(const DevCtx<real> &d, const WallInfo &wi, int w, const real *tab,
                                                    int l, real Tdev, real Pdev)
{
    NodeCoef<real> k;
    const int law = d.layer_law[wi.layer_off + l];
    k.law = law != HYGRO_LAW_AFFINE;
    if (!k.law) {
        const LayerC<real> c = load_layer(tab, l);
        k.khM = fma(c.kMb, Pdev, c.kMa);
        k.khT = fma(c.kTb, Pdev, c.kTa);
        k.khX = (real)(d.Lv * wi.nu) * k.khM;
        k.A = fma(c.Ab, Pdev, c.Aa);
        k.B = fma(c.Bb, Pdev, c.Ba);
        k.C = c.chi * k.A;
        return k;
    }
    const LawCoef<real> m = table1_law<real>(law, d.Tref[w] + Tdev, d.Pref[w] + Pdev, (real)d.Lv);
    const real inv2dx = (real)(0.5 / wi.dx), s = (real)(wi.dx / (2.0 * d.dt));
    k.khM = m.kM * inv2dx;
    k.khT = m.kTT * inv2dx;
    k.khX = m.kTM * inv2dx;
    k.A = m.cM * s;
    k.B = m.cTT * s;
    k.C = m.cTM * s;
    return k;
}

// One node of a wall with Table-1 layers: the balance of [eq:DF_NL] with every coefficient of level n from
// node_coef; faces arithmetic inside a layer and harmonic across layers (the kTM face of two affine layers
// is nu Lv times their kM face, as in the affine walls).
template <typename real>
__device__ __forceinline__ void law_node(const DevCtx<real> &d, const WallInfo &wi, int w, int g, int j, int l,
                                         const real *tab, const real *Tc, const real *Pc, real &pp, real &tp,
                                         real hM, real hT, real qi, real gi, real fT, real fP, real &dP, real &dT)
{
    const real half = real(0.5);
    const int N = wi.N;
    const NodeCoef<real> k = node_coef(d, wi, w, tab, l, Tc[g], Pc[g]);
    real FMl = 0, FTl = 0, FXl = 0, FMr = 0, FTr = 0, FXr = 0, Tl = 0, Pl = 0, Tr = 0, Pr = 0;
    auto face = [&](const NodeCoef<real> &o, bool same, real &FM, real &FT, real &FX) {
        FM = same ? k.khM + o.khM : face_harmonic(k.khM, o.khM);
        FT = same ? k.khT + o.khT : face_harmonic(k.khT, o.khT);
        if (!k.law && !o.law)
            FX = (real)(d.Lv * wi.nu) * FM;
        else
            FX = same ? k.khX + o.khX : face_harmonic(k.khX, o.khX);
    };
    if (j > 0) {
        const int ll = d.node_layer[g - 1];
        Tl = Tc[g - 1];
        Pl = Pc[g - 1];
        face(node_coef(d, wi, w, tab, ll, Tl, Pl), ll == l, FMl, FTl, FXl);
    }
    if (j < N - 1) {
        const int lr = d.node_layer[g + 1];
        Tr = Tc[g + 1];
        Pr = Pc[g + 1];
        face(node_coef(d, wi, w, tab, lr, Tr, Pr), lr == l, FMr, FTr, FXr);
    }
    const real wgt = (j == 0 || j == N - 1) ? half : real(1);
    const real A = k.A * wgt, B = k.B * wgt, C = k.C * wgt;
    const real numP = fma(hM, fP - pp, fma(FMl, Pl - pp, FMr * (Pr - pp)) + gi);
    dP = fast_div(numP, fma(half, FMl + FMr + hM, A));
    const real Pbar = fma(half, dP, pp);
    const real Lv = (real)d.Lv;
    real numT = fma(FTl, Tl - tp, FTr * (Tr - tp));
    numT = fma(FXl, Pl - Pbar, fma(FXr, Pr - Pbar, numT));
    numT = fma(-C, dP, numT);
    numT = fma(hT, fT - tp, fma(Lv, hM * (fP - Pbar), numT + qi));
    dT = fast_div(numT, fma(half, FTl + FTr + hT, B));
}

template <typename real>
__global__ void __launch_bounds__(256)
    df1d_plain_kernel(const DevCtx<real> d, int64_t n, int32_t sample_idx, real *samples)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= d.total_nodes) return;
    const int w = d.node_wall[g];
    const WallInfo wi = d.walls[w];
    const int j = g - wi.node_off;
    const int N = wi.N;
    const real *Tc = d.T[d.cur];
    const real *Pc = d.P[d.cur];
    real *Tn = d.T[1 - d.cur];   // holds level n-1 on entry, level n+1 on exit
    real *Pn = d.P[1 - d.cur];
    const real *tab = d.layer_tab + (size_t)wi.layer_off * kLayerStride;
    const int l = d.node_layer[g];
    const LayerC<real> c = load_layer(tab, l);
    const real half = real(0.5);
    if (wi.has_law) {
        const int face = j == 0 ? 0 : (j == N - 1 ? 1 : -1);
        real hM = 0, hT = 0, qi = 0, gi = 0, fT = 0, fP = 0;
        if (face >= 0) {
            const FaceInfo &fi = d.faces[(size_t)w * 2 + face];
            if (fi.kind == HYGRO_BC_AMBIENT) {
                hM = (real)fi.hM;
                hT = (real)fi.hT;
                qi = (real)fi.q_inf;
                gi = (real)fi.g_inf;
                ambient_at(fi, d.noise, n, d.t0, d.dt, fT, fP);
            }
        }
        real pp = Pn[g], tp = Tn[g], dP, dT;
        law_node(d, wi, w, g, j, l, tab, Tc, Pc, pp, tp, hM, hT, qi, gi, fT, fP, dP, dT);
        const real Pnew = pp + dP, Tnew = tp + dT;
        Pn[g] = Pnew;
        Tn[g] = Tnew;
        if (!(isfinite(Pnew) && isfinite(Tnew))) atomicExch(d.nonfinite, 1);
        if (face >= 0) {
            const real Lv = (real)d.Lv;
            const real Pbar = fma(half, dP, pp), Tbar = fma(half, dT, tp);
            const real hm = hM * (fP - Pbar);
            const real q = fma(hT, fT - Tbar, fma(Lv, hm, qi));
            const real gflux = hm + gi;
            double *cu = d.cumul + (size_t)w * 4 + face * 2;
            double *fl = d.flast + (size_t)w * 4 + face * 2;
            cu[0] += d.dt * (double)q;
            cu[1] += d.dt * (double)gflux;
            fl[0] = (double)q;
            fl[1] = (double)gflux;
            if (samples != nullptr && sample_idx >= 0) {
                real *o = samples + ((size_t)sample_idx * d.W + w) * 4 + face * 2;
                o[0] = d.Tref[w] + Tnew;
                o[1] = d.Pref[w] + Pnew;
            }
        }
        return;
    }

    const real Pk = Pc[g];
    const real khM = fma(c.kMb, Pk, c.kMa), khT = fma(c.kTb, Pk, c.kTa);
    real FMl = 0, FTl = 0, FMr = 0, FTr = 0, Tl = 0, Pl = 0, Tr = 0, Pr = 0;
    if (j > 0) {
        const int ll = d.node_layer[g - 1];
        const LayerC<real> cl = (ll == l) ? c : load_layer(tab, ll);
        Tl = Tc[g - 1];
        Pl = Pc[g - 1];
        const real a = fma(cl.kMb, Pl, cl.kMa), b = fma(cl.kTb, Pl, cl.kTa);
        FMl = ll == l ? a + khM : face_harmonic(a, khM);
        FTl = ll == l ? b + khT : face_harmonic(b, khT);
    }
    if (j < N - 1) {
        const int lr = d.node_layer[g + 1];
        const LayerC<real> cr = (lr == l) ? c : load_layer(tab, lr);
        Tr = Tc[g + 1];
        Pr = Pc[g + 1];
        const real a = fma(cr.kMb, Pr, cr.kMa), b = fma(cr.kTb, Pr, cr.kTa);
        FMr = lr == l ? khM + a : face_harmonic(khM, a);
        FTr = lr == l ? khT + b : face_harmonic(khT, b);
    }
    const real wgt = (j == 0 || j == N - 1) ? half : real(1);
    const real A = fma(c.Ab, Pk, c.Aa) * wgt;
    const real B = fma(c.Bb, Pk, c.Ba) * wgt;

    const int face = j == 0 ? 0 : (j == N - 1 ? 1 : -1);
    real hM = 0, hT = 0, qi = 0, gi = 0, fT = 0, fP = 0;
    if (face >= 0) {
        const FaceInfo &fi = d.faces[(size_t)w * 2 + face];
        if (fi.kind == HYGRO_BC_AMBIENT) {
            hM = (real)fi.hM;
            hT = (real)fi.hT;
            qi = (real)fi.q_inf;
            gi = (real)fi.g_inf;
            ambient_at(fi, d.noise, n, d.t0, d.dt, fT, fP);
        }
    }

    // vapour pressure first
    const real pp = Pn[g];
    const real numP = fma(hM, fP - pp, fma(FMl, Pl - pp, FMr * (Pr - pp)) + gi);
    const real denP = fma(half, FMl + FMr + hM, A);
    const real dP = fast_div(numP, denP);
    const real Pbar = fma(half, dP, pp);
    // then temperature with Pv^{n+1}
    const real tp = Tn[g];
    const real Lv = (real)d.Lv;
    const real hm = hM * (fP - Pbar);
    real numT = fma(FTl, Tl - tp, FTr * (Tr - tp));
    // latent heat of the moisture flux inside the wall (kTM = nu Lv kM); the surface keeps Lv hM
    numT = fma((real)(d.Lv * wi.nu), fma(FMl, Pl - Pbar, FMr * (Pr - Pbar)), numT);
    numT = fma(-c.chi * A, dP, numT);
    numT = fma(hT, fT - tp, fma(Lv, hm, numT + qi));
    const real denT = fma(half, FTl + FTr + hT, B);
    const real dT = fast_div(numT, denT);
    const real Pnew = pp + dP, Tnew = tp + dT;
    Pn[g] = Pnew;
    Tn[g] = Tnew;
    if (!(isfinite(Pnew) && isfinite(Tnew))) atomicExch(d.nonfinite, 1);

    if (face >= 0) {
        const real Tbar = fma(half, dT, tp);
        const real q = fma(hT, fT - Tbar, fma(Lv, hm, qi));
        const real gflux = hm + gi;
        double *cu = d.cumul + (size_t)w * 4 + face * 2;
        double *fl = d.flast + (size_t)w * 4 + face * 2;
        cu[0] += d.dt * (double)q;
        cu[1] += d.dt * (double)gflux;
        fl[0] = (double)q;
        fl[1] = (double)gflux;
        if (samples != nullptr && sample_idx >= 0) {
            real *o = samples + ((size_t)sample_idx * d.W + w) * 4 + face * 2;
            o[0] = d.Tref[w] + Tnew;
            o[1] = d.Pref[w] + Pnew;
        }
    }
}

// Discrete balance of one step n -> n+1 per wall and field (the identity S = B + D of the DF scheme):
// storage S = sum_j w dx (c (u^{n+1} - u^{n-1}) [+ cTM (Pv^{n+1} - Pv^{n-1})]) / (2 dt), boundary B = the surface
// fluxes into the wall with the time-averaged surface values ([eq:HAM_BC]), DF defect D = sum over interior
// faces of (k_f / dx) ((u_{j+1}^n - ubar_{j+1}) + (u_j^n - ubar_j)) (plus the kTM cross terms for T), and M the
// sum of the magnitudes of all terms. Levels: Tp, Pp = n-1, d.T[cur], d.P[cur] = n, Tn, Pn = n+1.
// bal[w][field: 0 T, 1 Pv][4] = S, B, D, M, accumulated in FP64 (zeroed by the caller).
template <typename real>
__global__ void __launch_bounds__(256)
    df1d_balance_kernel(const DevCtx<real> d, const real *Tp, const real *Pp, const real *Tn, const real *Pn,
                        int64_t n, double *bal)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= d.total_nodes) return;
    const int w = d.node_wall[g];
    const WallInfo wi = d.walls[w];
    const int j = g - wi.node_off;
    const int N = wi.N;
    const real *Tc = d.T[d.cur], *Pc = d.P[d.cur];
    const real *tab = d.layer_tab + (size_t)wi.layer_off * kLayerStride;
    const int l = d.node_layer[g];
    const LayerC<real> c = load_layer(tab, l);
    const real half = real(0.5), Lv = (real)d.Lv, LvN = (real)(d.Lv * wi.nu);
    double *bT = bal + (size_t)w * 8, *bP = bT + 4;
    const real wgt = (j == 0 || j == N - 1) ? half : real(1);
    const real A = fma(c.Ab, Pc[g], c.Aa) * wgt, B = fma(c.Bb, Pc[g], c.Ba) * wgt;
    const real dP = Pn[g] - Pp[g], dT = Tn[g] - Tp[g];
    const double sP = (double)(A * dP), sT = (double)fma(B, dT, c.chi * A * dP);
    atomicAdd(bP + 0, sP);
    atomicAdd(bP + 3, fabs(sP));
    atomicAdd(bT + 0, sT);
    atomicAdd(bT + 3, fabs(sT));
    if (j < N - 1) {
        // the face (j, j+1), counted once, by node j
        const int lr = d.node_layer[g + 1];
        const LayerC<real> cr = (lr == l) ? c : load_layer(tab, lr);
        const real a = fma(c.kMb, Pc[g], c.kMa), b = fma(cr.kMb, Pc[g + 1], cr.kMa);
        const real at = fma(c.kTb, Pc[g], c.kTa), bt = fma(cr.kTb, Pc[g + 1], cr.kTa);
        const real FM = lr == l ? a + b : face_harmonic(a, b);
        const real FT = lr == l ? at + bt : face_harmonic(at, bt);
        const real Pb0 = half * (Pn[g] + Pp[g]), Pb1 = half * (Pn[g + 1] + Pp[g + 1]);
        const real Tb0 = half * (Tn[g] + Tp[g]), Tb1 = half * (Tn[g + 1] + Tp[g + 1]);
        const real eP = (Pc[g + 1] - Pb1) + (Pc[g] - Pb0), eT = (Tc[g + 1] - Tb1) + (Tc[g] - Tb0);
        atomicAdd(bP + 2, (double)(FM * eP));
        atomicAdd(bT + 2, (double)fma(FT, eT, LvN * FM * eP));
        atomicAdd(bP + 3, (double)(FM * (fabs(Pc[g + 1] - Pb0) + fabs(Pc[g] - Pb1))));
        atomicAdd(bT + 3, (double)(FT * (fabs(Tc[g + 1] - Tb0) + fabs(Tc[g] - Tb1)) +
                                   LvN * FM * (fabs(Pc[g + 1] - Pb0) + fabs(Pc[g] - Pb1))));
    }
    const int face = j == 0 ? 0 : (j == N - 1 ? 1 : -1);
    if (face >= 0) {
        const FaceInfo &fi = d.faces[(size_t)w * 2 + face];
        if (fi.kind == HYGRO_BC_AMBIENT) {
            real fT, fP;
            ambient_at(fi, d.noise, n, d.t0, d.dt, fT, fP);
            const real Tbar = half * (Tn[g] + Tp[g]), Pbar = half * (Pn[g] + Pp[g]);
            const real hm = (real)fi.hM * (fP - Pbar);
            const real gflux = hm + (real)fi.g_inf;
            const real q = fma((real)fi.hT, fT - Tbar, fma(Lv, hm, (real)fi.q_inf));
            atomicAdd(bP + 1, (double)gflux);
            atomicAdd(bP + 3, fabs((double)gflux));
            atomicAdd(bT + 1, (double)q);
            atomicAdd(bT + 3, fabs((double)q));
        }
    }
}

template <typename real>
static cudaError_t launch_balance(const DevCtx<real> &d, const real *Tp, const real *Pp, const real *Tn,
                                  const real *Pn, int64_t n, double *bal, cudaStream_t s)
{
    const int grid = (d.total_nodes + 255) / 256;
    df1d_balance_kernel<real><<<grid, 256, 0, s>>>(d, Tp, Pp, Tn, Pn, n, bal);
    return cudaGetLastError();
}

cudaError_t launch_balance_f32(const DevCtx<float> &d, const float *Tp, const float *Pp, const float *Tn,
                               const float *Pn, int64_t n, double *bal, cudaStream_t s)
{
    return launch_balance(d, Tp, Pp, Tn, Pn, n, bal, s);
}

cudaError_t launch_balance_f64(const DevCtx<double> &d, const double *Tp, const double *Pp, const double *Tn,
                               const double *Pn, int64_t n, double *bal, cudaStream_t s)
{
    return launch_balance(d, Tp, Pp, Tn, Pn, n, bal, s);
}

// First step by explicit Euler substeps (hygro_start_euler): one block per wall, its levels in shared
// memory. Level 1 from level 0 by m substeps of tau = dt / m, the coefficients re-evaluated at every
// substep, Pv first and T with the substep's Pv change in the cTM storage term, the ambient air at each
// substep's time; m = ceil(dt / tau_max) with tau_max the explicit stability bound of the wall at level 0,
// min over nodes of C / (sum of the face conductances + h) for both fields (C = w dx c). In the kh form
// of the layer table: C_Pv = 2 dt w (Aa + Ab P'), C_T = 2 dt w (Ba + Bb P'), C_TM = chi C_Pv. The flux sums
// receive tau times the surface fluxes of every substep. Writes level 1 into the level n-1 buffer.
// m_out[w] receives the substep count (0 if it exceeded max_sub: the wall is then left unchanged).
template <typename real>
__global__ void __launch_bounds__(128) df1d_euler_start_kernel(const DevCtx<real> d, int64_t max_sub, int64_t *m_out)
{
    extern __shared__ __align__(16) unsigned char es_raw[];
    __shared__ double s_red[4];
    const int w = blockIdx.x, tid = threadIdx.x;
    const WallInfo wi = d.walls[w];
    const int N = wi.N;
    real *T = reinterpret_cast<real *>(es_raw), *P = T + N, *Tn = P + N, *Pn = Tn + N;
    const real *tab = d.layer_tab + (size_t)wi.layer_off * kLayerStride;
    const int8_t *lay = d.node_layer + wi.node_off;
    const real *T0 = d.T[d.cur] + wi.node_off, *P0 = d.P[d.cur] + wi.node_off;
    for (int j = tid; j < N; j += blockDim.x) {
        T[j] = T0[j];
        P[j] = P0[j];
    }
    const FaceInfo &f0 = d.faces[(size_t)w * 2], &f1 = d.faces[(size_t)w * 2 + 1];
    const bool a0 = f0.kind == HYGRO_BC_AMBIENT, a1 = f1.kind == HYGRO_BC_AMBIENT;
    const real hM0 = a0 ? (real)f0.hM : real(0), hT0 = a0 ? (real)f0.hT : real(0);
    const real hM1 = a1 ? (real)f1.hM : real(0), hT1 = a1 ? (real)f1.hT : real(0);
    const real g0 = a0 ? (real)f0.g_inf : real(0), q0 = a0 ? (real)f0.q_inf : real(0);
    const real g1 = a1 ? (real)f1.g_inf : real(0), q1 = a1 ? (real)f1.q_inf : real(0);
    const real Lv = (real)d.Lv, LvN = (real)(d.Lv * wi.nu), two_dt = (real)(2.0 * d.dt);
    if (tid == 0) s_red[0] = d.dt;
    __syncthreads();
    // face conductances of node j (kh sums, harmonic across layers); left and right
    auto faces = [&](int j, real &FMl, real &FTl, real &FMr, real &FTr) {
        const LayerC<real> c = load_layer(tab, lay[j]);
        const real khM = fma(c.kMb, P[j], c.kMa), khT = fma(c.kTb, P[j], c.kTa);
        FMl = FTl = FMr = FTr = real(0);
        if (j > 0) {
            const LayerC<real> cl = load_layer(tab, lay[j - 1]);
            const real a = fma(cl.kMb, P[j - 1], cl.kMa), b = fma(cl.kTb, P[j - 1], cl.kTa);
            FMl = lay[j - 1] == lay[j] ? a + khM : face_harmonic(a, khM);
            FTl = lay[j - 1] == lay[j] ? b + khT : face_harmonic(b, khT);
        }
        if (j < N - 1) {
            const LayerC<real> cr = load_layer(tab, lay[j + 1]);
            const real a = fma(cr.kMb, P[j + 1], cr.kMa), b = fma(cr.kTb, P[j + 1], cr.kTa);
            FMr = lay[j + 1] == lay[j] ? khM + a : face_harmonic(khM, a);
            FTr = lay[j + 1] == lay[j] ? khT + b : face_harmonic(khT, b);
        }
    };
    // the stability bound at level 0
    double tmin = d.dt;
    for (int j = tid; j < N; j += blockDim.x) {
        const LayerC<real> c = load_layer(tab, lay[j]);
        const real wj = (j == 0 || j == N - 1) ? real(0.5) : real(1);
        real FMl, FTl, FMr, FTr;
        faces(j, FMl, FTl, FMr, FTr);
        const real GM = FMl + FMr + (j == 0 ? hM0 : real(0)) + (j == N - 1 ? hM1 : real(0));
        const real GT = FTl + FTr + (j == 0 ? hT0 : real(0)) + (j == N - 1 ? hT1 : real(0));
        const double CP = (double)(two_dt * wj * fma(c.Ab, P[j], c.Aa)), CT = (double)(two_dt * wj * fma(c.Bb, P[j], c.Ba));
        if (GM > real(0)) tmin = fmin(tmin, CP / (double)GM);
        if (GT > real(0)) tmin = fmin(tmin, CT / (double)GT);
    }
    for (int o = 16; o > 0; o >>= 1) tmin = fmin(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
    if ((tid & 31) == 0) atomicMin(reinterpret_cast<unsigned long long *>(&s_red[0]), __double_as_longlong(tmin));
    __syncthreads();
    const double tau_max = s_red[0];   // positive doubles order like their bit patterns
    int64_t m = (int64_t)ceil(d.dt / tau_max);
    if (m < 1) m = 1;
    if (m > max_sub) {
        if (tid == 0) m_out[w] = 0;
        return;
    }
    const double tau = d.dt / (double)m;
    const real tau_r = (real)tau;
    double cq0 = 0.0, cg0 = 0.0, cq1 = 0.0, cg1 = 0.0, lq0 = 0.0, lg0 = 0.0, lq1 = 0.0, lg1 = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        real aT0 = real(0), aP0 = real(0), aT1 = real(0), aP1 = real(0);
        for (int j = tid; j < N; j += blockDim.x) {
            const LayerC<real> c = load_layer(tab, lay[j]);
            const real wj = (j == 0 || j == N - 1) ? real(0.5) : real(1);
            real FMl, FTl, FMr, FTr;
            faces(j, FMl, FTl, FMr, FTr);
            real rP = real(0), rT = real(0);
            if (j > 0) {
                rP = fma(FMl, P[j - 1] - P[j], rP);
                rT = fma(FTl, T[j - 1] - T[j], fma(LvN * FMl, P[j - 1] - P[j], rT));
            }
            if (j < N - 1) {
                rP = fma(FMr, P[j + 1] - P[j], rP);
                rT = fma(FTr, T[j + 1] - T[j], fma(LvN * FMr, P[j + 1] - P[j], rT));
            }
            if (j == 0 && a0) {
                double x, y;
                ambient_at(f0, d.noise, i, d.t0, tau, x, y);
                aT0 = (real)x;
                aP0 = (real)y;
                const real hm = hM0 * (aP0 - P[j]);
                const real gq = hm + g0, qq = fma(hT0, aT0 - T[j], fma(Lv, hm, q0));
                rP += gq;
                rT += qq;
                cq0 += tau * (double)qq;
                cg0 += tau * (double)gq;
                lq0 = (double)qq;
                lg0 = (double)gq;
            }
            if (j == N - 1 && a1) {
                double x, y;
                ambient_at(f1, d.noise, i, d.t0, tau, x, y);
                aT1 = (real)x;
                aP1 = (real)y;
                const real hm = hM1 * (aP1 - P[j]);
                const real gq = hm + g1, qq = fma(hT1, aT1 - T[j], fma(Lv, hm, q1));
                rP += gq;
                rT += qq;
                cq1 += tau * (double)qq;
                cg1 += tau * (double)gq;
                lq1 = (double)qq;
                lg1 = (double)gq;
            }
            const real CP = two_dt * wj * fma(c.Ab, P[j], c.Aa), CT = two_dt * wj * fma(c.Bb, P[j], c.Ba);
            const real dP = tau_r * rP / CP;
            Pn[j] = P[j] + dP;
            Tn[j] = T[j] + tau_r * rT / CT - c.chi * CP / CT * dP;
        }
        __syncthreads();
        for (int j = tid; j < N; j += blockDim.x) {
            T[j] = Tn[j];
            P[j] = Pn[j];
        }
        __syncthreads();
    }
    real *T1 = d.T[1 - d.cur] + wi.node_off, *P1 = d.P[1 - d.cur] + wi.node_off;
    bool bad = false;
    for (int j = tid; j < N; j += blockDim.x) {
        T1[j] = T[j];
        P1[j] = P[j];
        bad |= !(isfinite(T[j]) && isfinite(P[j]));
    }
    if (bad) atomicExch(d.nonfinite, 1);
    if (tid == 0) {
        d.cumul[(size_t)w * 4 + 0] += cq0;
        d.cumul[(size_t)w * 4 + 1] += cg0;
        d.flast[(size_t)w * 4 + 0] = lq0;
        d.flast[(size_t)w * 4 + 1] = lg0;
        m_out[w] = m;
    }
    if (tid == (N - 1) % (int)blockDim.x) {
        d.cumul[(size_t)w * 4 + 2] += cq1;
        d.cumul[(size_t)w * 4 + 3] += cg1;
        d.flast[(size_t)w * 4 + 2] = lq1;
        d.flast[(size_t)w * 4 + 3] = lg1;
    }
}

template <typename real>
static cudaError_t launch_euler(const DevCtx<real> &d, int Nmax, int64_t max_sub, int64_t *m_out, cudaStream_t s)
{
    const size_t smem = (size_t)4 * Nmax * sizeof(real);
    cudaError_t e = cudaFuncSetAttribute(df1d_euler_start_kernel<real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    df1d_euler_start_kernel<real><<<d.W, 128, smem, s>>>(d, max_sub, m_out);
    return cudaGetLastError();
}

cudaError_t launch_euler_start_f32(const DevCtx<float> &d, int Nmax, int64_t max_sub, int64_t *m_out, cudaStream_t s)
{
    return launch_euler(d, Nmax, max_sub, m_out, s);
}

cudaError_t launch_euler_start_f64(const DevCtx<double> &d, int Nmax, int64_t max_sub, int64_t *m_out, cudaStream_t s)
{
    return launch_euler(d, Nmax, max_sub, m_out, s);
}

cudaError_t launch_plain_step_f32(const DevCtx<float> &d, int64_t n, int32_t sample_idx, float *samples,
                                  cudaStream_t s)
{
    const int grid = (d.total_nodes + 255) / 256;
    df1d_plain_kernel<float><<<grid, 256, 0, s>>>(d, n, sample_idx, samples);
    return cudaGetLastError();
}

cudaError_t launch_plain_step_f64(const DevCtx<double> &d, int64_t n, int32_t sample_idx, double *samples,
                                  cudaStream_t s)
{
    const int grid = (d.total_nodes + 255) / 256;
    df1d_plain_kernel<double><<<grid, 256, 0, s>>>(d, n, sample_idx, samples);
    return cudaGetLastError();
}

}  // namespace hygro
