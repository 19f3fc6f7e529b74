// Plain DF kernel: one thread per node, one launch per step, both levels in
// global memory. The same scheme as the persistent kernel (coefficients at
// level n, face means, Pv then T, half-cell Robin surfaces; paper Sec. 3.1
// [eq:DF_NL] and Appendix A), in its most direct GPU form.
#include "df1d_common.cuh"

namespace hygro {

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
    numT = fma(Lv, fma(FMl, Pl - Pbar, FMr * (Pr - Pbar)), numT);
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
    const real half = real(0.5), Lv = (real)d.Lv;
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
        atomicAdd(bT + 2, (double)fma(FT, eT, Lv * FM * eP));
        atomicAdd(bP + 3, (double)(FM * (fabs(Pc[g + 1] - Pb0) + fabs(Pc[g] - Pb1))));
        atomicAdd(bT + 3, (double)(FT * (fabs(Tc[g + 1] - Tb0) + fabs(Tc[g] - Tb1)) +
                                   Lv * FM * (fabs(Pc[g + 1] - Pb0) + fabs(Pc[g] - Pb1))));
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
