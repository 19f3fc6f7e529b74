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
