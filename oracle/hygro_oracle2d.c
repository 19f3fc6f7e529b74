/*
 * FP64 CPU oracle of the Dufort-Frankel update on 2D wall sections (uniform grid, dx = dy = h).
 * TEST INFRASTRUCTURE ONLY (see hygro_oracle.h). The 1D balance of [eq:DF_NL] extended to a
 * 5-point stencil: every node j owns the control area wx wy h^2 (wx, wy = 1/2 on the domain edges),
 * each face between two nodes has the length of its perpendicular half-cell weight times h, and a
 * Robin face on the domain edge ([eq:HAM_BC]) has length w_perp h:
 *   wx wy h^2 c (u^{n+1} - u^{n-1}) / (2 dt)
 *       = sum_faces w_perp h k_f (u_nb^n - ubar) / h + sum_edges w_perp h [h_s (u_inf - ubar) + src]
 * with ubar = (u^{n+1} + u^{n-1}) / 2, coefficients at level n, face values as in 1D (arithmetic
 * inside a material region, harmonic across regions), Pv first, then T with Pv^{n+1}.
 * Faces of the section: 0: x = 0, 1: x = Lx, 2: y = 0, 3: y = Ly.
 */
#include "hygro_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { L_KM0, L_A, L_CM0, L_B, L_KTT0, L_AT, L_CTT0, L_BT, L_CHI };

static double face_mean(double a, double b, int same) { return same ? 0.5 * (a + b) : 2.0 * a * b / (a + b); }

/* One DF step of grid g; new levels are written into Tp / Pp. */
static void grid_step(const orc2d_problem *p, int32_t g, double t, double *Tp, const double *Tc, double *Pp,
                      const double *Pc, double *buf)
{
    const int32_t nx = p->nx, ny = p->ny;
    const size_t n = (size_t)nx * ny;
    const double h = p->h, dt = p->dt, Lv = p->Lv;
    const uint8_t *reg = p->region + (size_t)g * n;
    const double *par = p->region_par + (size_t)g * p->n_regions * ORC_NLAYER_PAR;
    double *kM = buf, *cM = buf + n, *kTT = buf + 2 * n, *cTT = buf + 3 * n, *cTM = buf + 4 * n, *Pn = buf + 5 * n;
    for (size_t c = 0; c < n; ++c) {
        const double *q = par + (size_t)reg[c] * ORC_NLAYER_PAR;
        double r = Pc[c] / p->Psat;
        kM[c] = q[L_KM0] * (1.0 + q[L_A] * r);
        cM[c] = q[L_CM0] * (1.0 + q[L_B] * r);
        kTT[c] = q[L_KTT0] * (1.0 + q[L_AT] * r);
        cTT[c] = q[L_CTT0] * (1.0 + q[L_BT] * r);
        cTM[c] = q[L_CHI] * cM[c];
    }
    /* air of the ambient faces at t^n */
    double Tinf[4], Pinf[4], hT[4], hM[4], qs[4], gs[4];
    for (int f = 0; f < 4; ++f) {
        const double *b = p->bc_par + ((size_t)g * 4 + f) * ORC_NBC_PAR;
        hT[f] = hM[f] = qs[f] = gs[f] = Tinf[f] = Pinf[f] = 0.0;
        if (p->bc_kind[g * 4 + f] != ORC_BC_AMBIENT) continue;
        hT[f] = b[0];
        hM[f] = b[1];
        qs[f] = b[2];
        gs[f] = b[3];
        double T = b[4], P = b[6];
        const double period_P = b[12] > 0.0 ? b[12] : b[8];   /* Pv sinusoid period (<= 0: the T period) */
        if (b[8] > 0.0) T += b[5] * sin(6.283185307179586476925286766559 * t / b[8] + b[9]);
        if (period_P > 0.0) P += b[7] * sin(6.283185307179586476925286766559 * t / period_P + b[10]);
        if (p->noise[f] != NULL && p->noise_len[f] > 0 && b[11] > 0.0) {
            const float *tab = p->noise[f] + (size_t)g * p->noise_len[f] * 2;
            double x = t / b[11];
            int32_t len = p->noise_len[f];
            double nT, nP;
            if (x <= 0.0) {
                nT = tab[0];
                nP = tab[1];
            } else if (x >= (double)(len - 1)) {
                nT = tab[(size_t)(len - 1) * 2];
                nP = tab[(size_t)(len - 1) * 2 + 1];
            } else {
                double i = floor(x), fr = x - i;
                size_t k = (size_t)i;
                nT = (1.0 - fr) * tab[k * 2] + fr * tab[(k + 1) * 2];
                nP = (1.0 - fr) * tab[k * 2 + 1] + fr * tab[(k + 1) * 2 + 1];
            }
            T += nT;
            P += nP;
        }
        Tinf[f] = T;
        Pinf[f] = P;
    }
    /* neighbours: di, dj, face length uses the perpendicular weight */
    static const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
    for (int pass = 0; pass < 2; ++pass) {
        for (int32_t j = 0; j < ny; ++j)
            for (int32_t i = 0; i < nx; ++i) {
                const size_t c = (size_t)j * nx + i;
                const double wx = (i == 0 || i == nx - 1) ? 0.5 : 1.0;
                const double wy = (j == 0 || j == ny - 1) ? 0.5 : 1.0;
                double S = 0, nb = 0, H = 0, src = 0, cross = 0;
                const double Pbar = pass == 1 ? 0.5 * (Pn[c] + Pp[c]) : 0.0;
                for (int d = 0; d < 4; ++d) {
                    const int32_t ii = i + di[d], jj = j + dj[d];
                    const double len = d < 2 ? wy : wx;
                    if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) continue;
                    const size_t e = (size_t)jj * nx + ii;
                    const int same = reg[c] == reg[e];
                    if (pass == 0) {
                        const double G = len * face_mean(kM[c], kM[e], same) / h;
                        S += G;
                        nb += G * Pc[e];
                    } else {
                        const double G = len * face_mean(kTT[c], kTT[e], same) / h;
                        const double GM = len * Lv * face_mean(kM[c], kM[e], same) / h;
                        S += G;
                        nb += G * Tc[e];
                        cross += GM * (Pc[e] - Pbar);
                    }
                }
                /* Robin edges: face f lies at i = 0 (0), i = nx-1 (1), j = 0 (2), j = ny-1 (3) */
                const int on[4] = {i == 0, i == nx - 1, j == 0, j == ny - 1};
                for (int f = 0; f < 4; ++f) {
                    if (!on[f]) continue;
                    const double len = f < 2 ? wy : wx;
                    if (pass == 0) {
                        H += len * hM[f];
                        src += len * (hM[f] * Pinf[f] + gs[f]);
                    } else {
                        H += len * hT[f];
                        src += len * (hT[f] * Tinf[f] + Lv * hM[f] * (Pinf[f] - Pbar) + qs[f]);
                    }
                }
                if (pass == 0) {
                    const double A = wx * wy * h * cM[c] / (2.0 * dt);
                    Pn[c] = ((A - 0.5 * S - 0.5 * H) * Pp[c] + nb + src) / (A + 0.5 * S + 0.5 * H);
                } else {
                    const double B = wx * wy * h * cTT[c] / (2.0 * dt);
                    const double C = wx * wy * h * cTM[c] / (2.0 * dt);
                    const double Tn = ((B - 0.5 * S - 0.5 * H) * Tp[c] + nb + cross + src - C * (Pn[c] - Pp[c])) /
                                      (B + 0.5 * S + 0.5 * H);
                    Tp[c] = Tn;
                }
            }
    }
    for (size_t c = 0; c < n; ++c) Pp[c] = Pn[c];
}

int orc2d_run(const orc2d_problem *p, orc2d_state *s, int64_t n_steps, int32_t n_threads)
{
    if (p == NULL || s == NULL || n_steps < 0 || p->nx < 2 || p->ny < 2 || p->n_grids < 0 || !(p->h > 0))
        return -1;
    const size_t n = (size_t)p->nx * p->ny;
    if (n_threads <= 0) n_threads = 1;
    int rc = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads)
#endif
    {
        double *buf = (double *)malloc(sizeof(double) * n * 6);
        if (buf == NULL) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            rc = -2;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (int32_t g = 0; g < p->n_grids; ++g) {
                double *Tp = s->T_prev + (size_t)g * n, *Tc = s->T_cur + (size_t)g * n;
                double *Pp = s->P_prev + (size_t)g * n, *Pc = s->P_cur + (size_t)g * n;
                for (int64_t it = 0; it < n_steps; ++it) {
                    const double t = p->t0 + (double)(s->step + it) * p->dt;
                    grid_step(p, g, t, Tp, Tc, Pp, Pc, buf);
                    double *x = Tp;
                    Tp = Tc;
                    Tc = x;
                    x = Pp;
                    Pp = Pc;
                    Pc = x;
                }
                if (n_steps % 2 == 1) {
                    /* the newest level sits in the *_prev array: swap contents back into place */
                    double *a = s->T_prev + (size_t)g * n, *b = s->T_cur + (size_t)g * n;
                    double *c2 = s->P_prev + (size_t)g * n, *d = s->P_cur + (size_t)g * n;
                    for (size_t k = 0; k < n; ++k) {
                        double x = a[k];
                        a[k] = b[k];
                        b[k] = x;
                        x = c2[k];
                        c2[k] = d[k];
                        d[k] = x;
                    }
                }
            }
            free(buf);
        }
    }
    if (rc == 0) s->step += n_steps;
    return rc;
}
