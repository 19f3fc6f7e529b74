/*
 * The paper's comparison schemes on the CPU (Sec. 4 and Sec. 5.2): Euler implicit with fixed-point
 * sub-iterations, and Euler explicit within its stability bound. TEST INFRASTRUCTURE ONLY: they are
 * timed next to the DF oracle on the same host cores (the paper's DF / implicit cost ratio) and serve as
 * independent solvers of the same semi-discrete problem.
 *
 * Both use the DF oracle's spatial operator: half-cell finite volumes (weight 1/2 at the surface nodes),
 * face values arithmetic inside a layer and harmonic across layers, the Robin exchanges of [eq:HAM_BC]
 * (fluxes positive into the wall), the coefficients of Sec. 2 (affine laws or the Table-1 material), the
 * room air node of Sec. 5.1 with the latent terms and the vapour part of the air's heat capacity.
 *
 * Euler implicit (the problem statement of Sec. 5.2, [eq:wbse_tn_imp]): the step n -> n+1 solves
 *   w dx cM (P+ - P) / dt = faces kM (P+_nb - P+) / dx + hM (Pinf+ - P+) + ginf,
 *   w dx [cTT (T+ - T) + cTM (P+ - P)] / dt = faces [kTT (T+_nb - T+) + kTM (P+_nb - P+)] / dx
 *                                             + hT (Tinf+ - T+) + Lv hM (Pinf+ - P+) + qinf,
 * with the air at t^{n+1} and the room air of level n+1, and the room air balances with the walls' surface
 * values of level n+1. Because the coefficients depend on the unknowns and walls and rooms are coupled,
 * it is solved by the fixed-point iteration of Alg. 1: from the iterate (u^k, ua^k) (k = 0: level n), the
 * walls' linear systems (tridiagonal, Pv then T) with the coefficients at u^k and the room air ua^k give
 * u^{k+1}; the rooms' balances with the surface values of u^{k+1} give ua^{k+1}; the iteration stops when
 * the largest relative change of any value is below eta.
 *
 * Euler explicit: a step of dt in m substeps tau = dt / m, m the smallest count with tau within the
 * explicit stability bound of every node and room at the step's start (per node: w dx c divided by the sum
 * of its face conductances / dx and surface h, for cM and for cTT; per room: the capacity over its total
 * exchange conductance), times refine >= 1. It is the dimensional, per-node form of the bounds
 * [eq:cfl_heat_Eq], [eq:cfl_moisture_Eq]. Coefficients, air and room air are taken at every substep's start.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "oracle_internal.h"

typedef struct {
    double *kM, *cM, *kTT, *cTT, *kTM, *cTM, *kMf, *kTTf, *kTMf;
    double *a, *b, *c, *d, *x;   /* tridiagonal system */
    double *Tk, *Pk;             /* the iterate's levels */
} work;

static int work_alloc(work *w, int32_t N)
{
    double *buf = (double *)malloc(sizeof(double) * (size_t)N * 16);
    if (buf == NULL) return -2;
    double **f[] = {&w->kM, &w->cM, &w->kTT, &w->cTT, &w->kTM, &w->cTM, &w->kMf, &w->kTTf, &w->kTMf,
                    &w->a, &w->b, &w->c, &w->d, &w->x, &w->Tk, &w->Pk};
    for (int i = 0; i < 16; ++i) *f[i] = buf + (size_t)i * N;
    return 0;
}

/* Thomas algorithm: a[j] x[j-1] + b[j] x[j] + c[j] x[j+1] = d[j], j = 0..N-1 (b, d overwritten). */
static void thomas(int32_t N, const double *a, double *b, const double *c, double *d, double *x)
{
    for (int32_t j = 1; j < N; ++j) {
        const double m = a[j] / b[j - 1];
        b[j] -= m * c[j - 1];
        d[j] -= m * d[j - 1];
    }
    x[N - 1] = d[N - 1] / b[N - 1];
    for (int32_t j = N - 2; j >= 0; --j) x[j] = (d[j] - c[j] * x[j + 1]) / b[j];
}

/* One backward-Euler solve of one wall from level n (Tn, Pn) with the coefficients of the iterate
 * (w->Tk, w->Pk) and the boundary air bc: the new levels in Tout, Pout. */
static void implicit_wall(const orc_problem *p, const wall_view *v, const face_bc bc[2], const double *Tn,
                          const double *Pn, work *w, double *Tout, double *Pout)
{
    const int32_t N = v->N;
    const double dx = v->dx, dt = p->dt, Lv = p->Lv;
    coefficients(p, v, w->Tk, w->Pk, w->kM, w->cM, w->kTT, w->cTT, w->kTM, w->cTM, w->kMf, w->kTTf, w->kTMf);
    /* vapour pressure */
    for (int32_t j = 0; j < N; ++j) {
        const double wj = (j == 0 || j == N - 1) ? 0.5 : 1.0;
        const double m = wj * dx * w->cM[j] / dt;
        w->a[j] = j > 0 ? -w->kMf[j - 1] / dx : 0.0;
        w->c[j] = j < N - 1 ? -w->kMf[j] / dx : 0.0;
        w->b[j] = m - w->a[j] - w->c[j];
        w->d[j] = m * Pn[j];
        if (j == 0) {
            w->b[j] += bc[0].hM;
            w->d[j] += bc[0].hM * bc[0].P_inf + bc[0].g_inf;
        }
        if (j == N - 1) {
            w->b[j] += bc[1].hM;
            w->d[j] += bc[1].hM * bc[1].P_inf + bc[1].g_inf;
        }
    }
    thomas(N, w->a, w->b, w->c, w->d, Pout);
    /* temperature with the new Pv in the cross flux and the cTM storage */
    for (int32_t j = 0; j < N; ++j) {
        const double wj = (j == 0 || j == N - 1) ? 0.5 : 1.0;
        const double m = wj * dx * w->cTT[j] / dt;
        w->a[j] = j > 0 ? -w->kTTf[j - 1] / dx : 0.0;
        w->c[j] = j < N - 1 ? -w->kTTf[j] / dx : 0.0;
        w->b[j] = m - w->a[j] - w->c[j];
        double rhs = m * Tn[j] - wj * dx * w->cTM[j] * (Pout[j] - Pn[j]) / dt;
        if (j > 0) rhs += w->kTMf[j - 1] / dx * (Pout[j - 1] - Pout[j]);
        if (j < N - 1) rhs += w->kTMf[j] / dx * (Pout[j + 1] - Pout[j]);
        for (int f = 0; f < 2; ++f)
            if ((f == 0 && j == 0) || (f == 1 && j == N - 1)) {
                w->b[j] += bc[f].hT + bc[f].hR;
                rhs += bc[f].hT * bc[f].T_inf + Lv * bc[f].hM * (bc[f].P_inf - Pout[j]) + bc[f].q_inf + bc[f].qR;
            }
        w->d[j] = rhs;
    }
    thomas(N, w->a, w->b, w->c, w->d, Tout);
}

/* Surface fluxes into the wall at the values (T, P) of its surface nodes. */
static void surface_flux(const orc_problem *p, const face_bc bc[2], const double *T, const double *P, int32_t N,
                         double fl[2][2])
{
    for (int f = 0; f < 2; ++f) {
        const int32_t j = f == 0 ? 0 : N - 1;
        const double g = bc[f].hM * (bc[f].P_inf - P[j]) + bc[f].g_inf;
        fl[f][0] = bc[f].hT * (bc[f].T_inf - T[j]) + p->Lv * bc[f].hM * (bc[f].P_inf - P[j]) + bc[f].q_inf +
                   bc[f].qR - bc[f].hR * T[j];
        fl[f][1] = g;
    }
}

/* Surface values [n_walls][2 faces][T, Pv] of the levels T, P. */
static void surface_values(const orc_problem *p, const int64_t *node_off, const double *T, const double *P,
                           double *surf)
{
    for (int32_t w = 0; w < p->n_walls; ++w) {
        surf[w * 4 + 0] = T[node_off[w]];
        surf[w * 4 + 1] = P[node_off[w]];
        surf[w * 4 + 2] = T[node_off[w + 1] - 1];
        surf[w * 4 + 3] = P[node_off[w + 1] - 1];
    }
}

/* Room sums over the room-side faces: A hT, A hM, A hT Ts, A hM Ps with the walls' surface values in T, P. */
static void room_sums(const orc_problem *p, const int64_t *node_off, const double *T, const double *P,
                      double *sum /* [R][4] */)
{
    const int32_t R = p->n_rooms;
    for (int32_t i = 0; i < 4 * R; ++i) sum[i] = 0.0;
    for (int32_t w = 0; w < p->n_walls; ++w)
        for (int f = 0; f < 2; ++f) {
            if (p->bc_kind[w * 2 + f] != ORC_BC_ROOM) continue;
            const int32_t r = p->bc_room[w * 2 + f];
            const double *b = p->bc_par + ((size_t)w * 2 + f) * ORC_NBC_PAR;
            const int64_t j = f == 0 ? node_off[w] : node_off[w + 1] - 1;
            const double A = p->wall_area[w];
            sum[r * 4 + 0] += A * b[B_HT];
            sum[r * 4 + 1] += A * b[B_HM];
            sum[r * 4 + 2] += A * b[B_HT] * T[j];
            sum[r * 4 + 3] += A * b[B_HM] * P[j];
        }
}

/* Backward-Euler room air of level n+1 (Ta, Pa of level n in Tn_a, Pn_a) at time t = t^{n+1}, with the
 * capacity at the iterate's vapour pressure Pk_a and the room sums of the walls' new surface values. */
static void implicit_room(const orc_problem *p, int32_t r, double t, double Tn_a, double Pn_a, double Pk_a,
                          const double *sum, const double *lk, double *Ta, double *Pa)
{
    const double *q = p->room_par + (size_t)r * ORC_NROOM_PAR;
    const double dt = p->dt, Lv = p->Lv, Pref = q[R_PVREF];
    const double rhoV = q[R_RHOA] * q[R_VOL], gv = rhoV * q[R_ACH] / 3600.0;
    double T_out, P_out, g;
    room_sources(p, r, t, &T_out, &P_out, &g);
    const double w_out = P_out / Pref;
    const double CP = rhoV / Pref;
    const double G = lk[r * 3 + 0], GT = lk[r * 3 + 1], Gw = lk[r * 3 + 2];   /* linked rooms of the iterate */
    const double P1 = (CP / dt * Pn_a + g + gv * w_out + sum[r * 4 + 3] + Gw) /
                      (CP / dt + gv / Pref + sum[r * 4 + 1] + G / Pref);
    const double CT = rhoV * (q[R_CPA] + q[R_CPV] * Pk_a / Pref);
    const double rhs = CT / dt * Tn_a + q[R_QGAIN] + Lv * g + gv * q[R_CPA] * T_out + Lv * gv * (w_out - P1 / Pref) +
                       sum[r * 4 + 2] + Lv * (sum[r * 4 + 3] - sum[r * 4 + 1] * P1) + q[R_CPA] * GT +
                       Lv * (Gw - G * P1 / Pref);
    *Ta = rhs / (CT / dt + gv * q[R_CPA] + sum[r * 4 + 0] + G * q[R_CPA]);
    *Pa = P1;
}

int orc_euler_implicit_run(const orc_problem *p, orc_state *s, int64_t n_steps, double eta, int32_t max_iter,
                           int32_t norm, int64_t *iterations, int32_t n_threads)
{
    if (p == NULL || s == NULL || n_steps < 0 || !(eta > 0.0) || max_iter < 1 || norm < 0 || norm > 1) return -1;
    if (p->n_rooms > 0 && (s->room == NULL || p->room_par == NULL || p->wall_area == NULL)) return -1;
    const int32_t W = p->n_walls, R = p->n_rooms;
    int64_t *node_off = (int64_t *)calloc((size_t)W + 1, sizeof(int64_t));
    int64_t *layer_off = (int64_t *)calloc((size_t)W + 1, sizeof(int64_t));
    if (!node_off || !layer_off) {
        free(node_off);
        free(layer_off);
        return -2;
    }
    int32_t Nmax = 3;
    for (int32_t w = 0; w < W; ++w) {
        if (p->n_nodes[w] < 3) {
            free(node_off);
            free(layer_off);
            return -1;
        }
        node_off[w + 1] = node_off[w] + p->n_nodes[w];
        layer_off[w + 1] = layer_off[w] + p->n_layers[w];
        if (p->n_nodes[w] > Nmax) Nmax = p->n_nodes[w];
    }
    const int64_t tot = node_off[W];
    double *Tk = (double *)malloc(sizeof(double) * (size_t)tot * 4);
    double *ra = (double *)malloc(sizeof(double) * ((size_t)R * 8 + 1));
    if (!Tk || !ra) {
        free(node_off);
        free(layer_off);
        free(Tk);
        free(ra);
        return -2;
    }
    double *Pk = Tk + tot, *Tk1 = Tk + 2 * tot, *Pk1 = Tk + 3 * tot;
    double *rk = ra, *rsum = ra + 4 * R;   /* iterate's room air (Ta, Pa per room) and room sums */
    double *air = (double *)calloc((size_t)R * 4 + 1, sizeof(double));   /* rk in the room_state layout */
    double *surf = (double *)calloc((size_t)W * 4 + 1, sizeof(double));
    double *qrad = (double *)calloc((size_t)W * 4 + 1, sizeof(double));
    double *lk = (double *)calloc((size_t)R * 3 + 1, sizeof(double));
    if (air == NULL || surf == NULL || qrad == NULL || lk == NULL) {
        free(node_off);
        free(layer_off);
        free(Tk);
        free(ra);
        free(air);
        free(surf);
        free(qrad);
        free(lk);
        return -2;
    }
    if (n_threads <= 0) n_threads = 1;
    int rc = 0;
    for (int64_t it = 0; it < n_steps && rc == 0; ++it) {
        const double t1 = p->t0 + (double)(s->step + 1) * p->dt;
        memcpy(Tk, s->T_cur, sizeof(double) * (size_t)tot);
        memcpy(Pk, s->P_cur, sizeof(double) * (size_t)tot);
        for (int32_t r = 0; r < R; ++r) {
            rk[r * 2 + 0] = s->room[r * 4 + 1];
            rk[r * 2 + 1] = s->room[r * 4 + 3];
        }
        int32_t k = 0;
        double change = 0.0;
        do {
            /* walls from level n with the coefficients of the iterate, the room air of the iterate and the
             * radiative exchange of the iterate's surface temperatures */
            for (int32_t r = 0; r < R; ++r) {
                air[r * 4 + 1] = rk[r * 2 + 0];
                air[r * 4 + 3] = rk[r * 2 + 1];
            }
            if (R > 0) {
                surface_values(p, node_off, Tk, Pk, surf);
                room_radiation(p, surf, qrad);
            }
            int err = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads)
#endif
            {
                work wk;
                if (work_alloc(&wk, Nmax) != 0) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                    err = -2;
                } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
                    for (int32_t w = 0; w < W; ++w) {
                        const wall_view v = view_of(p, layer_off, w);
                        face_bc bc[2] = {face_of(p, w, 0, t1, air), face_of(p, w, 1, t1, air)};
                        for (int f = 0; f < 2 && R > 0; ++f) {
                            bc[f].hR = qrad[(w * 2 + f) * 2 + 0];
                            bc[f].qR = qrad[(w * 2 + f) * 2 + 1];
                        }
                        const int64_t o = node_off[w];
                        memcpy(wk.Tk, Tk + o, sizeof(double) * (size_t)v.N);
                        memcpy(wk.Pk, Pk + o, sizeof(double) * (size_t)v.N);
                        implicit_wall(p, &v, bc, s->T_cur + o, s->P_cur + o, &wk, Tk1 + o, Pk1 + o);
                    }
                    free(wk.kM);
                }
            }
            if (err != 0) {
                rc = err;
                break;
            }
            /* rooms with the walls' new surface values; the change of the iterate as the largest relative
             * change (norm 0) or the Euclidean norm of all relative changes (norm 1) */
            change = 0.0;
            double sq = 0.0;
            if (R > 0) {
                room_sums(p, node_off, Tk1, Pk1, rsum);
                room_links(p, air, lk);   /* the linked rooms' air of the iterate (air holds rk) */
                for (int32_t r = 0; r < R; ++r) {
                    double Ta, Pa;
                    implicit_room(p, r, t1, s->room[r * 4 + 1], s->room[r * 4 + 3], rk[r * 2 + 1], rsum, lk, &Ta, &Pa);
                    const double eT = fabs(Ta - rk[r * 2 + 0]) / fabs(Ta), eP = fabs(Pa - rk[r * 2 + 1]) / fabs(Pa);
                    change = fmax(change, fmax(eT, eP));
                    sq += eT * eT + eP * eP;
                    rk[r * 2 + 0] = Ta;
                    rk[r * 2 + 1] = Pa;
                }
            }
            for (int64_t i = 0; i < tot; ++i) {
                const double eT = fabs(Tk1[i] - Tk[i]) / fabs(Tk1[i]), eP = fabs(Pk1[i] - Pk[i]) / fabs(Pk1[i]);
                change = fmax(change, fmax(eT, eP));
                sq += eT * eT + eP * eP;
                Tk[i] = Tk1[i];
                Pk[i] = Pk1[i];
            }
            if (norm == 1) change = sqrt(sq);
            ++k;
        } while (rc == 0 && !(change < eta) && k < max_iter);
        if (rc != 0) break;
        if (!(change < eta)) rc = -3;
        if (iterations) *iterations += k;
        /* fluxes of level n+1 into the running sums */
        for (int32_t r = 0; r < R; ++r) {
            air[r * 4 + 1] = rk[r * 2 + 0];
            air[r * 4 + 3] = rk[r * 2 + 1];
        }
        if (R > 0) {
            surface_values(p, node_off, Tk, Pk, surf);
            room_radiation(p, surf, qrad);
        }
        for (int32_t w = 0; w < W; ++w) {
            const int64_t o = node_off[w];
            face_bc bc[2] = {face_of(p, w, 0, t1, air), face_of(p, w, 1, t1, air)};
            for (int f = 0; f < 2 && R > 0; ++f) {
                bc[f].hR = qrad[(w * 2 + f) * 2 + 0];
                bc[f].qR = qrad[(w * 2 + f) * 2 + 1];
            }
            double fl[2][2];
            surface_flux(p, bc, Tk + o, Pk + o, p->n_nodes[w], fl);
            for (int f = 0; f < 2; ++f)
                for (int c = 0; c < 2; ++c) s->cumul[w * 4 + f * 2 + c] += p->dt * fl[f][c];
        }
        memcpy(s->T_prev, s->T_cur, sizeof(double) * (size_t)tot);
        memcpy(s->P_prev, s->P_cur, sizeof(double) * (size_t)tot);
        memcpy(s->T_cur, Tk, sizeof(double) * (size_t)tot);
        memcpy(s->P_cur, Pk, sizeof(double) * (size_t)tot);
        for (int32_t r = 0; r < R; ++r) {
            s->room[r * 4 + 0] = s->room[r * 4 + 1];
            s->room[r * 4 + 1] = rk[r * 2 + 0];
            s->room[r * 4 + 2] = s->room[r * 4 + 3];
            s->room[r * 4 + 3] = rk[r * 2 + 1];
        }
        s->step += 1;
    }
    free(node_off);
    free(layer_off);
    free(Tk);
    free(ra);
    free(air);
    free(surf);
    free(qrad);
    free(lk);
    return rc;
}

/* The explicit stability bound (seconds) of one wall at (T, P) with boundary bc: the smallest over nodes
 * and both fields of w dx c / (sum of face conductances / dx + h). */
static double wall_tau(const orc_problem *p, const wall_view *v, const face_bc bc[2], const double *T,
                       const double *P, work *w)
{
    const int32_t N = v->N;
    const double dx = v->dx;
    coefficients(p, v, T, P, w->kM, w->cM, w->kTT, w->cTT, w->kTM, w->cTM, w->kMf, w->kTTf, w->kTMf);
    double tmax = INFINITY;
    for (int32_t j = 0; j < N; ++j) {
        const double wj = (j == 0 || j == N - 1) ? 0.5 : 1.0;
        double GM = 0.0, GT = 0.0;
        if (j > 0) {
            GM += w->kMf[j - 1] / dx;
            GT += w->kTTf[j - 1] / dx;
        }
        if (j < N - 1) {
            GM += w->kMf[j] / dx;
            GT += w->kTTf[j] / dx;
        }
        if (j == 0) {
            GM += bc[0].hM;
            GT += bc[0].hT;
        }
        if (j == N - 1) {
            GM += bc[1].hM;
            GT += bc[1].hT;
        }
        if (GM > 0.0) tmax = fmin(tmax, wj * dx * w->cM[j] / GM);
        if (GT > 0.0) tmax = fmin(tmax, wj * dx * w->cTT[j] / GT);
    }
    return tmax;
}

/* One forward-Euler substep tau of one wall: (T, P) -> (Tout, Pout), fluxes at the substep's start. */
static void explicit_wall(const orc_problem *p, const wall_view *v, const face_bc bc[2], const double *T,
                          const double *P, double tau, work *w, double *Tout, double *Pout, double fl[2][2])
{
    const int32_t N = v->N;
    const double dx = v->dx, Lv = p->Lv;
    coefficients(p, v, T, P, w->kM, w->cM, w->kTT, w->cTT, w->kTM, w->cTM, w->kMf, w->kTTf, w->kTMf);
    for (int32_t j = 0; j < N; ++j) {
        const double wj = (j == 0 || j == N - 1) ? 0.5 : 1.0;
        double g = 0.0;
        if (j > 0) g += w->kMf[j - 1] / dx * (P[j - 1] - P[j]);
        if (j < N - 1) g += w->kMf[j] / dx * (P[j + 1] - P[j]);
        if (j == 0) g += bc[0].hM * (bc[0].P_inf - P[j]) + bc[0].g_inf;
        if (j == N - 1) g += bc[1].hM * (bc[1].P_inf - P[j]) + bc[1].g_inf;
        Pout[j] = P[j] + tau * g / (wj * dx * w->cM[j]);
    }
    for (int32_t j = 0; j < N; ++j) {
        const double wj = (j == 0 || j == N - 1) ? 0.5 : 1.0;
        double q = 0.0;
        if (j > 0) q += (w->kTTf[j - 1] * (T[j - 1] - T[j]) + w->kTMf[j - 1] * (P[j - 1] - P[j])) / dx;
        if (j < N - 1) q += (w->kTTf[j] * (T[j + 1] - T[j]) + w->kTMf[j] * (P[j + 1] - P[j])) / dx;
        for (int f = 0; f < 2; ++f)
            if ((f == 0 && j == 0) || (f == 1 && j == N - 1))
                q += bc[f].hT * (bc[f].T_inf - T[j]) + Lv * bc[f].hM * (bc[f].P_inf - P[j]) + bc[f].q_inf +
                     bc[f].qR - bc[f].hR * T[j];
        q -= wj * dx * w->cTM[j] * (Pout[j] - P[j]) / tau;
        Tout[j] = T[j] + tau * q / (wj * dx * w->cTT[j]);
    }
    surface_flux(p, bc, T, P, N, fl);
}

int orc_euler_explicit_run(const orc_problem *p, orc_state *s, int64_t n_steps, double refine, int64_t *substeps,
                           int32_t n_threads)
{
    if (p == NULL || s == NULL || n_steps < 0 || !(refine >= 1.0)) return -1;
    if (p->n_rooms > 0 && (s->room == NULL || p->room_par == NULL || p->wall_area == NULL)) return -1;
    const int32_t W = p->n_walls, R = p->n_rooms;
    int64_t *node_off = (int64_t *)calloc((size_t)W + 1, sizeof(int64_t));
    int64_t *layer_off = (int64_t *)calloc((size_t)W + 1, sizeof(int64_t));
    if (!node_off || !layer_off) {
        free(node_off);
        free(layer_off);
        return -2;
    }
    int32_t Nmax = 3;
    for (int32_t w = 0; w < W; ++w) {
        if (p->n_nodes[w] < 3) {
            free(node_off);
            free(layer_off);
            return -1;
        }
        node_off[w + 1] = node_off[w] + p->n_nodes[w];
        layer_off[w + 1] = layer_off[w] + p->n_layers[w];
        if (p->n_nodes[w] > Nmax) Nmax = p->n_nodes[w];
    }
    const int64_t tot = node_off[W];
    double *T = (double *)malloc(sizeof(double) * (size_t)tot * 4);
    double *ra = (double *)malloc(sizeof(double) * ((size_t)R * 10 + 4));
    double *tw = (double *)malloc(sizeof(double) * ((size_t)W + 1));
    double *surf = (double *)calloc((size_t)W * 4 + 1, sizeof(double));
    double *qrad = (double *)calloc((size_t)W * 4 + 1, sizeof(double));
    double *lk = (double *)calloc((size_t)R * 3 + 1, sizeof(double));
    if (!T || !ra || !tw || !surf || !qrad || !lk) {
        free(node_off);
        free(layer_off);
        free(T);
        free(ra);
        free(tw);
        free(surf);
        free(qrad);
        free(lk);
        return -2;
    }
    double *P = T + tot, *T1 = T + 2 * tot, *P1 = T + 3 * tot;
    double *air = ra, *rsum = ra + 4 * R + 2;   /* room air in the room_state layout, room sums */
    if (n_threads <= 0) n_threads = 1;
    int rc = 0;
    for (int64_t it = 0; it < n_steps && rc == 0; ++it) {
        const double t0 = p->t0 + (double)s->step * p->dt;
        memcpy(T, s->T_cur, sizeof(double) * (size_t)tot);
        memcpy(P, s->P_cur, sizeof(double) * (size_t)tot);
        for (int32_t r = 0; r < R; ++r) {
            air[r * 4 + 1] = s->room[r * 4 + 1];
            air[r * 4 + 3] = s->room[r * 4 + 3];
        }
        /* substeps: the stability bound at the step's start, walls and rooms */
        double tmax = p->dt;
        int err = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads)
#endif
        {
            work wk;
            if (work_alloc(&wk, Nmax) != 0) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                err = -2;
            } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
                for (int32_t w = 0; w < W; ++w) {
                    const wall_view v = view_of(p, layer_off, w);
                    const face_bc bc[2] = {face_of(p, w, 0, t0, air), face_of(p, w, 1, t0, air)};
                    tw[w] = wall_tau(p, &v, bc, T + node_off[w], P + node_off[w], &wk);
                }
                free(wk.kM);
            }
        }
        if (err != 0) {
            rc = err;
            break;
        }
        for (int32_t w = 0; w < W; ++w) tmax = fmin(tmax, tw[w]);
        if (R > 0) {
            room_sums(p, node_off, T, P, rsum);
            for (int32_t r = 0; r < R; ++r) {
                const double *q = p->room_par + (size_t)r * ORC_NROOM_PAR;
                const double rhoV = q[R_RHOA] * q[R_VOL], gv = rhoV * q[R_ACH] / 3600.0, Pref = q[R_PVREF];
                double G = 0.0;
                for (int32_t l = 0; l < p->n_links; ++l)
                    if (p->link_zone[2 * l] == r || p->link_zone[2 * l + 1] == r) G += p->link_flow[l];
                const double kP = gv / Pref + rsum[r * 4 + 1] + G / Pref;
                const double kT = gv * q[R_CPA] + rsum[r * 4 + 0] + G * q[R_CPA];
                tmax = fmin(tmax, (rhoV / Pref) / kP);
                tmax = fmin(tmax, rhoV * (q[R_CPA] + q[R_CPV] * air[r * 4 + 3] / Pref) / kT);
            }
        }
        int64_t m = (int64_t)ceil(refine * p->dt / tmax);
        if (m < 1) m = 1;
        const double tau = p->dt / (double)m;
        for (int64_t i = 0; i < m && rc == 0; ++i) {
            const double t = t0 + (double)i * tau;
            if (R > 0) {
                surface_values(p, node_off, T, P, surf);
                room_radiation(p, surf, qrad);
                room_links(p, air, lk);
            }
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads)
#endif
            {
                work wk;
                if (work_alloc(&wk, Nmax) != 0) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                    err = -2;
                } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
                    for (int32_t w = 0; w < W; ++w) {
                        const wall_view v = view_of(p, layer_off, w);
                        face_bc bc[2] = {face_of(p, w, 0, t, air), face_of(p, w, 1, t, air)};
                        for (int f = 0; f < 2 && R > 0; ++f) {
                            bc[f].hR = qrad[(w * 2 + f) * 2 + 0];
                            bc[f].qR = qrad[(w * 2 + f) * 2 + 1];
                        }
                        const int64_t o = node_off[w];
                        double fl[2][2];
                        explicit_wall(p, &v, bc, T + o, P + o, tau, &wk, T1 + o, P1 + o, fl);
                        for (int f = 0; f < 2; ++f)
                            for (int c = 0; c < 2; ++c) s->cumul[w * 4 + f * 2 + c] += tau * fl[f][c];
                    }
                    free(wk.kM);
                }
            }
            if (err != 0) {
                rc = err;
                break;
            }
            /* rooms: forward Euler with the walls' surface values at the substep's start */
            if (R > 0) {
                room_sums(p, node_off, T, P, rsum);
                for (int32_t r = 0; r < R; ++r) {
                    const double *q = p->room_par + (size_t)r * ORC_NROOM_PAR;
                    const double Lv = p->Lv, Pref = q[R_PVREF];
                    const double rhoV = q[R_RHOA] * q[R_VOL], gv = rhoV * q[R_ACH] / 3600.0;
                    double T_out, P_out, g;
                    room_sources(p, r, t, &T_out, &P_out, &g);
                    const double w_out = P_out / Pref, Ta = air[r * 4 + 1], Pa = air[r * 4 + 3];
                    const double G = lk[r * 3 + 0], GT = lk[r * 3 + 1], Gw = lk[r * 3 + 2];
                    const double dP = (g + gv * (w_out - Pa / Pref) + rsum[r * 4 + 3] - rsum[r * 4 + 1] * Pa +
                                       Gw - G * Pa / Pref) /
                                      (rhoV / Pref);
                    const double CT = rhoV * (q[R_CPA] + q[R_CPV] * Pa / Pref);
                    const double dT = (q[R_QGAIN] + Lv * g + gv * q[R_CPA] * (T_out - Ta) + Lv * gv * (w_out - Pa / Pref) +
                                       rsum[r * 4 + 2] - rsum[r * 4 + 0] * Ta + Lv * (rsum[r * 4 + 3] - rsum[r * 4 + 1] * Pa) +
                                       q[R_CPA] * (GT - G * Ta) + Lv * (Gw - G * Pa / Pref)) /
                                      CT;
                    air[r * 4 + 1] = Ta + tau * dT;
                    air[r * 4 + 3] = Pa + tau * dP;
                }
            }
            double *sw = T;
            T = T1;
            T1 = sw;
            sw = P;
            P = P1;
            P1 = sw;
        }
        if (rc != 0) break;
        if (substeps) *substeps += m;
        memcpy(s->T_prev, s->T_cur, sizeof(double) * (size_t)tot);
        memcpy(s->P_prev, s->P_cur, sizeof(double) * (size_t)tot);
        memcpy(s->T_cur, T, sizeof(double) * (size_t)tot);
        memcpy(s->P_cur, P, sizeof(double) * (size_t)tot);
        for (int32_t r = 0; r < R; ++r) {
            s->room[r * 4 + 0] = s->room[r * 4 + 1];
            s->room[r * 4 + 1] = air[r * 4 + 1];
            s->room[r * 4 + 2] = s->room[r * 4 + 3];
            s->room[r * 4 + 3] = air[r * 4 + 3];
        }
        s->step += 1;
    }
    /* T, P may point into either half of the buffer after the swaps: free the allocation's start */
    free(T < T1 ? T : T1);
    free(node_off);
    free(layer_off);
    free(ra);
    free(tw);
    free(surf);
    free(qrad);
    free(lk);
    return rc;
}
