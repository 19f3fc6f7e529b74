/*
 * FP64 CPU oracle: plain statement of the Dufort-Frankel hygrothermal wall
 * update (arXiv:1703.10119). TEST INFRASTRUCTURE ONLY; see hygro_oracle.h
 * for what each part follows. Scalar loops, no blocking, no reordering.
 */
#include "hygro_oracle.h"
#include "oracle_internal.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif


/* Linear interpolation of an evenly spaced (T, Pv) noise table at time t,
 * held constant beyond its ends. */
static double noise_at(const float *tab, int32_t len, double noise_dt, double t, int field)
{
    if (tab == NULL || len <= 0 || noise_dt <= 0.0) return 0.0;
    double x = t / noise_dt;
    if (x <= 0.0) return (double)tab[field];
    if (x >= (double)(len - 1)) return (double)tab[(size_t)(len - 1) * 2 + field];
    double i = floor(x);
    size_t k = (size_t)i;
    double f = x - i;
    return (1.0 - f) * (double)tab[k * 2 + field] + f * (double)tab[(k + 1) * 2 + field];
}

/* Ambient air of an exterior face: daily sinusoid plus interpolated noise
 * (the T_inf, Pv_inf of [eq:HAM_BC]). */
void orc_ambient(const orc_problem *p, int32_t w, int32_t face, double t, double *T_inf, double *P_inf)
{
    const double *b = p->bc_par + ((size_t)w * 2 + face) * ORC_NBC_PAR;
    const float *tab = NULL;
    if (p->noise[face] != NULL && p->noise_len[face] > 0)
        tab = p->noise[face] + (size_t)w * (size_t)p->noise_len[face] * 2;
    double T = b[B_TMEAN], P = b[B_PMEAN];
    const double period_P = b[B_PERIODP] > 0.0 ? b[B_PERIODP] : b[B_PERIOD];
    if (b[B_PERIOD] > 0.0) T += b[B_TAMP] * sin(TWO_PI * t / b[B_PERIOD] + b[B_PHT]);
    if (period_P > 0.0) P += b[B_PAMP] * sin(TWO_PI * t / period_P + b[B_PHP]);
    T += noise_at(tab, p->noise_len[face], b[B_NDT], t, 0);
    P += noise_at(tab, p->noise_len[face], b[B_NDT], t, 1);
    *T_inf = T;
    *P_inf = P;
}


wall_view view_of(const orc_problem *p, const int64_t *layer_off, int32_t w)
{
    wall_view v;
    v.N = p->n_nodes[w];
    v.dx = p->thickness[w] / (double)(v.N - 1);
    v.nl = p->n_layers[w];
    v.first = p->layer_first + layer_off[w];
    v.par = p->layer_par + (size_t)layer_off[w] * ORC_NLAYER_PAR;
    v.law = p->layer_law != NULL ? p->layer_law + layer_off[w] : NULL;
    v.nu = p->vapour_frac != NULL ? p->vapour_frac[w] : 1.0;
    return v;
}

static int32_t layer_of(const wall_view *v, int32_t j)
{
    int32_t l = 0;
    while (l + 1 < v->nl && j >= v->first[l + 1]) ++l;
    return l;
}

/* The load bearing material of Sec. 4, Table 1 (see hygro_oracle.h for the formulas and the readings of
 * the parts the paper leaves open). The storage coefficient is the derivative of the sorption isotherm
 * with respect to Pv, cM = f'(phi) / Ps = (df / dPc) (dPc / dPv) with dPc / dPv = rho_l Rv T / Pv. */
void orc_table1(int32_t law, double T, double Pv, double Lv, double *out, double *ps, double *fw)
{
    const double rho_l = 1000.0, Rv = 461.5, c1 = 1.25e-5, c2 = 1.8e-5;
    const double rho0 = 790.0, c0 = 870.0, cw = 4180.0;
    const double theta = T - 273.15;
    const double Ps = 610.94 * exp(17.625 * theta / (theta + 243.04));
    /* above saturation the isotherm has no values: the capillary pressure is held at 0 (saturated) */
    const double Pc = fmin(0.0, rho_l * Rv * T * log(Pv / Ps));
    const double x1 = -c1 * Pc, x2 = -c2 * Pc;
    const double f = 47.1 * pow(1.0 + pow(x1, 1.65), -0.39) + 109.9 * pow(1.0 + pow(x2, 6.0), -0.83);
    /* df/dPc: each term a (1 + (-c Pc)^m)^-e gives a e m c (-c Pc)^(m-1) (1 + (-c Pc)^m)^(-e-1) */
    const double dfdPc = 47.1 * 0.39 * 1.65 * c1 * pow(x1, 0.65) * pow(1.0 + pow(x1, 1.65), -1.39) +
                         109.9 * 0.83 * 6.0 * c2 * pow(x2, 5.0) * pow(1.0 + pow(x2, 6.0), -1.83);
    const double cM = dfdPc * rho_l * Rv * T / Pv;
    const double s = 1.0 - f / 157.0;
    const double dv = 1.88e-6 / T * s / (0.503 * s * s + 0.497);
    const double x = 2.0 * Pv / Ps;
    double liquid;
    if (law == ORC_LAW_TABLE1_A) {
        const double y = -8.0 * x - 2.0;
        liquid = exp(y * y);
    } else if (law == ORC_LAW_TABLE1_C) {
        liquid = exp(-8.0 * (x - 2.0) * (x - 2.0));
    } else {
        const double e = exp(-8.0 * x - 2.0);
        liquid = e * e;
    }
    const double kM = 1.97e-10 * exp(-0.07 * log10(x) + 1.44) + 1.77e-7 * liquid;
    out[0] = kM;
    out[1] = cM;
    out[2] = 0.2 + 0.0045 * f;
    out[3] = rho0 * c0 + f * cw;
    out[4] = Lv * dv;
    out[5] = cw * theta * cM;
    if (ps) *ps = Ps;
    if (fw) *fw = f;
}

/* Material coefficients of Sec. 2 evaluated at level n (explicitly, as the
 * paper prescribes for the DF scheme in Sec. 3.1), then their face values:
 * arithmetic mean of the two nodes inside a layer (for coefficients affine
 * in Pv this equals the coefficient at the face-mean Pv, Sec. 3.1) and the
 * harmonic mean across an interface between two layers. Affine layers:
 * kTM_f = nu Lv kM_f. Layers of a Table-1 law: their kTM = Lv dv takes the
 * face rule of the other conductances. */
void coefficients(const orc_problem *p, const wall_view *v, const double *T, const double *P,
                         double *kM, double *cM, double *kTT, double *cTT, double *kTM, double *cTM,
                         double *kMf, double *kTTf, double *kTMf)
{
    for (int32_t j = 0; j < v->N; ++j) {
        const int32_t l = layer_of(v, j);
        const int32_t law = v->law != NULL ? v->law[l] : ORC_LAW_AFFINE;
        if (law != ORC_LAW_AFFINE) {
            double c[6];
            orc_table1(law, T[j], P[j], p->Lv, c, NULL, NULL);
            kM[j] = c[0];
            cM[j] = c[1];
            kTT[j] = c[2];
            cTT[j] = c[3];
            kTM[j] = c[4];
            cTM[j] = c[5];
            continue;
        }
        const double *q = v->par + (size_t)l * ORC_NLAYER_PAR;
        double r = P[j] / p->Psat;
        kM[j] = q[L_KM0] * (1.0 + q[L_A] * r);
        cM[j] = q[L_CM0] * (1.0 + q[L_B] * r);
        kTT[j] = q[L_KTT0] * (1.0 + q[L_AT] * r);
        cTT[j] = q[L_CTT0] * (1.0 + q[L_BT] * r);
        kTM[j] = v->nu * p->Lv * kM[j];
        cTM[j] = q[L_CHI] * cM[j];
    }
    for (int32_t j = 0; j + 1 < v->N; ++j) {
        const int32_t l0 = layer_of(v, j), l1 = layer_of(v, j + 1);
        const int affine = v->law == NULL || (v->law[l0] == ORC_LAW_AFFINE && v->law[l1] == ORC_LAW_AFFINE);
        if (l0 == l1) {
            kMf[j] = 0.5 * (kM[j] + kM[j + 1]);
            kTTf[j] = 0.5 * (kTT[j] + kTT[j + 1]);
            kTMf[j] = affine ? v->nu * p->Lv * kMf[j] : 0.5 * (kTM[j] + kTM[j + 1]);
        } else {
            kMf[j] = 2.0 * kM[j] * kM[j + 1] / (kM[j] + kM[j + 1]);
            kTTf[j] = 2.0 * kTT[j] * kTT[j + 1] / (kTT[j] + kTT[j + 1]);
            kTMf[j] = affine ? v->nu * p->Lv * kMf[j] : 2.0 * kTM[j] * kTM[j + 1] / (kTM[j] + kTM[j + 1]);
        }
    }
}

void orc_coefficients(const orc_problem *p, int32_t w, const double *T, const double *P, double *node6,
                      double *face3)
{
    int64_t *off = (int64_t *)calloc((size_t)p->n_walls + 1, sizeof(int64_t));
    for (int32_t i = 0; i < p->n_walls; ++i) off[i + 1] = off[i] + p->n_layers[i];
    wall_view v = view_of(p, off, w);
    int32_t N = v.N;
    double *buf = (double *)malloc(sizeof(double) * (size_t)(9 * N));
    coefficients(p, &v, T != NULL ? T : P, P, buf, buf + N, buf + 2 * N, buf + 3 * N, buf + 4 * N, buf + 5 * N,
                 buf + 6 * N, buf + 7 * N, buf + 8 * N);
    for (int32_t j = 0; j < N; ++j)
        for (int k = 0; k < 6; ++k) node6[j * 6 + k] = buf[k * N + j];
    for (int32_t j = 0; j + 1 < N; ++j)
        for (int k = 0; k < 3; ++k) face3[j * 3 + k] = buf[(6 + k) * N + j];
    free(buf);
    free(off);
}


face_bc face_of(const orc_problem *p, int32_t w, int32_t f, double t, const double *room_state)
{
    face_bc s;
    memset(&s, 0, sizeof s);
    const double *b = p->bc_par + ((size_t)w * 2 + f) * ORC_NBC_PAR;
    int32_t kind = p->bc_kind[w * 2 + f];
    if (kind == ORC_BC_ADIABATIC) return s;
    s.hT = b[B_HT];
    s.hM = b[B_HM];
    s.q_inf = b[B_QINF];
    s.g_inf = b[B_GINF];
    if (kind == ORC_BC_ROOM) {
        /* explicit coupling [eq:wbse_tn_exp]: the wall sees the room air at level n */
        int32_t r = p->bc_room[w * 2 + f];
        s.T_inf = room_state[r * 4 + 1];
        s.P_inf = room_state[r * 4 + 3];
    } else {
        orc_ambient(p, w, f, t, &s.T_inf, &s.P_inf);
    }
    return s;
}

typedef struct {
    double *kM, *cM, *kTT, *cTT, *kTM, *cTM, *kMf, *kTTf, *kTMf, *Pn, *Tn;
} scratch;

/* One DF step of one wall. On return Tp / Pp hold level n+1.
 *
 * Per node j, with half-cell weight w_j (1/2 at the two surface nodes),
 * the DF balance of [eq:DF_NL] in conservative form reads
 *   w_j dx c_j (u_j^{n+1} - u_j^{n-1}) / (2 dt)
 *      = sum_{faces f of j} k_f (u_nb^n - ubar_j) / dx + surface terms,
 *   ubar_j = (u_j^{n+1} + u_j^{n-1}) / 2,
 * which is solved for u_j^{n+1}. Pv is advanced first ([eq:DF_eq1]); the T
 * equation then carries the kTM cross flux and the cTM storage term with
 * Pv^{n+1} ([eq:DF_eq2]). At a surface node the Robin exchange enters with
 * the time-averaged surface value, which is what the ghost node of
 * [eq:ghost_node_v0] / [eq:ghost_node_u0] substitutes. */
static void wall_step(const orc_problem *p, const wall_view *v, const face_bc bc[2],
                      double *Tp, const double *Tc, double *Pp, const double *Pc, scratch *sc,
                      double flux[2][2], double bal[2][4])
{
    const int32_t N = v->N;
    const double dx = v->dx, dt = p->dt, Lv = p->Lv;
    coefficients(p, v, Tc, Pc, sc->kM, sc->cM, sc->kTT, sc->cTT, sc->kTM, sc->cTM, sc->kMf, sc->kTTf,
                 sc->kTMf);

    /* vapour pressure first */
    for (int32_t j = 0; j < N; ++j) {
        double w = (j == 0 || j == N - 1) ? 0.5 : 1.0;
        double A = w * dx * sc->cM[j] / (2.0 * dt);
        double S = 0.0, nb = 0.0, H = 0.0, src = 0.0;
        if (j > 0) {
            S += sc->kMf[j - 1] / dx;
            nb += sc->kMf[j - 1] / dx * Pc[j - 1];
        }
        if (j < N - 1) {
            S += sc->kMf[j] / dx;
            nb += sc->kMf[j] / dx * Pc[j + 1];
        }
        if (j == 0) {
            H += bc[0].hM;
            src += bc[0].hM * bc[0].P_inf + bc[0].g_inf;
        }
        if (j == N - 1) {
            H += bc[1].hM;
            src += bc[1].hM * bc[1].P_inf + bc[1].g_inf;
        }
        sc->Pn[j] = ((A - 0.5 * S - 0.5 * H) * Pp[j] + nb + src) / (A + 0.5 * S + 0.5 * H);
    }

    /* then temperature, using Pv^{n+1} of the same node */
    for (int32_t j = 0; j < N; ++j) {
        double w = (j == 0 || j == N - 1) ? 0.5 : 1.0;
        double B = w * dx * sc->cTT[j] / (2.0 * dt);
        double C = w * dx * sc->cTM[j] / (2.0 * dt);
        double Pbar = 0.5 * (sc->Pn[j] + Pp[j]);
        double S = 0.0, nb = 0.0, cross = 0.0, H = 0.0, src = 0.0;
        if (j > 0) {
            S += sc->kTTf[j - 1] / dx;
            nb += sc->kTTf[j - 1] / dx * Tc[j - 1];
            cross += sc->kTMf[j - 1] / dx * (Pc[j - 1] - Pbar);
        }
        if (j < N - 1) {
            S += sc->kTTf[j] / dx;
            nb += sc->kTTf[j] / dx * Tc[j + 1];
            cross += sc->kTMf[j] / dx * (Pc[j + 1] - Pbar);
        }
        for (int f = 0; f < 2; ++f) {
            if ((f == 0 && j == 0) || (f == 1 && j == N - 1)) {
                H += bc[f].hT + bc[f].hR;
                src += bc[f].hT * bc[f].T_inf + Lv * bc[f].hM * (bc[f].P_inf - Pbar) + bc[f].q_inf + bc[f].qR;
            }
        }
        sc->Tn[j] = ((B - 0.5 * S - 0.5 * H) * Tp[j] + nb + cross + src - C * (sc->Pn[j] - Pp[j])) /
                    (B + 0.5 * S + 0.5 * H);
    }

    /* surface fluxes into the wall, [eq:HAM_BC] with the time-averaged surface values */
    for (int f = 0; f < 2; ++f) {
        int32_t j = f == 0 ? 0 : N - 1;
        double Tbar = 0.5 * (sc->Tn[j] + Tp[j]);
        double Pbar = 0.5 * (sc->Pn[j] + Pp[j]);
        double g = bc[f].hM * (bc[f].P_inf - Pbar) + bc[f].g_inf;
        double q = bc[f].hT * (bc[f].T_inf - Tbar) + Lv * bc[f].hM * (bc[f].P_inf - Pbar) + bc[f].q_inf +
                   bc[f].qR - bc[f].hR * Tbar;
        flux[f][0] = q;
        flux[f][1] = g;
    }

    /* discrete balance of this step: storage S, boundary B, DF defect D */
    if (bal != NULL) {
        double S_T = 0, S_P = 0, M_T = 0, M_P = 0, D_T = 0, D_P = 0;
        for (int32_t j = 0; j < N; ++j) {
            double w = (j == 0 || j == N - 1) ? 0.5 : 1.0;
            double sP = w * dx * sc->cM[j] * (sc->Pn[j] - Pp[j]) / (2.0 * dt);
            double sT = w * dx * (sc->cTT[j] * (sc->Tn[j] - Tp[j]) + sc->cTM[j] * (sc->Pn[j] - Pp[j])) /
                        (2.0 * dt);
            S_P += sP;
            S_T += sT;
            M_P += fabs(sP);
            M_T += fabs(sT);
        }
        for (int32_t j = 0; j + 1 < N; ++j) {
            double Pb0 = 0.5 * (sc->Pn[j] + Pp[j]), Pb1 = 0.5 * (sc->Pn[j + 1] + Pp[j + 1]);
            double Tb0 = 0.5 * (sc->Tn[j] + Tp[j]), Tb1 = 0.5 * (sc->Tn[j + 1] + Tp[j + 1]);
            double dP = sc->kMf[j] / dx * ((Pc[j + 1] - Pb1) + (Pc[j] - Pb0));
            double dT = sc->kTTf[j] / dx * ((Tc[j + 1] - Tb1) + (Tc[j] - Tb0)) +
                        sc->kTMf[j] / dx * ((Pc[j + 1] - Pb1) + (Pc[j] - Pb0));
            D_P += dP;
            D_T += dT;
            M_P += sc->kMf[j] / dx * (fabs(Pc[j + 1] - Pb0) + fabs(Pc[j] - Pb1));
            M_T += sc->kTTf[j] / dx * (fabs(Tc[j + 1] - Tb0) + fabs(Tc[j] - Tb1)) +
                   sc->kTMf[j] / dx * (fabs(Pc[j + 1] - Pb0) + fabs(Pc[j] - Pb1));
        }
        double B_T = flux[0][0] + flux[1][0], B_P = flux[0][1] + flux[1][1];
        M_T += fabs(flux[0][0]) + fabs(flux[1][0]);
        M_P += fabs(flux[0][1]) + fabs(flux[1][1]);
        bal[0][0] = S_T; bal[0][1] = B_T; bal[0][2] = D_T; bal[0][3] = M_T;
        bal[1][0] = S_P; bal[1][1] = B_P; bal[1][2] = D_P; bal[1][3] = M_P;
    }

    for (int32_t j = 0; j < N; ++j) {
        Tp[j] = sc->Tn[j];
        Pp[j] = sc->Pn[j];
    }
}

/* Outdoor air of a room's ventilation and the occupants' vapour production (Sec. 5.1: base load plus
 * the daily pulse) at time t. */
void room_sources(const orc_problem *p, int32_t r, double t, double *T_out, double *P_out, double *g_vap)
{
    const double *q = p->room_par + (size_t)r * ORC_NROOM_PAR;
    double T = q[R_TMEAN], P = q[R_PMEAN];
    const double period_P = q[R_PERIODP] > 0.0 ? q[R_PERIODP] : q[R_PERIOD];
    if (q[R_PERIOD] > 0.0) T += q[R_TAMP] * sin(TWO_PI * t / q[R_PERIOD] + q[R_PHT]);
    if (period_P > 0.0) P += q[R_PAMP] * sin(TWO_PI * t / period_P + q[R_PHP]);
    double g = q[R_GVAP];
    if (q[R_PPER] > 0.0) {
        const double ph = fmod(t, q[R_PPER]);
        if (ph >= q[R_PON] && ph < q[R_POFF]) g += q[R_GPULSE];
    }
    *T_out = T;
    *P_out = P;
    *g_vap = g;
}

/* Room air node of Sec. 5.1 ([eq:LAV_equation] with the sources of the
 * occupants and of ventilation, the wall exchanges [eq:LAV_couplage]),
 * humidity ratio w = Pva / Pv_ref. The wall surface values enter at level n
 * as in [eq:wbse_tn_exp]; the room node itself is advanced with the DF
 * replacement (Ta^{n+1} + Ta^{n-1}) / 2 of its own value, vapour first. */
/* q_rw = s eps sigma sum over the room's faces of (T'^4 - Ts^4) (Sec. 2). Each term factors exactly as
 * h' (T' - Ts) with the radiative conductance h' = s eps sigma (T'^2 + Ts^2)(T' + Ts), symmetric in the two
 * surfaces; written so, q_rw has the form of DF faces to the other surfaces: conductances and the other
 * surfaces' temperatures of level n, the face's own value averaged over levels n+1 and n-1 (a level-n own
 * value would be a leapfrog term, unstable in DF). rad = (hR, qR) = (sum h', sum h' T'), the face receiving
 * qR - hR Ts. */
void room_radiation(const orc_problem *p, const double *surf, double *rad)
{
    const int32_t W = p->n_walls;
    for (int32_t i = 0; i < 4 * W; ++i) rad[i] = 0.0;
    if (p->face_emis == NULL || p->room_view == NULL) return;
    for (int32_t w = 0; w < W; ++w)
        for (int f = 0; f < 2; ++f) {
            if (p->bc_kind[w * 2 + f] != ORC_BC_ROOM) continue;
            const int32_t r = p->bc_room[w * 2 + f];
            const double Ts = surf[w * 4 + f * 2];
            const double c = p->room_view[r] * p->face_emis[w * 2 + f] * ORC_SIGMA;
            double hR = 0.0, qR = 0.0;
            for (int32_t u = 0; u < W; ++u)
                for (int g = 0; g < 2; ++g) {
                    if (p->bc_kind[u * 2 + g] != ORC_BC_ROOM || p->bc_room[u * 2 + g] != r) continue;
                    if (u == w && g == f) continue;
                    const double To = surf[u * 4 + g * 2];
                    const double h = c * (To * To + Ts * Ts) * (To + Ts);
                    hR += h;
                    qR += h * To;
                }
            rad[(w * 2 + f) * 2 + 0] = hR;
            rad[(w * 2 + f) * 2 + 1] = qR;
        }
}

void room_links(const orc_problem *p, const double *rs, double *lk)
{
    for (int32_t i = 0; i < 3 * p->n_rooms; ++i) lk[i] = 0.0;
    for (int32_t l = 0; l < p->n_links; ++l) {
        const double g = p->link_flow[l];
        for (int e = 0; e < 2; ++e) {
            const int32_t r = p->link_zone[2 * l + e], o = p->link_zone[2 * l + 1 - e];
            const double *qo = p->room_par + (size_t)o * ORC_NROOM_PAR;
            lk[r * 3 + 0] += g;
            lk[r * 3 + 1] += g * rs[o * 4 + 1];
            lk[r * 3 + 2] += g * rs[o * 4 + 3] / qo[R_PVREF];
        }
    }
}

/* lk: this room's interzone sums (room_links) at level n. */
static void room_step(const orc_problem *p, int32_t r, double t, double *rs,
                      const double *sum_AhT, const double *sum_AhM, const double *sum_AhTTs,
                      const double *sum_AhMPs, const double *lk)
{
    const double *q = p->room_par + (size_t)r * ORC_NROOM_PAR;
    const double dt = p->dt, Lv = p->Lv;
    double Ta_p = rs[0], Ta_c = rs[1], Pa_p = rs[2], Pa_c = rs[3];
    double rhoV = q[R_RHOA] * q[R_VOL];
    double gv = rhoV * q[R_ACH] / 3600.0;                        /* kg/s of exchanged air */
    double T_out, P_out, g_vap;
    room_sources(p, r, t, &T_out, &P_out, &g_vap);
    double Pref = q[R_PVREF];
    double w_out = P_out / Pref;
    /* interzone airflow: G_inz = sum g (w_o - w), Q_inz = sum g [cpa (T_o - Ta) + Lv (w_o - w)] */
    const double G = lk[0], GT = lk[1], Gw = lk[2];
    if (q[R_SCHEME] == 1.0) {
        /* the explicit Euler update of Sec. 5.2: every term of both balances at level n */
        double Pa_n = Pa_c + dt / (rhoV / Pref) * (g_vap + gv * (w_out - Pa_c / Pref) + sum_AhMPs[r] - sum_AhM[r] * Pa_c +
                                                   Gw - G * Pa_c / Pref);
        double CT0 = rhoV * (q[R_CPA] + q[R_CPV] * Pa_c / Pref);
        double rhs0 = q[R_QGAIN] + Lv * g_vap + gv * q[R_CPA] * (T_out - Ta_c) + Lv * gv * (w_out - Pa_c / Pref) +
                      sum_AhTTs[r] - sum_AhT[r] * Ta_c + Lv * (sum_AhMPs[r] - sum_AhM[r] * Pa_c) +
                      q[R_CPA] * (GT - G * Ta_c) + Lv * (Gw - G * Pa_c / Pref);
        double Ta_n = Ta_c + dt / CT0 * rhs0;
        rs[0] = Ta_c;
        rs[1] = Ta_n;
        rs[2] = Pa_c;
        rs[3] = Pa_n;
        return;
    }
    /* vapour: rhoV/Pref dPa/dt = g_vap + gv (w_out - Pa/Pref) + sum A hM (Ps - Pa) */
    double CP = rhoV / Pref;
    double a_p = CP / (2.0 * dt);
    double k_p = gv / Pref + sum_AhM[r] + G / Pref;
    double Pa_n = ((a_p - 0.5 * k_p) * Pa_p + g_vap + gv * w_out + sum_AhMPs[r] + Gw) / (a_p + 0.5 * k_p);
    double Pa_bar = 0.5 * (Pa_n + Pa_p);
    /* heat: rhoV (cpa + cpv w) dTa/dt = Q + Lv g_vap + gv cpa (T_out - Ta) + Lv gv (w_out - w)
     *       + sum A [hT (Ts - Ta) + Lv hM (Ps - Pa)] */
    double CT = rhoV * (q[R_CPA] + q[R_CPV] * Pa_c / Pref);
    double a_t = CT / (2.0 * dt);
    double k_t = gv * q[R_CPA] + sum_AhT[r] + G * q[R_CPA];
    double rhs = q[R_QGAIN] + Lv * g_vap + gv * q[R_CPA] * T_out + Lv * gv * (w_out - Pa_bar / Pref) +
                 sum_AhTTs[r] + Lv * (sum_AhMPs[r] - sum_AhM[r] * Pa_bar) + q[R_CPA] * GT +
                 Lv * (Gw - G * Pa_bar / Pref);
    double Ta_n = ((a_t - 0.5 * k_t) * Ta_p + rhs) / (a_t + 0.5 * k_t);
    rs[0] = Ta_c;
    rs[1] = Ta_n;
    rs[2] = Pa_c;
    rs[3] = Pa_n;
}

/* Start by explicit Euler substeps (an option of the first step): level 1 from level 0 by m explicit
 * Euler steps of tau = dt / m, the coefficients of Sec. 2 re-evaluated at every substep, Pv first and T
 * with the substep's Pv change in the cTM storage term, the ambient air at each substep's time. m is the
 * smallest count with tau within the explicit stability bound of every node at level 0,
 * tau <= w dx c / (sum of the face conductances k_f/dx + h) for both fields, times refine (>= 1).
 * Afterwards level n-1 holds level 0, level n holds level 1, and the step is 1; the flux sums receive
 * the sum over substeps of tau times the surface fluxes (surface values at each substep's start). */
int orc_euler_start(const orc_problem *p, orc_state *s, double refine, int32_t n_threads)
{
    if (p == NULL || s == NULL || s->step != 0 || !(refine >= 1.0) || p->n_rooms > 0) return -1;
    const int32_t W = p->n_walls;
    int64_t *node_off = (int64_t *)calloc((size_t)W + 1, sizeof(int64_t));
    int64_t *layer_off = (int64_t *)calloc((size_t)W + 1, sizeof(int64_t));
    if (!node_off || !layer_off) {
        free(node_off);
        free(layer_off);
        return -2;
    }
    int32_t Nmax = 3;
    for (int32_t w = 0; w < W; ++w) {
        node_off[w + 1] = node_off[w] + p->n_nodes[w];
        layer_off[w + 1] = layer_off[w] + p->n_layers[w];
        if (p->n_nodes[w] > Nmax) Nmax = p->n_nodes[w];
    }
    if (n_threads <= 0) n_threads = 1;
    int rc = 0;
#ifdef _OPENMP
#pragma omp parallel for num_threads(n_threads) schedule(dynamic, 1)
#endif
    for (int32_t w = 0; w < W; ++w) {
        double *buf = (double *)malloc(sizeof(double) * (size_t)Nmax * 13);
        if (buf == NULL) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            rc = -2;
            continue;
        }
        scratch sc;
        sc.kM = buf; sc.cM = buf + Nmax; sc.kTT = buf + 2 * Nmax; sc.cTT = buf + 3 * Nmax;
        sc.kTM = buf + 4 * Nmax; sc.cTM = buf + 5 * Nmax; sc.kMf = buf + 6 * Nmax;
        sc.kTTf = buf + 7 * Nmax; sc.kTMf = buf + 8 * Nmax; sc.Pn = buf + 9 * Nmax; sc.Tn = buf + 10 * Nmax;
        double *T = buf + 11 * Nmax, *P = buf + 12 * Nmax;
        wall_view v = view_of(p, layer_off, w);
        const int32_t N = v.N;
        const double dx = v.dx, dt = p->dt, Lv = p->Lv;
        const int64_t o = node_off[w];
        for (int32_t j = 0; j < N; ++j) {
            T[j] = s->T_cur[o + j];
            P[j] = s->P_cur[o + j];
        }
        /* the stability bound at level 0 */
        coefficients(p, &v, T, P, sc.kM, sc.cM, sc.kTT, sc.cTT, sc.kTM, sc.cTM, sc.kMf, sc.kTTf, sc.kTMf);
        face_bc b0[2] = {face_of(p, w, 0, p->t0, NULL), face_of(p, w, 1, p->t0, NULL)};
        double tmax = dt;
        for (int32_t j = 0; j < N; ++j) {
            const double wj = (j == 0 || j == N - 1) ? 0.5 : 1.0;
            double GM = 0.0, GT = 0.0;
            if (j > 0) {
                GM += sc.kMf[j - 1] / dx;
                GT += sc.kTTf[j - 1] / dx;
            }
            if (j < N - 1) {
                GM += sc.kMf[j] / dx;
                GT += sc.kTTf[j] / dx;
            }
            if (j == 0) {
                GM += b0[0].hM;
                GT += b0[0].hT;
            }
            if (j == N - 1) {
                GM += b0[1].hM;
                GT += b0[1].hT;
            }
            if (GM > 0.0 && wj * dx * sc.cM[j] / GM < tmax) tmax = wj * dx * sc.cM[j] / GM;
            if (GT > 0.0 && wj * dx * sc.cTT[j] / GT < tmax) tmax = wj * dx * sc.cTT[j] / GT;
        }
        int64_t m = (int64_t)ceil(refine * dt / tmax);
        if (m < 1) m = 1;
        const double tau = dt / (double)m;
        for (int64_t i = 0; i < m; ++i) {
            const double t = p->t0 + (double)i * tau;
            face_bc bc[2] = {face_of(p, w, 0, t, NULL), face_of(p, w, 1, t, NULL)};
            coefficients(p, &v, T, P, sc.kM, sc.cM, sc.kTT, sc.cTT, sc.kTM, sc.cTM, sc.kMf, sc.kTTf, sc.kTMf);
            /* surface fluxes with the values at the substep's start */
            for (int f = 0; f < 2; ++f) {
                const int32_t j = f == 0 ? 0 : N - 1;
                const double g = bc[f].hM * (bc[f].P_inf - P[j]) + bc[f].g_inf;
                const double q = bc[f].hT * (bc[f].T_inf - T[j]) + Lv * bc[f].hM * (bc[f].P_inf - P[j]) + bc[f].q_inf;
                s->cumul[w * 4 + f * 2 + 0] += tau * q;
                s->cumul[w * 4 + f * 2 + 1] += tau * g;
            }
            for (int32_t j = 0; j < N; ++j) {
                const double wj = (j == 0 || j == N - 1) ? 0.5 : 1.0;
                double rP = 0.0, rT = 0.0;
                if (j > 0) {
                    rP += sc.kMf[j - 1] / dx * (P[j - 1] - P[j]);
                    rT += sc.kTTf[j - 1] / dx * (T[j - 1] - T[j]) + sc.kTMf[j - 1] / dx * (P[j - 1] - P[j]);
                }
                if (j < N - 1) {
                    rP += sc.kMf[j] / dx * (P[j + 1] - P[j]);
                    rT += sc.kTTf[j] / dx * (T[j + 1] - T[j]) + sc.kTMf[j] / dx * (P[j + 1] - P[j]);
                }
                for (int f = 0; f < 2; ++f)
                    if ((f == 0 && j == 0) || (f == 1 && j == N - 1)) {
                        rP += bc[f].hM * (bc[f].P_inf - P[j]) + bc[f].g_inf;
                        rT += bc[f].hT * (bc[f].T_inf - T[j]) + Lv * bc[f].hM * (bc[f].P_inf - P[j]) + bc[f].q_inf;
                    }
                const double dP = tau * rP / (wj * dx * sc.cM[j]);
                sc.Pn[j] = P[j] + dP;
                sc.Tn[j] = T[j] + tau * rT / (wj * dx * sc.cTT[j]) - sc.cTM[j] / sc.cTT[j] * dP;
            }
            for (int32_t j = 0; j < N; ++j) {
                T[j] = sc.Tn[j];
                P[j] = sc.Pn[j];
            }
        }
        for (int32_t j = 0; j < N; ++j) {
            s->T_prev[o + j] = s->T_cur[o + j];
            s->P_prev[o + j] = s->P_cur[o + j];
            s->T_cur[o + j] = T[j];
            s->P_cur[o + j] = P[j];
        }
        free(buf);
    }
    free(node_off);
    free(layer_off);
    if (rc == 0) s->step = 1;
    return rc;
}

int orc_run(const orc_problem *p, orc_state *s, int64_t n_steps, int32_t sample_every,
            double *samples, double *room_samples, double *flux_last, double *balance_last,
            int32_t n_threads)
{
    if (p == NULL || s == NULL || n_steps < 0 || p->n_walls < 0) return -1;
    if ((samples != NULL || room_samples != NULL) && sample_every <= 0) return -1;
    const int32_t W = p->n_walls;
    for (int32_t w = 0; w < W; ++w)
        if (p->n_nodes[w] < 3 || p->n_layers[w] < 1 || !(p->thickness[w] > 0.0)) return -1;
    if (p->n_rooms > 0 && (s->room == NULL || p->room_par == NULL || p->wall_area == NULL)) return -1;

    int64_t *node_off = (int64_t *)calloc((size_t)W + 1, sizeof(int64_t));
    int64_t *layer_off = (int64_t *)calloc((size_t)W + 1, sizeof(int64_t));
    if (!node_off || !layer_off) {
        free(node_off);
        free(layer_off);
        return -2;
    }
    int32_t Nmax = 3;
    for (int32_t w = 0; w < W; ++w) {
        node_off[w + 1] = node_off[w] + p->n_nodes[w];
        layer_off[w + 1] = layer_off[w] + p->n_layers[w];
        if (p->n_nodes[w] > Nmax) Nmax = p->n_nodes[w];
    }
    const int32_t R = p->n_rooms;
    double *surf = (double *)calloc((size_t)W * 4 + 1, sizeof(double)); /* Ts^n, Ps^n of face 0, face 1 */
    double *rsum = (double *)calloc((size_t)R * 4 + 1, sizeof(double));
    double *flux = (double *)calloc((size_t)W * 4 + 1, sizeof(double));
    double *qrad = (double *)calloc((size_t)W * 4 + 1, sizeof(double));   /* radiative hR, qR of each face */
    double *lk = (double *)calloc((size_t)R * 3 + 1, sizeof(double));     /* interzone sums of each room */
    double *rs0 = (double *)calloc((size_t)R * 4 + 1, sizeof(double));    /* room states of level n */
    if (!surf || !rsum || !flux || !qrad || !lk || !rs0) {
        free(node_off); free(layer_off); free(surf); free(rsum); free(flux); free(qrad); free(lk); free(rs0);
        return -2;
    }
    if (n_threads <= 0) n_threads = 1;
    int rc = 0;

    for (int64_t it = 0; it < n_steps; ++it) {
        const int64_t n = s->step;
        const double t = p->t0 + (double)n * p->dt;
        const int last = (it == n_steps - 1);
        /* wall surface values at level n, used by the room balance of this step */
        for (int32_t w = 0; w < W; ++w) {
            surf[w * 4 + 0] = s->T_cur[node_off[w]];
            surf[w * 4 + 1] = s->P_cur[node_off[w]];
            surf[w * 4 + 2] = s->T_cur[node_off[w] + p->n_nodes[w] - 1];
            surf[w * 4 + 3] = s->P_cur[node_off[w] + p->n_nodes[w] - 1];
        }
        /* long-wave exchange among each room's surfaces at level n (explicit, a surface heat source) */
        if (R > 0) room_radiation(p, surf, qrad);
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads)
#endif
        {
            scratch sc;
            double *buf = (double *)malloc(sizeof(double) * (size_t)Nmax * 11);
            if (buf == NULL) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                rc = -2;
            } else {
                sc.kM = buf; sc.cM = buf + Nmax; sc.kTT = buf + 2 * Nmax; sc.cTT = buf + 3 * Nmax;
                sc.kTM = buf + 4 * Nmax; sc.cTM = buf + 5 * Nmax; sc.kMf = buf + 6 * Nmax;
                sc.kTTf = buf + 7 * Nmax; sc.kTMf = buf + 8 * Nmax; sc.Pn = buf + 9 * Nmax;
                sc.Tn = buf + 10 * Nmax;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
                for (int32_t w = 0; w < W; ++w) {
                    wall_view v = view_of(p, layer_off, w);
                    face_bc bc[2] = {face_of(p, w, 0, t, s->room), face_of(p, w, 1, t, s->room)};
                    for (int f = 0; f < 2 && R > 0; ++f) {
                        bc[f].hR = qrad[(w * 2 + f) * 2 + 0];
                        bc[f].qR = qrad[(w * 2 + f) * 2 + 1];
                    }
                    double fl[2][2], bl[2][4];
                    int64_t o = node_off[w];
                    wall_step(p, &v, bc, s->T_prev + o, s->T_cur + o, s->P_prev + o, s->P_cur + o, &sc,
                              fl, (last && balance_last) ? bl : NULL);
                    for (int f = 0; f < 2; ++f)
                        for (int k = 0; k < 2; ++k) {
                            flux[w * 4 + f * 2 + k] = fl[f][k];
                            s->cumul[w * 4 + f * 2 + k] += p->dt * fl[f][k];
                        }
                    if (last && balance_last)
                        for (int f = 0; f < 2; ++f)
                            for (int k = 0; k < 4; ++k) balance_last[(size_t)w * 8 + f * 4 + k] = bl[f][k];
                    /* rotate: level n becomes n-1, level n+1 (written into *_prev) becomes n */
                    for (int32_t j = 0; j < v.N; ++j) {
                        double tt = s->T_prev[o + j];
                        s->T_prev[o + j] = s->T_cur[o + j];
                        s->T_cur[o + j] = tt;
                        double pp = s->P_prev[o + j];
                        s->P_prev[o + j] = s->P_cur[o + j];
                        s->P_cur[o + j] = pp;
                    }
                }
                free(buf);
            }
        }
        if (rc != 0) break;

        if (R > 0) {
            /* per-room sums over the room-side wall faces, surface values at level n */
            double *AhT = rsum, *AhM = rsum + R, *AhTTs = rsum + 2 * R, *AhMPs = rsum + 3 * R;
            for (int32_t i = 0; i < 4 * R; ++i) rsum[i] = 0.0;
            for (int32_t w = 0; w < W; ++w)
                for (int f = 0; f < 2; ++f) {
                    if (p->bc_kind[w * 2 + f] != ORC_BC_ROOM) continue;
                    int32_t r = p->bc_room[w * 2 + f];
                    const double *b = p->bc_par + ((size_t)w * 2 + f) * ORC_NBC_PAR;
                    double A = p->wall_area[w];
                    AhT[r] += A * b[B_HT];
                    AhM[r] += A * b[B_HM];
                    AhTTs[r] += A * b[B_HT] * surf[w * 4 + f * 2 + 0];
                    AhMPs[r] += A * b[B_HM] * surf[w * 4 + f * 2 + 1];
                }
            /* interzone exchange with the linked rooms' air of level n */
            for (int32_t i = 0; i < 4 * R; ++i) rs0[i] = s->room[i];
            room_links(p, rs0, lk);
            for (int32_t r = 0; r < R; ++r) room_step(p, r, t, s->room + r * 4, AhT, AhM, AhTTs, AhMPs, lk + r * 3);
        }

        s->step = n + 1;
        if (sample_every > 0 && (it + 1) % sample_every == 0) {
            int64_t k = (it + 1) / sample_every - 1;
            if (samples != NULL)
                for (int32_t w = 0; w < W; ++w) {
                    double *o = samples + ((size_t)k * W + w) * 4;
                    o[0] = s->T_cur[node_off[w]];
                    o[1] = s->P_cur[node_off[w]];
                    o[2] = s->T_cur[node_off[w] + p->n_nodes[w] - 1];
                    o[3] = s->P_cur[node_off[w] + p->n_nodes[w] - 1];
                }
            if (room_samples != NULL)
                for (int32_t r = 0; r < R; ++r) {
                    room_samples[((size_t)k * R + r) * 2 + 0] = s->room[r * 4 + 1];
                    room_samples[((size_t)k * R + r) * 2 + 1] = s->room[r * 4 + 3];
                }
        }
        if (last && flux_last != NULL) memcpy(flux_last, flux, sizeof(double) * (size_t)W * 4);
    }
    free(node_off);
    free(layer_off);
    free(surf);
    free(rsum);
    free(flux);
    free(qrad);
    free(lk);
    free(rs0);
    return rc;
}
