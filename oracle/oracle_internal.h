/*
 * Internal helpers shared by the oracle's translation units (hygro_oracle.c and the CPU comparator
 * schemes in hygro_comparators.c). TEST INFRASTRUCTURE ONLY, like the rest of the oracle.
 */
#ifndef HYGRO_ORACLE_INTERNAL_H
#define HYGRO_ORACLE_INTERNAL_H

#include "hygro_oracle.h"

enum { L_KM0, L_A, L_CM0, L_B, L_KTT0, L_AT, L_CTT0, L_BT, L_CHI };
enum { B_HT, B_HM, B_QINF, B_GINF, B_TMEAN, B_TAMP, B_PMEAN, B_PAMP, B_PERIOD, B_PHT, B_PHP, B_NDT, B_PERIODP };
enum { R_VOL, R_ACH, R_QGAIN, R_GVAP, R_TMEAN, R_TAMP, R_PMEAN, R_PAMP, R_PERIOD, R_PHT, R_PHP,
       R_RHOA, R_CPA, R_CPV, R_PVREF, R_SCHEME, R_PERIODP, R_GPULSE, R_PON, R_POFF, R_PPER };

static const double TWO_PI = 6.283185307179586476925286766559;

typedef struct {
    int32_t N;
    double dx;
    int32_t nl;
    const int32_t *first;
    const double *par;
    const int32_t *law;    /* coefficient law of each layer (NULL: all affine) */
    double nu;             /* kTM = nu Lv kM */
} wall_view;

wall_view view_of(const orc_problem *p, const int64_t *layer_off, int32_t w);

/* Node coefficients at (T, P) of one level and their face values (see hygro_oracle.c). */
void coefficients(const orc_problem *p, const wall_view *v, const double *T, const double *P,
                  double *kM, double *cM, double *kTT, double *cTT, double *kTM, double *cTM,
                  double *kMf, double *kTTf, double *kTMf);

/* Surface exchange data of one face for this step: the air state and the
 * coefficients of [eq:HAM_BC]. An adiabatic face exchanges nothing. */
typedef struct {
    double hT, hM, q_inf, g_inf, T_inf, P_inf;
    /* long-wave exchange with the other surfaces of a room (zero elsewhere): the face receives
     * qR - hR Ts, the coefficient hR and the emission qR of level n */
    double hR, qR;
} face_bc;

face_bc face_of(const orc_problem *p, int32_t w, int32_t f, double t, const double *room_state);

/* Long-wave exchange q_rw (Sec. 2) of every room face at the surface temperatures surf ([n_walls][2 faces]
 * [T, Pv]) of level n, in the form qR - hR Ts of faces to the room's other surfaces: rad[w][f][0] = hR = sum
 * of the radiative conductances h' = s eps sigma (T'^2 + Ts^2)(T' + Ts) and rad[w][f][1] = qR = sum h' T';
 * zero on other faces. */
void room_radiation(const orc_problem *p, const double *surf, double *rad);

/* Interzone exchange of every room with the air of the rooms it is linked to, at the room states rs
 * ([n_rooms][Ta_prev, Ta, Pa_prev, Pa]): per room the total link flow G (kg/s) and the sums G T_o, G w_o of
 * the linked rooms' level values (w = Pa / Pv_ref); lk[r][3]. */
void room_links(const orc_problem *p, const double *rs, double *lk);

/* Outdoor air and vapour production of room r at time t (Sec. 5.1). */
void room_sources(const orc_problem *p, int32_t r, double t, double *T_out, double *P_out, double *g_vap);

#endif
