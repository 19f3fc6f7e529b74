/*
 * FP64 CPU oracle for the Dufort-Frankel (DF) hygrothermal wall update of
 * Gasparin, Berger, Dutykh & Mendes, "An improved explicit scheme for
 * whole-building hygrothermal simulation" (arXiv:1703.10119).
 *
 * TEST INFRASTRUCTURE ONLY. This code is the plain, slow, obviously correct
 * statement of what the CUDA library computes. Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark load it; the CUDA
 * library neither links nor calls it, and the two share no source.
 *
 * What it follows (paper sections / equations, LaTeX labels in brackets):
 *   - the coupled moisture (Pv) and heat (T) equations [eq:HAM_equation2],
 *     with coefficients kM, cM, kTT, cTT, kTM, cTM (Sec. 2) taken in the
 *     affine form kM = kM0 (1 + a Pv/Psat), cM = cM0 (1 + b Pv/Psat),
 *     kTT = kTT0 (1 + aT Pv/Psat), cTT = cTT0 (1 + bT Pv/Psat),
 *     kTM = nu Lv kM (nu = 1 unless a wall's vapour fraction says otherwise:
 *     Sec. 2 defines kTM = Lv delta_v with delta_v the vapour part of kM), cTM = chi cM;
 *   - Robin surface exchanges [eq:HAM_BC] (fluxes counted positive INTO the
 *     wall at both faces), uniform initial state [eq:HAM_ic];
 *   - the nonlinear DF scheme [eq:DF_NL], [eq:DF_NL_RHS]: coefficients
 *     evaluated explicitly at level n, face values from the two adjacent
 *     nodes, u_j^n replaced by (u_j^{n+1} + u_j^{n-1})/2 in the diagonal;
 *   - the coupled order of Appendix A: Pv first [eq:DF_eq1], then T using
 *     Pv^{n+1} [eq:DF_eq2], [eq:DF_eq2b];
 *   - the surface nodes through the ghost-node treatment of Appendix A
 *     [eq:bc_v], [eq:ghost_node_v0], [eq:ghost_node_u0], written in its
 *     equivalent half-cell form (identical algebra, no ghost storage);
 *   - the room air balance of Sec. 5.1 [eq:LAV_equation], [eq:LAV_couplage]
 *     advanced explicitly with the wall surface values at level n as in
 *     [eq:wbse_tn_exp], the room node itself taking the DF form.
 *
 * Layout: walls are concatenated; the nodes of wall w are
 * node_offset[w] .. node_offset[w] + n_nodes[w] - 1, node 0 at x = 0 (face 0),
 * node N-1 at x = L (face 1), dx = L / (N - 1).
 */
#ifndef HYGRO_ORACLE_H
#define HYGRO_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_NLAYER_PAR 9   /* kM0, a, cM0, b, kTT0, aT, cTT0, bT, chi */
#define ORC_NBC_PAR 13     /* hT, hM, q_inf, g_inf, T_mean, T_amp, P_mean, P_amp, period, phase_T, phase_P, noise_dt,
                              period_P (period of the Pv sinusoid; <= 0: period) */
#define ORC_NROOM_PAR 21   /* volume, ach, Q_gain, g_vap, T_out_mean, T_out_amp, P_out_mean, P_out_amp,
                              period, phase_T, phase_P, rho_a, cp_a, cp_v, Pv_ref, scheme (0: the room
                              as one more DF node, 1: the explicit Euler update of Sec. 5.2), period_P
                              (outdoor Pv; <= 0: period), g_pulse, pulse_on, pulse_off, pulse_period (the
                              vapour production is g_vap + g_pulse while pulse_on <= t mod pulse_period
                              < pulse_off; no pulse when pulse_period <= 0) */

enum { ORC_BC_AMBIENT = 0, ORC_BC_ADIABATIC = 1, ORC_BC_ROOM = 2 };

/* Coefficient law of a layer. ORC_LAW_AFFINE: the affine laws above (layer_par). The others: the load
 * bearing material of Sec. 4 (Table 1), whose coefficients depend on T and Pv, layer_par unused:
 *   Ps(T) = 610.94 exp(17.625 theta / (theta + 243.04)) Pa, theta = T - 273.15 (the paper gives no
 *           saturation pressure; this is the Magnus form of Alduchov & Eskridge, 1996);
 *   Pc = rho_l Rv T ln(Pv / Ps) (Kelvin relation, Sec. 2), rho_l = 1000 kg/m3, Rv = 461.5 J/(kg K),
 *        held at 0 (saturation) for Pv > Ps, where the isotherm has no values;
 *   f = 47.1 [1 + (-c1 Pc)^1.65]^-0.39 + 109.9 [1 + (-c2 Pc)^6]^-0.83 kg/m3, c1 = 1.25e-5, c2 = 1.8e-5;
 *   cM = df/dPv (through the Kelvin relation with ln), dv = 1.88e-6 / T (1 - f/157) / (0.503 (1 -
 *   f/157)^2 + 0.497), kTT = 0.2 + 0.0045 f, cTT = rho0 c0 + f cw (rho0 = 790, c0 = 870, cw = 4180),
 *   kTM = Lv dv, cTM = cw theta cM (theta in degrees Celsius);
 *   kM = 1.97e-10 exp(-0.07 log10(x) + 1.44) + 1.77e-7 L(x), x = 2 Pv / Ps, with the liquid term L read
 *   from Table 1's garbled bracket as (exp(-8 x - 2))^2 (ORC_LAW_TABLE1), exp((-8 x - 2)^2)
 *   (ORC_LAW_TABLE1_A) or exp(-8 (x - 2)^2) (ORC_LAW_TABLE1_C). */
enum { ORC_LAW_AFFINE = 0, ORC_LAW_TABLE1 = 1, ORC_LAW_TABLE1_A = 2, ORC_LAW_TABLE1_C = 3 };

/* The six coefficients (kM, cM, kTT, cTT, kTM, cTM) of a Table-1 law at (T [K], Pv [Pa]), out[6];
 * also the saturation pressure and the sorption isotherm f (kg/m3) through ps / fw when not NULL. */
void orc_table1(int32_t law, double T, double Pv, double Lv, double *out, double *ps, double *fw);

typedef struct {
    int32_t n_walls;
    const int32_t *n_nodes;      /* [n_walls], each >= 3 */
    const double *thickness;     /* [n_walls] */
    const int32_t *n_layers;     /* [n_walls], each >= 1 */
    const int32_t *layer_first;  /* [sum n_layers]: first local node of each layer (0 for the first) */
    const double *layer_par;     /* [sum n_layers][ORC_NLAYER_PAR] */
    const int32_t *bc_kind;      /* [n_walls][2] */
    const double *bc_par;        /* [n_walls][2][ORC_NBC_PAR] */
    const int32_t *bc_room;      /* [n_walls][2]: room index of BC_ROOM faces */
    const float *noise[2];       /* per face: [n_walls][noise_len[f]][2] (T, Pv) or NULL */
    int32_t noise_len[2];
    double dt, t0, Lv, Psat;
    int32_t n_rooms;
    const double *room_par;      /* [n_rooms][ORC_NROOM_PAR] */
    const double *wall_area;     /* [n_walls], m^2, used by room faces */
    const double *vapour_frac;   /* [n_walls] nu of kTM = nu Lv kM inside the wall, or NULL (all 1) */
    const int32_t *layer_law;    /* [sum n_layers] ORC_LAW_* of each layer, or NULL (all affine) */
    /* long-wave radiation among a room's wall surfaces (Sec. 2, q_rw): a room face of wall w receives
     * s_r eps_wf sigma sum over the room's faces (Ts'^4 - Ts^4), surface temperatures of level n */
    const double *face_emis;     /* [n_walls][2] emissivity eps of each face (room faces), or NULL (none) */
    const double *room_view;     /* [n_rooms] view factor s of each room, or NULL (none) */
    /* interzone airflow (Sec. 5.1, Q_inz and G_inz): link l carries link_flow[l] kg/s of air between rooms
     * link_zone[2l] and link_zone[2l+1] in both directions */
    int32_t n_links;
    const int32_t *link_zone;    /* [n_links][2] */
    const double *link_flow;     /* [n_links] */
} orc_problem;

#define ORC_SIGMA 5.670374419e-8   /* Stefan-Boltzmann constant, W/(m2 K4) */

typedef struct {
    int64_t step;                /* n: T_cur / P_cur hold level n, T_prev / P_prev level n-1 */
    double *T_prev, *T_cur;      /* [sum n_nodes] */
    double *P_prev, *P_cur;      /* [sum n_nodes] */
    double *cumul;               /* [n_walls][2 faces][2] sum over steps of dt * flux (heat, moisture) */
    double *room;                /* [n_rooms][4]: Ta_prev, Ta_cur, Pa_prev, Pa_cur (may be NULL) */
} orc_state;

/* Advance n_steps DF steps.
 *   samples:      [n_steps / sample_every][n_walls][2 faces][2] surface (T, Pv) at level n+1
 *                 after every sample_every-th step of this call, or NULL
 *   room_samples: [n_steps / sample_every][n_rooms][2] room (Ta, Pva), or NULL
 *   flux_last:    [n_walls][2 faces][2] heat (W/m2) and moisture (kg/m2/s) flux of the last step, or NULL
 *   balance_last: [n_walls][2 fields (T, Pv)][4] storage S, boundary B, DF defect D, scale M of the
 *                 last step (S = B + D in exact arithmetic; M = sum of the magnitudes of all terms), or NULL
 * Returns 0 on success, -1 on invalid arguments, -2 on allocation failure. */
int orc_run(const orc_problem *p, orc_state *s, int64_t n_steps, int32_t sample_every,
            double *samples, double *room_samples, double *flux_last, double *balance_last,
            int32_t n_threads);

/* The first step by explicit Euler substeps instead of DF with level -1 := level 0 (state at step 0, walls
 * without rooms): level 1 from level 0 by m substeps of dt / m, m = ceil(refine * dt / tau_max) with
 * tau_max the explicit stability bound at level 0. Afterwards the step is 1. 0 on success. */
int orc_euler_start(const orc_problem *p, orc_state *s, double refine, int32_t n_threads);

/* The paper's comparison schemes (hygro_comparators.c; Sec. 4, Sec. 5.2), on the DF oracle's spatial
 * operator. Both advance n_steps steps of dt from the state's level n; afterwards T_prev / P_prev hold the
 * level before the last and T_cur / P_cur the last, the room air likewise, and the flux sums grow.
 *
 * Euler implicit with the fixed-point sub-iterations of Alg. 1: each step iterates walls (backward Euler,
 * coefficients at the iterate, room air of the iterate) and rooms (backward Euler with the walls' new surface
 * values) until the largest relative change of any value is below eta; *iterations (if not NULL) grows by the
 * sub-iterations done. The change is the largest relative change of any value (norm 0) or the Euclidean
 * norm of the relative changes of all values (norm 1; the paper does not name its norm). Returns 0, -1
 * (invalid), -2 (allocation), -3 (a step did not converge in max_iter).
 *
 * Euler explicit: each step in m substeps, m = ceil(refine dt / tau) with tau the explicit stability bound of
 * every node and room at the step's start; *substeps (if not NULL) grows by the substeps done. */
int orc_euler_implicit_run(const orc_problem *p, orc_state *s, int64_t n_steps, double eta, int32_t max_iter,
                           int32_t norm, int64_t *iterations, int32_t n_threads);
int orc_euler_explicit_run(const orc_problem *p, orc_state *s, int64_t n_steps, double refine, int64_t *substeps,
                           int32_t n_threads);

/* Ambient air state (T_inf, Pv_inf) seen by an ambient face at time t. */
void orc_ambient(const orc_problem *p, int32_t wall, int32_t face, double t, double *T_inf, double *P_inf);

/* Per-node coefficients (kM, cM, kTT, cTT, kTM, cTM) of wall w at temperatures T[0..N-1] (used by the
 * Table-1 laws only; may be NULL for affine walls) and vapour pressures P[0..N-1], and face values
 * (kM_f, kTT_f, kTM_f) for the N-1 interior faces. */
void orc_coefficients(const orc_problem *p, int32_t wall, const double *T, const double *P,
                      double *node6 /* [N][6] */, double *face3 /* [N-1][3] */);

/* 2D wall sections (hygro_oracle2d.c): G grids of nx x ny nodes, spacing h in x and y. */
typedef struct {
    int32_t n_grids, nx, ny;
    double h;                    /* m */
    const uint8_t *region;       /* [G][ny][nx] material region of every node */
    int32_t n_regions;           /* rows per grid in region_par */
    const double *region_par;    /* [G][n_regions][ORC_NLAYER_PAR] */
    const int32_t *bc_kind;      /* [G][4] faces 0: x = 0, 1: x = Lx, 2: y = 0, 3: y = Ly (ambient or adiabatic) */
    const double *bc_par;        /* [G][4][ORC_NBC_PAR] */
    const float *noise[4];       /* per face: [G][noise_len[f]][2] or NULL */
    int32_t noise_len[4];
    double dt, t0, Lv, Psat;
} orc2d_problem;

typedef struct {
    int64_t step;
    double *T_prev, *T_cur, *P_prev, *P_cur;   /* [G][ny][nx] */
} orc2d_state;

/* Advance n_steps DF steps of every grid (OpenMP over grids). 0 on success. */
int orc2d_run(const orc2d_problem *p, orc2d_state *s, int64_t n_steps, int32_t n_threads);

/* Sensor misfit of the surface values (hygro_adjoint.c): samples after every sample_every-th step,
 * obs[k][w][f] = (T, Pv) observed at face f of wall w after step (k+1) * sample_every. */
typedef struct {
    int32_t sample_every;
    const double *obs;           /* [n_steps / sample_every][n_walls][2][2] */
    double wT, wP;               /* weights of the squared T and Pv mismatches */
    const double *T_init;        /* [n_walls] uniform initial state of each wall */
    const double *P_init;
} orc_misfit;

/* Loss and its gradient dL/d(layer_par) ([sum n_layers][ORC_NLAYER_PAR], or NULL for the loss alone)
 * by the reverse-time adjoint of the DF step. Walls without room faces, kTM = Lv kM. 0 on success. */
int orc_loss_adjoint(const orc_problem *p, int64_t n_steps, const orc_misfit *m, double *loss, double *grad,
                     int32_t n_threads);

/* Loss and its derivative along dir ([sum n_layers][ORC_NLAYER_PAR]) by forward-mode dual numbers. */
int orc_loss_tangent(const orc_problem *p, int64_t n_steps, const orc_misfit *m, const double *dir, double *loss,
                     double *dloss);

#ifdef __cplusplus
}
#endif
#endif
