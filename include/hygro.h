/*
 * hygro: GB300 (sm_103a) library for the Dufort-Frankel (DF) explicit update
 * of coupled heat and moisture transfer in porous building walls, after
 * Gasparin, Berger, Dutykh & Mendes, "An improved explicit scheme for
 * whole-building hygrothermal simulation" (arXiv:1703.10119).
 *
 * Problem (paper Sec. 2, [eq:HAM_equation2]): on each wall x in [0, L],
 *     cM  dPv/dt            = d/dx( kM  dPv/dx )
 *     cTT dT/dt + cTM dPv/dt = d/dx( kTT dT/dx + kTM dPv/dx )
 * with coefficients re-evaluated at every step from the vapour pressure
 * (affine form per layer, Psat = desc.Psat):
 *     kM = kM0 (1 + a Pv/Psat), cM = cM0 (1 + b Pv/Psat),
 *     kTT = kTT0 (1 + aT Pv/Psat), cTT = cTT0 (1 + bT Pv/Psat),
 *     kTM = Lv kM, cTM = chi cM,
 * Robin exchanges at both faces ([eq:HAM_BC]; fluxes positive INTO the wall)
 *     g = hM (Pv_inf - Pv_s) + g_inf
 *     q = hT (T_inf - T_s) + Lv hM (Pv_inf - Pv_s) + q_inf
 * and a uniform initial state ([eq:HAM_ic]).
 *
 * Discretisation (Sec. 3.1 [eq:DF_NL], Appendix A [eq:DF_eq1], [eq:DF_eq2],
 * [eq:ghost_node_v0], [eq:ghost_node_u0]): N uniform nodes per wall
 * (node 0 at x = 0 = face 0, node N-1 at x = L = face 1, dx = L/(N-1)),
 * three time levels; level n+1 follows from levels n and n-1 with the
 * coefficients taken at level n, face values = arithmetic mean of the two
 * nodes inside a layer and harmonic mean across a layer interface, the
 * diagonal u_j^n replaced by (u_j^{n+1} + u_j^{n-1})/2, Pv advanced before
 * T, surface nodes as half cells (the ghost-node form of Appendix A). The
 * first step uses level -1 := level 0.
 *
 * Conventions of every call:
 *   - returns a hygro_status and never throws across the ABI;
 *   - validates its arguments before changing any state: a call that fails
 *     with HYGRO_E_INVALID leaves the context as it was;
 *   - inputs are copied (the caller keeps ownership of its arrays);
 *   - output pointers may be host or device memory (device memory is
 *     recognised with cudaPointerGetAttributes); with device outputs the
 *     call is stream-ordered on the context's stream and returns after
 *     enqueueing, with host outputs it returns when the data are there;
 *   - what the set-up calls copied in is in place before the next run's
 *     kernels start, on any stream: on a non-blocking context stream, a
 *     call that launches work first waits for the copies (not while the
 *     stream is being captured into a graph);
 *   - calls on one context are not thread-safe; separate contexts are;
 *   - hygro_last_error gives a readable message for the last failure.
 * Walls are concatenated: the nodes of wall w occupy
 * [node_offset(w), node_offset(w) + n_nodes[w]) in field arrays, with
 * node_offset(w) = n_nodes[0] + ... + n_nodes[w-1].
 */
#ifndef HYGRO_H
#define HYGRO_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HYGRO_API __attribute__((visibility("default")))
#else
#define HYGRO_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hygro_ctx hygro_ctx;   /* opaque, owned by the library */

typedef enum {
    HYGRO_OK = 0,
    HYGRO_E_INVALID = -1,      /* bad argument; nothing changed */
    HYGRO_E_NOMEM = -2,        /* host or device allocation failed */
    HYGRO_E_CUDA = -3,         /* a CUDA call failed (message in hygro_last_error) */
    HYGRO_E_STATE = -4,        /* call out of order (e.g. run before set_materials / set_bc) */
    HYGRO_E_NONFINITE = -5,    /* a wall produced a NaN or infinity */
    HYGRO_E_TIMEOUT = -6,      /* a bounded device wait gave up */
    HYGRO_E_UNSUPPORTED = -7   /* valid request the library does not handle (e.g. N too large) */
} hygro_status;

/* Fault injection for tests of the caller's error handling: with the environment variable
 * HYGRO_FAULT=<entry point>:<n> (e.g. "hygro_run:3"), the n-th call of that entry point in the process,
 * counted from 1, returns HYGRO_E_CUDA with an "injected fault" message before it changes anything or
 * touches the device. The variable is read at the first call of any entry point; without it nothing
 * is injected. hygro_get_step, hygro_last_error and hygro_destroy have no fault point. */

enum { HYGRO_FP32 = 0, HYGRO_FP64 = 1 };

/* How hygro_run advances the walls.
 * PERSISTENT: one launch per hygro_run; each wall is owned by one warp that
 *   keeps its two time levels in registers for the whole time loop (walls of
 *   3..512 nodes).
 * PLAIN: one thread per node, one launch per step, levels in global memory
 *   (any N >= 3); the straightforward GPU form of the scheme. */
enum { HYGRO_KERNEL_PERSISTENT = 0, HYGRO_KERNEL_PLAIN = 1 };

enum { HYGRO_BC_AMBIENT = 0, HYGRO_BC_ADIABATIC = 1, HYGRO_BC_ROOM = 2 };

/* Largest wall the persistent kernel accepts (32 lanes x 16 nodes). */
#define HYGRO_PERSISTENT_MAX_NODES 512
/* Largest number of layers in one wall. */
#define HYGRO_MAX_LAYERS 8

typedef struct {
    int32_t n_walls;           /* >= 1 */
    const int32_t *n_nodes;    /* [n_walls], each >= 3 (copied) */
    const double *thickness;   /* [n_walls] metres, > 0 (copied) */
    double dt;                 /* time step, seconds, > 0 */
    double t0;                 /* time of level 0, seconds */
    double Lv;                 /* latent heat of evaporation, J/kg */
    double Psat;               /* saturation pressure of the coefficient laws, Pa, > 0 */
    int32_t precision;         /* HYGRO_FP32 or HYGRO_FP64 */
    int32_t kernel;            /* HYGRO_KERNEL_PERSISTENT or HYGRO_KERNEL_PLAIN */
    int32_t device;            /* CUDA device ordinal */
    void *stream;              /* cudaStream_t to run on, or NULL for the default stream */
} hygro_desc;

/* One material layer (paper Sec. 2 coefficient definitions, affine in Pv). */
typedef struct {
    double kM0, a;             /* moisture permeability kM0 (s) and its Pv slope */
    double cM0, b;             /* moisture storage cM0 (s^2/m^2) and its Pv slope */
    double kTT0, aT;           /* thermal conductivity (W/m/K) and its Pv slope */
    double cTT0, bT;           /* volumetric heat capacity (J/m^3/K) and its Pv slope */
    double chi;                /* cTM = chi * cM (J/kg/K) */
} hygro_layer;

/* One face of one wall ([eq:HAM_BC]). For HYGRO_BC_AMBIENT the air state is
 *   T_inf(t)  = T_mean + T_amp sin(2 pi t/period + phase_T) + noise_T(t)
 *   Pv_inf(t) = P_mean + P_amp sin(2 pi t/period_P + phase_P) + noise_P(t)
 * (the T sinusoid is dropped when period <= 0; period_P <= 0 means period_P = period, and the Pv
 * sinusoid is dropped when that is <= 0), noise(t) being the linear interpolation at t/noise_dt of the
 * table noise[k][2] = (T, Pv), k = 0 .. noise_len-1, held at its end values outside it. HYGRO_BC_ROOM
 * faces see the air of room `room` at level n (paper Sec. 5.2 [eq:wbse_tn_exp]).
 * HYGRO_BC_ADIABATIC faces exchange nothing. */
typedef struct {
    int32_t kind;
    int32_t room;
    double hT, hM;             /* W/m^2/K, s/m */
    double q_inf, g_inf;       /* extra heat (W/m^2) and moisture (kg/m^2/s) fluxes into the wall */
    double T_mean, T_amp, P_mean, P_amp, period, phase_T, phase_P;
    const float *noise;        /* host (pageable or page-locked) or device memory, [noise_len][2], or NULL (copied) */
    int32_t noise_len;
    double noise_dt;
    double period_P;           /* period of the Pv sinusoid, s (<= 0: period) */
} hygro_bc;

/* One room: a perfectly mixed air zone (paper Sec. 5.1, [eq:LAV_equation], [eq:LAV_couplage]).
 * Air state Ta (K) and Pva (Pa), humidity ratio w = Pva / Pv_ref. Per step, with the wall surface
 * values Ts, Pvs of the room's walls at level n (explicit coupling, Sec. 5.2 [eq:wbse_tn_exp]):
 *   rho V / Pv_ref dPva/dt = g(t) + gv (w_out - w) + sum_walls A hM (Pvs - Pva)
 *   rho V (cp_a + cp_v w) dTa/dt = Q_gain + Lv g(t) + gv cp_a (T_out - Ta) + Lv gv (w_out - w)
 *                                  + sum_walls A [hT (Ts - Ta) + Lv hM (Pvs - Pva)]
 * gv = rho V ach / 3600 (kg/s), outdoor air T_out, Pv_out as the ambient sinusoids of hygro_bc
 * (no noise). The vapour production g(t) = g_vap, plus g_pulse while pulse_on <= (t mod pulse_period)
 * < pulse_off (no pulse when pulse_period <= 0): the occupants' load of Sec. 5.1, whose latent heat
 * Q_o = Lv g enters the heat balance. Each room equation is advanced as one more DF node (its own value
 * at level n replaced by the mean of levels n+1 and n-1; the heat capacity at level n), vapour first. */
typedef struct {
    double volume, ach, Q_gain, g_vap;   /* m^3, 1/h, W, kg/s */
    double T_out_mean, T_out_amp, P_out_mean, P_out_amp, period, phase_T, phase_P;
    double rho_a, cp_a, cp_v, Pv_ref;    /* kg/m^3, J/kg/K, J/kg/K, Pa */
    double Ta0, Pa0;                     /* initial air state (both stored levels) */
    double period_P;                     /* period of the outdoor Pv sinusoid, s (<= 0: period) */
    double g_pulse, pulse_on, pulse_off, pulse_period;   /* kg/s, s, s, s */
} hygro_room;

/* Most walls one room may have (each wall has at most one face on a room). */
#define HYGRO_MAX_ROOM_WALLS 8

/* Options of a context (hygro_set_option). */
enum { HYGRO_OPT_ROOM_SCHEME = 1 };
/* HYGRO_OPT_ROOM_SCHEME values: how each room air node is advanced.
 * HYGRO_ROOM_DF (default): one more DF node (its own level-n value in its balance replaced by the mean
 *   of levels n+1 and n-1), explicit in the wall surface values; stable at the whole-building time steps.
 * HYGRO_ROOM_EULER: the explicit Euler update of paper Sec. 5.2 (every term at level n); unstable when
 *   dt exceeds twice the room's time constant (heat capacity over total exchange conductance). */
enum { HYGRO_ROOM_DF = 0, HYGRO_ROOM_EULER = 1 };

/* Create a context on desc->device. *out receives the context. */
HYGRO_API hygro_status hygro_create(const hygro_desc *desc, hygro_ctx **out);

/* Layer map, materials and uniform initial state ([eq:HAM_ic]).
 *   n_layers[w] in 1..HYGRO_MAX_LAYERS; the layers of wall w are the next
 *   n_layers[w] entries of layer_first / layers; layer_first holds the first
 *   node of each layer (0 for the first layer, strictly increasing, < N).
 * Resets both stored levels to (T_init[w], P_init[w]) and the step to 0.
 * All arrays are host memory. */
HYGRO_API hygro_status hygro_set_materials(hygro_ctx *ctx, const int32_t *n_layers, const int32_t *layer_first,
                                 const hygro_layer *layers, const double *T_init, const double *P_init);

/* Boundary description of one face (0: x = 0, 1: x = L) for every wall;
 * bc[w] for w in 0..n_walls-1, host memory. The noise tables of the ambient faces are copied to the
 * device during the call (the caller's tables may be freed afterwards); each value is checked on the
 * way. A non-finite value gives HYGRO_E_INVALID naming the wall, as does any other invalid field, and
 * a refused call leaves the face's previous description and tables in place. Setting one face does not
 * copy the other face's tables again, nor does hygro_set_materials. The copy uses up to 8 host threads
 * and two host staging chunks of up to 64 MB each (pinned when the allocation succeeds), which the
 * context keeps for its next uploads; the call returns when the tables are on the device. When every run
 * of tables adjacent in memory starts in page-locked host memory (cudaHostAlloc, cudaHostRegister) or in
 * device memory, the tables skip the host threads: one DMA copy per run lands them in the device staging
 * area, and a device kernel checks their values before they replace the face's tables. */
HYGRO_API hygro_status hygro_set_bc(hygro_ctx *ctx, int32_t face, const hygro_bc *bc);

/* Rooms of the whole-building model: rooms[r] for r in 0..n_rooms-1, wall_area[w] (m^2) the area
 * of wall w seen by the room its HYGRO_BC_ROOM face points at (host memory, copied). Resets the room
 * air to (Ta0, Pa0). Rooms need the persistent kernel. */
HYGRO_API hygro_status hygro_set_rooms(hygro_ctx *ctx, int32_t n_rooms, const hygro_room *rooms,
                                       const double *wall_area);

/* Long-wave radiation among the wall surfaces of each room (paper Sec. 2: q_rw, the heat a room face
 * receives, = s eps sigma sum over the room's faces of (T'^4 - Ts^4), sigma the Stefan-Boltzmann constant).
 * emissivity[w][f] (host, [n_walls][2], in [0, 1]) applies to room faces; view[r] (host, [n_rooms], in
 * [0, 1]) is the view factor s of room r. Each term is taken as h' (T' - Ts) with the conductance
 * h' = s eps sigma (T'^2 + Ts^2)(T' + Ts) (an exact factorisation): h' and the other faces' T' of level n,
 * the face's own Ts averaged over levels n+1 and n-1 as for the convective exchange (the level-n form of
 * the face's own term is unstable in DF). Radiating faces run the general code variant. Both arrays are
 * copied. HYGRO_E_INVALID for a NULL array or a value outside [0, 1] (NaN included); HYGRO_E_STATE before
 * hygro_set_rooms, which clears the radiation. */
HYGRO_API hygro_status hygro_set_radiation(hygro_ctx *ctx, const double *emissivity, const double *view);

/* Interzone airflow (paper Sec. 5.1: Q_inz = g (cpa (T_j - T_i)) + Lv g (w_j - w_i), G_inz = g (w_j - w_i) in
 * both rooms of a link; the paper writes cw for the air's heat capacity, read as the room's cp_a).
 * zones[l] (host, [n_links][2]) two different rooms, flow[l] >= 0 kg/s of air exchanged both ways. A room's
 * own values enter as the mean of levels n+1 and n-1 (the room node's DF form), the linked room's as level
 * n. Both arrays are copied; n_links = 0 removes every link. Rooms linked together run in one block: a
 * linked group holds at most 4 rooms and 3 links per room, and its walls plus one air warp per room fill
 * at most 16 warps (hygro_run reports HYGRO_E_STATE otherwise). HYGRO_E_INVALID for n_links < 0, a NULL
 * array with links, a link between a room and itself or to a room that does not exist, or a negative or
 * non-finite flow; HYGRO_E_STATE before hygro_set_rooms, which clears the links. */
HYGRO_API hygro_status hygro_set_interzone(hygro_ctx *ctx, int32_t n_links, const int32_t *zones, const double *flow);

/* Set an option (HYGRO_OPT_*) of the context; it applies from the next run. */
HYGRO_API hygro_status hygro_set_option(hygro_ctx *ctx, int32_t option, int64_t value);

/* Share of the moisture permeability that carries latent heat, per wall: the cross conductivity of
 * the heat equation is kTM = nu Lv kM at the faces inside the wall (paper Sec. 2: kTM = Lv delta_v with
 * delta_v the vapour part of kM), while the surface exchange keeps Lv hM ([eq:HAM_BC]). nu[w] >= 0,
 * finite; the default is 1 (kTM = Lv kM). nu (host memory, [n_walls]) is copied; it may be set at any
 * time and applies from the next step. The adjoint (hygro_loss_grad) supports nu = 1 only. */
HYGRO_API hygro_status hygro_set_vapour_fraction(hygro_ctx *ctx, const double *nu);

/* Coefficient law of each layer (paper Sec. 4, Table 1: the load bearing material whose coefficients
 * depend on T and Pv). law[l] for every layer l of hygro_set_materials' order (host memory, copied):
 *   HYGRO_LAW_AFFINE    the affine laws of the layer's hygro_layer parameters (the default);
 *   HYGRO_LAW_TABLE1    Table 1: the sorption isotherm f through the Kelvin relation (natural logarithm),
 *                       cM = df/dPv, lambda, the vapour permeability dv, kTM = Lv dv, cTT = rho0 c0 + cw f,
 *                       cTM = cw (T - 273.15) cM, the saturation pressure of the Magnus form (Alduchov &
 *                       Eskridge 1996; the paper gives none), the capillary pressure held at 0 above
 *                       saturation; kM's liquid term read as (exp(-8x-2))^2, x = 2 Pv / Ps;
 *   HYGRO_LAW_TABLE1_A  the same with the liquid term read as exp((-8x-2)^2) (overflows in FP32);
 *   HYGRO_LAW_TABLE1_C  the same with the liquid term read as exp(-8 (x-2)^2).
 * The coefficients of a Table-1 layer come from each node's absolute T and Pv of level n (explicit, as
 * Sec. 3.1 prescribes); faces take the arithmetic mean inside a layer and the harmonic mean across layers,
 * kTM included. The hygro_layer parameters of a Table-1 layer are not used. hygro_set_materials resets
 * every layer to HYGRO_LAW_AFFINE. Walls with a Table-1 layer run on the plain kernel only: hygro_run of a
 * context of the persistent kernel, a wall facing a room and hygro_loss_grad refuse them with
 * HYGRO_E_UNSUPPORTED. HYGRO_E_INVALID for an unknown law; HYGRO_E_STATE before hygro_set_materials. */
#define HYGRO_LAW_AFFINE 0
#define HYGRO_LAW_TABLE1 1
#define HYGRO_LAW_TABLE1_A 2
#define HYGRO_LAW_TABLE1_C 3
HYGRO_API hygro_status hygro_set_layer_law(hygro_ctx *ctx, const int32_t *law);

/* Room air state of level 0 (n) or 1 (n-1): Ta[n_rooms], Pa[n_rooms] (host or device memory). */
HYGRO_API hygro_status hygro_get_rooms(hygro_ctx *ctx, int32_t level, double *Ta, double *Pa);

/* Advance n_steps DF steps (n_steps >= 0).
 * samples: NULL, or [n_steps / sample_every][n_walls][2 faces][2] of float
 *   (FP32 contexts) or double (FP64 contexts) receiving the surface (T, Pv)
 *   at level n+1 after every sample_every-th step of this call;
 *   samples_bytes must cover it. */
HYGRO_API hygro_status hygro_run(hygro_ctx *ctx, int64_t n_steps, int32_t sample_every, void *samples,
                       size_t samples_bytes);

/* Start option: the first step by explicit Euler substeps instead of the DF step with level -1 := level 0
 * (DF is stated for n >= 1; the paper's explicit scheme is bounded by the stability condition it gives).
 * Level 1 follows from level 0 by m explicit Euler substeps of dt / m per wall, the coefficients
 * re-evaluated at every substep, Pv first and T with the substep's Pv change in the cTM storage term, the
 * ambient air at each substep's time; m = ceil(dt / tau_max), tau_max = the wall's explicit stability
 * bound at level 0 (min over nodes and both fields of w dx c / (sum of face conductances + h)). The flux
 * sums receive dt / m times every substep's surface fluxes. Requires the context at step 0 (right after
 * hygro_set_materials / hygro_set_fields); afterwards the step is 1 and the stored levels are (0, 1), and
 * hygro_run continues with DF. A wall needing more than 2^24 substeps makes the call fail with
 * HYGRO_E_UNSUPPORTED and no state changed. Walls with a room face: HYGRO_E_UNSUPPORTED. Synchronous. */
HYGRO_API hygro_status hygro_start_euler(hygro_ctx *ctx);

/* Wait for the context's stream; HYGRO_E_NONFINITE if any wall went
 * non-finite in the runs since the last check. */
HYGRO_API hygro_status hygro_sync(hygro_ctx *ctx);

/* Surface fluxes into the wall of the last step, [n_walls][2 faces][2]
 * (heat W/m^2, moisture kg/m^2/s), and their running sums over all steps
 * of dt * flux (J/m^2, kg/m^2), accumulated in FP64. Either may be NULL. */
HYGRO_API hygro_status hygro_fluxes(hygro_ctx *ctx, double *flux, double *cumulative);

/* Discrete balance of the next step n -> n+1, computed from the stored levels without advancing them
 * (the step, the levels and the flux sums are left as they were). Per wall and field (0: T, 1: Pv):
 * bal[w][f][0] storage S = sum_j w_j dx (c (u^{n+1} - u^{n-1}) [+ cTM (Pv^{n+1} - Pv^{n-1}) for T]) / (2 dt),
 * bal[w][f][1] boundary B = the surface fluxes into the wall with the time-averaged surface values,
 * bal[w][f][2] DF defect D = sum over interior faces of (k_f/dx)((u_{j+1}^n - ubar_{j+1}) + (u_j^n - ubar_j))
 *              (plus the kTM terms for T), ubar = (u^{n+1} + u^{n-1}) / 2,
 * bal[w][f][3] M = the sum of the magnitudes of every term.
 * The scheme satisfies S = B + D exactly in exact arithmetic ([eq:DF_NL] summed over the nodes; D is the
 * O(dt^2) conservation defect of DF). Sums in FP64; bal is [n_walls][2][4], host or device memory. Walls
 * with a room face are not supported (HYGRO_E_UNSUPPORTED). */
HYGRO_API hygro_status hygro_balance(hygro_ctx *ctx, double *bal);

/* Stored levels as absolute values in FP64: level 0 is the newest (n),
 * level 1 the previous (n-1). T and P hold sum(n_nodes) values each. */
HYGRO_API hygro_status hygro_get_fields(hygro_ctx *ctx, int32_t level, double *T, double *P);

/* Overwrite one stored level (absolute values, host or device memory). */
HYGRO_API hygro_status hygro_set_fields(hygro_ctx *ctx, int32_t level, const double *T, const double *P);

/* Index n of the newest stored level. */
HYGRO_API hygro_status hygro_get_step(const hygro_ctx *ctx, int64_t *step);

/* Checkpoint of the whole evolving state (levels, step, flux sums, room
 * air). With buf == NULL, *bytes receives the size; otherwise *bytes must
 * be at least that size. Restoring with hygro_set_state into a context
 * created with the same description, materials and boundaries continues
 * the run bit for bit. Host memory. */
HYGRO_API hygro_status hygro_get_state(hygro_ctx *ctx, void *buf, size_t *bytes);
HYGRO_API hygro_status hygro_set_state(hygro_ctx *ctx, const void *buf, size_t bytes);

/* Autotuner of the persistent kernel's wall schedule (the walls each block runs, dealt by the
 * longest-processing-time rule with a step-time model a + b K per code variant). From the current
 * state it runs probe_steps steps (16 .. 2^20) with every wall's start and end recorded on the GPU
 * clock, fits the model to the walls' measured time per step (least squares per variant), then times
 * the same probe with the current schedule and with the schedule of the refitted model (CUDA events)
 * and keeps the faster one. The stored levels, step and flux sums are restored afterwards; results of
 * later runs do not depend on the schedule. model[0..3] = a, model[4..7] = b of the fitted model
 * (nanoseconds; may be NULL); ms[0], ms[1] = probe time with the previous and the refitted schedule (may
 * be NULL). Walls facing rooms run in the room kernel and are not scheduled: HYGRO_E_UNSUPPORTED for a
 * context with rooms or with the plain kernel. Synchronous. The paper has no counterpart: the schedule
 * changes where the walls run, not what the scheme computes. */
HYGRO_API hygro_status hygro_autotune(hygro_ctx *ctx, int32_t probe_steps, double *model, double *ms);

/* Size of the fixed device array behind hygro_run_noalloc: 8 MiB. */
#define HYGRO_NOALLOC_SCRATCH_BYTES (8u << 20)

/* hygro_run for callers that cannot allocate device memory when they call it: a process whose device
 * memory is held by its own pool allocator (PyTorch's caching allocator, for instance), where a
 * direct cudaMalloc can fail or split the pool, or a time-critical loop that must not allocate.
 * Same arguments, results and stream ordering as hygro_run; it calls no cudaMalloc, cudaFree or
 * allocating library routine. Where hygro_run stages samples bound for host memory in a buffer it
 * allocates, this call stages them in a fixed array of HYGRO_NOALLOC_SCRATCH_BYTES that the library
 * keeps in global memory on every GPU that loads it, until the process exits; a call whose samples
 * need more returns HYGRO_E_UNSUPPORTED and changes nothing. The first call on a device looks up the
 * array's device address with that device current; make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents (each call overwrites in full what
 * it stages, so nothing needs clearing); calls whose GPU work overlaps (other threads, streams or
 * contexts) race on it. The paper has no counterpart to this entry point. */
HYGRO_API hygro_status hygro_run_noalloc(hygro_ctx *ctx, int64_t n_steps, int32_t sample_every, void *samples,
                                         size_t samples_bytes);

/* Sensor misfit of a run and its gradient with respect to the material parameters, by the reverse-time
 * adjoint of the DF step (the paper has no adjoint; this differentiates the scheme described above).
 * The run starts from the uniform initial state given to hygro_set_materials (level -1 := level 0) at t0
 * and lasts n_steps; the context's stored levels, step and flux sums are left as they were.
 *   loss = sum over samples k (after every sample_every-th step, k = 0 .. n_steps / sample_every - 1),
 *          walls w and faces f of  wT (T_f - obs[k][w][f][0])^2 + wP (Pv_f - obs[k][w][f][1])^2,
 *   T_f, Pv_f the surface node values (node 0 for face 0, node N-1 for face 1); obs holds absolute values,
 *   float, host or device memory, [n_steps / sample_every][n_walls][2][2].
 * *loss (host) receives the loss, accumulated in FP64. grad (host or device memory, or NULL) receives
 * dloss/dtheta, [total layers][9] in the order of hygro_layer (kM0, a, cM0, b, kTT0, aT, cTT0, bT, chi),
 * accumulated in FP64. The forward saves (level n-1, level n) every checkpoint_every steps (0: about
 * sqrt(n_steps)), and the reverse recomputes each stretch from its checkpoint. With checkpoint_every >=
 * n_steps the forward keeps every level instead and nothing is recomputed (faster, at about
 * walls x 2 x (n_steps + 2) x 32 x slots-per-lane reals of device memory). Device memory for the
 * checkpoints and the stretch levels is allocated by the call, per wall about (checkpoints x 4 +
 * (stride + 2) x 2) x 32 x slots-per-lane reals (slots per lane: the longest lane run of the wall,
 * about N / 32); HYGRO_E_NOMEM if it does not fit.
 * Walls with a room face are not supported (HYGRO_E_UNSUPPORTED). The arithmetic runs in the context's
 * precision. */
HYGRO_API hygro_status hygro_loss_grad(hygro_ctx *ctx, int64_t n_steps, int32_t sample_every, const float *obs,
                                       double wT, double wP, int32_t checkpoint_every, double *loss, double *grad);

/* Message of the last failed call on ctx (or of the last failed
 * hygro_create when ctx is NULL). Never NULL. */
HYGRO_API const char *hygro_last_error(const hygro_ctx *ctx);

/* Release everything the context owns. NULL is accepted. */
HYGRO_API void hygro_destroy(hygro_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* HYGRO_H */
