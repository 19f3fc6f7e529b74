/*
 * hygro2d: the Dufort-Frankel (DF) update of coupled heat and moisture transfer on 2D wall sections
 * (thermal-bridge corners), GB300 (sm_103a). Companion of hygro.h (same status codes, material and
 * face descriptions); the paper solves the 1D problem, and this is its extension to a 5-point stencil.
 *
 * Problem: on each section (x, y) in [0, (nx-1) h] x [0, (ny-1) h] the equations of hygro.h
 * ([eq:HAM_equation2]) with d/dx(k d/dx) replaced by div(k grad), the coefficients affine in Pv per
 * material region, Robin exchanges ([eq:HAM_BC], fluxes positive into the section) or no flux on
 * each of the four faces, a uniform initial state ([eq:HAM_ic]).
 *
 * Discretisation ([eq:DF_NL] in two dimensions): nodes on a uniform grid of spacing h (node (i, j)
 * at x = i h, y = j h). Node (i, j) owns the control area wx wy h^2, with wx = 1/2 for i = 0 or
 * nx - 1 and 1 otherwise (wy likewise in j). Its four faces to the neighbouring nodes have the
 * length of the perpendicular weight times h (wy h for the x-faces, wx h for the y-faces), a face
 * conductivity equal to the arithmetic mean of the two nodes' values inside a region and to the
 * harmonic mean across regions, and a Robin face of the section enters an edge node with its length
 * (wy h on the faces x = const, wx h on y = const; a corner node takes both). Per step, with the
 * coefficients at level n and u^n of the node replaced by (u^{n+1} + u^{n-1})/2:
 *   wx wy h c (u^{n+1} - u^{n-1}) / (2 dt) = sum_faces len k_f (u_nb^n - ubar) / h
 *                                            + sum_Robin len [h_s (u_inf - ubar) + source]
 * Pv first, then T with Pv^{n+1} and the latent term Lv kM; level -1 := level 0 at the start.
 *
 * Faces of a section: 0: x = 0, 1: x = (nx-1) h, 2: y = 0, 3: y = (ny-1) h.
 * Field arrays are [n_grids][ny][nx] (x fastest), FP64 absolute values at the ABI.
 * The conventions of hygro.h hold: every call validates before it changes state, copies its
 * inputs, accepts host or device output pointers, and is not thread-safe on one context.
 */
#ifndef HYGRO2D_H
#define HYGRO2D_H

#include "hygro.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hygro2d_ctx hygro2d_ctx;   /* opaque, owned by the library */

/* Most material regions per section. */
#define HYGRO2D_MAX_REGIONS 8

typedef struct {
    int32_t n_grids;           /* sections, >= 1 */
    int32_t nx, ny;            /* nodes per section in x and y, each >= 2 */
    double h;                  /* node spacing in x and y, metres, > 0 */
    double dt, t0, Lv, Psat;   /* as in hygro_desc */
    int32_t precision;         /* HYGRO_FP32 or HYGRO_FP64 */
    int32_t steps_per_launch;  /* DF steps fused in one launch (temporal blocking depth), 1..4, or 0 for 4 */
    int32_t device;            /* CUDA device ordinal */
    void *stream;              /* cudaStream_t to run on, or NULL for the default stream */
} hygro2d_desc;

/* Create a context on desc->device. Fails with HYGRO_E_UNSUPPORTED when a section is too large for
 * 32-bit node indices or the device lacks the shared memory of one tile. */
HYGRO_API hygro_status hygro2d_create(const hygro2d_desc *desc, hygro2d_ctx **out);

/* Material map and uniform initial state.
 *   region: [n_grids][ny][nx] region index of every node, each < n_regions (host memory);
 *   layers: [n_grids][n_regions] material of each region (hygro_layer, the affine laws of hygro.h);
 *   T_init, P_init: [n_grids] uniform initial state of each section.
 * Resets both stored levels to the initial state and the step to 0. */
HYGRO_API hygro_status hygro2d_set_materials(hygro2d_ctx *ctx, int32_t n_regions, const uint8_t *region,
                                             const hygro_layer *layers, const double *T_init, const double *P_init);

/* Boundary description of one face (0..3, see above) for every section: bc[g], g in 0..n_grids-1,
 * HYGRO_BC_AMBIENT or HYGRO_BC_ADIABATIC (host memory, copied). */
HYGRO_API hygro_status hygro2d_set_bc(hygro2d_ctx *ctx, int32_t face, const hygro_bc *bc);

/* Advance n_steps DF steps (n_steps >= 0): ceil(n_steps / steps_per_launch) launches, stream-ordered on
 * the context's stream; returns after enqueueing. Whole intervals of HYGRO2D_OPT_GRAPH_LAUNCHES launches
 * (64 by default) are replayed from a CUDA graph of that interval, built on first use and kept until the
 * materials, a boundary or an option changes; the rest of the run is launched one by one. The launches
 * and their results are the same either way (the graph's launches read their step index from a device
 * counter that the graph advances). */
HYGRO_API hygro_status hygro2d_run(hygro2d_ctx *ctx, int64_t n_steps);

/* Options (hygro2d_set_option / hygro2d_get_option):
 *   HYGRO2D_OPT_STEPS_PER_LAUNCH: DF steps fused per launch (temporal blocking depth), 1..4;
 *   HYGRO2D_OPT_GRAPH_LAUNCHES:   launches per CUDA graph interval, an even count up to 4096, 0 for none.
 * The paper has no counterpart: these shape the launches, not the scheme. Setting an option waits for
 * the context's stream. HYGRO_E_INVALID for an unknown option or a value out of range. */
#define HYGRO2D_OPT_STEPS_PER_LAUNCH 1
#define HYGRO2D_OPT_GRAPH_LAUNCHES 2
HYGRO_API hygro_status hygro2d_set_option(hygro2d_ctx *ctx, int32_t option, int64_t value);
HYGRO_API hygro_status hygro2d_get_option(const hygro2d_ctx *ctx, int32_t option, int64_t *value);

/* Autotuner of the temporal blocking depth: from the current state, times probe_steps steps (1..100000)
 * at each depth 1..4 (a warm-up launch first, CUDA events on the context's stream), restores the state
 * after each, and keeps the fastest depth as HYGRO2D_OPT_STEPS_PER_LAUNCH. *k_best (may be NULL)
 * receives it and ms_per_step[0..3] (may be NULL) the time per step of each depth. The state, the step
 * and the results of later runs are unchanged: every depth gives the same bits. Temporarily allocates
 * two copies of the stored levels. Synchronous. The paper has no counterpart. */
HYGRO_API hygro_status hygro2d_autotune(hygro2d_ctx *ctx, int32_t probe_steps, int32_t *k_best,
                                        double *ms_per_step);

/* Wait for the context's stream. HYGRO_E_NONFINITE if a node went non-finite, HYGRO_E_TIMEOUT if a
 * bounded device wait gave up, since the last check. */
HYGRO_API hygro_status hygro2d_sync(hygro2d_ctx *ctx);

/* Stored level 0 (n) or 1 (n-1) as absolute FP64 values, [n_grids][ny][nx] each (T or P may be NULL). */
HYGRO_API hygro_status hygro2d_get_fields(hygro2d_ctx *ctx, int32_t level, double *T, double *P);

/* Overwrite one stored level (absolute values, [n_grids][ny][nx], host or device memory). */
HYGRO_API hygro_status hygro2d_set_fields(hygro2d_ctx *ctx, int32_t level, const double *T, const double *P);

/* Index n of the newest stored level. */
HYGRO_API hygro_status hygro2d_get_step(const hygro2d_ctx *ctx, int64_t *step);

/* Message of the last failed call on ctx (or of the last failed hygro2d_create when ctx is NULL). */
HYGRO_API const char *hygro2d_last_error(const hygro2d_ctx *ctx);

/* Release everything the context owns. NULL is accepted. */
HYGRO_API void hygro2d_destroy(hygro2d_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* HYGRO2D_H */
