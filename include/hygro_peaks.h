/*
 * Arithmetic peaks of the GPU the hygro library runs on, measured by
 * microbenchmark: the denominators of the roofline fractions of the 1D wall
 * kernels, whose work is FP32 arithmetic (HBM traffic is only forcing and
 * samples). The paper has no counterpart: it states no hardware roof.
 *
 * Each probe launches a grid of (SM count x 4) blocks of 256 threads; every
 * thread runs 8 independent dependency chains of one instruction kind for a
 * number of iterations chosen so that the timed launch lasts about
 * target_ms (a short calibration launch first), and writes nothing to
 * memory but one result guarded by a comparison that never holds (so the
 * chains cannot be removed). The time is taken with CUDA events on the given
 * stream after a warm-up launch. Operations counted, per thread lane:
 *   HYGRO_PEAK_FFMA   fma.rn.f32          one operation per instruction
 *   HYGRO_PEAK_FFMA2  fma.rn.f32x2        two operations per instruction (a packed pair)
 *   HYGRO_PEAK_RCP    rcp.approx.ftz.f32  one operation per instruction (each chain step adds a
 *                                         constant first, which keeps consecutive reciprocals from
 *                                         cancelling; the adds are not counted)
 *   HYGRO_PEAK_DFMA   fma.rn.f64          one operation per instruction
 * Results: *ops_per_s (lane operations per second over the whole GPU) and
 * *ms (the timed launch). The clock the GPU ran at is not controlled here:
 * sample it while the probe runs.
 */
#ifndef HYGRO_PEAKS_H
#define HYGRO_PEAKS_H

#include <stdint.h>

#include "hygro.h"

#ifdef __cplusplus
extern "C" {
#endif

enum { HYGRO_PEAK_FFMA = 0, HYGRO_PEAK_FFMA2 = 1, HYGRO_PEAK_RCP = 2, HYGRO_PEAK_DFMA = 3 };

/* Run one probe on `device` (the current device when < 0), on `stream` (a cudaStream_t, NULL for the
 * legacy default stream). HYGRO_E_INVALID for an unknown kind, a NULL output or target_ms outside
 * [1, 10000]; HYGRO_E_CUDA when a CUDA call fails. Synchronous. */
HYGRO_API hygro_status hygro_peak_probe(int32_t kind, int32_t device, void *stream, double target_ms,
                                        double *ops_per_s, double *ms);

#ifdef __cplusplus
}
#endif
#endif
