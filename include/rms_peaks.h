/*
 * rms_peaks.h -- machine peaks behind the rooflines of the walker step.
 *
 * The paper has no counterpart: these calls measure, on the current device,
 * the rates that bound the random-walker step of Sec. 2.2, so that a
 * measured walker-step rate can be stated as a fraction of a measured peak.
 *   - The label lookup of Sec. 2.1.1 is one dependent 2-byte gather across
 *     each face a walker meets; its ceiling is the rate of random 2-byte
 *     gathers from a uint16 volume of the same size, served by L2 when the
 *     volume fits there and by HBM when it does not.
 *   - The plain FP64 form is bound by GB300's FP64 pipe: its ceiling is the
 *     rate of independent FP64 adds and multiplies (the form is compiled
 *     without FMA contraction, so adds and multiplies are what it issues).
 *
 * Every call allocates what it needs on the current device (cudaMalloc),
 * runs one untimed launch, then times `reps` launches with CUDA events on
 * `stream` and reports the best.  Not for use inside stream capture.
 */
#ifndef RMS_PEAKS_H
#define RMS_PEAKS_H

#include <stdint.h>

#include "rms.h"

#ifdef __cplusplus
extern "C" {
#endif

/* kinds of rms_measure_peak */
#define RMS_PEAK_FP64_ADD 0   /* independent FP64 adds (__dadd_rn), 8 chains per thread, op/s */
#define RMS_PEAK_FP64_MUL 1   /* independent FP64 multiplies (__dmul_rn), op/s */
#define RMS_PEAK_FP64_FMA 2   /* independent FP64 fused multiply-adds, op/s (one FMA = one op) */
#define RMS_PEAK_GATHER 3     /* independent random 2-byte gathers (read-only path) from a uint16 volume of
                                 `volume_elems` elements, 8 in flight per thread: gathers/s */
#define RMS_PEAK_GATHER_DEP 4 /* the same with one gather in flight per thread (each address depends on the
                                 previous label, as a walker's face events do): gathers/s */

/* Measure one peak.  volume_elems: for the gather kinds, the number of
 * uint16 elements of the volume, a power of two in [2^10, 2^31] (2^24 = 32
 * MiB stays in GB300's 129 MB L2; 2^28 = 512 MiB does not); ignored
 * otherwise.  target_ms: approximate duration of one timed launch (> 0;
 * e.g. 20).  reps: timed launches, >= 1.  Outputs: *rate = operations or
 * gathers per second of the best launch, *ms = its duration (either may be
 * NULL).  Errors: RMS_E_INVALID_ARG (unknown kind, bad size), RMS_E_OOM,
 * RMS_E_CUDA. */
rms_status rms_measure_peak(int32_t kind, int64_t volume_elems, double target_ms, int32_t reps, void *stream,
                            double *rate, double *ms);

/* Number of streaming multiprocessors of the current device
 * (cudaDevAttrMultiProcessorCount), for the issue-slot peak.  RMS_E_CUDA. */
rms_status rms_device_sm_count(int32_t *sm_count);

#ifdef __cplusplus
}
#endif

#endif /* RMS_PEAKS_H */
