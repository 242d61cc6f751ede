/* rich_peaks.h -- throughput microbenchmarks of the GPU units the photon
 * trace relies on, exported by librich.so beside the propagator (rich.h).
 *
 * The paper has no counterpart: these are the measured denominators of the
 * trace kernel's roofline (the slower of the FP32 bound and the L2 bound of
 * its bytes per photon). Peaks derived from unit counts and the nominal
 * clock overstate what a kernel can reach at the clocks the GPU actually
 * runs; these are measured on the device, at its current clocks.
 */
#ifndef RICH_PEAKS_H
#define RICH_PEAKS_H

#include <stdint.h>

#if defined(__GNUC__)
#define RICH_PEAKS_API __attribute__((visibility("default")))
#else
#define RICH_PEAKS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rich_peaks {
    double fp32_fma_flops;   /* FP32 fused multiply-adds x 2 per second: 8
                                independent FMA chains per thread, 64 warps
                                per SM                                      */
    double fp32_minmax_ops;  /* FP32 min/max operations per second (the ALU
                                pipe), same shape                           */
    double mufu_ops;         /* approximate reciprocals per second (the
                                special-function unit), each fed by an FMA
                                so that no two can be folded               */
    double l2_read_bytes;    /* bytes per second read from L2 by 16-byte
                                loads that bypass L1 (ld.global.cg), over a
                                48 MiB buffer read 20 times by 4 x 512
                                threads per SM                              */
    int32_t n_sm;            /* streaming multiprocessors                   */
    int32_t reserved;
    double sm_clock_mhz_max; /* the device's maximum SM clock (attribute)   */
} rich_peaks;

/* Runs the four microbenchmarks on `device` (made current for the call and
 * restored after) on `stream` (a cudaStream_t, NULL for the legacy default
 * stream), each the best of three runs after one warm-up, timed with CUDA
 * events on that stream; takes about half a second. Allocates 49 MiB of
 * device memory for the call and frees it. *out (host) receives the rates;
 * a rate that could not be measured is 0. Returns 0 on success, 1 for a
 * NULL out, 2 for a CUDA error, 3 if the allocation failed
 * (rich_peaks_last_error describes it). Synchronous. */
RICH_PEAKS_API int rich_measure_peaks(int device, void *stream, rich_peaks *out);

/* Message of the calling thread's last failed rich_measure_peaks. */
RICH_PEAKS_API const char *rich_peaks_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RICH_PEAKS_H */
