/*
 * wave_peaks.h -- on-device microbenchmarks behind the ALU and shared-memory
 * roofs that the benchmark reports beside the HBM roof of the sweep.
 *
 * The paper bounds its operators by a roofline of memory bandwidth and
 * floating-point peak (Sec. 5.4.2, Sec. 5.5); these two numbers are the
 * corresponding ceilings of the GPU the library runs on, measured, not taken
 * from a data sheet.  They are not part of the modelling path.
 */
#ifndef WAVETILE_WAVE_PEAKS_H
#define WAVETILE_WAVE_PEAKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Measure on the current device, on `stream` (a cudaStream_t; NULL = legacy
 * default stream), and wait for the result:
 *   fp32_tflops (HOST out)  FP32 FMA throughput in TFLOP/s (one FMA = 2 flops),
 *                           every SM running independent paired-FP32 FMA chains
 *                           (the instruction form the sweep's arithmetic uses);
 *   smem_tbs    (HOST out)  shared-memory load bandwidth in TB/s summed over all
 *                           SMs, conflict-free 16-byte loads.
 * Each kernel runs a few milliseconds; the best of three runs is kept.  Uses
 * no device memory beyond a 64-byte result buffer in the library's static
 * storage.  Returns WAVE_OK (0), WAVE_EINVAL (-1) for NULL outputs or
 * WAVE_ECUDA (-3). */
int32_t wave_measure_peaks(double *fp32_tflops, double *smem_tbs, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* WAVETILE_WAVE_PEAKS_H */
