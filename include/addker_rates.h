/*
 * addker_rates.h - device-rate microbenchmark of the GB300 library for additive-kernel products.
 *
 * Measurement tooling, not part of the product interface (include/addker.h): the rates bound the
 * product's spread and gather kernels and serve the benchmark's roofline accounting. Built into its own
 * shared library (libaddker_rates.so) beside libaddker.so; status codes are those of addker.h.
 */
#ifndef ADDKER_RATES_H
#define ADDKER_RATES_H

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Device rates for roofline accounting (not in the paper; needs no plan). On the current device,
 * each rate from a kernel that does nothing else, median of 3 timed launches after a warm-up:
 *   out[0] SMs   out[1] SM clock under FP32 load, MHz (clock64 against the global timer)
 *   out[2] FFMA TFLOP/s   out[3] packed FFMA2 TFLOP/s (an FMA counts 2 flops)
 *   out[4] shared-memory float atomic adds, 10^9/s (distinct words)
 *   out[5] global float atomic adds into a 1 MiB L2-resident grid, 10^9/s (rows of 32 words)
 *   out[6] milliseconds of the FFMA launch
 *   out[7] global double atomic adds into a 2 MiB L2-resident grid, 10^9/s (rows of 32 words).
 * Writes up to `cap` values (host doubles) and returns the number available (8); synchronous,
 * about 0.2 s of GPU time. ADDKER_ECUDA / ADDKER_ENOMEM on failure.
 */
int addker_device_rates(double* out, int cap);

#ifdef __cplusplus
}
#endif
#endif /* ADDKER_RATES_H */
