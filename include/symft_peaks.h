/*
 * symft_peaks.h -- peak-rate microbenchmarks of the current GPU, the
 * denominators of the rooflines that HBM bandwidth and tensor throughput do
 * not cover.  The sampler's sign path is integer work (Philox draws, 32-bit
 * XOR / LOP3, shared-memory atomics) and its on-chip dense executors are FP32
 * / FP64 arithmetic on shared memory, so their fractions of peak are taken
 * against these measured rates.  The paper has no counterpart: this is
 * measurement infrastructure of this library.
 *
 * symft_measure_peaks runs six short kernels on the current device (a few
 * tens of milliseconds in total) and fills *out with whole-GPU rates:
 *   int32_lop3_per_s       3-input LOP3 lane operations per second
 *   int32_imad_wide_per_s  32x32->64 multiplies (IMAD.WIDE) per second
 *   philox_blocks_per_s    Philox4x32-10 blocks (128 random bits) per second
 *   fp32_fma_per_s         FP32 fused multiply-adds per second
 *   fp64_fma_per_s         FP64 fused multiply-adds per second
 *   smem_bytes_per_s       shared-memory load bytes per second (conflict-free
 *                          16-byte loads)
 * plus the SM count and the clock the device reports.  Each rate comes from
 * one CUDA-event-timed launch of many independent chains per thread on
 * 8 CTAs x 256 threads per SM.  The call allocates 16 bytes of device memory
 * for a result sink and synchronises the device.  Returns 0, or a negative
 * code: SYMFT_PEAK_E_ARG for a NULL argument, SYMFT_PEAK_E_CUDA when a CUDA
 * call fails (the fields measured before the failure are kept).
 */
#ifndef SYMFT_PEAKS_H
#define SYMFT_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

enum { SYMFT_PEAK_OK = 0, SYMFT_PEAK_E_ARG = -3, SYMFT_PEAK_E_CUDA = -6 };

typedef struct {
  int sm_count;
  double sm_clock_mhz_attr;
  double int32_lop3_per_s;
  double int32_imad_wide_per_s;
  double philox_blocks_per_s;
  double fp32_fma_per_s;
  double fp64_fma_per_s;
  double smem_bytes_per_s;
} symft_peaks;

int symft_measure_peaks(symft_peaks* out);

#ifdef __cplusplus
}
#endif

#endif /* SYMFT_PEAKS_H */
