// Peak-rate microbenchmarks of one GPU (the denominators of the rooflines that
// are not HBM or tensor bound): 32-bit integer logic (LOP3), 32x32->64
// integer multiply-add (IMAD.WIDE), the Philox4x32-10 block function of the
// random-stream specification, FP32 FMA, FP64 FMA and shared-memory load
// bandwidth.  Each kernel runs many independent dependency chains per thread
// over a grid of several CTAs per SM, so the measured rate is the pipe's
// throughput, not its latency.  Results are operations per second for the
// whole GPU, timed with CUDA events around one launch after a warm-up launch.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "device.cuh"
#include "symft_peaks.h"

namespace symft {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;          // independent chains per thread

// 3-input XOR, one LOP3 per step and chain
__global__ void __launch_bounds__(kPeakThreads) peak_lop3_kernel(uint32_t iters, uint32_t seed, uint32_t* sink) {
  uint32_t a[kChains], b = seed ^ threadIdx.x, c = seed * 0x9E3779B9u + blockIdx.x;
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = seed + k * 0x1234567u + threadIdx.x;
  for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      uint32_t r;
      asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(a[k]), "r"(b), "r"(c));
      a[k] = r;
    }
    b += 1u;
  }
  uint32_t x = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) x ^= a[k];
  if (x == 0x13579BDFu) sink[0] = x;
}

// 32x32 -> 64-bit multiply, one IMAD.WIDE per step and chain
__global__ void __launch_bounds__(kPeakThreads) peak_imad_kernel(uint32_t iters, uint32_t seed, uint32_t* sink) {
  uint32_t a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = seed + k * 0x1234567u + threadIdx.x;
  for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      uint64_t r;
      asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(r) : "r"(a[k]), "r"(0xD2511F53u));
      a[k] = (uint32_t)(r >> 32) ^ (uint32_t)r;
    }
  }
  uint32_t x = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) x ^= a[k];
  if (x == 0x13579BDFu) sink[0] = x;
}

// Philox4x32-10 blocks with precomputed round keys, two independent counters
// per thread
__global__ void __launch_bounds__(kPeakThreads) peak_philox_kernel(uint32_t iters, PhiloxKeys K, uint32_t* sink) {
  uint4 c0 = make_uint4(threadIdx.x, blockIdx.x, 0u, 1u), c1 = make_uint4(threadIdx.x, blockIdx.x, 0u, 2u);
  uint32_t x = 0;
  for (uint32_t i = 0; i < iters; ++i) {
    c0.z = i;
    c1.z = i;
    const uint4 o0 = philox(c0, K), o1 = philox(c1, K);
    x ^= o0.x ^ o0.y ^ o0.z ^ o0.w ^ o1.x ^ o1.y ^ o1.z ^ o1.w;
  }
  if (x == 0x13579BDFu) sink[0] = x;
}

template <typename Real>
__global__ void __launch_bounds__(kPeakThreads) peak_fma_kernel(uint32_t iters, Real s, uint32_t* sink) {
  Real a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (Real)(threadIdx.x + k) * (Real)1e-3;
  const Real m = (Real)0.999999, c = s;
  for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = a[k] * m + c;
  }
  Real x = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) x += a[k];
  if (x == (Real)-1.2345) sink[0] = 1u;
}

// 16-byte shared-memory loads, conflict-free (consecutive lanes, consecutive
// 16-byte words), four independent loads per step
__global__ void __launch_bounds__(kPeakThreads) peak_smem_kernel(uint32_t iters, uint32_t seed, uint32_t* sink) {
  __shared__ uint4 buf[kPeakThreads * 4];
  for (int i = threadIdx.x; i < kPeakThreads * 4; i += kPeakThreads) buf[i] = make_uint4(i, seed, i ^ seed, 1u);
  __syncthreads();
  uint4 acc = make_uint4(0u, 0u, 0u, 0u);
  uint32_t off = threadIdx.x;
  for (uint32_t i = 0; i < iters; ++i) {
    const uint4 v0 = buf[off], v1 = buf[(off + kPeakThreads) & (kPeakThreads * 4 - 1)];
    const uint4 v2 = buf[(off + 2 * kPeakThreads) & (kPeakThreads * 4 - 1)];
    const uint4 v3 = buf[(off + 3 * kPeakThreads) & (kPeakThreads * 4 - 1)];
    acc = xor4(acc, xor4(xor4(v0, v1), xor4(v2, v3)));
    off = (off + 32 + (acc.x & 0u)) & (kPeakThreads * 4 - 1);
  }
  if ((acc.x ^ acc.y ^ acc.z ^ acc.w) == 0x13579BDFu) sink[0] = 1u;
}

}  // namespace
}  // namespace symft

using namespace symft;

namespace {

// time one launch (after a warm-up launch) of `launch(iters)`
template <typename F>
int time_kernel(F launch, uint32_t iters, double* ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return SYMFT_PEAK_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return SYMFT_PEAK_E_CUDA;
  }
  launch(iters / 8 + 1);
  cudaEventRecord(e0);
  launch(iters);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return SYMFT_PEAK_E_CUDA;
  *ms = t;
  return SYMFT_PEAK_OK;
}

}  // namespace

extern "C" int symft_measure_peaks(symft_peaks* out) {
  if (!out) return SYMFT_PEAK_E_ARG;
  std::memset(out, 0, sizeof(*out));
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SYMFT_PEAK_E_CUDA;
  int sms = 0, clk_khz = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SYMFT_PEAK_E_CUDA;
  if (cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev) != cudaSuccess) clk_khz = 0;
  out->sm_count = sms;
  out->sm_clock_mhz_attr = clk_khz / 1000.0;
  uint32_t* sink = nullptr;
  if (cudaMalloc(&sink, 16) != cudaSuccess) return SYMFT_PEAK_E_CUDA;
  const int grid = sms * 8;
  const double threads = (double)grid * kPeakThreads;
  double ms = 0.0;
  int rc;
  const uint32_t it = 1u << 14;
  rc = time_kernel([&](uint32_t n) { peak_lop3_kernel<<<grid, kPeakThreads>>>(n, 7u, sink); }, it, &ms);
  if (rc == SYMFT_PEAK_OK) out->int32_lop3_per_s = threads * it * kChains / (ms * 1e-3);
  if (rc == SYMFT_PEAK_OK)
    rc = time_kernel([&](uint32_t n) { peak_imad_kernel<<<grid, kPeakThreads>>>(n, 7u, sink); }, it, &ms);
  if (rc == SYMFT_PEAK_OK) out->int32_imad_wide_per_s = threads * it * kChains / (ms * 1e-3);
  const PhiloxKeys K = make_philox_keys(0x1234ABCDull);
  const uint32_t itp = 1u << 10;
  if (rc == SYMFT_PEAK_OK)
    rc = time_kernel([&](uint32_t n) { peak_philox_kernel<<<grid, kPeakThreads>>>(n, K, sink); }, itp, &ms);
  if (rc == SYMFT_PEAK_OK) out->philox_blocks_per_s = threads * itp * 2 / (ms * 1e-3);
  if (rc == SYMFT_PEAK_OK)
    rc = time_kernel([&](uint32_t n) { peak_fma_kernel<float><<<grid, kPeakThreads>>>(n, 1e-7f, sink); }, it, &ms);
  if (rc == SYMFT_PEAK_OK) out->fp32_fma_per_s = threads * it * kChains / (ms * 1e-3);
  const uint32_t itd = 1u << 10;
  if (rc == SYMFT_PEAK_OK)
    rc = time_kernel([&](uint32_t n) { peak_fma_kernel<double><<<grid, kPeakThreads>>>(n, 1e-7, sink); }, itd, &ms);
  if (rc == SYMFT_PEAK_OK) out->fp64_fma_per_s = threads * itd * kChains / (ms * 1e-3);
  if (rc == SYMFT_PEAK_OK)
    rc = time_kernel([&](uint32_t n) { peak_smem_kernel<<<grid, kPeakThreads>>>(n, 7u, sink); }, it, &ms);
  if (rc == SYMFT_PEAK_OK) out->smem_bytes_per_s = threads * it * 4 * 16 / (ms * 1e-3);
  cudaFree(sink);
  return rc;
}
