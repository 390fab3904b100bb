// symft_sample_noalloc: sampling for callers that cannot allocate device memory.
//
// Some hosts of this library own the whole device heap (a framework with its
// own caching allocator, a service with a fixed memory budget) and cannot let
// a library call cudaMalloc.  This
// entry point runs the sign, warp-executor and finalize kernels of
// symft_sample_ex but takes every byte of device memory it needs beyond the
// caller's outputs -- the copy of the
// plan, the dense-sign columns, the active-outcome columns, the status word
// and any global active vectors -- from one fixed array in this file.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds kNoAllocBytes for it until the process exits.  Host code only
// sees a stand-in symbol, so the device address is fetched once per device
// with cudaGetSymbolAddress (on the first call made with that device current)
// and passed to the kernels.  All calls share the array: calls that overlap on
// the GPU (different streams, or different host threads) race on it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "internal.hpp"
#include "plan_dev.hpp"
#include "plan_host.hpp"
#include "symft.h"

namespace symft {
namespace {

constexpr size_t kNoAllocBytes = size_t(32) << 20;   // 32 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_setup_mu;
unsigned char* g_base[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};

thread_local std::string g_noalloc_error;

int fail(int code, const std::string& msg) {
  g_noalloc_error = msg;
  return code;
}

inline size_t up256(size_t v) { return (v + 255) & ~size_t(255); }

// Device address of the array on `dev` (which must be current).
cudaError_t setup(int dev, unsigned char** base, int* sms) {
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (g_base[dev] == nullptr) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_base[dev] = static_cast<unsigned char*>(ptr);
    g_sm_count[dev] = n;
  }
  *base = g_base[dev];
  *sms = g_sm_count[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace symft

using namespace symft;

extern "C" const char* symft_noalloc_last_error(void) { return g_noalloc_error.c_str(); }

extern "C" int symft_sample_noalloc(const symft_plan* plan, uint64_t shots, uint64_t seed,
                                    uint64_t shot_offset, uint64_t* meas_out, uint64_t* det_out,
                                    uint64_t* obs_out, uint64_t* discard_out, int precision,
                                    void* stream) {
  g_noalloc_error.clear();
  if (!plan) return fail(SYMFT_E_ARG, "null plan");
  if (shots == 0) return fail(SYMFT_E_ARG, "shots must be >= 1");
  if (shot_offset % kNoiseBlock)
    return fail(SYMFT_E_ARG, "shot_offset must be a multiple of " + std::to_string(kNoiseBlock));
  if (shots + shot_offset > (1ull << 39)) return fail(SYMFT_E_ARG, "shot index beyond 2^39");
  if (precision != SYMFT_FP32 && precision != SYMFT_FP64) return fail(SYMFT_E_ARG, "bad precision");
  const HostPlan& h = plan->hp;
  const uint64_t W = (shots + 63) / 64;
  const uint64_t nblk = (shots + kNoiseBlock - 1) / kNoiseBlock;
  const uint32_t G = static_cast<uint32_t>(h.dense.size());
  if (h.n_records == 0) meas_out = nullptr;
  if (h.n_dets == 0) det_out = nullptr;
  if (h.n_obs == 0) obs_out = nullptr;
  const bool need_det_scratch = h.postselect && det_out == nullptr && h.n_dets > 0;
  const bool fp64 = precision == SYMFT_FP64;

  // dense launch shape (as symft_sample_ex chooses it)
  const size_t amp = fp64 ? 16 : 8;
  const size_t m3bytes = ((h.n_m3 + 31) / 32) * 4;
  const size_t vec_bytes = (static_cast<size_t>(1) << h.k_max) * amp;
  const bool dense_smem = vec_bytes + m3bytes <= 48 * 1024;
  const int dense_wpb = dense_smem
                            ? static_cast<int>(std::min<size_t>(8, std::max<size_t>(1, (160 * 1024) / (vec_bytes + m3bytes + 16))))
                            : 4;

  // carve the array: plan | status | dense signs | m3 | detector scratch | vectors
  const size_t o_plan = 0;
  const size_t o_status = up256(plan->blob.size());
  const size_t o_signs = o_status + 256;
  const size_t o_m3 = o_signs + up256(static_cast<size_t>(G) * W * 8);
  const size_t o_det = o_m3 + up256(static_cast<size_t>(h.n_m3) * W * 8);
  const size_t o_vec = o_det + (need_det_scratch ? up256(static_cast<size_t>(h.n_dets) * W * 8) : 0);
  size_t need = o_vec;
  uint64_t dense_grid_cap = 0;
  if (G && !dense_smem) {
    // at least one warp slot of global vector space; the grid shrinks to what fits
    if (need + vec_bytes * dense_wpb > kNoAllocBytes)
      return fail(SYMFT_E_CAPACITY, "active vectors of 2^" + std::to_string(h.k_max) +
                                        " amplitudes do not fit the 32 MiB no-allocation array");
    dense_grid_cap = (kNoAllocBytes - need) / (vec_bytes * dense_wpb);
    need += dense_grid_cap * dense_wpb * vec_bytes;
  }
  if (need > kNoAllocBytes)
    return fail(SYMFT_E_CAPACITY, "request needs " + std::to_string(need) +
                                      " bytes of device scratch, more than the 32 MiB no-allocation "
                                      "array; sample fewer shots per call");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(SYMFT_E_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(SYMFT_E_ARG, "device ordinal out of range");
  unsigned char* base = nullptr;
  int sms = 0;
  e = setup(dev, &base, &sms);
  if (e != cudaSuccess) return fail(SYMFT_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  e = set_smem_limits();
  if (e != cudaSuccess) return fail(SYMFT_E_CUDA, cudaGetErrorString(e));

  // the plan image goes into the array on every call (calls may alternate plans)
  e = cudaMemcpyAsync(base + o_plan, plan->blob.data(), plan->blob.size(), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail(SYMFT_E_CUDA, cudaGetErrorString(e));
  DevPlan dp{};
  bind_plan(plan, base + o_plan, &dp);
  uint64_t* signs = G ? reinterpret_cast<uint64_t*>(base + o_signs) : nullptr;
  uint64_t* m3 = h.n_m3 ? reinterpret_cast<uint64_t*>(base + o_m3) : nullptr;
  uint64_t* det = need_det_scratch ? reinterpret_cast<uint64_t*>(base + o_det) : det_out;
  int* status = reinterpret_cast<int*>(base + o_status);

  if (h.n_slots > 0) {
    SignArgs s{};
    s.p = dp;
    s.seed = seed;
    s.keys = make_philox_keys(seed);
    s.block0 = shot_offset / kNoiseBlock;
    s.n_blocks = nblk;
    s.W = W;
    s.shots = shots;
    s.meas = meas_out;
    s.det = det;
    s.obs = obs_out;
    s.signs = signs;
    s.status = status;
    if (sign_smem_bytes(dp) > 220 * 1024) return fail(SYMFT_E_CAPACITY, "too many bit-packed slots");
    int per_sm = 1;
    e = sign_occupancy(dp, &per_sm);
    if (e != cudaSuccess) return fail(SYMFT_E_CUDA, cudaGetErrorString(e));
    const uint64_t cap = static_cast<uint64_t>(sms) * std::max(1, per_sm);
    e = launch_sign(s, static_cast<int>(std::max<uint64_t>(1, std::min(nblk, cap))), st);
    if (e != cudaSuccess) return fail(SYMFT_E_CUDA, cudaGetErrorString(e));
  }
  if (G) {
    // active outcomes are OR-ed in by the dense kernel: clear the previous call's bits
    if (h.n_m3) {
      e = cudaMemsetAsync(m3, 0, static_cast<size_t>(h.n_m3) * W * 8, st);
      if (e != cudaSuccess) return fail(SYMFT_E_CUDA, cudaGetErrorString(e));
    }
    DenseArgs d{};
    d.p = dp;
    d.seed = seed;
    d.keys = make_philox_keys(seed);
    d.shot0 = shot_offset;
    d.shots = shots;
    d.W = W;
    d.signs = signs;
    d.m3_out = m3 ? m3 : reinterpret_cast<uint64_t*>(base + o_m3);
    d.kmax = h.k_max;
    d.status = status;
    // early exit under postselection reads the detector columns the sign
    // kernel has just written (as symft_sample_ex does)
    d.det_exo = dp.post_chk_off ? det : nullptr;
    size_t smem;
    uint64_t cap = static_cast<uint64_t>(sms) * (dense_smem ? 16 : 8);
    if (dense_smem) {
      d.use_smem = 1;
      smem = dense_warp_smem_bytes(dp, dense_wpb, vec_bytes, true);
    } else {
      d.use_smem = 0;
      smem = dense_warp_smem_bytes(dp, dense_wpb, vec_bytes, false);
      cap = std::min<uint64_t>(cap, std::max<uint64_t>(1, dense_grid_cap));
      d.gvec = base + o_vec;
      d.gvec_stride = static_cast<uint64_t>(1) << h.k_max;
    }
    const uint64_t want = (shots + dense_wpb - 1) / dense_wpb;
    const int grid = static_cast<int>(std::max<uint64_t>(1, std::min(want, cap)));
    e = launch_dense(d, fp64, dense_wpb, grid, smem, st);
    if (e != cudaSuccess) return fail(SYMFT_E_CUDA, cudaGetErrorString(e));
  }
  if (h.n_m3 > 0 || h.postselect || discard_out != nullptr) {
    FinalArgs f{};
    f.p = dp;
    f.W = W;
    f.shots = shots;
    f.m3 = m3;
    f.meas = meas_out;
    f.det = det;
    f.obs = obs_out;
    f.discard = discard_out;
    e = launch_finalize(f, st);
    if (e != cudaSuccess) return fail(SYMFT_E_CUDA, cudaGetErrorString(e));
  }
  return SYMFT_OK;
}
