// Host-side plan object shared by the C ABI translation units.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "internal.hpp"
#include "plan_dev.hpp"

namespace symft {

struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t need) {
    if (need <= bytes) return cudaSuccess;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&ptr, need);
    if (e == cudaSuccess) bytes = need;
    return e;
  }
  void release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
  }
};

// Byte offsets of the plan arrays inside the device blob.
struct BlobOffsets {
  size_t ch, q, ct, t4, qi, qs, pc, m1t, m1o, m1g, tco, tca, sc, li, gi, gv, pe, dn, dc, m3t, sm1, sm1o, pco, pch;
  size_t plc, plo, pls;
  size_t clt, clo;
  size_t ctg;
  uint32_t n_ctg = 0;
  size_t snz, odl, ors, pid;
  uint32_t n_pth = 0;
  uint32_t n_snz = 0, n_odl = 0, n_ors = 0;
};

cudaError_t launch_sign(const SignArgs& a, int grid, cudaStream_t st);
size_t sign_smem_bytes(const DevPlan& p);
cudaError_t sign_occupancy(const DevPlan& p, int* ctas_per_sm);
// shots_per_warp 2: two shots per warp, each on 16 lanes (the smem size is
// then that of 2 * warps_per_block shots)
cudaError_t launch_dense(const DenseArgs& a, bool fp64, int warps_per_block, int grid, size_t smem,
                         cudaStream_t st, int shots_per_warp = 1);
cudaError_t launch_finalize(const FinalArgs& a, cudaStream_t st);
cudaError_t launch_count(const CountArgs& a, int sm_count, cudaStream_t st);
cudaError_t set_smem_limits();
size_t plain_smem_bytes(const DevPlan& p, uint32_t kmax, bool fp64);
size_t dense_reg_smem_bytes(const DevPlan& p);
size_t dense_warp_smem_bytes(const DevPlan& p, int wpb, size_t vec_bytes, bool vec_in_smem);
size_t dense_pc_smem_bytes(const DevPlan& p, int wpb, size_t ws_bytes, bool ws_in_smem);
size_t dense_cta_smem_bytes(const DevPlan& p, size_t vec_bytes, bool vec_in_smem);
cudaError_t launch_dense_cta(const DenseArgs& a, bool fp64, int grid, size_t smem, cudaStream_t st);
cudaError_t launch_dense_reg(const DenseArgs& a, bool fp64, int grid, cudaStream_t st);
// shots one CTA of the register executor holds at a time
uint32_t dense_reg_shots_per_cta(uint32_t kmax, bool fp64);
cudaError_t launch_dense_pc(const DenseArgs& a, bool fp64, int warps_per_block, int grid, size_t smem,
                            cudaStream_t st);
// resident CTAs per SM of the product-component warp executor for a launch shape
cudaError_t dense_pc_occupancy(bool fp64, int warps_per_block, size_t smem, int* ctas_per_sm);
cudaError_t launch_dense_pc_cta(const DenseArgs& a, bool fp64, int grid, size_t smem, cudaStream_t st);
cudaError_t launch_plain(const PlainArgs& a, bool fp64, int grid, cudaStream_t st);
// all dense instructions for one batch of the wide executor (host_dense: the
// plan's instruction stream in host memory, for the per-instruction launches)
// (tile_bits: amplitudes per fused-window tile as a power of two, 0 = default)
cudaError_t launch_wide_batch(const WideArgs& a, const DenseInstrDev* host_dense, bool fp64, int sm_count,
                              cudaStream_t st, int* launches,
                              uint32_t tile_bits = 0);
// amplitudes one shot moves through HBM in the wide executor's passes
uint64_t wide_amp_traffic(const DenseInstrDev* d, uint32_t G, bool fp64, uint32_t tile_bits = 0);
// the fused-window tile bits the wide executor uses for a request (0 = default)
uint32_t wide_tile_bits_in_use(bool fp64, uint32_t tile_bits);

// Launch shapes chosen by symft_autotune (0 = built-in heuristic).
struct Tune {
  bool tuned = false;
  int sign_ctas_per_sm = 0;  // sign kernel: resident CTAs per SM (0 = occupancy limit)
  int dense_grid_mult = 8;   // register / warp executors: CTAs per SM
  int dense_wpb = 0;         // warp executor: warps (shots) per CTA
  int cta_grid_mult = 2;     // CTA executor with global vectors: CTAs per SM
  int wide_tile_bits = 0;    // wide executor: fused-window tile of 2^bits amplitudes (0 = default)
  int dense_kind = 0;        // dense executor (1 register, 2 warp, 3 CTA, 4 wide, 5 / 6 product
                             // components on a warp / a CTA; 0 = the cost model's choice)
  float best_ms_per_shot = 0.0f;
};

}  // namespace symft

struct symft_plan {
  symft::HostPlan hp;
  std::vector<unsigned char> blob;   // device image of the plan, built at compile time
  symft::BlobOffsets off{};
  std::mutex mu;
  bool uploaded = false;
  int device = -1;
  symft::DevBuf plan_buf;
  symft::DevPlan dp{};
  symft::DevBuf signs, m3, det_scratch, gvec, status, wide;
  std::vector<symft::DenseInstrDev> dense_host;   // host copy of the instruction stream
  uint32_t post_grp0 = 0xFFFFFFFFu;                // early-exit check before any dense work
  symft::DevBuf obs_scratch, disc_scratch;      // tallies without obs / discard outputs
  symft::DevBuf h_meas, h_det, h_obs, h_disc;   // staging for host outputs
  symft::DevBuf h_prob, h_counts;
  symft::DevBuf t_meas, t_det, t_obs, t_disc;   // outputs of autotuning probes
  symft::Tune tune[2];                          // FP32, FP64
  int sm_count = 0;
  // product-component warp executor (FP32, FP64): workspace in shared memory
  // (1) or global memory (0), warps per CTA and resident CTAs per SM, chosen
  // by occupancy (pc_wpb 0 = not yet chosen)
  int pc_smem[2] = {0, 0}, pc_wpb[2] = {0, 0}, pc_cps[2] = {0, 0};
};

namespace symft {
// Build the device image of a compiled plan (throws Error on capacity limits).
void build_blob(symft_plan* P);
// Point the DevPlan arrays into a copy of the blob at `base` (device address).
void bind_plan(const symft_plan* P, unsigned char* base, DevPlan* d);
}  // namespace symft
