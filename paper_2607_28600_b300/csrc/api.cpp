// C ABI (include/symft.h): compile, plan info, sampling, errors.
//
// The plan owns its host description, its device copy (uploaded by the first
// sampling call) and a workspace that grows to the largest request seen and
// is reused by later calls (Sec. 6, reuse of prepared buffers).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.hpp"
#include "plan_dev.hpp"
#include "plan_host.hpp"
#include "symft.h"




using namespace symft;

namespace {
thread_local std::string g_last_error;
thread_local int g_last_launches = 0;

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

}  // namespace

namespace {

template <class T>
size_t push(std::vector<unsigned char>& blob, const std::vector<T>& v) {
  size_t off = (blob.size() + 15) & ~size_t(15);
  blob.resize(off + v.size() * sizeof(T) + 16);
  if (!v.empty()) std::memcpy(blob.data() + off, v.data(), v.size() * sizeof(T));
  return off;
}

}  // namespace

namespace symft {

void build_blob(symft_plan* P) {
  const HostPlan& h = P->hp;
  std::vector<ChannelDev> ch(h.n_channels);
  for (uint32_t c = 0; c < h.n_channels; ++c)
    ch[c] = ChannelDev{h.ch_theta_last[c], h.ch_qtab[c], h.ch_ctab[c], h.ch_comp0[c], h.ch_ncomp[c]};
  std::vector<uint32_t> theta4(((h.n_channels + 3) / 4) * 4, 0u);
  for (uint32_t c = 0; c < h.n_channels; ++c) theta4[c] = h.ch_theta_last[c];
  std::vector<uint32_t> qtheta;
  std::vector<float> qinv;
  for (auto& q : h.qtabs) {
    qtheta.insert(qtheta.end(), q.theta, q.theta + kNoiseBlock);
    double l = std::log1p(-q.q);
    qinv.push_back((q.q > 0.0 && q.q < 1.0) ? static_cast<float>(1.0 / l) : 0.0f);
  }
  std::vector<CellTableDev> ct(h.ctabs.size());
  for (size_t i = 0; i < h.ctabs.size(); ++i) {
    ct[i].ncell = h.ctabs[i].ncell;
    std::memcpy(ct[i].phi, h.ctabs[i].phi, sizeof(ct[i].phi));
    std::memcpy(ct[i].mask, h.ctabs[i].mask, sizeof(ct[i].mask));
  }
  std::vector<DenseInstrDev> dn(h.dense.size());
  for (size_t g = 0; g < h.dense.size(); ++g) {
    const DenseInstr& d = h.dense[g];
    DenseInstrDev& o = dn[g];
    o.kind = d.kind;
    o.k = d.k;
    o.h = d.h;
    o.mu = d.mu;
    o.a = d.a;
    o.b = d.b;
    o.eta = d.eta;
    o.m3 = d.m3;
    o.c = d.c;
    o.s = d.s;
    o.sign_target_col = d.sign_target - h.n_records;
    o.causal_off = d.causal_off;
    o.causal_n = d.causal_n;
    o.t = d.t;
  }
  std::vector<unsigned char>& blob = P->blob;
  blob.clear();
  P->off.ch = push(blob, ch);
  P->off.q = push(blob, qtheta);
  P->off.ct = push(blob, ct);
  P->off.t4 = push(blob, theta4);
  P->off.qi = push(blob, qinv);
  // packed incidence lists (16-bit targets, 24-bit offsets, 8-bit counts)
  if (h.n_slots >= 65536) throw Error(SYMFT_E_CAPACITY, "more than 65535 bit-packed slots");
  if (h.comp_tgt.size() >= (1u << 24)) throw Error(SYMFT_E_CAPACITY, "too many sign incidences");
  if (h.n_channels >= (1u << 28)) throw Error(SYMFT_E_CAPACITY, "too many noise channels");
  std::vector<uint32_t> comp_rng(h.n_comp);
  for (uint32_t k = 0; k < h.n_comp; ++k) {
    const uint32_t off = h.comp_off[k], n = h.comp_off[k + 1] - off;
    bool inl = n <= 2;
    for (uint32_t j = 0; j < n && inl; ++j) inl = h.comp_tgt[off + j] < 16384;
    if (inl) {
      uint32_t t0 = n > 0 ? h.comp_tgt[off] : 0, t1 = n > 1 ? h.comp_tgt[off + 1] : 0;
      comp_rng[k] = 0x80000000u | (n << 28) | (t1 << 14) | t0;
    } else {
      if (n >= 256) throw Error(SYMFT_E_CAPACITY, "a noise component reaches more than 255 targets");
      if (off >= (1u << 23)) throw Error(SYMFT_E_CAPACITY, "too many sign incidences");
      comp_rng[k] = (off << 8) | n;
    }
  }
  std::vector<uint16_t> comp_tgt(h.comp_tgt.begin(), h.comp_tgt.end());
  P->off.co = push(blob, comp_rng);
  P->off.ctg = push(blob, comp_tgt);
  P->off.m1t = push(blob, h.m1_t);
  P->off.m1o = push(blob, h.m1_off);
  P->off.m1g = push(blob, h.m1_tgt);
  P->off.tco = push(blob, h.tgt_causal_off);
  P->off.tca = push(blob, h.tgt_causal);
  P->off.sc = push(blob, h.slot_const);
  P->off.po = push(blob, h.par_off);
  P->off.pa = push(blob, h.par);
  P->off.lo = push(blob, h.lvl_off);
  P->off.lr = push(blob, h.lvl_rec);
  P->off.go = push(blob, h.gat_off);
  P->off.gr = push(blob, h.gat_rec);
  P->off.pe = push(blob, h.post_events);
  P->off.dn = push(blob, dn);
  P->off.dc = push(blob, h.dense_causal);
  P->off.plc = push(blob, h.plain_const);
  P->off.plo = push(blob, h.plain_off);
  P->off.pls = push(blob, h.plain_sym);
}

void bind_plan(const symft_plan* P, unsigned char* base, DevPlan* dptr) {
  const HostPlan& h = P->hp;
  auto at = [&](size_t off) { return base + off; };
  DevPlan& d = *dptr;
  d.n_channels = h.n_channels;
  d.ch = reinterpret_cast<const ChannelDev*>(at(P->off.ch));
  d.theta4 = reinterpret_cast<const uint4*>(at(P->off.t4));
  d.n_qtab = static_cast<uint32_t>(h.qtabs.size());
  d.n_ctab = static_cast<uint32_t>(h.ctabs.size());
  d.qtheta = reinterpret_cast<const uint32_t*>(at(P->off.q));
  d.qinv = reinterpret_cast<const float*>(at(P->off.qi));
  d.ctabs = reinterpret_cast<const CellTableDev*>(at(P->off.ct));
  d.comp_rng = reinterpret_cast<const uint32_t*>(at(P->off.co));
  d.comp_tgt = reinterpret_cast<const uint16_t*>(at(P->off.ctg));
  d.n_m1 = static_cast<uint32_t>(h.m1_t.size());
  d.m1_t = reinterpret_cast<const uint32_t*>(at(P->off.m1t));
  d.m1_off = reinterpret_cast<const uint32_t*>(at(P->off.m1o));
  d.m1_tgt = reinterpret_cast<const uint32_t*>(at(P->off.m1g));
  d.n_targets = h.n_targets;
  d.tgt_det0 = h.tgt_det0;
  d.tgt_obs0 = h.tgt_obs0;
  d.tgt_sign0 = h.tgt_sign0;
  d.n_slots = h.n_slots;
  d.slot_const = reinterpret_cast<const uint8_t*>(at(P->off.sc));
  d.par_off = reinterpret_cast<const uint32_t*>(at(P->off.po));
  d.par = reinterpret_cast<const uint32_t*>(at(P->off.pa));
  d.n_levels = h.lvl_off.empty() ? 0 : static_cast<uint32_t>(h.lvl_off.size() - 1);
  d.lvl_off = reinterpret_cast<const uint32_t*>(at(P->off.lo));
  d.lvl_rec = reinterpret_cast<const uint32_t*>(at(P->off.lr));
  d.gat_off = reinterpret_cast<const uint32_t*>(at(P->off.go));
  d.gat_rec = reinterpret_cast<const uint32_t*>(at(P->off.gr));
  d.tgt_causal_off = reinterpret_cast<const uint32_t*>(at(P->off.tco));
  d.tgt_causal = reinterpret_cast<const uint32_t*>(at(P->off.tca));
  d.n_post_events = static_cast<uint32_t>(h.post_events.size());
  d.post_events = reinterpret_cast<const int32_t*>(at(P->off.pe));
  d.n_dense = static_cast<uint32_t>(h.dense.size());
  d.dense = reinterpret_cast<const DenseInstrDev*>(at(P->off.dn));
  d.dense_causal = reinterpret_cast<const uint32_t*>(at(P->off.dc));
  d.n_m3 = h.n_m3;
  d.n_records = h.n_records;
  d.n_dets = h.n_dets;
  d.n_obs = h.n_obs;
  d.postselect = h.postselect;
  d.n_comp = h.n_comp;
  d.plain_const = reinterpret_cast<const uint8_t*>(at(P->off.plc));
  d.plain_off = reinterpret_cast<const uint32_t*>(at(P->off.plo));
  d.plain_sym = reinterpret_cast<const uint32_t*>(at(P->off.pls));
}

}  // namespace symft

namespace {

cudaError_t upload(symft_plan* P) {
  cudaError_t e = P->plan_buf.ensure(P->blob.size());
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(P->plan_buf.ptr, P->blob.data(), P->blob.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  bind_plan(P, static_cast<unsigned char*>(P->plan_buf.ptr), &P->dp);
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  P->device = dev;
  e = cudaDeviceGetAttribute(&P->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  P->uploaded = true;
  return cudaSuccess;
}

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess)                                                               \
      return set_error(_e == cudaErrorMemoryAllocation ? SYMFT_E_NOMEM : SYMFT_E_CUDA,   \
                       std::string(#expr) + ": " + cudaGetErrorString(_e));              \
  } while (0)

int sample_impl(symft_plan* P, const symft_sample_args* a) {
  const HostPlan& h = P->hp;
  if (a->shots == 0) return set_error(SYMFT_E_ARG, "shots must be >= 1");
  if (a->shot_offset % kNoiseBlock) return set_error(SYMFT_E_ARG, "shot_offset must be a multiple of 128");
  if (a->shots + a->shot_offset > (1ull << 39)) return set_error(SYMFT_E_ARG, "shot index beyond 2^39");
  if (a->precision != SYMFT_FP32 && a->precision != SYMFT_FP64) return set_error(SYMFT_E_ARG, "bad precision");
  if (a->out_location != SYMFT_OUT_DEVICE && a->out_location != SYMFT_OUT_HOST)
    return set_error(SYMFT_E_ARG, "bad out_location");
  cudaStream_t st = static_cast<cudaStream_t>(a->stream);
  if (!P->uploaded) {
    try {
      CUDA_TRY(upload(P));
    } catch (const Error& e) {
      return set_error(e.code, e.what());
    }
  }
  int launches = 0;
  const uint64_t W = (a->shots + 63) / 64;
  const uint64_t nblk = (a->shots + kNoiseBlock - 1) / kNoiseBlock;
  const bool host = a->out_location == SYMFT_OUT_HOST;

  uint64_t *meas = a->meas_out, *det = a->det_out, *obs = a->obs_out, *disc = a->discard_out;
  if (host) {
    if (meas) { CUDA_TRY(P->h_meas.ensure(std::max<uint64_t>(1, h.n_records * W) * 8)); meas = (uint64_t*)P->h_meas.ptr; }
    if (det) { CUDA_TRY(P->h_det.ensure(std::max<uint64_t>(1, h.n_dets * W) * 8)); det = (uint64_t*)P->h_det.ptr; }
    if (obs) { CUDA_TRY(P->h_obs.ensure(std::max<uint64_t>(1, h.n_obs * W) * 8)); obs = (uint64_t*)P->h_obs.ptr; }
    if (disc) { CUDA_TRY(P->h_disc.ensure(W * 8)); disc = (uint64_t*)P->h_disc.ptr; }
  }
  if (h.n_records == 0) meas = nullptr;
  if (h.n_dets == 0) det = nullptr;
  if (h.n_obs == 0) obs = nullptr;
  const bool need_final = h.n_m3 > 0 || h.postselect || disc != nullptr;
  if (h.postselect && det == nullptr && h.n_dets > 0) {
    CUDA_TRY(P->det_scratch.ensure(h.n_dets * W * 8));
    det = static_cast<uint64_t*>(P->det_scratch.ptr);
  }
  const uint32_t G = static_cast<uint32_t>(h.dense.size());
  uint64_t* signs = nullptr;
  if (G) {
    CUDA_TRY(P->signs.ensure(G * W * 8));
    signs = static_cast<uint64_t*>(P->signs.ptr);
  }
  CUDA_TRY(P->status.ensure(16));
  int* status = static_cast<int*>(P->status.ptr);
  if (a->check) CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));

  // --- plain form: one CTA per shot -----------------------------------------
  if (a->plain) {
    const bool fp64 = a->precision == SYMFT_FP64;
    if (plain_smem_bytes(P->dp, h.k_max, fp64) > 200 * 1024)
      return set_error(SYMFT_E_CAPACITY, "plain form: per-shot state exceeds shared memory");
    if (meas) CUDA_TRY(cudaMemsetAsync(meas, 0, h.n_records * W * 8, st));
    if (det) CUDA_TRY(cudaMemsetAsync(det, 0, h.n_dets * W * 8, st));
    if (obs) CUDA_TRY(cudaMemsetAsync(obs, 0, h.n_obs * W * 8, st));
    if (disc) CUDA_TRY(cudaMemsetAsync(disc, 0, W * 8, st));
    PlainArgs pa{};
    pa.p = P->dp;
    pa.seed = a->seed;
    pa.shot0 = a->shot_offset;
    pa.shots = a->shots;
    pa.W = W;
    pa.meas = meas;
    pa.det = det;
    pa.obs = obs;
    pa.discard = disc;
    pa.kmax = h.k_max;
    pa.status = status;
    const uint64_t cap = static_cast<uint64_t>(P->sm_count) * 16;
    CUDA_TRY(launch_plain(pa, fp64, static_cast<int>(std::max<uint64_t>(1, std::min<uint64_t>(a->shots, cap))), st));
    ++launches;
  }
  // --- sign kernel ---------------------------------------------------------
  if (!a->plain && h.n_slots > 0) {
    SignArgs s{};
    s.p = P->dp;
    s.seed = a->seed;
    s.block0 = a->shot_offset / kNoiseBlock;
    s.n_blocks = nblk;
    s.W = W;
    s.shots = a->shots;
    s.meas = meas;
    s.det = det;
    s.obs = obs;
    s.signs = signs;
    s.status = status;
    const size_t smem = sign_smem_bytes(P->dp);
    if (smem > 220 * 1024)
      return set_error(SYMFT_E_CAPACITY, "too many bit-packed slots for shared memory (" +
                                             std::to_string(h.n_slots) + ")");
    const int nb_cta = sign_blocks_per_cta(P->dp);
    const uint64_t chunks = (nblk + nb_cta - 1) / nb_cta;
    int per_sm = 1;
    CUDA_TRY(sign_occupancy(P->dp, &per_sm));
    uint64_t cap = static_cast<uint64_t>(P->sm_count) * std::max(1, per_sm);
    int grid = static_cast<int>(std::max<uint64_t>(1, std::min(chunks, cap)));
    CUDA_TRY(launch_sign(s, grid, st));
    ++launches;
  }
  // --- dense kernel --------------------------------------------------------
  if (!a->plain && G) {
    const bool fp64 = a->precision == SYMFT_FP64;
    CUDA_TRY(P->m3.ensure(std::max<uint64_t>(1, h.n_m3 * W) * 8));
    if (h.n_m3) CUDA_TRY(cudaMemsetAsync(P->m3.ptr, 0, h.n_m3 * W * 8, st));
    DenseArgs d{};
    d.p = P->dp;
    d.seed = a->seed;
    d.shot0 = a->shot_offset;
    d.shots = a->shots;
    d.W = W;
    d.signs = signs;
    d.m3_out = static_cast<uint64_t*>(P->m3.ptr);
    d.kmax = h.k_max;
    d.status = status;
    const size_t amp = fp64 ? 16 : 8;
    const size_t m3bytes = ((h.n_m3 + 31) / 32) * 4;
    const size_t vec_bytes = (static_cast<size_t>(1) << h.k_max) * amp;
    int wpb = 4;
    size_t smem;
    if (vec_bytes + m3bytes <= 48 * 1024) {
      wpb = static_cast<int>(std::min<size_t>(8, std::max<size_t>(1, (160 * 1024) / (vec_bytes + m3bytes + 16))));
      d.use_smem = 1;
      smem = ((wpb * m3bytes + 15) & ~size_t(15)) + wpb * vec_bytes;
    } else {
      d.use_smem = 0;
      smem = wpb * m3bytes + 16;
    }
    if (h.k_max <= 5 && dense_reg_smem_bytes(P->dp) <= 96 * 1024) {
      // register-resident form: lane x holds amplitude x
      const uint64_t want_r = (a->shots + 7) / 8;
      const uint64_t cap_r = static_cast<uint64_t>(P->sm_count) * 8;
      CUDA_TRY(launch_dense_reg(d, fp64, static_cast<int>(std::max<uint64_t>(1, std::min(want_r, cap_r))), st));
      ++launches;
      goto dense_done;
    }
    if (!d.use_smem) {
      // large k: one CTA per shot, vector in shared memory up to ~200 KB, else a
      // global slot per resident CTA (sized to stay L2-resident)
      const bool in_smem = dense_cta_smem_bytes(P->dp, vec_bytes, true) <= 200 * 1024;
      const size_t csmem = dense_cta_smem_bytes(P->dp, vec_bytes, in_smem);
      int grid_c = P->sm_count * (in_smem ? 1 : 2);
      grid_c = static_cast<int>(std::max<uint64_t>(1, std::min<uint64_t>(a->shots, grid_c)));
      d.use_smem = in_smem ? 1 : 0;
      if (!in_smem) {
        d.gvec_stride = static_cast<uint64_t>(1) << h.k_max;
        CUDA_TRY(P->gvec.ensure(static_cast<size_t>(grid_c) * vec_bytes));
        d.gvec = P->gvec.ptr;
      }
      CUDA_TRY(launch_dense_cta(d, fp64, grid_c, csmem, st));
      ++launches;
      goto dense_done;
    }
    {
    uint64_t want = (a->shots + wpb - 1) / wpb;
    uint64_t cap = static_cast<uint64_t>(P->sm_count) * (d.use_smem ? 16 : 8);
    if (!d.use_smem) {
      // bound the global-memory vectors to ~8 GB of resident warp slots
      uint64_t max_warps = std::max<uint64_t>(1, (8ull << 30) / vec_bytes);
      cap = std::min<uint64_t>(cap, std::max<uint64_t>(1, max_warps / wpb));
    }
    int grid = static_cast<int>(std::max<uint64_t>(1, std::min(want, cap)));
    if (!d.use_smem) {
      d.gvec_stride = static_cast<uint64_t>(1) << h.k_max;
      CUDA_TRY(P->gvec.ensure(static_cast<size_t>(grid) * wpb * vec_bytes));
      d.gvec = P->gvec.ptr;
    }
    CUDA_TRY(launch_dense(d, fp64, wpb, grid, smem, st));
    ++launches;
    }
  dense_done:;
  }
  // --- finalize ------------------------------------------------------------
  if (!a->plain && need_final) {
    FinalArgs f{};
    f.p = P->dp;
    f.W = W;
    f.shots = a->shots;
    f.m3 = h.n_m3 ? static_cast<const uint64_t*>(P->m3.ptr) : nullptr;
    f.meas = meas;
    f.det = det;
    f.obs = obs;
    f.discard = disc;
    CUDA_TRY(launch_finalize(f, st));
    ++launches;
  }
  if (host) {
    if (a->meas_out && meas) CUDA_TRY(cudaMemcpyAsync(a->meas_out, meas, h.n_records * W * 8, cudaMemcpyDeviceToHost, st));
    if (a->det_out && det) CUDA_TRY(cudaMemcpyAsync(a->det_out, det, h.n_dets * W * 8, cudaMemcpyDeviceToHost, st));
    if (a->obs_out && obs) CUDA_TRY(cudaMemcpyAsync(a->obs_out, obs, h.n_obs * W * 8, cudaMemcpyDeviceToHost, st));
    if (a->discard_out && disc) CUDA_TRY(cudaMemcpyAsync(a->discard_out, disc, W * 8, cudaMemcpyDeviceToHost, st));
  }
  g_last_launches = launches;
  if (host || a->check) CUDA_TRY(cudaStreamSynchronize(st));
  if (a->check) {
    int hs = 0;
    CUDA_TRY(cudaMemcpy(&hs, status, sizeof(int), cudaMemcpyDeviceToHost));
    if (hs != 0) return set_error(SYMFT_E_DEVICE, "device status " + std::to_string(hs));
  }
  return SYMFT_OK;
}

}  // namespace

extern "C" {

int symft_compile_ex(const char* text, const symft_options* opt, symft_plan** out) {
  g_last_error.clear();
  if (!text || !out) return set_error(SYMFT_E_ARG, "null argument");
  *out = nullptr;
  symft_options o{};
  if (opt) o = *opt;
  if (o.postselect != SYMFT_POSTSELECT_NONE && o.postselect != SYMFT_POSTSELECT_ALL)
    return set_error(SYMFT_E_ARG, "bad postselect mode");
  try {
    Circuit c = parse_circuit(text);
    symft_plan* p = new symft_plan();
    try {
      p->hp = compile_plan(c, o);
      build_blob(p);
    } catch (...) {
      delete p;
      throw;
    }
    *out = p;
    return SYMFT_OK;
  } catch (const Error& e) {
    return set_error(e.code, e.what());
  } catch (const std::bad_alloc&) {
    return set_error(SYMFT_E_NOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return set_error(SYMFT_E_PARSE, e.what());
  }
}

int symft_compile(const char* text, symft_plan** out) { return symft_compile_ex(text, nullptr, out); }

int symft_plan_info(const symft_plan* p, symft_info* info) {
  if (!p || !info) return set_error(SYMFT_E_ARG, "null argument");
  const HostPlan& h = p->hp;
  std::memset(info, 0, sizeof(*info));
  info->n_qubits = h.n_qubits;
  info->n_meas_events = h.n_meas;
  info->n_records = h.n_records;
  info->n_dets = h.n_dets;
  info->n_obs = h.n_obs;
  info->n_channels = h.n_channels;
  info->k_max = h.k_max;
  for (int i = 0; i < 7; ++i) info->n_instr[i] = h.hist[i];
  info->max_expr_weight = h.max_expr_weight;
  info->n_noise_components = h.n_comp;
  info->n_targets = h.n_slots;
  info->n_causal = h.n_m3;
  info->sign_xor_terms = h.sign_xor_terms;
  return SYMFT_OK;
}

void symft_plan_free(symft_plan* p) {
  if (!p) return;
  p->plan_buf.release();
  p->signs.release();
  p->m3.release();
  p->det_scratch.release();
  p->gvec.release();
  p->status.release();
  p->h_meas.release();
  p->h_det.release();
  p->h_obs.release();
  p->h_disc.release();
  delete p;
}

int symft_sample_ex(const symft_plan* plan, const symft_sample_args* args) {
  g_last_error.clear();
  g_last_launches = 0;
  if (!plan || !args) return set_error(SYMFT_E_ARG, "null argument");
  symft_plan* P = const_cast<symft_plan*>(plan);
  std::lock_guard<std::mutex> lk(P->mu);
  try {
    return sample_impl(P, args);
  } catch (const std::bad_alloc&) {
    return set_error(SYMFT_E_NOMEM, "host allocation failed");
  }
}

int symft_sample(const symft_plan* plan, uint64_t shots, uint64_t seed, uint64_t* meas_out,
                 uint64_t* det_out, uint64_t* obs_out, void* stream) {
  symft_sample_args a{};
  a.shots = shots;
  a.seed = seed;
  a.meas_out = meas_out;
  a.det_out = det_out;
  a.obs_out = obs_out;
  a.stream = stream;
  return symft_sample_ex(plan, &a);
}

const char* symft_last_error(void) { return g_last_error.c_str(); }

int symft_last_launch_count(void) { return g_last_launches; }

}  // extern "C"
