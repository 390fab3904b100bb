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

// the warp executor runs two shots per warp (16 lanes each) up to this k_max
// (measured: k = 8 circuits 1.3-1.7x faster, k = 10 slower; four shots per
// warp slower at k = 8)
constexpr uint32_t kWarpPairMaxK = 8;

static_assert(kNoiseBlock == SYMFT_SHOT_ALIGN, "shot alignment is the noise block");

void build_blob(symft_plan* P) {
  const HostPlan& h = P->hp;
  std::vector<ChannelDev> ch(h.n_channels);
  for (uint32_t c = 0; c < h.n_channels; ++c)
    ch[c] = ChannelDev{h.ch_theta_last[c], h.ch_qtab[c], h.ch_ctab[c], h.ch_comp0[c], h.ch_cell0[c]};
  std::vector<uint32_t> theta4(((h.n_channels + 3) / 4) * 4, 0u);
  for (uint32_t c = 0; c < h.n_channels; ++c) theta4[c] = h.ch_theta_last[c];
  std::vector<uint32_t> qtheta, qshift;
  std::vector<uint16_t> qstart;
  for (auto& q : h.qtabs) {
    qtheta.insert(qtheta.end(), q.theta, q.theta + kNoiseBlock);
    // lane-search buckets (plan_dev.hpp, kQBuckets)
    const uint32_t last = q.theta[kNoiseBlock - 1];
    uint32_t sh = 0;
    while (sh < 32 && (static_cast<uint64_t>(last) >> sh) >= static_cast<uint64_t>(kQBuckets)) ++sh;
    qshift.push_back(sh);
    uint32_t j = 0;
    for (uint32_t i = 0; i < static_cast<uint32_t>(kQBuckets); ++i) {
      const uint64_t lo = static_cast<uint64_t>(i) << sh;
      while (j < static_cast<uint32_t>(kNoiseBlock) && q.theta[j] <= lo) ++j;
      qstart.push_back(static_cast<uint16_t>(j));
    }
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
    o.cf = static_cast<float>(d.c);
    o.sf = static_cast<float>(d.s);
    o.sign_target_col = d.sign_target - h.n_records;
    o.causal_off = d.causal_off;
    o.causal_n = d.causal_n;
    o.t = d.t;
    o.post_grp = kNoGroup;
    o.pad = 0;
  }
  // early exit only where it can pay: after an active measurement whose
  // detector group is not empty and with at least kEarlyExitWork amplitudes
  // of dense work still to come (below that the check costs more than it saves)
  {
    constexpr uint64_t kEarlyExitWork = 1024;
    std::vector<uint64_t> rest(dn.size() + 1, 0);
    for (size_t g = dn.size(); g-- > 0;) rest[g] = rest[g + 1] + (1ull << dn[g].k);
    const bool ps = h.postselect && !h.post_chk.empty();
    for (size_t g = 0; g < dn.size(); ++g) {
      if (!ps || (dn[g].kind != I_ACTIVE_DIAG_MEAS && dn[g].kind != I_ACTIVE_PAIR_MEAS)) continue;
      const uint32_t q = static_cast<uint32_t>(dn[g].m3) + 1;
      if (h.post_chk_off[q + 1] > h.post_chk_off[q] && rest[g + 1] >= kEarlyExitWork) dn[g].post_grp = q;
    }
    P->post_grp0 = (ps && h.post_chk_off[1] > h.post_chk_off[0] && rest[0] >= kEarlyExitWork) ? 0u : kNoGroup;
  }
  P->dense_host = dn;
  std::vector<unsigned char>& blob = P->blob;
  blob.clear();
  P->off.ch = push(blob, ch);
  P->off.q = push(blob, qtheta);
  P->off.ct = push(blob, ct);
  P->off.t4 = push(blob, theta4);
  P->off.qi = push(blob, qshift);
  P->off.qs = push(blob, qstart);
  if (h.n_slots >= 65536) throw Error(SYMFT_E_CAPACITY, "more than 65535 bit-packed slots");
  if (h.n_channels >= (1u << 28)) throw Error(SYMFT_E_CAPACITY, "too many noise channels");
  // (channel, cell) target entries: up to 7 word offsets inline, else a list
  const size_t n_cells = h.cell_off.size() - 1;
  std::vector<uint4> cellt(std::max<size_t>(1, n_cells));
  std::vector<uint32_t> cell_ovf;
  for (size_t e = 0; e < n_cells; ++e) {
    const uint32_t off = h.cell_off[e], n = h.cell_off[e + 1] - off;
    bool inl = n <= 7;
    for (uint32_t j = 0; j < n && inl; ++j) inl = h.cell_tgt[off + j] < 4096;
    uint16_t f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (inl) {
      f[0] = static_cast<uint16_t>(n);
      for (uint32_t j = 0; j < n; ++j) f[1 + j] = static_cast<uint16_t>(h.cell_tgt[off + j] * 16);
      std::memcpy(&cellt[e], f, 16);
    } else {
      cellt[e] = make_uint4(0xFFFFu, static_cast<uint32_t>(cell_ovf.size()), n, 0u);
      for (uint32_t j = 0; j < n; ++j) cell_ovf.push_back(h.cell_tgt[off + j] * 16);
    }
  }
  if (cell_ovf.empty()) cell_ovf.push_back(0);
  P->off.clt = push(blob, cellt);
  P->off.clo = push(blob, cell_ovf);
  P->off.m1t = push(blob, h.m1_t);
  P->off.m1o = push(blob, h.m1_off);
  P->off.m1g = push(blob, h.m1_tgt);
  P->off.tco = push(blob, h.tgt_causal_off);
  P->off.tca = push(blob, h.tgt_causal);
  {
    std::vector<uint4> ctg;
    for (uint32_t i = 0; i + 1 < h.tgt_causal_off.size(); ++i) {
      const uint32_t b = h.tgt_causal_off[i], e = h.tgt_causal_off[i + 1];
      if (e > b) ctg.push_back(make_uint4(i, b, e - b, 0u));
    }
    P->off.n_ctg = static_cast<uint32_t>(ctg.size());
    if (ctg.empty()) ctg.push_back(make_uint4(0u, 0u, 0u, 0u));
    P->off.ctg = push(blob, ctg);
  }
  P->off.sc = push(blob, h.slot_const);
  // slot -> constant and random-measurement sources (inverse of the m1 lists)
  std::vector<uint32_t> sm1_nsrc(h.n_slots, 0);
  {
    std::vector<std::vector<uint32_t>> src(h.n_slots);
    for (size_t j = 0; j < h.m1_t.size(); ++j)
      for (uint32_t q = h.m1_off[j]; q < h.m1_off[j + 1]; ++q) src[h.m1_tgt[q]].push_back(static_cast<uint32_t>(j));
    for (uint32_t i = 0; i < h.n_slots; ++i) sm1_nsrc[i] = static_cast<uint32_t>(src[i].size());
    std::vector<uint4> sm1(std::max<size_t>(1, h.n_slots));
    std::vector<uint32_t> ovf;
    for (uint32_t i = 0; i < h.n_slots; ++i) {
      const uint32_t cbit = h.slot_const[i] ? 0x8000u : 0u;
      const auto& v = src[i];
      bool inl = v.size() <= 7;
      for (uint32_t j : v) inl = inl && j < 65536;
      uint16_t f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      if (inl) {
        f[0] = static_cast<uint16_t>(v.size() | cbit);
        for (size_t q = 0; q < v.size(); ++q) f[1 + q] = static_cast<uint16_t>(v[q]);
        std::memcpy(&sm1[i], f, 16);
      } else {
        sm1[i] = make_uint4(0x7FFFu | cbit, static_cast<uint32_t>(ovf.size()), static_cast<uint32_t>(v.size()), 0u);
        ovf.insert(ovf.end(), v.begin(), v.end());
      }
    }
    if (ovf.empty()) ovf.push_back(0);
    P->off.sm1 = push(blob, sm1);
    P->off.sm1o = push(blob, ovf);
  }
  // record chains as paths: from each root that has a child, the chain of
  // single children (the compile step gives every record at most one parent
  // and at most one child)
  {
    std::vector<int64_t> child(h.n_records, -1);
    for (uint32_t r = 0; r < h.n_records; ++r) {
      const uint32_t np = h.par_off[r + 1] - h.par_off[r];
      if (np > 1) throw Error(SYMFT_E_DEVICE, "internal: a record with more than one parent");
      if (np == 1) {
        const uint32_t pa = h.par[h.par_off[r]];
        if (child[pa] >= 0) throw Error(SYMFT_E_DEVICE, "internal: a record with more than one child");
        child[pa] = r;
      }
    }
    // 16 fields of 16 bits per path (two 16-byte items), unused ones 0xFFFF
    std::vector<uint16_t> ids;
    for (uint32_t r = 0; r < h.n_records; ++r) {
      if (h.par_off[r + 1] != h.par_off[r] || child[r] < 0) continue;
      const size_t x = ids.size();
      ids.resize(x + kMaxLevels, 0xFFFFu);
      size_t n = 0;
      for (int64_t q = r; q >= 0; q = child[q], ++n) {
        if (n == static_cast<size_t>(kMaxLevels) || q >= 0xFFFF)
          throw Error(SYMFT_E_DEVICE, "internal: a record chain path of more than 16 records or a record index "
                                      "beyond 16 bits");
        ids[x + n] = static_cast<uint16_t>(q);
      }
    }
    P->off.n_pth = static_cast<uint32_t>(ids.size() / kMaxLevels);
    if (ids.empty()) ids.resize(kMaxLevels, 0xFFFFu);
    P->off.pid = push(blob, ids);
  }
  // detector / observable gathers: up to seven records inline, else a list
  const size_t n_gat = h.gat_off.size() - 1;
  std::vector<uint4> gat_item(std::max<size_t>(1, n_gat));
  std::vector<uint32_t> gat_ovf;
  for (size_t j = 0; j < n_gat; ++j) {
    const uint32_t off = h.gat_off[j], n = h.gat_off[j + 1] - off;
    uint16_t f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (n <= 7) {
      f[0] = static_cast<uint16_t>(n);
      for (uint32_t q = 0; q < n; ++q) f[1 + q] = static_cast<uint16_t>(h.gat_rec[off + q]);
      std::memcpy(&gat_item[j], f, 16);
    } else {
      gat_item[j] = make_uint4(0xFFFFu, static_cast<uint32_t>(gat_ovf.size()), n, 0u);
      for (uint32_t q = 0; q < n; ++q) gat_ovf.push_back(h.gat_rec[off + q]);
    }
  }
  if (gat_ovf.empty()) gat_ovf.push_back(0);
  // slots that do not start at zero
  {
    std::vector<uint32_t> nz;
    for (uint32_t i = 0; i < h.n_slots; ++i)
      if (h.slot_const[i] || sm1_nsrc[i]) nz.push_back(i);
    P->off.n_snz = static_cast<uint32_t>(nz.size());
    if (nz.empty()) nz.push_back(0);
    P->off.snz = push(blob, nz);
  }
  // outputs that equal one slot before the record chains (exo(b) = delta_b ^
  // exo(a) when a is b's only parent, so exo(a) ^ exo(b) = delta_b), and the rest
  {
    std::vector<uint2> dl;
    std::vector<uint32_t> rest;
    auto npar = [&](uint32_t r) { return h.par_off[r + 1] - h.par_off[r]; };
    for (uint32_t j = 0; j < n_gat; ++j) {
      const uint32_t off = h.gat_off[j], n = h.gat_off[j + 1] - off;
      int64_t slot = -1;
      if (n == 1 && npar(h.gat_rec[off]) == 0) {
        slot = h.gat_rec[off];
      } else if (n == 2) {
        const uint32_t a = std::min(h.gat_rec[off], h.gat_rec[off + 1]);
        const uint32_t b = std::max(h.gat_rec[off], h.gat_rec[off + 1]);
        if (npar(b) == 1 && h.par[h.par_off[b]] == a) slot = b;
      }
      if (slot >= 0) dl.push_back(make_uint2(j, static_cast<uint32_t>(slot)));
      else rest.push_back(j);
    }
    P->off.n_odl = static_cast<uint32_t>(dl.size());
    P->off.n_ors = static_cast<uint32_t>(rest.size());
    if (dl.empty()) dl.push_back(make_uint2(0u, 0u));
    if (rest.empty()) rest.push_back(0);
    P->off.odl = push(blob, dl);
    P->off.ors = push(blob, rest);
  }
  P->off.m3t = push(blob, h.m3_t);
  P->off.pco = push(blob, h.post_chk_off);
  P->off.pch = push(blob, h.post_chk);
  P->off.gi = push(blob, gat_item);
  P->off.gv = push(blob, gat_ovf);
  P->off.pe = push(blob, h.post_events);
  P->off.dn = push(blob, dn);
  P->off.pc = push(blob, h.pc.ops);
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
  d.qshift = reinterpret_cast<const uint32_t*>(at(P->off.qi));
  d.qstart = reinterpret_cast<const uint16_t*>(at(P->off.qs));
  d.ctabs = reinterpret_cast<const CellTableDev*>(at(P->off.ct));
  d.cellt = reinterpret_cast<const CellTargetsDev*>(at(P->off.clt));
  d.cell_ovf = reinterpret_cast<const uint32_t*>(at(P->off.clo));
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
  d.slot_m1 = reinterpret_cast<const uint4*>(at(P->off.sm1));
  d.slot_m1_ovf = reinterpret_cast<const uint32_t*>(at(P->off.sm1o));
  d.n_paths = P->off.n_pth;
  d.path_ids = reinterpret_cast<const uint4*>(at(P->off.pid));
  d.m3_t = reinterpret_cast<const uint32_t*>(at(P->off.m3t));
  const bool early = h.postselect && !h.post_chk.empty();
  d.post_chk_off = early ? reinterpret_cast<const uint32_t*>(at(P->off.pco)) : nullptr;
  d.post_chk = early ? reinterpret_cast<const uint32_t*>(at(P->off.pch)) : nullptr;
  d.post_grp0 = P->post_grp0;
  d.gat_item = reinterpret_cast<const uint4*>(at(P->off.gi));
  d.gat_ovf = reinterpret_cast<const uint32_t*>(at(P->off.gv));
  d.n_slot_nz = P->off.n_snz;
  d.slot_nz = reinterpret_cast<const uint32_t*>(at(P->off.snz));
  d.n_out_delta = P->off.n_odl;
  d.n_out_rest = P->off.n_ors;
  d.out_delta = reinterpret_cast<const uint2*>(at(P->off.odl));
  d.out_rest = reinterpret_cast<const uint32_t*>(at(P->off.ors));
  d.tgt_causal_off = reinterpret_cast<const uint32_t*>(at(P->off.tco));
  d.tgt_causal = reinterpret_cast<const uint32_t*>(at(P->off.tca));
  d.n_causal_tgt = P->off.n_ctg;
  d.causal_tgt = reinterpret_cast<const uint4*>(at(P->off.ctg));
  d.n_post_events = static_cast<uint32_t>(h.post_events.size());
  d.post_events = reinterpret_cast<const int32_t*>(at(P->off.pe));
  d.n_dense = static_cast<uint32_t>(h.dense.size());
  d.dense = reinterpret_cast<const DenseInstrDev*>(at(P->off.dn));
  d.n_pc = static_cast<uint32_t>(h.pc.ops.size());
  d.pc = reinterpret_cast<const PCOp*>(at(P->off.pc));
  d.pc_capacity = h.pc.capacity;
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

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Whether dense executor `kind` (1 register, 2 warp with the vector in shared
// memory, 3 CTA with the vector in shared memory, 4 wide with vectors in HBM,
// 5 warp running the product-component program, 6 CTA running it with the
// workspace in shared memory) can run this plan at this precision.
bool dense_kind_valid(const symft_plan* P, const HostPlan& h, bool fp64, int kind) {
  const size_t amp = fp64 ? 16 : 8;
  const size_t m3bytes = ((h.n_m3 + 31) / 32) * 4;
  const size_t vec_bytes = (static_cast<size_t>(1) << h.k_max) * amp;
  switch (kind) {
    case 1: return h.k_max >= 1 && h.k_max <= 5 && dense_reg_smem_bytes(P->dp) <= 96 * 1024;
    case 2: return vec_bytes + m3bytes <= 48 * 1024 && dense_warp_smem_bytes(P->dp, 1, vec_bytes, true) <= 200 * 1024;
    case 3: return dense_cta_smem_bytes(P->dp, vec_bytes, true) <= 200 * 1024;
    case 4: return true;
    case 5: return !h.pc.ops.empty() && h.pc.capacity <= (1u << 22);
    case 6: return !h.pc.ops.empty() &&
                   dense_cta_smem_bytes(P->dp, static_cast<size_t>(h.pc.capacity) * amp, true) <= 200 * 1024;
  }
  return false;
}

// The executor for a plan: the tuned choice when it is valid, else the
// product-component executor on one warp per shot when its cost model
// selected it (measured faster than one CTA per shot on the component
// programs here: a CTA pays a barrier per op on mostly small components), else
// the first valid kind in the order register, warp, CTA, wide (smallest
// footprint first).
int dense_kind_for(const symft_plan* P, const HostPlan& h, bool fp64, int tuned) {
  if (tuned && dense_kind_valid(P, h, fp64, tuned)) return tuned;
  if (h.pc.use && dense_kind_valid(P, h, fp64, 5)) return 5;
  for (int k = 1; k <= 4; ++k)
    if (dense_kind_valid(P, h, fp64, k)) return k;
  return 4;
}

// Launch shapes and workspace pointers of one sampling request.  prepare()
// allocates and decides everything on the host; enqueue() only issues
// memsets and kernel launches, so it can also run inside a stream capture.
struct Prep {
  uint64_t W = 0, nblk = 0, shots = 0;
  bool plain = false, fp64 = false, need_final = false;
  uint64_t *meas = nullptr, *det = nullptr, *obs = nullptr, *disc = nullptr;
  uint64_t *signs = nullptr, *m3 = nullptr;
  double* prob = nullptr;
  uint64_t* counts = nullptr;
  int* status = nullptr;
  int sign_grid = 0;
  int dense_kind = 0;   // 0 none, 1 register, 2 warp, 3 CTA per shot, 4 wide (HBM)
  int dense_grid = 0, dense_wpb = 0, dense_use_smem = 0;
  size_t dense_smem = 0;
  void* gvec = nullptr;
  uint64_t gvec_stride = 0;
  int plain_grid = 0;
  // wide executor: batch size and workspace pieces
  uint32_t wide_nb = 0;
  uint32_t wide_tile_bits = 0;   // 0: the executor's default
  int dense_spw = 1;             // warp executor: shots per warp
  void* wide_vec[2] = {nullptr, nullptr};
  uint32_t* wide_m3b = nullptr;
  uint8_t* wide_lam = nullptr;
  double* wide_sums = nullptr;
  double* wide_scale = nullptr;
  float* wide_scalef = nullptr;
  uint8_t* wide_lab = nullptr;
  uint8_t* wide_alive = nullptr;
};

int validate(const symft_sample_args* a) {
  if (a->shots == 0) return set_error(SYMFT_E_ARG, "shots must be >= 1");
  if (a->shot_offset % kNoiseBlock)
    return set_error(SYMFT_E_ARG, "shot_offset must be a multiple of " + std::to_string(kNoiseBlock));
  if (a->shots + a->shot_offset > (1ull << 39)) return set_error(SYMFT_E_ARG, "shot index beyond 2^39");
  if (a->precision != SYMFT_FP32 && a->precision != SYMFT_FP64) return set_error(SYMFT_E_ARG, "bad precision");
  if (a->out_location != SYMFT_OUT_DEVICE && a->out_location != SYMFT_OUT_HOST)
    return set_error(SYMFT_E_ARG, "bad out_location");
  if (a->plain != SYMFT_PLAIN_OFF && a->plain != SYMFT_PLAIN_IN_KERNEL && a->plain != SYMFT_PLAIN_PREPASS)
    return set_error(SYMFT_E_ARG, "bad plain form");
  return SYMFT_OK;
}

// outputs: the device pointers the kernels write (caller's or host staging)
int prepare(symft_plan* P, const symft_sample_args* a, uint64_t* meas, uint64_t* det, uint64_t* obs,
            uint64_t* disc, double* prob, uint64_t* counts, Prep* o) {
  const HostPlan& h = P->hp;
  if (!P->uploaded) {
    try {
      CUDA_TRY(upload(P));
    } catch (const Error& e) {
      return set_error(e.code, e.what());
    }
  }
  CUDA_TRY(set_smem_limits());
  const Tune& t = P->tune[a->precision == SYMFT_FP64 ? 1 : 0];
  o->W = (a->shots + 63) / 64;
  o->shots = a->shots;
  o->nblk = (a->shots + kNoiseBlock - 1) / kNoiseBlock;
  o->plain = a->plain == SYMFT_PLAIN_IN_KERNEL;
  o->fp64 = a->precision == SYMFT_FP64;
  const uint64_t W = o->W;
  if (h.n_records == 0) meas = nullptr;
  if (h.n_dets == 0) det = nullptr;
  if (h.n_obs == 0) obs = nullptr;
  if (h.postselect && det == nullptr && h.n_dets > 0) {
    CUDA_TRY(P->det_scratch.ensure(h.n_dets * W * 8));
    det = static_cast<uint64_t*>(P->det_scratch.ptr);
  }
  if (counts) {   // the tallies read the observable and discard columns
    if (h.n_obs && obs == nullptr) {
      CUDA_TRY(P->obs_scratch.ensure(h.n_obs * W * 8));
      obs = static_cast<uint64_t*>(P->obs_scratch.ptr);
    }
    if (h.postselect && disc == nullptr) {
      CUDA_TRY(P->disc_scratch.ensure(W * 8));
      disc = static_cast<uint64_t*>(P->disc_scratch.ptr);
    }
  }
  o->need_final = h.n_m3 > 0 || h.postselect || disc != nullptr;
  o->prob = h.n_m3 ? prob : nullptr;
  o->counts = counts;
  o->meas = meas;
  o->det = det;
  o->obs = obs;
  o->disc = disc;
  const uint32_t G = static_cast<uint32_t>(h.dense.size());
  CUDA_TRY(P->status.ensure(16));
  o->status = static_cast<int*>(P->status.ptr);
  if (o->plain) {
    if (plain_smem_bytes(P->dp, h.k_max, o->fp64) > 200 * 1024)
      return set_error(SYMFT_E_CAPACITY, "plain form: per-shot state exceeds shared memory");
    const uint64_t cap = static_cast<uint64_t>(P->sm_count) * 16;
    o->plain_grid = static_cast<int>(std::max<uint64_t>(1, std::min<uint64_t>(a->shots, cap)));
    return SYMFT_OK;
  }
  if (G) {
    CUDA_TRY(P->signs.ensure(G * W * 8));
    o->signs = static_cast<uint64_t*>(P->signs.ptr);
    CUDA_TRY(P->m3.ensure(std::max<uint64_t>(1, h.n_m3 * W) * 8));
    o->m3 = static_cast<uint64_t*>(P->m3.ptr);
  }
  if (h.n_slots > 0) {
    if (sign_smem_bytes(P->dp) > 220 * 1024)
      return set_error(SYMFT_E_CAPACITY, "too many bit-packed slots for shared memory (" +
                                             std::to_string(h.n_slots) + ")");
    int per_sm = 1;
    CUDA_TRY(sign_occupancy(P->dp, &per_sm));
    if (t.sign_ctas_per_sm > 0) per_sm = std::min(per_sm, t.sign_ctas_per_sm);
    const uint64_t cap = static_cast<uint64_t>(P->sm_count) * std::max(1, per_sm);
    o->sign_grid = static_cast<int>(std::max<uint64_t>(1, std::min(o->nblk, cap)));
  }
  if (G) {
    const size_t amp = o->fp64 ? 16 : 8;
    const size_t m3bytes = ((h.n_m3 + 31) / 32) * 4;
    const size_t vec_bytes = (static_cast<size_t>(1) << h.k_max) * amp;
    if (a->plain == SYMFT_PLAIN_PREPASS) {
      // the paper's GPU design with its device-side prepass: one CTA per shot,
      // the whole vector in shared memory, signs from the packed columns
      if (dense_cta_smem_bytes(P->dp, vec_bytes, true) > 200 * 1024)
        return set_error(SYMFT_E_CAPACITY, "plain prepass form: per-shot vector exceeds shared memory");
      o->dense_kind = 3;
      o->dense_smem = dense_cta_smem_bytes(P->dp, vec_bytes, true);
      o->dense_use_smem = 1;
      const uint64_t cap = static_cast<uint64_t>(P->sm_count) * 16;
      o->dense_grid = static_cast<int>(std::max<uint64_t>(1, std::min<uint64_t>(a->shots, cap)));
    } else if (dense_kind_for(P, h, o->fp64, t.dense_kind) == 6) {
      // product components, one CTA per shot, workspace in shared memory
      o->dense_kind = 6;
      o->dense_smem = dense_cta_smem_bytes(P->dp, static_cast<size_t>(h.pc.capacity) * amp, true);
      o->dense_use_smem = 1;
      const uint64_t cap = static_cast<uint64_t>(P->sm_count) * 8 * t.cta_grid_mult;
      o->dense_grid = static_cast<int>(std::max<uint64_t>(1, std::min<uint64_t>(a->shots, cap)));
    } else if (dense_kind_for(P, h, o->fp64, t.dense_kind) == 5) {
      // product components: one warp per shot, its component workspace in
      // shared memory or in a global slot per warp, whichever keeps more
      // warps resident per SM (the workspaces bound them in shared memory,
      // registers in global memory, where the workspaces of the resident
      // warps mostly stay in L2); a shot is a chain of dependent accesses,
      // so resident warps are what hides their latency
      o->dense_kind = 5;
      const size_t ws_bytes = static_cast<size_t>(h.pc.capacity) * amp;
      const int pi = o->fp64 ? 1 : 0;
      constexpr int kGlobalWpb = 4;
      if (P->pc_wpb[pi] == 0) {
        int best = 0, bw = 1, bc = 0;
        for (int c = 1; c <= 8 && ws_bytes + m3bytes <= 227 * 1024; ++c) {
          const size_t sm = dense_pc_smem_bytes(P->dp, c, ws_bytes, true);
          if (sm > 227 * 1024) break;
          int n = 0;
          CUDA_TRY(dense_pc_occupancy(o->fp64, c, sm, &n));
          if (n * c > best) {
            best = n * c;
            bw = c;
            bc = n;
          }
        }
        int ng = 0;
        CUDA_TRY(dense_pc_occupancy(o->fp64, kGlobalWpb, dense_pc_smem_bytes(P->dp, kGlobalWpb, 0, false), &ng));
        const bool sm = best > 0 && best >= ng * kGlobalWpb;
        P->pc_smem[pi] = sm ? 1 : 0;
        P->pc_wpb[pi] = sm ? bw : kGlobalWpb;
        P->pc_cps[pi] = sm ? bc : ng;
      }
      const bool in_smem = P->pc_smem[pi] != 0;
      int wpb = t.dense_wpb ? t.dense_wpb : P->pc_wpb[pi];
      while (in_smem && wpb > 1 && dense_pc_smem_bytes(P->dp, wpb, ws_bytes, true) > 227 * 1024) --wpb;
      o->dense_wpb = wpb;
      o->dense_use_smem = in_smem ? 1 : 0;
      o->dense_smem = dense_pc_smem_bytes(P->dp, wpb, in_smem ? ws_bytes : 0, in_smem);
      int cps = P->pc_cps[pi];
      if (wpb != P->pc_wpb[pi]) CUDA_TRY(dense_pc_occupancy(o->fp64, wpb, o->dense_smem, &cps));
      // resident CTAs times dense_grid_mult / 8 waves: the default, 8, is one
      // wave of persistent warps (four waves measured no faster, and would
      // hold four times the global workspace slots)
      const uint64_t want = (a->shots + wpb - 1) / wpb;
      const uint64_t cap = static_cast<uint64_t>(P->sm_count) * std::max(1, cps) * std::max(1, t.dense_grid_mult / 8);
      o->dense_grid = static_cast<int>(std::max<uint64_t>(1, std::min(want, cap)));
      if (!in_smem) {
        o->gvec_stride = h.pc.capacity;
        CUDA_TRY(P->gvec.ensure(static_cast<size_t>(o->dense_grid) * wpb * ws_bytes));
        o->gvec = P->gvec.ptr;
      }
    } else if (dense_kind_for(P, h, o->fp64, t.dense_kind) == 1) {
      o->dense_kind = 1;   // register-resident: 32 / 2^k_max segments per warp, lane x of a
                           // shot's segment holds amplitude x (in one or two register sets)
      const uint64_t per_cta = dense_reg_shots_per_cta(h.k_max, o->fp64);
      const uint64_t want = (a->shots + per_cta - 1) / per_cta;
      const uint64_t cap = static_cast<uint64_t>(P->sm_count) * t.dense_grid_mult;
      o->dense_grid = static_cast<int>(std::max<uint64_t>(1, std::min(want, cap)));
    } else if (dense_kind_for(P, h, o->fp64, t.dense_kind) == 2) {
      o->dense_kind = 2;   // vector in shared memory; small vectors two shots per warp (16 lanes each)
      const int spw = h.k_max <= kWarpPairMaxK ? 2 : 1;
      o->dense_spw = spw;
      const size_t bk = dense_warp_smem_bytes(P->dp, 1, 0, false);
      int wpb = t.dense_wpb ? t.dense_wpb
                            : static_cast<int>(std::min<size_t>(8, std::max<size_t>(1, (160 * 1024) / (spw * (vec_bytes + bk + 16)))));
      while (wpb > 1 && dense_warp_smem_bytes(P->dp, wpb * spw, vec_bytes, true) > 200 * 1024) --wpb;
      o->dense_wpb = wpb;
      o->dense_use_smem = 1;
      o->dense_smem = dense_warp_smem_bytes(P->dp, wpb * spw, vec_bytes, true);
      const uint64_t want = (a->shots + wpb * spw - 1) / (wpb * spw);
      const uint64_t cap = static_cast<uint64_t>(P->sm_count) * t.dense_grid_mult * 2;
      o->dense_grid = static_cast<int>(std::max<uint64_t>(1, std::min(want, cap)));
    } else if (dense_kind_for(P, h, o->fp64, t.dense_kind) == 3) {
      o->dense_kind = 3;   // CTA per shot, vector in shared memory
      o->dense_smem = dense_cta_smem_bytes(P->dp, vec_bytes, true);
      o->dense_use_smem = 1;
      const int grid = P->sm_count * t.cta_grid_mult;
      o->dense_grid = static_cast<int>(std::max<uint64_t>(1, std::min<uint64_t>(a->shots, grid)));
    } else {
      // wide executor: batches of shots with their vectors in HBM (two
      // buffers each), instruction by instruction; ~8 GB of vectors
      o->dense_kind = 4;
      o->wide_tile_bits = static_cast<uint32_t>(t.wide_tile_bits);
      const uint64_t per_shot = 2 * vec_bytes;
      const uint64_t nb = std::min<uint64_t>({a->shots, std::max<uint64_t>(1, (8ull << 30) / per_shot), 65535});
      o->wide_nb = static_cast<uint32_t>(nb);
      const size_t m3w = (h.n_m3 + 31) / 32;
      const size_t off_m3b = 2 * nb * vec_bytes;
      const size_t off_lam = align_up(off_m3b + nb * m3w * 4, 256);
      const size_t off_sums = align_up(off_lam + std::max<size_t>(1, G) * nb, 256);
      const size_t off_scale = off_sums + nb * 16;
      const size_t off_scalef = off_scale + nb * 8;
      const size_t off_lab = off_scalef + nb * 4;
      const size_t off_alive = off_lab + nb;
      const size_t total = off_alive + nb;
      CUDA_TRY(P->wide.ensure(total));
      unsigned char* base = static_cast<unsigned char*>(P->wide.ptr);
      o->wide_vec[0] = base;
      o->wide_vec[1] = base + nb * vec_bytes;
      o->wide_m3b = reinterpret_cast<uint32_t*>(base + off_m3b);
      o->wide_lam = base + off_lam;
      o->wide_sums = reinterpret_cast<double*>(base + off_sums);
      o->wide_scale = reinterpret_cast<double*>(base + off_scale);
      o->wide_scalef = reinterpret_cast<float*>(base + off_scalef);
      o->wide_lab = base + off_lab;
      o->wide_alive = base + off_alive;
      o->gvec_stride = static_cast<uint64_t>(1) << h.k_max;
    }
  }
  return SYMFT_OK;
}

// tallies after the outputs are final (same stream, so in order)
int enqueue_counts(symft_plan* P, const Prep& o, cudaStream_t st, int* launches) {
  if (!o.counts) return SYMFT_OK;
  const HostPlan& h = P->hp;
  CUDA_TRY(cudaMemsetAsync(o.counts, 0, (2 + static_cast<size_t>(h.n_obs)) * 8, st));
  CountArgs c{};
  c.W = o.W;
  c.shots = o.shots;
  c.n_obs = o.obs ? h.n_obs : 0;
  c.obs = o.obs;
  c.discard = o.disc;
  c.counts = reinterpret_cast<unsigned long long*>(o.counts);
  CUDA_TRY(launch_count(c, P->sm_count, st));
  ++*launches;
  return SYMFT_OK;
}

int enqueue(symft_plan* P, const symft_sample_args* a, const Prep& o, cudaStream_t st, int* launches) {
  const HostPlan& h = P->hp;
  const uint64_t W = o.W;
  if (o.plain) {
    if (o.meas) CUDA_TRY(cudaMemsetAsync(o.meas, 0, h.n_records * W * 8, st));
    if (o.det) CUDA_TRY(cudaMemsetAsync(o.det, 0, h.n_dets * W * 8, st));
    if (o.obs) CUDA_TRY(cudaMemsetAsync(o.obs, 0, h.n_obs * W * 8, st));
    if (o.disc) CUDA_TRY(cudaMemsetAsync(o.disc, 0, W * 8, st));
    PlainArgs pa{};
    pa.p = P->dp;
    pa.seed = a->seed;
    pa.shot0 = a->shot_offset;
    pa.shots = a->shots;
    pa.W = W;
    pa.meas = o.meas;
    pa.det = o.det;
    pa.obs = o.obs;
    pa.discard = o.disc;
    pa.kmax = h.k_max;
    pa.status = o.status;
    pa.prob = o.prob;
    CUDA_TRY(launch_plain(pa, o.fp64, o.plain_grid, st));
    ++*launches;
    return enqueue_counts(P, o, st, launches);
  }
  if (o.sign_grid > 0) {
    SignArgs s{};
    s.p = P->dp;
    s.seed = a->seed;
    s.keys = make_philox_keys(a->seed);
    s.block0 = a->shot_offset / kNoiseBlock;
    s.n_blocks = o.nblk;
    s.W = W;
    s.shots = a->shots;
    s.meas = o.meas;
    s.det = o.det;
    s.obs = o.obs;
    s.signs = o.signs;
    s.status = o.status;
    CUDA_TRY(launch_sign(s, o.sign_grid, st));
    ++*launches;
  }
  if (o.dense_kind) {
    if (h.n_m3) CUDA_TRY(cudaMemsetAsync(o.m3, 0, h.n_m3 * W * 8, st));
    DenseArgs d{};
    d.p = P->dp;
    d.seed = a->seed;
    d.keys = make_philox_keys(a->seed);
    d.shot0 = a->shot_offset;
    d.shots = a->shots;
    d.W = W;
    d.signs = o.signs;
    d.m3_out = o.m3;
    d.kmax = h.k_max;
    d.status = o.status;
    d.use_smem = o.dense_use_smem;
    d.gvec = o.gvec;
    d.gvec_stride = o.gvec_stride;
    d.prob = o.prob;
    // early exit under postselection reads the detector columns the sign
    // kernel has just written
    d.det_exo = P->dp.post_chk_off ? o.det : nullptr;
    if (o.dense_kind == 4) {
      WideArgs wa{};
      wa.p = P->dp;
      wa.keys = d.keys;
      wa.shots = a->shots;
      wa.W = W;
      wa.stride = o.gvec_stride;
      wa.vec[0] = o.wide_vec[0];
      wa.vec[1] = o.wide_vec[1];
      wa.signs = o.signs;
      wa.m3_out = o.m3;
      wa.prob = o.prob;
      wa.m3b = o.wide_m3b;
      wa.lam = o.wide_lam;
      wa.sums = o.wide_sums;
      wa.scale = o.wide_scale;
      wa.scalef = o.wide_scalef;
      wa.det_exo = d.det_exo;
      wa.alive = o.wide_alive;
      wa.lab = o.wide_lab;
      wa.status = o.status;
      for (uint64_t s0 = 0; s0 < a->shots; s0 += o.wide_nb) {
        wa.shot0 = a->shot_offset + s0;
        wa.r0 = s0;
        wa.nb = static_cast<uint32_t>(std::min<uint64_t>(o.wide_nb, a->shots - s0));
        wa.cur = 0;
        int l = 0;
        CUDA_TRY(launch_wide_batch(wa, P->dense_host.data(), o.fp64, P->sm_count, st, &l, o.wide_tile_bits));
        *launches += l;
      }
      --*launches;   // counted once below
    } else if (o.dense_kind == 1) CUDA_TRY(launch_dense_reg(d, o.fp64, o.dense_grid, st));
    else if (o.dense_kind == 5) CUDA_TRY(launch_dense_pc(d, o.fp64, o.dense_wpb, o.dense_grid, o.dense_smem, st));
    else if (o.dense_kind == 6) CUDA_TRY(launch_dense_pc_cta(d, o.fp64, o.dense_grid, o.dense_smem, st));
    else if (o.dense_kind == 2)
      CUDA_TRY(launch_dense(d, o.fp64, o.dense_wpb, o.dense_grid, o.dense_smem, st, o.dense_spw));
    else CUDA_TRY(launch_dense_cta(d, o.fp64, o.dense_grid, o.dense_smem, st));
    ++*launches;
  }
  if (o.need_final) {
    FinalArgs f{};
    f.p = P->dp;
    f.W = W;
    f.shots = a->shots;
    f.m3 = h.n_m3 ? o.m3 : nullptr;
    f.meas = o.meas;
    f.det = o.det;
    f.obs = o.obs;
    f.discard = o.disc;
    CUDA_TRY(launch_finalize(f, st));
    ++*launches;
  }
  return enqueue_counts(P, o, st, launches);
}

int sample_impl(symft_plan* P, const symft_sample_args* a) {
  const HostPlan& h = P->hp;
  int rc = validate(a);
  if (rc != SYMFT_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(a->stream);
  const uint64_t W = (a->shots + 63) / 64;
  const bool host = a->out_location == SYMFT_OUT_HOST;
  uint64_t *meas = a->meas_out, *det = a->det_out, *obs = a->obs_out, *disc = a->discard_out;
  double* prob = a->prob_out;
  uint64_t* counts = a->counts_out;
  if (host) {
    if (meas) { CUDA_TRY(P->h_meas.ensure(std::max<uint64_t>(1, h.n_records * W) * 8)); meas = (uint64_t*)P->h_meas.ptr; }
    if (det) { CUDA_TRY(P->h_det.ensure(std::max<uint64_t>(1, h.n_dets * W) * 8)); det = (uint64_t*)P->h_det.ptr; }
    if (obs) { CUDA_TRY(P->h_obs.ensure(std::max<uint64_t>(1, h.n_obs * W) * 8)); obs = (uint64_t*)P->h_obs.ptr; }
    if (disc) { CUDA_TRY(P->h_disc.ensure(W * 8)); disc = (uint64_t*)P->h_disc.ptr; }
    if (prob && h.n_m3) { CUDA_TRY(P->h_prob.ensure(h.n_m3 * a->shots * 8)); prob = (double*)P->h_prob.ptr; }
    if (counts) { CUDA_TRY(P->h_counts.ensure((2 + h.n_obs) * 8)); counts = (uint64_t*)P->h_counts.ptr; }
  }
  Prep o;
  rc = prepare(P, a, meas, det, obs, disc, prob, counts, &o);
  if (rc != SYMFT_OK) return rc;
  if (a->check) CUDA_TRY(cudaMemsetAsync(o.status, 0, sizeof(int), st));
  int launches = 0;
  rc = enqueue(P, a, o, st, &launches);
  g_last_launches = launches;
  if (rc != SYMFT_OK) return rc;
  if (host) {
    if (a->meas_out && o.meas) CUDA_TRY(cudaMemcpyAsync(a->meas_out, o.meas, h.n_records * W * 8, cudaMemcpyDeviceToHost, st));
    if (a->det_out && o.det) CUDA_TRY(cudaMemcpyAsync(a->det_out, o.det, h.n_dets * W * 8, cudaMemcpyDeviceToHost, st));
    if (a->obs_out && o.obs) CUDA_TRY(cudaMemcpyAsync(a->obs_out, o.obs, h.n_obs * W * 8, cudaMemcpyDeviceToHost, st));
    if (a->discard_out && o.disc) CUDA_TRY(cudaMemcpyAsync(a->discard_out, o.disc, W * 8, cudaMemcpyDeviceToHost, st));
    if (a->prob_out && o.prob)
      CUDA_TRY(cudaMemcpyAsync(a->prob_out, o.prob, h.n_m3 * a->shots * 8, cudaMemcpyDeviceToHost, st));
    if (a->counts_out && o.counts)
      CUDA_TRY(cudaMemcpyAsync(a->counts_out, o.counts, (2 + h.n_obs) * 8, cudaMemcpyDeviceToHost, st));
  }
  if (host || a->check) CUDA_TRY(cudaStreamSynchronize(st));
  if (a->check) {
    int hs = 0;
    CUDA_TRY(cudaMemcpy(&hs, o.status, sizeof(int), cudaMemcpyDeviceToHost));
    if (hs != 0) return set_error(SYMFT_E_DEVICE, "device status " + std::to_string(hs));
  }
  return SYMFT_OK;
}

// ---- autotuning: pick launch shapes by timing candidates on the plan --------
int autotune_impl(symft_plan* P, uint64_t shots, int precision, cudaStream_t st) {
  const HostPlan& h = P->hp;
  const uint64_t W = (shots + 63) / 64;
  CUDA_TRY(P->t_meas.ensure(std::max<uint64_t>(1, h.n_records * W) * 8));
  CUDA_TRY(P->t_det.ensure(std::max<uint64_t>(1, h.n_dets * W) * 8));
  CUDA_TRY(P->t_obs.ensure(std::max<uint64_t>(1, h.n_obs * W) * 8));
  CUDA_TRY(P->t_disc.ensure(W * 8));
  symft_sample_args a{};
  a.shots = shots;
  a.seed = 12345;
  a.precision = precision;
  a.stream = st;
  Tune& t = P->tune[precision == SYMFT_FP64 ? 1 : 0];
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  auto time_cfg = [&](float* ms) -> int {
    Prep o;
    int rc = prepare(P, &a, static_cast<uint64_t*>(P->t_meas.ptr), static_cast<uint64_t*>(P->t_det.ptr),
                     static_cast<uint64_t*>(P->t_obs.ptr), static_cast<uint64_t*>(P->t_disc.ptr), nullptr, nullptr, &o);
    if (rc != SYMFT_OK) return rc;
    int l = 0;
    rc = enqueue(P, &a, o, st, &l);   // warm-up
    if (rc != SYMFT_OK) return rc;
    CUDA_TRY(cudaEventRecord(e0, st));
    for (int i = 0; i < 3; ++i) {
      a.seed = 12346 + i;
      rc = enqueue(P, &a, o, st, &l);
      if (rc != SYMFT_OK) return rc;
    }
    CUDA_TRY(cudaEventRecord(e1, st));
    CUDA_TRY(cudaEventSynchronize(e1));
    CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
    return SYMFT_OK;
  };
  int rc = SYMFT_OK;
  float best = 0.0f;
  Tune base = t;
  rc = time_cfg(&best);
  // sign kernel: resident CTAs per SM
  if (rc == SYMFT_OK && h.n_slots > 0) {
    for (int cps : {2, 3, 4}) {
      Tune cand = base;
      cand.sign_ctas_per_sm = cps;
      t = cand;
      float ms = 0.0f;
      rc = time_cfg(&ms);
      if (rc != SYMFT_OK) break;
      if (ms < best) { best = ms; base = cand; }
    }
    t = base;
  }
  // dense executor kind: every kind that can run the plan, default shapes
  if (rc == SYMFT_OK && !h.dense.empty()) {
    const bool fp64 = precision == SYMFT_FP64;
    for (int kind = 1; kind <= 6; ++kind) {
      if (!dense_kind_valid(P, h, fp64, kind) || kind == dense_kind_for(P, h, fp64, base.dense_kind)) continue;
      Tune cand = base;
      cand.dense_kind = kind;
      t = cand;
      float ms = 0.0f;
      rc = time_cfg(&ms);
      if (rc != SYMFT_OK) break;
      if (ms < best) { best = ms; base = cand; }
    }
    t = base;
  }
  // dense executor: grid size (register / warp kernels), warps per CTA, CTA slots
  if (rc == SYMFT_OK && !h.dense.empty()) {
    std::vector<Tune> cands;
    for (int gm : {2, 4, 8, 16, 32}) { Tune c = base; c.dense_grid_mult = gm; cands.push_back(c); }
    for (int wpb : {2, 4, 8}) { Tune c = base; c.dense_wpb = wpb; cands.push_back(c); }
    for (int cm : {1, 2, 4}) { Tune c = base; c.cta_grid_mult = cm; cands.push_back(c); }
    // the wide executor's fused-window tile (shape of the tiles it streams)
    if (dense_kind_for(P, h, precision == SYMFT_FP64, base.dense_kind) == 4) {
      const int hi = precision == SYMFT_FP64 ? static_cast<int>(kWideTileBitsMaxF64) : static_cast<int>(kWideTileBitsMaxF32);
      for (int tb = static_cast<int>(kWideTileBitsMin); tb <= hi; ++tb) { Tune c = base; c.wide_tile_bits = tb; cands.push_back(c); }
    }
    for (const Tune& cand : cands) {
      t = cand;
      float ms = 0.0f;
      rc = time_cfg(&ms);
      if (rc != SYMFT_OK) break;
      if (ms < best) { best = ms; base = cand; }
    }
    t = base;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SYMFT_OK) return rc;
  t.tuned = true;
  t.best_ms_per_shot = best / 3.0f / static_cast<float>(shots);
  return SYMFT_OK;
}

// ---- batched jobs captured into one CUDA graph --------------------------------
struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> ev;
  ~GraphCache() {
    if (exec) cudaGraphExecDestroy(exec);
    for (auto s : branch) cudaStreamDestroy(s);
    for (auto e : ev) cudaEventDestroy(e);
    if (cap) cudaStreamDestroy(cap);
  }
};
thread_local GraphCache g_graph;

int batch_impl(const symft_plan* const* plans, int n_plans, const symft_job* jobs, int n_jobs,
               cudaStream_t user) {
  if (!plans || !jobs || n_plans <= 0 || n_jobs <= 0) return set_error(SYMFT_E_ARG, "empty batch");
  std::vector<symft_sample_args> args(n_jobs);
  std::vector<uint64_t> max_shots(n_plans, 0);
  std::vector<char> any_counts(n_plans, 0);
  for (int j = 0; j < n_jobs; ++j) {
    const symft_job& J = jobs[j];
    if (J.plan >= static_cast<uint32_t>(n_plans) || !plans[J.plan])
      return set_error(SYMFT_E_ARG, "job " + std::to_string(j) + ": bad plan index");
    symft_sample_args& a = args[j];
    a = symft_sample_args{};
    a.shots = J.shots;
    a.seed = J.seed;
    a.shot_offset = J.shot_offset;
    a.meas_out = J.meas_out;
    a.det_out = J.det_out;
    a.obs_out = J.obs_out;
    a.discard_out = J.discard_out;
    a.precision = J.precision;
    a.plain = J.plain;
    a.counts_out = J.counts_out;
    int rc = validate(&a);
    if (rc != SYMFT_OK) return set_error(rc, "job " + std::to_string(j) + ": " + g_last_error);
    max_shots[J.plan] = std::max(max_shots[J.plan], J.shots);
    if (J.counts_out) any_counts[J.plan] = 1;
  }
  // size every plan's workspace for its largest job first, so no later
  // prepare() moves a buffer another job of the same plan already uses
  for (int p = 0; p < n_plans; ++p) {
    if (!max_shots[p]) continue;
    symft_plan* P = const_cast<symft_plan*>(plans[p]);
    for (int prec : {SYMFT_FP32, SYMFT_FP64}) {
      symft_sample_args a{};
      a.shots = max_shots[p];
      a.precision = prec;
      Prep o;
      int rc = prepare(P, &a, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, &o);
      if (rc != SYMFT_OK) return rc;
      if (P->hp.postselect && P->hp.n_dets) CUDA_TRY(P->det_scratch.ensure(P->hp.n_dets * o.W * 8));
      if (any_counts[p]) {
        if (P->hp.n_obs) CUDA_TRY(P->obs_scratch.ensure(P->hp.n_obs * o.W * 8));
        if (P->hp.postselect) CUDA_TRY(P->disc_scratch.ensure(o.W * 8));
      }
    }
  }
  std::vector<Prep> preps(n_jobs);
  for (int j = 0; j < n_jobs; ++j) {
    symft_plan* P = const_cast<symft_plan*>(plans[jobs[j].plan]);
    int rc = prepare(P, &args[j], args[j].meas_out, args[j].det_out, args[j].obs_out, args[j].discard_out,
                     nullptr, args[j].counts_out, &preps[j]);
    if (rc != SYMFT_OK) return set_error(rc, "job " + std::to_string(j) + ": " + g_last_error);
  }
  // capture: one branch per plan (jobs of a plan share its workspace, in order)
  GraphCache& G = g_graph;
  if (!G.cap) CUDA_TRY(cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking));
  const int nbr = std::min(n_plans, 32);
  while (static_cast<int>(G.branch.size()) < nbr) {
    cudaStream_t s;
    CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    G.branch.push_back(s);
  }
  while (static_cast<int>(G.ev.size()) < nbr + 1) {
    cudaEvent_t e;
    CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    G.ev.push_back(e);
  }
  CUDA_TRY(cudaStreamBeginCapture(G.cap, cudaStreamCaptureModeThreadLocal));
  int launches = 0;
  int rc = SYMFT_OK;
  cudaError_t ce = cudaEventRecord(G.ev[nbr], G.cap);
  std::vector<char> used(nbr, 0);
  for (int j = 0; j < n_jobs && rc == SYMFT_OK && ce == cudaSuccess; ++j) {
    const int b = static_cast<int>(jobs[j].plan) % nbr;
    if (!used[b]) {
      ce = cudaStreamWaitEvent(G.branch[b], G.ev[nbr], 0);
      used[b] = 1;
    }
    if (ce == cudaSuccess)
      rc = enqueue(const_cast<symft_plan*>(plans[jobs[j].plan]), &args[j], preps[j], G.branch[b], &launches);
  }
  for (int b = 0; b < nbr && ce == cudaSuccess; ++b) {
    if (!used[b]) continue;
    ce = cudaEventRecord(G.ev[b], G.branch[b]);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(G.cap, G.ev[b], 0);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t ee = cudaStreamEndCapture(G.cap, &graph);
  if (rc != SYMFT_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return set_error(SYMFT_E_CUDA, std::string("batch capture: ") + cudaGetErrorString(ce));
  }
  if (ee != cudaSuccess) return set_error(SYMFT_E_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ee));
  bool ok = false;
  if (G.exec) {
    cudaGraphExecUpdateResultInfo info;
    ok = cudaGraphExecUpdate(G.exec, graph, &info) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      cudaGraphExecDestroy(G.exec);
      G.exec = nullptr;
    }
  }
  if (!ok) {
    cudaError_t ie = cudaGraphInstantiate(&G.exec, graph, 0);
    if (ie != cudaSuccess) {
      cudaGraphDestroy(graph);
      G.exec = nullptr;
      return set_error(SYMFT_E_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
    }
  }
  cudaGraphDestroy(graph);
  CUDA_TRY(cudaGraphLaunch(G.exec, user));
  g_last_launches = launches;
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
  if (o.postselect != SYMFT_POSTSELECT_NONE && o.postselect != SYMFT_POSTSELECT_ALL &&
      o.postselect != SYMFT_POSTSELECT_LISTED)
    return set_error(SYMFT_E_ARG, "bad postselect mode");
  if (o.postselect == SYMFT_POSTSELECT_LISTED && o.n_post_dets > 0 && o.post_dets == nullptr)
    return set_error(SYMFT_E_ARG, "postselect LISTED: null post_dets");
  try {
    Circuit c = parse_circuit(text);
    if (o.postselect == SYMFT_POSTSELECT_LISTED)
      for (uint32_t i = 0; i < o.n_post_dets; ++i)
        if (o.post_dets[i] >= c.n_dets)
          return set_error(SYMFT_E_ARG, "postselect LISTED: detector " + std::to_string(o.post_dets[i]) +
                                            " out of range (" + std::to_string(c.n_dets) + " detectors)");
    if (o.executor < 0 || o.executor > 6) return set_error(SYMFT_E_ARG, "bad executor preference");
    if (o.wide_tile_bits != 0 && (o.wide_tile_bits < static_cast<int>(kWideTileBitsMin) || o.wide_tile_bits > 16))
      return set_error(SYMFT_E_ARG, "wide_tile_bits out of range");
    symft_plan* p = new symft_plan();
    try {
      p->hp = compile_plan(c, o);
      build_blob(p);
      p->tune[0].dense_kind = p->tune[1].dense_kind = o.executor;
      p->tune[0].wide_tile_bits = p->tune[1].wide_tile_bits = o.wide_tile_bits;
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
  uint64_t traffic = 0, flops = 0;
  for (const DenseInstr& d : h.dense) {
    const uint64_t n = 1ull << d.k;
    if (d.kind == I_PROMOTE_ROT) traffic += 3 * n;
    else if (d.kind == I_ACTIVE_DIAG_ROT || d.kind == I_ACTIVE_PAIR_ROT) traffic += 2 * n;
    else traffic += n + n + n / 2;
    switch (d.kind) {
      case I_PROMOTE_ROT: flops += 4 * n; break;
      case I_ACTIVE_DIAG_ROT: flops += 6 * n; break;
      case I_ACTIVE_PAIR_ROT: flops += 10 * n; break;
      case I_ACTIVE_DIAG_MEAS: flops += 5 * n; break;
      default: flops += 13 * n; break;
    }
  }
  info->dense_amp_traffic = traffic;
  info->dense_flops = flops;
  // algorithmic integer work of the sign kernel per noise block (512 shots):
  // Philox blocks the stream specification needs, expected fires, and 32-bit
  // XOR operations (random-measurement sources, record parents and output
  // gather terms over 16 words per slot, plus one XOR per fired target)
  {
    double philox = static_cast<double>(h.m1_t.size()) * (kNoiseBlock / kWordPair);
    double fires = 0.0, xor_ops = 0.0;
    const uint32_t n_groups = (h.n_channels + 3) / 4;
    for (uint32_t g = 0; g < n_groups; ++g) {
      bool live = false;
      for (uint32_t c = 4 * g; c < std::min(h.n_channels, 4 * g + 4); ++c) live |= h.ch_theta_last[c] != 0;
      if (live) philox += 1.0;
    }
    for (uint32_t c = 0; c < h.n_channels; ++c) {
      if (h.ch_theta_last[c] == 0) continue;
      const double q = h.qtabs[h.ch_qtab[c]].q;
      const CellTable& ct = h.ctabs[h.ch_ctab[c]];
      const double d = ct.ncell > 1 ? 2.0 : 1.0;            // tail draws per fire
      // N ~ Binomial(512, q) fires; ceil(d N / 4) tail blocks
      double pk = std::pow(1.0 - q, kNoiseBlock), tail = 0.0;
      for (int k = 0; k <= kNoiseBlock && (k < 8 || pk > 1e-18); ++k) {
        tail += pk * std::ceil(d * k / 4.0);
        pk *= (static_cast<double>(kNoiseBlock - k) / (k + 1)) * (q / (1.0 - q));
      }
      philox += tail;
      const double nf = kNoiseBlock * q;
      fires += nf;
      // mean number of target slots of a fired cell, weighted by the cell law
      double prev = 0.0, tg = 0.0;
      for (uint32_t k = 0; k < ct.ncell; ++k) {
        const double hi = k + 1 < ct.ncell ? ct.phi[k] / 4294967296.0 : 1.0;
        const uint32_t e = h.ch_cell0[c] + k;
        tg += (hi - prev) * (h.cell_off[e + 1] - h.cell_off[e]);
        prev = hi;
      }
      xor_ops += nf * tg;
    }
    xor_ops += 16.0 * (static_cast<double>(h.m1_tgt.size()) + h.par.size() + h.gat_rec.size());
    info->sign_model[0] = philox;
    info->sign_model[1] = fires;
    info->sign_model[2] = xor_ops;
  }
  info->wide_amp_traffic[0] = wide_amp_traffic(p->dense_host.data(), static_cast<uint32_t>(p->dense_host.size()), false,
                                                static_cast<uint32_t>(p->tune[0].wide_tile_bits));
  info->wide_amp_traffic[1] = wide_amp_traffic(p->dense_host.data(), static_cast<uint32_t>(p->dense_host.size()), true,
                                                static_cast<uint32_t>(p->tune[1].wide_tile_bits));
  info->pc_capacity = h.pc.capacity;
  info->pc_selected = h.pc.use ? 1u : 0u;
  info->pc_work[0] = h.pc.work_pc;
  info->pc_work[1] = h.pc.work_mono;
  info->simplified[0] = h.n_fused;
  info->simplified[1] = h.n_cancelled;
  info->simplified[2] = h.n_branch_phase;
  info->wide_tile_bits[0] = wide_tile_bits_in_use(false, static_cast<uint32_t>(p->tune[0].wide_tile_bits));
  info->wide_tile_bits[1] = wide_tile_bits_in_use(true, static_cast<uint32_t>(p->tune[1].wide_tile_bits));
  for (int i = 0; i < 2; ++i) {
    info->tuned_ns_per_shot[i] = p->tune[i].tuned ? p->tune[i].best_ms_per_shot * 1e6f : 0.0f;
    info->dense_executor[i] = h.dense.empty() ? 0u
        : static_cast<uint32_t>(dense_kind_for(p, h, i == 1, p->tune[i].dense_kind));
  }
  return SYMFT_OK;
}

int symft_plan_active_meas(const symft_plan* p, uint32_t* t_out, uint32_t capacity) {
  if (!p) return set_error(SYMFT_E_ARG, "null plan");
  if (capacity > 0 && t_out == nullptr) return set_error(SYMFT_E_ARG, "null t_out");
  const auto& t = p->hp.m3_t;
  for (uint32_t j = 0; j < capacity && j < t.size(); ++j) t_out[j] = t[j];
  return static_cast<int>(t.size());
}

void symft_plan_free(symft_plan* p) {
  if (!p) return;
  p->plan_buf.release();
  p->signs.release();
  p->m3.release();
  p->det_scratch.release();
  p->obs_scratch.release();
  p->disc_scratch.release();
  p->h_prob.release();
  p->h_counts.release();
  p->gvec.release();
  p->wide.release();
  p->status.release();
  p->h_meas.release();
  p->h_det.release();
  p->h_obs.release();
  p->h_disc.release();
  p->t_meas.release();
  p->t_det.release();
  p->t_obs.release();
  p->t_disc.release();
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

int symft_autotune(symft_plan* plan, uint64_t shots, int precision, void* stream) {
  g_last_error.clear();
  if (!plan) return set_error(SYMFT_E_ARG, "null plan");
  if (shots == 0) return set_error(SYMFT_E_ARG, "shots must be >= 1");
  if (precision != SYMFT_FP32 && precision != SYMFT_FP64) return set_error(SYMFT_E_ARG, "bad precision");
  std::lock_guard<std::mutex> lk(plan->mu);
  try {
    return autotune_impl(plan, shots, precision, static_cast<cudaStream_t>(stream));
  } catch (const std::bad_alloc&) {
    return set_error(SYMFT_E_NOMEM, "host allocation failed");
  }
}

int symft_sample_batch(const symft_plan* const* plans, int n_plans, const symft_job* jobs, int n_jobs,
                       void* stream) {
  g_last_error.clear();
  g_last_launches = 0;
  try {
    return batch_impl(plans, n_plans, jobs, n_jobs, static_cast<cudaStream_t>(stream));
  } catch (const std::bad_alloc&) {
    return set_error(SYMFT_E_NOMEM, "host allocation failed");
  }
}

const char* symft_last_error(void) { return g_last_error.c_str(); }

int symft_last_launch_count(void) { return g_last_launches; }

}  // extern "C"
