// Device plan layout and kernel argument blocks (host- and device-visible PODs).
#pragma once

#include <cstdint>

#include <vector_types.h>

namespace symft {

// stream tags (counter word 3)
constexpr uint32_t kTagHead = 1, kTagTail = 2, kTagMbit = 3, kTagMfrac = 4;

// shots per noise block of the stream specification: a channel's head draw
// and its block-geometric process cover lanes 0..kNoiseBlock-1 of one block
constexpr int kNoiseBlock = 512;
// shots per packed random-measurement Philox block (two 64-shot words)
constexpr int kWordPair = 128;
// records per chain path at most (the compile step starts a new path there)
constexpr int kMaxLevels = 16;

struct ChannelDev {        // 16 bytes, one per noise channel
  uint32_t theta_last;     // THETA_{kNoiseBlock-1}: u >= this means no fire in the block
  uint16_t qtab, ctab;
  uint32_t comp0;          // first noise component (plain form)
  uint32_t cell0;          // first (channel, cell) target entry (sign kernel)
};

// Targets of one (channel, Pauli cell), 16 bytes as eight 16-bit fields:
// f0 = n <= 7 and f1..f(n) = slot * 16 (the slot's first 32-bit word); or
// f0 = 0xFFFF and (y, z) = (offset, count) of a list of slot * 16 in cell_ovf.
using CellTargetsDev = uint4;

struct CellTableDev {
  uint32_t ncell;
  uint32_t phi[15];
  uint8_t mask[16];
};

// Lane-search buckets of a threshold table: with shift s the smallest value
// such that THETA_{kNoiseBlock-1} >> s < kQBuckets, bucket i holds
// min{j : THETA_j > i << s}, the first lane a uniform u with u >> s == i can
// fire at.  The search starts there and steps up while u >= THETA_j, so its
// answer is the table's own, and it takes kNoiseBlock / kQBuckets extra steps
// on average for a uniform below THETA_{kNoiseBlock-1}.
constexpr int kQBuckets = 512;

struct DenseInstrDev {
  int32_t kind, k, h, mu;
  uint32_t a, b;
  int32_t eta, m3;
  double c, s;
  uint32_t sign_target_col;   // column of the exogenous sign in the scratch
  uint32_t causal_off, causal_n;
  uint32_t t;
  uint32_t post_grp;          // active measurement: detector group to check for early
                              // exit after it, or kNoGroup
  float cf, sf;               // c and s rounded to FP32 (to nearest) on the host: the
                              // FP32 executors' coefficients, so no lane converts
                              // from FP64 (a slow pipe on B300) per instruction
  uint32_t pad;
};

// The rotation coefficients (c, s) of an instruction in the vector's precision.
template <typename Real>
__host__ __device__ inline Real coef_c(const DenseInstrDev& I) {
  if constexpr (sizeof(Real) == 4) return I.cf;
  else return I.c;
}
template <typename Real>
__host__ __device__ inline Real coef_s(const DenseInstrDev& I) {
  if constexpr (sizeof(Real) == 4) return I.sf;
  else return I.s;
}

constexpr uint32_t kNoGroup = 0xFFFFFFFFu;

// fused-window tile sizes (log2 amplitudes) the wide executor accepts
constexpr uint32_t kWideTileBitsMin = 10, kWideTileBitsMaxF32 = 13, kWideTileBitsMaxF64 = 12;

// The warp executors copy the instruction stream (and the product-component
// program) into shared memory, in front of their per-warp words, when it
// takes at most kStageBytes; else they read it from the plan in global memory.
constexpr size_t kStageBytes = 24 * 1024;
__host__ __device__ inline size_t stage_bytes(size_t program_bytes) {
  return program_bytes <= kStageBytes ? (program_bytes + 15) & ~(size_t)15 : 0;
}

// Product-component program (Sec. 6, adaptive product-component
// representation): one op per component initialisation, Kronecker merge or
// dense instruction, with the component's place in the per-shot workspace.
enum PCOpKind : uint32_t { PC_INIT = 0, PC_MERGE = 1, PC_APPLY = 2 };

struct PCOp {
  uint32_t op;        // PCOpKind
  uint32_t g;         // dense instruction (INIT: its PromoteRot; APPLY: the instruction)
  uint32_t off;       // workspace offset (amplitudes) of the target component
  uint32_t k;         // APPLY: the component's width before the instruction
  uint32_t a, b;      // APPLY: masks in the component's local bits
  int32_t h;          // APPLY (measurement): local pivot bit
  uint32_t offA, kA;  // MERGE: first factor (its bits become the low bits)
  uint32_t offB, kB;  // MERGE: second factor
  uint32_t out;       // APPLY (measurement): offset the kept half is written to (off: in place)
};

struct DevPlan {
  uint32_t n_channels;
  const ChannelDev* ch;
  const uint4* theta4;          // THETA_{kNoiseBlock-1} of channels 4g..4g+3 (0 = never fires)
  uint32_t n_qtab, n_ctab;
  const uint32_t* qtheta;       // [n_qtab][kNoiseBlock]
  const uint32_t* qshift;       // [n_qtab] bucket shift s
  const uint16_t* qstart;       // [n_qtab][kQBuckets] first lane of each bucket
  const CellTableDev* ctabs;
  const CellTargetsDev* cellt;  // per (channel, cell)
  const uint32_t* cell_ovf;     // long target lists (slot * 16)
  uint32_t n_m1;
  const uint32_t* m1_t;
  const uint32_t* m1_off;
  const uint32_t* m1_tgt;
  // outputs in finalize numbering [records][dets][obs] (tgt_sign0 = count)
  uint32_t n_targets, tgt_det0, tgt_obs0, tgt_sign0;
  const uint32_t* tgt_causal_off;
  const uint32_t* tgt_causal;
  // the outputs with causal terms only: n_causal_tgt items, x = output index,
  // y = first entry in tgt_causal, z = count
  uint32_t n_causal_tgt;
  const uint4* causal_tgt;
  // sign-kernel slots [records][dense signs]
  uint32_t n_slots;
  const uint8_t* slot_const;
  // per slot: its constant and its random-measurement sources, 16 bytes as
  // eight 16-bit fields: f0 = n | const << 15 with n <= 7 and f1..f(n) = m1
  // indices, or n = 0x7FFF and (y, z) = (offset, count) of a list in slot_m1_ovf
  const uint4* slot_m1;
  const uint32_t* slot_m1_ovf;
  // record chains as paths (every record has at most one parent and at most
  // one child): path p is path_ids[2p], path_ids[2p + 1], its 2..kMaxLevels
  // records as 16-bit fields in order, each the parent of the next, the
  // unused fields 0xFFFF
  uint32_t n_paths;
  const uint4* path_ids;
  // det / obs -> records: f0 = n <= 7 and f1..f(n) = records, or f0 = 0xFFFF
  // and (y, z) = (offset, count) of a record list in gat_ovf
  const uint4* gat_item;
  const uint32_t* gat_ovf;
  // slots that do not start at zero (a constant or random-measurement sources)
  uint32_t n_slot_nz;
  const uint32_t* slot_nz;
  // detectors / observables (index j < n_dets + n_obs) that equal one slot as
  // it stands before the record chains: x = j, y = slot (a record without
  // parents, or the later record of a two-record gather whose only parent is
  // the other one); every other output is gathered after the chains
  uint32_t n_out_delta, n_out_rest;
  const uint2* out_delta;
  const uint32_t* out_rest;
  // postselection walk in circuit order: record r as r (>= 0), detector i as
  // -1 - (2 i + p) with p = 1 when detector i is postselected
  uint32_t n_post_events;
  const int32_t* post_events;
  // early exit of the dense executors: postselected detectors grouped by the
  // number of active measurements before them (n_m3 + 2 offsets; group q is
  // final once active measurement q - 1 is decided); null without postselection
  const uint32_t* post_chk_off;
  const uint32_t* post_chk;
  uint32_t post_grp0;           // 0: check group 0 before a shot's dense work; else kNoGroup
  uint32_t n_dense;
  const DenseInstrDev* dense;
  uint32_t n_pc;                // product-component program (0: not built)
  const PCOp* pc;
  uint32_t pc_capacity;         // its workspace amplitudes per shot
  const uint32_t* dense_causal;
  uint32_t n_m3;
  const uint32_t* m3_t;         // measurement ordinal of each active measurement
  uint32_t n_records, n_dets, n_obs;
  int postselect;               // non-zero when any detector is postselected
  // plain (per-shot) form
  uint32_t n_comp;
  const uint8_t* plain_const;   // [records][dets][obs][dense signs]
  const uint32_t* plain_off;
  const uint32_t* plain_sym;
};


// Philox4x32-10 round keys of a seed: k[2r] = k0 + r * 0x9E3779B9,
// k[2r+1] = k1 + r * 0xBB67AE85 (mod 2^32), r = 0..9, with (k0, k1) the low
// and high words of the seed.  Kernels read them from the launch parameters.
struct PhiloxKeys {
  uint32_t k[20];
};

inline PhiloxKeys make_philox_keys(uint64_t seed) {
  PhiloxKeys K;
  uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    K.k[2 * r] = k0;
    K.k[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return K;
}

struct SignArgs {
  DevPlan p;
  PhiloxKeys keys;        // round keys of `seed`
  uint64_t seed;
  uint64_t block0;        // global index of the first noise block (kNoiseBlock shots)
  uint64_t n_blocks;      // local noise blocks
  uint64_t W;             // words per column
  uint64_t shots;
  uint64_t* meas;         // may be null
  uint64_t* det;
  uint64_t* obs;
  uint64_t* signs;        // dense sign scratch (n_dense columns) or null
  int* status;
};

struct DenseArgs {
  DevPlan p;
  PhiloxKeys keys;        // round keys of `seed`
  uint64_t seed;
  uint64_t shot0;         // absolute index of local shot 0
  uint64_t shots;
  uint64_t W;
  const uint64_t* signs;  // exogenous sign columns (n_dense x W)
  uint64_t* m3_out;       // active outcomes (n_m3 x W), zeroed before launch
  void* gvec;             // global vector scratch (per resident warp) or null
  uint64_t gvec_stride;   // amplitudes per warp slot in gvec
  uint32_t kmax;
  int use_smem;
  int* status;
  double* prob;           // Pr(m = 0) per active measurement and shot (n_m3 x shots) or null
  const uint64_t* det_exo;   // detector columns from the sign kernel (exogenous parts), or
                             // null: no early exit
};

// One batch of the wide (instruction-major) dense executor.
struct WideArgs {
  DevPlan p;
  PhiloxKeys keys;        // round keys of the seed
  uint64_t shot0;         // absolute index of batch shot 0
  uint64_t r0;            // request-local index of batch shot 0
  uint64_t shots;         // shots of the whole request (prob_out row length)
  uint64_t W;             // words per output column of the request
  uint32_t nb;            // shots in this batch
  int cur;                // buffer holding the current vectors (0 or 1)
  uint64_t stride;        // amplitudes per shot in a buffer (2^k_max)
  void* vec[2];           // [nb][stride] amplitudes each
  const uint64_t* signs;  // exogenous sign columns (n_dense x W)
  uint64_t* m3_out;       // active outcomes (n_m3 x W), zeroed before the first batch
  double* prob;           // Pr(m = 0) per active measurement and shot, or null
  uint32_t* m3b;          // [nb][ceil(n_m3 / 32)] active outcomes of each shot
  uint8_t* lam;           // [n_dense][nb] sign of each dense instruction
  double* sums;           // [nb][2] branch sums of the current measurement
  double* scale;          // [nb] renormalisation after the current measurement
  float* scalef;          // [nb] the same, rounded to FP32 (FP32 vectors)
  uint8_t* lab;           // [nb] kept branch label
  const uint64_t* det_exo;   // as in DenseArgs (early exit), or null
  uint8_t* alive;         // [nb] 0 once the shot is rejected by postselection
  int* status;            // set non-zero on a device-side failure (a bounded wait that ran out)
};

struct PlainArgs {
  DevPlan p;
  uint64_t seed;
  uint64_t shot0;         // absolute index of local shot 0
  uint64_t shots;
  uint64_t W;
  uint64_t* meas;         // zeroed before launch (bits are OR-ed in)
  uint64_t* det;
  uint64_t* obs;
  uint64_t* discard;
  uint32_t kmax;
  int* status;
  double* prob;           // as in DenseArgs
};

struct FinalArgs {
  DevPlan p;
  uint64_t W;
  uint64_t shots;
  const uint64_t* m3;     // may be null when n_m3 == 0
  uint64_t* meas;
  uint64_t* det;          // required when postselecting
  uint64_t* obs;
  uint64_t* discard;
};

// Tallies of one request: kept shots, discarded shots, and per observable the
// kept shots whose observable bit is 1.
struct CountArgs {
  uint64_t W;
  uint64_t shots;
  uint32_t n_obs;
  const uint64_t* obs;      // may be null when n_obs == 0
  const uint64_t* discard;  // may be null (no postselection)
  unsigned long long* counts;   // 2 + n_obs, zeroed before launch
};

}  // namespace symft
