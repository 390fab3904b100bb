// Host-side data structures of the compile step and the lowered device plan.
#pragma once

#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "plan_dev.hpp"
#include "symft.h"

namespace symft {

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

// ---------------------------------------------------------------------------
// Circuit model (Sec. 2) after parsing and REPEAT unrolling.
// ---------------------------------------------------------------------------
enum GateId : int {
  G_I, G_H, G_S, G_S_DAG, G_SQRT_X, G_SQRT_X_DAG, G_X, G_Y, G_Z,
  G_CX, G_CY, G_CZ, G_SWAP
};

enum OpKind : int { OP_CLIFF, OP_ROT, OP_MEAS, OP_FB, OP_NOISE, OP_DET, OP_OBS };

// Noise channel families.  Components are the symplectic bits the channel
// can flip, listed per qubit of its support as (x, z).
enum ChanType : int { CH_X, CH_Y, CH_Z, CH_XYZ, CH_D2 };

struct PauliTerm {
  uint32_t q;
  char p;  // 'X' 'Y' 'Z'
};

struct Op {
  OpKind kind;
  int gate = 0;
  uint32_t q0 = 0, q1 = 0;
  std::vector<PauliTerm> pauli;   // rotation / measurement / feedback Pauli
  double theta = 0.0;
  uint32_t t = 0;                 // measurement ordinal
  int32_t rec = -1;               // record index, -1 hidden
  std::vector<uint32_t> conds;    // ordinals (feedback / detector / observable)
  uint32_t channel = 0;           // noise ordinal
  int chan = 0;                   // ChanType
  double q = 0.0;                 // total error probability
  std::vector<double> weights;    // cell weights (CH_XYZ: X, Y, Z)
  uint32_t index = 0;             // detector / observable index
};

struct Circuit {
  std::vector<Op> ops;
  uint32_t n_qubits = 0, n_meas = 0, n_records = 0, n_channels = 0, n_dets = 0, n_obs = 0;
  std::vector<uint32_t> record_ordinal;
};

Circuit parse_circuit(const std::string& text);

// ---------------------------------------------------------------------------
// Lowered plan.
// ---------------------------------------------------------------------------
enum InstrKind : int {
  I_PROMOTE_ROT = 0, I_ACTIVE_DIAG_ROT = 1, I_ACTIVE_PAIR_ROT = 2,
  I_RANDOM_MEAS = 3, I_DET_MEAS = 4, I_ACTIVE_DIAG_MEAS = 5, I_ACTIVE_PAIR_MEAS = 6
};

constexpr int kMaxActive = 24;       // build limit on k_max

// One dense-state instruction (the sign is target sign_target + causal list).
struct DenseInstr {
  int kind;
  int k;             // active width before the instruction
  uint32_t a, b;     // active masks (bit j = coordinate j+1)
  int h;             // pivot bit (active measurements)
  int mu;            // power of i
  int eta;
  double c, s;       // cos(theta/2), sin(theta/2)
  uint32_t sign_target;   // exogenous part of lambda (target slot)
  uint32_t causal_off, causal_n;   // m3 indices in the causal list
  int32_t m3;        // active measurement: index of its outcome among m3 symbols
  uint32_t t;        // measurement ordinal (active measurements)
  int32_t rec;       // record index or -1
};

// Distinct noise-probability tables.
struct QTable {
  double q;
  uint32_t theta[kNoiseBlock];
};

struct CellTable {
  uint32_t ncell;
  uint32_t phi[15];          // thresholds PHI_k, k < ncell-1
  uint8_t mask[16];          // component mask per cell
};

struct PCProgram {
  std::vector<PCOp> ops;
  uint32_t capacity = 0;      // workspace amplitudes per shot
  uint64_t work_pc = 0;       // amplitudes touched per shot by the program
  uint64_t work_mono = 0;     // amplitudes touched per shot by the monolithic vector
  bool use = false;           // selected by the cost model
};

PCProgram build_product_components(const std::vector<DenseInstr>& dense, uint32_t k_max);

struct HostPlan {
  uint32_t n_qubits = 0, n_meas = 0, n_records = 0, n_dets = 0, n_obs = 0, n_channels = 0;
  uint32_t k_max = 0;
  uint32_t hist[7] = {0, 0, 0, 0, 0, 0, 0};
  uint32_t max_expr_weight = 0;
  int postselect = 0;

  // noise channels in ordinal order
  std::vector<uint32_t> ch_theta_last;   // THETA_127 (0: never fires)
  std::vector<uint16_t> ch_qtab, ch_ctab;
  std::vector<uint32_t> ch_comp0;        // first component id
  std::vector<uint8_t> ch_ncomp;
  std::vector<uint32_t> ch_cell0;        // first (channel, cell) entry of cell_off
  std::vector<QTable> qtabs;
  std::vector<CellTable> ctabs;

  // component -> targets (CSR)
  uint32_t n_comp = 0;
  std::vector<uint32_t> comp_off, comp_tgt;
  // (channel, Pauli cell) -> targets (CSR): the slots a fired cell flips, i.e.
  // the XOR of its components' target sets (pairs that cancel removed)
  std::vector<uint32_t> cell_off, cell_tgt;

  // random measurements (m1): ordinal and targets (CSR)
  std::vector<uint32_t> m1_t, m1_off, m1_tgt;

  // outputs in finalize numbering: [records][dets][obs]; tgt_sign0 = their count
  uint32_t n_targets = 0, tgt_rec0 = 0, tgt_det0 = 0, tgt_obs0 = 0, tgt_sign0 = 0;
  std::vector<uint32_t> tgt_causal_off, tgt_causal;   // m3 indices per output

  // sign-kernel slots: [records][dense signs]; a record slot accumulates
  // const + delta (noise and random bits) and then XORs in its parent record
  uint32_t n_slots = 0;
  std::vector<uint8_t> slot_const;
  std::vector<uint32_t> par_off, par;        // record -> parent record (CSR, at most one)
  std::vector<uint32_t> gat_off, gat_rec;    // det / obs -> records (CSR)

  // plain (per-shot, unpacked) form: full exogenous expression of every output
  // [records][dets][obs][dense signs] as symbol lists; symbol < n_comp is a
  // noise component, else n_comp + m1 index
  std::vector<uint8_t> plain_const;
  std::vector<uint32_t> plain_off, plain_sym;

  // postselection order: events in circuit order, record r (>= 0) or
  // detector i (-1 - (2 i + p), p = 1 when detector i is postselected)
  std::vector<int32_t> post_events;
  // postselected detectors grouped by the active measurements before them:
  // group q (q = 0 .. n_m3) = post_chk[post_chk_off[q] .. post_chk_off[q+1])
  std::vector<uint32_t> post_chk_off, post_chk;

  // dense executor
  std::vector<DenseInstr> dense;
  std::vector<uint32_t> dense_causal;    // m3 index lists
  uint32_t n_m3 = 0;
  std::vector<uint32_t> m3_t;            // ordinal of each m3 symbol

  uint64_t sign_xor_terms = 0;
  // commutation-aware simplification: rotations merged into an earlier one,
  // merged rotations removed (angle a multiple of 2 pi), rotations removed as
  // branch phases of a later same-body measurement
  uint32_t n_fused = 0, n_cancelled = 0, n_branch_phase = 0;
  // product-component form of the dense instruction stream
  PCProgram pc;
};

HostPlan compile_plan(const Circuit& c, const symft_options& opt);

}  // namespace symft
