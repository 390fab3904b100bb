// Compile step: symbolic Clifford-Pauli frame factorization (Sec. 3),
// stabilizer-coordinate planning (Sec. 4) and lowering to the device plan
// (Sec. 6: precompiled instruction descriptors, packed independent symbols).
//
// Representation choices (all host side, run once per circuit):
//  * Paulis are i^e X^x Z^z over n qubits with x, z as 64-bit word vectors.
//  * The Clifford frame C_t is kept as its pull-back map (images of X_q, Z_q
//    under P -> C_t^dag P C_t); a new gate g updates it by
//    T_new(Q) = T_old(g^dag Q g) (Sec. 3, rule C_t = g C_{t-1}).
//  * The symbolic Pauli frame E_t is kept in column form over the pulled-back
//    qubits: Ex[j] / Ez[j] are affine expressions (bitsets over symbols plus a
//    constant bit) giving E's X and Z exponents on qubit j.  Noise uses the
//    symplectic component bits of each channel (x_q, z_q per qubit of its
//    support); since the anticommutation indicator is bilinear this gives the
//    same sign as the one-hot variables of Eq. symbolic-noise-sign.
//  * lambda_t = omega(E_{t-1}, P') is read off the columns of P' (Sec. 3).
//  * The planner follows Sec. 4 case by case; symbolic corrections of the
//    measurement cases are appended to E, so later signs pick them up.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.hpp"

namespace symft {
namespace {

inline int popc(uint64_t v) { return __builtin_popcountll(v); }

// ---------------------------------------------------------------- Paulis ----
struct Pauli {
  std::vector<uint64_t> x, z;
  int e = 0;  // power of i
};

struct PauliAlg {
  int nw;
  explicit PauliAlg(int n) : nw((n + 63) / 64) {}
  Pauli identity() const {
    Pauli p;
    p.x.assign(nw, 0);
    p.z.assign(nw, 0);
    return p;
  }
  Pauli single(uint32_t q, bool xb, bool zb, int e = 0) const {
    Pauli p = identity();
    if (xb) p.x[q >> 6] |= 1ull << (q & 63);
    if (zb) p.z[q >> 6] |= 1ull << (q & 63);
    p.e = e & 3;
    return p;
  }
  // a <- a * b
  void mul_into(Pauli& a, const Pauli& b) const {
    int cnt = 0;
    for (int w = 0; w < nw; ++w) {
      cnt += popc(a.z[w] & b.x[w]);
      a.x[w] ^= b.x[w];
      a.z[w] ^= b.z[w];
    }
    a.e = (a.e + b.e + 2 * cnt) & 3;
  }
  int omega(const Pauli& a, const Pauli& b) const {
    uint64_t acc = 0;
    for (int w = 0; w < nw; ++w) acc ^= (a.x[w] & b.z[w]) ^ (a.z[w] & b.x[w]);
    return popc(acc) & 1;
  }
  bool same_support(const Pauli& a, const Pauli& b) const {
    return a.x == b.x && a.z == b.z;
  }
};

// ------------------------------------------------- affine expressions ----
// Bitset over NS symbols; bit NS is the constant term.
struct Expr {
  std::vector<uint64_t> w;
};

struct ExprAlg {
  uint32_t ns, nw;
  explicit ExprAlg(uint32_t nsym) : ns(nsym), nw((nsym + 1 + 63) / 64) {}
  Expr zero() const { return Expr{std::vector<uint64_t>(nw, 0)}; }
  Expr sym(uint32_t s) const {
    Expr e = zero();
    e.w[s >> 6] |= 1ull << (s & 63);
    return e;
  }
  void flip(Expr& e, uint32_t s) const { e.w[s >> 6] ^= 1ull << (s & 63); }
  bool get(const Expr& e, uint32_t s) const { return (e.w[s >> 6] >> (s & 63)) & 1; }
  void xor_into(Expr& a, const Expr& b) const {
    for (uint32_t i = 0; i < nw; ++i) a.w[i] ^= b.w[i];
  }
  bool constant(const Expr& e) const { return get(e, ns); }
  template <class F>
  void for_each(const Expr& e, uint32_t lo, uint32_t hi, F f) const {
    for (uint32_t wi = lo >> 6; wi <= ((hi - 1) >> 6) && wi < nw && lo < hi; ++wi) {
      uint64_t v = e.w[wi];
      while (v) {
        uint32_t s = wi * 64 + __builtin_ctzll(v);
        v &= v - 1;
        if (s >= lo && s < hi) f(s);
      }
    }
  }
};

// ------------------------------------------ gate Heisenberg images ----
// g^dag Q g for the local generators Q in {X_a, Z_a, X_b, Z_b}, as
// (x bits, z bits, e) over the local qubits (bit 0 = a, bit 1 = b).
struct LocalPauli {
  int x, z, e;
};

void gate_images(int g, LocalPauli img[4]) {
  // defaults: identity map
  img[0] = {1, 0, 0};  // X_a
  img[1] = {0, 1, 0};  // Z_a
  img[2] = {2, 0, 0};  // X_b
  img[3] = {0, 2, 0};  // Z_b
  switch (g) {
    case G_I: break;
    case G_H: img[0] = {0, 1, 0}; img[1] = {1, 0, 0}; break;
    case G_S: img[0] = {1, 1, 3}; break;            // S^dag X S = -Y = -i X Z
    case G_S_DAG: img[0] = {1, 1, 1}; break;        // S X S^dag = Y = i X Z
    case G_X: img[1] = {0, 1, 2}; break;            // X Z X = -Z
    case G_Z: img[0] = {1, 0, 2}; break;            // Z X Z = -X
    case G_Y: img[0] = {1, 0, 2}; img[1] = {0, 1, 2}; break;
    case G_SQRT_X: img[1] = {1, 1, 1}; break;       // Z -> Y
    case G_SQRT_X_DAG: img[1] = {1, 1, 3}; break;   // Z -> -Y
    case G_CX:  // control a, target b (self-inverse)
      img[0] = {3, 0, 0};   // X_a -> X_a X_b
      img[3] = {0, 3, 0};   // Z_b -> Z_a Z_b
      break;
    case G_CZ:
      img[0] = {1, 2, 0};   // X_a -> X_a Z_b
      img[2] = {2, 1, 0};   // X_b -> Z_a X_b
      break;
    case G_CY:
      img[0] = {3, 2, 1};   // X_a -> X_a Y_b = i X_a X_b Z_b
      img[2] = {2, 1, 0};   // X_b -> Z_a X_b
      img[3] = {0, 3, 0};   // Z_b -> Z_a Z_b
      break;
    case G_SWAP:
      img[0] = {2, 0, 0}; img[1] = {0, 2, 0}; img[2] = {1, 0, 0}; img[3] = {0, 1, 0};
      break;
    default: throw Error(SYMFT_E_UNSUPPORTED, "unknown gate");
  }
}

// ---------------------------------------------------------- compiler ----
struct RawInstr {
  int kind;
  uint32_t t = 0;
  uint32_t a = 0, b = 0;
  int h = 0, mu = 0, eta = 0, k = 0;
  double theta = 0.0;
  Expr lam;
};

class Compiler {
 public:
  Compiler(const Circuit& c, const symft_options& opt)
      : c_(c), opt_(opt), n_(c.n_qubits), pa_(std::max<uint32_t>(c.n_qubits, 1)),
        ea_(1) {}

  HostPlan run();

 private:
  const Circuit& c_;
  symft_options opt_;
  uint32_t n_;
  PauliAlg pa_;
  ExprAlg ea_;
  uint32_t n_comp_ = 0;
  std::vector<uint32_t> chan_comp0_;
  std::vector<uint8_t> chan_ncomp_;

  // Clifford frame as pull-back map
  std::vector<Pauli> TX_, TZ_;
  // symbolic Pauli frame, column form
  std::vector<Expr> Ex_, Ez_;
  // planner tableau
  std::vector<Pauli> Zb_, Xb_;
  uint32_t k_ = 0, kmax_ = 0;
  std::vector<RawInstr> instrs_;

  // Factorized operator sequence (Sec. 3): rotations R_P(theta) and Pauli
  // measurements with P pulled back through the Clifford frame and the sign
  // lam from the noise and feedback terms of the Pauli frame; detectors and
  // observables are segment boundaries.
  struct FOp {
    int kind;          // 0 rotation, 1 measurement, 2 detector / observable boundary
    Pauli p;
    double theta = 0.0;
    uint32_t t = 0;
    Expr lam;
    bool dead = false;
  };
  uint32_t n_fused_ = 0, n_cancelled_ = 0, n_branch_phase_ = 0;

  bool symbol_free(const Expr& e) const {
    for (uint32_t w = 0; w < ea_.nw; ++w) {
      uint64_t v = e.w[w];
      if (w == (ea_.ns >> 6)) v &= ~(1ull << (ea_.ns & 63));
      if (v) return false;
    }
    return true;
  }

  // Commutation-aware simplification before planning (Sec. 6): conservative
  // local rewrites inside each segment between detector positions.
  //  - Rotation fusion: a rotation whose Pauli body equals that of an earlier
  //    rotation, with every operation in between commuting with it and with
  //    signs that differ by a constant (lam_i ^ lam_j has no symbol), is
  //    merged into the earlier one; the merged rotation is removed when its
  //    angle is a multiple of 2 pi (the identity up to a global phase).
  //  - Branch phase: a rotation followed, across operations that all commute
  //    with it, by a measurement of the same Pauli body acts on each outcome's
  //    eigenspace as a phase only, so it is removed.
  // Measurements never move, so record order, detector boundaries and the
  // measurement symbols every sign uses stay as they were.
  void simplify(std::vector<FOp>& f) {
    constexpr size_t kScan = 512;   // operations examined per rewrite search
    for (size_t j = 0; j < f.size(); ++j) {
      if (f[j].kind != 0 || f[j].dead) continue;
      size_t steps = 0;
      for (size_t i = j; i-- > 0 && steps < kScan; ++steps) {
        FOp& o = f[i];
        if (o.dead) continue;
        if (o.kind == 2) break;
        if (o.kind == 0 && pa_.same_support(o.p, f[j].p)) {
          Expr d = o.lam;
          ea_.xor_into(d, f[j].lam);
          if (symbol_free(d)) {
            // P_j = s P_i with s = +-1 from the phases; signed angles add
            const int rel = (ea_.constant(d) ? 1 : 0) ^ ((((o.p.e - f[j].p.e) & 3) == 2) ? 1 : 0);
            o.theta += rel ? -f[j].theta : f[j].theta;
            f[j].dead = true;
            ++n_fused_;
            const double two_pi = 6.283185307179586;
            const double r = std::fabs(std::remainder(o.theta, two_pi));
            if (r < 1e-12) {
              o.dead = true;
              ++n_cancelled_;
            }
            break;
          }
        }
        if (pa_.omega(o.p, f[j].p)) break;
      }
    }
    for (size_t i = 0; i < f.size(); ++i) {
      if (f[i].kind != 0 || f[i].dead) continue;
      size_t steps = 0;
      for (size_t j = i + 1; j < f.size() && steps < kScan; ++j, ++steps) {
        const FOp& o = f[j];
        if (o.dead) continue;
        if (o.kind == 2) break;
        if (o.kind == 1 && pa_.same_support(o.p, f[i].p)) {
          f[i].dead = true;
          ++n_branch_phase_;
          break;
        }
        if (pa_.omega(o.p, f[i].p)) break;
      }
    }
  }

  uint32_t msym(uint32_t t) const { return n_comp_ + t; }

  Pauli pull_back_local(const LocalPauli& lp, uint32_t qa, uint32_t qb) const {
    Pauli out = pa_.identity();
    out.e = lp.e;
    uint32_t qs[2] = {qa, qb};
    for (int j = 0; j < 2; ++j)
      if ((lp.x >> j) & 1) pa_.mul_into(out, TX_[qs[j]]);
    for (int j = 0; j < 2; ++j)
      if ((lp.z >> j) & 1) pa_.mul_into(out, TZ_[qs[j]]);
    return out;
  }

  Pauli pull_back(const std::vector<PauliTerm>& p) const {
    Pauli out = pa_.identity();
    int ny = 0;
    for (auto& t : p)
      if (t.p == 'Y') ++ny;
    out.e = ny & 3;  // Y = i X Z
    for (auto& t : p)
      if (t.p == 'X' || t.p == 'Y') pa_.mul_into(out, TX_[t.q]);
    for (auto& t : p)
      if (t.p == 'Z' || t.p == 'Y') pa_.mul_into(out, TZ_[t.q]);
    return out;
  }

  void apply_gate(const Op& op) {
    LocalPauli img[4];
    gate_images(op.gate, img);
    bool two = op.gate >= G_CX;
    uint32_t qa = op.q0, qb = two ? op.q1 : op.q0;
    Pauli nxa = pull_back_local(img[0], qa, qb);
    Pauli nza = pull_back_local(img[1], qa, qb);
    if (two) {
      Pauli nxb = pull_back_local(img[2], qa, qb);
      Pauli nzb = pull_back_local(img[3], qa, qb);
      TX_[qb] = std::move(nxb);
      TZ_[qb] = std::move(nzb);
    }
    TX_[qa] = std::move(nxa);
    TZ_[qa] = std::move(nza);
  }

  // E <- Q^{expr} E   (column form; Q pulled back)
  void frame_add_symbol(const Pauli& q, uint32_t sym) {
    for (int w = 0; w < pa_.nw; ++w) {
      uint64_t vx = q.x[w], vz = q.z[w];
      while (vx) {
        uint32_t j = w * 64 + __builtin_ctzll(vx);
        vx &= vx - 1;
        ea_.flip(Ex_[j], sym);
      }
      while (vz) {
        uint32_t j = w * 64 + __builtin_ctzll(vz);
        vz &= vz - 1;
        ea_.flip(Ez_[j], sym);
      }
    }
  }
  void frame_add_expr(const Pauli& q, const Expr& ex) {
    for (int w = 0; w < pa_.nw; ++w) {
      uint64_t vx = q.x[w], vz = q.z[w];
      while (vx) {
        uint32_t j = w * 64 + __builtin_ctzll(vx);
        vx &= vx - 1;
        ea_.xor_into(Ex_[j], ex);
      }
      while (vz) {
        uint32_t j = w * 64 + __builtin_ctzll(vz);
        vz &= vz - 1;
        ea_.xor_into(Ez_[j], ex);
      }
    }
  }
  Expr frame_sign(const Pauli& p) const {
    Expr lam = ea_.zero();
    for (int w = 0; w < pa_.nw; ++w) {
      uint64_t vz = p.z[w], vx = p.x[w];
      while (vz) {
        uint32_t j = w * 64 + __builtin_ctzll(vz);
        vz &= vz - 1;
        ea_.xor_into(lam, Ex_[j]);
      }
      while (vx) {
        uint32_t j = w * 64 + __builtin_ctzll(vx);
        vx &= vx - 1;
        ea_.xor_into(lam, Ez_[j]);
      }
    }
    return lam;
  }

  // --- Sec. 4: decomposition P = mu Xbar_A^a Zbar_A^b Xbar_D^d Zbar_D^c ---
  struct Decomp {
    uint32_t a = 0, b = 0;
    int first_d = -1;               // lowest dormant index with d = 1
    std::vector<uint8_t> d, c;      // dormant bits, index j - k
    int mu = 0;
  };
  Decomp decompose(const Pauli& p, bool need_mu) const {
    Decomp D;
    D.d.assign(n_ - k_, 0);
    D.c.assign(n_ - k_, 0);
    for (uint32_t j = 0; j < k_; ++j) {
      if (pa_.omega(p, Zb_[j])) D.a |= 1u << j;
      if (pa_.omega(p, Xb_[j])) D.b |= 1u << j;
    }
    for (uint32_t j = k_; j < n_; ++j) {
      D.d[j - k_] = pa_.omega(p, Zb_[j]);
      D.c[j - k_] = pa_.omega(p, Xb_[j]);
      if (D.d[j - k_] && D.first_d < 0) D.first_d = static_cast<int>(j);
    }
    if (need_mu && D.first_d < 0) {
      Pauli q = pa_.identity();
      for (uint32_t j = 0; j < k_; ++j)
        if ((D.a >> j) & 1) pa_.mul_into(q, Xb_[j]);
      for (uint32_t j = 0; j < k_; ++j)
        if ((D.b >> j) & 1) pa_.mul_into(q, Zb_[j]);
      for (uint32_t j = k_; j < n_; ++j)
        if (D.c[j - k_]) pa_.mul_into(q, Zb_[j]);
      if (!pa_.same_support(p, q)) throw Error(SYMFT_E_DEVICE, "internal: tableau does not span P");
      D.mu = (p.e - q.e) & 3;
    }
    return D;
  }

  // symplectic coordinate change with dormant pivot h (Sec. 4.1 / 4.2)
  void dormant_pivot_update(const Pauli& p, const Decomp& D, uint32_t h) {
    const Pauli zh = Zb_[h];
    for (uint32_t j = 0; j < k_; ++j) {
      if ((D.a >> j) & 1) pa_.mul_into(Zb_[j], zh);
      if ((D.b >> j) & 1) pa_.mul_into(Xb_[j], zh);
    }
    for (uint32_t j = k_; j < n_; ++j) {
      if (j == h) continue;
      if (D.d[j - k_]) pa_.mul_into(Zb_[j], zh);
      if (D.c[j - k_]) pa_.mul_into(Xb_[j], zh);
    }
    Xb_[h] = p;
  }
  void swap_pair(uint32_t i, uint32_t j) {
    std::swap(Zb_[i], Zb_[j]);
    std::swap(Xb_[i], Xb_[j]);
  }
  void retire_active(uint32_t h) {
    Pauli zp = Zb_[h], xp = Xb_[h];
    for (uint32_t j = h; j + 1 < k_; ++j) {
      Zb_[j] = std::move(Zb_[j + 1]);
      Xb_[j] = std::move(Xb_[j + 1]);
    }
    Zb_[k_ - 1] = std::move(zp);
    Xb_[k_ - 1] = std::move(xp);
    --k_;
  }

  void plan_rotation(const Pauli& p, double theta, Expr lam) {
    Decomp D = decompose(p, true);
    RawInstr I;
    I.theta = theta;
    I.k = static_cast<int>(k_);
    if (D.first_d >= 0) {
      uint32_t h = static_cast<uint32_t>(D.first_d);
      dormant_pivot_update(p, D, h);
      if (h != k_) swap_pair(h, k_);
      ++k_;
      if (k_ > kMaxActive)
        throw Error(SYMFT_E_CAPACITY, "active width exceeds the build limit of " + std::to_string(kMaxActive));
      kmax_ = std::max(kmax_, k_);
      I.kind = I_PROMOTE_ROT;
      I.lam = std::move(lam);
      instrs_.push_back(std::move(I));
      return;
    }
    if (D.a == 0 && D.b == 0) return;  // global phase only
    I.a = D.a;
    I.b = D.b;
    I.mu = D.mu;
    I.lam = std::move(lam);
    I.kind = D.a == 0 ? I_ACTIVE_DIAG_ROT : I_ACTIVE_PAIR_ROT;
    if (I.kind == I_ACTIVE_DIAG_ROT && (D.mu & 1))
      throw Error(SYMFT_E_DEVICE, "internal: non-real phase in diagonal rotation");
    instrs_.push_back(std::move(I));
  }

  void plan_measurement(const Pauli& p, uint32_t t, Expr lam) {
    Decomp D = decompose(p, true);
    RawInstr I;
    I.t = t;
    I.k = static_cast<int>(k_);
    if (D.first_d >= 0) {
      // dormant-nondiagonal: random measurement, correction (Xbar_h'')^{m xor lambda}
      uint32_t h = static_cast<uint32_t>(D.first_d);
      dormant_pivot_update(p, D, h);
      Pauli zh = Zb_[h];
      Zb_[h] = p;
      Xb_[h] = zh;
      Expr corr = lam;
      ea_.flip(corr, msym(t));
      frame_add_expr(Xb_[h], corr);
      I.kind = I_RANDOM_MEAS;
      instrs_.push_back(std::move(I));
      return;
    }
    if (D.a == 0 && D.b == 0) {
      if (D.mu & 1) throw Error(SYMFT_E_DEVICE, "internal: non-Hermitian deterministic measurement");
      I.kind = I_DET_MEAS;
      I.eta = D.mu >> 1;
      I.lam = std::move(lam);
      instrs_.push_back(std::move(I));
      return;
    }
    if (D.a == 0) {
      // active-diagonal measurement, pivot = highest set bit of b
      if (D.mu & 1) throw Error(SYMFT_E_DEVICE, "internal: non-Hermitian diagonal measurement");
      int eta = D.mu >> 1;
      uint32_t h = 31 - __builtin_clz(D.b);
      const Pauli xh = Xb_[h];
      for (uint32_t j = 0; j < k_; ++j)
        if (j != h && ((D.b >> j) & 1)) pa_.mul_into(Xb_[j], xh);
      for (uint32_t j = k_; j < n_; ++j)
        if (D.c[j - k_]) pa_.mul_into(Xb_[j], xh);
      Pauli zn = p;
      zn.e = (zn.e + 2 * eta) & 3;
      Zb_[h] = std::move(zn);
      Expr corr = lam;
      ea_.flip(corr, msym(t));
      if (eta) ea_.flip(corr, ea_.ns);
      frame_add_expr(Xb_[h], corr);
      retire_active(h);
      I.kind = I_ACTIVE_DIAG_MEAS;
      I.b = D.b;
      I.h = static_cast<int>(h);
      I.eta = eta;
      I.lam = std::move(lam);
      instrs_.push_back(std::move(I));
      return;
    }
    // active-nondiagonal measurement, pivot = highest set bit of a
    uint32_t h = 31 - __builtin_clz(D.a);
    const Pauli zh = Zb_[h];
    for (uint32_t j = 0; j < k_; ++j) {
      if (j == h) continue;
      if ((D.a >> j) & 1) pa_.mul_into(Zb_[j], zh);
      if ((D.b >> j) & 1) pa_.mul_into(Xb_[j], zh);
    }
    for (uint32_t j = k_; j < n_; ++j)
      if (D.c[j - k_]) pa_.mul_into(Xb_[j], zh);
    Zb_[h] = p;
    Xb_[h] = zh;
    Expr corr = lam;
    ea_.flip(corr, msym(t));
    frame_add_expr(Xb_[h], corr);
    retire_active(h);
    I.kind = I_ACTIVE_PAIR_MEAS;
    I.a = D.a;
    I.b = D.b;
    I.h = static_cast<int>(h);
    I.mu = D.mu;
    I.lam = std::move(lam);
    instrs_.push_back(std::move(I));
  }

  void lower(HostPlan& P);
};

int chan_ncomp(int chan) {
  switch (chan) {
    case CH_X: case CH_Z: return 1;
    case CH_Y: case CH_XYZ: return 2;
    case CH_D2: return 4;
  }
  return 0;
}

HostPlan Compiler::run() {
  // symbols: noise components first, then measurement ordinals
  chan_comp0_.assign(c_.n_channels, 0);
  chan_ncomp_.assign(c_.n_channels, 0);
  for (auto& op : c_.ops)
    if (op.kind == OP_NOISE) {
      chan_comp0_[op.channel] = n_comp_;
      chan_ncomp_[op.channel] = static_cast<uint8_t>(chan_ncomp(op.chan));
      n_comp_ += chan_ncomp_[op.channel];
    }
  ea_ = ExprAlg(n_comp_ + c_.n_meas);
  uint32_t nq = std::max<uint32_t>(n_, 1);
  TX_.resize(nq);
  TZ_.resize(nq);
  Zb_.resize(nq);
  Xb_.resize(nq);
  for (uint32_t q = 0; q < nq; ++q) {
    TX_[q] = pa_.single(q, true, false);
    TZ_[q] = pa_.single(q, false, true);
    Zb_[q] = pa_.single(q, false, true);
    Xb_[q] = pa_.single(q, true, false);
  }
  Ex_.assign(nq, ea_.zero());
  Ez_.assign(nq, ea_.zero());

  // 1. factorization: the frame holds the noise and feedback terms only
  std::vector<FOp> fops;
  for (const Op& op : c_.ops) {
    switch (op.kind) {
      case OP_CLIFF:
        apply_gate(op);
        break;
      case OP_NOISE: {
        uint32_t s = chan_comp0_[op.channel];
        uint32_t qs[2] = {op.q0, op.q1};
        int nqb = op.chan == CH_D2 ? 2 : 1;
        for (int j = 0; j < nqb; ++j) {
          bool hx = op.chan != CH_Z, hz = op.chan != CH_X;
          if (hx) frame_add_symbol(TX_[qs[j]], s++);
          if (hz) frame_add_symbol(TZ_[qs[j]], s++);
        }
        break;
      }
      case OP_FB: {
        Pauli q = pull_back(op.pauli);
        Expr ex = ea_.zero();
        for (uint32_t t : op.conds) ea_.flip(ex, msym(t));
        frame_add_expr(q, ex);
        break;
      }
      case OP_ROT: {
        FOp f;
        f.kind = 0;
        f.p = pull_back(op.pauli);
        f.lam = frame_sign(f.p);
        f.theta = op.theta;
        fops.push_back(std::move(f));
        break;
      }
      case OP_MEAS: {
        FOp f;
        f.kind = 1;
        f.p = pull_back(op.pauli);
        f.lam = frame_sign(f.p);
        f.t = op.t;
        fops.push_back(std::move(f));
        break;
      }
      case OP_DET:
      case OP_OBS: {
        FOp f;
        f.kind = 2;
        fops.push_back(std::move(f));
        break;
      }
    }
  }
  // 2. commutation-aware simplification
  if (!opt_.no_simplify) simplify(fops);
  // 3. planning (Sec. 4): the frame now accumulates the planner's measurement
  //    corrections, and an operation's sign is its factorized sign XOR theirs
  for (uint32_t q = 0; q < nq; ++q) {
    Ex_[q] = ea_.zero();
    Ez_[q] = ea_.zero();
  }
  for (FOp& f : fops) {
    if (f.dead || f.kind == 2) continue;
    Expr lam = frame_sign(f.p);
    ea_.xor_into(lam, f.lam);
    if (f.kind == 0) plan_rotation(f.p, f.theta, std::move(lam));
    else plan_measurement(f.p, f.t, std::move(lam));
  }
  HostPlan P;
  lower(P);
  P.n_fused = n_fused_;
  P.n_cancelled = n_cancelled_;
  P.n_branch_phase = n_branch_phase_;
  P.pc = build_product_components(P.dense, P.k_max);
  if (opt_.no_product_components) P.pc.use = false;
  return P;
}

// ------------------------------------------------------------- lowering ----
void Compiler::lower(HostPlan& P) {
  P.n_qubits = c_.n_qubits;
  P.n_meas = c_.n_meas;
  P.n_records = c_.n_records;
  P.n_dets = c_.n_dets;
  P.n_obs = c_.n_obs;
  P.n_channels = c_.n_channels;
  P.k_max = kmax_;
  P.n_comp = n_comp_;
  for (auto& I : instrs_) P.hist[I.kind]++;

  const uint32_t NM = c_.n_meas;
  // symbol classes of measurement ordinals
  std::vector<int> cls(NM, -1);           // 1: m1, 2: m2, 3: m3
  std::vector<int32_t> m1_index(NM, -1), m3_index(NM, -1);
  std::vector<const RawInstr*> det_of(NM, nullptr);
  for (auto& I : instrs_) {
    if (I.kind == I_RANDOM_MEAS) {
      cls[I.t] = 1;
      m1_index[I.t] = static_cast<int32_t>(P.m1_t.size());
      P.m1_t.push_back(I.t);
    } else if (I.kind == I_DET_MEAS) {
      cls[I.t] = 2;
      det_of[I.t] = &I;
    } else if (I.kind == I_ACTIVE_DIAG_MEAS || I.kind == I_ACTIVE_PAIR_MEAS) {
      cls[I.t] = 3;
      m3_index[I.t] = static_cast<int32_t>(P.m3_t.size());
      P.m3_t.push_back(I.t);
    }
  }
  P.n_m3 = static_cast<uint32_t>(P.m3_t.size());
  for (uint32_t t = 0; t < NM; ++t)
    if (cls[t] < 0) throw Error(SYMFT_E_DEVICE, "internal: measurement without instruction");

  // resolve deterministic outcomes: res[t] over {components, m1, m3, const}
  const uint32_t NS = ea_.ns;
  std::vector<Expr> res(NM);
  auto resolve = [&](const Expr& in) {
    Expr out = in;
    // clear measurement symbols of class m2 and substitute
    for (uint32_t wi = n_comp_ >> 6; wi < ea_.nw; ++wi) {
      uint64_t v = in.w[wi];
      while (v) {
        uint32_t s = wi * 64 + __builtin_ctzll(v);
        v &= v - 1;
        if (s < n_comp_ || s >= NS) continue;
        uint32_t t = s - n_comp_;
        if (cls[t] == 2) {
          ea_.flip(out, s);
          ea_.xor_into(out, res[t]);
        }
      }
    }
    return out;
  };
  std::vector<Expr> dense_lam;
  std::vector<const RawInstr*> dense_src;
  for (auto& I : instrs_) {
    if (I.kind == I_RANDOM_MEAS) {
      res[I.t] = ea_.sym(msym(I.t));
    } else if (I.kind == I_DET_MEAS) {
      Expr r = resolve(I.lam);
      if (I.eta) ea_.flip(r, NS);
      res[I.t] = std::move(r);
      uint32_t w = 0;
      ea_.for_each(res[I.t], 0, NS, [&](uint32_t) { ++w; });
      P.max_expr_weight = std::max(P.max_expr_weight, w);
    } else {
      Expr r = resolve(I.lam);
      uint32_t w = 0;
      ea_.for_each(r, 0, NS, [&](uint32_t) { ++w; });
      P.max_expr_weight = std::max(P.max_expr_weight, w);
      dense_lam.push_back(std::move(r));
      dense_src.push_back(&I);
      if (I.kind == I_ACTIVE_DIAG_MEAS || I.kind == I_ACTIVE_PAIR_MEAS)
        res[I.t] = ea_.sym(msym(I.t));
    }
  }

  // ---- outputs: records, detectors, observables (full expressions) ----
  const uint32_t R = c_.n_records, Dn = c_.n_dets, O = c_.n_obs;
  const uint32_t G = static_cast<uint32_t>(dense_lam.size());
  P.tgt_rec0 = 0;
  P.tgt_det0 = R;
  P.tgt_obs0 = R + Dn;
  P.tgt_sign0 = R + Dn + O;
  P.n_targets = R + Dn + O;
  std::vector<Expr> full(P.n_targets);
  for (uint32_t r = 0; r < R; ++r) full[r] = res[c_.record_ordinal[r]];
  std::vector<std::vector<uint32_t>> gat(Dn + O);
  for (uint32_t i = 0; i < Dn + O; ++i) full[R + i] = ea_.zero();
  std::vector<int32_t> rec_of_t(NM, -1);
  for (uint32_t r = 0; r < R; ++r) rec_of_t[c_.record_ordinal[r]] = static_cast<int32_t>(r);
  for (const Op& op : c_.ops) {
    if (op.kind != OP_DET && op.kind != OP_OBS) continue;
    uint32_t slot = (op.kind == OP_DET ? 0 : Dn) + op.index;
    for (uint32_t t : op.conds) {
      ea_.xor_into(full[R + slot], res[t]);
      gat[slot].push_back(static_cast<uint32_t>(rec_of_t[t]));
    }
  }
  // gather lists with duplicates cancelled (parity)
  P.gat_off.assign(Dn + O + 1, 0);
  for (uint32_t i = 0; i < Dn + O; ++i) {
    std::sort(gat[i].begin(), gat[i].end());
    std::vector<uint32_t> keep;
    for (size_t j = 0; j < gat[i].size();) {
      size_t e = j;
      while (e < gat[i].size() && gat[i][e] == gat[i][j]) ++e;
      if ((e - j) & 1) keep.push_back(gat[i][j]);
      j = e;
    }
    P.gat_rec.insert(P.gat_rec.end(), keep.begin(), keep.end());
    P.gat_off[i + 1] = static_cast<uint32_t>(P.gat_rec.size());
  }
  // causal (active-outcome) parts of every output, for the finalize pass
  P.tgt_causal_off.assign(P.n_targets + 1, 0);
  for (uint32_t i = 0; i < P.n_targets; ++i) {
    ea_.for_each(full[i], n_comp_, NS, [&](uint32_t s) {
      uint32_t t = s - n_comp_;
      if (cls[t] == 3) P.tgt_causal.push_back(static_cast<uint32_t>(m3_index[t]));
      else if (cls[t] == 2) throw Error(SYMFT_E_DEVICE, "internal: unresolved deterministic symbol");
    });
    P.tgt_causal_off[i + 1] = static_cast<uint32_t>(P.tgt_causal.size());
  }

  // ---- plain form: full exogenous symbol lists of every output and dense sign ----
  {
    const uint32_t NTP = R + Dn + O + G;
    P.plain_const.assign(NTP, 0);
    P.plain_off.assign(NTP + 1, 0);
    for (uint32_t i = 0; i < NTP; ++i) {
      const Expr& e = i < R + Dn + O ? full[i] : dense_lam[i - (R + Dn + O)];
      P.plain_const[i] = ea_.constant(e);
      ea_.for_each(e, 0, NS, [&](uint32_t sidx) {
        if (sidx < n_comp_) {
          P.plain_sym.push_back(sidx);
        } else {
          uint32_t t = sidx - n_comp_;
          if (cls[t] == 1) P.plain_sym.push_back(n_comp_ + static_cast<uint32_t>(m1_index[t]));
        }
      });
      P.plain_off[i + 1] = static_cast<uint32_t>(P.plain_sym.size());
    }
  }

  // ---- exogenous record parts, delta-chained to earlier records ----
  // The sign kernel evaluates exo_r = const ^ delta_r ^ exo(parent).  A parent
  // is taken when it removes enough weighted incidences: a noise component
  // costs work only in the rare blocks where it fires, a random-measurement
  // bit every block, a parent one word-XOR per block.
  Expr m3mask = ea_.zero(), m1mask = ea_.zero();
  for (uint32_t t = 0; t < NM; ++t) {
    if (cls[t] == 3) ea_.flip(m3mask, msym(t));
    if (cls[t] == 1) ea_.flip(m1mask, msym(t));
  }
  auto strip_causal = [&](const Expr& e) {
    Expr o = e;
    for (uint32_t w = 0; w < ea_.nw; ++w) o.w[w] &= ~m3mask.w[w];
    return o;
  };
  const uint32_t sym_words = ea_.nw;
  const uint64_t const_bit_mask_word = NS >> 6;
  const uint64_t const_bit = 1ull << (NS & 63);
  auto cost = [&](const Expr& e) {
    uint64_t c = 0;
    for (uint32_t w = 0; w < sym_words; ++w) {
      uint64_t v = e.w[w];
      if (w == const_bit_mask_word) v &= ~const_bit;
      c += __builtin_popcountll(v) + 15ull * __builtin_popcountll(v & m1mask.w[w]);
    }
    return c;
  };
  std::vector<Expr> exo(R);
  for (uint32_t r = 0; r < R; ++r) exo[r] = strip_causal(full[r]);
  std::vector<std::vector<uint32_t>> parents(R);
  std::vector<Expr> delta(R);
  std::vector<std::vector<uint32_t>> inv(NS);       // symbol -> records containing it
  constexpr uint64_t kParentGain = 20;
  constexpr size_t kMaxCand = 96;
  // The chains are paths: a record takes at most one parent, and a record is
  // the parent of at most one other, so the sign kernel walks each path in one
  // thread with no barrier between its records.  (More parents, or several
  // children per parent, remove more incidences -- d=7: 2.61 against 3.31
  // targets per fired cell -- but the kernel then resolves the records level
  // by level with a CTA barrier per level, measured slower.)  Paths are cut
  // after kMaxLevels records.
  constexpr int kMaxParents = 1;
  constexpr uint32_t kMaxLevel = kMaxLevels - 1;
  std::vector<uint32_t> level(R, 0);
  std::vector<uint8_t> has_child(R, 0);
  std::vector<uint32_t> seen_mark(R, 0xFFFFFFFFu);
  for (uint32_t r = 0; r < R; ++r) {
    Expr resid = exo[r];
    uint64_t cres = cost(resid);
    for (int it = 0; it < kMaxParents && cres > kParentGain; ++it) {
      // candidates: earlier records sharing a symbol with the residual
      std::vector<uint32_t> cand;
      ea_.for_each(resid, 0, NS, [&](uint32_t sidx) {
        if (cand.size() >= kMaxCand) return;
        const auto& lst = inv[sidx];
        for (size_t j = lst.size(); j-- > 0 && cand.size() < kMaxCand;) {
          uint32_t p = lst[j];
          if (level[p] >= kMaxLevel || has_child[p]) continue;
          if (seen_mark[p] != r * 8 + it) {
            seen_mark[p] = r * 8 + it;
            cand.push_back(p);
          }
        }
      });
      uint64_t best_c = cres;
      int64_t best = -1;
      for (uint32_t p : cand) {
        Expr x = resid;
        ea_.xor_into(x, exo[p]);
        uint64_t c = cost(x);
        if (c < best_c) {
          best_c = c;
          best = p;
        }
      }
      if (best < 0 || cres - best_c < kParentGain) break;
      ea_.xor_into(resid, exo[best]);
      cres = best_c;
      parents[r].push_back(static_cast<uint32_t>(best));
      has_child[best] = 1;
      level[r] = std::max(level[r], level[best] + 1);
    }
    delta[r] = std::move(resid);
    ea_.for_each(exo[r], 0, NS, [&](uint32_t sidx) { inv[sidx].push_back(r); });
  }
  P.par_off.assign(R + 1, 0);
  for (uint32_t r = 0; r < R; ++r) {
    P.par.insert(P.par.end(), parents[r].begin(), parents[r].end());
    P.par_off[r + 1] = static_cast<uint32_t>(P.par.size());
  }

  // ---- sign-kernel slots: [records (deltas)][dense signs (exogenous part)] ----
  P.n_slots = R + G;
  std::vector<Expr> slot_expr(P.n_slots);
  for (uint32_t r = 0; r < R; ++r) slot_expr[r] = std::move(delta[r]);
  std::vector<std::vector<uint32_t>> sign_causal(G);
  for (uint32_t g = 0; g < G; ++g) {
    slot_expr[R + g] = strip_causal(dense_lam[g]);
    ea_.for_each(dense_lam[g], n_comp_, NS, [&](uint32_t sidx) {
      uint32_t t = sidx - n_comp_;
      if (cls[t] == 3) sign_causal[g].push_back(static_cast<uint32_t>(m3_index[t]));
    });
  }
  std::vector<std::vector<uint32_t>> comp_t(n_comp_), m1_t(P.m1_t.size());
  P.slot_const.assign(P.n_slots, 0);
  for (uint32_t i = 0; i < P.n_slots; ++i) {
    const Expr& e = slot_expr[i];
    P.slot_const[i] = ea_.constant(e);
    ea_.for_each(e, 0, NS, [&](uint32_t sidx) {
      if (sidx < n_comp_) {
        comp_t[sidx].push_back(i);
        P.sign_xor_terms++;
      } else {
        uint32_t t = sidx - n_comp_;
        if (cls[t] == 1) {
          m1_t[m1_index[t]].push_back(i);
          P.sign_xor_terms++;
        } else {
          throw Error(SYMFT_E_DEVICE, "internal: non-exogenous symbol in a slot");
        }
      }
    });
  }
  P.comp_off.assign(n_comp_ + 1, 0);
  for (uint32_t sidx = 0; sidx < n_comp_; ++sidx)
    P.comp_off[sidx + 1] = P.comp_off[sidx] + static_cast<uint32_t>(comp_t[sidx].size());
  P.comp_tgt.reserve(P.comp_off[n_comp_]);
  for (auto& v : comp_t) P.comp_tgt.insert(P.comp_tgt.end(), v.begin(), v.end());
  P.m1_off.assign(P.m1_t.size() + 1, 0);
  for (size_t j = 0; j < m1_t.size(); ++j) P.m1_off[j + 1] = P.m1_off[j] + static_cast<uint32_t>(m1_t[j].size());
  for (auto& v : m1_t) P.m1_tgt.insert(P.m1_tgt.end(), v.begin(), v.end());

  // dense instruction stream
  for (uint32_t g = 0; g < G; ++g) {
    const RawInstr& I = *dense_src[g];
    DenseInstr D{};
    D.kind = I.kind;
    D.k = I.k;
    D.a = I.a;
    D.b = I.b;
    D.h = I.h;
    D.mu = I.mu;
    D.eta = I.eta;
    D.c = std::cos(I.theta / 2.0);
    D.s = std::sin(I.theta / 2.0);
    D.sign_target = R + g;
    D.causal_off = static_cast<uint32_t>(P.dense_causal.size());
    const auto& cl = sign_causal[g];
    D.causal_n = static_cast<uint32_t>(cl.size());
    P.dense_causal.insert(P.dense_causal.end(), cl.begin(), cl.end());
    D.m3 = -1;
    D.t = I.t;
    D.rec = -1;
    if (I.kind == I_ACTIVE_DIAG_MEAS || I.kind == I_ACTIVE_PAIR_MEAS) D.m3 = m3_index[I.t];
    P.dense.push_back(D);
  }

  // noise channel tables
  P.ch_theta_last.assign(c_.n_channels, 0);
  P.ch_qtab.assign(c_.n_channels, 0);
  P.ch_ctab.assign(c_.n_channels, 0);
  P.ch_comp0 = chan_comp0_;
  P.ch_ncomp = chan_ncomp_;
  for (const Op& op : c_.ops) {
    if (op.kind != OP_NOISE) continue;
    // q table
    int qi = -1;
    for (size_t i = 0; i < P.qtabs.size(); ++i)
      if (P.qtabs[i].q == op.q) qi = static_cast<int>(i);
    if (qi < 0) {
      QTable qt;
      qt.q = op.q;
      double r = 1.0 - op.q, rp = r;
      for (int j = 0; j < kNoiseBlock; ++j) {
        double v = std::floor((1.0 - rp) * 4294967296.0);
        qt.theta[j] = v >= 4294967295.0 ? 0xFFFFFFFFu : static_cast<uint32_t>(v);
        rp = rp * r;
      }
      qi = static_cast<int>(P.qtabs.size());
      P.qtabs.push_back(qt);
      if (P.qtabs.size() > 65535) throw Error(SYMFT_E_CAPACITY, "too many distinct noise probabilities");
    }
    // cell table
    CellTable ct{};
    std::vector<int> masks;
    switch (op.chan) {
      case CH_X: case CH_Z: masks = {1}; break;
      case CH_Y: masks = {3}; break;
      case CH_XYZ: masks = {1, 3, 2}; break;
      case CH_D2:
        for (int k = 1; k < 16; ++k) {
          int pa = k >> 2, pb = k & 3;
          auto bits = [](int p) { return p == 1 ? 1 : (p == 2 ? 3 : (p == 3 ? 2 : 0)); };
          masks.push_back(bits(pa) | (bits(pb) << 2));
        }
        break;
    }
    ct.ncell = static_cast<uint32_t>(masks.size());
    for (size_t i = 0; i < masks.size(); ++i) ct.mask[i] = static_cast<uint8_t>(masks[i]);
    double total = 0.0;
    for (double w : op.weights) total = total + w;
    double run = 0.0;
    for (size_t i = 0; i + 1 < op.weights.size(); ++i) {
      run = run + op.weights[i];
      double v = std::floor(run / total * 4294967296.0);
      ct.phi[i] = v >= 4294967295.0 ? 0xFFFFFFFFu : static_cast<uint32_t>(v);
    }
    int ci = -1;
    for (size_t i = 0; i < P.ctabs.size(); ++i)
      if (std::memcmp(&P.ctabs[i], &ct, sizeof(CellTable)) == 0) ci = static_cast<int>(i);
    if (ci < 0) {
      ci = static_cast<int>(P.ctabs.size());
      P.ctabs.push_back(ct);
      if (P.ctabs.size() > 65535) throw Error(SYMFT_E_CAPACITY, "too many distinct noise channels");
    }
    P.ch_qtab[op.channel] = static_cast<uint16_t>(qi);
    P.ch_ctab[op.channel] = static_cast<uint16_t>(ci);
    // a channel whose components reach no target never needs drawing
    bool live = false;
    for (uint32_t s = chan_comp0_[op.channel]; s < chan_comp0_[op.channel] + chan_ncomp_[op.channel]; ++s)
      live |= P.comp_off[s + 1] > P.comp_off[s];
    P.ch_theta_last[op.channel] = live ? P.qtabs[qi].theta[kNoiseBlock - 1] : 0;
  }

  // targets of each (channel, cell): a fired cell applies all its components
  // at once, so the sampler flips the XOR of their target sets
  P.ch_cell0.assign(c_.n_channels, 0);
  P.cell_off.assign(1, 0);
  for (uint32_t ch = 0; ch < c_.n_channels; ++ch) {
    P.ch_cell0[ch] = static_cast<uint32_t>(P.cell_off.size() - 1);
    const CellTable& ct = P.ctabs[P.ch_ctab[ch]];
    for (uint32_t k = 0; k < ct.ncell; ++k) {
      std::vector<uint32_t> t;
      for (int bp = 0; bp < 4; ++bp) {
        if (!((ct.mask[k] >> bp) & 1)) continue;
        const uint32_t comp = chan_comp0_[ch] + bp;
        t.insert(t.end(), P.comp_tgt.begin() + P.comp_off[comp], P.comp_tgt.begin() + P.comp_off[comp + 1]);
      }
      std::sort(t.begin(), t.end());
      for (size_t i = 0; i < t.size();) {
        size_t j = i;
        while (j < t.size() && t[j] == t[i]) ++j;
        if ((j - i) & 1) P.cell_tgt.push_back(t[i]);
        i = j;
      }
      P.cell_off.push_back(static_cast<uint32_t>(P.cell_tgt.size()));
    }
  }

  // postselection event order (Sec. 6, detector postselection): which
  // detectors reject a shot, and where each sits among the records
  std::vector<uint8_t> post(c_.n_dets, 0);
  if (opt_.postselect == SYMFT_POSTSELECT_ALL) {
    std::fill(post.begin(), post.end(), 1);
  } else if (opt_.postselect == SYMFT_POSTSELECT_LISTED) {
    for (uint32_t i = 0; i < opt_.n_post_dets; ++i) post[opt_.post_dets[i]] = 1;
  }
  P.postselect = 0;
  for (uint8_t v : post) P.postselect |= v;
  for (const Op& op : c_.ops) {
    if (op.kind == OP_MEAS && op.rec >= 0) {
      P.post_events.push_back(op.rec);
    } else if (op.kind == OP_DET) {
      P.post_events.push_back(-1 - static_cast<int32_t>(2 * op.index + post[op.index]));
    }
  }
  // early exit: postselected detectors grouped by the number of active
  // measurements that precede them in circuit order.  Once the dense
  // executor has decided active measurement j, every record and detector up
  // to the detectors of group j + 1 is final, so a shot whose first fired
  // postselected detector lies there needs no further dense work.
  P.post_chk_off.assign(P.n_m3 + 2, 0);
  if (P.postselect && P.n_m3 > 0) {
    std::vector<std::vector<uint32_t>> grp(P.n_m3 + 1);
    uint32_t seen = 0;
    for (const Op& op : c_.ops) {
      if (op.kind == OP_MEAS && cls[op.t] == 3) ++seen;
      else if (op.kind == OP_DET && post[op.index]) grp[seen].push_back(op.index);
    }
    for (uint32_t q = 0; q <= P.n_m3; ++q) {
      P.post_chk.insert(P.post_chk.end(), grp[q].begin(), grp[q].end());
      P.post_chk_off[q + 1] = static_cast<uint32_t>(P.post_chk.size());
    }
  }
}

}  // namespace

HostPlan compile_plan(const Circuit& c, const symft_options& opt) {
  Compiler comp(c, opt);
  return comp.run();
}

}  // namespace symft
