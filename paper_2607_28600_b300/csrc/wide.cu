// Wide dense executor: the dense-state instructions of Sec. 4 for active
// widths whose vectors do not fit on chip (2^k amplitudes per shot above
// ~200 KB).  Work is instruction-major: a batch of shots keeps its vectors in
// HBM ([shot][2^k_max] amplitudes, two buffers), and the dense instructions
// run as grid-wide passes over all shots of the batch, so each pass streams
// whole vectors with full memory-level parallelism.
//
//   rotations    a run of consecutive rotations whose pair and new bits fit
//                a shared-memory tile is one fused pass (below); a lone
//                rotation is one pass in place (PromoteRot writes the upper
//                half, ActivePairRot updates disjoint pairs (x0, x0 ^ a))
//   measurements branch sums per shot (block partials added into FP64
//                accumulators), a per-shot decision (shared uniform rule,
//                record / causal bits, renormalisation, signs of the
//                following instructions), and compaction into the other
//                buffer
//
// A shot's signs lam(g) = exogenous bit ^ causal residual (Sec. 5) are
// evaluated per shot whenever its active outcomes change: at the start of the
// batch for the instructions up to the first measurement, and by each
// measurement's decision for those up to the next one.
#include <cuda_runtime.h>

#include <cstdint>

#include "device.cuh"

namespace symft {

namespace {

constexpr int kWideThreads = 256;
constexpr int kWideItems = 4;     // elements per thread per block-pass

template <typename Real>
struct Amp {
  Real re, im;
};

__device__ __forceinline__ uint32_t wide_insert_bit(uint32_t z, int h, uint32_t d) {
  const uint32_t low = z & ((1u << h) - 1u);
  return low | (d << h) | ((z >> h) << (h + 1));
}

// Element updates shared by every rotation pass (lone, fused in shared
// memory, fused in registers), so all give the same bits.  Pair rotation:
// v' = c v + s z w with w the partner element, s = -1 when `neg` (the
// partner's (-1)^{b.x}) and z = -i i^mu sg s, which is real for odd mu and
// imaginary for even mu, so z w takes two products; zr is z's non-zero part
// (k = s zr) and `odd` selects which part it is.
template <typename Real>
__device__ __forceinline__ Amp<Real> pair_update_k(Amp<Real> v, Amp<Real> w, Real c, Real k, bool odd) {
  const Real pr = odd ? w.re : -w.im;
  const Real pi = odd ? w.im : w.re;
  Amp<Real> o;
  o.re = fma(c, v.re, k * pr);
  o.im = fma(c, v.im, k * pi);
  return o;
}

// the same with mu's parity known at compile time (no selects)
template <bool ODD, typename Real>
__device__ __forceinline__ Amp<Real> pair_update_t(Amp<Real> v, Amp<Real> w, Real c, Real k) {
  Amp<Real> o;
  if constexpr (ODD) {
    o.re = fma(c, v.re, k * w.re);
    o.im = fma(c, v.im, k * w.im);
  } else {
    o.re = fma(c, v.re, k * -w.im);
    o.im = fma(c, v.im, k * w.re);
  }
  return o;
}

template <typename Real>
__device__ __forceinline__ Amp<Real> pair_update(Amp<Real> v, Amp<Real> w, Real c, Real zr, bool odd, bool neg) {
  return pair_update_k(v, w, c, neg ? -zr : zr, odd);
}

// the non-zero part of z = -i i^mu sg s (odd mu: real, even mu: imaginary)
template <typename Real>
__device__ __forceinline__ Real pair_z(int mu, Real sgs) {
  // i^mu times -i: mu = 0 -> -i, 1 -> 1, 2 -> i, 3 -> -1
  return (mu & 3) == 0 || (mu & 3) == 3 ? -sgs : sgs;
}

// Diagonal rotation: a' = (c - i f) a with f = +-mu s
template <typename Real>
__device__ __forceinline__ Amp<Real> diag_update(Amp<Real> a, Real c, Real f) {
  Amp<Real> r;
  r.re = fma(f, a.im, c * a.re);
  r.im = fma(-f, a.re, c * a.im);
  return r;
}

__device__ __forceinline__ uint64_t wide_meas_U(const PhiloxKeys& K, uint32_t t, uint64_t r) {
  const uint64_t w = r >> 6;
  const uint4 ob = philox(make_uint4(t, (uint32_t)(w >> 1), (uint32_t)(w >> 33), kTagMbit), K);
  const uint64_t word = (w & 1) ? ((uint64_t)ob.z | ((uint64_t)ob.w << 32)) : ((uint64_t)ob.x | ((uint64_t)ob.y << 32));
  const uint64_t bit = (word >> (r & 63)) & 1ull;
  const uint4 of = philox(make_uint4(t, (uint32_t)(r >> 1), (uint32_t)(r >> 33), kTagMfrac), K);
  const uint64_t fw = (r & 1) ? ((uint64_t)of.z | ((uint64_t)of.w << 32)) : ((uint64_t)of.x | ((uint64_t)of.y << 32));
  return (bit << 52) + (fw >> 12);
}

// signs of instructions g0, g0+1, ... up to and including the next active
// measurement, for shot b (whose active outcomes so far are in m3b)
__device__ void wide_signs_from(const WideArgs& A, uint32_t b, uint32_t g0) {
  const uint64_t r = A.r0 + b;
  const uint32_t m3w = (A.p.n_m3 + 31) / 32;
  const uint32_t* mb = A.m3b + (size_t)b * m3w;
  for (uint32_t g = g0; g < A.p.n_dense; ++g) {
    const DenseInstrDev I = A.p.dense[g];
    uint32_t lam = (uint32_t)((__ldg(A.signs + (uint64_t)I.sign_target_col * A.W + (r >> 6)) >> (r & 63)) & 1ull);
    for (uint32_t q = 0; q < I.causal_n; ++q) {
      const uint32_t j = __ldg(A.p.dense_causal + I.causal_off + q);
      lam ^= (mb[j >> 5] >> (j & 31)) & 1u;
    }
    A.lam[(size_t)g * A.nb + b] = (uint8_t)lam;
    if (I.kind == 5 || I.kind == 6) break;
  }
}

}  // namespace

template <typename Real>
__global__ void wide_init_kernel(WideArgs A) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= A.nb) return;
  Amp<Real>* v = reinterpret_cast<Amp<Real>*>(A.vec[A.cur]) + (size_t)b * A.stride;
  v[0].re = (Real)1;
  v[0].im = (Real)0;
  const uint32_t m3w = (A.p.n_m3 + 31) / 32;
  for (uint32_t i = 0; i < m3w; ++i) A.m3b[(size_t)b * m3w + i] = 0u;
  A.sums[2 * b] = 0.0;
  A.sums[2 * b + 1] = 0.0;
  wide_signs_from(A, b, 0);
  // early exit: a shot rejected before any active measurement is skipped
  A.alive[b] = (A.det_exo && A.p.post_grp0 == 0 &&
                group_rejects(A.p, A.det_exo, A.W, A.r0 + b, 0, A.m3b + (size_t)b * m3w)) ? 0 : 1;
}

// PromoteRot / ActiveDiagRot / ActivePairRot of instruction g on every shot:
// one flat index over (shot, element), element count 2^lg per shot
template <typename Real>
__global__ void __launch_bounds__(kWideThreads) wide_rot_kernel(WideArgs A, uint32_t g) {
  const DenseInstrDev I = A.p.dense[g];
  const uint32_t n = 1u << I.k;
  const int lg = I.kind == 2 ? I.k - 1 : I.k;          // pairs for ActivePairRot
  const uint64_t total = (uint64_t)A.nb << lg;
  const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
  const Real c = coef_c<Real>(I), s = coef_s<Real>(I);
  const uint8_t* lamg = A.lam + (size_t)g * A.nb;
  Amp<Real>* vbase = reinterpret_cast<Amp<Real>*>(A.vec[A.cur]);
  if (I.kind == 0) {                    // a'_x = c a_x, a'_{x+n} = -i sg s a_x
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += step) {
      const uint32_t b = (uint32_t)(i >> lg), x = (uint32_t)i & (n - 1);
      if (!A.alive[b]) continue;
      Amp<Real>* v = vbase + (size_t)b * A.stride;
      const Real sgs = lamg[b] ? -s : s;
      Amp<Real> a = v[x], hi;
      hi.re = sgs * a.im;
      hi.im = -sgs * a.re;
      v[x + n] = hi;
      a.re *= c;
      a.im *= c;
      v[x] = a;
    }
  } else if (I.kind == 1) {             // a_x *= c - i sg mu (-1)^{b.x} s
    const Real mus = I.mu == 0 ? s : -s;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += step) {
      const uint32_t b = (uint32_t)(i >> lg), x = (uint32_t)i & (n - 1);
      if (!A.alive[b]) continue;
      Amp<Real>* v = vbase + (size_t)b * A.stride;
      const Real f = (lamg[b] ? -mus : mus) * ((__popc(x & I.b) & 1) ? (Real)-1 : (Real)1);
      v[x] = diag_update(v[x], c, f);
    }
  } else {                              // pairs (x0, x0 ^ a), coefficient -i mu sg s (-1)^{b.x}
    const int pb = 31 - __clz(I.a);
    const bool odd = (I.mu & 1) != 0;
    const uint32_t half_mask = (n >> 1) - 1;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += step) {
      const uint32_t b = (uint32_t)(i >> lg), z = (uint32_t)i & half_mask;
      if (!A.alive[b]) continue;
      Amp<Real>* v = vbase + (size_t)b * A.stride;
      const Real zr = pair_z<Real>(I.mu, lamg[b] ? -s : s);
      const uint32_t x0 = wide_insert_bit(z, pb, 0u), x1 = x0 ^ I.a;
      const Amp<Real> v0 = v[x0], v1 = v[x1];
      v[x0] = pair_update(v0, v1, c, zr, odd, (__popc(x1 & I.b) & 1) != 0);
      v[x1] = pair_update(v1, v0, c, zr, odd, (__popc(x0 & I.b) & 1) != 0);
    }
  }
}

// conj(mu) of a pair measurement
template <typename Real>
__device__ __forceinline__ void wide_conj_mu(int mu, Real& mcr, Real& mci) {
  switch (mu & 3) {
    case 0: mcr = 1; mci = 0; break;
    case 1: mcr = 0; mci = -1; break;
    case 2: mcr = -1; mci = 0; break;
    default: mcr = 0; mci = 1; break;
  }
}

// outcome of measurement g for shot b from its branch sums: the shared
// uniform rule on p0 = S_{label 0} / (S0 + S1), records, renormalisation,
// and the signs of the following instructions; returns the kept label and
// the scale
template <typename Real>
__device__ void wide_decide_one(const WideArgs& A, uint32_t g, uint32_t b, double S0, double S1,
                                uint32_t& lab_out, double& scale_out) {
  const DenseInstrDev I = A.p.dense[g];
  const uint64_t r = A.r0 + b, rg = A.shot0 + b;
  const uint32_t lam = A.lam[(size_t)g * A.nb + b];
  const uint32_t l0 = I.kind == 5 ? (lam ^ (uint32_t)I.eta) : lam;
  const uint64_t U = wide_meas_U(A.keys, I.t, rg);
  double pd = (l0 ? S1 : S0) / (S0 + S1);
  // FP32 vectors: p0 rounded to FP32; p0 * 2^53 is exact in FP64 either way,
  // so the comparison below is the exact rule U < p0 * 2^53
  if (sizeof(Real) == 4) pd = (double)(float)pd;
  const uint32_t m = (double)U < pd * 9007199254740992.0 ? 0u : 1u;
  if (A.prob) A.prob[(uint64_t)I.m3 * A.shots + r] = pd;
  lab_out = l0 ^ m;
  scale_out = 1.0 / sqrt(lab_out ? S1 : S0);
  if (m) {
    const uint32_t m3w = (A.p.n_m3 + 31) / 32;
    A.m3b[(size_t)b * m3w + (I.m3 >> 5)] |= 1u << (I.m3 & 31);
    atomicOr(reinterpret_cast<unsigned long long*>(A.m3_out) + (uint64_t)I.m3 * A.W + (r >> 6),
             1ull << (r & 63));
  }
  wide_signs_from(A, b, g + 1);
  // early exit once a postselected detector that is now final fires
  if (A.det_exo && I.post_grp != kNoGroup) {
    const uint32_t m3w = (A.p.n_m3 + 31) / 32;
    if (group_rejects(A.p, A.det_exo, A.W, r, I.post_grp, A.m3b + (size_t)b * m3w)) A.alive[b] = 0;
  }
}

template <typename Real>
__global__ void wide_decide_kernel(WideArgs A, uint32_t g) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= A.nb || !A.alive[b]) return;
  uint32_t lab;
  double scale;
  wide_decide_one<Real>(A, g, b, A.sums[2 * b], A.sums[2 * b + 1], lab, scale);
  A.lab[b] = (uint8_t)lab;
  A.scale[b] = scale;
  A.scalef[b] = (float)scale;
  A.sums[2 * b] = 0.0;
  A.sums[2 * b + 1] = 0.0;
}

// compaction of shot b's measurement g: element z of the kept half
template <typename Real>
__device__ __forceinline__ Amp<Real> wide_kept(const Amp<Real>* v, const DenseInstrDev& I, uint32_t z, uint32_t lab,
                                               Real scale, Real mcr, Real mci) {
  const int h = I.h;
  Amp<Real> a;
  if (I.kind == 5) {
    const uint32_t u = wide_insert_bit(z, h, lab);
    a = v[u ^ ((uint32_t)(__popc(u & I.b & ~(1u << h)) & 1) << h)];
    a.re *= scale;
    a.im *= scale;
  } else {
    const Real inv_sqrt2 = (Real)0.70710678118654752440;
    const uint32_t u0 = wide_insert_bit(z, h, 0u);
    const Amp<Real> a0 = v[u0], a1 = v[u0 ^ I.a];
    Real sb = (__popc(I.b & u0) & 1) ? (Real)-1 : (Real)1;
    if (lab) sb = -sb;
    const Real tr = sb * (mcr * a1.re - mci * a1.im), ti = sb * (mcr * a1.im + mci * a1.re);
    a.re = (a0.re + tr) * inv_sqrt2 * scale;
    a.im = (a0.im + ti) * inv_sqrt2 * scale;
  }
  return a;
}

// branch sums of shot b's measurement g over elements e0, e0+step, ...:
// terms in the vector's precision, summed in runs of kWideRun terms in that
// precision and the runs in FP64 (B300's FP64 rate is a small fraction of its
// FP32 rate, so FP32 vectors keep FP64 work to one add per run)
constexpr uint32_t kWideRun = 16;

template <typename Real>
__device__ __forceinline__ void wide_partial_sums(const Amp<Real>* v, const DenseInstrDev& I, uint32_t e0,
                                                  uint32_t step, double& S0, double& S1) {
  const uint32_t n = 1u << I.k;
  if (I.kind == 5) {
    for (uint32_t x0 = e0; x0 < n; x0 += step * kWideRun) {
      Real r0 = 0, r1 = 0;
      for (uint32_t j = 0, x = x0; j < kWideRun && x < n; ++j, x += step) {
        const Amp<Real> a = v[x];
        const Real w = a.re * a.re + a.im * a.im;
        if (__popc(x & I.b) & 1) r1 += w; else r0 += w;
      }
      S0 += (double)r0;
      S1 += (double)r1;
    }
  } else {
    Real mcr, mci;
    wide_conj_mu<Real>(I.mu, mcr, mci);
    const Real inv_sqrt2 = (Real)0.70710678118654752440;
    const uint32_t half = n >> 1;
    for (uint32_t z0 = e0; z0 < half; z0 += step * kWideRun) {
      Real r0 = 0, r1 = 0;
      for (uint32_t j = 0, z = z0; j < kWideRun && z < half; ++j, z += step) {
        const uint32_t u0 = wide_insert_bit(z, I.h, 0u);
        const Amp<Real> a0 = v[u0], a1 = v[u0 ^ I.a];
        const Real sb = (__popc(I.b & u0) & 1) ? (Real)-1 : (Real)1;
        const Real tr = sb * (mcr * a1.re - mci * a1.im), ti = sb * (mcr * a1.im + mci * a1.re);
        const Real b0r = (a0.re + tr) * inv_sqrt2, b0i = (a0.im + ti) * inv_sqrt2;
        const Real b1r = (a0.re - tr) * inv_sqrt2, b1i = (a0.im - ti) * inv_sqrt2;
        r0 += b0r * b0r + b0i * b0i;
        r1 += b1r * b1r + b1i * b1i;
      }
      S0 += (double)r0;
      S1 += (double)r1;
    }
  }
}

// a whole measurement of a small vector (2^k <= kWideSmall): one warp per
// shot computes the sums, decides, and compacts into the other buffer
constexpr uint32_t kWideSmall = 4096;

template <typename Real>
__global__ void __launch_bounds__(kWideThreads) wide_meas_small_kernel(WideArgs A, uint32_t g) {
  const uint32_t b = blockIdx.x * (kWideThreads / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= A.nb || !A.alive[b]) return;        // whole warps leave together
  const DenseInstrDev I = A.p.dense[g];
  const Amp<Real>* v = reinterpret_cast<const Amp<Real>*>(A.vec[A.cur]) + (size_t)b * A.stride;
  Amp<Real>* o = reinterpret_cast<Amp<Real>*>(A.vec[A.cur ^ 1]) + (size_t)b * A.stride;
  double S0 = 0.0, S1 = 0.0;
  wide_partial_sums<Real>(v, I, (uint32_t)lane, 32u, S0, S1);
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    S0 += __shfl_xor_sync(0xffffffffu, S0, off);
    S1 += __shfl_xor_sync(0xffffffffu, S1, off);
  }
  uint32_t lab = 0;
  double scale = 0.0;
  if (lane == 0) wide_decide_one<Real>(A, g, b, S0, S1, lab, scale);
  lab = __shfl_sync(0xffffffffu, lab, 0);
  scale = __shfl_sync(0xffffffffu, scale, 0);
  Real mcr = 0, mci = 0;
  if (I.kind == 6) wide_conj_mu<Real>(I.mu, mcr, mci);
  const uint32_t half = 1u << (I.k - 1);
  for (uint32_t z = (uint32_t)lane; z < half; z += 32) o[z] = wide_kept<Real>(v, I, z, lab, (Real)scale, mcr, mci);
}

// branch sums S0 (label 0) and S1 of measurement g, FP64 accumulation: a 2D
// grid of (chunk, shot) blocks adding block partials into the shot's sums
template <typename Real>
__global__ void __launch_bounds__(kWideThreads) wide_sums_kernel(WideArgs A, uint32_t g) {
  __shared__ double red[2][kWideThreads / 32];
  const uint32_t b = blockIdx.y;
  if (!A.alive[b]) return;                     // the whole block leaves
  const DenseInstrDev I = A.p.dense[g];
  const Amp<Real>* v = reinterpret_cast<const Amp<Real>*>(A.vec[A.cur]) + (size_t)b * A.stride;
  double S0 = 0.0, S1 = 0.0;
  wide_partial_sums<Real>(v, I, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, S0, S1);
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    S0 += __shfl_xor_sync(0xffffffffu, S0, o);
    S1 += __shfl_xor_sync(0xffffffffu, S1, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][warp] = S0;
    red[1][warp] = S1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int w = 0; w < kWideThreads / 32; ++w) {
      t0 += red[0][w];
      t1 += red[1][w];
    }
    atomicAdd(A.sums + 2 * b, t0);
    atomicAdd(A.sums + 2 * b + 1, t1);
  }
}

// compaction of measurement g into the other buffer (2^(k-1) amplitudes per
// shot), one flat index over (shot, element)
template <typename Real>
__global__ void __launch_bounds__(kWideThreads) wide_compact_kernel(WideArgs A, uint32_t g) {
  const DenseInstrDev I = A.p.dense[g];
  const int lg = I.k - 1;
  const uint64_t total = (uint64_t)A.nb << lg;
  const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
  Real mcr = 0, mci = 0;
  if (I.kind == 6) wide_conj_mu<Real>(I.mu, mcr, mci);
  const Amp<Real>* vb = reinterpret_cast<const Amp<Real>*>(A.vec[A.cur]);
  Amp<Real>* ob = reinterpret_cast<Amp<Real>*>(A.vec[A.cur ^ 1]);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += step) {
    const uint32_t b = (uint32_t)(i >> lg), z = (uint32_t)i & ((1u << lg) - 1u);
    if (!A.alive[b]) continue;
    const Real sc = sizeof(Real) == 4 ? (Real)A.scalef[b] : (Real)A.scale[b];
    ob[(size_t)b * A.stride + z] = wide_kept<Real>(vb + (size_t)b * A.stride, I, z, A.lab[b], sc, mcr, mci);
  }
}

// ---------------------------------------------------------------------------
// Fused rotation windows.  A run of consecutive PromoteRot / ActiveDiagRot /
// ActivePairRot instructions whose pair bits (the bits of a), new bits (the
// coordinate a PromoteRot adds) and the five lowest bits together number at
// most T is applied in ONE pass over HBM: each CTA stages a tile of 2^T
// amplitudes -- the "inner" bits vary inside the tile, the other ("outer")
// bits are fixed per tile -- in shared memory, runs the whole window on it
// and writes it back.  The five lowest bits are always inner, so a tile is
// 2^(T-5) runs of 32 consecutive amplitudes (coalesced).  A diagonal phase
// needs no pairing, so only pair and new bits constrain a window.  In tile
// coordinates an instruction's masks are the inner parts of a and b gathered
// onto the tile's bit positions; the outer part of b adds a parity that is
// fixed per tile.
// ---------------------------------------------------------------------------
constexpr int kFuseMax = 48;        // instructions per window
// tile bits: 2^12 FP32 / 2^11 FP64 amplitudes = 32 KB of shared memory (larger
// tiles make the pass compute-bound before they save HBM traffic)
constexpr uint32_t kFuseBitsF32 = 12, kFuseBitsF64 = 11;
// the tile bits in use: the requested ones clamped to what the kernels take
// (a 2^T-amplitude tile, two of them in the bulk form, within 200 KB), else
// the default
template <typename Real>
inline uint32_t wide_tile_bits(uint32_t requested) {
  const uint32_t def = sizeof(Real) == 4 ? kFuseBitsF32 : kFuseBitsF64;
  const uint32_t hi = sizeof(Real) == 4 ? kWideTileBitsMaxF32 : kWideTileBitsMaxF64;
  if (requested == 0) return def;
  return requested < kWideTileBitsMin ? kWideTileBitsMin : (requested > hi ? hi : requested);
}

struct FuseInstr {
  uint32_t b_out;      // b & outer bits (parity fixed per tile)
  uint16_t a_loc;      // a gathered onto the tile bits (pair rotations)
  uint16_t b_loc;      // b & inner bits gathered onto the tile bits
  uint8_t kind;        // 0 PromoteRot, 1 ActiveDiagRot, 2 ActivePairRot
  uint8_t p_loc;       // tile bit of the new coordinate (PromoteRot) or of a's pivot (pair)
  uint16_t e_loc;      // tile bits of coordinates not yet promoted: elements with
                       // any of them set do not exist yet (zero) and are skipped
  uint8_t ra, rb;      // register phases: a (PromoteRot: the new bit) and b
                       // gathered onto the phase's register bits
};

// A phase of a window: rotations q0 .. q0 + n - 1 applied in registers on the
// register bits R (a mask of kRegBits tile bits >= 5), or (R == 0) one
// rotation applied on the tile in shared memory.
struct FusePhase {
  uint16_t q0, n, R, pad;
};

struct WideFuse {
  uint32_t g0, n;          // instructions g0 .. g0 + n - 1
  uint32_t inner;          // inner (tile) bits, |inner| = T
  uint32_t outer;          // outer bits: [0, k_start) without the inner bits
  uint32_t T, kstart, kend;
  uint32_t hi_shift;       // 5: inner bits 0..4 are the tile's low bits
  uint32_t n_ph;           // phases
  FuseInstr ins[kFuseMax];
  FusePhase ph[kFuseMax];
};

// register bits of a phase: 2^kRegBits amplitudes per thread (16 FP32 / 8 FP64)
template <typename Real>
struct RegBits {
  static constexpr int M = sizeof(Real) == 4 ? 4 : 3;
};
constexpr uint32_t reg_bits(bool fp64) { return fp64 ? 3u : 4u; }

// x with the bits of v placed at the set positions of mask, lowest first
__host__ __device__ __forceinline__ uint32_t deposit_bits(uint32_t v, uint32_t mask) {
  uint32_t x = 0;
  for (uint32_t m = mask; m; m &= m - 1) {
    if (v & 1u) x |= m & (~m + 1u);
    v >>= 1;
  }
  return x;
}

// One rotation of a fused window on the whole tile in shared memory: the
// tile of shot b whose outer bits are `off` (element i of the tile is
// amplitude off + the inner bits of i); elements of coordinates not yet
// promoted are skipped (they are zero).
template <typename Real>
__device__ __forceinline__ void apply_rot_smem(const WideArgs& A, const WideFuse& F, Amp<Real>* tile, uint32_t b,
                                               uint32_t off, uint32_t tid, uint32_t q) {
  const uint32_t n = 1u << F.T;
  const FuseInstr& L = F.ins[q];
  const uint32_t g = F.g0 + q;
  const DenseInstrDev& I = A.p.dense[g];
  const Real c = coef_c<Real>(I), s = coef_s<Real>(I);
  const Real sgs = A.lam[(size_t)g * A.nb + b] ? -s : s;
  const uint32_t po = __popc(L.b_out & off) & 1u;
  if (L.kind == 0) {                              // a'_x = c a_x, a'_{x+new} = -i sg s a_x
    const uint32_t pb = 1u << L.p_loc;
    for (uint32_t z = tid; z < (n >> 1); z += blockDim.x) {
      const uint32_t i0 = wide_insert_bit(z, L.p_loc, 0u);
      if (i0 & L.e_loc) continue;
      Amp<Real> a = tile[i0], hi;
      hi.re = sgs * a.im;
      hi.im = -sgs * a.re;
      a.re *= c;
      a.im *= c;
      tile[i0] = a;
      tile[i0 | pb] = hi;
    }
  } else if (L.kind == 1) {                       // a_x *= c - i sg mu (-1)^{b.x} s
    const Real mus = I.mu == 0 ? sgs : -sgs;
    for (uint32_t i = tid; i < n; i += blockDim.x) {
      if (i & L.e_loc) continue;
      const Real f = ((__popc(i & L.b_loc) ^ po) & 1u) ? -mus : mus;
      tile[i] = diag_update(tile[i], c, f);
    }
  } else {                                        // pairs (x0, x0 ^ a)
    const Real zr = pair_z<Real>(I.mu, sgs);
    const bool odd = (I.mu & 1) != 0;
    for (uint32_t z = tid; z < (n >> 1); z += blockDim.x) {
      const uint32_t i0 = wide_insert_bit(z, L.p_loc, 0u), i1 = i0 ^ L.a_loc;
      if (i0 & L.e_loc) continue;
      const Amp<Real> v0 = tile[i0], v1 = tile[i1];
      const bool n1 = ((__popc(i1 & L.b_loc) ^ po) & 1u) != 0u;
      const bool n0 = ((__popc(i0 & L.b_loc) ^ po) & 1u) != 0u;
      tile[i0] = pair_update(v0, v1, c, zr, odd, n1);
      tile[i1] = pair_update(v1, v0, c, zr, odd, n0);
    }
  }
}

// ---------------------------------------------------------------------------
// Register phases.  A warp holds 2^(5+M) amplitudes of the tile: lane l and
// register j hold element base | l | dep(j), where the lanes run over tile bits
// 0..4 (so every shared-memory access of the warp is 32 consecutive elements),
// dep(j) places the M bits of j on the phase's register bits R, and base sets
// the remaining (warp) bits.  A rotation whose pair bits above bit 4 lie in R
// pairs element x with x ^ a: register j ^ aR of lane l ^ aL, reached by a
// register copy and, for aL != 0, a shuffle.  Every element takes its new
// value from itself and its partner with the same formulas as the
// shared-memory form, so a phase of several rotations costs one load and one
// store of the tile.
// ---------------------------------------------------------------------------
template <typename Real>
__device__ __forceinline__ Amp<Real> shfl_amp(Amp<Real> v, uint32_t lanemask) {
  Amp<Real> w;
  w.re = __shfl_xor_sync(0xffffffffu, v.re, lanemask);
  w.im = __shfl_xor_sync(0xffffffffu, v.im, lanemask);
  return w;
}

// compile-time bit helpers of the register loops
__host__ __device__ constexpr int ctz_c(int x) { return x & 1 ? 0 : 1 + ctz_c(x >> 1); }
__host__ __device__ constexpr int msb_c(int x) { return x > 1 ? 1 + msb_c(x >> 1) : 0; }
__host__ __device__ constexpr int nth_bit_c(int mask, int n) { return n == 0 ? ctz_c(mask) : nth_bit_c(mask & (mask - 1), n - 1); }
__host__ __device__ constexpr int deposit_c(int v, int mask) {
  return mask == 0 ? 0 : ((v & 1) ? (mask & -mask) : 0) | deposit_c(v >> 1, mask & (mask - 1));
}

// k times the sign of chi (+-1): a multiplication in FP32; in FP64 (a slow
// pipe on B300) an XOR of the sign bit
__device__ __forceinline__ float mul_sign(float k, float chi) { return k * chi; }
__device__ __forceinline__ double mul_sign(double k, double chi) {
  return __longlong_as_double(__double_as_longlong(k) ^ (__double_as_longlong(chi) & (long long)0x8000000000000000ull));
}

// Pair rotation with register part AR of a and lane part aL.  The partner
// signs follow a character of the register bits: chi[k] = -1 when bit k of
// b's register part is set, so walking the register indices in Gray-code
// order gives every element's coefficient k = +-zr with one (exact)
// multiplication by +-1; k starts as element 0's, and chiAR relates element
// j1 = j0 ^ AR to j0.  Step T of the walk is a template argument, so every
// register index is a compile-time constant.
template <int AR, int M, int T, bool ODD, typename Real>
__device__ __forceinline__ void reg_pair_step(Amp<Real> (&v)[1 << M], uint32_t aL, Real c, Real k,
                                              const Real (&chi)[M], Real chiAR) {
  constexpr int NJ = 1 << M;
  if constexpr (AR == 0) {
    if constexpr (T < NJ) {
      if constexpr (T > 0) k = mul_sign(k, chi[ctz_c(T)]);
      constexpr int j = T ^ (T >> 1);
      const Amp<Real> w = shfl_amp(v[j], aL);
      v[j] = pair_update_t<ODD>(v[j], w, c, k);
      reg_pair_step<AR, M, T + 1, ODD, Real>(v, aL, c, k, chi, chiAR);
    }
  } else {
    if constexpr (T < NJ / 2) {
      constexpr int FM = (NJ - 1) & ~(1 << msb_c(AR));   // register bits other than a's pivot
      if constexpr (T > 0) k = mul_sign(k, chi[nth_bit_c(FM, ctz_c(T))]);
      constexpr int j0 = deposit_c(T ^ (T >> 1), FM);
      constexpr int j1 = j0 ^ AR;
      Amp<Real> w0 = v[j1], w1 = v[j0];
      if (aL) {
        w0 = shfl_amp(w0, aL);
        w1 = shfl_amp(w1, aL);
      }
      const Amp<Real> o0 = pair_update_t<ODD>(v[j0], w0, c, k);
      const Amp<Real> o1 = pair_update_t<ODD>(v[j1], w1, c, mul_sign(k, chiAR));
      v[j0] = o0;
      v[j1] = o1;
      reg_pair_step<AR, M, T + 1, ODD, Real>(v, aL, c, k, chi, chiAR);
    }
  }
}

// Diagonal rotation in registers: coefficient f of element 0, the others by
// the same Gray-code walk
template <int M, int T, typename Real>
__device__ __forceinline__ void reg_diag_step(Amp<Real> (&v)[1 << M], Real c, Real f, const Real (&chi)[M]) {
  if constexpr (T < (1 << M)) {
    if constexpr (T > 0) f = mul_sign(f, chi[ctz_c(T)]);
    constexpr int j = T ^ (T >> 1);
    v[j] = diag_update(v[j], c, f);
    reg_diag_step<M, T + 1, Real>(v, c, f, chi);
  }
}

// PromoteRot with the new coordinate on register bit PR
template <int PR, int M, typename Real>
__device__ __forceinline__ void reg_promote(Amp<Real> (&v)[1 << M], Real c, Real sgs) {
  constexpr int NJ = 1 << M;
#pragma unroll
  for (int j0 = 0; j0 < NJ; ++j0) {
    if ((j0 >> PR) & 1) continue;
    Amp<Real> a = v[j0], hi;
    hi.re = sgs * a.im;
    hi.im = -sgs * a.re;
    a.re *= c;
    a.im *= c;
    v[j0] = a;
    v[j0 | (1 << PR)] = hi;
  }
}

template <int M, typename Real>
__device__ __forceinline__ void reg_pair_dispatch(uint32_t ar, Amp<Real> (&v)[1 << M], uint32_t aL, Real c, Real k0,
                                                  const Real (&chi)[M], Real chiAR, bool odd) {
  // (ar, mu odd) -> one instantiation each
  switch (ar | (odd ? 16u : 0u)) {
#define SYMFT_PAIR_CASE(k)                                                                         \
  case k:                                                                                          \
    if constexpr (k < (1 << M)) reg_pair_step<k, M, 0, false, Real>(v, aL, c, k0, chi, chiAR);     \
    break;                                                                                         \
  case k + 16:                                                                                     \
    if constexpr (k < (1 << M)) reg_pair_step<k, M, 0, true, Real>(v, aL, c, k0, chi, chiAR);      \
    break;
    SYMFT_PAIR_CASE(0) SYMFT_PAIR_CASE(1) SYMFT_PAIR_CASE(2) SYMFT_PAIR_CASE(3)
    SYMFT_PAIR_CASE(4) SYMFT_PAIR_CASE(5) SYMFT_PAIR_CASE(6) SYMFT_PAIR_CASE(7)
    SYMFT_PAIR_CASE(8) SYMFT_PAIR_CASE(9) SYMFT_PAIR_CASE(10) SYMFT_PAIR_CASE(11)
    SYMFT_PAIR_CASE(12) SYMFT_PAIR_CASE(13) SYMFT_PAIR_CASE(14) SYMFT_PAIR_CASE(15)
#undef SYMFT_PAIR_CASE
    default: break;
  }
}

// One register phase of a window on the tile of shot b with outer bits `off`.
template <typename Real>
__device__ __forceinline__ void apply_phase_reg(const WideArgs& A, const WideFuse& F, Amp<Real>* tile, uint32_t b,
                                                uint32_t off, const FusePhase P) {
  constexpr int M = RegBits<Real>::M;
  constexpr int NJ = 1 << M;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const uint32_t Wb = ((1u << F.T) - 1u) & ~31u & ~(uint32_t)P.R;
  uint32_t rb[M];
  {
    uint32_t m = P.R;
#pragma unroll
    for (int k = 0; k < M; ++k) {
      rb[k] = m & (~m + 1u);
      m &= m - 1u;
    }
  }
  auto dep = [&](int j) {
    uint32_t x = 0;
#pragma unroll
    for (int k = 0; k < M; ++k)
      if ((j >> k) & 1) x |= rb[k];
    return x;
  };
  // elements with a warp bit of a coordinate not yet promoted are zero for
  // the whole phase (the phase promotes only register or lane bits)
  const uint32_t e_w = F.ins[P.q0].e_loc & Wb;
  const uint32_t nsub = 1u << (F.T - 5 - M);
  for (uint32_t sub = warp; sub < nsub; sub += nwarps) {
    const uint32_t base = deposit_bits(sub, Wb);
    if (base & e_w) continue;                       // uniform over the warp
    const uint32_t x0 = base | lane;
    Amp<Real> v[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) v[j] = tile[x0 | dep(j)];
    for (uint32_t q = P.q0; q < (uint32_t)P.q0 + P.n; ++q) {
      const FuseInstr& L = F.ins[q];
      const uint32_t g = F.g0 + q;
      const DenseInstrDev& I = A.p.dense[g];
      const Real c = coef_c<Real>(I), s = coef_s<Real>(I);
      const Real sgs = A.lam[(size_t)g * A.nb + b] ? -s : s;
      // parity of b over the outer and warp bits of the element
      const uint32_t pw = (__popc(L.b_out & off) ^ __popc(base & L.b_loc)) & 1u;
      const uint32_t bL = L.b_loc & 31u;
      Real chi[M];
#pragma unroll
      for (int k = 0; k < M; ++k) chi[k] = ((L.rb >> k) & 1u) ? (Real)-1 : (Real)1;
      if (L.kind == 0) {
        if (L.p_loc >= 5) {
          switch (L.ra) {
            case 1: reg_promote<0, M, Real>(v, c, sgs); break;
            case 2: reg_promote<1, M, Real>(v, c, sgs); break;
            case 4: reg_promote<2, M, Real>(v, c, sgs); break;
            default: if constexpr (M > 3) reg_promote<3, M, Real>(v, c, sgs); break;
          }
        } else {
          const uint32_t pb = 1u << L.p_loc;
          const bool upper = (lane & pb) != 0u;
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            const Amp<Real> w = shfl_amp(v[j], pb);
            Amp<Real> o;
            if (upper) {
              o.re = sgs * w.im;
              o.im = -sgs * w.re;
            } else {
              o.re = v[j].re * c;
              o.im = v[j].im * c;
            }
            v[j] = o;
          }
        }
      } else if (L.kind == 1) {
        const Real mus = I.mu == 0 ? sgs : -sgs;
        const uint32_t pt = (pw ^ __popc(lane & bL)) & 1u;
        reg_diag_step<M, 0, Real>(v, c, pt ? -mus : mus, chi);
      } else {
        const Real zr = pair_z<Real>(I.mu, sgs);
        const bool odd = (I.mu & 1) != 0;
        const uint32_t aL = L.a_loc & 31u;
        // sign of the partner x ^ a of element j: parity of (x ^ a) & b
        const uint32_t pt = (pw ^ __popc((lane ^ aL) & bL) ^ __popc((uint32_t)L.ra & L.rb)) & 1u;
        const Real chiAR = (__popc((uint32_t)L.ra & L.rb) & 1u) ? (Real)-1 : (Real)1;
        reg_pair_dispatch<M, Real>(L.ra, v, aL, c, pt ? -zr : zr, chi, chiAR, odd);
      }
    }
#pragma unroll
    for (int j = 0; j < NJ; ++j) tile[x0 | dep(j)] = v[j];
  }
}

// One fused window on a tile held in shared memory, phase by phase.  Ends with
// the CTA synchronised.
template <typename Real>
__device__ __forceinline__ void apply_window(const WideArgs& A, const WideFuse& F, Amp<Real>* tile, uint32_t b,
                                             uint32_t off, uint32_t tid) {
  for (uint32_t ph = 0; ph < F.n_ph; ++ph) {
    const FusePhase P = F.ph[ph];
    if (P.R == 0) apply_rot_smem<Real>(A, F, tile, b, off, tid, P.q0);
    else apply_phase_reg<Real>(A, F, tile, b, off, P);
    __syncthreads();
  }
}

template <typename Real>
__global__ void __launch_bounds__(kWideThreads) wide_fused_rot_kernel(WideArgs A, WideFuse F) {
  extern __shared__ __align__(16) unsigned char fsm[];
  Amp<Real>* tile = reinterpret_cast<Amp<Real>*>(fsm);
  uint32_t* hi_tab = reinterpret_cast<uint32_t*>(fsm + ((size_t)sizeof(Amp<Real>) << F.T));
  const uint32_t n = 1u << F.T;
  const uint32_t tid = threadIdx.x;
  // global offsets of the tile's high inner index (i >> 5)
  const uint32_t inner_hi = F.inner & ~31u;
  for (uint32_t j = tid; j < (n >> 5); j += blockDim.x) hi_tab[j] = deposit_bits(j, inner_hi);
  __syncthreads();
  const uint32_t tiles = 1u << (F.kend - F.T);
  const uint64_t total = (uint64_t)A.nb * tiles;
  const uint32_t kst_mask = F.kstart >= 32 ? ~0u : (1u << F.kstart) - 1u;
  for (uint64_t t = blockIdx.x; t < total; t += gridDim.x) {
    const uint32_t b = (uint32_t)(t / tiles), o = (uint32_t)(t - (uint64_t)b * tiles);
    if (!A.alive[b]) continue;                       // uniform over the CTA
    const uint32_t off = deposit_bits(o, F.outer);
    Amp<Real>* v = reinterpret_cast<Amp<Real>*>(A.vec[A.cur]) + (size_t)b * A.stride;
    for (uint32_t i = tid; i < n; i += blockDim.x) {
      const uint32_t x = off + hi_tab[i >> 5] + (i & 31u);
      Amp<Real> a;
      a.re = (Real)0;
      a.im = (Real)0;
      if ((x & ~kst_mask) == 0u) a = v[x];           // coordinates not yet promoted are 0
      tile[i] = a;
    }
    __syncthreads();
    apply_window<Real>(A, F, tile, b, off, tid);
    for (uint32_t i = tid; i < n; i += blockDim.x) v[off + hi_tab[i >> 5] + (i & 31u)] = tile[i];
    __syncthreads();
  }
}

// ---- bulk asynchronous copies (Blackwell copy engine) ------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* m, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(m)), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for phase `parity` of m to complete, for at most ~2^32 SM clocks
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* m, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(m, parity))
    if (clock64() - t0 > (1ll << 32)) return false;
  return true;
}
// global -> shared, completing `bytes` on the mbarrier (both addresses 16-byte
// aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* m) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(m))
               : "memory");
}
// shared -> global in this thread's current bulk group
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// this thread's bulk stores have read their shared-memory sources
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// this thread's bulk stores are complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// order this thread's generic shared-memory accesses before later async-proxy ones
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// The fused window with tiles streamed by the copy engine: a tile is n / 32
// chunks of 32 consecutive amplitudes (the inner bits include bits 0..4, so a
// chunk is 256 B in FP32, 512 B in FP64, aligned to its size).  Each CTA walks
// its tiles with two buffers: while it applies the window to one tile, the
// next tile's chunks arrive by bulk copies that complete on that buffer's
// mbarrier, and the previous tile leaves by bulk stores.  A buffer is refilled
// only after the stores issued from it have read it.  Chunks of coordinates not
// yet promoted (a whole chunk, since F.kstart >= 5) are zero-filled instead of
// copied.  A bounded wait that runs out sets *A.status and ends the CTA.
template <typename Real>
__global__ void __launch_bounds__(kWideThreads, 3) wide_fused_bulk_kernel(WideArgs A, WideFuse F) {
  extern __shared__ __align__(128) unsigned char bsm[];
  const uint32_t n = 1u << F.T;
  const size_t tb = sizeof(Amp<Real>) << F.T;       // tile bytes
  auto buf = [&](int s) { return reinterpret_cast<Amp<Real>*>(bsm + (size_t)s * tb); };
  uint32_t* hi_tab = reinterpret_cast<uint32_t*>(bsm + 2 * tb);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(bsm + 2 * tb + ((size_t)4 << (F.T - 5)));
  const uint32_t tid = threadIdx.x;
  const uint32_t nch = n >> 5;                       // chunks per tile
  constexpr uint32_t cb = 32u * sizeof(Amp<Real>);  // chunk bytes
  const uint32_t inner_hi = F.inner & ~31u;
  const uint32_t kst_mask = F.kstart >= 32 ? ~0u : (1u << F.kstart) - 1u;
  for (uint32_t j = tid; j < nch; j += blockDim.x) hi_tab[j] = deposit_bits(j, inner_hi);
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
  }
  fence_async_shared();
  __syncthreads();
  // chunks of a tile that exist (their inner high bits below k_start): the
  // same for every tile whose outer bits are below k_start, none otherwise
  uint32_t nlive = 0;
  for (uint32_t j = 0; j < nch; ++j) nlive += (hi_tab[j] & ~kst_mask) == 0u;
  const uint32_t tiles = 1u << (F.kend - F.T);
  const uint64_t total = (uint64_t)A.nb * tiles;
  auto next_live = [&](uint64_t t) {
    while (t < total && !A.alive[t / tiles]) t += gridDim.x;
    return t;
  };
  auto issue_load = [&](uint64_t t, int s) {
    const uint32_t b = (uint32_t)(t / tiles), o = (uint32_t)(t - (uint64_t)b * tiles);
    const uint32_t off = deposit_bits(o, F.outer);
    const Amp<Real>* v = reinterpret_cast<const Amp<Real>*>(A.vec[A.cur]) + (size_t)b * A.stride;
    const bool outer_live = (off & ~kst_mask) == 0u;
    if (tid == 0) mbar_arrive_expect(&mbar[s], outer_live ? nlive * cb : 0u);
    __syncthreads();                                 // the expected bytes precede every copy
    for (uint32_t j = tid; j < nch; j += blockDim.x)
      if (outer_live && (hi_tab[j] & ~kst_mask) == 0u) bulk_load(buf(s) + 32 * j, v + off + hi_tab[j], cb, &mbar[s]);
    // chunks that are not copied are zero, written element-strided across the
    // CTA (consecutive threads, consecutive banks)
    if (!outer_live || nlive < nch) {
      Amp<Real> z;
      z.re = (Real)0;
      z.im = (Real)0;
      for (uint32_t i = tid; i < n; i += blockDim.x)
        if (!outer_live || (hi_tab[i >> 5] & ~kst_mask) != 0u) buf(s)[i] = z;
    }
  };
  uint32_t phase = 0u;                               // bit s: parity of buffer s's next phase
  uint64_t t = next_live(blockIdx.x);
  if (t < total) issue_load(t, 0);
  bool failed = false, pending = false;
  int ps = 0;
  for (uint32_t it = 0; t < total; ++it) {
    const int s = it & 1;
    const uint64_t tn = next_live(t + gridDim.x);
    if (tn < total) {
      bulk_wait_read();                              // the stores from buffer s ^ 1 have read it
      __syncthreads();
      issue_load(tn, s ^ 1);
      pending = true;
      ps = s ^ 1;
    } else {
      pending = false;
    }
    const bool ok = mbar_wait_bounded(&mbar[s], (phase >> s) & 1u);
    phase ^= 1u << s;
    if (__syncthreads_or(!ok)) {                     // also orders the zero fills
      failed = true;
      break;
    }
    const uint32_t b = (uint32_t)(t / tiles), o = (uint32_t)(t - (uint64_t)b * tiles);
    const uint32_t off = deposit_bits(o, F.outer);
    apply_window<Real>(A, F, buf(s), b, off, tid);
    fence_async_shared();
    __syncthreads();
    Amp<Real>* v = reinterpret_cast<Amp<Real>*>(A.vec[A.cur]) + (size_t)b * A.stride;
    for (uint32_t j = tid; j < nch; j += blockDim.x) bulk_store(v + off + hi_tab[j], buf(s) + 32 * j, cb);
    bulk_commit();
    t = tn;
  }
  if (failed) {
    if (tid == 0 && A.status) atomicExch(A.status, 3);
    if (pending) (void)mbar_wait_bounded(&mbar[ps], (phase >> ps) & 1u);
  }
  bulk_wait_all();
}

// bit positions of mask, gathered: the index of each set bit of x & mask
static uint32_t gather_bits(uint32_t x, uint32_t mask) {
  uint32_t r = 0, k = 0;
  for (uint32_t m = mask; m; m &= m - 1, ++k)
    if (x & m & (~m + 1u)) r |= 1u << k;
  return r;
}

// Greedy window from instruction g0 (a rotation): consecutive rotations while
// the inner bits fit in T.  Returns the number of instructions taken.
static uint32_t build_window(const DenseInstrDev* d, uint32_t G, uint32_t g0, uint32_t T, WideFuse* F,
                             uint32_t M) {
  const uint32_t kstart = (uint32_t)d[g0].k;
  uint32_t inner = 0u;
  for (uint32_t j = 0; j < 5; ++j) inner |= 1u << j;
  uint32_t g = g0, kend = kstart;
  while (g < G && d[g].kind <= 2 && g - g0 < (uint32_t)kFuseMax) {
    uint32_t need = 0u;
    if (d[g].kind == 0) need = 1u << d[g].k;
    else if (d[g].kind == 2) need = d[g].a;
    const uint32_t nx = inner | need;
    if ((uint32_t)__builtin_popcount(nx) > T) break;
    inner = nx;
    if (d[g].kind == 0) kend = (uint32_t)d[g].k + 1;
    ++g;
  }
  const uint32_t n = g - g0;
  // the tile: at most T bits of [0, kend); pad with the lowest free bits
  const uint32_t Te = kend < T ? kend : T;
  const uint32_t kmask = kend >= 32 ? ~0u : (1u << kend) - 1u;
  inner &= kmask;
  for (uint32_t j = 0; j < kend && (uint32_t)__builtin_popcount(inner) < Te; ++j) inner |= 1u << j;
  F->g0 = g0;
  F->n = n;
  F->inner = inner;
  F->T = (uint32_t)__builtin_popcount(inner);
  F->kstart = kstart;
  F->kend = kend;
  F->outer = (kstart >= 32 ? ~0u : (1u << kstart) - 1u) & ~inner;
  F->hi_shift = 5;
  for (uint32_t q = 0; q < n; ++q) {
    const DenseInstrDev& I = d[g0 + q];
    FuseInstr& L = F->ins[q];
    L.kind = (uint8_t)I.kind;
    L.b_out = I.b & F->outer;
    L.b_loc = (uint16_t)gather_bits(I.b, inner);
    L.a_loc = (uint16_t)gather_bits(I.a, inner);
    L.p_loc = 0;
    if (I.kind == 0) L.p_loc = (uint8_t)__builtin_popcount(inner & ((1u << I.k) - 1u));
    else if (I.kind == 2) L.p_loc = (uint8_t)(31 - __builtin_clz((uint32_t)L.a_loc));
    L.e_loc = (uint16_t)gather_bits(~((1u << I.k) - 1u), inner);
    L.ra = L.rb = 0;
  }
  // phases: consecutive rotations whose tile bits above bit 4 (pair bits, new
  // bit) fit in M register bits; a rotation that needs more is a phase of its
  // own in shared memory.  Tiles too small for a warp's 2^(5+M) elements use
  // shared memory throughout.
  F->n_ph = 0;
  const uint32_t tmask = (1u << F->T) - 1u;
  auto high_need = [&](const FuseInstr& L) -> uint32_t {
    if (L.kind == 0) return L.p_loc >= 5 ? (1u << L.p_loc) : 0u;
    if (L.kind == 2) return L.a_loc & ~31u;
    return 0u;
  };
  auto close = [&](uint32_t q0, uint32_t cnt, uint32_t R) {
    // pad R to M bits with the lowest free tile bits above bit 4
    for (uint32_t j = 5; j < F->T && (uint32_t)__builtin_popcount(R) < M; ++j)
      if (!((R >> j) & 1u)) R |= 1u << j;
    for (uint32_t q = q0; q < q0 + cnt; ++q) {
      FuseInstr& L = F->ins[q];
      L.ra = (uint8_t)gather_bits(L.kind == 0 ? high_need(L) : L.a_loc, R);
      L.rb = (uint8_t)gather_bits(L.b_loc, R);
    }
    F->ph[F->n_ph++] = FusePhase{(uint16_t)q0, (uint16_t)cnt, (uint16_t)R, 0};
  };
  if (F->T < 5 + M) {
    for (uint32_t q = 0; q < n; ++q) F->ph[F->n_ph++] = FusePhase{(uint16_t)q, 1, 0, 0};
    return n;
  }
  uint32_t q0 = 0, R = 0;
  for (uint32_t q = 0; q < n; ++q) {
    const uint32_t need = high_need(F->ins[q]) & tmask;
    if ((uint32_t)__builtin_popcount(R | need) <= M) {
      R |= need;
      continue;
    }
    if (q > q0) close(q0, q - q0, R);
    if ((uint32_t)__builtin_popcount(need) > M) {
      F->ph[F->n_ph++] = FusePhase{(uint16_t)q, 1, 0, 0};
      q0 = q + 1;
      R = 0;
    } else {
      q0 = q;
      R = need;
    }
  }
  if (n > q0) close(q0, n - q0, R);
  return n;
}

// ---------------------------------------------------------------------------
// host: one batch of shots through the whole dense instruction stream
// ---------------------------------------------------------------------------
// blocks of a flat pass over `total` elements: enough to fill the GPU
static unsigned wide_flat_blocks(uint64_t total, int sm_count) {
  const uint64_t want = (total + (uint64_t)kWideThreads * kWideItems - 1) / ((uint64_t)kWideThreads * kWideItems);
  const uint64_t cap = (uint64_t)sm_count * 32;
  uint64_t x = want < cap ? want : cap;
  return (unsigned)(x < 1 ? 1 : x);
}

// chunks per shot of a 2D (chunk, shot) pass over `elems` elements per shot
static unsigned wide_chunks(uint64_t elems, int sm_count, uint32_t nb) {
  const uint64_t want = (elems + (uint64_t)kWideThreads * kWideItems - 1) / ((uint64_t)kWideThreads * kWideItems);
  const uint64_t fill = ((uint64_t)sm_count * 16 + nb - 1) / nb;
  uint64_t x = want < fill ? want : fill;
  if (x < 1) x = 1;
  if (x > 65535) x = 65535;
  return (unsigned)x;
}

template <typename Real>
static cudaError_t wide_batch_t(WideArgs A, const DenseInstrDev* host_dense, int sm_count, cudaStream_t st,
                                int* launches, uint32_t tile_bits) {
  const unsigned nb_blocks = (A.nb + 127) / 128;
  wide_init_kernel<Real><<<nb_blocks, 128, 0, st>>>(A);
  ++*launches;
  const uint32_t T = wide_tile_bits<Real>(tile_bits);
  for (uint32_t g = 0; g < A.p.n_dense; ++g) {
    const DenseInstrDev& I = host_dense[g];
    const uint64_t n = 1ull << I.k;
    if (I.kind <= 2) {
      WideFuse F;
      const uint32_t nw = build_window(host_dense, A.p.n_dense, g, T, &F, RegBits<Real>::M);
      if (nw >= 2 && F.kend >= 5) {
        // one pass over HBM for the whole window
        const uint64_t tiles = (uint64_t)A.nb << (F.kend - F.T);
        static bool attr_set = false;
        static int bulk_per_sm[32] = {};   // resident CTAs per SM by tile bits (at the full tile)
        const size_t smem_bulk = 2 * (sizeof(Amp<Real>) << F.T) + ((size_t)4 << (F.T - 5)) + 16;
        if (!attr_set) {
          cudaError_t e = cudaFuncSetAttribute((const void*)wide_fused_rot_kernel<Real>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
          if (e == cudaSuccess)
            e = cudaFuncSetAttribute((const void*)wide_fused_bulk_kernel<Real>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
          if (e != cudaSuccess) return e;
          attr_set = true;
        }
        if (bulk_per_sm[T] == 0) {
          const size_t smem_max = 2 * (sizeof(Amp<Real>) << T) + ((size_t)4 << (T - 5)) + 16;
          cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bulk_per_sm[T], wide_fused_bulk_kernel<Real>,
                                                                        kWideThreads, smem_max);
          if (e != cudaSuccess) return e;
          if (bulk_per_sm[T] == 0) bulk_per_sm[T] = -1;   // does not fit: thread loads and stores
        }
        if (F.kstart >= 5 && bulk_per_sm[T] > 0) {
          // tiles streamed by bulk copies; one resident wave of CTAs walks them
          const uint64_t cap = (uint64_t)sm_count * bulk_per_sm[T];
          const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
          wide_fused_bulk_kernel<Real><<<grid, kWideThreads, smem_bulk, st>>>(A, F);
        } else {
          const size_t smem = (sizeof(Amp<Real>) << F.T) + ((size_t)4 << (F.T - 5));
          const uint64_t cap = (uint64_t)sm_count * 8;
          const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
          wide_fused_rot_kernel<Real><<<grid, kWideThreads, smem, st>>>(A, F);
        }
        ++*launches;
        g += nw - 1;
      } else {
        const uint64_t per_shot = I.kind == 2 ? n / 2 : n;
        wide_rot_kernel<Real><<<wide_flat_blocks(per_shot * A.nb, sm_count), kWideThreads, 0, st>>>(A, g);
        ++*launches;
      }
    } else if (n <= kWideSmall) {
      wide_meas_small_kernel<Real><<<(A.nb + kWideThreads / 32 - 1) / (kWideThreads / 32), kWideThreads, 0, st>>>(A, g);
      ++*launches;
      A.cur ^= 1;
    } else {
      const uint64_t elems = I.kind == 5 ? n : n / 2;
      wide_sums_kernel<Real><<<dim3(wide_chunks(elems, sm_count, A.nb), A.nb), kWideThreads, 0, st>>>(A, g);
      wide_decide_kernel<Real><<<nb_blocks, 128, 0, st>>>(A, g);
      wide_compact_kernel<Real><<<wide_flat_blocks((n / 2) * A.nb, sm_count), kWideThreads, 0, st>>>(A, g);
      *launches += 3;
      A.cur ^= 1;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Amplitudes one shot moves through HBM in the passes wide_batch_t issues
// (every shot running to the end): a fused window reads the 2^k_start
// existing amplitudes and writes 2^k_end; a lone PromoteRot reads 2^k and
// writes 2^(k+1), a lone diagonal or pair rotation reads and writes 2^k; a
// measurement reads 2^k for its sums, reads up to 2^k for the compaction and
// writes 2^(k-1).
uint32_t wide_tile_bits_in_use(bool fp64, uint32_t tile_bits) {
  return fp64 ? wide_tile_bits<double>(tile_bits) : wide_tile_bits<float>(tile_bits);
}

uint64_t wide_amp_traffic(const DenseInstrDev* d, uint32_t G, bool fp64, uint32_t tile_bits) {
  const uint32_t T = fp64 ? wide_tile_bits<double>(tile_bits) : wide_tile_bits<float>(tile_bits);
  uint64_t amps = 0;
  for (uint32_t g = 0; g < G; ++g) {
    const uint64_t n = 1ull << d[g].k;
    if (d[g].kind <= 2) {
      WideFuse F;
      const uint32_t nw = build_window(d, G, g, T, &F, reg_bits(fp64));
      if (nw >= 2 && F.kend >= 5) {
        amps += (1ull << F.kstart) + (1ull << F.kend);
        g += nw - 1;
      } else {
        amps += d[g].kind == 0 ? 3 * n : 2 * n;
      }
    } else {
      amps += n + n + n / 2;
    }
  }
  return amps;
}

cudaError_t launch_wide_batch(const WideArgs& a, const DenseInstrDev* host_dense, bool fp64, int sm_count,
                              cudaStream_t st, int* launches, uint32_t tile_bits) {
  return fp64 ? wide_batch_t<double>(a, host_dense, sm_count, st, launches, tile_bits)
              : wide_batch_t<float>(a, host_dense, sm_count, st, launches, tile_bits);
}

}  // namespace symft
