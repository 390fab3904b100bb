// Dense-state, plain-form, finalize and tally kernels (Sec. 5, single-shot
// algorithm, run for many shots at once).
//
//  dense_reg_kernel  k_max <= 5: 32 / 2^k_max shots per warp (twice that in
//                    FP32), lane x of a shot's segment holds amplitude x
//  dense_kernel      one shot per warp (two on 16-lane groups up to k_max 8),
//                    active vector in shared memory
//  dense_pc_kernel   one shot per warp on its product-component workspace
//  dense_cta_kernel  one CTA per shot, vector in shared memory
//                    -- all of them run PromoteRot, ActiveDiagRot, ActivePairRot,
//                    ActiveDiagMeas and ActivePairMeas (Sec. 4) on the shot's
//                    active vector, completing each sign with the causal
//                    residual of the active outcomes sampled earlier in the shot
//  plain_kernel      one CTA per shot with unpacked per-shot noise and signs
//                    (the comparison form)
//  finalize_kernel   one thread per 64-shot word: folds the active outcomes into
//                    records / detectors / observables, applies postselection
//  count_kernel      kept / discarded / observable tallies
#include <cuda_runtime.h>

#include <cstdint>

#include "device.cuh"

namespace symft {

const void* sign_kernel_fn();

// ---------------------------------------------------------------------------
// Dense executor: a warp (or a group of its lanes) per shot, active vector in
// shared or global memory.
// ---------------------------------------------------------------------------
template <typename Real>
struct Cplx {
  Real re, im;
};



__device__ __forceinline__ uint32_t insert_bit(uint32_t z, int h, uint32_t d) {
  uint32_t low = z & ((1u << h) - 1u);
  return low | (d << h) | ((z >> h) << (h + 1));
}

__device__ __forceinline__ double meas_uniform(uint64_t seed, uint32_t t, uint64_t r) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  uint64_t w = r >> 6;
  uint4 ob = philox(make_uint4(t, (uint32_t)(w >> 1), (uint32_t)(w >> 33), kTagMbit), k0, k1);
  uint64_t word = (w & 1) ? ((uint64_t)ob.z | ((uint64_t)ob.w << 32)) : ((uint64_t)ob.x | ((uint64_t)ob.y << 32));
  uint64_t bit = (word >> (r & 63)) & 1ull;
  uint4 of = philox(make_uint4(t, (uint32_t)(r >> 1), (uint32_t)(r >> 33), kTagMfrac), k0, k1);
  uint64_t fw = (r & 1) ? ((uint64_t)of.z | ((uint64_t)of.w << 32)) : ((uint64_t)of.x | ((uint64_t)of.y << 32));
  uint64_t f = fw >> 12;
  return (double)((bit << 52) + f) * 0x1p-53;
}

template <typename Real>
__device__ __forceinline__ double norm2(Cplx<Real> v) {
  return (double)v.re * (double)v.re + (double)v.im * (double)v.im;
}

// U = u * 2^53 of the shared measurement rule: an integer below 2^53
__device__ __forceinline__ uint64_t meas_U(const PhiloxKeys& K, uint32_t t, uint64_t r) {
  const uint64_t w = r >> 6;
  const uint4 ob = philox(make_uint4(t, (uint32_t)(w >> 1), (uint32_t)(w >> 33), kTagMbit), K);
  const uint64_t word = (w & 1) ? ((uint64_t)ob.z | ((uint64_t)ob.w << 32)) : ((uint64_t)ob.x | ((uint64_t)ob.y << 32));
  const uint64_t bit = (word >> (r & 63)) & 1ull;
  const uint4 of = philox(make_uint4(t, (uint32_t)(r >> 1), (uint32_t)(r >> 33), kTagMfrac), K);
  const uint64_t fw = (r & 1) ? ((uint64_t)of.z | ((uint64_t)of.w << 32)) : ((uint64_t)of.x | ((uint64_t)of.y << 32));
  return (bit << 52) + (fw >> 12);
}

// The uniforms of a shot's active measurements, one chunk at a time: the
// shot's lanes (a segment of 2^lw lanes from lane `base`; the whole warp when
// lw = 5) hold U of active measurements (c << lw) + l for the current chunk c,
// lane l holding one; a measurement reads its value by a shuffle and moves to
// the next chunk when it leaves this one.
struct ShotUniforms {
  uint64_t uc = 0;
  uint32_t chunk = 0xFFFFFFFFu;
  __device__ __forceinline__ uint64_t get(const DenseArgs& A, uint32_t j, uint64_t rg, int l, uint32_t lw = 5,
                                          int base = 0) {
    if ((j >> lw) != chunk) {
      chunk = j >> lw;
      const uint32_t jj = (chunk << lw) + (uint32_t)l;
      uc = jj < A.p.n_m3 ? meas_U(A.keys, __ldg(A.p.m3_t + jj), rg) : 0ull;
    }
    return __shfl_sync(0xffffffffu, uc, base + (int)(j & ((1u << lw) - 1u)));
  }
};

// recorded bit: 0 iff u < p0, i.e. U < p0 * 2^53 (both sides exact in FP64)
__device__ __forceinline__ uint32_t decide64(uint64_t U, double p0) {
  return (double)U < p0 * 9007199254740992.0 ? 0u : 1u;
}

// the same rule for an FP32 p0, in integers: U < p0 * 2^53 <=> U < ceil(p0 * 2^53)
__device__ __forceinline__ uint32_t decide32(uint64_t U, float p0) {
  if (!(p0 > 0.0f)) return 1u;
  if (p0 >= 1.0f) return 0u;
  const uint32_t bits = __float_as_uint(p0);
  const int e = (int)((bits >> 23) & 0xFFu);
  uint64_t mant;
  int shift;                                   // p0 * 2^53 = mant * 2^shift
  if (e == 0) {
    mant = bits & 0x7FFFFFu;
    shift = -149 + 53;
  } else {
    mant = (bits & 0x7FFFFFu) | 0x800000u;
    shift = e - 127 - 23 + 53;                 // <= 29 since p0 < 1
  }
  uint64_t T;
  if (shift >= 0) T = mant << shift;
  else if (-shift >= 40) T = 1;                // 0 < p0 * 2^53 < 1
  else T = (mant + ((1ull << -shift) - 1)) >> -shift;
  return U < T ? 0u : 1u;
}

// the sums over a group of kGW lanes (a whole warp for 32, else the aligned
// half or quarter that holds this lane)
template <uint32_t kGW, typename Acc>
__device__ __forceinline__ void group_sum2(Acc& a, Acc& b) {
#pragma unroll
  for (int o = (int)kGW / 2; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
}

template <typename Acc>
__device__ __forceinline__ void warp_sum2(Acc& a, Acc& b) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
}

// Branch sums of an active measurement over this thread's share of the vector:
// diagonal -> S_y over parity(b.x) = y; pair -> S_y = sum_z |beta_z(y)|^2.
template <typename Real, typename Acc>
__device__ __forceinline__ void branch_sums(const Cplx<Real>* vec, const DenseInstrDev& I, uint32_t n,
                                            uint32_t start, uint32_t stride, Real mcr, Real mci,
                                            Acc& S0, Acc& S1) {
  // terms in the vector's precision, summed in runs of 16 in that precision
  // and the runs in Acc (one Acc add per run keeps FP64 work off the
  // per-element path of FP32 vectors)
  constexpr uint32_t kRun = 16;
  const Real inv_sqrt2 = (Real)0.70710678118654752440;
  if (I.kind == 5) {
    for (uint32_t x0 = start; x0 < n; x0 += stride * kRun) {
      Real r0 = 0, r1 = 0;
      for (uint32_t j = 0, x = x0; j < kRun && x < n; ++j, x += stride) {
        const Cplx<Real> a = vec[x];
        const Real v = a.re * a.re + a.im * a.im;
        if (__popc(x & I.b) & 1) r1 += v; else r0 += v;
      }
      S0 += (Acc)r0;
      S1 += (Acc)r1;
    }
  } else {
    const uint32_t half = n >> 1;
    for (uint32_t z0 = start; z0 < half; z0 += stride * kRun) {
      Real r0 = 0, r1 = 0;
      for (uint32_t j = 0, z = z0; j < kRun && z < half; ++j, z += stride) {
        const uint32_t u0 = insert_bit(z, I.h, 0u);
        const Cplx<Real> a0 = vec[u0], a1 = vec[u0 ^ I.a];
        const Real sb = (__popc(I.b & u0) & 1) ? (Real)-1 : (Real)1;
        const Real tr = sb * (mcr * a1.re - mci * a1.im), ti = sb * (mcr * a1.im + mci * a1.re);
        const Real b0r = (a0.re + tr) * inv_sqrt2, b0i = (a0.im + ti) * inv_sqrt2;
        const Real b1r = (a0.re - tr) * inv_sqrt2, b1i = (a0.im - ti) * inv_sqrt2;
        r0 += b0r * b0r + b0i * b0i;
        r1 += b1r * b1r + b1i * b1i;
      }
      S0 += (Acc)r0;
      S1 += (Acc)r1;
    }
  }
}

// Per-element arithmetic of the dense instructions, shared by the
// per-element and the batched loops below.
// PromoteRot: a'_x = c a_x, a'_{x+n} = -i sg s a_x
template <typename Real>
__device__ __forceinline__ void promote_elem(Cplx<Real>* vec, uint32_t x, uint32_t n, Cplx<Real> v, Real sg,
                                             Real s, Real c) {
  Cplx<Real> hi;
  hi.re = sg * s * v.im;
  hi.im = -sg * s * v.re;
  vec[x + n] = hi;
  v.re *= c;
  v.im *= c;
  vec[x] = v;
}
// ActiveDiagRot: a_x *= c - i f, f = sg mu s (-1)^{b.x}
template <typename Real>
__device__ __forceinline__ void diag_elem(Cplx<Real>* vec, uint32_t x, Cplx<Real> v, Real sgmus, uint32_t b, Real c) {
  const Real f = sgmus * ((__popc(x & b) & 1) ? (Real)-1 : (Real)1);
  Cplx<Real> o;
  o.re = c * v.re + f * v.im;
  o.im = c * v.im - f * v.re;
  vec[x] = o;
}
// ActivePairRot on the pair (x0, x1 = x0 ^ a): coefficient (cr + i ci) on
// the partner, with its sign (-1)^{b.partner}
// (pab = parity of a.b: parity(b.x1) = parity(b.x0) xor pab)
template <typename Real>
__device__ __forceinline__ void pair_elem(Cplx<Real>* vec, uint32_t x0, uint32_t x1, Cplx<Real> v0, Cplx<Real> v1,
                                          uint32_t b, uint32_t pab, Real c, Real cr, Real ci) {
  const uint32_t p0 = __popc(x0 & b) & 1;
  const Real s1 = (p0 ^ pab) ? (Real)-1 : (Real)1;              // applied to a_{x1} in a'_{x0}
  const Real s0 = p0 ? (Real)-1 : (Real)1;
  Cplx<Real> o0, o1;
  o0.re = c * v0.re + s1 * (cr * v1.re - ci * v1.im);
  o0.im = c * v0.im + s1 * (cr * v1.im + ci * v1.re);
  o1.re = c * v1.re + s0 * (cr * v0.re - ci * v0.im);
  o1.im = c * v1.im + s0 * (cr * v0.im + ci * v0.re);
  vec[x0] = o0;
  vec[x1] = o1;
}
// kept amplitude z of an active measurement with label lab, scaled
template <typename Real>
__device__ __forceinline__ Cplx<Real> kept_elem(const Cplx<Real>* vec, const DenseInstrDev& I, uint32_t z,
                                                uint32_t lab, Real mcr, Real mci, Real scale) {
  const Real inv_sqrt2 = (Real)0.70710678118654752440;
  const int h = I.h;
  Cplx<Real> val;
  if (I.kind == 5) {
    const uint32_t u = insert_bit(z, h, lab);
    // x(b,u): bit h = u_h xor parity of b over the other bits
    const uint32_t x = u ^ ((uint32_t)(__popc(u & I.b & ~(1u << h)) & 1) << h);
    val = vec[x];
  } else {
    const uint32_t u0 = insert_bit(z, h, 0u);
    const Cplx<Real> a0 = vec[u0], a1 = vec[u0 ^ I.a];
    Real sb = (__popc(I.b & u0) & 1) ? (Real)-1 : (Real)1;
    if (lab) sb = -sb;
    const Real tr = sb * (mcr * a1.re - mci * a1.im), ti = sb * (mcr * a1.im + mci * a1.re);
    val.re = (a0.re + tr) * inv_sqrt2;
    val.im = (a0.im + ti) * inv_sqrt2;
  }
  val.re *= scale;
  val.im *= scale;
  return val;
}

// One dense instruction (Sec. 4: PromoteRot, ActiveDiagRot, ActivePairRot,
// ActiveDiagMeas, ActivePairMeas) on a vector of n = 2^k amplitudes held by
// a group of kGW lanes (the whole warp, or the half that starts at lane
// gbase; `lane` is the lane's index in its group), in shared or global
// memory, with the instruction's sign lam; the masks a, b and the pivot h of
// I are those of the vector's own bits.  A measurement writes the kept half
// to out: in place (out == vec) when h is the highest bit of a (pair) or any
// bit of b (diagonal), else to a disjoint region.  A group whose shot is not
// live computes along but decides nothing and writes no outcome.
//
// kBatch > 1: an instruction over at least kGW kBatch elements (amplitudes,
// pairs or kept amplitudes) runs in steps of kBatch elements per lane whose
// loads are all issued before the step's stores, so their shared-memory
// latencies overlap; the elements of a step are disjoint, and a
// measurement's in-place compaction reads every source of a step before any
// of its writes (a source is never below its destination).  Batching costs
// registers, so only executors whose occupancy is set by shared memory take it.
template <typename Real, uint32_t kBatch, uint32_t kGW = 32>
__device__ __forceinline__ void warp_instr(const DenseArgs& A, Cplx<Real>* vec, Cplx<Real>* out, uint32_t n,
                                           const DenseInstrDev& I, uint32_t lam, uint64_t r, uint64_t rg, uint64_t w,
                                           uint64_t bitmask, uint32_t* m3bits, ShotUniforms& su, int lane,
                                           int gbase = 0, bool live = true) {
  constexpr uint32_t kLgGW = kGW == 32 ? 5 : (kGW == 16 ? 4 : 3);
  const Real sg = lam ? (Real)-1 : (Real)1;
  const Real c = coef_c<Real>(I), s = coef_s<Real>(I);

  switch (I.kind) {
    case 0: {  // PromoteRot: a'_{x} = c a_x, a'_{x+2^k} = -i sg s a_x
      if (kBatch > 1 && n >= kGW * kBatch) {
        for (uint32_t x0 = lane; x0 < n; x0 += kGW * kBatch) {
          Cplx<Real> v[kBatch];
#pragma unroll
          for (uint32_t j = 0; j < kBatch; ++j) v[j] = vec[x0 + kGW * j];
#pragma unroll
          for (uint32_t j = 0; j < kBatch; ++j) promote_elem(vec, x0 + kGW * j, n, v[j], sg, s, c);
        }
      } else {
        for (uint32_t x = lane; x < n; x += kGW) promote_elem(vec, x, n, vec[x], sg, s, c);
      }
      break;
    }
    case 1: {  // ActiveDiagRot: a_x *= c - i sg mu (-1)^{b.x} s
      const Real mu = I.mu == 0 ? (Real)1 : (Real)-1;
      const Real sgmus = sg * mu * s;
      if (kBatch > 1 && n >= kGW * kBatch) {
        for (uint32_t x0 = lane; x0 < n; x0 += kGW * kBatch) {
          Cplx<Real> v[kBatch];
#pragma unroll
          for (uint32_t j = 0; j < kBatch; ++j) v[j] = vec[x0 + kGW * j];
#pragma unroll
          for (uint32_t j = 0; j < kBatch; ++j) diag_elem(vec, x0 + kGW * j, v[j], sgmus, I.b, c);
        }
      } else {
        for (uint32_t x = lane; x < n; x += kGW) diag_elem(vec, x, vec[x], sgmus, I.b, c);
      }
      break;
    }
    case 2: {  // ActivePairRot on pairs (x0, x0 ^ a)
      const int p = 31 - __clz(I.a);
      // coefficient -i mu sg s (-1)^{b.x} for mu = i^mu
      Real cr, ci;  // -i * i^mu
      switch (I.mu & 3) {
        case 0: cr = 0; ci = -1; break;
        case 1: cr = 1; ci = 0; break;
        case 2: cr = 0; ci = 1; break;
        default: cr = -1; ci = 0; break;
      }
      cr *= sg * s;
      ci *= sg * s;
      const uint32_t nh = n >> 1;
      const uint32_t pab = __popc(I.a & I.b) & 1;
      if (kBatch > 1 && nh >= kGW * kBatch) {
        for (uint32_t z0 = lane; z0 < nh; z0 += kGW * kBatch) {
          Cplx<Real> v0[kBatch], v1[kBatch];
#pragma unroll
          for (uint32_t j = 0; j < kBatch; ++j) {
            const uint32_t x0 = insert_bit(z0 + kGW * j, p, 0u);
            v0[j] = vec[x0];
            v1[j] = vec[x0 ^ I.a];
          }
#pragma unroll
          for (uint32_t j = 0; j < kBatch; ++j) {
            const uint32_t x0 = insert_bit(z0 + kGW * j, p, 0u);
            pair_elem(vec, x0, x0 ^ I.a, v0[j], v1[j], I.b, pab, c, cr, ci);
          }
        }
      } else {
        for (uint32_t z = lane; z < nh; z += kGW) {
          const uint32_t x0 = insert_bit(z, p, 0u), x1 = x0 ^ I.a;
          pair_elem(vec, x0, x1, vec[x0], vec[x1], I.b, pab, c, cr, ci);
        }
      }
      break;
    }
    case 5:
    case 6: {  // active measurements
      Real mcr = 0, mci = 0;       // conj(mu)
      if (I.kind == 6) {
        switch (I.mu & 3) {
          case 0: mcr = 1; mci = 0; break;
          case 1: mcr = 0; mci = -1; break;
          case 2: mcr = -1; mci = 0; break;
          default: mcr = 0; mci = 1; break;
        }
      }
      // label for m = 0: diag -> parity lam^eta ; pair -> y = lam
      const uint32_t l0 = I.kind == 5 ? (lam ^ (uint32_t)I.eta) : lam;
      uint32_t m = 0;
      Real scale;
      if (sizeof(Real) == 8 || n >= (1u << 14)) {      // FP64 sums
        double S0 = 0.0, S1 = 0.0;
        branch_sums<Real, double>(vec, I, n, lane, kGW, mcr, mci, S0, S1);
        group_sum2<kGW>(S0, S1);
        const uint64_t U = su.get(A, (uint32_t)I.m3, rg, lane, kLgGW, gbase);
        if (lane == 0 && live) {
          const double p0 = (l0 ? S1 : S0) / (S0 + S1);
          m = decide64(U, p0);
          if (A.prob) A.prob[(uint64_t)I.m3 * A.shots + r] = p0;
        }
        m = __shfl_sync(0xffffffffu, m, gbase);
        scale = (Real)(1.0 / sqrt((l0 ^ m) ? S1 : S0));
      } else {                                         // FP32 sums below 2^14 terms
        float S0 = 0.0f, S1 = 0.0f;
        branch_sums<Real, float>(vec, I, n, lane, kGW, mcr, mci, S0, S1);
        group_sum2<kGW>(S0, S1);
        const uint64_t U = su.get(A, (uint32_t)I.m3, rg, lane, kLgGW, gbase);
        // the renormalisation scale 1 / sqrt(S_m) in FP32 on one lane: every
        // later branch probability is self-normalised, so the scale only
        // sets the vector's overall norm (an FP64 scale measured 2.4-3x
        // slower on B300, whose FP64 pipe is a small fraction of FP32's)
        float sc = 0.0f;
        if (lane == 0 && live) {
          const float p0 = (l0 ? S1 : S0) / (S0 + S1);
          m = decide32(U, p0);
          if (A.prob) A.prob[(uint64_t)I.m3 * A.shots + r] = (double)p0;
          sc = rsqrtf((l0 ^ m) ? S1 : S0);
        }
        m = __shfl_sync(0xffffffffu, m, gbase);
        scale = (Real)__shfl_sync(0xffffffffu, sc, gbase);
      }
      const uint32_t lab = l0 ^ m;
      // compaction in increasing z order (in place, sources are never below z)
      const uint32_t half = n >> 1;
      if (kBatch > 1 && half >= kGW * kBatch) {
        for (uint32_t z0 = lane; z0 < half; z0 += kGW * kBatch) {
          Cplx<Real> val[kBatch];
#pragma unroll
          for (uint32_t j = 0; j < kBatch; ++j) val[j] = kept_elem(vec, I, z0 + kGW * j, lab, mcr, mci, scale);
          __syncwarp();
#pragma unroll
          for (uint32_t j = 0; j < kBatch; ++j) out[z0 + kGW * j] = val[j];
          __syncwarp();
        }
      } else {
        for (uint32_t z0 = 0; z0 < half; z0 += kGW) {
          const uint32_t z = z0 + lane;
          Cplx<Real> val;
          val.re = 0;
          val.im = 0;
          if (z < half) val = kept_elem(vec, I, z, lab, mcr, mci, scale);
          __syncwarp();
          if (z < half) out[z] = val;
          __syncwarp();
        }
      }
      if (m) {
        if (lane == 0) {
          m3bits[I.m3 >> 5] |= 1u << (I.m3 & 31);
          atomicOr(reinterpret_cast<unsigned long long*>(A.m3_out) + (uint64_t)I.m3 * A.W + w,
                   (unsigned long long)bitmask);
        }
      }
      break;
    }
    default:
      if (lane == 0 && A.status) atomicExch(A.status, 1);
      break;
  }
}

template <typename Real, uint32_t kGroups>
__global__ void __launch_bounds__(256) dense_kernel(DenseArgs A) {
  // kGroups shots per warp, each on a group of kGW lanes with its own vector:
  // every instruction is decoded once for all of them
  constexpr uint32_t kGW = 32 / kGroups;
  extern __shared__ unsigned char dsm[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const uint32_t gid = (uint32_t)lane / kGW;             // this lane's shot in the warp
  const int gl = lane & (int)(kGW - 1);                  // its lane in the shot's group
  const int gbase = (int)(gid * kGW);
  const uint32_t vwpb = (uint32_t)wpb * kGroups;         // shots per CTA
  const uint32_t vw = (uint32_t)wib * kGroups + gid;     // this shot's slot in the CTA
  const uint32_t S = 1u << A.kmax;
  const uint32_t m3w = (A.p.n_m3 + 31) / 32;
  const uint32_t G = A.p.n_dense;
  const uint32_t bkw = m3w + (G + 31) / 32;     // per-shot words: m3 bits, then sign bits
  // the instruction stream, staged in shared memory when it is small enough
  const size_t stb = stage_bytes((size_t)G * sizeof(DenseInstrDev));
  const DenseInstrDev* ins = A.p.dense;
  if (stb) {
    for (uint32_t i = threadIdx.x; i < G * (sizeof(DenseInstrDev) / 4); i += blockDim.x)
      reinterpret_cast<uint32_t*>(dsm)[i] = reinterpret_cast<const uint32_t*>(A.p.dense)[i];
    ins = reinterpret_cast<const DenseInstrDev*>(dsm);
  }
  uint32_t* m3bits = reinterpret_cast<uint32_t*>(dsm + stb) + (size_t)vw * bkw;
  uint32_t* sgn = m3bits + m3w;
  Cplx<Real>* vec;
  const uint64_t slot_global = (uint64_t)blockIdx.x * vwpb + vw;
  if (A.use_smem) {
    size_t off = stb + (((size_t)vwpb * bkw * 4 + 15) & ~(size_t)15);
    vec = reinterpret_cast<Cplx<Real>*>(dsm + off) + (size_t)vw * S;
  } else {
    vec = reinterpret_cast<Cplx<Real>*>(A.gvec) + slot_global * A.gvec_stride;
  }
  __syncthreads();

  for (uint64_t r0 = (uint64_t)blockIdx.x * vwpb + (uint64_t)wib * kGroups; r0 < A.shots;
       r0 += (uint64_t)gridDim.x * vwpb) {
    const uint64_t r = r0 + gid;         // request-local shot of this group
    const bool inreq = r < A.shots;
    const uint64_t rg = A.shot0 + r;     // absolute shot index
    const uint64_t w = r >> 6;
    const uint64_t bitmask = 1ull << (r & 63);
    for (uint32_t i = gl; i < m3w; i += kGW) m3bits[i] = 0u;
    // the shot's exogenous sign bits, kGW instructions per ballot, fetched
    // together before the instruction loop
    for (uint32_t base = 0; base < G; base += kGW) {
      const uint32_t g = base + gl;
      bool bit = false;
      if (inreq && g < G) bit = (__ldg(A.signs + (uint64_t)ins[g].sign_target_col * A.W + w) & bitmask) != 0;
      const uint32_t bal = __ballot_sync(0xffffffffu, bit);
      if (gl == 0) {
        if (kGW == 32) {
          sgn[base >> 5] = bal;
        } else {
          const uint32_t part = (bal >> gbase) & ((1u << kGW) - 1u);
          if ((base & 31) == 0) sgn[base >> 5] = part;
          else sgn[base >> 5] |= part << (base & 31);
        }
      }
    }
    ShotUniforms su;
    if (gl == 0) {
      vec[0].re = (Real)1;
      vec[0].im = (Real)0;
    }
    __syncwarp();
    // a shot rejected before any active measurement needs no dense work; a
    // warp runs while any of its shots is live, the others stepping masked
    bool live = inreq && !(A.det_exo && A.p.post_grp0 == 0 && group_rejects(A.p, A.det_exo, A.W, r, 0, m3bits));
    uint32_t livem = __ballot_sync(0xffffffffu, live);
    __syncwarp();
    if (livem == 0) continue;
    uint32_t k = 0;
    for (uint32_t g = 0; g < G; ++g) {
      const DenseInstrDev I = ins[g];
      // sign: exogenous bit xor causal residual over m3 bits of this shot
      uint32_t lam = (sgn[g >> 5] >> (g & 31)) & 1u;
      for (uint32_t q = 0; q < I.causal_n; ++q) {
        const uint32_t j = __ldg(A.p.dense_causal + I.causal_off + q);
        lam ^= (m3bits[j >> 5] >> (j & 31)) & 1u;
      }
      const uint32_t n = 1u << k;
      warp_instr<Real, 1, kGW>(A, vec, vec, n, I, lam, r, rg, w, bitmask, m3bits, su, gl, gbase, live);
      if (I.kind == 0) ++k;
      else if (I.kind == 5 || I.kind == 6) --k;
      __syncwarp();
      if (A.det_exo && I.post_grp != kNoGroup) {           // early exit once rejected
        if (live) live = !group_rejects(A.p, A.det_exo, A.W, r, I.post_grp, m3bits);
        livem = __ballot_sync(0xffffffffu, live);
        __syncwarp();
        if (livem == 0) break;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Product-component executor (Sec. 6, adaptive product-component
// representation): one warp per shot runs the plan's component program on a
// workspace of pc_capacity amplitudes (shared memory, or a per-warp global
// slot): INIT opens a one-coordinate component with the PromoteRot's factor
// (c, -i sg s); MERGE writes the Kronecker product C[xA + 2^kA xB] =
// A[xA] B[xB] into a fresh region; APPLY runs a dense instruction on one
// component with local masks.  Signs, outcomes and early exit as in the
// monolithic warp executor.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(256) dense_pc_kernel(DenseArgs A) {
  // warp_instr's batch: a shot's steps are a chain of dependent
  // shared-memory or L2 round trips, so 4 FP32 elements per lane and step
  // (measured fastest: 8 needs 127 registers, which halves the resident
  // warps); FP64 measured no faster batched
  constexpr uint32_t kPcBatch = sizeof(Real) == 4 ? 4 : 1;
  extern __shared__ unsigned char dsm[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const uint32_t m3w = (A.p.n_m3 + 31) / 32;
  const uint32_t G = A.p.n_dense;
  const uint32_t bkw = m3w + (G + 31) / 32;
  // the instruction stream and the component program, staged in shared
  // memory when they are small enough
  const size_t ib = (size_t)G * sizeof(DenseInstrDev);
  const size_t stb = stage_bytes(ib + (size_t)A.p.n_pc * sizeof(PCOp));
  const DenseInstrDev* ins = A.p.dense;
  const PCOp* prog = A.p.pc;
  if (stb) {
    for (uint32_t i = threadIdx.x; i < G * (sizeof(DenseInstrDev) / 4); i += blockDim.x)
      reinterpret_cast<uint32_t*>(dsm)[i] = reinterpret_cast<const uint32_t*>(A.p.dense)[i];
    for (uint32_t i = threadIdx.x; i < A.p.n_pc * (sizeof(PCOp) / 4); i += blockDim.x)
      reinterpret_cast<uint32_t*>(dsm + ib)[i] = reinterpret_cast<const uint32_t*>(A.p.pc)[i];
    ins = reinterpret_cast<const DenseInstrDev*>(dsm);
    prog = reinterpret_cast<const PCOp*>(dsm + ib);
  }
  uint32_t* m3bits = reinterpret_cast<uint32_t*>(dsm + stb) + (size_t)wib * bkw;
  uint32_t* sgn = m3bits + m3w;
  const uint64_t warp_global = (uint64_t)blockIdx.x * wpb + wib;
  Cplx<Real>* ws;
  if (A.use_smem) {
    const size_t off = stb + (((size_t)wpb * bkw * 4 + 15) & ~(size_t)15);
    ws = reinterpret_cast<Cplx<Real>*>(dsm + off) + (size_t)wib * A.p.pc_capacity;
  } else {
    ws = reinterpret_cast<Cplx<Real>*>(A.gvec) + warp_global * A.gvec_stride;
  }
  __syncthreads();
  for (uint64_t r = warp_global; r < A.shots; r += (uint64_t)gridDim.x * wpb) {
    const uint64_t rg = A.shot0 + r;
    const uint64_t w = r >> 6;
    const uint64_t bitmask = 1ull << (r & 63);
    for (uint32_t i = lane; i < m3w; i += 32) m3bits[i] = 0u;
    for (uint32_t base = 0; base < G; base += 32) {
      const uint32_t g = base + lane;
      bool bit = false;
      if (g < G) bit = (__ldg(A.signs + (uint64_t)ins[g].sign_target_col * A.W + w) & bitmask) != 0;
      const uint32_t bal = __ballot_sync(0xffffffffu, bit);
      if (lane == 0) sgn[base >> 5] = bal;
    }
    ShotUniforms su;
    __syncwarp();
    const bool dead0 = A.det_exo && A.p.post_grp0 == 0 && group_rejects(A.p, A.det_exo, A.W, r, 0, m3bits);
    __syncwarp();
    if (dead0) continue;
    for (uint32_t q = 0; q < A.p.n_pc; ++q) {
      const PCOp O = prog[q];
      if (O.op == PC_MERGE) {
        const uint32_t na = 1u << O.kA, nc = 1u << (O.kA + O.kB);
        const Cplx<Real>* pa = ws + O.offA;
        const Cplx<Real>* pb = ws + O.offB;
        Cplx<Real>* pc = ws + O.off;
        auto kron = [&](uint32_t x, const Cplx<Real>& u, const Cplx<Real>& v) {
          Cplx<Real> t;
          t.re = u.re * v.re - u.im * v.im;
          t.im = u.re * v.im + u.im * v.re;
          pc[x] = t;
        };
        if (kPcBatch > 1 && nc >= 32 * kPcBatch) {     // fresh region: disjoint from both factors
          for (uint32_t x0 = lane; x0 < nc; x0 += 32 * kPcBatch) {
            Cplx<Real> u[kPcBatch], v[kPcBatch];
#pragma unroll
            for (uint32_t j = 0; j < kPcBatch; ++j) {
              u[j] = pa[(x0 + 32 * j) & (na - 1)];
              v[j] = pb[(x0 + 32 * j) >> O.kA];
            }
#pragma unroll
            for (uint32_t j = 0; j < kPcBatch; ++j) kron(x0 + 32 * j, u[j], v[j]);
          }
        } else {
          for (uint32_t x = lane; x < nc; x += 32) kron(x, pa[x & (na - 1)], pb[x >> O.kA]);
        }
        __syncwarp();
        continue;
      }
      DenseInstrDev I = ins[O.g];
      uint32_t lam = (sgn[O.g >> 5] >> (O.g & 31)) & 1u;
      for (uint32_t c = 0; c < I.causal_n; ++c) {
        const uint32_t j = __ldg(A.p.dense_causal + I.causal_off + c);
        lam ^= (m3bits[j >> 5] >> (j & 31)) & 1u;
      }
      Cplx<Real>* vec = ws + O.off;
      if (O.op == PC_INIT) {
        if (lane == 0) {
          vec[0].re = (Real)1;
          vec[0].im = (Real)0;
        }
        __syncwarp();
        warp_instr<Real, kPcBatch>(A, vec, vec, 1u, I, lam, r, rg, w, bitmask, m3bits, su, lane);
        __syncwarp();
        continue;
      }
      I.a = O.a;
      I.b = O.b;
      I.h = O.h;
      warp_instr<Real, kPcBatch>(A, vec, ws + O.out, 1u << O.k, I, lam, r, rg, w, bitmask, m3bits, su, lane);
      __syncwarp();
      if (A.det_exo && I.post_grp != kNoGroup) {           // early exit once rejected
        const bool dead = group_rejects(A.p, A.det_exo, A.W, r, I.post_grp, m3bits);
        __syncwarp();
        if (dead) break;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Register-resident dense executor for k_max <= 5: a warp holds 32 / 2^k_max
// shots, one per segment of 2^k_max lanes; lane x of a segment holds its
// shot's amplitude alpha_x (zero beyond 2^k), and PromoteRot, pair partners,
// compaction sources and branch sums are shuffles inside the segment.  The
// instruction stream sits in shared memory and is decoded once for all the
// warp's shots; each shot's exogenous sign bits come in one coalesced pass
// (the warp's shots share one 32-shot half-word of every sign column).
// ---------------------------------------------------------------------------
constexpr int kRegWarps = 8;

template <typename Real>
__device__ __forceinline__ Real shfl_r(Real v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}

// Shots per warp of the register executor: 32 / 2^k_max segments, times the
// register sets a lane carries (kRegSetsF32 in FP32: every instruction is
// decoded once for twice the shots, and a lane has independent work per set;
// one in FP64, whose pipe bounds it either way).
constexpr uint32_t kRegSetsF32 = 2;

template <typename Real, uint32_t kLw, uint32_t kSets>
__global__ void __launch_bounds__(kRegWarps * 32) dense_reg_kernel(DenseArgs A) {
  extern __shared__ __align__(16) unsigned char rsm[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const uint32_t G = A.p.n_dense;
  const uint32_t m3w = (A.p.n_m3 + 31) / 32;
  constexpr uint32_t lw = kLw;                       // log2 lanes per shot (= k_max)
  constexpr uint32_t Wd = 1u << lw;
  constexpr uint32_t S = 32u >> lw;                  // segments per warp
  constexpr uint32_t SW = S * kSets;                 // shots per warp (<= 64)
  const uint32_t seg = (uint32_t)lane >> lw;         // this lane's segment
  const uint32_t sl = (uint32_t)lane & (Wd - 1u);    // its amplitude index
  const int base = (int)(seg << lw);                 // the segment's first lane
  DenseInstrDev* ins = reinterpret_cast<DenseInstrDev*>(rsm);
  // per warp: the sign word of each instruction (64 shots), then the active
  // outcomes of each of its shots
  uint32_t* wbase = reinterpret_cast<uint32_t*>(rsm + align16((size_t)G * sizeof(DenseInstrDev))) +
                    (size_t)warp * (2 * G + 64 * m3w);
  uint64_t* sgw = reinterpret_cast<uint64_t*>(wbase);
  uint32_t* m3all = wbase + 2 * G;
  for (uint32_t i = threadIdx.x; i < G * (sizeof(DenseInstrDev) / 4); i += blockDim.x)
    reinterpret_cast<uint32_t*>(ins)[i] = reinterpret_cast<const uint32_t*>(A.p.dense)[i];
  __syncthreads();

  uint32_t lead_mask = 0u;                           // lane 0 of every segment
  for (uint32_t q = 0; q < S; ++q) lead_mask |= 1u << (q << lw);
  const uint64_t wstride = (uint64_t)gridDim.x * kRegWarps * SW;
  for (uint64_t r0 = ((uint64_t)blockIdx.x * kRegWarps + warp) * SW; r0 < A.shots; r0 += wstride) {
    // set j of this segment holds request-local shot r0 + j S + seg; r0 is a
    // multiple of SW, which divides 64, so all of the warp's shots share the
    // 64-shot word r0 / 64
    const uint64_t w = r0 >> 6;
    uint64_t r[kSets];
    uint32_t* m3b[kSets];
#pragma unroll
    for (uint32_t j = 0; j < kSets; ++j) {
      r[j] = r0 + j * S + seg;
      m3b[j] = m3all + (size_t)(j * S + seg) * m3w;
    }
    for (uint32_t g = lane; g < G; g += 32)
      sgw[g] = __ldg(A.signs + (uint64_t)ins[g].sign_target_col * A.W + w);
    for (uint32_t i = lane; i < SW * m3w; i += 32) m3all[i] = 0u;
    __syncwarp();
    // shots past the request, or rejected before any active measurement, need
    // no dense work; their sets step along masked while others run
    bool dead[kSets];
    uint32_t deadm[kSets];
    bool all_dead = true;
#pragma unroll
    for (uint32_t j = 0; j < kSets; ++j) {
      dead[j] = r[j] >= A.shots;
      if (!dead[j] && sl == 0 && A.det_exo && A.p.post_grp0 == 0)
        dead[j] = group_rejects(A.p, A.det_exo, A.W, r[j], 0, m3b[j]);
      deadm[j] = __ballot_sync(0xffffffffu, sl == 0 && dead[j]);
      dead[j] = (deadm[j] >> base) & 1u;
      all_dead = all_dead && (deadm[j] & lead_mask) == lead_mask;
    }
    __syncwarp();
    if (all_dead) continue;
    ShotUniforms su[kSets];
    Real re[kSets], im[kSets];
#pragma unroll
    for (uint32_t j = 0; j < kSets; ++j) {
      re[j] = sl == 0 ? (Real)1 : (Real)0;
      im[j] = (Real)0;
    }
    uint32_t k = 0;
    for (uint32_t g = 0; g < G; ++g) {
      const DenseInstrDev& I = ins[g];
      const uint64_t sw = sgw[g];
      Real sg[kSets];
      uint32_t lam[kSets];
#pragma unroll
      for (uint32_t j = 0; j < kSets; ++j) {
        lam[j] = (uint32_t)(sw >> (r[j] & 63)) & 1u;
        for (uint32_t q = 0; q < I.causal_n; ++q) {
          const uint32_t jj = __ldg(A.p.dense_causal + I.causal_off + q);
          lam[j] ^= (m3b[j][jj >> 5] >> (jj & 31)) & 1u;
        }
        sg[j] = lam[j] ? (Real)-1 : (Real)1;
      }
      const Real c = coef_c<Real>(I), s = coef_s<Real>(I);
      const uint32_t n = 1u << k;
      if (I.kind == 0) {                       // PromoteRot
        const int src = base + (int)(sl >= n ? sl - n : sl);
#pragma unroll
        for (uint32_t j = 0; j < kSets; ++j) {
          const Real ore = shfl_r(re[j], src), oim = shfl_r(im[j], src);
          if (sl < n) {
            re[j] *= c;
            im[j] *= c;
          } else if (sl < 2 * n) {
            re[j] = sg[j] * s * oim;           // -i sg s alpha
            im[j] = -sg[j] * s * ore;
          }
        }
        ++k;
      } else if (I.kind == 1) {                // ActiveDiagRot
        const Real mu = I.mu == 0 ? (Real)1 : (Real)-1;
        const Real par = (__popc(sl & I.b) & 1) ? (Real)-1 : (Real)1;
#pragma unroll
        for (uint32_t j = 0; j < kSets; ++j) {
          const Real f = sg[j] * mu * s * par;
          const Real nre = c * re[j] + f * im[j], nim = c * im[j] - f * re[j];
          re[j] = nre;
          im[j] = nim;
        }
      } else if (I.kind == 2) {                // ActivePairRot
        Real cr, ci;                           // -i * i^mu
        switch (I.mu & 3) {
          case 0: cr = 0; ci = -1; break;
          case 1: cr = 1; ci = 0; break;
          case 2: cr = 0; ci = 1; break;
          default: cr = -1; ci = 0; break;
        }
        const uint32_t partner = (sl ^ I.a) & (Wd - 1u);
        const Real ps = (__popc(partner & I.b) & 1) ? (Real)-1 : (Real)1;
#pragma unroll
        for (uint32_t j = 0; j < kSets; ++j) {
          const Real pre = shfl_r(re[j], base + (int)partner), pim = shfl_r(im[j], base + (int)partner);
          const Real sp = ps * sg[j] * s;
          const Real nre = c * re[j] + sp * (cr * pre - ci * pim), nim = c * im[j] + sp * (cr * pim + ci * pre);
          if (sl < n) {
            re[j] = nre;
            im[j] = nim;
          }
        }
      } else {                                 // active measurements
        const int h = I.h;
        const uint32_t half = n >> 1;
        const Real inv_sqrt2 = (Real)0.70710678118654752440;
        const uint32_t z = sl;
        const uint32_t u0 = insert_bit(z & (half - 1 + (half == 0)), h, 0u);
        Real mcr = 0, mci = 0;
        if (I.kind == 6) {
          switch (I.mu & 3) {
            case 0: mcr = 1; mci = 0; break;
            case 1: mcr = 0; mci = -1; break;
            case 2: mcr = -1; mci = 0; break;
            default: mcr = 0; mci = 1; break;
          }
        }
        const int l0s = base + (int)(u0 & (Wd - 1u)), l1s = base + (int)((u0 ^ I.a) & (Wd - 1u));
        const Real sb = (__popc(I.b & u0) & 1) ? (Real)-1 : (Real)1;
        const bool podd = __popc(sl & I.b) & 1;
        bool stop = true;
#pragma unroll
        for (uint32_t j = 0; j < kSets; ++j) {
          // diag: partition by parity(b.x); pair: beta_z(y) from (u0, u0^a)
          Real b0re = 0, b0im = 0, b1re = 0, b1im = 0;
          Real s0 = 0, s1 = 0;                 // this lane's share (one amplitude)
          if (I.kind == 5) {
            if (sl < n) {
              const Real v = re[j] * re[j] + im[j] * im[j];
              if (podd) s1 = v; else s0 = v;
            }
          } else {
            const Real a0re = shfl_r(re[j], l0s), a0im = shfl_r(im[j], l0s);
            const Real a1re = shfl_r(re[j], l1s), a1im = shfl_r(im[j], l1s);
            const Real tr = sb * (mcr * a1re - mci * a1im), ti = sb * (mcr * a1im + mci * a1re);
            b0re = (a0re + tr) * inv_sqrt2; b0im = (a0im + ti) * inv_sqrt2;
            b1re = (a0re - tr) * inv_sqrt2; b1im = (a0im - ti) * inv_sqrt2;
            if (z < half) {
              s0 = b0re * b0re + b0im * b0im;
              s1 = b1re * b1re + b1im * b1im;
            }
          }
          // at most 32 terms, summed over the segment in the vector's own precision
          for (uint32_t o = Wd >> 1; o; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, (int)o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, (int)o);
          }
          const uint32_t l0 = I.kind == 5 ? (lam[j] ^ (uint32_t)I.eta) : lam[j];
          uint32_t m = 0;
          const uint64_t U = su[j].get(A, (uint32_t)I.m3, A.shot0 + r[j], (int)sl, lw, base);
          // decision and the renormalisation scale 1 / sqrt(S_m) on the
          // segment's first lane, in the vector's precision (self-normalised
          // probabilities make the scale matter only for the overall norm)
          Real sc = 0;
          if (sl == 0 && !dead[j]) {
            if (sizeof(Real) == 8) {
              const double pd = (double)(l0 ? s1 : s0) / (double)(s0 + s1);
              m = decide64(U, pd);
              if (A.prob) A.prob[(uint64_t)I.m3 * A.shots + r[j]] = pd;
            } else {
              const float pf = (float)((l0 ? s1 : s0) / (s0 + s1));
              m = decide32(U, pf);
              if (A.prob) A.prob[(uint64_t)I.m3 * A.shots + r[j]] = (double)pf;
            }
            sc = sizeof(Real) == 8 ? (Real)(1.0 / sqrt((double)((l0 ^ m) ? s1 : s0)))
                                   : (Real)rsqrtf((float)((l0 ^ m) ? s1 : s0));
          }
          m = __shfl_sync(0xffffffffu, m, base);
          const uint32_t lab = l0 ^ m;
          const Real scale = shfl_r(sc, base);
          if (I.kind == 5) {
            const uint32_t u = insert_bit(z & (half - 1 + (half == 0)), h, lab);
            const uint32_t x = u ^ ((uint32_t)(__popc(u & I.b & ~(1u << h)) & 1) << h);
            const int xs = base + (int)(x & (Wd - 1u));
            const Real nre = shfl_r(re[j], xs), nim = shfl_r(im[j], xs);
            re[j] = z < half ? nre * scale : (Real)0;
            im[j] = z < half ? nim * scale : (Real)0;
          } else {
            re[j] = z < half ? (lab ? b1re : b0re) * scale : (Real)0;
            im[j] = z < half ? (lab ? b1im : b0im) * scale : (Real)0;
          }
          if (m && sl == 0) {                  // m is 0 on dead segments
            m3b[j][I.m3 >> 5] |= 1u << (I.m3 & 31);
            atomicOr(reinterpret_cast<unsigned long long*>(A.m3_out) + (uint64_t)I.m3 * A.W + w,
                     1ull << (r[j] & 63));
          }
        }
        --k;
        __syncwarp();
        if (A.det_exo && I.post_grp != kNoGroup) {   // early exit once rejected
#pragma unroll
          for (uint32_t j = 0; j < kSets; ++j) {
            bool d2 = dead[j];
            if (!d2 && sl == 0) d2 = group_rejects(A.p, A.det_exo, A.W, r[j], I.post_grp, m3b[j]);
            deadm[j] = __ballot_sync(0xffffffffu, sl == 0 && d2);
            dead[j] = (deadm[j] >> base) & 1u;
            stop = stop && (deadm[j] & lead_mask) == lead_mask;
          }
          if (stop) break;
        }
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// CTA-per-shot dense executor for vectors up to ~200 KB: the whole CTA works
// on one shot's vector in shared memory.  (The kernel can also keep the vector
// in a per-CTA global slot when use_smem is 0; the library sends vectors that
// exceed shared memory to the wide executor instead, so it launches this
// kernel with use_smem = 1 only.)
// ---------------------------------------------------------------------------
constexpr int kCtaThreads = 256;

// One dense instruction on a vector of n = 2^k amplitudes held by a whole
// CTA (shared or global memory), with the instruction's sign lam (the CTA
// executor's body; red and bcast are the CTA's reduction and broadcast
// scratch).  A measurement writes the kept half to out, in place when out ==
// vec (pivot h the highest bit of a for a pair measurement), else to a
// disjoint region.
template <typename Real>
__device__ __forceinline__ void cta_instr(const DenseArgs& A, Cplx<Real>* vec, Cplx<Real>* out, uint32_t n,
                                          const DenseInstrDev& I, uint32_t lam, uint64_t rg, uint64_t r, uint64_t w,
                                          uint64_t bitmask, uint32_t* m3b, double* red, int* bcast, uint32_t tid) {
  const Real sg = lam ? (Real)-1 : (Real)1;
  const Real c = coef_c<Real>(I), s = coef_s<Real>(I);
  if (I.kind == 0) {
    for (uint32_t x = tid; x < n; x += blockDim.x) {
      Cplx<Real> v = vec[x], hi;
      hi.re = sg * s * v.im;
      hi.im = -sg * s * v.re;
      vec[x + n] = hi;
      v.re *= c;
      v.im *= c;
      vec[x] = v;
    }
  } else if (I.kind == 1) {
    const Real mu = I.mu == 0 ? (Real)1 : (Real)-1;
    for (uint32_t x = tid; x < n; x += blockDim.x) {
      const Real f = sg * mu * s * ((__popc(x & I.b) & 1) ? (Real)-1 : (Real)1);
      const Cplx<Real> v = vec[x];
      Cplx<Real> o;
      o.re = c * v.re + f * v.im;
      o.im = c * v.im - f * v.re;
      vec[x] = o;
    }
  } else if (I.kind == 2) {
    const int pb = 31 - __clz(I.a);
    Real cr, ci;
    switch (I.mu & 3) {
      case 0: cr = 0; ci = -1; break;
      case 1: cr = 1; ci = 0; break;
      case 2: cr = 0; ci = 1; break;
      default: cr = -1; ci = 0; break;
    }
    cr *= sg * s;
    ci *= sg * s;
    for (uint32_t z = tid; z < (n >> 1); z += blockDim.x) {
      const uint32_t x0 = insert_bit(z, pb, 0u), x1 = x0 ^ I.a;
      const Cplx<Real> v0 = vec[x0], v1 = vec[x1];
      const Real s1 = (__popc(x1 & I.b) & 1) ? (Real)-1 : (Real)1;
      const Real s0 = (__popc(x0 & I.b) & 1) ? (Real)-1 : (Real)1;
      Cplx<Real> o0, o1;
      o0.re = c * v0.re + s1 * (cr * v1.re - ci * v1.im);
      o0.im = c * v0.im + s1 * (cr * v1.im + ci * v1.re);
      o1.re = c * v1.re + s0 * (cr * v0.re - ci * v0.im);
      o1.im = c * v1.im + s0 * (cr * v0.im + ci * v0.re);
      vec[x0] = o0;
      vec[x1] = o1;
    }
  } else {
    const int h = I.h;
    const Real inv_sqrt2 = (Real)0.70710678118654752440;
    Real mcr = 0, mci = 0;
    if (I.kind == 6) {
      switch (I.mu & 3) {
        case 0: mcr = 1; mci = 0; break;
        case 1: mcr = 0; mci = -1; break;
        case 2: mcr = -1; mci = 0; break;
        default: mcr = 0; mci = 1; break;
      }
    }
    const uint32_t l0 = I.kind == 5 ? (lam ^ (uint32_t)I.eta) : lam;
    double S0 = 0.0, S1 = 0.0;
    if (sizeof(Real) == 8 || n >= (1u << 14)) {    // FP64 sums
      branch_sums<Real, double>(vec, I, n, tid, blockDim.x, mcr, mci, S0, S1);
      warp_sum2(S0, S1);
    } else {                                       // FP32 sums below 2^14 terms
      float F0 = 0.0f, F1 = 0.0f;
      branch_sums<Real, float>(vec, I, n, tid, blockDim.x, mcr, mci, F0, F1);
      warp_sum2(F0, F1);
      S0 = F0;
      S1 = F1;
    }
    if ((tid & 31) == 0) {
      red[tid >> 5] = S0;
      red[kCtaThreads / 32 + (tid >> 5)] = S1;
    }
    __syncthreads();
    S0 = 0.0;
    S1 = 0.0;
    for (int w2 = 0; w2 < kCtaThreads / 32; ++w2) {
      S0 += red[w2];
      S1 += red[kCtaThreads / 32 + w2];
    }
    if (tid == 0) {
      const double p0 = (l0 ? S1 : S0) / (S0 + S1);
      const uint32_t m = decide64(meas_U(A.keys, I.t, rg), p0);
      if (A.prob) A.prob[(uint64_t)I.m3 * A.shots + r] = p0;
      bcast[1] = (int)m;
      if (m) {
        m3b[I.m3 >> 5] |= 1u << (I.m3 & 31);
        atomicOr(reinterpret_cast<unsigned long long*>(A.m3_out) + (uint64_t)I.m3 * A.W + w,
                 (unsigned long long)bitmask);
      }
    }
    __syncthreads();
    const uint32_t m = (uint32_t)bcast[1];
    const uint32_t lab = l0 ^ m;
    const Real scale = (Real)(1.0 / sqrt(lab ? S1 : S0));
    const uint32_t half = n >> 1;
    for (uint32_t z0 = 0; z0 < half; z0 += blockDim.x) {
      const uint32_t z = z0 + tid;
      Cplx<Real> v;
      v.re = 0;
      v.im = 0;
      if (z < half) {
        if (I.kind == 5) {
          const uint32_t u = insert_bit(z, h, lab);
          v = vec[u ^ ((uint32_t)(__popc(u & I.b & ~(1u << h)) & 1) << h)];
        } else {
          const uint32_t u0 = insert_bit(z, h, 0u);
          const Cplx<Real> a0 = vec[u0], a1 = vec[u0 ^ I.a];
          Real sb = (__popc(I.b & u0) & 1) ? (Real)-1 : (Real)1;
          if (lab) sb = -sb;
          const Real tr = sb * (mcr * a1.re - mci * a1.im), tim = sb * (mcr * a1.im + mci * a1.re);
          v.re = (a0.re + tr) * inv_sqrt2;
          v.im = (a0.im + tim) * inv_sqrt2;
        }
        v.re *= scale;
        v.im *= scale;
      }
      __syncthreads();
      if (z < half) out[z] = v;
      __syncthreads();
    }
  }
}

template <typename Real>
__global__ void __launch_bounds__(kCtaThreads) dense_cta_kernel(DenseArgs A) {
  extern __shared__ __align__(16) unsigned char csm[];
  const uint32_t tid = threadIdx.x;
  const uint32_t G = A.p.n_dense;
  const uint32_t m3w = (A.p.n_m3 + 31) / 32;
  uint32_t* m3b = reinterpret_cast<uint32_t*>(csm);
  double* red = reinterpret_cast<double*>(csm + align16(m3w * 4 + 16));
  int* bcast = reinterpret_cast<int*>(red + 2 * (kCtaThreads / 32));
  Cplx<Real>* vec = A.use_smem
                        ? reinterpret_cast<Cplx<Real>*>(csm + align16(m3w * 4 + 16) + align16(2 * (kCtaThreads / 32) * 8 + 16))
                        : reinterpret_cast<Cplx<Real>*>(A.gvec) + (uint64_t)blockIdx.x * A.gvec_stride;
  for (uint64_t r = blockIdx.x; r < A.shots; r += gridDim.x) {
    const uint64_t rg = A.shot0 + r;
    const uint64_t w = r >> 6;
    const uint64_t bitmask = 1ull << (r & 63);
    for (uint32_t i = tid; i < m3w; i += blockDim.x) m3b[i] = 0u;
    if (tid == 0) {
      vec[0].re = (Real)1;
      vec[0].im = (Real)0;
    }
    __syncthreads();
    // a shot rejected before any active measurement needs no dense work
    const bool dead0 = A.det_exo && A.p.post_grp0 == 0 && group_rejects(A.p, A.det_exo, A.W, r, 0, m3b);
    __syncthreads();
    if (dead0) continue;
    uint32_t k = 0;
    for (uint32_t g = 0; g < G; ++g) {
      const DenseInstrDev I = A.p.dense[g];
      if (tid == 0) {
        uint32_t lam = (uint32_t)((__ldg(A.signs + (uint64_t)I.sign_target_col * A.W + w) & bitmask) != 0);
        for (uint32_t q = 0; q < I.causal_n; ++q) {
          const uint32_t j = __ldg(A.p.dense_causal + I.causal_off + q);
          lam ^= (m3b[j >> 5] >> (j & 31)) & 1u;
        }
        bcast[0] = (int)lam;
      }
      __syncthreads();
      const uint32_t lam = (uint32_t)bcast[0];
      const uint32_t n = 1u << k;
      cta_instr<Real>(A, vec, vec, n, I, lam, rg, r, w, bitmask, m3b, red, bcast, tid);
      if (I.kind == 0) {
        ++k;
      } else if (I.kind == 5 || I.kind == 6) {
        --k;
        if (A.det_exo && I.post_grp != kNoGroup) {   // early exit once rejected
          const bool dead = group_rejects(A.p, A.det_exo, A.W, r, I.post_grp, m3b);
          __syncthreads();
          if (dead) break;
        }
      }
      __syncthreads();
    }
  }
}

// Product-component program on one CTA per shot: the component workspace
// (pc_capacity amplitudes) in shared memory or a per-CTA global slot, every
// INIT / MERGE / APPLY op executed by the whole CTA (for components of
// thousands of amplitudes, where one warp per shot leaves the SM idle).
template <typename Real>
__global__ void __launch_bounds__(kCtaThreads) dense_pc_cta_kernel(DenseArgs A) {
  extern __shared__ __align__(16) unsigned char csm[];
  const uint32_t tid = threadIdx.x;
  const uint32_t m3w = (A.p.n_m3 + 31) / 32;
  uint32_t* m3b = reinterpret_cast<uint32_t*>(csm);
  double* red = reinterpret_cast<double*>(csm + align16(m3w * 4 + 16));
  int* bcast = reinterpret_cast<int*>(red + 2 * (kCtaThreads / 32));
  Cplx<Real>* ws = A.use_smem
                       ? reinterpret_cast<Cplx<Real>*>(csm + align16(m3w * 4 + 16) + align16(2 * (kCtaThreads / 32) * 8 + 16))
                       : reinterpret_cast<Cplx<Real>*>(A.gvec) + (uint64_t)blockIdx.x * A.gvec_stride;
  for (uint64_t r = blockIdx.x; r < A.shots; r += gridDim.x) {
    const uint64_t rg = A.shot0 + r;
    const uint64_t w = r >> 6;
    const uint64_t bitmask = 1ull << (r & 63);
    for (uint32_t i = tid; i < m3w; i += blockDim.x) m3b[i] = 0u;
    __syncthreads();
    const bool dead0 = A.det_exo && A.p.post_grp0 == 0 && group_rejects(A.p, A.det_exo, A.W, r, 0, m3b);
    __syncthreads();
    if (dead0) continue;
    for (uint32_t q = 0; q < A.p.n_pc; ++q) {
      const PCOp O = A.p.pc[q];
      if (O.op == PC_MERGE) {
        const uint32_t na = 1u << O.kA, nc = 1u << (O.kA + O.kB);
        const Cplx<Real>* pa = ws + O.offA;
        const Cplx<Real>* pb = ws + O.offB;
        Cplx<Real>* pcv = ws + O.off;
        for (uint32_t x = tid; x < nc; x += blockDim.x) {
          const Cplx<Real> u = pa[x & (na - 1)], v = pb[x >> O.kA];
          Cplx<Real> t;
          t.re = u.re * v.re - u.im * v.im;
          t.im = u.re * v.im + u.im * v.re;
          pcv[x] = t;
        }
        __syncthreads();
        continue;
      }
      DenseInstrDev I = A.p.dense[O.g];
      if (tid == 0) {
        uint32_t lam = (uint32_t)((__ldg(A.signs + (uint64_t)I.sign_target_col * A.W + w) & bitmask) != 0);
        for (uint32_t c = 0; c < I.causal_n; ++c) {
          const uint32_t j = __ldg(A.p.dense_causal + I.causal_off + c);
          lam ^= (m3b[j >> 5] >> (j & 31)) & 1u;
        }
        bcast[0] = (int)lam;
        if (O.op == PC_INIT) {
          ws[O.off].re = (Real)1;
          ws[O.off].im = (Real)0;
        }
      }
      __syncthreads();
      const uint32_t lam = (uint32_t)bcast[0];
      Cplx<Real>* vec = ws + O.off;
      if (O.op == PC_INIT) {
        cta_instr<Real>(A, vec, vec, 1u, I, lam, rg, r, w, bitmask, m3b, red, bcast, tid);
        __syncthreads();
        continue;
      }
      I.a = O.a;
      I.b = O.b;
      I.h = O.h;
      cta_instr<Real>(A, vec, ws + O.out, 1u << O.k, I, lam, rg, r, w, bitmask, m3b, red, bcast, tid);
      if (I.kind == 5 || I.kind == 6) {
        if (A.det_exo && I.post_grp != kNoGroup) {   // early exit once rejected
          const bool dead = group_rejects(A.p, A.det_exo, A.W, r, I.post_grp, m3b);
          __syncthreads();
          if (dead) break;
        }
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// Plain form (the paper's GPU design rebuilt, for comparison): one CTA per
// shot; the shot draws its own noise components and random bits from the
// same streams, evaluates every sign unpacked from its full symbol list, runs
// the dense instructions on a vector in shared memory and OR-s its output bits
// into the (zeroed) columns.
// ---------------------------------------------------------------------------
constexpr int kPlainThreads = 128;

struct PlainLayout {
  size_t fired, m1, val, m3, vec, red, total;
};

__host__ __device__ inline PlainLayout plain_layout(const DevPlan& p, uint32_t kmax, size_t amp) {
  PlainLayout L;
  const uint32_t NTP = p.tgt_sign0 + p.n_dense;
  L.fired = 0;
  L.m1 = L.fired + align16(((p.n_comp + 31) / 32) * 4);
  L.val = L.m1 + align16(((p.n_m1 + 31) / 32) * 4);
  L.m3 = L.val + align16(NTP);
  L.vec = L.m3 + align16(((p.n_m3 + 31) / 32) * 4 + 16);
  L.red = L.vec + align16(((size_t)1 << kmax) * amp);
  L.total = L.red + 2 * kPlainThreads * sizeof(double) + 32;
  return L;
}

__device__ __forceinline__ int first_above_global(const uint32_t* __restrict__ th, uint32_t u) {
  int lo = 0, hi = kNoiseBlock;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (u < __ldg(th + mid)) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// block-wide sum of two doubles (all threads get the result)
__device__ __forceinline__ void block_sum2(double& a, double& b, double* red) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[warp] = a;
    red[kPlainThreads / 32 + warp] = b;
  }
  __syncthreads();
  a = 0.0;
  b = 0.0;
  for (int w = 0; w < kPlainThreads / 32; ++w) {
    a += red[w];
    b += red[kPlainThreads / 32 + w];
  }
  __syncthreads();
}

template <typename Real>
__global__ void __launch_bounds__(kPlainThreads) plain_kernel(PlainArgs A) {
  extern __shared__ __align__(16) unsigned char psm[];
  const DevPlan& P = A.p;
  const PlainLayout Lay = plain_layout(P, A.kmax, sizeof(Cplx<Real>));
  uint32_t* fired = reinterpret_cast<uint32_t*>(psm + Lay.fired);
  uint32_t* m1b = reinterpret_cast<uint32_t*>(psm + Lay.m1);
  uint8_t* val = psm + Lay.val;
  uint32_t* m3b = reinterpret_cast<uint32_t*>(psm + Lay.m3);
  Cplx<Real>* vec = reinterpret_cast<Cplx<Real>*>(psm + Lay.vec);
  double* red = reinterpret_cast<double*>(psm + Lay.red);
  int* bcast = reinterpret_cast<int*>(red + 2 * kPlainThreads);
  const uint32_t tid = threadIdx.x;
  const uint32_t k0 = (uint32_t)A.seed, k1 = (uint32_t)(A.seed >> 32);
  const uint32_t R = P.n_records, NO = P.tgt_sign0;
  const uint32_t NTP = NO + P.n_dense;
  const uint32_t n_groups = (P.n_channels + 3) >> 2;

  for (uint64_t r = blockIdx.x; r < A.shots; r += gridDim.x) {
    const uint64_t rg = A.shot0 + r;
    const uint32_t gb = (uint32_t)(rg / kNoiseBlock), my_lane = (uint32_t)(rg % kNoiseBlock);
    const uint64_t w = r >> 6;
    const uint64_t bitmask = 1ull << (r & 63);
    for (uint32_t i = tid; i < (P.n_comp + 31) / 32; i += blockDim.x) fired[i] = 0u;
    for (uint32_t i = tid; i < (P.n_m1 + 31) / 32; i += blockDim.x) m1b[i] = 0u;
    for (uint32_t i = tid; i < (P.n_m3 + 31) / 32; i += blockDim.x) m3b[i] = 0u;
    __syncthreads();
    // 1. this shot's noise: run each channel's process up to the shot's lane
    for (uint32_t g = tid; g < n_groups; g += blockDim.x) {
      const uint4 th4 = __ldg(P.theta4 + g);
      if (!(th4.x | th4.y | th4.z | th4.w)) continue;
      const uint4 head = philox(make_uint4(g, gb, 0u, kTagHead), k0, k1);
      for (uint32_t s2 = 0; s2 < 4; ++s2) {
        const uint32_t c = 4 * g + s2;
        if (c >= P.n_channels) break;
        uint32_t u = pick(head, s2);
        if (u >= pick(th4, s2)) continue;
        const uint4 raw = __ldg(reinterpret_cast<const uint4*>(P.ch) + c);
        const uint32_t* th = P.qtheta + (size_t)(raw.y & 0xFFFFu) * kNoiseBlock;
        const CellTableDev* ct = P.ctabs + (raw.y >> 16);
        const uint32_t ncell = ct->ncell;
        uint32_t ti = 0;
        int L = 0;
        for (int guard = 0; guard <= kNoiseBlock; ++guard) {
          const int j = first_above_global(th, u);
          if (j > kNoiseBlock - 1 - L) break;
          const int lanebit = L + j;
          if ((uint32_t)lanebit > my_lane) break;
          uint32_t cell = 0;
          if (ncell > 1) {
            const uint4 t4 = philox(make_uint4(c, gb, ti >> 2, kTagTail), k0, k1);
            const uint32_t v = pick(t4, ti & 3);
            ++ti;
            cell = ncell - 1;
            for (uint32_t kk = 0; kk + 1 < ncell; ++kk)
              if (v < ct->phi[kk]) { cell = kk; break; }
          }
          if ((uint32_t)lanebit == my_lane) {
            uint32_t mask = ct->mask[cell];
            while (mask) {
              const uint32_t comp = raw.z + (__ffs(mask) - 1);
              mask &= mask - 1;
              atomicOr(fired + (comp >> 5), 1u << (comp & 31));
            }
            break;
          }
          L = lanebit + 1;
          if (L >= kNoiseBlock) break;
          const uint4 t4 = philox(make_uint4(c, gb, ti >> 2, kTagTail), k0, k1);
          u = pick(t4, ti & 3);
          ++ti;
        }
      }
    }
    // 2. random measurement bits
    for (uint32_t j = tid; j < P.n_m1; j += blockDim.x) {
      const uint64_t wg = rg >> 6;
      const uint4 o = philox(make_uint4(__ldg(P.m1_t + j), (uint32_t)(wg >> 1), (uint32_t)(wg >> 33), kTagMbit), k0, k1);
      const uint64_t word = (wg & 1) ? ((uint64_t)o.z | ((uint64_t)o.w << 32)) : ((uint64_t)o.x | ((uint64_t)o.y << 32));
      if ((word >> (rg & 63)) & 1ull) atomicOr(m1b + (j >> 5), 1u << (j & 31));
    }
    __syncthreads();
    // 3. every exogenous sign, unpacked, from its full symbol list
    for (uint32_t i = tid; i < NTP; i += blockDim.x) {
      uint32_t v = __ldg(P.plain_const + i);
      const uint32_t e = __ldg(P.plain_off + i + 1);
      for (uint32_t q = __ldg(P.plain_off + i); q < e; ++q) {
        const uint32_t sy = __ldg(P.plain_sym + q);
        v ^= sy < P.n_comp ? (fired[sy >> 5] >> (sy & 31)) & 1u
                           : (m1b[(sy - P.n_comp) >> 5] >> ((sy - P.n_comp) & 31)) & 1u;
      }
      val[i] = (uint8_t)v;
    }
    if (tid == 0) {
      vec[0].re = (Real)1;
      vec[0].im = (Real)0;
    }
    __syncthreads();
    // early exit (this design ends a rejected shot at once): whether a
    // postselected detector of group q fires, from the shot's unpacked
    // exogenous detector values and its active outcomes so far
    auto plain_rejects = [&](uint32_t q) -> bool {
      if (!P.post_chk_off) return false;
      const uint32_t e1 = __ldg(P.post_chk_off + q + 1);
      for (uint32_t e = __ldg(P.post_chk_off + q); e < e1; ++e) {
        const uint32_t i = R + __ldg(P.post_chk + e);     // the detector's output index
        uint32_t v = val[i];
        const uint32_t ce = __ldg(P.tgt_causal_off + i + 1);
        for (uint32_t c = __ldg(P.tgt_causal_off + i); c < ce; ++c) {
          const uint32_t j = __ldg(P.tgt_causal + c);
          v ^= (m3b[j >> 5] >> (j & 31)) & 1u;
        }
        if (v) return true;
      }
      return false;
    };
    // 4. dense instructions on the shot's vector (skipped once rejected)
    uint32_t k = 0;
    const bool dead0 = plain_rejects(0);
    for (uint32_t g = 0; g < P.n_dense && !dead0; ++g) {
      const DenseInstrDev I = P.dense[g];
      if (tid == 0) {
        uint32_t lam = val[NO + g];
        for (uint32_t q = 0; q < I.causal_n; ++q) {
          const uint32_t j = __ldg(P.dense_causal + I.causal_off + q);
          lam ^= (m3b[j >> 5] >> (j & 31)) & 1u;
        }
        bcast[0] = (int)lam;
      }
      __syncthreads();
      const uint32_t lam = (uint32_t)bcast[0];
      const Real sg = lam ? (Real)-1 : (Real)1;
      const Real c = coef_c<Real>(I), s = coef_s<Real>(I);
      const uint32_t n = 1u << k;
      if (I.kind == 0) {
        for (uint32_t x = tid; x < n; x += blockDim.x) {
          Cplx<Real> v = vec[x], hi;
          hi.re = sg * s * v.im;
          hi.im = -sg * s * v.re;
          vec[x + n] = hi;
          v.re *= c;
          v.im *= c;
          vec[x] = v;
        }
        ++k;
      } else if (I.kind == 1) {
        const Real mu = I.mu == 0 ? (Real)1 : (Real)-1;
        for (uint32_t x = tid; x < n; x += blockDim.x) {
          const Real f = sg * mu * s * ((__popc(x & I.b) & 1) ? (Real)-1 : (Real)1);
          const Cplx<Real> v = vec[x];
          Cplx<Real> o;
          o.re = c * v.re + f * v.im;
          o.im = c * v.im - f * v.re;
          vec[x] = o;
        }
      } else if (I.kind == 2) {
        const int pb = 31 - __clz(I.a);
        Real cr, ci;
        switch (I.mu & 3) {
          case 0: cr = 0; ci = -1; break;
          case 1: cr = 1; ci = 0; break;
          case 2: cr = 0; ci = 1; break;
          default: cr = -1; ci = 0; break;
        }
        cr *= sg * s;
        ci *= sg * s;
        for (uint32_t z = tid; z < (n >> 1); z += blockDim.x) {
          const uint32_t x0 = insert_bit(z, pb, 0u), x1 = x0 ^ I.a;
          const Cplx<Real> v0 = vec[x0], v1 = vec[x1];
          const Real s1 = (__popc(x1 & I.b) & 1) ? (Real)-1 : (Real)1;
          const Real s0 = (__popc(x0 & I.b) & 1) ? (Real)-1 : (Real)1;
          Cplx<Real> o0, o1;
          o0.re = c * v0.re + s1 * (cr * v1.re - ci * v1.im);
          o0.im = c * v0.im + s1 * (cr * v1.im + ci * v1.re);
          o1.re = c * v1.re + s0 * (cr * v0.re - ci * v0.im);
          o1.im = c * v1.im + s0 * (cr * v0.im + ci * v0.re);
          vec[x0] = o0;
          vec[x1] = o1;
        }
      } else {
        const int h = I.h;
        const Real inv_sqrt2 = (Real)0.70710678118654752440;
        Real mcr = 0, mci = 0;
        if (I.kind == 6) {
          switch (I.mu & 3) {
            case 0: mcr = 1; mci = 0; break;
            case 1: mcr = 0; mci = -1; break;
            case 2: mcr = -1; mci = 0; break;
            default: mcr = 0; mci = 1; break;
          }
        }
        double S0 = 0.0, S1 = 0.0;
        if (I.kind == 5) {
          for (uint32_t x = tid; x < n; x += blockDim.x) {
            const double v = norm2(vec[x]);
            if (__popc(x & I.b) & 1) S1 += v; else S0 += v;
          }
        } else {
          for (uint32_t z = tid; z < (n >> 1); z += blockDim.x) {
            const uint32_t u0 = insert_bit(z, h, 0u);
            const Cplx<Real> a0 = vec[u0], a1 = vec[u0 ^ I.a];
            const Real sb = (__popc(I.b & u0) & 1) ? (Real)-1 : (Real)1;
            const Real tr = sb * (mcr * a1.re - mci * a1.im), tim = sb * (mcr * a1.im + mci * a1.re);
            Cplx<Real> b0, b1;
            b0.re = (a0.re + tr) * inv_sqrt2; b0.im = (a0.im + tim) * inv_sqrt2;
            b1.re = (a0.re - tr) * inv_sqrt2; b1.im = (a0.im - tim) * inv_sqrt2;
            S0 += norm2(b0);
            S1 += norm2(b1);
          }
        }
        block_sum2(S0, S1, red);
        const uint32_t l0 = I.kind == 5 ? (lam ^ (uint32_t)I.eta) : lam;
        const double p0 = (l0 ? S1 : S0) / (S0 + S1);
        if (tid == 0) {
          const uint32_t m = meas_uniform(A.seed, I.t, rg) < p0 ? 0u : 1u;
          if (A.prob) A.prob[(uint64_t)I.m3 * A.shots + r] = p0;
          bcast[1] = (int)m;
          if (m) m3b[I.m3 >> 5] |= 1u << (I.m3 & 31);
        }
        __syncthreads();
        const uint32_t m = (uint32_t)bcast[1];
        const uint32_t lab = l0 ^ m;
        const Real scale = (Real)(1.0 / sqrt(lab ? S1 : S0));
        const uint32_t half = n >> 1;
        for (uint32_t z0 = 0; z0 < half; z0 += blockDim.x) {
          const uint32_t z = z0 + tid;
          Cplx<Real> v;
          v.re = 0;
          v.im = 0;
          if (z < half) {
            if (I.kind == 5) {
              const uint32_t u = insert_bit(z, h, lab);
              v = vec[u ^ ((uint32_t)(__popc(u & I.b & ~(1u << h)) & 1) << h)];
            } else {
              const uint32_t u0 = insert_bit(z, h, 0u);
              const Cplx<Real> a0 = vec[u0], a1 = vec[u0 ^ I.a];
              Real sb = (__popc(I.b & u0) & 1) ? (Real)-1 : (Real)1;
              if (lab) sb = -sb;
              const Real tr = sb * (mcr * a1.re - mci * a1.im), tim = sb * (mcr * a1.im + mci * a1.re);
              v.re = (a0.re + tr) * inv_sqrt2;
              v.im = (a0.im + tim) * inv_sqrt2;
            }
            v.re *= scale;
            v.im *= scale;
          }
          __syncthreads();
          if (z < half) vec[z] = v;
          __syncthreads();
        }
        --k;
        const bool dead = plain_rejects((uint32_t)I.m3 + 1);
        __syncthreads();
        if (dead) break;
      }
      __syncthreads();
    }
    // 5. outputs: causal residuals, postselection, OR into the columns
    for (uint32_t i = tid; i < NO; i += blockDim.x) {
      uint32_t v = val[i];
      const uint32_t e = __ldg(P.tgt_causal_off + i + 1);
      for (uint32_t q = __ldg(P.tgt_causal_off + i); q < e; ++q) {
        const uint32_t j = __ldg(P.tgt_causal + q);
        v ^= (m3b[j >> 5] >> (j & 31)) & 1u;
      }
      val[i] = (uint8_t)v;
    }
    __syncthreads();
    if (tid == 0) {
      int cut = 0;
      if (P.postselect) {
        for (uint32_t e = 0; e < P.n_post_events; ++e) {
          const int32_t ev = __ldg(P.post_events + e);
          if (ev >= 0) {
            if (cut) val[ev] = 0;
          } else {
            const uint32_t code = (uint32_t)(-1 - ev);
            const uint32_t di = R + (code >> 1);
            if (cut) val[di] = 0;
            else if ((code & 1u) && val[di]) cut = 1;
          }
        }
        if (cut)
          for (uint32_t j = 0; j < P.n_obs; ++j) val[R + P.n_dets + j] = 0;
      }
      bcast[2] = cut;
    }
    __syncthreads();
    for (uint32_t i = tid; i < NO; i += blockDim.x) {
      if (!val[i]) continue;
      uint64_t* col;
      uint64_t idx;
      if (i < R) { col = A.meas; idx = i; }
      else if (i < R + P.n_dets) { col = A.det; idx = i - R; }
      else { col = A.obs; idx = i - R - P.n_dets; }
      if (col) atomicOr(reinterpret_cast<unsigned long long*>(col + idx * A.W + w), (unsigned long long)bitmask);
    }
    if (tid == 0 && bcast[2] && A.discard)
      atomicOr(reinterpret_cast<unsigned long long*>(A.discard + w), (unsigned long long)bitmask);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Finalize: causal residuals of records/detectors/observables and postselection.
// ---------------------------------------------------------------------------


__global__ void finalize_kernel(FinalArgs A) {
  constexpr uint32_t kEv = 8;   // columns (outputs, postselection events) whose words are loaded together
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < A.W; w += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t pad = ~0ull;
    if (w == A.W - 1 && (A.shots & 63)) pad = (1ull << (A.shots & 63)) - 1;
    if (A.m3) {
      // outputs with causal terms: XOR in the active outcomes they name.
      // Each output is its own column, so a batch's words are all loaded
      // before any is stored.
      for (uint32_t t0 = 0; t0 < A.p.n_causal_tgt; t0 += kEv) {
        const uint32_t nt = min(kEv, A.p.n_causal_tgt - t0);
        uint64_t* ptr[kEv];
        uint64_t val[kEv], acc[kEv];
#pragma unroll
        for (uint32_t j = 0; j < kEv; ++j) {
          ptr[j] = nullptr;
          val[j] = 0;
          acc[j] = 0;
          if (j < nt) {
            const uint4 it = __ldg(A.p.causal_tgt + t0 + j);
            for (uint32_t q = it.y; q < it.y + it.z; ++q)
              acc[j] ^= A.m3[(uint64_t)__ldg(A.p.tgt_causal + q) * A.W + w];
            const uint32_t i = it.x;
            if (i < A.p.tgt_det0) ptr[j] = A.meas ? A.meas + (uint64_t)i * A.W + w : nullptr;
            else if (i < A.p.tgt_obs0) ptr[j] = A.det ? A.det + (uint64_t)(i - A.p.tgt_det0) * A.W + w : nullptr;
            else ptr[j] = A.obs ? A.obs + (uint64_t)(i - A.p.tgt_obs0) * A.W + w : nullptr;
            if (ptr[j]) val[j] = *ptr[j];
          }
        }
#pragma unroll
        for (uint32_t j = 0; j < kEv; ++j)
          if (ptr[j]) *ptr[j] = val[j] ^ (acc[j] & pad);
      }
    }
    if (A.p.postselect) {
      // the walk in circuit order: every record and detector after the first
      // fired postselected detector is cleared.  Each event is its own
      // column, so a batch's words are all loaded before any is stored.
      uint64_t cut = 0;
      for (uint32_t e0 = 0; e0 < A.p.n_post_events; e0 += kEv) {
        const uint32_t ne = min(kEv, A.p.n_post_events - e0);
        uint64_t* ptr[kEv];
        uint64_t val[kEv];
#pragma unroll
        for (uint32_t j = 0; j < kEv; ++j) {
          ptr[j] = nullptr;
          val[j] = 0;
          if (j < ne) {
            const int32_t ev = __ldg(A.p.post_events + e0 + j);
            if (ev >= 0) ptr[j] = A.meas ? A.meas + (uint64_t)ev * A.W + w : nullptr;
            else ptr[j] = A.det + (uint64_t)((uint32_t)(-1 - ev) >> 1) * A.W + w;
            if (ptr[j]) val[j] = *ptr[j];
          }
        }
#pragma unroll
        for (uint32_t j = 0; j < kEv; ++j) {
          if (j < ne) {
            const int32_t ev = __ldg(A.p.post_events + e0 + j);
            const uint64_t v = val[j] & ~cut;
            if (ptr[j]) *ptr[j] = v;
            if (ev < 0 && (((uint32_t)(-1 - ev)) & 1u)) cut |= v;
          }
        }
      }
      if (A.obs)
        for (uint32_t j = 0; j < A.p.n_obs; ++j) A.obs[(uint64_t)j * A.W + w] &= ~cut;
      if (A.discard) A.discard[w] = cut & pad;
    } else if (A.discard) {
      A.discard[w] = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// Tallies of a request: kept and discarded shots, and for each observable the
// kept shots that read 1 (the undetected logical errors of a memory or
// distillation experiment).  Pass j = 0 counts kept/discarded, pass j >= 1
// observable j - 1; each warp adds its partial counts with one atomic.
// ---------------------------------------------------------------------------
__global__ void count_kernel(CountArgs A) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t w0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (uint32_t j = 0; j <= A.n_obs; ++j) {
    unsigned long long c0 = 0, c1 = 0;
    for (uint64_t w = w0; w < A.W; w += stride) {
      uint64_t pad = ~0ull;
      if (w == A.W - 1 && (A.shots & 63)) pad = (1ull << (A.shots & 63)) - 1;
      const uint64_t d = A.discard ? (A.discard[w] & pad) : 0ull;
      if (j == 0) {
        c0 += (unsigned long long)__popcll(pad & ~d);
        c1 += (unsigned long long)__popcll(d);
      } else {
        c0 += (unsigned long long)__popcll(A.obs[(uint64_t)(j - 1) * A.W + w] & pad & ~d);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      c0 += __shfl_down_sync(0xffffffffu, c0, o);
      c1 += __shfl_down_sync(0xffffffffu, c1, o);
    }
    if ((threadIdx.x & 31) == 0) {
      if (j == 0) {
        if (c0) atomicAdd(A.counts + 0, c0);
        if (c1) atomicAdd(A.counts + 1, c1);
      } else if (c0) {
        atomicAdd(A.counts + 1 + j, c0);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// launch wrappers (host)
// ---------------------------------------------------------------------------
cudaError_t set_smem_limits();

template <typename Real>
cudaError_t launch_dense_t(const DenseArgs& a, int warps_per_block, int grid, size_t smem, cudaStream_t st,
                           int shots_per_warp) {
  if (shots_per_warp == 2) dense_kernel<Real, 2><<<grid, warps_per_block * 32, smem, st>>>(a);
  else dense_kernel<Real, 1><<<grid, warps_per_block * 32, smem, st>>>(a);
  return cudaGetLastError();
}

size_t dense_cta_smem_bytes(const DevPlan& p, size_t vec_bytes, bool vec_in_smem) {
  return align16(((p.n_m3 + 31) / 32) * 4 + 16) + align16(2 * (kCtaThreads / 32) * 8 + 16) +
         (vec_in_smem ? vec_bytes : 0);
}

cudaError_t launch_dense_cta(const DenseArgs& a, bool fp64, int grid, size_t smem, cudaStream_t st) {
  if (fp64) dense_cta_kernel<double><<<grid, kCtaThreads, smem, st>>>(a);
  else dense_cta_kernel<float><<<grid, kCtaThreads, smem, st>>>(a);
  return cudaGetLastError();
}

size_t dense_warp_smem_bytes(const DevPlan& p, int wpb, size_t vec_bytes, bool vec_in_smem) {
  const size_t bk = ((size_t)(p.n_m3 + 31) / 32 + (p.n_dense + 31) / 32) * 4;   // per warp
  return stage_bytes((size_t)p.n_dense * sizeof(DenseInstrDev)) + (((size_t)wpb * bk + 15) & ~(size_t)15) +
         (vec_in_smem ? (size_t)wpb * vec_bytes : 0);
}

size_t dense_pc_smem_bytes(const DevPlan& p, int wpb, size_t ws_bytes, bool ws_in_smem) {
  const size_t bk = ((size_t)(p.n_m3 + 31) / 32 + (p.n_dense + 31) / 32) * 4;   // per warp
  return stage_bytes((size_t)p.n_dense * sizeof(DenseInstrDev) + (size_t)p.n_pc * sizeof(PCOp)) +
         (((size_t)wpb * bk + 15) & ~(size_t)15) + (ws_in_smem ? (size_t)wpb * ws_bytes : 0);
}

size_t dense_reg_smem_bytes(const DevPlan& p) {
  const size_t G = p.n_dense;
  return align16((size_t)G * sizeof(DenseInstrDev)) + (size_t)kRegWarps * (2 * G + 64 * ((p.n_m3 + 31) / 32)) * 4 + 16;
}

template <typename Real>
static void launch_dense_reg_t(const DenseArgs& a, int grid, size_t smem, cudaStream_t st) {
  constexpr uint32_t K = sizeof(Real) == 4 ? kRegSetsF32 : 1;
  switch (a.kmax) {
    case 1: dense_reg_kernel<Real, 1, K><<<grid, kRegWarps * 32, smem, st>>>(a); break;
    case 2: dense_reg_kernel<Real, 2, K><<<grid, kRegWarps * 32, smem, st>>>(a); break;
    case 3: dense_reg_kernel<Real, 3, K><<<grid, kRegWarps * 32, smem, st>>>(a); break;
    case 4: dense_reg_kernel<Real, 4, K><<<grid, kRegWarps * 32, smem, st>>>(a); break;
    default: dense_reg_kernel<Real, 5, K><<<grid, kRegWarps * 32, smem, st>>>(a); break;
  }
}

uint32_t dense_reg_shots_per_cta(uint32_t kmax, bool fp64) {
  return (uint32_t)kRegWarps * (32u >> kmax) * (fp64 ? 1u : kRegSetsF32);
}

cudaError_t launch_dense_reg(const DenseArgs& a, bool fp64, int grid, cudaStream_t st) {
  if (a.kmax < 1 || a.kmax > 5) return cudaErrorInvalidValue;
  const size_t smem = dense_reg_smem_bytes(a.p);
  if (fp64) launch_dense_reg_t<double>(a, grid, smem, st);
  else launch_dense_reg_t<float>(a, grid, smem, st);
  return cudaGetLastError();
}

cudaError_t launch_dense_pc(const DenseArgs& a, bool fp64, int warps_per_block, int grid, size_t smem, cudaStream_t st) {
  if (fp64) dense_pc_kernel<double><<<grid, warps_per_block * 32, smem, st>>>(a);
  else dense_pc_kernel<float><<<grid, warps_per_block * 32, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t dense_pc_occupancy(bool fp64, int warps_per_block, size_t smem, int* ctas_per_sm) {
  cudaError_t e = set_smem_limits();
  if (e != cudaSuccess) return e;
  const void* f = fp64 ? (const void*)dense_pc_kernel<double> : (const void*)dense_pc_kernel<float>;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, f, warps_per_block * 32, smem);
}

cudaError_t launch_dense_pc_cta(const DenseArgs& a, bool fp64, int grid, size_t smem, cudaStream_t st) {
  if (fp64) dense_pc_cta_kernel<double><<<grid, kCtaThreads, smem, st>>>(a);
  else dense_pc_cta_kernel<float><<<grid, kCtaThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_dense(const DenseArgs& a, bool fp64, int warps_per_block, int grid, size_t smem, cudaStream_t st,
                         int shots_per_warp) {
  return fp64 ? launch_dense_t<double>(a, warps_per_block, grid, smem, st, shots_per_warp)
              : launch_dense_t<float>(a, warps_per_block, grid, smem, st, shots_per_warp);
}

size_t plain_smem_bytes(const DevPlan& p, uint32_t kmax, bool fp64) {
  return plain_layout(p, kmax, fp64 ? 16 : 8).total;
}

// Raise every kernel's dynamic shared-memory limit once (host call, outside
// any stream capture); launches then only enqueue.
cudaError_t set_smem_limits() {
  static bool done = false;
  if (done) return cudaSuccess;
  const int lim = 227 * 1024;
  const void* fns[] = {sign_kernel_fn(),
                       (const void*)dense_kernel<float, 1>, (const void*)dense_kernel<double, 1>,
                       (const void*)dense_kernel<float, 2>, (const void*)dense_kernel<double, 2>,
                       (const void*)dense_pc_kernel<float>, (const void*)dense_pc_kernel<double>,
                       (const void*)dense_pc_cta_kernel<float>, (const void*)dense_pc_cta_kernel<double>,
                       (const void*)dense_reg_kernel<float, 1, kRegSetsF32>,
                       (const void*)dense_reg_kernel<float, 2, kRegSetsF32>,
                       (const void*)dense_reg_kernel<float, 3, kRegSetsF32>,
                       (const void*)dense_reg_kernel<float, 4, kRegSetsF32>,
                       (const void*)dense_reg_kernel<float, 5, kRegSetsF32>, (const void*)dense_reg_kernel<double, 1, 1>,
                       (const void*)dense_reg_kernel<double, 2, 1>, (const void*)dense_reg_kernel<double, 3, 1>,
                       (const void*)dense_reg_kernel<double, 4, 1>, (const void*)dense_reg_kernel<double, 5, 1>,
                       (const void*)dense_cta_kernel<float>, (const void*)dense_cta_kernel<double>,
                       (const void*)plain_kernel<float>, (const void*)plain_kernel<double>};
  for (const void* f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e != cudaSuccess) return e;
  }
  done = true;
  return cudaSuccess;
}

cudaError_t launch_plain(const PlainArgs& a, bool fp64, int grid, cudaStream_t st) {
  const size_t smem = plain_smem_bytes(a.p, a.kmax, fp64);
  if (fp64) plain_kernel<double><<<grid, kPlainThreads, smem, st>>>(a);
  else plain_kernel<float><<<grid, kPlainThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalArgs& a, cudaStream_t st) {
  // one thread per 64-shot word; small CTAs spread the words over every SM
  int threads = 64;
  uint64_t blocks = (a.W + threads - 1) / threads;
  if (blocks > 65535) blocks = 65535;
  if (blocks == 0) blocks = 1;
  finalize_kernel<<<(unsigned)blocks, threads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_count(const CountArgs& a, int sm_count, cudaStream_t st) {
  const int threads = 256;
  uint64_t blocks = (a.W + threads - 1) / threads;
  const uint64_t cap = static_cast<uint64_t>(sm_count > 0 ? sm_count : 1) * 4;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  count_kernel<<<(unsigned)blocks, threads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace symft
