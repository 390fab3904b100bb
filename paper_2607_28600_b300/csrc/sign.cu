// Bit-packed sign kernel (Sec. 6, sampling of the independent symbols, run for
// 512 shots per CTA iteration): draws the noise of every channel and the
// random-measurement bits from the counter-based streams, scatters them into
// the bit-packed record / dense-sign accumulators held in shared memory (64
// shots per word), resolves the record chains and gathers detectors and
// observables, and writes the columns out.  This is the exogenous part of
// every affine sign.
#include <cuda_runtime.h>

#include <cstdint>

#include "device.cuh"

namespace symft {

namespace {

constexpr int kQueue = 96;          // per-warp ring of fire states (< 32 + 64 live)
constexpr int kSignWarps = 8;       // warps per CTA

// smallest j in [0, kNoiseBlock) with u < theta[j], for a u below
// theta[kNoiseBlock-1]: the lane-search bucket of u (plan_dev.hpp, kQBuckets)
// gives the first lane u can fire at, and exact integer comparisons step up
// from there, so the result is the threshold table's own answer
__device__ __forceinline__ int first_above(const uint32_t* th, const uint16_t* bk, uint32_t sh, uint32_t u) {
  int j = bk[u >> sh];
  while (j < kNoiseBlock - 1 && u >= th[j]) ++j;
  return j;
}

// x mod kQueue for x < 2 kQueue (every ring index sum below stays under that:
// qh < kQueue, at most 64 entries live after a drain, lane / popc <= 32)
__device__ __forceinline__ uint32_t ring(uint32_t x) { return x >= (uint32_t)kQueue ? x - kQueue : x; }

// XOR `bit` into word `wb` of the first n (<= 7) slots of a cell target entry
__device__ __forceinline__ void scatter7(uint32_t* sw, uint4 tg, uint32_t n, uint32_t wb, uint32_t bit) {
  const uint32_t f[7] = {tg.x >> 16, tg.y & 0xFFFFu, tg.y >> 16, tg.z & 0xFFFFu, tg.z >> 16,
                         tg.w & 0xFFFFu, tg.w >> 16};
#pragma unroll
  for (uint32_t k = 0; k < 7; ++k) {
    if (k >= n) break;
    atomicXor(sw + f[k] + wb, bit);
  }
}

// 128-lane sub-blocks of a noise block; a slot holds one uint4 per sub-block
constexpr int kSub = kNoiseBlock / 128;
// a chain path's record ids are two 16-byte items of eight 32-bit words
static_assert(kMaxLevels == 16, "the path walk reads 16 record ids per path");

// This thread's 16-byte column pieces in a noise block: sub-block t % kSub of
// every (blockDim / kSub)-th column, so consecutive threads cover consecutive
// pieces of one column and the padding masks are per thread.  Full pieces
// (both words hold only real shots, W even and the array 16-byte aligned, so
// every piece is too) are one 16-byte store; the request's last piece is
// masked.
struct Piece {
  uint32_t b;          // sub-block
  uint64_t wa;         // first 64-shot word of the piece
  bool live, full, hb; // real shots in the piece; unmasked store; second word exists
  uint64_t m0, m1;     // padding masks of the two words
  __device__ __forceinline__ void put(uint64_t* d, uint4 v, bool al) const {
    if (full && al) {
      *reinterpret_cast<uint4*>(d) = v;
    } else {
      d[0] = (((uint64_t)v.y << 32) | v.x) & m0;
      if (hb) d[1] = (((uint64_t)v.w << 32) | v.z) & m1;
    }
  }
};

__device__ __forceinline__ Piece piece_of(const SignArgs& A, uint64_t sub0, uint32_t nsub) {
  Piece p;
  p.b = threadIdx.x % kSub;
  p.wa = 2 * (sub0 + p.b);
  p.live = p.b < nsub;
  p.full = 64 * (p.wa + 2) <= A.shots && (A.W & 1) == 0;
  const uint64_t la = p.live ? A.shots - 64 * p.wa : 0;   // shots in word wa (>= 1 when live)
  p.m0 = la < 64 ? (1ull << la) - 1 : ~0ull;
  p.hb = p.wa + 1 < A.W;
  const uint64_t lb = p.hb ? A.shots - 64 * (p.wa + 1) : 0;
  p.m1 = !p.hb ? 0ull : (lb < 64 ? (1ull << lb) - 1 : ~0ull);
  return p;
}

// column piece of detector / observable j (null when the caller skipped it)
__device__ __forceinline__ uint64_t* out_col(const SignArgs& A, const Piece& p, uint32_t j, bool& al) {
  const uint32_t ND = A.p.n_dets;
  if (j < ND) {
    al = (reinterpret_cast<uintptr_t>(A.det) & 15) == 0;
    return A.det ? A.det + (uint64_t)j * A.W + p.wa : nullptr;
  }
  al = (reinterpret_cast<uintptr_t>(A.obs) & 15) == 0;
  return A.obs ? A.obs + (uint64_t)(j - ND) * A.W + p.wa : nullptr;
}

struct SignLayout {
  size_t q_off, qs_off, qk_off, c_off, slot_off, qa_off, qb_off, cnt_off, total;
};

__host__ __device__ inline SignLayout sign_layout(uint32_t n_qtab, uint32_t n_ctab, uint32_t n_slots) {
  SignLayout L;
  L.q_off = 0;
  L.qs_off = align16((size_t)n_qtab * kNoiseBlock * 4);
  L.qk_off = L.qs_off + align16((size_t)n_qtab * 4);
  L.c_off = L.qk_off + align16((size_t)n_qtab * kQBuckets * 2);
  L.slot_off = L.c_off + align16((size_t)n_ctab * sizeof(CellTableDev));
  L.qa_off = L.slot_off + (size_t)n_slots * kSub * 16;
  L.qb_off = L.qa_off + (size_t)kSignWarps * kQueue * 16;
  L.cnt_off = L.qb_off + (size_t)kSignWarps * kQueue * 4;
  L.total = L.cnt_off + 64;
  return L;
}

}  // namespace

// One CTA iteration samples one noise block (kNoiseBlock = 512 consecutive
// shots, 8 words of 64 shots per column).  Shared memory: the noise tables,
// then
//   slots  n_slots x kSub x uint4  (lane l: bit l&31 of word l>>5 of the slot)
//   queue  kSignWarps x kQueue x {uint4 (c, u, L | draw << 9, qtab | ctab << 16),
//                                 uint32 first (channel, cell) target entry}
__global__ void __launch_bounds__(kSignWarps * 32, 5) sign_kernel(SignArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const uint32_t NT = A.p.n_slots;
  const SignLayout Lay = sign_layout(A.p.n_qtab, A.p.n_ctab, NT);
  uint32_t* sq = reinterpret_cast<uint32_t*>(smem_raw + Lay.q_off);
  uint32_t* sqs = reinterpret_cast<uint32_t*>(smem_raw + Lay.qs_off);
  uint16_t* sqb = reinterpret_cast<uint16_t*>(smem_raw + Lay.qk_off);
  CellTableDev* sc = reinterpret_cast<CellTableDev*>(smem_raw + Lay.c_off);
  uint4* slots = reinterpret_cast<uint4*>(smem_raw + Lay.slot_off);
  uint4* qa = reinterpret_cast<uint4*>(smem_raw + Lay.qa_off) + warp * kQueue;
  uint32_t* qb = reinterpret_cast<uint32_t*>(smem_raw + Lay.qb_off) + warp * kQueue;
  uint32_t* sqn = reinterpret_cast<uint32_t*>(smem_raw + Lay.cnt_off);

  for (uint32_t i = threadIdx.x; i < A.p.n_qtab * kNoiseBlock; i += blockDim.x) sq[i] = __ldg(A.p.qtheta + i);
  for (uint32_t i = threadIdx.x; i < A.p.n_qtab; i += blockDim.x) sqs[i] = __ldg(A.p.qshift + i);
  for (uint32_t i = threadIdx.x; i < A.p.n_qtab * kQBuckets; i += blockDim.x) sqb[i] = __ldg(A.p.qstart + i);
  for (uint32_t i = threadIdx.x; i < A.p.n_ctab; i += blockDim.x) sc[i] = A.p.ctabs[i];
  __syncthreads();

  const uint32_t n_groups = (A.p.n_channels + 3) >> 2;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint32_t R = A.p.n_records;
  uint32_t* sw = reinterpret_cast<uint32_t*>(slots);

  for (uint64_t blk = blockIdx.x; blk < A.n_blocks; blk += gridDim.x) {
    const uint32_t gblk = (uint32_t)(A.block0 + blk);      // global noise block
    const uint64_t sub0 = blk * kSub;                       // local 128-shot sub-block
    const uint32_t nsub = (uint32_t)min((uint64_t)kSub, (A.shots + 127) / 128 - sub0);
    // 1+2. constants and random-measurement bits m1: one Philox block = the
    //    128 bits of a sub-block (64-shot words 2s and 2s+1 of global
    //    sub-block s).  With few m1 symbols their words are staged in the
    //    (still unused) queue area and every slot gathers its own sources;
    //    otherwise the words are scattered into the slots with atomics.
    if ((size_t)A.p.n_m1 * kSub * 16 <= (size_t)kSignWarps * kQueue * 16) {
      // every slot starts at zero; the slots with a constant or random
      // sources are then set from their items
      for (uint32_t i = threadIdx.x; i < NT * kSub; i += blockDim.x) slots[i] = make_uint4(0u, 0u, 0u, 0u);
      uint4* mw = reinterpret_cast<uint4*>(smem_raw + Lay.qa_off);    // [n_m1][kSub]
      for (uint32_t it = threadIdx.x; it < nsub * A.p.n_m1; it += blockDim.x) {
        const uint32_t b = it / A.p.n_m1, j = it - b * A.p.n_m1;
        const uint64_t gs = (uint64_t)gblk * kSub + b;
        mw[j * kSub + b] = philox(make_uint4(__ldg(A.p.m1_t + j), (uint32_t)gs, (uint32_t)(gs >> 32), kTagMbit), A.keys);
      }
      __syncthreads();
      for (uint32_t x = threadIdx.x; x < A.p.n_slot_nz * kSub; x += blockDim.x) {
        const uint32_t b = x % kSub;
        const uint32_t i = __ldg(A.p.slot_nz + x / kSub) * kSub + b;
        const uint4 e = __ldg(A.p.slot_m1 + i / kSub);
        const uint32_t c = (e.x & 0x8000u) ? ~0u : 0u;
        uint4 v = make_uint4(c, c, c, c);
        const uint32_t n = e.x & 0x7FFFu;
        if (b < nsub) {
          if (n == 0x7FFFu) {
            for (uint32_t q = e.y; q < e.y + e.z; ++q) v = xor4(v, mw[__ldg(A.p.slot_m1_ovf + q) * kSub + b]);
          } else {
            const uint32_t f[7] = {e.x >> 16, e.y & 0xFFFFu, e.y >> 16, e.z & 0xFFFFu, e.z >> 16,
                                   e.w & 0xFFFFu, e.w >> 16};
#pragma unroll
            for (uint32_t k = 0; k < 7; ++k) {
              if (k >= n) break;
              v = xor4(v, mw[f[k] * kSub + b]);
            }
          }
        }
        slots[i] = v;
      }
      __syncthreads();
    } else {
      for (uint32_t i = threadIdx.x; i < NT * kSub; i += blockDim.x) {
        const uint32_t v = A.p.slot_const[i / kSub] ? ~0u : 0u;
        slots[i] = make_uint4(v, v, v, v);
      }
      __syncthreads();
      for (uint32_t it = threadIdx.x; it < nsub * A.p.n_m1; it += blockDim.x) {
        const uint32_t b = it / A.p.n_m1, j = it - b * A.p.n_m1;
        const uint64_t gs = (uint64_t)gblk * kSub + b;
        const uint4 o = philox(make_uint4(__ldg(A.p.m1_t + j), (uint32_t)gs, (uint32_t)(gs >> 32), kTagMbit), A.keys);
        const uint32_t e = __ldg(A.p.m1_off + j + 1);
        for (uint32_t q = __ldg(A.p.m1_off + j); q < e; ++q) {
          uint32_t* t = reinterpret_cast<uint32_t*>(slots + (size_t)__ldg(A.p.m1_tgt + q) * kSub + b);
          atomicXor(t + 0, o.x);
          atomicXor(t + 1, o.y);
          atomicXor(t + 2, o.z);
          atomicXor(t + 3, o.w);
        }
      }
    }
    // 3. noise.  Phase A: each lane draws the head uniforms of four channels
    //    (one Philox block) and queues the channels that fire in this block.
    //    Phase B: each lane takes one queued (channel, u, L, draw index) state,
    //    resolves exactly one fire -- lane L + j*, its Pauli cell and the
    //    scatter of its components -- and re-queues the channel if its
    //    block-geometric process continues, so every step costs the same.
    uint32_t qn = 0, qh = 0;     // ring buffer: entries (qh + i) % kQueue, i < qn
    // Resolve the fire of one queued state (whose uniform is known to fire):
    // its Pauli cell (whose target entry is loaded right away, so the load is
    // in flight during the lane search and the re-queue), its lane, and the
    // word and bit that scatter() XORs into the entry's slots.  The next
    // uniform is tested here; returns true (and the next state) only if the
    // channel fires again.
    auto fire_step = [&](uint4 ent, uint32_t cell0, uint4& next, uint4& tg, uint32_t& wb, uint32_t& bit) -> bool {
      const uint32_t c = ent.x;
      const int L = (int)(ent.z & 0x1FFu);
      uint32_t ti = ent.z >> 9;
      const uint32_t qt = ent.w & 0xFFFFu;
      const CellTableDev* ct = sc + (ent.w >> 16);
      const uint32_t ncell = ct->ncell;
      // the draws of one fire (cell, next u) lie in one Philox block
      const uint4 tail = philox(make_uint4(c, gblk, ti >> 2, kTagTail), A.keys);
      uint32_t cell = 0;
      if (ncell > 1) {
        const uint32_t v = pick(tail, ti & 3);
        ++ti;
        // min{k : v < phi_k}: equal-weight guess, then exact correction
        int cc = (int)(((uint64_t)v * ncell) >> 32);
        while (cc > 0 && v < ct->phi[cc - 1]) --cc;
        while (cc < (int)ncell - 1 && v >= ct->phi[cc]) ++cc;
        cell = (uint32_t)cc;
      }
      tg = __ldg(A.p.cellt + cell0 + cell);
      const uint32_t* th = sq + (size_t)qt * kNoiseBlock;
      const int lanebit = L + first_above(th, sqb + qt * kQBuckets, sqs[qt], ent.y);   // <= kNoiseBlock-1 by construction
      const uint32_t u2 = pick(tail, ti & 3);        // next uniform, draw index ti
      wb = (uint32_t)lanebit >> 5;                   // word offset inside a slot
      bit = 1u << (lanebit & 31);
      if (lanebit >= kNoiseBlock - 1) return false;
      const int L2 = lanebit + 1;
      if (u2 >= th[kNoiseBlock - 1 - L2]) return false;   // no further fire in lanes L2..end
      next = make_uint4(c, u2, (uint32_t)L2 | ((ti + 1) << 9), ent.w);
      return true;
    };
    auto scatter = [&](uint4 tg, uint32_t wb, uint32_t bit) {
      const uint32_t ntg = tg.x & 0xFFFFu;
      if (ntg == 0xFFFFu) {
        for (uint32_t q = tg.y; q < tg.y + tg.z; ++q) atomicXor(sw + __ldg(A.p.cell_ovf + q) + wb, bit);
      } else {
        scatter7(sw, tg, ntg, wb, bit);
      }
    };
    // full-warp drain of the 32 oldest queued states; continuing channels are
    // re-queued at the back of the ring
    auto drain32 = [&]() {
      const uint32_t src = ring(qh + lane);
      const uint4 ent = qa[src];
      const uint32_t cell0 = qb[src];
      __syncwarp();
      qh = ring(qh + 32);
      qn -= 32;
      uint4 next = make_uint4(0u, 0u, 0u, 0u), tg;
      uint32_t wb, bit;
      const bool more = fire_step(ent, cell0, next, tg, wb, bit);
      const uint32_t bal = __ballot_sync(0xffffffffu, more);
      if (more) {
        const uint32_t pos = ring(qh + qn + __popc(bal & lt_mask));
        qa[pos] = next;
        qb[pos] = cell0;
      }
      qn += __popc(bal);
      scatter(tg, wb, bit);
      __syncwarp();
    };
    for (uint32_t base = warp * 32; base < n_groups; base += kSignWarps * 32) {
      const uint32_t g = base + lane;
      const bool valid = g < n_groups;
      uint4 head = make_uint4(0u, 0u, 0u, 0u), th4 = make_uint4(0u, 0u, 0u, 0u);
      if (valid) {
        th4 = __ldg(A.p.theta4 + g);
        if (th4.x | th4.y | th4.z | th4.w)
          head = philox(make_uint4(g, gblk, 0u, kTagHead), A.keys);
      }
      // queue the firing channels, two channel slots at a time (<= 64 new states)
#pragma unroll
      for (uint32_t h2 = 0; h2 < 4; h2 += 2) {
        const bool f0 = valid && pick(head, h2) < pick(th4, h2);
        const bool f1 = valid && pick(head, h2 + 1) < pick(th4, h2 + 1);
        const uint32_t b0m = __ballot_sync(0xffffffffu, f0), b1m = __ballot_sync(0xffffffffu, f1);
        if (b0m | b1m) {
          // slot order: lane-major pairs; position = entries of lower lanes + own
          const uint32_t lower = __popc(b0m & lt_mask) + __popc(b1m & lt_mask);
          uint32_t pos = ring(qh + qn + lower);
          if (f0) {
            const uint32_t c = 4 * g + h2;
            const uint4 raw = __ldg(reinterpret_cast<const uint4*>(A.p.ch) + c);
            qa[pos] = make_uint4(c, pick(head, h2), 0u, raw.y);
            qb[pos] = raw.w;
            pos = pos + 1 == kQueue ? 0 : pos + 1;
          }
          if (f1) {
            const uint32_t c = 4 * g + h2 + 1;
            const uint4 raw = __ldg(reinterpret_cast<const uint4*>(A.p.ch) + c);
            qa[pos] = make_uint4(c, pick(head, h2 + 1), 0u, raw.y);
            qb[pos] = raw.w;
          }
          qn += __popc(b0m) + __popc(b1m);
          __syncwarp();
          while (qn >= 32) drain32();
        }
      }
    }
    // pool the leftover states of all warps and finish each channel in one
    // thread (few continue past one more fire)
    __syncthreads();
    if (lane == 0) sqn[warp] = qn;
    __syncthreads();
    uint32_t off = 0, total = 0;
    for (int w2 = 0; w2 < kSignWarps; ++w2) {
      const uint32_t n2 = sqn[w2];
      if (w2 < warp) off += n2;
      total += n2;
    }
    // gather into the pool area (the queues of all warps, read before written)
    uint4 mine = make_uint4(0u, 0u, 0u, 0u);
    uint32_t mineb = 0;
    if ((uint32_t)lane < qn) {
      mine = qa[ring(qh + lane)];
      mineb = qb[ring(qh + lane)];
    }
    __syncthreads();
    uint4* pool_a = reinterpret_cast<uint4*>(smem_raw + Lay.qa_off);
    uint32_t* pool_b = reinterpret_cast<uint32_t*>(smem_raw + Lay.qb_off);
    if ((uint32_t)lane < qn) {
      pool_a[off + lane] = mine;
      pool_b[off + lane] = mineb;
    }
    __syncthreads();
    for (uint32_t x = threadIdx.x; x < total; x += blockDim.x) {
      uint4 ent = pool_a[x];
      const uint32_t cell0 = pool_b[x];
      for (int guard = 0; guard < kNoiseBlock; ++guard) {
        uint4 next, tg;
        uint32_t wb, bit;
        const bool more = fire_step(ent, cell0, next, tg, wb, bit);
        scatter(tg, wb, bit);
        if (!more) break;
        ent = next;
      }
    }
    __syncthreads();
    const uint32_t step = blockDim.x / kSub;
    const uint32_t i0 = threadIdx.x / kSub;
    // 4. detectors and observables that equal one slot before the chains
    {
      const Piece pc = piece_of(A, sub0, nsub);
      if (pc.live && (A.det || A.obs)) {
        for (uint32_t x = i0; x < A.p.n_out_delta; x += step) {
          const uint2 e = __ldg(A.p.out_delta + x);
          bool al;
          uint64_t* d = out_col(A, pc, e.x, al);
          if (d) pc.put(d, slots[(size_t)e.y * kSub + pc.b], al);
        }
      }
    }
    __syncthreads();
    // 5. records: each chain path walked by one thread per sub-block, no
    //    barrier between its records (exo_r = delta_r ^ exo_parent)
    //    The path's record ids (two 16-byte items) are loaded up front.
    for (uint32_t x = threadIdx.x; x < A.p.n_paths * kSub; x += blockDim.x) {
      const uint4 w0 = __ldg(A.p.path_ids + 2 * (x / kSub)), w1 = __ldg(A.p.path_ids + 2 * (x / kSub) + 1);
      const uint32_t f[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
      const uint32_t bb = x % kSub;
      uint4 acc = slots[(size_t)(f[0] & 0xFFFFu) * kSub + bb];
#pragma unroll
      for (int i = 1; i < kMaxLevels; ++i) {
        const uint32_t id = (i & 1) ? (f[i >> 1] >> 16) : (f[i >> 1] & 0xFFFFu);
        if (id == 0xFFFFu) break;
        uint4* sl = slots + (size_t)id * kSub + bb;
        acc = xor4(acc, *sl);
        *sl = acc;
      }
    }
    __syncthreads();
    // 6. write the records, the gathered detectors / observables (XOR of
    //    records) and the dense signs
    const Piece pc = piece_of(A, sub0, nsub);
    const uint32_t b = pc.b;
    const uint64_t wa = pc.wa;
    if (pc.live) {
      const uint64_t cstep = (uint64_t)step * A.W;
      if (A.meas) {
        uint64_t* d = A.meas + (uint64_t)i0 * A.W + wa;
        const uint4* sl = slots + (size_t)i0 * kSub + b;
        const bool al = ((reinterpret_cast<uintptr_t>(A.meas) & 15) == 0);
        for (uint32_t i = i0; i < R; i += step, d += cstep, sl += (size_t)step * kSub) pc.put(d, *sl, al);
      }
      auto gather = [&](uint32_t j) {
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        const uint4 gi = __ldg(A.p.gat_item + j);
        const uint32_t n = gi.x & 0xFFFFu;
        if (n == 0xFFFFu) {
          for (uint32_t q = gi.y; q < gi.y + gi.z; ++q) v = xor4(v, slots[__ldg(A.p.gat_ovf + q) * kSub + b]);
        } else {
          const uint32_t f[7] = {gi.x >> 16, gi.y & 0xFFFFu, gi.y >> 16, gi.z & 0xFFFFu, gi.z >> 16,
                                 gi.w & 0xFFFFu, gi.w >> 16};
#pragma unroll
          for (uint32_t k = 0; k < 7; ++k) {
            if (k >= n) break;
            v = xor4(v, slots[f[k] * kSub + b]);
          }
        }
        return v;
      };
      if (A.det || A.obs) {
        for (uint32_t x = i0; x < A.p.n_out_rest; x += step) {
          const uint32_t j = __ldg(A.p.out_rest + x);
          bool al;
          uint64_t* d = out_col(A, pc, j, al);
          if (d) pc.put(d, gather(j), al);
        }
      }
      if (A.signs) {
        uint64_t* d = A.signs + (uint64_t)i0 * A.W + wa;
        const bool al = ((reinterpret_cast<uintptr_t>(A.signs) & 15) == 0);
        for (uint32_t g = i0; g < NT - R; g += step, d += cstep) pc.put(d, slots[(size_t)(R + g) * kSub + b], al);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// launch wrappers (host)
// ---------------------------------------------------------------------------
cudaError_t set_smem_limits();

const void* sign_kernel_fn() { return (const void*)sign_kernel; }

size_t sign_smem_bytes(const DevPlan& p) { return sign_layout(p.n_qtab, p.n_ctab, p.n_slots).total; }

cudaError_t sign_occupancy(const DevPlan& p, int* ctas_per_sm) {
  const size_t smem = sign_smem_bytes(p);
  cudaError_t e = set_smem_limits();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute((const void*)sign_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, sign_kernel, kSignWarps * 32, smem);
}

cudaError_t launch_sign(const SignArgs& a, int grid, cudaStream_t st) {
  sign_kernel<<<grid, kSignWarps * 32, sign_smem_bytes(a.p), st>>>(a);
  return cudaGetLastError();
}

}  // namespace symft
