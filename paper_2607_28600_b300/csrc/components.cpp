// Adaptive product-component representation (Sec. 6): a deterministic pass
// over the planned dense instruction stream that finds the exact product
// structure of the active coefficient tensor.  Each independent component is
// one small dense vector; a PromoteRot opens a new one-coordinate component
// (its update c a_x, -i sg s a_x is a Kronecker factor (c, -i sg s)); an
// instruction whose support (the coordinates of its masks a and b) lies in one
// component updates that component alone; one whose support spans several
// first merges them by an exact Kronecker product.  Components are never split
// again, except that a measurement removes its pivot coordinate, and a
// component left with no coordinate is a global phase and is dropped.  The
// local masks, pivots, merge schedule and a static placement of the
// components in one per-shot workspace are computed here once for all shots.
#include <algorithm>
#include <map>
#include <vector>

#include "internal.hpp"

namespace symft {

namespace {

// First-fit placement of power-of-two regions in an amplitude address space.
struct Placer {
  std::map<uint32_t, uint32_t> free_;   // offset -> length
  uint32_t end = 0, peak = 0;
  uint32_t alloc(uint32_t n) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        const uint32_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > n) free_[off + n] = len - n;
        return off;
      }
    }
    const uint32_t off = end;
    end += n;
    peak = std::max(peak, end);
    return off;
  }
  void release(uint32_t off, uint32_t n) {
    if (n == 0) return;
    auto it = free_.emplace(off, n).first;
    // merge with the next and previous free ranges
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
        it = pv;
      }
    }
    if (it->first + it->second == end) {
      end = it->first;
      free_.erase(it);
    }
  }
};

struct Comp {
  std::vector<uint32_t> coords;   // local bit i <-> active coordinate coords[i]
  uint32_t off = 0;
  bool live = false;
};

}  // namespace

PCProgram build_product_components(const std::vector<DenseInstr>& dense, uint32_t k_max) {
  PCProgram P;
  std::vector<Comp> comps;
  std::vector<int> comp_of;          // active coordinate -> component
  Placer pl;
  uint64_t work_pc = 0, work_mono = 0;
  auto local_mask = [&](const Comp& c, uint32_t m) {
    uint32_t r = 0;
    for (size_t i = 0; i < c.coords.size(); ++i)
      if ((m >> c.coords[i]) & 1u) r |= 1u << i;
    return r;
  };
  // merge every component touched by mask m into one; returns its index
  auto merge_support = [&](uint32_t g, uint32_t m) -> int {
    std::vector<int> touched;
    for (uint32_t j = 0; m >> j; ++j)
      if ((m >> j) & 1u) {
        const int c = comp_of[j];
        if (std::find(touched.begin(), touched.end(), c) == touched.end()) touched.push_back(c);
      }
    std::sort(touched.begin(), touched.end());
    int cur = touched[0];
    for (size_t t = 1; t < touched.size(); ++t) {
      Comp& A = comps[cur];
      Comp& B = comps[touched[t]];
      const uint32_t kA = static_cast<uint32_t>(A.coords.size()), kB = static_cast<uint32_t>(B.coords.size());
      Comp C;
      C.coords = A.coords;
      C.coords.insert(C.coords.end(), B.coords.begin(), B.coords.end());
      C.off = pl.alloc(1u << (kA + kB));
      C.live = true;
      PCOp op{};
      op.op = PC_MERGE;
      op.g = g;
      op.off = C.off;
      op.offA = A.off;
      op.kA = kA;
      op.offB = B.off;
      op.kB = kB;
      P.ops.push_back(op);
      work_pc += 1ull << (kA + kB);
      pl.release(A.off, 1u << kA);
      pl.release(B.off, 1u << kB);
      A.live = B.live = false;
      comps.push_back(C);
      const int ci = static_cast<int>(comps.size()) - 1;
      for (uint32_t j : comps[ci].coords) comp_of[j] = ci;
      cur = ci;
    }
    return cur;
  };
  for (uint32_t g = 0; g < dense.size(); ++g) {
    const DenseInstr& I = dense[g];
    work_mono += 1ull << I.k;
    if (I.kind == I_PROMOTE_ROT) {
      Comp c;
      c.coords = {static_cast<uint32_t>(I.k)};
      c.off = pl.alloc(2);
      c.live = true;
      comps.push_back(c);
      comp_of.push_back(static_cast<int>(comps.size()) - 1);
      PCOp op{};
      op.op = PC_INIT;
      op.g = g;
      op.off = c.off;
      op.k = 0;
      P.ops.push_back(op);
      work_pc += 1;
      continue;
    }
    const uint32_t support = I.a | I.b | (I.kind >= I_ACTIVE_DIAG_MEAS ? (1u << I.h) : 0u);
    const int ci = merge_support(g, support);
    Comp& C = comps[ci];
    const uint32_t kc = static_cast<uint32_t>(C.coords.size());
    PCOp op{};
    op.op = PC_APPLY;
    op.g = g;
    op.off = C.off;
    op.k = kc;
    op.a = local_mask(C, I.a);
    op.b = local_mask(C, I.b);
    op.h = 0;
    op.out = C.off;
    work_pc += 1ull << kc;
    if (I.kind == I_ACTIVE_DIAG_MEAS || I.kind == I_ACTIVE_PAIR_MEAS) {
      const auto hp = std::find(C.coords.begin(), C.coords.end(), static_cast<uint32_t>(I.h));
      op.h = static_cast<int>(hp - C.coords.begin());
      // The compaction removes the pivot's local bit.  In place it reads every
      // source at or above its destination only when the pivot is the highest
      // local bit of a (the planner's choice in the monolithic order); a pair
      // measurement whose pivot landed lower in the component writes its kept
      // half to a fresh region instead.
      const bool fresh = I.kind == I_ACTIVE_PAIR_MEAS && op.h != 31 - __builtin_clz(op.a);
      if (fresh) {
        op.out = pl.alloc(1u << (kc - 1));
        pl.release(C.off, 1u << kc);
        C.off = op.out;
      } else {
        op.out = C.off;
        pl.release(C.off + (1u << (kc - 1)), 1u << (kc - 1));
      }
      P.ops.push_back(op);
      // a component left without coordinates is a global phase
      C.coords.erase(hp);
      if (C.coords.empty()) {
        pl.release(C.off, 1);
        C.live = false;
      }
      // the planner retires coordinate h: the coordinates above it move down
      comp_of.erase(comp_of.begin() + I.h);
      for (Comp& x : comps)
        if (x.live)
          for (uint32_t& j : x.coords)
            if (j > static_cast<uint32_t>(I.h)) --j;
    } else {
      P.ops.push_back(op);
    }
  }
  P.capacity = std::max<uint32_t>(pl.peak, 1);
  P.work_pc = work_pc;
  P.work_mono = work_mono;
  // used only when it clearly pays: at most half the monolithic vector work,
  // and only where the monolithic vector would not be register-resident (a
  // warp holds k <= 5 in registers, faster than any shared-memory workspace)
  P.use = k_max > 5 && work_pc * 2 <= work_mono;
  return P;
}

}  // namespace symft
