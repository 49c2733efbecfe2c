// color_device.cuh -- device side of the ordered coloring (Sec. III-B static
// Random order, first fit), shared by the per-round kernel and the
// small-round engine.  Internal header of the CUDA library.
#pragma once

#include "common.cuh"

namespace picasso {

// Publish a new state word (the low half of the 64-bit state; the priority
// in the high half never changes).
__device__ __forceinline__ void publish(uint64_t* state, int32_t v, uint32_t w) {
  __stcg(reinterpret_cast<uint32_t*>(state + v), w);
}

// ---------------------------------------------------------------------------
// Ordered persistent coloring.  `order` lists the round's vertices in exact
// coloring order; warp w takes positions w, w + W, w + 2W, ... (W = warps in
// the grid).  A vertex that has to wait polls the neighbour holding it up
// instead of leaving for a later sweep.  No deadlock: the earliest unfinished
// position's warp is working on it (all its earlier positions are done), and
// that vertex waits only on earlier positions, which are finished; the
// cooperative launch guarantees every warp is resident.  A poll budget
// bounds every wait (a.max_polls polls; the context's wait_polls, by default
// kMaxPolls): when it runs out the kernel sets *err = 1 and the warp returns;
// the caller then recolors the round with the sweep kernel.
// ---------------------------------------------------------------------------

constexpr int kOrderedGroup = 2;  // run chunks of 32 whose loads are in flight together

// Loads of the conflict structure (read-only while the coloring runs):
// through the read-only cache when earlier launches built it; plain loads
// when it was written earlier in the same launch (FRESH, the small-round
// engine), where the read-only path may hold lines from before the write
// and the grid barrier orders plain loads after the writes.
template <bool FRESH, class T>
__device__ __forceinline__ T ld_run(const T* p) {
  if (FRESH) return *p;
  return __ldg(p);
}
constexpr int kListBatch = 32 / kClistWords;   // candidates checked against their lists together
constexpr int kClistSlots = kClistWords - 1;   // colored vertices a list records per color

// Scan the run [rs, rs + ntot) of candidate c to the end: true if an earlier
// neighbour took c; waits (bounded) on earlier neighbours still undecided at
// or below c.  *fail is set when a wait runs out.
template <bool FRESH>
__device__ __forceinline__ bool run_blocked(const ColorArgs& a, int32_t v, uint32_t pv, uint32_t c, int64_t rs,
                                            int64_t ntot, int lane, int& polls, bool* fail) {
  for (int64_t e0 = 0; e0 < ntot;) {
    int32_t u[kOrderedGroup];
    uint64_t su[kOrderedGroup];
    bool past = false;  // ranked ids: a later neighbour ends the prefix
#pragma unroll
    for (int j = 0; j < kOrderedGroup; ++j) {
      const int64_t e = e0 + 32 * j + lane;
      u[j] = e < ntot ? ld_run<FRESH>(a.col + rs + e) : -1;
      if (a.ranked && u[j] > v) {
        u[j] = -1;
        past = true;
      }
    }
#pragma unroll
    for (int j = 0; j < kOrderedGroup; ++j) su[j] = u[j] >= 0 ? __ldcg(&a.state[u[j]]) : 0ull;
    bool lb = false;
    uint32_t wm[kOrderedGroup];
#pragma unroll
    for (int j = 0; j < kOrderedGroup; ++j) {
      bool lw = false;
      if (u[j] >= 0) {
        const uint32_t pu = (uint32_t)(su[j] >> 32);
        if (a.ranked || pu < pv || (pu == pv && u[j] < v)) {
          const uint32_t wu = (uint32_t)su[j], st = wu & 3u, cu = wu >> 2;
          lb = lb || (st == kColored && cu == c);
          lw = st == kUndecided && cu <= c;
        }
      }
      wm[j] = __ballot_sync(0xffffffffu, lw);
    }
    if (__any_sync(0xffffffffu, lb)) return true;
    int jw = -1;
#pragma unroll
    for (int j = kOrderedGroup - 1; j >= 0; --j)
      if (wm[j]) jw = j;
    if (jw < 0) {
      if (__any_sync(0xffffffffu, past)) return false;
      e0 += 32 * kOrderedGroup;
      continue;
    }
    // wait for the first neighbour holding us up, then rescan from its chunk
    uint32_t m = 0u;
    int32_t uw = -1;
#pragma unroll
    for (int j = 0; j < kOrderedGroup; ++j)
      if (j == jw) {
        m = wm[j];
        uw = u[j];
      }
    const int32_t wu_id = __shfl_sync(0xffffffffu, uw, __ffs(m) - 1);
    while (true) {
      const uint32_t w = (uint32_t)__ldcg(&a.state[wu_id]);
      if ((w & 3u) != kUndecided || (w >> 2) > c) break;
      if (++polls > a.max_polls) {
        *fail = true;
        return true;
      }
      __nanosleep(64);
    }
    e0 += 32 * jw;
  }
  return false;
}

// One vertex.  The run offsets and colors of 32 candidates are loaded at
// once (lane k holds candidate k's).  With colored lists (a.clist),
// kListBatch candidates at a time are first checked against the vertices
// already colored with them: kClistWords lanes per candidate read the
// candidate's list (a count and the ranks of its first kClistSlots colored
// vertices) and test commutation with those ranked before v.  A hit proves the candidate
// blocked (that vertex is an earlier neighbour holding the color); nothing
// else is concluded from the list.  Every candidate not proven blocked, in
// list order, is settled by scanning its whole run (run_blocked), which is
// exact; the first one no earlier neighbour can take is v's color.
template <bool FRESH>
__device__ __forceinline__ bool ordered_vertex(const ColorArgs& a, int32_t v, int lane, int32_t* err) {
  const int64_t row = ld_run<FRESH>(a.loff + v);
  const int L = (int)(ld_run<FRESH>(a.loff + v + 1) - row);
  const uint32_t pv = (uint32_t)(__ldcg(&a.state[v]) >> 32);
  const bool lists = a.clist != nullptr;
  const bool wide = a.qw > 1;  // strings of more than one word per part
  uint64_t xv = 0, zv = 0;
  if (lists && !wide) {
    xv = ld_run<FRESH>(a.xz + 2 * (int64_t)v);
    zv = ld_run<FRESH>(a.xz + 2 * (int64_t)v + 1);
  }
  int polls = 0;
  for (int kb = 0; kb < L; kb += 32) {
    const int kl = kb + lane;
    int64_t my_rs = 0, my_re = 0;
    if (kl < L) {
      my_rs = ld_run<FRESH>(a.runoff + row + kl) - a.cbase;
      my_re = ld_run<FRESH>(a.runoff + row + kl + 1) - a.cbase;
    }
    const uint32_t my_c = kl < L ? (uint32_t)ld_run<FRESH>(a.lists + row + kl) : 0u;
    const int kend = min(L - kb, 32);
    for (int k0 = 0; k0 < kend; k0 += kListBatch) {
      uint32_t proven = 0u;  // bit b: candidate k0 + b is blocked
      if (lists) {
        const int kq = k0 + lane / kClistWords, w = lane % kClistWords;
        const uint32_t cq = __shfl_sync(0xffffffffu, my_c, min(kq, 31));
        const uint32_t word = (kq < kend && w > 0) ? __ldcg(a.clist + (size_t)cq * kClistWords + w) : 0u;
        bool lb = false;
        if (word != 0u && (int32_t)(word - 1) < v) {
          const int64_t u = (int64_t)(word - 1);
          if (wide)
            lb = commuteW(a.xz + 2 * a.qw * (int64_t)v, a.xz + 2 * a.qw * u, a.qw);
          else
            lb = commute1(xv, zv, ld_run<FRESH>(a.xz + 2 * u), ld_run<FRESH>(a.xz + 2 * u + 1));
        }
        const uint32_t bm = __ballot_sync(0xffffffffu, lb);
#pragma unroll
        for (int b = 0; b < kListBatch; ++b)
          if ((bm >> (kClistWords * b)) & ((1u << kClistWords) - 1u)) proven |= 1u << b;
      }
#pragma unroll 1
      for (int b = 0; b < kListBatch; ++b) {
        const int kk = k0 + b;
        if (kk >= kend) break;
        if ((proven >> b) & 1u) continue;
        const uint32_t c = __shfl_sync(0xffffffffu, my_c, kk);
        const int64_t rs = __shfl_sync(0xffffffffu, my_rs, kk);
        const int64_t re = __shfl_sync(0xffffffffu, my_re, kk);
        if (kb + kk > 0 && lane == 0) publish(a.state, v, (c << 2) | kUndecided);
        bool fail = false;
        const bool blk = run_blocked<FRESH>(a, v, pv, c, rs, re - rs, lane, polls, &fail);
        if (fail) {
          if (lane == 0) atomicExch(err, 1);
          return false;
        }
        if (!blk) {
          if (lane == 0) {
            if (lists) {
              const uint32_t slot = atomicAdd(a.clist + (size_t)c * kClistWords, 1u);
              if (slot < (uint32_t)kClistSlots)
                __stcg(a.clist + (size_t)c * kClistWords + 1 + slot, (uint32_t)v + 1u);
            }
            publish(a.state, v, (c << 2) | kColored);
          }
          return true;
        }
      }
    }
  }
  if (lane == 0) publish(a.state, v, (kFailedColor << 2) | kFailed);
  return true;
}


// ---------------------------------------------------------------------------
// Mask coloring (bit layout).  Bucket c keeps two 512-bit masks over its
// member slots: colored (the member took c) and resolved (the member will
// never take c: it passed c or took another color).  For vertex v and its
// candidate c with row bits r (the earlier members of bucket c that commute
// with v):
//   r & colored != 0                 c is taken by an earlier neighbour;
//   r & ~(colored | resolved) == 0   no earlier neighbour can still take c:
//                                    v takes c (first fit);
//   otherwise                        v waits (bounded) for those members.
// A vertex publishes its passes (resolved bits) before it waits and, once
// decided, its color (colored bit) and every other list color (resolved),
// so each bit only ever changes from 0 to 1 and a decision taken from any
// value read is final.  Candidates are examined kMaskCands at a time, four
// lanes per candidate.
// ---------------------------------------------------------------------------
constexpr int kMaskCands = 8;

// Mark list entries [from, to) of v (row = loff[v]) except `skip`: resolved.
// Entries kb .. kb + 31 come from the lanes' registers (lane t holds entry
// kb + t's color c and packed word rb), the others (lists of more than 32
// colors) from memory.
template <bool FRESH>
__device__ __forceinline__ void mask_resolve(const ColorArgs& a, int64_t row, int from, int to, int skip, int lane,
                                             int kb, uint32_t c, int64_t rb) {
  const int t = kb + lane;
  if (t >= from && t < to && t != skip) {
    const int slot = rinfo_slot(rb);
    atomicOr(a.cmask + (size_t)c * 32 + 16 + (slot >> 5), 1u << (slot & 31));
  }
  for (int u = from + lane; u < to; u += 32) {
    if (u == skip || (u >= kb && u < kb + 32)) continue;
    const uint32_t cu = (uint32_t)ld_run<FRESH>(a.lists + row + u);
    const int slot = rinfo_slot(ld_run<FRESH>(a.rinfo + row + u));
    atomicOr(a.cmask + (size_t)cu * 32 + 16 + (slot >> 5), 1u << (slot & 31));
  }
}

// Lane's list entry of v (color and packed word), or 0 past the list: the
// first loads of mask_vertex, which a caller may issue ahead of time.
template <bool FRESH>
__device__ __forceinline__ void mask_entry(const ColorArgs& a, int32_t v, int lane, uint32_t* c, int64_t* rb) {
  const int64_t row = a.Lu ? (int64_t)v * a.Lu : ld_run<FRESH>(a.loff + v);
  const int L = a.Lu ? a.Lu : (int)(ld_run<FRESH>(a.loff + v + 1) - row);
  *c = lane < L ? (uint32_t)ld_run<FRESH>(a.lists + row + lane) : 0u;
  *rb = lane < L ? ld_run<FRESH>(a.rinfo + row + lane) : 0;
}

// pre: c0 / rb0 hold mask_entry(v) (entries 0 .. 31 need no load).
template <bool FRESH>
__device__ __forceinline__ bool mask_vertex(const ColorArgs& a, int32_t v, int lane, int32_t* err, bool pre = false,
                                            uint32_t c0 = 0u, int64_t rb0 = 0) {
  // lists of one length (a single set): the row is known without a load
  const int64_t row = a.Lu ? (int64_t)v * a.Lu : ld_run<FRESH>(a.loff + v);
  const int L = a.Lu ? a.Lu : (int)(ld_run<FRESH>(a.loff + v + 1) - row);
  int polls = 0;
  int kdone = 0;  // entries [0, kdone) passed and marked resolved
  for (int kb = 0; kb < L; kb += 32) {
    const int kl = kb + lane;
    uint32_t my_c = 0u;
    int64_t my_rb = 0;
    if (pre && kb == 0) {
      my_c = c0;
      my_rb = rb0;
    } else if (kl < L) {
      my_c = (uint32_t)ld_run<FRESH>(a.lists + row + kl);
      my_rb = ld_run<FRESH>(a.rinfo + row + kl);
    }
    const int kend = min(L - kb, 32);
    for (int k0 = 0; k0 < kend; k0 += kMaskCands) {
      // lanes 4 j .. 4 j + 3 take candidate k0 + j: lane 4 j + q holds its
      // row words 4 q .. 4 q + 3 and the same words of its bucket's masks
      // (one 16-byte load each)
      const int kq = k0 + (lane >> 2), w0 = 4 * (lane & 3);
      const uint32_t cq = __shfl_sync(0xffffffffu, my_c, min(kq, 31));
      const int64_t rq = __shfl_sync(0xffffffffu, my_rb, min(kq, 31));
      const int nw = kq < kend ? (rinfo_slot(rq) >> 5) + 1 : 0;  // row words
      bool bl = false, pe = false;
      if (w0 < nw) {
        const uint4 tk = __ldcg(reinterpret_cast<const uint4*>(a.cmask + (size_t)cq * 32 + w0));
        const uint4 nv = __ldcg(reinterpret_cast<const uint4*>(a.cmask + (size_t)cq * 32 + 16 + w0));
        const uint32_t* rp = a.rmask + rinfo_addr(rq) + w0;
        const int m = nw - w0;
        const uint32_t r0 = ld_run<FRESH>(rp);
        const uint32_t r1 = m > 1 ? ld_run<FRESH>(rp + 1) : 0u;
        const uint32_t r2 = m > 2 ? ld_run<FRESH>(rp + 2) : 0u;
        const uint32_t r3 = m > 3 ? ld_run<FRESH>(rp + 3) : 0u;
        bl = ((r0 & tk.x) | (r1 & tk.y) | (r2 & tk.z) | (r3 & tk.w)) != 0u;
        pe = ((r0 & ~(tk.x | nv.x)) | (r1 & ~(tk.y | nv.y)) | (r2 & ~(tk.z | nv.z)) | (r3 & ~(tk.w | nv.w))) != 0u;
      }
      // nibble j of each ballot: candidate k0 + j taken / pending; bit 4 j of
      // `open`: candidate k0 + j exists and is not taken
      uint32_t taken = __ballot_sync(0xffffffffu, bl), pend = __ballot_sync(0xffffffffu, pe);
      taken |= taken >> 1;
      taken |= taken >> 2;
      pend |= pend >> 1;
      pend |= pend >> 2;
      const int ncand = min(kMaskCands, kend - k0);
      uint32_t open = ~taken & 0x11111111u & (ncand >= 8 ? 0xffffffffu : (1u << (4 * ncand)) - 1u);
      while (open != 0u) {
        const int j = (__ffs(open) - 1) >> 2;
        open &= open - 1u;
        const int kk = k0 + j;
        // earlier candidates are passed: say so before waiting or deciding
        mask_resolve<FRESH>(a, row, kdone, kb + kk, -1, lane, kb, my_c, my_rb);
        kdone = kb + kk;
        bool blocked = false;
        if ((pend >> (4 * j)) & 1u) {
          // wait for the earlier neighbours that may still take c
          const uint32_t c = __shfl_sync(0xffffffffu, my_c, kk);
          const int64_t rb = __shfl_sync(0xffffffffu, my_rb, kk);
          const bool act = lane < 16 && lane <= (rinfo_slot(rb) >> 5);
          const uint32_t r = act ? ld_run<FRESH>(a.rmask + rinfo_addr(rb) + lane) : 0u;
          while (true) {
            const uint32_t cc = act ? __ldcg(a.cmask + (size_t)c * 32 + lane) : 0u;
            const uint32_t ss = act ? __ldcg(a.cmask + (size_t)c * 32 + 16 + lane) : 0u;
            if (__any_sync(0xffffffffu, (r & cc) != 0u)) {
              blocked = true;
              break;
            }
            if (!__any_sync(0xffffffffu, (r & ~(cc | ss)) != 0u)) break;
            if (++polls > a.max_polls) {
              if (lane == 0) atomicExch(err, 1);
              return false;
            }
            __nanosleep(64);
          }
        }
        if (blocked) continue;
        // v takes c: colored bit, every other list color resolved
        const uint32_t c = __shfl_sync(0xffffffffu, my_c, kk);
        const int slot = rinfo_slot(__shfl_sync(0xffffffffu, my_rb, kk));
        mask_resolve<FRESH>(a, row, kdone, L, kb + kk, lane, kb, my_c, my_rb);
        if (lane == 0) {
          atomicOr(a.cmask + (size_t)c * 32 + (slot >> 5), 1u << (slot & 31));
          publish(a.state, v, (c << 2) | kColored);
        }
        return true;
      }
    }
    if (kb + 32 >= L) {
      // every candidate taken: v fails and will never take any of them
      mask_resolve<FRESH>(a, row, kdone, L, -1, lane, kb, my_c, my_rb);
      break;
    }
  }
  if (lane == 0) publish(a.state, v, (kFailedColor << 2) | kFailed);
  return true;
}

}  // namespace picasso
