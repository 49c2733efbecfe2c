// kernels_dynamic.cu -- Alg. 2's dynamic order on the GPU (the parallel rule).
//
// Alg. 2 colors the most constrained vertex first: the lowest bucket of
// remaining-list sizes, a color drawn from the remaining list, and that color
// leaves the lists of the vertex's uncolored neighbours.  Strictly sequential
// as written; here each step colors, at once, every uncolored vertex whose
// (remaining size, rank) is smaller than that of each uncolored neighbour
// (no two such vertices are adjacent), then removes their colors from the
// neighbours' lists.  A vertex whose list empties is left uncolored at the
// start of the next step.  Round-local ids are ranks in ascending
// (priority, global id), so the rank orders ties as (priority, id) would.
//
// A vertex's remaining list is a bit mask over its list entries (L <= 64);
// the conflict rows are the two-sided canonical ones (FULL form), so a
// colored vertex reaches every neighbour holding its color through the run
// of that color.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace picasso {

namespace {
// Position of the idx-th set bit (0-based) of m (idx < popc(m)).
__device__ __forceinline__ int nth_set_bit(uint64_t m, int idx) {
  const uint32_t lo = (uint32_t)m, hi = (uint32_t)(m >> 32);
  const int nlo = __popc(lo);
  if (idx < nlo) return __fns(lo, 0, idx + 1);
  return 32 + __fns(hi, 0, idx - nlo + 1);
}

// Position of color c in the sorted list [p, p + L), or -1.
__device__ __forceinline__ int list_pos(const int32_t* __restrict__ p, int L, int32_t c) {
  int lo = 0, hi = L - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int32_t x = p[mid];
    if (x == c) return mid;
    if (x < c)
      lo = mid + 1;
    else
      hi = mid - 1;
  }
  return -1;
}
}  // namespace

// The order of a step: (remaining list size, rank), smaller first.
__device__ __forceinline__ bool key_less(int cu, int32_t u, int cv, int32_t v) {
  return cu < cv || (cu == cv && u < v);
}

// Push v on the next step's work list once per step (stamp = step + 1).
__device__ __forceinline__ void push_next(const DynArgs& d, int32_t v, int32_t stamp, int32_t* list,
                                          int32_t* len) {
  if (atomicExch(d.stamp + v, stamp) != stamp) list[atomicAdd(len, 1)] = v;
}

constexpr int kScanChunks = 4;   // 32-entry chunks of a row scan in flight per warp
constexpr int kMaxParts = 16;    // warps sharing one vertex's strike or drain
constexpr int kMaxLongParts = 64;                  // warps sharing one long row scan
constexpr int64_t kHeadEntries = 64 * kScanChunks;  // row entries the first pass scans

// Warps per item when `items` items share the grid's nw warps.
__device__ __forceinline__ int64_t parts_for(int64_t items, int64_t nw, int64_t cap = kMaxParts) {
  if (items >= nw) return 1;
  const int64_t g = nw / items;
  return g < cap ? g : cap;
}

// Part j of G of examining vertex v at a step (one warp per part).  A vertex
// is active while its mask is nonzero (colored vertices and emptied lists
// have mask 0).  The part scans chunks j, j + G, ... of v's row entries from
// `skip` on, at most `limit` of them (chunks of 32 x kScanChunks entries,
// the next chunk's ids loaded while the current one's masks arrive), for an
// active neighbour smaller in (size, rank); on finding one it records it in
// blk[v] (the chunk's largest such neighbour in that order) and marks v
// blocked for this step (bstep[v] = stamp).
//   First pass (G = 1, skip 0, limit kHeadEntries): no blocker and nothing
//   left to scan makes v a local minimum (to sel); no blocker with entries
//   left puts v on the long list (lng).
//   Second pass (the long list, skip kHeadEntries, G parts): the part that
//   finishes last appends v to sel when no part found a blocker.
__device__ __forceinline__ void dyn_examine(const DynArgs& d, int32_t v, int64_t j, int64_t G, int lane,
                                            int32_t stamp, int32_t* slen, int64_t skip, int64_t limit,
                                            int32_t* llen) {
  const uint64_t m = __ldcg(d.mask + v);
  if (m == 0) return;  // finished (all parts see the same)
  const int cnt = __popcll(m);
  const int64_t r0 = d.runoff[d.loff[v]], rend = d.runoff[d.loff[v + 1]];
  const int64_t rs = r0 + skip, re = min(rend, rs + limit);
  constexpr int64_t CH = 32 * kScanChunks;
  bool found = false;
  int32_t u[kScanChunks], un[kScanChunks];
  auto load_cols = [&](int64_t e0, int32_t* dst) {
#pragma unroll
    for (int k = 0; k < kScanChunks; ++k) {
      const int64_t e = e0 + 32 * k + lane;
      dst[k] = e < re ? d.col[e] : -1;
    }
  };
  load_cols(rs + j * CH, u);
  for (int64_t e0 = rs + j * CH; e0 < re; e0 += G * CH) {
    uint64_t mu[kScanChunks];
#pragma unroll
    for (int k = 0; k < kScanChunks; ++k) mu[k] = u[k] >= 0 ? __ldcg(d.mask + u[k]) : 0ull;
    load_cols(e0 + G * CH, un);  // the next chunk's ids while the masks arrive
    int cb = -1;
    int32_t ub = -1;
#pragma unroll
    for (int k = 0; k < kScanChunks; ++k) {
      if (mu[k] != 0) {
        const int cu = __popcll(mu[k]);
        if (key_less(cu, u[k], cnt, v) && (cu > cb || (cu == cb && u[k] > ub))) {
          cb = cu;
          ub = u[k];
        }
      }
    }
    if (__any_sync(0xffffffffu, cb >= 0)) {
      const int cmax = __reduce_max_sync(0xffffffffu, cb);
      const int32_t umax = __reduce_max_sync(0xffffffffu, cb == cmax ? ub : -1);
      if (lane == 0) {
        d.blk[v] = umax;
        d.bstep[v] = stamp;
      }
      found = true;
      break;
    }
    if (G > 1 && __ldcg(d.bstep + v) == stamp) {  // another part found one
      found = true;
      break;
    }
#pragma unroll
    for (int k = 0; k < kScanChunks; ++k) u[k] = un[k];
  }
  if (lane != 0) return;
  if (llen != nullptr) {  // first pass
    if (!found) {
      if (re < rend)
        d.lng[atomicAdd(llen, 1)] = v;
      else
        d.sel[atomicAdd(slen, 1)] = v;
    }
    return;
  }
  if (G == 1) {
    if (!found) d.sel[atomicAdd(slen, 1)] = v;
    return;
  }
  __threadfence();
  if (atomicAdd(d.parts + v, 1) == (int32_t)(G - 1)) {
    d.parts[v] = 0;
    __threadfence();
    if (__ldcg(d.bstep + v) != stamp) d.sel[atomicAdd(slen, 1)] = v;
  }
}

// Part j of G of coloring v (a local minimum): v takes the color its draw
// picks from its remaining list; the part strikes that color from the lists
// of entries j, j + G, ... (32 at a time) of v's run of it.  A neighbour
// whose list empties is finished (state 2, put on fin); one whose new size
// puts it below the neighbour it was blocked by goes on the next work list.
__device__ __forceinline__ void dyn_apply(const DynArgs& d, int32_t v, int64_t j, int64_t G, int lane,
                                          int32_t stamp, int32_t* wnext, int32_t* wlen, int32_t* flen) {
  const uint64_t m = __ldcg(d.mask + v);
  const int cnt = __popcll(m);
  const int64_t g = d.gid[v];
  const int k = d.nsets > 1 ? set_of(d.soff, d.nsets, g) : 0;
  const uint32_t x = philox_block(d.sets[k].seed, d.round, g - d.soff[k], kTagDynamic, 0u).x;
  const int idx = (int)(((uint64_t)x * (uint64_t)cnt) >> 32);
  const int pos = nth_set_bit(m, idx);
  const int64_t e = d.loff[v] + pos;
  const int32_t c = d.lists[e];
  if (j == 0 && lane == 0) {
    d.color[v] = c;
    d.state[v] = 1;
  }
  const int64_t rs = d.runoff[e], re = d.runoff[e + 1];
  for (int64_t q = rs + 32 * j + lane; q < re; q += 32 * G) {
    const int32_t u = d.col[q];
    if (__ldcg(d.mask + u) == 0) continue;
    const int64_t lu = d.loff[u];
    const int p = list_pos(d.lists + lu, (int)(d.loff[u + 1] - lu), c);
    if (p < 0) continue;
    const uint64_t bit = 1ull << p;
    const uint64_t old = atomicAnd((unsigned long long*)(d.mask + u), ~bit);
    if (!(old & bit)) continue;
    const uint64_t now = old & ~bit;
    if (now == 0) {
      d.state[u] = 2;
      d.fin[atomicAdd(flen, 1)] = u;
      continue;
    }
    // still blocked by the same neighbour unless u now sorts below it (a
    // stale, larger size of the blocker only sends u to be re-examined)
    const int32_t b = __ldcg(d.blk + u);
    if (b < 0 || !key_less(__popcll(__ldcg(d.mask + b)), b, __popcll(now), u)) push_next(d, u, stamp, wnext, wlen);
  }
}

// Every step of a round in one cooperative launch, driven by events.  A
// vertex is examined at a step only if it is new (step 0), its blocker
// finished at the previous step, or its list shrank below its blocker's; any
// other active vertex is still blocked by its recorded neighbour (which is
// still active, and whose size only shrinks), so the steps take the same
// local minima as examining every vertex at every step.  Per step:
//   S  examine the work list: local minima to sel, blocked ones record blk
//      (a list longer than a quarter of the grid's warps: a first pass over
//      each row's head, then, after a barrier, the rows still undecided split
//      over all warps; a shorter one: several warps per row from the start);
//   A  the minima take colors and strike them; lists struck empty to fin;
//      neighbours whose size crossed their blocker's to the next list;
//   D  the minima's masks to 0; the waiters of each finished vertex (sel and
//      fin), neighbours w with blk[w] = that vertex, to the next list;
// with a grid barrier after each.  Short lists spread each item over up to
// kMaxParts warps.  ctl: [0..1] work list lengths (by step parity), [2..3]
// sel lengths, [4..5] fin lengths, [6] steps that colored a vertex, [7]
// long list length.  The
// smallest active vertex is never blocked, so it is on the work list while
// any vertex is active; every step finishes it, so the list is empty after
// at most n + 1 steps.
__global__ void k_dyn_all(DynArgs d) {
  int32_t* const ctl = d.ctl;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int64_t step = 0; step <= d.n; ++step) {
    const int p = (int)(step & 1);
    const int32_t* cur = p ? d.wb : d.wa;
    int32_t* nxt = p ? d.wa : d.wb;
    const int32_t stamp = (int32_t)(step + 1);
    const int64_t m = __ldcg(ctl + p);
    if (m == 0) break;
    constexpr int64_t kAll = (int64_t)1 << 62;
    if (4 * m > nw) {
      // S, long work list: first pass, one warp per vertex over its row head
      for (int64_t i = gw; i < m; i += nw)
        dyn_examine(d, __ldcg(cur + i), 0, 1, lane, stamp, ctl + 2 + p, 0, kHeadEntries, ctl + 7);
      if (!grid_sync_bounded(reinterpret_cast<unsigned int*>(ctl + 8), ctl + 10, kBarrierLimitNs, ctl + 11)) return;
      // second pass: the rows still undecided, split over the warps
      const int64_t nl = __ldcg(ctl + 7);
      if (nl > 0) {
        const int64_t G = parts_for(nl, nw, kMaxLongParts);
        for (int64_t w = gw; w < nl * G; w += nw)
          dyn_examine(d, __ldcg(d.lng + w / G), w % G, G, lane, stamp, ctl + 2 + p, kHeadEntries, kAll, nullptr);
      }
    } else {
      // S, short work list: at least four warps per vertex, whole rows
      const int64_t G = parts_for(m, nw);
      for (int64_t w = gw; w < m * G; w += nw)
        dyn_examine(d, __ldcg(cur + w / G), w % G, G, lane, stamp, ctl + 2 + p, 0, kAll, nullptr);
    }
    if (!grid_sync_bounded(reinterpret_cast<unsigned int*>(ctl + 8), ctl + 10, kBarrierLimitNs, ctl + 11)) return;
    // A
    const int64_t ns = __ldcg(ctl + 2 + p);
    if (ns > 0) {
      const int64_t G = parts_for(ns, nw);
      for (int64_t w = gw; w < ns * G; w += nw)
        dyn_apply(d, __ldcg(d.sel + w / G), w % G, G, lane, stamp, nxt, ctl + 1 - p, ctl + 4 + p);
    }
    if (!grid_sync_bounded(reinterpret_cast<unsigned int*>(ctl + 8), ctl + 10, kBarrierLimitNs, ctl + 11)) return;
    // D
    const int64_t nf = __ldcg(ctl + 4 + p), nt = ns + nf;
    if (nt > 0) {
      const int64_t G = parts_for(nt, nw);
      for (int64_t w = gw; w < nt * G; w += nw) {
        const int64_t i = w / G, j = w % G;
        const int32_t f = i < ns ? __ldcg(d.sel + i) : __ldcg(d.fin + (i - ns));
        if (i < ns && j == 0 && lane == 0) d.mask[f] = 0;
        const int64_t rs = d.runoff[d.loff[f]], re = d.runoff[d.loff[f + 1]];
        for (int64_t q = rs + 32 * j + lane; q < re; q += 32 * G) {
          const int32_t u = d.col[q];
          if (__ldcg(d.blk + u) == f && __ldcg(d.mask + u) != 0) push_next(d, u, stamp, nxt, ctl + 1 - p);
        }
      }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ctl[p] = 0;          // read by S of this step only
      ctl[2 + 1 - p] = 0;  // the next step's sel and fin
      ctl[4 + 1 - p] = 0;
      ctl[7] = 0;          // read after the first pass of this step's S only
      if (ns > 0) ctl[6] += 1;
    }
    if (!grid_sync_bounded(reinterpret_cast<unsigned int*>(ctl + 8), ctl + 10, kBarrierLimitNs, ctl + 11)) return;
  }
}

// Masks of full lists, every vertex on the first work list; state words for
// the carry at the end.
__global__ void k_dyn_init(DynArgs d) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < kDynCtlWords) d.ctl[v] = v == 0 ? (int32_t)d.n : 0;
  if (v >= d.n) return;
  const int L = (int)(d.loff[v + 1] - d.loff[v]);
  d.mask[v] = L >= 64 ? ~0ull : ((1ull << L) - 1ull);
  d.state[v] = 0;
  d.stamp[v] = 0;
  d.bstep[v] = 0;
  d.parts[v] = 0;
  d.blk[v] = -1;
  d.wa[v] = (int32_t)v;
}

__global__ void k_dyn_finish(DynArgs d, uint64_t* __restrict__ words) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.n) return;
  words[v] = d.state[v] == 1 ? (((uint64_t)(uint32_t)d.color[v] << 2) | kColored)
                             : (((uint64_t)kFailedColor << 2) | kFailed);
}

cudaError_t launch_dyn_init(const DynArgs& d, cudaStream_t s) {
  k_dyn_init<<<(unsigned)((std::max<int64_t>(d.n, 8) + 255) / 256), 256, 0, s>>>(d);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_dyn_all(const DynArgs& d, cudaStream_t s) {
  if (d.n <= 0) return cudaSuccess;
  int dev = 0, sms = 148, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dyn_all, 256, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  // up to 4 CTAs per SM: warps to hide the scans' load latency
  int64_t blocks = (int64_t)std::min(per_sm, 4) * sms;
  const int64_t want = (d.n + 7) / 8;
  if (want < blocks) blocks = want > 0 ? want : 1;
  blocks = debug_grid(blocks);
  DynArgs args = d;
  void* params[] = {(void*)&args};
  e = cudaLaunchCooperativeKernel((const void*)k_dyn_all, dim3((unsigned)blocks), dim3(256), params, 0, s);
  count_launches(1);
  return e;
}

cudaError_t launch_dyn_finish(const DynArgs& d, uint64_t* words, cudaStream_t s) {
  if (d.n <= 0) return cudaSuccess;
  k_dyn_finish<<<(unsigned)((d.n + 255) / 256), 256, 0, s>>>(d, words);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace picasso
