// kernels_color.cu -- Alg. 1 coloring of G_c and the carry to the next round.
//
// The order is the static Random order of Sec. III-B with first fit: in
// ascending (priority, round-local id) order each vertex takes the smallest
// list color that no earlier conflict neighbour took.  The sweeps below
// reproduce that sequential result in parallel.  A vertex v with candidate
// c (its k-th list color) looks only at the earlier neighbours that hold c
// (run k of its row) and
//   * moves to its next list color as soon as one of them is colored c;
//   * takes c once every one of them is colored differently, failed, or still
//     undecided with a candidate above c (candidates only grow, so such a
//     neighbour can never take c);
//   * otherwise records the first neighbour it waits on and is looked at
//     again only once that neighbour no longer holds it up (decided, or
//     undecided with a candidate above c).
// Each state word changes only along undecided(c0) -> undecided(c1) -> ... ->
// colored / failed, so any value a concurrent reader sees is a true past
// state and every decision taken from it is final.  The earliest undecided
// vertex never waits, so every sweep makes progress.
#include <cooperative_groups.h>

#include "common.cuh"
#include <algorithm>

#include "color_device.cuh"

namespace cg = cooperative_groups;

namespace picasso {

// ---------------------------------------------------------------------------
// Approximate priority order of the first work list: counting sort on the
// top priority bits.  The order only affects how fast decisions propagate
// inside one sweep (warps pick work in list order), never the result.
// ---------------------------------------------------------------------------
__global__ void k_prio_hist(const uint32_t* __restrict__ prio, int64_t n, int shift, uint32_t* __restrict__ hist) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) atomicAdd(&hist[prio[v] >> shift], 1u);
}

__global__ void k_prio_scatter(const uint32_t* __restrict__ prio, int64_t n, int shift,
                               const int64_t* __restrict__ hoff, uint32_t* __restrict__ cursor,
                               int32_t* __restrict__ work) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const uint32_t b = prio[v] >> shift;
  work[hoff[b] + atomicAdd(&cursor[b], 1u)] = (int32_t)v;
}

// Exact order inside each bin: insertion sort of the bin's (short) segment by
// (priority, vertex).  After it the whole list is in ascending (priority,
// round-local id) order, the coloring order.
__global__ void k_prio_bin_sort(const uint32_t* __restrict__ prio, const int64_t* __restrict__ hoff, int nbins,
                                int32_t* __restrict__ work) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbins) return;
  const int64_t lo = hoff[b], hi = hoff[b + 1];
  for (int64_t x = lo + 1; x < hi; ++x) {
    const int32_t v = work[x];
    const uint64_t kv = ((uint64_t)prio[v] << 32) | (uint32_t)v;
    int64_t y = x - 1;
    while (y >= lo) {
      const int32_t w = work[y];
      if ((((uint64_t)prio[w] << 32) | (uint32_t)w) <= kv) break;
      work[y + 1] = w;
      --y;
    }
    work[y + 1] = v;
  }
}

int prio_bins_for(int64_t n) {
  // about one vertex a bin: the insertion sorts stay a few elements long
  int bins = 2;
  while (bins < n && bins < (1 << 20)) bins <<= 1;
  return bins;
}

cudaError_t launch_prio_order(const uint32_t* prio, int64_t n, int nbins, uint32_t* hist, int64_t* hoff, void* tmp,
                              int32_t* work, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int bits = 0;
  while ((1 << bits) < nbins) ++bits;
  const int shift = 32 - bits;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * nbins, s);
  if (e != cudaSuccess) return e;
  k_prio_hist<<<blocks, 256, 0, s>>>(prio, n, shift, hist);
  count_launches(1);
  e = launch_scan_u32(hist, nbins, hoff, tmp, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * nbins, s);
  if (e != cudaSuccess) return e;
  k_prio_scatter<<<blocks, 256, 0, s>>>(prio, n, shift, hoff, hist, work);
  count_launches(1);
  k_prio_bin_sort<<<(unsigned)((nbins + 255) / 256), 256, 0, s>>>(prio, hoff, nbins, work);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void k_color_init(ColorArgs a, const uint32_t* __restrict__ prio, int32_t* __restrict__ nwork) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v == 0) *nwork = (int32_t)a.n;
  if (v >= a.n) return;
  a.state[v] = ((uint64_t)prio[v] << 32) | (((uint64_t)(uint32_t)a.lists[a.loff[v]] << 2) | kUndecided);
  a.kcur[v] = 0;
  a.rcur[v] = 0;
  a.blk[v] = -1;
}

cudaError_t launch_color_init(const ColorArgs& a, const uint32_t* prio, int32_t* nwork, cudaStream_t s) {
  const int64_t blocks = (a.n + 255) / 256;
  k_color_init<<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, s>>>(a, prio, nwork);
  count_launches(1);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Evaluation of one vertex by one warp: advance past blocked candidates, then
// take the candidate, fail, or record what v waits on and append v to
// work_out.  The loop runs at most L + 1 times.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void eval_vertex(const ColorArgs& a, int32_t v, int lane, int32_t* __restrict__ work_out,
                                            int32_t* __restrict__ nwork_out) {
  const int64_t row = a.loff[v];
  const int L = (int)(a.loff[v + 1] - row);
  const uint32_t pv = (uint32_t)(__ldcg(&a.state[v]) >> 32);
  int k = a.kcur[v];
  uint32_t cur = a.rcur[v];
  while (true) {
    if (k >= L) {
      if (lane == 0) publish(a.state, v, (kFailedColor << 2) | kFailed);
      return;
    }
    const uint32_t c = (uint32_t)a.lists[row + k];
    bool blocked = false;
    int64_t first_wait = -1;
    int32_t wait_u = -1;
    int64_t rs = 0, r1 = 0;
    if (a.rinfo) {
      // bit layout: cur counts resolved partner slots; every partner is
      // ranked before v
      const int64_t rb = a.rinfo[row + k];
      const int64_t pb = a.bboff[c];
      const int slot = rinfo_slot(rb);
      const int64_t w0 = rinfo_addr(rb);
      r1 = rinfo_len(rb) ? slot : 0;
      for (int64_t W = cur >> 5; (W << 5) < r1; ++W) {
        const int64_t t = (W << 5) + lane;
        const uint32_t wd = a.rmask[w0 + W];
        int32_t u = -1;
        if (t < slot && ((wd >> lane) & 1u)) u = a.bpid[pb + t];
        bool lb = false, lw = false;
        if (u >= 0) {
          const uint32_t wu = (uint32_t)__ldcg(&a.state[u]);
          const uint32_t st = wu & 3u, cu = wu >> 2;
          lb = st == kColored && cu == c;
          lw = st == kUndecided && cu <= c;
        }
        if (__any_sync(0xffffffffu, lb)) {
          blocked = true;
          break;
        }
        const uint32_t wm = __ballot_sync(0xffffffffu, lw);
        if (wm && first_wait < 0) {
          const int src = __ffs(wm) - 1;
          first_wait = (W << 5) + src;
          wait_u = __shfl_sync(0xffffffffu, u, src);
        }
      }
    } else {
      rs = a.runoff[row + k] - a.cbase;
      r1 = a.runoff[row + k + 1] - a.cbase;
    }
    // the run of c: the neighbours that hold c
    for (int64_t e0 = rs + cur; !a.rinfo && e0 < r1; e0 += 32) {
      const int64_t e = e0 + lane;
      bool lb = false, lw = false;
      int32_t u = -1;
      uint32_t wu = 0;
      if (e < r1) {
        u = a.col[e];
        if (a.ranked && u > v) u = -1;  // past the earlier neighbours
        const uint64_t su = u >= 0 ? __ldcg(&a.state[u]) : 0ull;
        const uint32_t pu = (uint32_t)(su >> 32);
        if (u >= 0 && (a.ranked || pu < pv || (pu == pv && u < v))) {
          wu = (uint32_t)su;
          const uint32_t st = wu & 3u, cu = wu >> 2;
          lb = st == kColored && cu == c;
          lw = st == kUndecided && cu <= c;
        }
      }
      if (__any_sync(0xffffffffu, lb)) {
        blocked = true;
        break;
      }
      const uint32_t wm = __ballot_sync(0xffffffffu, lw);
      if (wm && first_wait < 0) {
        const int src = __ffs(wm) - 1;
        first_wait = e0 + src;
        wait_u = __shfl_sync(0xffffffffu, u, src);
      }
      // ranked ids: the run ascends, so a later neighbour ends the prefix
      if (a.ranked && __any_sync(0xffffffffu, e < r1 && u < 0)) break;
    }
    if (blocked) {
      ++k;
      cur = 0;
      if (k < L && lane == 0) publish(a.state, v, ((uint32_t)a.lists[row + k] << 2) | kUndecided);
      continue;
    }
    if (wait_u >= 0) {
      if (lane == 0) {
        a.kcur[v] = (uint16_t)k;
        a.rcur[v] = (uint32_t)((first_wait >= 0 ? first_wait : r1) - rs);
        a.blk[v] = wait_u;
        a.blkw[v] = c;
        work_out[atomicAdd(nwork_out, 1)] = v;
      }
      return;
    }
    if (lane == 0) publish(a.state, v, (c << 2) | kColored);
    return;
  }
}

// Wake check of the pending items [b0, b0 + 32) of `in` by one warp: v stays
// pending without a rescan while the neighbour it waited on is still
// undecided with a candidate at or below v's candidate color (v could not
// decide anything new); otherwise v goes to the active list.  Appends are
// warp-aggregated.
__device__ __forceinline__ void wake_chunk(const ColorArgs& a, const int32_t* __restrict__ in, int64_t nin,
                                           int64_t b0, int lane, uint32_t lt, int32_t* __restrict__ active,
                                           int32_t* __restrict__ nactive, int32_t* __restrict__ out,
                                           int32_t* __restrict__ nout) {
  const int64_t w = b0 + lane;
  int32_t v = -1;
  bool stay = false;
  if (w < nin) {
    v = __ldcg(&in[w]);
    const int32_t b = a.blk[v];
    if (b >= 0) {
      const uint32_t wb = (uint32_t)__ldcg(&a.state[b]);
      stay = (wb & 3u) == kUndecided && (wb >> 2) <= a.blkw[v];
    }
  }
  const uint32_t ms = __ballot_sync(0xffffffffu, w < nin && stay);
  const uint32_t ma = __ballot_sync(0xffffffffu, w < nin && !stay);
  int32_t bs = 0, ba = 0;
  if (lane == 0) {
    if (ms) bs = atomicAdd(nout, __popc(ms));
    if (ma) ba = atomicAdd(nactive, __popc(ma));
  }
  bs = __shfl_sync(0xffffffffu, bs, 0);
  ba = __shfl_sync(0xffffffffu, ba, 0);
  if (w < nin) {
    if (stay)
      out[bs + __popc(ms & lt)] = v;
    else
      active[ba + __popc(ma & lt)] = v;
  }
}

// ---------------------------------------------------------------------------
// All sweeps of one round in a single cooperative launch: per sweep, a wake
// phase (thread per pending vertex) and an evaluation phase (warp per active
// vertex), separated by grid barriers; no host round trip between sweeps.
// ctl[0] pending count, ctl[1] next pending count, ctl[2] active count,
// ctl[3] sweeps run, ctl[4] set to 1 if max_sweeps ran out.  Every thread
// takes every barrier: the loop exits depend only on values all threads read
// after the same barrier.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 4) k_color_all(ColorArgs a, int32_t* __restrict__ wa, int32_t* __restrict__ wb,
                                                      int32_t* __restrict__ wact, int32_t* __restrict__ ctl,
                                                      int32_t max_sweeps) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = lanemask_lt();
  const int64_t gwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t wid = tid >> 5;
  int32_t* in = wa;
  int32_t* out = wb;
  int32_t sweep = 0;
  while (true) {
    const int32_t nin = __ldcg(&ctl[0]);
    if (nin == 0) break;
    if (sweep >= max_sweeps) {
      if (tid == 0) ctl[4] = 1;
      break;
    }
    if (tid == 0 && sweep < kSweepLog) {
      uint64_t t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      ctl[8 + sweep] = nin;
      reinterpret_cast<unsigned long long*>(ctl + 8 + kSweepLog)[sweep] = t;
    }
    for (int64_t b0 = wid * 32; b0 < nin; b0 += gwarps * 32)
      wake_chunk(a, in, nin, b0, lane, lt, wact, &ctl[2], out, &ctl[1]);
    if (!grid_sync_bounded(reinterpret_cast<unsigned int*>(ctl + kCtlBar), ctl + kCtlAbort, kBarrierLimitNs, ctl + kCtlSeen)) return;
    const int32_t nact = __ldcg(&ctl[2]);
    for (int64_t w = wid; w < nact; w += gwarps) eval_vertex(a, __ldcg(&wact[w]), lane, out, &ctl[1]);
    if (!grid_sync_bounded(reinterpret_cast<unsigned int*>(ctl + kCtlBar), ctl + kCtlAbort, kBarrierLimitNs, ctl + kCtlSeen)) return;
    if (tid == 0) {
      ctl[0] = __ldcg(&ctl[1]);
      ctl[1] = 0;
      ctl[2] = 0;
      ctl[3] = sweep + 1;
      if (sweep < kSweepLog) ctl[8 + 3 * kSweepLog + sweep] = nact;
    }
    if (!grid_sync_bounded(reinterpret_cast<unsigned int*>(ctl + kCtlBar), ctl + kCtlAbort, kBarrierLimitNs, ctl + kCtlSeen)) return;
    int32_t* t = in;
    in = out;
    out = t;
    ++sweep;
  }
}

__global__ void __launch_bounds__(256, 6) k_color_ordered(ColorArgs a, const int32_t* __restrict__ order,
                                                          int32_t* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int64_t gwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int64_t t = wid; t < a.n; t += gwarps) {
    if (!ordered_vertex<false>(a, order ? __ldcg(&order[t]) : (int32_t)(a.v0 + t), lane, err)) return;
  }
}

// The ordered pass of the bit layout with the buckets' masks (mask_vertex);
// vertices in rank order (ranked ids), one warp each.
__global__ void __launch_bounds__(256, 6) k_color_masks(ColorArgs a, int32_t* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int64_t gwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int64_t t = wid; t < a.n; t += gwarps) {
    if (!mask_vertex<false>(a, (int32_t)(a.v0 + t), lane, err)) return;
  }
}

cudaError_t launch_color_ordered(const ColorArgs& a, const int32_t* order, int32_t* err, cudaStream_t s,
                                 int per_sm_cap) {
  int dev = 0, sms = 148, per_sm = 0;
  const bool masks = a.cmask != nullptr;
  // the mask coloring reads the color masks 16 bytes at a time
  if (reinterpret_cast<uintptr_t>(a.cmask) & 15) return cudaErrorMisalignedAddress;
  const void* kern = masks ? (const void*)k_color_masks : (const void*)k_color_ordered;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  if (per_sm_cap > 0) per_sm = std::min(per_sm, per_sm_cap);
  int64_t blocks = (int64_t)per_sm * sms;
  const int64_t want = (a.n + 7) / 8;
  if (want < blocks) blocks = want > 0 ? want : 1;
  blocks = debug_grid(blocks);
  ColorArgs args = a;
  if (masks) {
    void* params[] = {(void*)&args, (void*)&err};
    e = cudaLaunchCooperativeKernel(kern, dim3((unsigned)blocks), dim3(256), params, 0, s);
  } else {
    void* params[] = {(void*)&args, (void*)&order, (void*)&err};
    e = cudaLaunchCooperativeKernel(kern, dim3((unsigned)blocks), dim3(256), params, 0, s);
  }
  count_launches(1);
  return e;
}

cudaError_t launch_color_all(const ColorArgs& a, int32_t* wa, int32_t* wb, int32_t* wact, int32_t* ctl,
                             cudaStream_t s) {
  int dev = 0, sms = 148, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_color_all, 256, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  int64_t blocks = (int64_t)per_sm * sms;
  const int64_t want = (a.n + 7) / 8;  // one warp per vertex at most
  if (want < blocks) blocks = want > 0 ? want : 1;
  blocks = debug_grid(blocks);
  ColorArgs args = a;
  int32_t max_sweeps = (int32_t)(a.n + 4 < 0x7fffffff ? a.n + 4 : 0x7fffffff);
  void* params[] = {(void*)&args, (void*)&wa, (void*)&wb, (void*)&wact, (void*)&ctl, (void*)&max_sweeps};
  e = cudaLaunchCooperativeKernel((const void*)k_color_all, dim3((unsigned)blocks), dim3(256), params, 0, s);
  count_launches(1);
  return e;
}

// Single-sweep kernels (the same two phases, one launch each), for callers
// that drive the sweeps from the host.
__global__ void __launch_bounds__(256) k_color_wake(ColorArgs a, const int32_t* __restrict__ work_in,
                                                    const int32_t* __restrict__ nwork_in, int32_t* __restrict__ active,
                                                    int32_t* __restrict__ nactive, int32_t* __restrict__ work_out,
                                                    int32_t* __restrict__ nwork_out) {
  const int64_t nin = *nwork_in;
  const int lane = threadIdx.x & 31;
  const uint32_t lt = lanemask_lt();
  const int64_t gwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int64_t b0 = wid * 32; b0 < nin; b0 += gwarps * 32)
    wake_chunk(a, work_in, nin, b0, lane, lt, active, nactive, work_out, nwork_out);
}

cudaError_t launch_color_wake(const ColorArgs& a, const int32_t* work_in, const int32_t* nwork_in, int32_t* active,
                              int32_t* nactive, int32_t* work_out, int32_t* nwork_out, cudaStream_t s) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (a.n + 255) / 256;
  const int64_t blocks = want < (int64_t)sms * 8 ? (want > 0 ? want : 1) : (int64_t)sms * 8;
  k_color_wake<<<(unsigned)blocks, 256, 0, s>>>(a, work_in, nwork_in, active, nactive, work_out, nwork_out);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256, 4) k_color_sweep(ColorArgs a, const int32_t* __restrict__ work_in,
                                                        const int32_t* __restrict__ nwork_in,
                                                        int32_t* __restrict__ work_out,
                                                        int32_t* __restrict__ nwork_out) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t nin = *nwork_in;
  for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < nin; w += nwarps)
    eval_vertex(a, work_in[w], lane, work_out, nwork_out);
}

cudaError_t launch_color_sweep(const ColorArgs& a, const int32_t* work_in, const int32_t* nwork_in,
                               int32_t* work_out, int32_t* nwork_out, cudaStream_t s) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (a.n + 7) / 8;
  const int64_t blocks = want < (int64_t)sms * 8 ? (want > 0 ? want : 1) : (int64_t)sms * 8;
  k_color_sweep<<<(unsigned)blocks, 256, 0, s>>>(a, work_in, nwork_in, work_out, nwork_out);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Carry
// ---------------------------------------------------------------------------
// Write colors to the output and flag the vertices that failed: the final
// color of a vertex of set k is base_k + (bucket color - cofs_k), written at
// its batch-global id.
__global__ void k_carry_flags(const uint64_t* __restrict__ state, int64_t n, const int32_t* __restrict__ gid,
                              const int32_t* __restrict__ perm, const int64_t* __restrict__ soff, int nsets,
                              const SetRound* __restrict__ sets, int32_t* __restrict__ color,
                              uint32_t* __restrict__ flag) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const uint32_t w = (uint32_t)state[v];
  const uint32_t st = w & 3u;
  if (st == kColored) {
    const int64_t g = gid ? (int64_t)gid[v] : v;
    const SetRound& sr = sets[nsets > 1 ? set_of(soff, nsets, g) : 0];
    color[g] = (int32_t)(sr.base + ((int64_t)(w >> 2) - sr.cofs));
  }
  flag[perm ? perm[v] : v] = st == kColored ? 0u : 1u;
}

cudaError_t launch_carry_flags(const uint64_t* state, int64_t n, const int32_t* gid, const int32_t* perm,
                               const int64_t* soff, int32_t nsets, const SetRound* sets, int32_t* color,
                               uint32_t* flag, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_carry_flags<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(state, n, gid, perm, soff, nsets, sets, color, flag);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void k_set_counts(const int32_t* __restrict__ gid, int64_t n, const int64_t* __restrict__ soff, int nsets,
                             uint32_t* __restrict__ hist) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int64_t g = gid ? (int64_t)gid[v] : v;
  atomicAdd(&hist[nsets > 1 ? set_of(soff, nsets, g) : 0], 1u);
}

cudaError_t launch_set_counts(const int32_t* gid, int64_t n, const int64_t* soff, int32_t nsets, uint32_t* hist,
                              cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * nsets, s);
  if (e != cudaSuccess || n <= 0) return e;
  k_set_counts<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(gid, n, soff, nsets, hist);
  count_launches(1);
  return cudaGetLastError();
}

// Conflict-structure bytes of every set in this round, counted like the
// byte budget: 8 (n_k + 1) row offsets + 4 per run entry, accumulated per
// vertex (the round's vertices of a set need not be contiguous).
__global__ void k_set_csr_bytes(const int64_t* __restrict__ loff, const int64_t* __restrict__ runoff,
                                const uint32_t* __restrict__ cnt, const int32_t* __restrict__ gid, int64_t n,
                                const int64_t* __restrict__ soff, int nsets, unsigned long long* __restrict__ out) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int64_t g = gid ? (int64_t)gid[v] : v;
  const int k = nsets > 1 ? set_of(soff, nsets, g) : 0;
  int64_t entries = 0;
  if (runoff) {
    entries = runoff[loff[v + 1]] - runoff[loff[v]];
  } else {
    for (int64_t e = loff[v]; e < loff[v + 1]; ++e) entries += cnt[e];
  }
  atomicAdd(&out[k], (unsigned long long)(8 + 4 * entries));
}


cudaError_t launch_set_csr_bytes(const int64_t* loff, const int64_t* runoff, const uint32_t* cnt, const int32_t* gid,
                                 int64_t n, const int64_t* soff, int32_t nsets, int64_t* out, cudaStream_t s) {
  if (nsets <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int64_t) * nsets, s);
  if (e != cudaSuccess || n <= 0) return e;
  k_set_csr_bytes<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(loff, runoff, cnt, gid, n, soff, nsets,
                                                               (unsigned long long*)out);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void k_rank_gather(const int32_t* __restrict__ perm, int64_t n, const int32_t* __restrict__ gid_in,
                              const uint64_t* __restrict__ xz_in, const uint32_t* __restrict__ prio_in,
                              int32_t* __restrict__ gid_out, uint64_t* __restrict__ xz_out,
                              uint32_t* __restrict__ prio_out, int32_t S) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int64_t i = perm[t];
  gid_out[t] = gid_in ? gid_in[i] : (int32_t)i;
  for (int w = 0; w < S; ++w) xz_out[S * t + w] = xz_in[S * i + w];
  prio_out[t] = prio_in[i];
}

cudaError_t launch_rank_gather(const int32_t* perm, int64_t n, const int32_t* gid_in, const uint64_t* xz_in,
                               const uint32_t* prio_in, int32_t* gid_out, uint64_t* xz_out, uint32_t* prio_out,
                               int32_t S, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_rank_gather<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(perm, n, gid_in, xz_in, prio_in, gid_out, xz_out,
                                                             prio_out, S);
  count_launches(1);
  return cudaGetLastError();
}

// Stable compaction of the flagged vertices (ascending global id is kept).
__global__ void k_carry_gather(const uint32_t* __restrict__ flag, const int64_t* __restrict__ pos, int64_t n,
                               const int32_t* __restrict__ gid, const uint64_t* __restrict__ xz,
                               int32_t* __restrict__ gid_out, uint64_t* __restrict__ xz_out, int32_t S) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n || !flag[v]) return;
  const int64_t p = pos[v];
  gid_out[p] = gid ? gid[v] : (int32_t)v;
  for (int w = 0; w < S; ++w) xz_out[S * p + w] = xz[S * v + w];
}

cudaError_t launch_carry_gather(const uint32_t* flag, const int64_t* pos, int64_t n, const int32_t* gid,
                                const uint64_t* xz, int32_t* gid_out, uint64_t* xz_out, int32_t S, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_carry_gather<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(flag, pos, n, gid, xz, gid_out, xz_out, S);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void k_gather_xz(const uint64_t* __restrict__ xz_all, const int32_t* __restrict__ gid, int64_t n,
                            uint64_t* __restrict__ xz_out, int32_t S) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int64_t g = gid[v];
  for (int w = 0; w < S; ++w) xz_out[S * v + w] = xz_all[S * g + w];
}

cudaError_t launch_gather_xz(const uint64_t* xz_all, const int32_t* gid, int64_t n, uint64_t* xz_out, int32_t S,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_gather_xz<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(xz_all, gid, n, xz_out, S);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void k_fill_i32(int32_t* out, int64_t n, int32_t v, int32_t step) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = step ? (int32_t)i : v;
}

cudaError_t launch_iota(int32_t* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_fill_i32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, 0, 1);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fill_i32(int32_t* out, int64_t n, int32_t v, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_fill_i32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, v, 0);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace picasso
