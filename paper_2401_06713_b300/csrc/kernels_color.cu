// kernels_color.cu -- Alg. 1 coloring of G_c and the carry to the next round.
//
// The order is the static Random order of Sec. III-B with first fit: in
// ascending (priority, round-local id) order each vertex takes the smallest
// list color that no earlier conflict neighbour took.  The sweep below
// reproduces that sequential result in parallel.  A vertex v with candidate
// c (its k-th list color) looks only at the earlier neighbours that hold c --
// run k of its row plus side-list k -- and
//   * moves to its next list color as soon as one of them is colored c;
//   * takes c once every one of them is colored differently, failed, or still
//     undecided with a candidate above c (candidates only grow, so such a
//     neighbour can never take c);
//   * otherwise waits for the next sweep.
// Each state word changes only along undecided(c0) -> undecided(c1) -> ... ->
// colored / failed, so any value a concurrent reader sees is a true past
// state and every decision taken from it is final.  The earliest undecided
// vertex never waits, so every sweep makes progress.
#include "common.cuh"

namespace picasso {

// Approximate priority order of the work list: counting sort on the top
// priority bits.  The order only affects how fast decisions propagate
// inside one sweep (warps pick work in list order), never the result.
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

int prio_bins_for(int64_t n) {
  int bins = 2;
  while (bins < n && bins < 65536) bins <<= 1;
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
  return cudaGetLastError();
}

__global__ void k_color_init(ColorArgs a, const uint32_t* __restrict__ prio, int32_t* __restrict__ nwork) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v == 0) *nwork = (int32_t)a.n;
  if (v >= a.n) return;
  a.state[v] = ((uint64_t)prio[v] << 32) | (((uint64_t)(uint32_t)a.lists[v * a.L] << 2) | kUndecided);
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

// Publish a new state word (the low half of the 64-bit state; the priority
// in the high half never changes).
__device__ __forceinline__ void publish(uint64_t* state, int32_t v, uint32_t w) {
  __stcg(reinterpret_cast<uint32_t*>(state + v), w);
}

__global__ void __launch_bounds__(256, 4) k_color_sweep(ColorArgs a, const int32_t* __restrict__ work_in,
                                                        const int32_t* __restrict__ nwork_in,
                                                        int32_t* __restrict__ work_out,
                                                        int32_t* __restrict__ nwork_out) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t nin = *nwork_in;
  const int L = a.L;
  for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < nin; w += nwarps) {
    const int32_t v = work_in[w];
    const uint32_t pv = (uint32_t)(__ldcg(&a.state[v]) >> 32);
    int k = a.kcur[v];
    uint32_t cur = a.rcur[v];
    const int64_t row = (int64_t)v * L;
    while (true) {
      if (k >= L) {
        if (lane == 0) publish(a.state, v, (kFailedColor << 2) | kFailed);
        break;
      }
      const uint32_t c = (uint32_t)a.lists[row + k];
      const int64_t rs = a.runoff[row + k], r1 = a.runoff[row + k + 1];
      bool blocked = false;
      int64_t first_wait = -1;
      int32_t wait_u = -1;
      uint32_t wait_w = 0;
      // the run of c: earlier neighbours whose smallest shared color is c
      for (int64_t e0 = rs + cur; e0 < r1; e0 += 32) {
        const int64_t e = e0 + lane;
        bool lb = false, lw = false;
        int32_t u = -1;
        uint32_t wu = 0;
        if (e < r1) {
          u = a.col[e];
          const uint64_t su = __ldcg(&a.state[u]);
          const uint32_t pu = (uint32_t)(su >> 32);
          if (pu < pv || (pu == pv && u < v)) {
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
          wait_w = __shfl_sync(0xffffffffu, wu, src);
        }
      }
      // side list of c: earlier neighbours holding c with a smaller shared color
      if (!blocked) {
        const int64_t x0 = a.xoff[row + k], x1 = a.xoff[row + k + 1];
        for (int64_t e0 = x0; e0 < x1; e0 += 32) {
          const int64_t e = e0 + lane;
          bool lb = false, lw = false;
          int32_t u = -1;
          uint32_t wu = 0;
          if (e < x1) {
            u = a.xcol[e];
            const uint64_t su = __ldcg(&a.state[u]);
            const uint32_t pu = (uint32_t)(su >> 32);
            if (pu < pv || (pu == pv && u < v)) {
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
          if (wm && wait_u < 0) {
            const int src = __ffs(wm) - 1;
            wait_u = __shfl_sync(0xffffffffu, u, src);
            wait_w = __shfl_sync(0xffffffffu, wu, src);
          }
        }
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
          a.blkw[v] = wait_w;
          work_out[atomicAdd(nwork_out, 1)] = v;
        }
        break;
      }
      if (lane == 0) publish(a.state, v, (c << 2) | kColored);
      break;
    }
  }
}

// Wake check, one thread per pending vertex: nothing can have changed for v
// while the neighbour it waited on still shows the state word v saw, so v
// stays pending without a rescan; otherwise v goes to the active list that
// the sweep evaluates.  Appends are warp-aggregated.
__global__ void __launch_bounds__(256) k_color_wake(const int32_t* __restrict__ blk, const uint32_t* __restrict__ blkw,
                                                    const uint64_t* __restrict__ state,
                                                    const int32_t* __restrict__ work_in,
                                                    const int32_t* __restrict__ nwork_in, int32_t* __restrict__ active,
                                                    int32_t* __restrict__ nactive, int32_t* __restrict__ work_out,
                                                    int32_t* __restrict__ nwork_out) {
  const int64_t nin = *nwork_in;
  const int lane = threadIdx.x & 31;
  const uint32_t lt = lanemask_lt();
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nin; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t w = base + threadIdx.x;
    int32_t v = -1;
    bool stay = false;
    if (w < nin) {
      v = work_in[w];
      const int32_t b = blk[v];
      stay = b >= 0 && (uint32_t)__ldcg(&state[b]) == blkw[v];
    }
    const uint32_t ms = __ballot_sync(0xffffffffu, w < nin && stay);
    const uint32_t ma = __ballot_sync(0xffffffffu, w < nin && !stay);
    int32_t bs = 0, ba = 0;
    if (lane == 0) {
      if (ms) bs = atomicAdd(nwork_out, __popc(ms));
      if (ma) ba = atomicAdd(nactive, __popc(ma));
    }
    bs = __shfl_sync(0xffffffffu, bs, 0);
    ba = __shfl_sync(0xffffffffu, ba, 0);
    if (w < nin) {
      if (stay)
        work_out[bs + __popc(ms & lt)] = v;
      else
        active[ba + __popc(ma & lt)] = v;
    }
  }
}

cudaError_t launch_color_wake(const ColorArgs& a, const int32_t* work_in, const int32_t* nwork_in, int32_t* active,
                              int32_t* nactive, int32_t* work_out, int32_t* nwork_out, cudaStream_t s) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (a.n + 255) / 256;
  const int64_t blocks = want < (int64_t)sms * 8 ? (want > 0 ? want : 1) : (int64_t)sms * 8;
  k_color_wake<<<(unsigned)blocks, 256, 0, s>>>(a.blk, a.blkw, a.state, work_in, nwork_in, active, nactive, work_out,
                                               nwork_out);
  count_launches(1);
  return cudaGetLastError();
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

// Carry: write colors to the global array and flag the vertices that failed.
__global__ void k_carry_flags(const uint64_t* __restrict__ state, int64_t n, const int32_t* __restrict__ gid,
                              int64_t base, int32_t* __restrict__ color, uint32_t* __restrict__ flag) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const uint32_t w = (uint32_t)state[v];
  const uint32_t st = w & 3u;
  if (st == kColored) color[gid ? gid[v] : v] = (int32_t)(base + (int64_t)(w >> 2));
  flag[v] = st == kColored ? 0u : 1u;
}

cudaError_t launch_carry_flags(const uint64_t* state, int64_t n, const int32_t* gid, int64_t base, int32_t* color,
                               uint32_t* flag, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_carry_flags<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(state, n, gid, base, color, flag);
  count_launches(1);
  return cudaGetLastError();
}

// Stable compaction of the flagged vertices (ascending global id is kept).
__global__ void k_carry_gather(const uint32_t* __restrict__ flag, const int64_t* __restrict__ pos, int64_t n,
                               const int32_t* __restrict__ gid, const uint64_t* __restrict__ xz,
                               int32_t* __restrict__ gid_out, uint64_t* __restrict__ xz_out) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n || !flag[v]) return;
  const int64_t p = pos[v];
  gid_out[p] = gid ? gid[v] : (int32_t)v;
  xz_out[2 * p] = xz[2 * v];
  xz_out[2 * p + 1] = xz[2 * v + 1];
}

cudaError_t launch_carry_gather(const uint32_t* flag, const int64_t* pos, int64_t n, const int32_t* gid,
                                const uint64_t* xz, int32_t* gid_out, uint64_t* xz_out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_carry_gather<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(flag, pos, n, gid, xz, gid_out, xz_out);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void k_gather_xz(const uint64_t* __restrict__ xz_all, const int32_t* __restrict__ gid, int64_t n,
                            uint64_t* __restrict__ xz_out) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int64_t g = gid[v];
  xz_out[2 * v] = xz_all[2 * g];
  xz_out[2 * v + 1] = xz_all[2 * g + 1];
}

cudaError_t launch_gather_xz(const uint64_t* xz_all, const int32_t* gid, int64_t n, uint64_t* xz_out,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_gather_xz<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(xz_all, gid, n, xz_out);
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
