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

__global__ void k_color_init(ColorArgs a, int32_t* __restrict__ work, int32_t* __restrict__ nwork) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v == 0) *nwork = (int32_t)a.n;
  if (v >= a.n) return;
  a.word[v] = ((uint32_t)a.lists[v * a.L] << 2) | kUndecided;
  a.kcur[v] = 0;
  work[v] = (int32_t)v;
}

cudaError_t launch_color_init(const ColorArgs& a, int32_t* work, int32_t* nwork, cudaStream_t s) {
  const int64_t blocks = (a.n + 255) / 256;
  k_color_init<<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, s>>>(a, work, nwork);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_color_sweep(ColorArgs a, const int32_t* __restrict__ work_in,
                                                     const int32_t* __restrict__ nwork_in,
                                                     int32_t* __restrict__ work_out, int32_t* __restrict__ nwork_out) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t nin = *nwork_in;
  const int L = a.L;
  for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < nin; w += nwarps) {
    const int32_t v = work_in[w];
    const uint32_t pv = a.prio[v];
    int k = a.kcur[v];
    const int64_t row = (int64_t)v * L;
    while (true) {
      if (k >= L) {
        if (lane == 0) __stcg(&a.word[v], (kFailedColor << 2) | kFailed);
        break;
      }
      const uint32_t c = (uint32_t)a.lists[row + k];
      bool blocked = false, wait = false;
      const int64_t r0 = a.runoff[row + k], r1 = a.runoff[row + k + 1];
      for (int64_t e = r0 + lane; e < r1; e += 32) {
        const int32_t u = a.col[e];
        const uint32_t pu = a.prio[u];
        if (pu < pv || (pu == pv && u < v)) {
          const uint32_t wu = __ldcg(&a.word[u]);
          const uint32_t st = wu & 3u, cu = wu >> 2;
          blocked |= (st == kColored && cu == c);
          wait |= (st == kUndecided && cu <= c);
        }
      }
      const int64_t x0 = a.xoff[row + k], x1 = a.xoff[row + k + 1];
      for (int64_t e = x0 + lane; e < x1; e += 32) {
        const int32_t u = a.xcol[e];
        const uint32_t pu = a.prio[u];
        if (pu < pv || (pu == pv && u < v)) {
          const uint32_t wu = __ldcg(&a.word[u]);
          const uint32_t st = wu & 3u, cu = wu >> 2;
          blocked |= (st == kColored && cu == c);
          wait |= (st == kUndecided && cu <= c);
        }
      }
      if (__any_sync(0xffffffffu, blocked)) {
        ++k;
        if (k < L && lane == 0) __stcg(&a.word[v], ((uint32_t)a.lists[row + k] << 2) | kUndecided);
        continue;
      }
      if (__any_sync(0xffffffffu, wait)) {
        if (lane == 0) {
          a.kcur[v] = (uint16_t)k;
          work_out[atomicAdd(nwork_out, 1)] = v;
        }
        break;
      }
      if (lane == 0) __stcg(&a.word[v], (c << 2) | kColored);
      break;
    }
  }
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
__global__ void k_carry_flags(const uint32_t* __restrict__ word, int64_t n, const int32_t* __restrict__ gid,
                              int64_t base, int32_t* __restrict__ color, uint32_t* __restrict__ flag) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const uint32_t w = word[v];
  const uint32_t st = w & 3u;
  if (st == kColored) color[gid ? gid[v] : v] = (int32_t)(base + (int64_t)(w >> 2));
  flag[v] = st == kColored ? 0u : 1u;
}

cudaError_t launch_carry_flags(const uint32_t* word, int64_t n, const int32_t* gid, int64_t base, int32_t* color,
                               uint32_t* flag, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_carry_flags<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(word, n, gid, base, color, flag);
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
