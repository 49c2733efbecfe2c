// kernels_scan.cu -- exclusive prefix sums (reduce / scan-of-partials /
// scan) used to turn per-row and per-run counts into CSR offsets.
#include "common.cuh"

namespace picasso {

namespace {
constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int64_t kChunk = (int64_t)kThreads * kItems;

__device__ __forceinline__ int64_t block_exclusive(int64_t v, int64_t* total) {
  __shared__ int64_t warp_sums[kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int64_t o = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += o;
  }
  if (lane == 31) warp_sums[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int64_t w = lane < kThreads / 32 ? warp_sums[lane] : 0;
    int64_t wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int64_t o = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += o;
    }
    if (lane < kThreads / 32) warp_sums[lane] = wi - w;
    if (lane == kThreads / 32 - 1) *total = wi;
  }
  __syncthreads();
  const int64_t r = warp_sums[wid] + incl - v;
  __syncthreads();
  return r;
}

template <typename T>
__global__ void k_reduce(const T* __restrict__ in, int64_t n, int64_t* __restrict__ partial) {
  const int64_t b0 = (int64_t)blockIdx.x * kChunk;
  int64_t s = 0;
  for (int i = 0; i < kItems; ++i) {
    const int64_t idx = b0 + (int64_t)i * kThreads + threadIdx.x;
    if (idx < n) s += (int64_t)in[idx];
  }
  __shared__ int64_t tot;
  block_exclusive(s, &tot);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <typename T>
__global__ void k_scan(const T* __restrict__ in, int64_t n, const int64_t* __restrict__ base,
                       int64_t* __restrict__ out) {
  const int64_t b0 = (int64_t)blockIdx.x * kChunk + (int64_t)threadIdx.x * kItems;
  int64_t vals[kItems];
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const int64_t idx = b0 + i;
    vals[i] = idx < n ? (int64_t)in[idx] : 0;
    s += vals[i];
  }
  __shared__ int64_t tot;
  int64_t run = block_exclusive(s, &tot) + (base ? base[blockIdx.x] : 0);
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const int64_t idx = b0 + i;
    if (idx < n) out[idx] = run;
    run += vals[i];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kThreads - 1) out[n] = run;
}

int64_t nblocks(int64_t n) { return (n + kChunk - 1) / kChunk; }

template <typename T>
cudaError_t scan_rec(const T* in, int64_t n, int64_t* out, int64_t* tmp, cudaStream_t s) {
  const int64_t nb = nblocks(n);
  if (nb <= 1) {
    k_scan<T><<<1, kThreads, 0, s>>>(in, n, nullptr, out);
    count_launches(1);
    return cudaGetLastError();
  }
  int64_t* partial = tmp;
  int64_t* partial_scan = tmp + nb;
  int64_t* rest = partial_scan + nb + 1;
  k_reduce<T><<<(unsigned)nb, kThreads, 0, s>>>(in, n, partial);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = scan_rec<int64_t>(partial, nb, partial_scan, rest, s);
  if (e != cudaSuccess) return e;
  k_scan<T><<<(unsigned)nb, kThreads, 0, s>>>(in, n, partial_scan, out);
  count_launches(1);
  return cudaGetLastError();
}
}  // namespace

size_t scan_tmp_bytes(int64_t n) {
  size_t words = 0;
  int64_t m = n;
  while (nblocks(m) > 1) {
    const int64_t nb = nblocks(m);
    words += (size_t)(2 * nb + 1);
    m = nb;
  }
  return (words + 16) * sizeof(int64_t);
}

__global__ void k_rinfo_lengths(const int64_t* __restrict__ rinfo, int64_t E, uint32_t* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < E) out[e] = (uint32_t)rinfo_len(rinfo[e]);
}

cudaError_t launch_rinfo_lengths(const int64_t* rinfo, int64_t E, uint32_t* out, cudaStream_t s) {
  if (E <= 0) return cudaSuccess;
  k_rinfo_lengths<<<(unsigned)((E + 255) / 256), 256, 0, s>>>(rinfo, E, out);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_scan_u32(const uint32_t* in, int64_t n, int64_t* out, void* tmp, cudaStream_t s) {
  if (n <= 0) {
    return cudaMemsetAsync(out, 0, sizeof(int64_t), s);
  }
  return scan_rec<uint32_t>(in, n, out, (int64_t*)tmp, s);
}

}  // namespace picasso
