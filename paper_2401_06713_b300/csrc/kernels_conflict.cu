// kernels_conflict.cu -- Alg. 1 construct_conflict_graph on sm_103a.
//
// G_c keeps a pair {u, v} of the round's vertices iff the two strings commute
// (edge of the complement graph G', Sec. II) and their color lists intersect
// (Sec. III-A).  Rows are color-major: row u holds, for each color c of u's
// list in ascending order, the neighbours v that also hold c, ascending in v
// (one "run" per list color).  A pair sharing m colors is listed in m runs of
// each row; the coloring step reads run k to find exactly the neighbours
// that hold the candidate color c_k.
//
// Both strategies below run a count pass (run lengths), an exclusive scan to
// offsets, and a fill pass that writes each run in ascending order -- no
// atomics on output positions, so the CSR is deterministic.
//
//   bucket join   one CTA per color c: the members of bucket c (vertices
//                 holding c) are staged in shared memory and every pair of
//                 members is tested there; the commuting pairs of bucket c
//                 are exactly run c of both rows.
//   all pairs     one warp per row u sweeping every column v (the paper's GPU
//                 kernel tests all |V|(|V|-1)/2 pairs, Sec. IV); the list
//                 intersection is a two-pointer merge.
#include <algorithm>
#include <cstdio>

#include "common.cuh"
#include "bits_device.cuh"
#include "warp_sort.cuh"

namespace picasso {

// ---------------------------------------------------------------------------
// Color buckets
// ---------------------------------------------------------------------------
__global__ void k_bucket_hist(const int32_t* __restrict__ lists, int64_t total, uint32_t* __restrict__ bcount) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&bcount[lists[i]], 1u);
}

cudaError_t launch_bucket_hist(const int32_t* lists, int64_t E, uint32_t* bcount, cudaStream_t s) {
  const int64_t total = E;
  if (total <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 148 * 16);
  k_bucket_hist<<<blocks, 256, 0, s>>>(lists, total, bcount);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void k_bucket_fill(const int32_t* __restrict__ lists, int64_t total, const int64_t* __restrict__ boff,
                              uint32_t* __restrict__ bcursor, int32_t* __restrict__ bmem) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = lists[i];
    const uint32_t pos = atomicAdd(&bcursor[c], 1u);
    bmem[boff[c] + pos] = (int32_t)i;  // list entry: ascending entry is ascending vertex
  }
}

cudaError_t launch_bucket_fill(const int32_t* lists, int64_t E, const int64_t* boff, uint32_t* bcursor,
                               int32_t* bmem, cudaStream_t s) {
  const int64_t total = E;
  if (total <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 148 * 16);
  k_bucket_fill<<<blocks, 256, 0, s>>>(lists, total, boff, bcursor, bmem);
  count_launches(1);
  return cudaGetLastError();
}

// Bucket sizes and places without global atomics.  The list entries are cut
// into G contiguous ranges of at most 65,535 entries (so a color occurs at
// most 65,535 times in one); block b counts its range's colors in shared
// memory (two 16-bit counters a word) and writes them to hist[b] (P rounded
// up to even, 16 bits a color).  A column pass turns hist[b][c] into the
// number of entries of color c in the ranges before b and sums bcount[c].
// The place pass runs over the same ranges, a block per range and slice of
// colors: the block keeps boff[c] + hist[b][c] of its colors in shared memory
// and gives entry e of color c in range b the next place (a shared-memory
// atomic), so each entry costs one global store.  Within a bucket the ranges
// are thus in entry order; the bucket sort orders each range's members.
constexpr int kHistThreads = 1024;
constexpr int64_t kPlaceSlice = 24576;  // colors of one place block (96 KB of places)

int64_t bucket_hist_blocks(int64_t E) {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max<int64_t>(sms, (E + 65534) / 65535);
}

__global__ void __launch_bounds__(kHistThreads) k_bucket_count(const int32_t* __restrict__ lists, int64_t E,
                                                               int64_t P, uint16_t* __restrict__ hist) {
  extern __shared__ uint32_t h2[];  // [(P + 1) / 2]
  const int64_t hw = (P + 1) / 2;
  for (int64_t i = threadIdx.x; i < hw; i += blockDim.x) h2[i] = 0u;
  __syncthreads();
  const int64_t e0 = E * blockIdx.x / gridDim.x, e1 = E * (blockIdx.x + 1) / gridDim.x;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int32_t c = lists[e];
    atomicAdd(&h2[c >> 1], 1u << (16 * (c & 1)));
  }
  __syncthreads();
  uint32_t* out = reinterpret_cast<uint32_t*>(hist + 2 * hw * (int64_t)blockIdx.x);
  for (int64_t i = threadIdx.x; i < hw; i += blockDim.x) out[i] = h2[i];
}

// Block of 256 threads: 32 colors x 8 parts of the ranges (warp w takes
// part w of the ranges for the block's 32 colors, so its loads are
// coalesced); each part's sum goes to shared memory, then every part writes
// its ranges' prefixes from the sum of the parts before it.
constexpr int kColsumParts = 8;
__global__ void __launch_bounds__(256) k_bucket_colsum(uint16_t* __restrict__ hist, int64_t P, int64_t G,
                                                       uint32_t* __restrict__ bcount) {
  __shared__ uint32_t part_sum[kColsumParts][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t stride = 2 * ((P + 1) / 2);
  const int64_t c = (int64_t)blockIdx.x * 32 + lane;
  const int64_t b0 = G * w / kColsumParts, b1 = G * (w + 1) / kColsumParts;
  uint32_t sum = 0;
  if (c < P)
    for (int64_t b = b0; b < b1; ++b) sum += __ldcg(hist + b * stride + c);
  part_sum[w][lane] = sum;
  __syncthreads();
  uint32_t run = 0;
  for (int k = 0; k < w; ++k) run += part_sum[k][lane];
  if (c < P) {
    // 8 ranges at a time: their loads are in flight together
    for (int64_t bb = b0; bb < b1; bb += 8) {
      uint32_t x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = bb + u < b1 ? (uint32_t)__ldcg(hist + (bb + u) * stride + c) : 0u;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (bb + u < b1) hist[(bb + u) * stride + c] = (uint16_t)run;  // exact while a bucket has <= 65,535 members
        run += x[u];
      }
    }
    if (w == kColsumParts - 1) bcount[c] = run;
  }
}

__global__ void __launch_bounds__(kHistThreads) k_bucket_place(const int32_t* __restrict__ lists, int64_t E,
                                                               int64_t P, int npass, const uint16_t* __restrict__ hist,
                                                               const int64_t* __restrict__ boff,
                                                               int32_t* __restrict__ bmem) {
  // block (range b, color slice p): the slice's next free places of range b
  // in shared memory, then the range's entries of those colors
  extern __shared__ uint32_t nxt[];
  const int64_t b = blockIdx.x / npass, p = blockIdx.x % npass;
  const int64_t cp0 = P * p / npass, cp1 = P * (p + 1) / npass;
  const uint16_t* pre = hist + 2 * ((P + 1) / 2) * b;
  for (int64_t c = cp0 + threadIdx.x; c < cp1; c += blockDim.x) nxt[c - cp0] = (uint32_t)(boff[c] + pre[c]);
  __syncthreads();
  const int64_t G = gridDim.x / npass;
  const int64_t e0 = E * b / G, e1 = E * (b + 1) / G;
  // four entries a thread at a time: their loads are in flight together
  for (int64_t e00 = e0; e00 < e1; e00 += 4 * (int64_t)blockDim.x) {
    int32_t c[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t e = e00 + u * (int64_t)blockDim.x + threadIdx.x;
      c[u] = e < e1 ? lists[e] : -1;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (c[u] >= cp0 && c[u] < cp1)
        bmem[atomicAdd(&nxt[c[u] - cp0], 1u)] = (int32_t)(e00 + u * (int64_t)blockDim.x + threadIdx.x);
  }
}

cudaError_t launch_bucket_count(const int32_t* lists, int64_t E, int64_t P, uint16_t* hist, int64_t G,
                                uint32_t* bcount, cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  if (P > kHistMaxP || G < 1 || E > 65535 * G) return cudaErrorInvalidValue;
  const size_t smem = sizeof(uint32_t) * (size_t)((P + 1) / 2);
  cudaError_t e = cudaFuncSetAttribute(k_bucket_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_bucket_count<<<(unsigned)G, kHistThreads, smem, s>>>(lists, E, P, hist);
  k_bucket_colsum<<<(unsigned)((P + 31) / 32), 256, 0, s>>>(hist, P, G, bcount);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_bucket_place(const int32_t* lists, int64_t E, int64_t P, const uint16_t* hist, int64_t G,
                                const int64_t* boff, int32_t* bmem, cudaStream_t s) {
  if (E <= 0 || P <= 0) return cudaSuccess;
  if (P > kHistMaxP || G < 1 || E > 65535 * G) return cudaErrorInvalidValue;
  // color slices of at most kPlaceSlice colors: two blocks per SM
  const int npass = (int)((P + kPlaceSlice - 1) / kPlaceSlice);
  const size_t smem = sizeof(uint32_t) * (size_t)((P + npass - 1) / npass);
  cudaError_t e = cudaFuncSetAttribute(k_bucket_place, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_bucket_place<<<(unsigned)(G * npass), kHistThreads, smem, s>>>(lists, E, P, npass, hist, boff, bmem);
  count_launches(1);
  return cudaGetLastError();
}

// Ascending order inside each bucket.  Buckets of up to 512 members: one warp
// per bucket, the keys in registers (lane l holds elements l*E .. l*E+E-1,
// E = m/32 for the padded size m): a bitonic network (partners closer than E
// in the same lane, farther ones exchanged by shuffles), or, with near (the
// members were placed by ranges, so each sits within a few places of its
// own), odd-even transposition passes that fall back to the network.
// Larger buckets: one CTA per bucket, the network in shared memory
// (k_bucket_sort).  GATHER (the bit pass, buckets of at most kWarpSortMax
// members): the same warp then writes the sorted members' words and vertex
// ids in slot order (bxz, bpid).
template <bool GATHER>
__global__ void __launch_bounds__(256, 4) k_bucket_sort_warp(const int64_t* __restrict__ boff, int64_t P,
                                                          int32_t* __restrict__ bmem, ConflictArgs a,
                                                          uint4* __restrict__ bxz, int32_t* __restrict__ bpid,
                                                          int near) {
  // the warp's bucket in shared memory (one pad word every 16), so that the
  // global reads and writes are coalesced and the lanes' runs of E
  // consecutive elements are read without bank conflicts
  __shared__ int32_t sbuf[8][kWarpSortMax + kWarpSortMax / 16];
  const int lane = threadIdx.x & 31;
  int32_t* sp = sbuf[(threadIdx.x >> 5) & 7];
  const int64_t gw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < P; b += gw) {
    const int64_t o = boff[b];
    const int s = (int)(boff[b + 1] - o);
    if (s > kWarpSortMax) continue;
    int32_t* p = bmem + o;
    __syncwarp();
    for (int i = lane; i < s; i += 32) sp[sort_at<true>(i)] = p[i];
    __syncwarp();
    if (s <= 1)
      ;
    else if (s <= 32)
      warp_sort_bucket<1, true>(sp, s, lane);
    else if (near) {
      if (s <= 64)
        warp_fix_bucket<2, true>(sp, s, lane);
      else if (s <= 128)
        warp_fix_bucket<4, true>(sp, s, lane);
      else if (s <= 256)
        warp_fix_bucket<8, true>(sp, s, lane);
      else
        warp_fix_bucket<16, true>(sp, s, lane);
    } else if (s <= 64)
      warp_sort_bucket<2, true>(sp, s, lane);
    else if (s <= 128)
      warp_sort_bucket<4, true>(sp, s, lane);
    else if (s <= 256)
      warp_sort_bucket<8, true>(sp, s, lane);
    else
      warp_sort_bucket<16, true>(sp, s, lane);
    __syncwarp();
    if (!GATHER) {
      for (int i = lane; i < s; i += 32) p[i] = sp[sort_at<true>(i)];
    } else {
      // four members a lane at a time, every load issued before the stores
      // (the words are 16-byte aligned: x, z of a vertex side by side)
      for (int i0 = 0; i0 < s; i0 += 128) {
        int32_t f[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + 32 * u + lane;
          f[u] = i < s ? sp[sort_at<true>(i)] : -1;
        }
        int32_t v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = f[u] < 0 ? 0 : (a.Lu ? f[u] / a.Lu : a.ent_v[f[u]]);
        uint4 w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          w[u] = f[u] < 0 ? make_uint4(0u, 0u, 0u, 0u) : __ldg(reinterpret_cast<const uint4*>(a.xz + 2 * (int64_t)v[u]));
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + 32 * u + lane;
          if (f[u] >= 0) {
            p[i] = f[u];
            bxz[o + i] = w[u];
            bpid[o + i] = v[u];
          }
        }
      }
    }
  }
}

__global__ void __launch_bounds__(512) k_bucket_sort(const int64_t* __restrict__ boff, int64_t P,
                                                     int32_t* __restrict__ bmem, int32_t* err) {
  __shared__ int32_t key[kBucketCap];
  for (int64_t b = blockIdx.x; b < P; b += gridDim.x) {
    const int64_t o = boff[b];
    const int s = (int)(boff[b + 1] - o);
    if (s <= kWarpSortMax) continue;
    if (s > kBucketCap) {
      if (threadIdx.x == 0) atomicExch(err, 1);
      continue;
    }
    int m = 1;
    while (m < s) m <<= 1;
    for (int i = threadIdx.x; i < m; i += blockDim.x) key[i] = i < s ? bmem[o + i] : 0x7fffffff;
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
          const int p = i ^ j;
          if (p > i) {
            const bool up = (i & k) == 0;
            const int32_t a = key[i], c = key[p];
            if ((a > c) == up) {
              key[i] = c;
              key[p] = a;
            }
          }
        }
        __syncthreads();
      }
    }
    for (int i = threadIdx.x; i < s; i += blockDim.x) bmem[o + i] = key[i];
    __syncthreads();
  }
}

cudaError_t launch_bucket_sort(const int64_t* boff, int64_t P, int32_t* bmem, int32_t* err, int32_t smax, bool near,
                               cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  const unsigned wblocks = (unsigned)std::min<int64_t>((P + 7) / 8, 148 * 16);
  k_bucket_sort_warp<false><<<wblocks, 256, 0, s>>>(boff, P, bmem, ConflictArgs{}, nullptr, nullptr, near ? 1 : 0);
  count_launches(1);
  if (smax > kWarpSortMax) {
    const unsigned blocks = (unsigned)std::min<int64_t>(P, 148 * 8);
    k_bucket_sort<<<blocks, 256, 0, s>>>(boff, P, bmem, err);
    count_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_bucket_sort_gather(const int64_t* boff, int64_t P, int32_t* bmem, int32_t smax, bool near,
                                      const ConflictArgs& a, uint4* bxz, int32_t* bpid, cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  if (smax > kWarpSortMax) return cudaErrorInvalidValue;
  // a member's words are read 16 bytes at a time
  if (reinterpret_cast<uintptr_t>(a.xz) & 15) return cudaErrorMisalignedAddress;
  const unsigned wblocks = (unsigned)std::min<int64_t>((P + 7) / 8, 148 * 16);
  k_bucket_sort_warp<true><<<wblocks, 256, 0, s>>>(boff, P, bmem, a, bxz, bpid, near ? 1 : 0);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void k_bucket_stats(const uint32_t* __restrict__ in, int64_t n, uint32_t* out32,
                               unsigned long long* out64) {
  uint32_t m = 0;
  unsigned long long q = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t x = in[i];
    m = max(m, x);
    q += (unsigned long long)x * (x > 0 ? x - 1 : 0);
  }
  for (int d = 16; d; d >>= 1) {
    m = max(m, __shfl_xor_sync(0xffffffffu, m, d));
    q += __shfl_xor_sync(0xffffffffu, q, d);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out32, m);
    atomicAdd(out64, q);
  }
}

cudaError_t launch_bucket_stats(const uint32_t* bcount, int64_t P, uint32_t* out32, unsigned long long* out64,
                                cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out32, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(out64, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess || P <= 0) return e;
  const unsigned blocks = (unsigned)std::min<int64_t>((P + 255) / 256, 148 * 4);
  k_bucket_stats<<<blocks, 256, 0, s>>>(bcount, P, out32, out64);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Bucket join
//
// Inside a bucket the commutation relation of all member pairs is a GF(2)
// bilinear form: bit(u, v) = parity(popc((x_u & z_v) ^ (z_u & x_v))) =
// sum_k x_u[k] z_v[k] + z_u[k] x_v[k] mod 2.  It is evaluated 32 x 32 pairs
// at a time by the "four Russians" method: for a block of 32 rows, the rows'
// bits are transposed into 32-bit columns a_k (bit r = bit k of row r) and,
// for every 4-bit chunk of the 128 (x|z) positions, the 16 XOR combinations
// of the chunk's four columns go to a shared-memory table.  A partner v then
// gets all 32 of its row bits with one table lookup per chunk, indexed by the
// chunk's 4 bits of v's (z|x) words: 32 lookups and 16 XORs for 32 pairs,
// where a direct test costs a POPC per pair.  The 16-entry tables sit in 16
// consecutive banks, so the warp's lookups never conflict.
//
// Mask words are stored block-major: the word of member row r (block R = r/32)
// for partners of block W is at base + (R * nwb + W) * 32 + (r % 32), so each
// 32 x 32 block is one coalesced 128-byte line.  When rows keep only their
// smaller-id partners (lower), only blocks W <= R exist, at base +
// (R (R + 1) / 2 + W) * 32 + (r % 32).
// ---------------------------------------------------------------------------
namespace {

constexpr int kMaskThreads = 256;
constexpr int kMaskWarps = kMaskThreads / 32;
constexpr int kEmitThreads = 256;

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline size_t mask_smem_bytes(int smax) {
  const int nwb = (smax + 31) >> 5;
  return align16(sizeof(uint4) * smax) + align16(sizeof(int32_t) * smax) * 2 + 256 +
         sizeof(uint32_t) * ((size_t)nwb * 128 + 64 + (size_t)kMaskWarps * kTabWords);
}

// The bit pass keeps a bucket's lower blocks row-major in shared memory: row
// r of block R at rm_pad_off(R) + r ((R + 1) | 1) + W (odd row strides, so a
// warp's 32 rows hit 32 banks), then copies them to HBM row-major without
// the padding: row r of block R at 16 R (R + 1) + r (R + 1).
__host__ __device__ inline int rm_pad_off(int R) { return 32 * (R * (R + 1) / 2 + R / 2); }

// Asynchronous global -> shared copies (the next bucket's members).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace

// Mask pass over one bucket per CTA iteration:
//  1. the members' words to shared memory;
//  2. bit columns of every 32-row block;
//  3. the blocks (I, J >= I) of the upper triangle, split evenly over the
//     warps: lane j of block (I, J) gets the word of row J*32+j against rows
//     I*32.. (commuting, i != j); a warp transpose gives the words of rows
//     I*32.. against partners J*32..; the relation is symmetric, so each
//     unordered pair is tested once.
// Per-row counts go to cnt at the member's list entry (the run of this
// bucket's color in the member's row).
__device__ __forceinline__ int mask_block(bool lower, int R, int W, int nwb) {
  return lower ? R * (R + 1) / 2 + W : R * nwb + W;
}

constexpr int kEmitChunk = 16;

// Rows of one staged chunk of NI partner words: lane rr keeps row rr's
// cursor; every lane reads it by shuffle, writes its partner if its bit is
// set, and the row's cursor advances by the word's popcount.
template <int NI>
__device__ __forceinline__ void emit_rows(const uint32_t* __restrict__ wbuf, const int32_t (&pv)[kEmitChunk],
                                          int64_t& rc, int nrows, int32_t* __restrict__ col, int lane, uint32_t lt,
                                          uint32_t rows = 0xffffffffu) {
  const uint32_t lbit = 1u << lane;
  for (int rr = 0; rr < nrows; ++rr) {
    if (!((rows >> rr) & 1u)) continue;
    int32_t* dst = col + __shfl_sync(0xffffffffu, rc, rr);
    int32_t at = 0;
#pragma unroll
    for (int t = 0; t < NI; ++t) {
      const uint32_t w = wbuf[t * 32 + rr];
      // predicated store: lane i writes partner i when bit i is set
      asm volatile(
          "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %0, 0;\n\t@p st.global.b32 [%1], %2;\n\t}"
          :
          : "r"(w & lbit), "l"(dst + at + __popc(w & lt)), "r"(pv[t]));
      at += __popc(w);
    }
    if (lane == rr) rc += at;
  }
}

// The unfused mask pass: members read through bmem and the strings; blocks
// (block-major) and per-entry counts to HBM, for the emit pass.
template <int QW, bool LOWER>
__global__ void __launch_bounds__(kMaskThreads, 4) k_bucket_mask(ConflictArgs a, const int64_t* __restrict__ boff,
                                                              const int32_t* __restrict__ bmem,
                                                              const int64_t* __restrict__ moff, int smax) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  uint8_t* p = smem_raw;
  uint4* w4 = (uint4*)p;
  p += align16(sizeof(uint4) * smax);
  int32_t* sfl = (int32_t*)p;
  p += align16(sizeof(int32_t) * smax);
  int32_t* cnt = (int32_t*)p;
  p += align16(sizeof(int32_t) * smax);
  // 256-byte aligned region: bit columns, then per-warp tables (table bases
  // need a zero low byte)
  {
    const uint32_t ad = (uint32_t)__cvta_generic_to_shared(p);
    p += (256u - (ad & 255u)) & 255u;
  }
  uint32_t* colw = (uint32_t*)p;  // [nwb][2 QW][32]
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t b = blockIdx.x; b < a.P; b += gridDim.x) {
    const int64_t o = boff[b];
    const int s = (int)(boff[b + 1] - o);
    if (s == 0) continue;
    for (int i = threadIdx.x; i < s; i += kMaskThreads) {
      const int32_t flat = bmem[o + i];
      const int64_t v = a.Lu ? flat / a.Lu : a.ent_v[flat];
      const uint64_t x = a.xz[2 * v], z = a.xz[2 * v + 1];
      w4[i] = make_uint4((uint32_t)x, (uint32_t)(x >> 32), (uint32_t)z, (uint32_t)(z >> 32));
      sfl[i] = flat;
      cnt[i] = 0;
    }
    __syncthreads();
    const int nwb = (s + 31) >> 5;
    for (int I = wid; I < nwb; I += kMaskWarps) {
      const int r = (I << 5) + lane;
      const uint4 w = r < s ? w4[r] : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
      for (int g = 0; g < 2 * QW; ++g) colw[(I * 2 * QW + g) * 32 + lane] = transpose32(word_of<QW>(w, g), lane);
    }
    const uint32_t tab_off = ((uint32_t)(nwb * 2 * QW * 32) + 63u) & ~63u;  // words; 256-byte aligned
    uint32_t* tab = colw + tab_off + wid * kTabWords;
    const uint32_t tab_addr = (uint32_t)__cvta_generic_to_shared(tab);
    __syncthreads();

    uint32_t* rmb = a.rmask + moff[b];
    const int nblk = nwb * (nwb + 1) / 2;  // blocks (I, J >= I)
    const int q0 = (int)((int64_t)nblk * wid / kMaskWarps), q1 = (int)((int64_t)nblk * (wid + 1) / kMaskWarps);
    int I = 0, J = 0;
    {
      int rem = q0;
      while (rem >= nwb - I) {
        rem -= nwb - I;
        ++I;
      }
      J = I + rem;
    }
    int tab_I = -1;
    for (int q = q0; q < q1; ++q) {
      if (tab_I != I) {
        build_tables<QW>(colw + I * 2 * QW * 32, tab, lane);
        tab_I = I;
      }
      const int ib = I << 5;
      const int j = (J << 5) + lane;
      const bool jv = j < s;
      const uint4 cwj = jv ? w4[j] : make_uint4(0u, 0u, 0u, 0u);
      const uint32_t anti = lookup<QW>(cwj, tab_addr);
      const uint32_t rows_ok = s - ib >= 32 ? 0xffffffffu : ((1u << (s - ib)) - 1u);
      uint32_t cw = jv ? (~anti & rows_ok) : 0u;
      // the diagonal block: no self pair; lower rows keep smaller partners
      if (I == J) cw &= LOWER ? ((1u << lane) - 1u) : ~(1u << lane);
      rmb[mask_block(LOWER, J, I, nwb) * 32 + lane] = cw;
      if (cw) atomicAdd(&cnt[j], __popc(cw));
      if (!LOWER && I != J) {
        const uint32_t tr = transpose32(cw, lane);
        rmb[(I * nwb + J) * 32 + lane] = tr;
        if (tr) atomicAdd(&cnt[ib + lane], __popc(tr));
      }
      if (++J == nwb) {
        ++I;
        J = I;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < s; i += kMaskThreads) a.cnt[sfl[i]] = (uint32_t)cnt[i];
    __syncthreads();
  }
}

// The bit pass (the default build; EARLIER form, buckets of at most
// kFusedMax members, strings of one word per part).  A CTA takes buckets
// b, b + G, ...; a bucket's members (words and entry ids, gathered in slot
// order beforehand) arrive by cp.async in one of two buffers while the CTA
// works on the other.  Per bucket, three CTA barriers:
//   1. (the bucket's members have landed; the previous bucket is done) warps
//      make the bit columns of the row blocks (warp transposes);
//   2. (columns done) every warp takes an even share of the lower blocks
//      (I, J >= I), builds the nibble tables of each row block I it meets,
//      and gets, by lookup, the word of row J*32 + lane against rows I*32 ..
//      (commuting, smaller slot), stored row-major in shared memory (odd row
//      strides), with the row's run length counted;
//   3. (every row is complete) the next bucket's copy starts; each entry's
//      packed word (row address, slot, run length), the bucket's run total,
//      and the rows to HBM row-major.
__host__ __device__ inline size_t bits2_smem_bytes(int smax) {
  const int nwb = (smax + 31) >> 5;
  return align16(sizeof(uint4) * 2 * smax) + align16(sizeof(int32_t) * 2 * smax) + align16(sizeof(int32_t) * smax) +
         sizeof(uint32_t) * (size_t)rm_pad_off(nwb) + 256 +
         sizeof(uint32_t) * ((size_t)kMaskWarps * kTabWords + (size_t)nwb * 128);
}

template <int QW>
__global__ void __launch_bounds__(kMaskThreads, 4) k_bucket_bits(ConflictArgs a, const int64_t* __restrict__ boff,
                                                              const int32_t* __restrict__ bmem,
                                                              const int64_t* __restrict__ moff, int smax) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  uint8_t* p = smem_raw;
  uint4* w4b = (uint4*)p;  // [2][smax]
  p += align16(sizeof(uint4) * 2 * smax);
  int32_t* sflb = (int32_t*)p;  // [2][smax]
  p += align16(sizeof(int32_t) * 2 * smax);
  int32_t* cnt = (int32_t*)p;  // [smax], zero between buckets
  p += align16(sizeof(int32_t) * smax);
  uint32_t* mwp = (uint32_t*)p;
  p += sizeof(uint32_t) * (size_t)rm_pad_off((smax + 31) >> 5);
  {
    // table bases need a zero low byte
    const uint32_t ad = (uint32_t)__cvta_generic_to_shared(p);
    p += (256u - (ad & 255u)) & 255u;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t* tab = (uint32_t*)p + wid * kTabWords;
  const uint32_t tab_addr = (uint32_t)__cvta_generic_to_shared(tab);
  uint32_t* colw = (uint32_t*)p + kMaskWarps * kTabWords;  // [nwb][2 QW][32] bit columns

  for (int i = threadIdx.x; i < smax; i += kMaskThreads) cnt[i] = 0;
  auto fetch = [&](int64_t b, int buf) {
    if (b >= a.P) return;
    const int64_t o = boff[b];
    const int sn = (int)(boff[b + 1] - o);
    for (int i = threadIdx.x; i < sn; i += kMaskThreads) {
      cp_async16(w4b + buf * smax + i, a.bxz + o + i);
      cp_async4(sflb + buf * smax + i, bmem + o + i);
    }
    cp_async_commit();
  };
  fetch(blockIdx.x, 0);
  int buf = 0;
  for (int64_t b = blockIdx.x; b < a.P; b += gridDim.x, buf ^= 1) {
    cp_async_wait_all();
    __syncthreads();
    const int64_t o = boff[b];
    const int s = (int)(boff[b + 1] - o);
    if (s == 0) {
      fetch(b + gridDim.x, buf ^ 1);
      continue;
    }
    const uint4* w4 = w4b + buf * smax;
    const int32_t* sfl = sflb + buf * smax;
    const int nwb = (s + 31) >> 5;
    for (int I = wid; I < nwb; I += kMaskWarps) {
      const int r = (I << 5) + lane;
      const uint4 w = r < s ? w4[r] : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
      for (int g = 0; g < 2 * QW; ++g) colw[(I * 2 * QW + g) * 32 + lane] = transpose32(word_of<QW>(w, g), lane);
    }
    __syncthreads();
    const int nblk = nwb * (nwb + 1) / 2;
    const int q0 = (int)((int64_t)nblk * wid / kMaskWarps), q1 = (int)((int64_t)nblk * (wid + 1) / kMaskWarps);
    int I = 0, J = 0;
    {
      int rem = q0;
      while (rem >= nwb - I) {
        rem -= nwb - I;
        ++I;
      }
      J = I + rem;
    }
    int tab_I = -1;
    for (int q = q0; q < q1; ++q) {
      if (tab_I != I) {
        build_tables<QW>(colw + I * 2 * QW * 32, tab, lane);
        tab_I = I;
      }
      const int ib = I << 5;
      const int j = (J << 5) + lane;
      const bool jv = j < s;
      const uint4 cwj = jv ? w4[j] : make_uint4(0u, 0u, 0u, 0u);
      const uint32_t anti = lookup<QW>(cwj, tab_addr);
      const uint32_t rows_ok = s - ib >= 32 ? 0xffffffffu : ((1u << (s - ib)) - 1u);
      uint32_t cw = jv ? (~anti & rows_ok) : 0u;
      // the diagonal block: no self pair, smaller partners only
      if (I == J) cw &= (1u << lane) - 1u;
      mwp[rm_pad_off(J) + lane * ((J + 1) | 1) + I] = cw;
      if (cw) atomicAdd(&cnt[j], __popc(cw));
      if (++J == nwb) {
        ++I;
        J = I;
      }
    }
    __syncthreads();
    // the next bucket's copy (the lookups, which share the shared-memory
    // pipe with it, are done)
    fetch(b + gridDim.x, buf ^ 1);
    // entry of member i: its row's first word, i and its run length; the
    // bucket's run total to *a.nnz
    uint32_t tot = 0;
    for (int i = threadIdx.x; i < s; i += kMaskThreads) {
      const int R = i >> 5;
      const int64_t w0 = moff[b] + 16 * R * (R + 1) + (i & 31) * (R + 1);
      const int ci = cnt[i];
      a.rinfo[sfl[i]] = rinfo_pack(w0, i, ci);
      cnt[i] = 0;
      tot += (uint32_t)ci;
    }
    tot = __reduce_add_sync(0xffffffffu, tot);
    if (lane == 0 && tot) atomicAdd(a.nnz, (unsigned long long)tot);
    // the rows to HBM, row-major: warp per row block, 32 words a step
    uint32_t* rmb = a.rmask + moff[b];
    for (int R = wid; R < nwb; R += kMaskWarps) {
      const uint32_t d = (uint32_t)(R + 1), m = (65536u + d - 1u) / d, sp = d | 1u;
      const uint32_t* src = mwp + rm_pad_off(R);
      uint32_t* dst = rmb + 16 * R * (R + 1);
      for (uint32_t o2 = lane; o2 < 32u * d; o2 += 32u) {
        const uint32_t r = (o2 * m) >> 16, w = o2 - r * d;  // o2 = r d + w (exact for o2 < 32 d, d <= 16)
        dst[o2] = src[r * sp + w];
      }
    }
  }
  cp_async_wait_all();
}

// Mask pass for strings of more than one word per part (q > 64): the
// outputs of the plain k_bucket_mask (mask blocks and per-entry counts)
// from a direct symplectic form per pair.  Block (I, J >= I) of the upper
// triangle goes to one warp; lane j keeps partner J*32+j's words in
// registers and every row I*32+r of the block is read from shared memory
// as a broadcast, so a warp forms 32 pairs per row.  WM >= qw words per part.
template <int WM, bool LOWER>
__global__ void __launch_bounds__(kMaskThreads) k_bucket_mask_wide(ConflictArgs a, const int64_t* __restrict__ boff,
                                                                   const int32_t* __restrict__ bmem,
                                                                   const int64_t* __restrict__ moff, int smax) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int W = a.qw, S = 2 * W;
  uint64_t* wv = reinterpret_cast<uint64_t*>(smem_raw);  // [smax][S] member words
  int32_t* sfl = reinterpret_cast<int32_t*>(wv + (size_t)smax * S);
  int32_t* cnt = sfl + smax;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t b = blockIdx.x; b < a.P; b += gridDim.x) {
    const int64_t o = boff[b];
    const int s = (int)(boff[b + 1] - o);
    if (s == 0) continue;
    for (int i = threadIdx.x; i < s; i += kMaskThreads) {
      sfl[i] = bmem[o + i];
      cnt[i] = 0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < s * S; t += kMaskThreads) {
      const int i = t / S, w = t - i * S;
      const int32_t flat = sfl[i];
      const int64_t v = a.Lu ? flat / a.Lu : a.ent_v[flat];
      wv[t] = a.xz[(int64_t)S * v + w];
    }
    __syncthreads();
    const int nwb = (s + 31) >> 5;
    const int nblk = nwb * (nwb + 1) / 2;
    uint32_t* rmb = a.rmask + moff[b];
    for (int qb = wid; qb < nblk; qb += kMaskWarps) {
      int I = 0, rem = qb;
      while (rem >= nwb - I) {
        rem -= nwb - I;
        ++I;
      }
      const int J = I + rem;
      const int ib = I << 5, j = (J << 5) + lane;
      const bool jv = j < s;
      uint64_t px[WM], pz[WM];
#pragma unroll
      for (int w = 0; w < WM; ++w) {
        px[w] = (jv && w < W) ? wv[(size_t)j * S + w] : 0ull;
        pz[w] = (jv && w < W) ? wv[(size_t)j * S + W + w] : 0ull;
      }
      const int nr = min(32, s - ib);
      uint32_t anti = 0u;
      for (int r = 0; r < nr; ++r) {
        const uint64_t* rw = wv + (size_t)(ib + r) * S;
        uint64_t acc = 0ull;
#pragma unroll
        for (int w = 0; w < WM; ++w)
          if (w < W) acc ^= (rw[w] & pz[w]) ^ (rw[W + w] & px[w]);
        anti |= (uint32_t)(__popcll(acc) & 1) << r;
      }
      const uint32_t rows_ok = nr >= 32 ? 0xffffffffu : ((1u << nr) - 1u);
      uint32_t cw = jv ? (~anti & rows_ok) : 0u;
      // the diagonal block: no self pair; lower rows keep smaller partners
      if (I == J) cw &= LOWER ? ((1u << lane) - 1u) : ~(1u << lane);
      rmb[mask_block(LOWER, J, I, nwb) * 32 + lane] = cw;
      if (cw) atomicAdd(&cnt[j], __popc(cw));
      if (!LOWER && I != J) {
        const uint32_t tr = transpose32(cw, lane);
        rmb[(I * nwb + J) * 32 + lane] = tr;
        if (tr) atomicAdd(&cnt[ib + lane], __popc(tr));
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < s; i += kMaskThreads) a.cnt[sfl[i]] = (uint32_t)cnt[i];
    __syncthreads();
  }
}

// Wide mask pass with nibble tables, for strings of 2 to kWideTabSlices
// words per part.  The symplectic form is a sum over 64-qubit slices, so a
// 32 x 32 anticommutation block is the XOR over slices of the q <= 64
// lookups: a warp keeps one table set per slice for its current row block
// (the bit columns of the block's rows, transposed in the warp), and each
// partner word group costs the lookups of the one-word pass.  Members' words
// are staged slice-major as (x lo, x hi, z lo, z hi).  Same outputs as the
// plain k_bucket_mask.
template <bool LOWER>
__global__ void __launch_bounds__(kMaskThreads) k_bucket_mask_wtab(ConflictArgs a, const int64_t* __restrict__ boff,
                                                                   const int32_t* __restrict__ bmem,
                                                                   const int64_t* __restrict__ moff, int smax) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int W = a.qw, S = 2 * W;
  uint8_t* p = smem_raw;
  uint4* wv4 = (uint4*)p;  // [W][smax]
  p += align16(sizeof(uint4) * (size_t)W * smax);
  int32_t* sfl = (int32_t*)p;
  p += align16(sizeof(int32_t) * smax);
  int32_t* cnt = (int32_t*)p;
  p += align16(sizeof(int32_t) * smax);
  {
    const uint32_t ad = (uint32_t)__cvta_generic_to_shared(p);
    p += (256u - (ad & 255u)) & 255u;  // table bases need a zero low byte
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // per warp: W table sets, then the bit columns of one slice [4][32]
  uint32_t* tab = (uint32_t*)p + (size_t)wid * (W * kTabWords + 128);
  uint32_t* colw = tab + W * kTabWords;
  const uint32_t tab_addr = (uint32_t)__cvta_generic_to_shared(tab);
  const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
  for (int64_t b = blockIdx.x; b < a.P; b += gridDim.x) {
    const int64_t o = boff[b];
    const int s = (int)(boff[b + 1] - o);
    if (s == 0) continue;
    for (int i = threadIdx.x; i < s; i += kMaskThreads) {
      sfl[i] = bmem[o + i];
      cnt[i] = 0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < s * W; t += kMaskThreads) {
      const int i = t / W, k = t - i * W;
      const int32_t flat = sfl[i];
      const int64_t v = a.Lu ? flat / a.Lu : a.ent_v[flat];
      const uint64_t x = a.xz[(int64_t)S * v + k], z = a.xz[(int64_t)S * v + W + k];
      wv4[(size_t)k * smax + i] = make_uint4((uint32_t)x, (uint32_t)(x >> 32), (uint32_t)z, (uint32_t)(z >> 32));
    }
    __syncthreads();
    const int nwb = (s + 31) >> 5;
    const int nblk = nwb * (nwb + 1) / 2;
    uint32_t* rmb = a.rmask + moff[b];
    // a contiguous range of upper-triangle blocks (I, J >= I) per warp, so a
    // row block's tables serve several partner blocks
    const int q0 = (int)((int64_t)nblk * wid / kMaskWarps), q1 = (int)((int64_t)nblk * (wid + 1) / kMaskWarps);
    int I = 0, J = 0;
    {
      int rem = q0;
      while (rem >= nwb - I) {
        rem -= nwb - I;
        ++I;
      }
      J = I + rem;
    }
    int tab_I = -1;
    for (int q = q0; q < q1; ++q) {
      if (tab_I != I) {
        const int r = (I << 5) + lane;
        for (int k = 0; k < W; ++k) {
          const uint4 w = r < s ? wv4[(size_t)k * smax + r] : zero4;
#pragma unroll
          for (int g = 0; g < 4; ++g) colw[g * 32 + lane] = transpose32(word_of<2>(w, g), lane);
          build_tables<2>(colw, tab + k * kTabWords, lane);
        }
        tab_I = I;
      }
      const int ib = I << 5;
      const int j = (J << 5) + lane;
      const bool jv = j < s;
      uint32_t anti = 0u;
      for (int k = 0; k < W; ++k) {
        const uint4 cwj = jv ? wv4[(size_t)k * smax + j] : zero4;
        anti ^= lookup<2>(cwj, tab_addr + (uint32_t)(k * kTabWords * 4));
      }
      const int nr = min(32, s - ib);
      const uint32_t rows_ok = nr >= 32 ? 0xffffffffu : ((1u << nr) - 1u);
      uint32_t cw = jv ? (~anti & rows_ok) : 0u;
      // the diagonal block: no self pair; lower rows keep smaller partners
      if (I == J) cw &= LOWER ? ((1u << lane) - 1u) : ~(1u << lane);
      rmb[mask_block(LOWER, J, I, nwb) * 32 + lane] = cw;
      if (cw) atomicAdd(&cnt[j], __popc(cw));
      if (!LOWER && I != J) {
        const uint32_t tr = transpose32(cw, lane);
        rmb[(I * nwb + J) * 32 + lane] = tr;
        if (tr) atomicAdd(&cnt[ib + lane], __popc(tr));
      }
      if (++J == nwb) {
        ++I;
        J = I;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < s; i += kMaskThreads) a.cnt[sfl[i]] = (uint32_t)cnt[i];
    __syncthreads();
  }
}

size_t wtab_mask_smem_bytes(int64_t smax, int32_t qw) {
  return align16(sizeof(uint4) * (size_t)qw * smax) + 2 * align16(sizeof(int32_t) * smax) + 256 +
         sizeof(uint32_t) * (size_t)kMaskWarps * (qw * kTabWords + 128);
}

size_t wide_mask_smem_bytes(int64_t smax, int32_t qw) { return (size_t)smax * (16 * (size_t)qw + 8); }

bool wide_mask_fits(int64_t smax, int32_t qw) {
  if (qw <= kWideTabSlices && wtab_mask_smem_bytes(smax, qw) <= kWideTabSmem) return true;
  return wide_mask_smem_bytes(smax, qw) <= kWideMaskSmem;
}

static cudaError_t launch_mask_wtab(const ConflictArgs& a, const int64_t* boff, const int32_t* bmem,
                                    const int64_t* moff, int32_t smax, cudaStream_t s) {
  const size_t bytes = wtab_mask_smem_bytes(smax, a.qw);
  auto kern = a.lower ? k_bucket_mask_wtab<true> : k_bucket_mask_wtab<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMaskThreads, bytes);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = debug_grid(std::min<int64_t>(a.P, (int64_t)sms * max(per_sm, 1)));
  kern<<<(unsigned)blocks, kMaskThreads, bytes, s>>>(a, boff, bmem, moff, smax);
  count_launches(1);
  return cudaGetLastError();
}

template <int WM>
static cudaError_t launch_mask_wide(const ConflictArgs& a, const int64_t* boff, const int32_t* bmem,
                                    const int64_t* moff, int32_t smax, cudaStream_t s) {
  const size_t bytes = wide_mask_smem_bytes(smax, a.qw);
  if (bytes > kWideMaskSmem) return cudaErrorInvalidValue;
  auto kern = a.lower ? k_bucket_mask_wide<WM, true> : k_bucket_mask_wide<WM, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMaskThreads, bytes);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = debug_grid(std::min<int64_t>(a.P, (int64_t)sms * max(per_sm, 1)));
  kern<<<(unsigned)blocks, kMaskThreads, bytes, s>>>(a, boff, bmem, moff, smax);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_bucket_bits(const ConflictArgs& a, const int64_t* boff, const int32_t* bmem, const int64_t* moff,
                               int32_t smax, int32_t q, cudaStream_t s, int per_sm_cap) {
  if (a.P <= 0 || a.n <= 0) return cudaSuccess;
  if (smax > kFusedMax || !a.lower || a.qw != 1) return cudaErrorInvalidValue;
  smax = max(smax, 1);
  const size_t bytes = bits2_smem_bytes(smax);
  auto kern = q <= 32 ? k_bucket_bits<1> : k_bucket_bits<2>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMaskThreads, bytes);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (per_sm_cap > 0) per_sm = min(per_sm, per_sm_cap);
  const int64_t blocks = debug_grid(std::min<int64_t>(a.P, (int64_t)sms * max(per_sm, 1)));
  kern<<<(unsigned)blocks, kMaskThreads, bytes, s>>>(a, boff, bmem, moff, smax);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_bucket_mask(const ConflictArgs& a, const int64_t* boff, const int32_t* bmem, const int64_t* moff,
                               int32_t smax, int32_t q, cudaStream_t s) {
  if (a.P <= 0 || a.n <= 0) return cudaSuccess;
  smax = max(smax, 1);
  if (a.qw > 1) {
    if (a.qw <= kWideTabSlices && wtab_mask_smem_bytes(smax, a.qw) <= kWideTabSmem)
      return launch_mask_wtab(a, boff, bmem, moff, smax, s);
    if (a.qw <= 2) return launch_mask_wide<2>(a, boff, bmem, moff, smax, s);
    if (a.qw <= 4) return launch_mask_wide<4>(a, boff, bmem, moff, smax, s);
    if (a.qw <= 8) return launch_mask_wide<8>(a, boff, bmem, moff, smax, s);
    if (a.qw <= 16) return launch_mask_wide<16>(a, boff, bmem, moff, smax, s);
    return cudaErrorInvalidValue;
  }
  const size_t bytes = mask_smem_bytes(smax);
  auto kern = q <= 32 ? (a.lower ? k_bucket_mask<1, true> : k_bucket_mask<1, false>)
                      : (a.lower ? k_bucket_mask<2, true> : k_bucket_mask<2, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMaskThreads, bytes);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = debug_grid(std::min<int64_t>(a.P, (int64_t)sms * max(per_sm, 1)));
  kern<<<(unsigned)blocks, kMaskThreads, bytes, s>>>(a, boff, bmem, moff, smax);
  count_launches(1);
  return cudaGetLastError();
}

// Mask words of bucket c: nwb x nwb blocks of 32 words (nwb (nwb + 1) / 2
// with lower), nwb = ceil(s_c / 32).
__global__ void k_bucket_words(const uint32_t* __restrict__ bcount, int64_t P, int32_t lower,
                               uint32_t* __restrict__ words) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < P) {
    const uint32_t nwb = (bcount[b] + 31u) >> 5;
    words[b] = (lower ? nwb * (nwb + 1) / 2 : nwb * nwb) * 32u;
  }
}

cudaError_t launch_bucket_words(const uint32_t* bcount, int64_t P, int32_t lower, uint32_t* words, cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  k_bucket_words<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(bcount, P, lower, words);
  count_launches(1);
  return cudaGetLastError();
}

// Row blocks of bucket c: nwb = ceil(s_c / 32) (the emit pass's work items).
__global__ void k_bucket_jblocks(const uint32_t* __restrict__ bcount, int64_t P, uint32_t* __restrict__ out) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < P) out[b] = (bcount[b] + 31u) >> 5;
}

cudaError_t launch_bucket_jblocks(const uint32_t* bcount, int64_t P, uint32_t* out, cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  k_bucket_jblocks<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(bcount, P, out);
  count_launches(1);
  return cudaGetLastError();
}

// ibkt[t] = the bucket of work item t, for t in [jboff[b], jboff[b + 1]).
__global__ void k_item_bucket(const int64_t* __restrict__ jboff, int64_t P, int32_t* __restrict__ ibkt) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= P) return;
  for (int64_t t = jboff[b]; t < jboff[b + 1]; ++t) ibkt[t] = (int32_t)b;
}

cudaError_t launch_item_bucket(const int64_t* jboff, int64_t P, int32_t* ibkt, cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  k_item_bucket<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(jboff, P, ibkt);
  count_launches(1);
  return cudaGetLastError();
}

// Emit pass: the mask words become CSR runs.  Work items are the 32-row
// blocks of all buckets (jboff = prefix of ceil(s_c / 32)); every warp takes
// items from a global counter, so no warp waits for another.  For an item the
// warp stages the rows' words, 16 partner blocks at a time (one coalesced
// 128-byte line each), and the partners' vertex ids in registers; it then
// writes the rows one after the other: the partners of a row's word go to
// consecutive positions (lane i writes partner i at the row's cursor plus the
// set bits below i), so each run comes out in ascending partner order and is
// written in one burst of stores.
__global__ void __launch_bounds__(kEmitThreads) k_bucket_emit(ConflictArgs a, const int64_t* __restrict__ boff,
                                                              const int32_t* __restrict__ bmem,
                                                              const int64_t* __restrict__ moff,
                                                              const int64_t* __restrict__ jboff,
                                                              const int32_t* __restrict__ ibkt,
                                                              int32_t* __restrict__ counter, int64_t lo,
                                                              int64_t hi, int64_t base) {
  __shared__ uint32_t wbuf_s[kEmitThreads / 32][kEmitChunk * 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t lt = lanemask_lt();
  uint32_t* wbuf = wbuf_s[wid];
  const int64_t items = jboff[a.P];
  // flat / Lu as the high word of flat * ceil(2^64 / Lu): exact for flat < 2^32
  const uint64_t invL = a.Lu > 1 ? ~0ull / (uint64_t)a.Lu + 1ull : 0ull;
  int64_t item = 0;
  if (lane == 0) item = atomicAdd(counter, 1);
  item = __shfl_sync(0xffffffffu, item, 0);
  while (item < items) {
    // the next item's id is fetched now and used at the end, so the atomic's
    // latency hides behind this item's stores
    int64_t next = 0;
    if (lane == 0) next = atomicAdd(counter, 1);
    const int64_t b = ibkt[item];
    const int J = (int)(item - jboff[b]);
    const int64_t o = boff[b];
    const int s = (int)(boff[b + 1] - o);
    const int nwb = (s + 31) >> 5;
    const uint32_t* rmb = a.rmask + moff[b];
    const int r = (J << 5) + lane;
    // lane r: row r's cursor; rows of vertices outside [lo, hi) are skipped
    bool in = false;
    int64_t rc = 0;
    if (r < s) {
      const int32_t f = bmem[o + r];
      const int64_t vr = a.Lu > 1 ? (int64_t)__umul64hi((uint64_t)f, invL) : a.Lu == 1 ? f : a.ent_v[f];
      in = vr >= lo && vr < hi;
      rc = a.runoff[f] - base;
    }
    const uint32_t rows_in = __ballot_sync(0xffffffffu, in);
    const int nrows = min(32, s - (J << 5));
    const int nwr = a.lower ? J + 1 : nwb;  // partner blocks of these rows
    const int blk0 = a.lower ? J * (J + 1) / 2 : J * nwb;
    for (int I0 = 0; I0 < nwr; I0 += kEmitChunk) {
      const int nI = min(kEmitChunk, nwr - I0);
      int32_t pv[kEmitChunk];
#pragma unroll
      for (int t = 0; t < kEmitChunk; ++t) {
        pv[t] = 0;
        if (t < nI) {
          wbuf[t * 32 + lane] = a.rowmajor ? __ldg(rmb + 16 * J * (J + 1) + lane * (J + 1) + I0 + t)
                                           : __ldg(rmb + (blk0 + I0 + t) * 32 + lane);
          const int pi = ((I0 + t) << 5) + lane;
          if (pi < s) {
            const int32_t f = __ldg(bmem + o + pi);
            pv[t] = a.Lu > 1 ? (int32_t)__umul64hi((uint64_t)f, invL) : a.Lu == 1 ? f : __ldg(a.ent_v + f);
          }
        }
      }
      __syncwarp();
      switch (nI) {
#define PICASSO_EMIT_CASE(N) \
  case N:                    \
    emit_rows<N>(wbuf, pv, rc, nrows, a.col, lane, lt, rows_in); \
    break;
        PICASSO_EMIT_CASE(1) PICASSO_EMIT_CASE(2) PICASSO_EMIT_CASE(3) PICASSO_EMIT_CASE(4)
        PICASSO_EMIT_CASE(5) PICASSO_EMIT_CASE(6) PICASSO_EMIT_CASE(7) PICASSO_EMIT_CASE(8)
        PICASSO_EMIT_CASE(9) PICASSO_EMIT_CASE(10) PICASSO_EMIT_CASE(11) PICASSO_EMIT_CASE(12)
        PICASSO_EMIT_CASE(13) PICASSO_EMIT_CASE(14) PICASSO_EMIT_CASE(15) PICASSO_EMIT_CASE(16)
#undef PICASSO_EMIT_CASE
        default:
          break;
      }
      __syncwarp();
    }
    item = __shfl_sync(0xffffffffu, next, 0);
  }
}

cudaError_t launch_bucket_emit(const ConflictArgs& a, const int64_t* boff, const int32_t* bmem, const int64_t* moff,
                               const int64_t* jboff, const int32_t* ibkt, int32_t* counter, int64_t lo, int64_t hi,
                               int64_t base, cudaStream_t s) {
  if (a.P <= 0 || a.n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bucket_emit, kEmitThreads, 0);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_bucket_emit<<<(unsigned)debug_grid(sms * max(per_sm, 1)), kEmitThreads, 0, s>>>(a, boff, bmem, moff, jboff, ibkt,
                                                                         counter, lo, hi, base);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// All pairs: warp per row u, lanes over the columns v; a commuting v joins
// u's run of every color the two lists share (two-pointer merge).
// ---------------------------------------------------------------------------
namespace {
constexpr int kApWarps = 8;
constexpr int kNoShare = 0x7fffffff;

// Next shared color index of u's list (rl) and v's list (lv) at or after the
// merge position (i, j); kNoShare when the lists have no further match.
__device__ __forceinline__ int next_shared(const int32_t* __restrict__ rl, int Lu, const int32_t* __restrict__ lv,
                                           int Lv, int& i, int& j) {
  while (i < Lu && j < Lv) {
    const int32_t x = rl[i], y = __ldg(lv + j);
    if (x == y) {
      const int k = i;
      ++i;
      ++j;
      return k;
    }
    if (x < y)
      ++i;
    else
      ++j;
  }
  return kNoShare;
}
}  // namespace

template <bool FILL>
__global__ void __launch_bounds__(kApWarps * 32) k_allpairs(ConflictArgs a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int Lm = a.Lmax;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // per warp: row list [Lmax] int32, run counters / cursors [Lmax] int64
  int32_t* rl = (int32_t*)smem_raw + (size_t)wid * Lm;
  int64_t* cur = (int64_t*)(smem_raw + ((sizeof(int32_t) * Lm * kApWarps + 15) & ~(size_t)15)) + (size_t)wid * Lm;
  const uint32_t lt = lanemask_lt();
  for (int64_t u = (int64_t)blockIdx.x * kApWarps + wid; u < a.n; u += (int64_t)gridDim.x * kApWarps) {
    const int64_t ru = a.loff[u];
    const int Lu = (int)(a.loff[u + 1] - ru);
    for (int t = lane; t < Lu; t += 32) {
      rl[t] = a.lists[ru + t];
      cur[t] = FILL ? a.runoff[ru + t] : 0;
    }
    __syncwarp();
    const bool wide = a.qw > 1;
    const uint64_t xu = wide ? 0 : a.xz[2 * u], zu = wide ? 0 : a.xz[2 * u + 1];
    const int64_t vend = a.lower ? u : a.n;  // lower rows: partners v < u only
    for (int64_t v0 = 0; v0 < vend; v0 += 32) {
      const int64_t v = v0 + lane;
      const int32_t* lv = nullptr;
      int Lv = 0, i = 0, j = 0, k = kNoShare;
      const bool cm = v < vend && v != u &&
                      (wide ? commuteW(a.xz + 2 * a.qw * u, a.xz + 2 * a.qw * v, a.qw)
                            : commute1(xu, zu, a.xz[2 * v], a.xz[2 * v + 1]));
      if (cm) {
        lv = a.lists + a.loff[v];
        Lv = (int)(a.loff[v + 1] - a.loff[v]);
        k = next_shared(rl, Lu, lv, Lv, i, j);
      }
      if (!FILL) {
        while (k != kNoShare) {
          atomicAdd((unsigned long long*)&cur[k], 1ull);
          k = next_shared(rl, Lu, lv, Lv, i, j);
        }
      } else {
        // runs in ascending color index; inside a run, lanes (= ascending v)
        // write in order
        while (true) {
          const int kmin = __reduce_min_sync(0xffffffffu, k);
          if (kmin == kNoShare) break;
          const bool mine = k == kmin;
          const uint32_t m = __ballot_sync(0xffffffffu, mine);
          if (mine) a.col[cur[kmin] + __popc(m & lt)] = (int32_t)v;
          __syncwarp();
          if (lane == 0) cur[kmin] += __popc(m);
          __syncwarp();
          if (mine) k = next_shared(rl, Lu, lv, Lv, i, j);
        }
      }
    }
    __syncwarp();
    if (!FILL)
      for (int t = lane; t < Lu; t += 32) a.cnt[ru + t] = (uint32_t)cur[t];
    __syncwarp();
  }
}

cudaError_t launch_allpairs(const ConflictArgs& a, bool fill, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const size_t bytes = ((sizeof(int32_t) * a.Lmax * kApWarps + 15) & ~(size_t)15) + sizeof(int64_t) * a.Lmax * kApWarps;
  auto kern = fill ? k_allpairs<true> : k_allpairs<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  const int64_t blocks = debug_grid(std::min<int64_t>((a.n + kApWarps - 1) / kApWarps, 148 * 8));
  kern<<<(unsigned)blocks, kApWarps * 32, bytes, s>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void k_row_offsets(const int64_t* __restrict__ runoff, const int64_t* __restrict__ loff, int64_t n,
                              int64_t* __restrict__ off) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u <= n) off[u] = runoff[loff[u]];
}

cudaError_t launch_row_offsets(const int64_t* runoff, const int64_t* loff, int64_t n, int64_t* off, cudaStream_t s) {
  k_row_offsets<<<(unsigned)((n + 1 + 255) / 256), 256, 0, s>>>(runoff, loff, n, off);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace picasso
