// kernels_conflict.cu -- Alg. 1 construct_conflict_graph on sm_103a.
//
// G_c keeps a pair {u, v} of the round's vertices iff the two strings commute
// (edge of the complement graph G', Sec. II) and their color lists intersect
// (Sec. III-A).  Rows are color-major: row u holds, for each color c of u's
// list in ascending order, the neighbours v whose smallest shared color with
// u is c, ascending in v (one "run" per list color).  Pairs sharing more than
// one color also go to a side list at each non-smallest shared color; the
// coloring step uses runs and side list to find, per list color, exactly the
// neighbours that hold it.
//
// Both strategies below run a count pass (run lengths), an exclusive scan to
// offsets, and a fill pass that recomputes every test and writes each run in
// ascending order with warp ballots -- no atomics on output positions, so
// the CSR is deterministic.
//
//   bucket join   one CTA per color c: the members of bucket c (vertices
//                 holding c) are staged in shared memory and every pair of
//                 members is tested there; a pair is a run entry at c iff c
//                 is the pair's smallest shared color, found exactly through
//                 a shared-memory hash of the members' smaller colors.
//   all pairs     one warp per row u sweeping every column v (the paper's GPU
//                 kernel tests all |V|(|V|-1)/2 pairs, Sec. IV); the list
//                 intersection is a two-pointer merge.
#include <algorithm>
#include <cstdio>

#include "common.cuh"

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

// Ascending order inside each bucket: a shared-memory bitonic sort per bucket.
__global__ void __launch_bounds__(512) k_bucket_sort(const int64_t* __restrict__ boff, int64_t P,
                                                     int32_t* __restrict__ bmem, int32_t* err) {
  __shared__ int32_t key[kBucketCap];
  for (int64_t b = blockIdx.x; b < P; b += gridDim.x) {
    const int64_t o = boff[b];
    const int s = (int)(boff[b + 1] - o);
    if (s <= 1) continue;
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

cudaError_t launch_bucket_sort(const int64_t* boff, int64_t P, int32_t* bmem, int32_t* err, cudaStream_t s) {
  const unsigned blocks = (unsigned)std::min<int64_t>(P, 148 * 8);
  k_bucket_sort<<<blocks, 256, 0, s>>>(boff, P, bmem, err);
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
// ---------------------------------------------------------------------------
namespace {

constexpr int kPairThreads = 512;
constexpr int kExCap = 2048;  // exclusion pairs per bucket before the exact fallback

struct BucketSmem {
  uint64_t* sx;
  uint64_t* sz;
  int32_t* sid;   // member vertex
  int32_t* sfl;   // member's list entry (bucket color's position)
  uint16_t* kk;   // position of the bucket color in the member's list
  int32_t* exo;   // [smax + 1]
  int32_t* excur; // [smax]
  int32_t* scnt;  // [smax] run counts
  int32_t* sxcnt; // [smax] side-list counts
  uint16_t* exv;  // [2 * kExCap]
  uint32_t* expair;
  uint32_t* tab;  // [hs]
  int32_t* misc;  // [4]: E, nexcl, slow
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline size_t bucket_smem_bytes(int smax, int hs) {
  size_t b = 0;
  b += align16(sizeof(uint64_t) * smax) * 2;
  b += align16(sizeof(int32_t) * smax) * 2;
  b += align16(sizeof(uint16_t) * smax);
  b += align16(sizeof(int32_t) * (smax + 1));
  b += align16(sizeof(int32_t) * smax);
  b += align16(sizeof(int32_t) * smax) * 2;
  b += align16(sizeof(uint16_t) * 2 * kExCap);
  b += align16(sizeof(uint32_t) * kExCap);
  b += align16(sizeof(uint32_t) * hs);
  b += align16(sizeof(int32_t) * 4);
  return b;
}

__device__ inline BucketSmem carve(uint8_t* p, int smax, int hs) {
  BucketSmem m;
  m.sx = (uint64_t*)p; p += align16(sizeof(uint64_t) * smax);
  m.sz = (uint64_t*)p; p += align16(sizeof(uint64_t) * smax);
  m.sid = (int32_t*)p; p += align16(sizeof(int32_t) * smax);
  m.sfl = (int32_t*)p; p += align16(sizeof(int32_t) * smax);
  m.kk = (uint16_t*)p; p += align16(sizeof(uint16_t) * smax);
  m.exo = (int32_t*)p; p += align16(sizeof(int32_t) * (smax + 1));
  m.excur = (int32_t*)p; p += align16(sizeof(int32_t) * smax);
  m.scnt = (int32_t*)p; p += align16(sizeof(int32_t) * smax);
  m.sxcnt = (int32_t*)p; p += align16(sizeof(int32_t) * smax);
  m.exv = (uint16_t*)p; p += align16(sizeof(uint16_t) * 2 * kExCap);
  m.expair = (uint32_t*)p; p += align16(sizeof(uint32_t) * kExCap);
  m.tab = (uint32_t*)p; p += align16(sizeof(uint32_t) * hs);
  m.misc = (int32_t*)p;
  return m;
}

// Does a[0..ka) meet b[0..kb)?  (both ascending)
__device__ inline bool share_prefix(const int32_t* __restrict__ a, int ka, const int32_t* __restrict__ b, int kb) {
  int i = 0, j = 0;
  while (i < ka && j < kb) {
    const int32_t x = __ldg(a + i), y = __ldg(b + j);
    if (x == y) return true;
    if (x < y)
      ++i;
    else
      ++j;
  }
  return false;
}


}  // namespace

// Mask pass over the pairs of a bucket, one 32 x 32 block (row chunk I,
// partner chunk J >= I) per warp step.  Lane t tests partner J*32 + t
// against each row of chunk I; the ballots give row words (partners of
// chunk J), and a 32-ballot bit transpose gives the words of the rows of
// chunk J for partners of chunk I -- every relation used (commutation,
// sharing a smaller color, i != j) is symmetric, so each unordered pair is
// tested once.  The run word keeps partners whose smallest shared color with
// the row is this bucket's color; the side word keeps the others.  Words of
// row i, chunk w live at masks + i * nwb + w; per-row counts accumulate in
// shared memory.
__device__ __forceinline__ uint32_t excl_bits(const BucketSmem& S, int i, int j0) {
  uint32_t exm = 0u;
  for (int e = S.exo[i], e1 = S.exo[i + 1]; e < e1; ++e) {
    const uint32_t d = (uint32_t)S.exv[e] - (uint32_t)j0;
    if (d < 32u) exm |= 1u << d;
  }
  return exm;
}

__device__ __forceinline__ void store_words(BucketSmem& S, int row, int s, int nwb, int w, uint32_t rm, uint32_t xm,
                                            uint32_t* __restrict__ rmask, uint32_t* __restrict__ xmask) {
  if (row < s) {
    rmask[(int64_t)row * nwb + w] = rm;
    xmask[(int64_t)row * nwb + w] = xm;
    if (rm) atomicAdd(&S.scnt[row], __popc(rm));
    if (xm) atomicAdd(&S.sxcnt[row], __popc(xm));
  }
}

// The 32 rows of chunk I against this lane's partner j: ballot words, the
// one for row I*32 + r kept by lane r.  DIAG: the block is on the diagonal
// (J == I), so partner j may be the row itself.
template <bool DIAG>
__device__ __forceinline__ uint32_t block_rows(const BucketSmem& S, int s, int ib, int j, bool valid, int lane,
                                               uint32_t xjl, uint32_t xjh, uint32_t zjl, uint32_t zjh) {
  uint32_t my_m = 0u;
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    const int i = ib + r;
    const bool rowok = i < s;
    uint64_t xi = 0ull, zi = 0ull;
    if (rowok) {
      xi = S.sx[i];
      zi = S.sz[i];
    }
    const uint32_t t = (((uint32_t)xi & zjl) ^ ((uint32_t)zi & xjl)) ^
                       (((uint32_t)(xi >> 32) & zjh) ^ ((uint32_t)(zi >> 32) & xjh));
    bool hit = valid && rowok && (__popc(t) & 1) == 0;
    if (DIAG) hit = hit && j != i;
    const uint32_t m = __ballot_sync(0xffffffffu, hit);
    my_m = lane == r ? m : my_m;
  }
  return my_m;
}

template <bool SLOW>
__device__ void mask_blocks(const ConflictArgs& a, BucketSmem& S, int s, int L, int lane, int wid, int nw,
                            uint32_t* __restrict__ rmask, uint32_t* __restrict__ xmask) {
  const int nwb = (s + 31) >> 5;
  const int nblk = nwb * (nwb + 1) / 2;
  for (int q = wid; q < nblk; q += nw) {
    // q -> (I, J), J >= I, row-major over the upper triangle
    int I = 0, rem = q;
    while (rem >= nwb - I) {
      rem -= nwb - I;
      ++I;
    }
    const int J = I + rem;
    const int ib = I << 5;
    const int j = (J << 5) + lane;
    const bool valid = j < s;
    const uint64_t xj = valid ? S.sx[j] : 0ull, zj = valid ? S.sz[j] : 0ull;
    const uint32_t xjl = (uint32_t)xj, xjh = (uint32_t)(xj >> 32);
    const uint32_t zjl = (uint32_t)zj, zjh = (uint32_t)(zj >> 32);
    const uint32_t my_m = J == I ? block_rows<true>(S, s, ib, j, valid, lane, xjl, xjh, zjl, zjh)
                                 : block_rows<false>(S, s, ib, j, valid, lane, xjl, xjh, zjl, zjh);
    // partners of this lane's row that share a smaller color go to the side word
    const int ir = ib + lane;
    uint32_t myex = 0u;
    if (!SLOW) {
      if (ir < s && S.exo[ir + 1] > S.exo[ir]) myex = excl_bits(S, ir, J << 5) & my_m;
    } else if (ir < s) {
      for (uint32_t bits = my_m; bits; bits &= bits - 1) {
        const int jj = (J << 5) + __ffs(bits) - 1;
        if (share_prefix(a.lists + (S.sfl[ir] - S.kk[ir]), S.kk[ir], a.lists + (S.sfl[jj] - S.kk[jj]), S.kk[jj]))
          myex |= bits & (0u - bits);
      }
    }
    const uint32_t my_r = my_m & ~myex, my_x = myex;
    store_words(S, ir, s, nwb, J, my_r, my_x, rmask, xmask);
    if (J != I) {
      uint32_t tr = 0u, tx = 0u;
#pragma unroll
      for (int b = 0; b < 32; ++b) {
        const uint32_t cr = __ballot_sync(0xffffffffu, (my_r >> b) & 1u);
        tr = lane == b ? cr : tr;
      }
      if (__any_sync(0xffffffffu, my_x != 0u)) {
#pragma unroll
        for (int b = 0; b < 32; ++b) {
          const uint32_t cx = __ballot_sync(0xffffffffu, (my_x >> b) & 1u);
          tx = lane == b ? cx : tx;
        }
      }
      store_words(S, (J << 5) + lane, s, nwb, I, tr, tx, rmask, xmask);
    }
  }
}

__global__ void __launch_bounds__(kPairThreads, 2) k_bucket_mask(ConflictArgs a, const int64_t* __restrict__ boff,
                                                              const int32_t* __restrict__ bmem,
                                                              const int64_t* __restrict__ moff, int smax,
                                                              int hs_log2) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int hs = 1 << hs_log2;
  BucketSmem S = carve(smem_raw, smax, hs);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int L = a.Lmax;

  for (int64_t b = blockIdx.x; b < a.P; b += gridDim.x) {
    const int64_t o = boff[b];
    const int s = (int)(boff[b + 1] - o);
    if (s == 0) continue;
    if (threadIdx.x < 4) S.misc[threadIdx.x] = 0;
    for (int i = threadIdx.x; i < s; i += blockDim.x) {
      const int32_t flat = bmem[o + i];  // list entry of color b in member v's list
      const int32_t v = a.Lu ? flat / a.Lu : a.ent_v[flat];
      S.sid[i] = v;
      S.sfl[i] = flat;
      S.sx[i] = a.xz[2 * (int64_t)v];
      S.sz[i] = a.xz[2 * (int64_t)v + 1];
      S.kk[i] = (uint16_t)(flat - (a.Lu ? (int64_t)v * a.Lu : a.loff[v]));
      S.excur[i] = 0;
      S.scnt[i] = 0;
      S.sxcnt[i] = 0;
    }
    __syncthreads();
    // E = number of (member, smaller color) entries
    {
      int e = 0;
      for (int i = threadIdx.x; i < s; i += blockDim.x) e += S.kk[i];
      for (int d = 16; d; d >>= 1) e += __shfl_xor_sync(0xffffffffu, e, d);
      if (lane == 0 && e) atomicAdd(&S.misc[0], e);
    }
    __syncthreads();
    if (S.misc[0] * 10 > hs * 7) {
      if (threadIdx.x == 0) S.misc[2] = 1;
    } else if (S.misc[0] > 0) {
      for (int i = threadIdx.x; i < hs; i += blockDim.x) S.tab[i] = 0u;
      __syncthreads();
      // Insert every smaller color of every member; an insert that passes an
      // entry of the same color found a pair sharing that color.
      // flattened over (member, list position) so that every thread's list
      // load is independent and the block's loads overlap
      for (int idx = threadIdx.x; idx < s * L; idx += blockDim.x) {
        const int i = idx / L, t = idx - i * L;
        if (t < S.kk[i]) {
          const uint32_t c = (uint32_t)__ldg(a.lists + (int64_t)(S.sfl[i] - S.kk[i]) + t);
          const uint32_t key = ((c + 1u) << 11) | (uint32_t)i;
          uint32_t slot = (c * 0x9E3779B1u) >> (32 - hs_log2);
          while (true) {
            const uint32_t old = atomicCAS(&S.tab[slot], 0u, key);
            if (old == 0u) break;
            if ((old >> 11) == c + 1u) {
              const int q = atomicAdd(&S.misc[1], 1);
              if (q < kExCap)
                S.expair[q] = ((old & 2047u) << 16) | (uint32_t)i;
              else
                S.misc[2] = 1;
            }
            slot = (slot + 1) & (hs - 1);
          }
        }
      }
    }
    __syncthreads();
    const bool slow = S.misc[2] != 0;
    const int npairs = min(S.misc[1], kExCap);
    if (!slow) {
      // per-member exclusion lists (counting sort of the pairs by member)
      for (int i = threadIdx.x; i <= s; i += blockDim.x) S.exo[i] = 0;
      __syncthreads();
      for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
        atomicAdd(&S.exo[(S.expair[p] >> 16) + 1], 1);
        atomicAdd(&S.exo[(S.expair[p] & 0xffffu) + 1], 1);
      }
      __syncthreads();
      if (wid == 0) {
        int carry = 0;
        for (int i0 = 1; i0 <= s; i0 += 32) {
          const int i = i0 + lane;
          int x = i <= s ? S.exo[i] : 0;
          for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
          }
          if (i <= s) S.exo[i] = x + carry;
          carry += __shfl_sync(0xffffffffu, x, 31);
        }
      }
      __syncthreads();
      for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
        const int i1 = S.expair[p] >> 16, i2 = S.expair[p] & 0xffff;
        S.exv[S.exo[i1] + atomicAdd(&S.excur[i1], 1)] = (uint16_t)i2;
        S.exv[S.exo[i2] + atomicAdd(&S.excur[i2], 1)] = (uint16_t)i1;
      }
      __syncthreads();
      // ascending partners per member (lists are short: insertion sort)
      for (int i = threadIdx.x; i < s; i += blockDim.x) {
        uint16_t* e = S.exv + S.exo[i];
        const int m = S.exo[i + 1] - S.exo[i];
        for (int x = 1; x < m; ++x) {
          const uint16_t key = e[x];
          int y = x - 1;
          while (y >= 0 && e[y] > key) {
            e[y + 1] = e[y];
            --y;
          }
          e[y + 1] = key;
        }
      }
      __syncthreads();
    }

    if (slow)
      mask_blocks<true>(a, S, s, L, lane, wid, nw, a.rmask + moff[b], a.xmask + moff[b]);
    else
      mask_blocks<false>(a, S, s, L, lane, wid, nw, a.rmask + moff[b], a.xmask + moff[b]);
    __syncthreads();
    for (int i = threadIdx.x; i < s; i += blockDim.x) {
      const int64_t slot = S.sfl[i];
      a.cnt[slot] = (uint32_t)S.scnt[i];
      a.xcnt[slot] = (uint32_t)S.sxcnt[i];
    }
    __syncthreads();
  }
}

cudaError_t launch_bucket_mask(const ConflictArgs& a, const int64_t* boff, const int32_t* bmem, const int64_t* moff,
                               int32_t smax, cudaStream_t s) {
  if (a.P <= 0 || a.n <= 0) return cudaSuccess;
  smax = max(smax, 1);
  int64_t want = (int64_t)smax * (int64_t)max(a.Lmax - 1, 1) * 3 / 2;
  int hs_log2 = 8;
  while ((1ll << hs_log2) < want && hs_log2 < 14) ++hs_log2;
  const size_t bytes = bucket_smem_bytes(smax, 1 << hs_log2);
  auto kern = k_bucket_mask;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPairThreads, bytes);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = std::min<int64_t>(a.P, (int64_t)sms * max(per_sm, 1));
  kern<<<(unsigned)blocks, kPairThreads, bytes, s>>>(a, boff, bmem, moff, smax, hs_log2);
  count_launches(1);
  return cudaGetLastError();
}

// Mask words of bucket c: s_c rows of ceil(s_c / 32) words.
__global__ void k_bucket_words(const uint32_t* __restrict__ bcount, int64_t P, uint32_t* __restrict__ words) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < P) words[b] = bcount[b] * ((bcount[b] + 31u) >> 5);
}

cudaError_t launch_bucket_words(const uint32_t* bcount, int64_t P, uint32_t* words, cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  k_bucket_words<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(bcount, P, words);
  count_launches(1);
  return cudaGetLastError();
}

// Emit pass: streaming compaction of the mask words into the CSR.  One warp
// per member row; the run's entries are written in ascending partner order
// (ballot positions within a word, words in ascending order).
__global__ void __launch_bounds__(512) k_bucket_emit(ConflictArgs a, const int64_t* __restrict__ boff,
                                                     const int32_t* __restrict__ bmem,
                                                     const int64_t* __restrict__ moff) {
  extern __shared__ __align__(16) int32_t emit_smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t lt = lanemask_lt();
  const int smax = a.smax;
  int32_t* vid = emit_smem;          // [smax] member vertex ids
  int32_t* flat = emit_smem + smax;  // [smax] member list entries
  for (int64_t b = blockIdx.x; b < a.P; b += gridDim.x) {
    const int64_t o = boff[b];
    const int s = (int)(boff[b + 1] - o);
    if (s == 0) continue;
    for (int i = threadIdx.x; i < s; i += blockDim.x) {
      const int32_t f = bmem[o + i];
      flat[i] = f;
      vid[i] = a.Lu ? f / a.Lu : a.ent_v[f];
    }
    __syncthreads();
    const int nwb = (s + 31) >> 5;
    const uint32_t* rmb = a.rmask + moff[b];
    const uint32_t* xmb = a.xmask + moff[b];
    for (int i = wid; i < s; i += nw) {
      const int64_t slot = flat[i];
      int32_t* rp = a.col + a.runoff[slot];
      const int64_t x0 = a.xoff[slot], x1 = a.xoff[slot + 1];
      const uint32_t* rrow = rmb + (int64_t)i * nwb;
      for (int w0 = 0; w0 < nwb; w0 += 32) {
        // each lane loads one word; the warp then walks them in order and
        // writes each word's partners with one coalesced store
        const int wl = w0 + lane;
        const uint32_t rml = wl < nwb ? __ldg(rrow + wl) : 0u;
        const int nwords = min(32, nwb - w0);
#pragma unroll 4
        for (int t = 0; t < nwords; ++t) {
          const uint32_t rm = __shfl_sync(0xffffffffu, rml, t);
          const int j = ((w0 + t) << 5) + lane;
          if ((rm >> lane) & 1u) rp[__popc(rm & lt)] = vid[j];
          rp += __popc(rm);
        }
      }
      if (x1 > x0) {  // side-list entries are rare: only rows that have some
        int32_t* xp = a.xcol + x0;
        const uint32_t* xrow = xmb + (int64_t)i * nwb;
        for (int w = 0; w < nwb; ++w) {
          const uint32_t xm = __ldg(xrow + w);
          const int j = (w << 5) + lane;
          if ((xm >> lane) & 1u) xp[__popc(xm & lt)] = vid[j];
          xp += __popc(xm);
        }
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_bucket_emit(const ConflictArgs& a, const int64_t* boff, const int32_t* bmem, const int64_t* moff,
                               int32_t smax, cudaStream_t s) {
  if (a.P <= 0 || a.n <= 0) return cudaSuccess;
  const size_t bytes = 2 * sizeof(int32_t) * (size_t)max(smax, 1);
  ConflictArgs args = a;
  args.smax = max(smax, 1);
  cudaError_t e = cudaFuncSetAttribute(k_bucket_emit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = std::min<int64_t>(a.P, (int64_t)sms * 4);
  k_bucket_emit<<<(unsigned)blocks, 512, bytes, s>>>(args, boff, bmem, moff);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// All pairs: warp per row, two-pointer list merge for commuting pairs.
// ---------------------------------------------------------------------------
namespace {
constexpr int kApWarps = 8;
}

template <bool FILL>
__global__ void __launch_bounds__(kApWarps * 32) k_allpairs(ConflictArgs a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int Lm = a.Lmax;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // per warp: row list [Lmax] int32, run counters/cursors [Lmax] int64, side [Lmax] int64
  int32_t* rl = (int32_t*)smem_raw + (size_t)wid * Lm;
  int64_t* cur = (int64_t*)(smem_raw + align16(sizeof(int32_t) * Lm * kApWarps)) + (size_t)wid * 2 * Lm;
  int64_t* xcur = cur + Lm;
  const uint32_t lt = lanemask_lt();
  for (int64_t u = (int64_t)blockIdx.x * kApWarps + wid; u < a.n; u += (int64_t)gridDim.x * kApWarps) {
    const int64_t ru = a.loff[u];
    const int Lu = (int)(a.loff[u + 1] - ru);
    for (int t = lane; t < Lu; t += 32) {
      rl[t] = a.lists[ru + t];
      cur[t] = FILL ? a.runoff[ru + t] : 0;
      xcur[t] = FILL ? a.xoff[ru + t] : 0;
    }
    __syncwarp();
    const uint64_t xu = a.xz[2 * u], zu = a.xz[2 * u + 1];
    for (int64_t v0 = 0; v0 < a.n; v0 += 32) {
      const int64_t v = v0 + lane;
      int k0 = -1, nshared = 0;
      if (v < a.n && v != u && commute1(xu, zu, a.xz[2 * v], a.xz[2 * v + 1])) {
        const int32_t* lv = a.lists + a.loff[v];
        const int Lv = (int)(a.loff[v + 1] - a.loff[v]);
        int i = 0, j = 0;
        while (i < Lu && j < Lv) {
          const int32_t x = rl[i], y = __ldg(lv + j);
          if (x == y) {
            if (k0 < 0) {
              k0 = i;
            } else if (!FILL) {
              atomicAdd((unsigned long long*)&xcur[i], 1ull);
            }
            ++nshared;
            ++i;
            ++j;
          } else if (x < y) {
            ++i;
          } else {
            ++j;
          }
        }
      }
      if (!FILL) {
        if (k0 >= 0) atomicAdd((unsigned long long*)&cur[k0], 1ull);
      } else {
        // run entries: lanes with the same run write in lane (= v) order
        const uint32_t act = __ballot_sync(0xffffffffu, k0 >= 0);
        if (act) {
          const uint32_t grp = __match_any_sync(0xffffffffu, k0);
          if (k0 >= 0) {
            const int64_t pos = cur[k0] + __popc(grp & lt);
            a.col[pos] = (int32_t)v;
          }
          __syncwarp();
          if (k0 >= 0 && (grp & lt) == 0u) cur[k0] += __popc(grp);
          __syncwarp();
        }
        // side-list entries, one lane at a time in lane order
        uint32_t more = __ballot_sync(0xffffffffu, nshared > 1);
        while (more) {
          const int l = __ffs(more) - 1;
          more &= more - 1;
          if (lane == l) {
            const int32_t* lv = a.lists + a.loff[v];
            const int Lv = (int)(a.loff[v + 1] - a.loff[v]);
            int i = 0, j = 0, seen = 0;
            while (i < Lu && j < Lv) {
              const int32_t x = rl[i], y = __ldg(lv + j);
              if (x == y) {
                if (seen++) a.xcol[xcur[i]++] = (int32_t)v;
                ++i;
                ++j;
              } else if (x < y) {
                ++i;
              } else {
                ++j;
              }
            }
          }
          __syncwarp();
        }
      }
    }
    __syncwarp();
    if (!FILL) {
      for (int t = lane; t < Lu; t += 32) {
        a.cnt[ru + t] = (uint32_t)cur[t];
        a.xcnt[ru + t] = (uint32_t)xcur[t];
      }
    }
    __syncwarp();
  }
}

cudaError_t launch_allpairs(const ConflictArgs& a, bool fill, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const size_t bytes = align16(sizeof(int32_t) * a.Lmax * kApWarps) + sizeof(int64_t) * 2 * a.Lmax * kApWarps;
  auto kern = fill ? k_allpairs<true> : k_allpairs<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  const int64_t blocks = std::min<int64_t>((a.n + kApWarps - 1) / kApWarps, 148 * 8);
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
