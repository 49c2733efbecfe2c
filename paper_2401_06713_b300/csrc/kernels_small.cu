// kernels_small.cu -- the small-round engine: every remaining round of a
// context (one set, or a batch of sets advancing together), once a round has
// at most kSmallRoundsMax vertices, in one cooperative launch.  Late rounds are small (the uncolored set shrinks geometrically),
// and as separate launches their cost is launch and synchronisation overhead;
// here each round is a sequence of grid-wide phases with no host round trip.
//
// A round follows Alg. 1 exactly as the per-round path does:
//   priorities (static Random order, Sec. III-B) -> ranks in ascending
//   (priority, global id) -> lists in that order (Floyd, as draw_list) ->
//   G_c in the bit layout by a join through per-color buckets -> ordered
//   first-fit coloring over the buckets' color masks (mask_vertex) -> colors
//   and the uncolored set in ascending global id (carry).
// The run of list entry (u, k) holds the vertices v < u that commute with u
// and also hold color c = list[u][k]: exactly the members of bucket c ranked
// before u that commute with u.  So a bucket gives every run of its color by
// commutation tests alone: sorted by list-entry index (r L + k, ascending
// with the rank r), member i against the members j < i, one bit each.
// (P, L) of a set come from a table the host fills with its own rule (indexed
// by the set's vertex count), so both paths use the same numbers.  In a
// batch, V_l in ascending global id holds the sets one after another; a
// vertex's Philox streams are keyed by its set's seed and its id within the
// set, its list colors carry the set's bucket-color offset (sum of the P of
// the sets before it), and it is ranked among its own set only.  Data the launch wrote in an earlier phase is read
// after a grid barrier with plain or L2 loads (ld_run<true>), never through
// the read-only path, which may hold lines from before the write.
//
// The engine stops, with the state of the round it could not finish intact
// (its vertex list; no color written), when the round's CSR exceeds the
// capacity or the byte budget, or when a bounded wait of the coloring runs
// out; the host then continues with the per-round path.
#include <cooperative_groups.h>

#include <algorithm>

#include "bits_device.cuh"
#include "color_device.cuh"
#include "common.cuh"
#include "warp_sort.cuh"

namespace cg = cooperative_groups;

namespace picasso {

namespace {
constexpr int kSmallThreads = 256;
constexpr int kSmallWarps = kSmallThreads / 32;
constexpr int kSmallBlocksPerSm = 2;
// dynamic shared memory of one warp: a bucket's member words (W words per
// part) and run lengths; for W = 1 also a block's bit columns and nibble
// tables (with room to align the tables to 256 bytes)
template <int W>
__host__ __device__ constexpr int warp_smem_bytes() {
  return W == 1 ? kSmallBucketCap * 20 + 128 * 4 + 256 + kTabWords * 4 : kSmallBucketCap * (16 * W + 4);
}

// Sum of x over the block (every thread gets it).  sm: 32 words.
__device__ __forceinline__ int64_t block_sum(int64_t x, int64_t* sm) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int d = 16; d; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
  __syncthreads();
  if (lane == 0) sm[wid] = x;
  __syncthreads();
  int64_t t = 0;
  for (int w = 0; w < nw; ++w) t += sm[w];
  return t;
}

// Exclusive scan of x over the block; *total gets the block's sum.  sm: 32 words.
__device__ __forceinline__ int64_t block_excl(int64_t x, int64_t* sm, int64_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int64_t inc = x;
  for (int d = 1; d < 32; d <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += y;
  }
  __syncthreads();
  if (lane == 31) sm[wid] = inc;
  __syncthreads();
  int64_t before = 0, t = 0;
  for (int w = 0; w < nw; ++w) {
    const int64_t y = sm[w];
    if (w < wid) before += y;
    t += y;
  }
  *total = t;
  return before + inc - x;
}

// Launch shapes of the engine: the cooperative grid (the larger rounds), one
// thread-block cluster, one block (the smallest rounds).
constexpr int kModeGrid = 0, kModeCluster = 1, kModeBlock = 2;

// Barrier of every thread of the launch: the cooperative grid's (bounded in
// time), the cluster's hardware barrier (release / acquire at cluster scope,
// which covers global memory written by the cluster's blocks), or the
// block's (which orders the block's global memory accesses as well).
template <int MODE>
__device__ __forceinline__ bool engine_sync(const SmallArgs& a, int site, int64_t round) {
  if constexpr (MODE == kModeCluster) {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    return true;
  } else if constexpr (MODE == kModeBlock) {
    __syncthreads();
    return true;
  } else {
    // a block that gives up records where (first one only) and the launch
    // ends with err[3] set
    int seen = -1;
    if (grid_sync_bounded(a.bar, a.err + 3, kBarrierLimitNs, &seen)) return true;
    if (threadIdx.x == 0 && seen >= 0 && atomicCAS((unsigned long long*)(a.ctl + 9), 0ull, (unsigned long long)site) == 0ull) {
      a.ctl[10] = round;
      a.ctl[11] = seen;
    }
    return false;
  }
}

// Exclusive scans of NV values per element over elements 0 .. m - 1, by the
// whole launch: block b takes the b-th contiguous chunk, adds the sums of the
// chunks before it (a.part: NV words per block) and hands each element's
// prefixes to put(i, ex); the last block calls put(m, totals).  get(i,
// first, y) gives element i's values, first on the summing pass and again
// (first = false) on the scanning pass.  Contains one barrier of the launch;
// every thread must call it.
template <int MODE, int NV, class Get, class Put>
__device__ bool engine_scan(const SmallArgs& a, int64_t round, int64_t m, int64_t* sm, Get get, Put put) {
  const int64_t chunk = (m + gridDim.x - 1) / gridDim.x;
  const int64_t lo = min(m, chunk * (int64_t)blockIdx.x), hi = min(m, lo + chunk);
  int64_t x[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) x[v] = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    int64_t y[NV];
    get(i, true, y);
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] += y[v];
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int64_t t = block_sum(x[v], sm);
    if (threadIdx.x == 0) a.part[NV * blockIdx.x + v] = t;
  }
  if (!engine_sync<MODE>(a, __LINE__, round)) return false;
  int64_t pre[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    int64_t p = 0;
    for (int64_t b = threadIdx.x; b < blockIdx.x; b += blockDim.x) p += __ldcg(a.part + NV * b + v);
    pre[v] = block_sum(p, sm);
  }
  for (int64_t t0 = lo; t0 < hi; t0 += blockDim.x) {
    const int64_t i = t0 + threadIdx.x;
    int64_t y[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) y[v] = 0;
    if (i < hi) get(i, false, y);
    int64_t ex[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      int64_t tot = 0;
      ex[v] = pre[v] + block_excl(y[v], sm, &tot);
      pre[v] += tot;
    }
    if (i < hi) put(i, ex);
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) put(m, pre);
  return true;
}

// One vertex's list drawn by a warp (Alg. 1 assign_rand_list_colors): the
// same picks as draw_list, Floyd's sampling on the same Philox words, in
// ascending order.  Lane t computes picks t and t + 32 as if unseen, the
// picks then take their final values one after another (a pick already
// chosen is replaced by j = P - L + m), and each goes to the place given by
// the number of smaller picks (the picks are distinct).  Writes out[0 .. L)
// (bucket colors: + cofs), owner[0 .. L) = rk, counts every color in
// bcount; returns the smallest color.  L <= 64.
__device__ __forceinline__ uint32_t warp_draw_list(uint64_t seed, int32_t round, int64_t g, int64_t P, int L,
                                                   int64_t cofs, int32_t* __restrict__ out,
                                                   int32_t* __restrict__ owner, int32_t rk,
                                                   uint32_t* __restrict__ bcount, int lane) {
  uint32_t t0 = 0u, t1 = 0u;
  if (lane < L) {
    const uint32_t x = pick(philox_block(seed, round, g, kTagList, (uint32_t)(lane >> 2)), (uint32_t)(lane & 3));
    t0 = (uint32_t)(((uint64_t)x * (uint64_t)(P - L + lane + 1)) >> 32);
  }
  if (lane + 32 < L) {
    const int m = lane + 32;
    const uint32_t x = pick(philox_block(seed, round, g, kTagList, (uint32_t)(m >> 2)), (uint32_t)(m & 3));
    t1 = (uint32_t)(((uint64_t)x * (uint64_t)(P - L + m + 1)) >> 32);
  }
  uint32_t s0 = 0xFFFFFFFFu, s1 = 0xFFFFFFFFu;
  for (int m = 0; m < L; ++m) {
    const uint32_t t = __shfl_sync(0xffffffffu, m < 32 ? t0 : t1, m & 31);
    const bool hit = (lane < m && s0 == t) || (lane + 32 < m && s1 == t);
    const uint32_t val = __any_sync(0xffffffffu, hit) ? (uint32_t)(P - L + m) : t;
    if (lane == (m & 31)) {
      if (m < 32)
        s0 = val;
      else
        s1 = val;
    }
  }
  int c0 = 0, c1 = 0;
  for (int m = 0; m < L; ++m) {
    const uint32_t v = __shfl_sync(0xffffffffu, m < 32 ? s0 : s1, m & 31);
    c0 += v < s0;
    c1 += v < s1;
  }
  if (lane < L) {
    const int32_t c = (int32_t)(cofs + s0);
    out[c0] = c;
    owner[lane] = rk;
    atomicAdd(bcount + c, 1u);
  }
  if (lane + 32 < L) {
    const int32_t c = (int32_t)(cofs + s1);
    out[c1] = c;
    owner[lane + 32] = rk;
    atomicAdd(bcount + c, 1u);
  }
  return (uint32_t)(cofs + __reduce_min_sync(0xffffffffu, min(s0, s1)));
}
}  // namespace


// Largest k with off[k] <= x (off ascending, off[0] <= x): the set holding
// position x when off holds the sets' offsets (empty sets are skipped).
__device__ __forceinline__ int find_set(const int64_t* off, int nsets, int64_t x) {
  int lo = 0, hi = nsets - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= x)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// The sets' offsets for a round from their vertex counts srem: vertices
// (svoff), bucket colors (scof, sum of P) and list entries (seoff, sum of
// n L).  Block 0 only; sm: 32 words.
__device__ void set_prefixes(const SmallArgs& a, int64_t* sm) {
  int64_t pv = 0, pc = 0, pe = 0;
  for (int k0 = 0; k0 < a.nsets; k0 += blockDim.x) {
    const int k = k0 + threadIdx.x;
    int64_t nk = 0, Pk = 0, Ek = 0;
    if (k < a.nsets) {
      nk = a.srem[k];
      if (nk > 0) {
        const int2 pl = a.ptab[nk];
        Pk = pl.x;
        Ek = nk * pl.y;
      }
    }
    int64_t tv, tc, te;
    const int64_t xv = block_excl(nk, sm, &tv);
    const int64_t xc = block_excl(Pk, sm, &tc);
    const int64_t xe = block_excl(Ek, sm, &te);
    if (k < a.nsets) {
      a.svoff[k] = pv + xv;
      a.scof[k] = pc + xc;
      a.seoff[k] = pe + xe;
    }
    pv += tv;
    pc += tc;
    pe += te;
  }
  if (threadIdx.x == 0) {
    a.svoff[a.nsets] = pv;
    a.scof[a.nsets] = pc;
    a.seoff[a.nsets] = pe;
  }
}

// The bit layout from the sorted buckets, by work items of 32 members of
// one bucket (item = bucket c, members i0 .. i0 + 31 = row block R): lane i
// tests its member against the members j < i (the smaller ranks), whose
// ranks and words the warp stages in shared memory, and writes its row of
// R + 1 words (bit t of word W: member 32 W + t commutes with i) at
// moff[c] + 16 R (R + 1) + (i % 32)(R + 1), and its entry's packed word
// (row address, slot, run length).  A warp takes a contiguous range of
// items, so it stages a bucket's members once, as far as its items reach.
// The run total goes to the set's count snnz and to the round's, ctl[3].
template <int W>
__device__ void bucket_bits(const SmallArgs& a, int32_t* R, uint64_t* X, int lane, int64_t gwarp, int64_t nwarps) {
  const int64_t nitems = __ldcg(a.ctl + 8);
  const int64_t per = (nitems + nwarps - 1) / nwarps;
  const int64_t it0 = min(nitems, gwarp * per), it1 = min(nitems, it0 + per);
  int64_t c = -1, b0 = 0;
  int s = 0, staged = 0, set = 0;
  for (int64_t it = it0; it < it1; ++it) {
    const int64_t cb = a.ibkt[it];
    const int i0 = (int)(it - a.iboff[cb]) * 32;
    if (cb != c) {
      c = cb;
      b0 = a.boff[c];
      s = (int)(a.boff[c + 1] - b0);
      staged = 0;
      set = a.nsets > 1 ? find_set(a.scof, a.nsets, c) : 0;
    }
    const int need = min(s, i0 + 32);
    if (need > staged) {
      __syncwarp();
      for (int i = staged + lane; i < need; i += 32) {
        R[i] = a.brank[b0 + i];
#pragma unroll
        for (int k = 0; k < 2 * W; ++k) X[2 * W * i + k] = a.bxz[2 * W * (b0 + i) + k];
      }
      staged = need;
      __syncwarp();
    }
    const int i = i0 + lane;
    const bool active = i < s;
    const int Rb = i0 >> 5;  // this item's row block
    int64_t addr = a.moff[c] + 16 * (int64_t)Rb * (Rb + 1) + (int64_t)lane * (Rb + 1);
    const int ilim = active ? i : 0;  // lanes past the bucket test nothing
    uint32_t tot = 0;
    // the symplectic form folded to one 32-bit word: parity of
    // x_i & z_j ^ z_i & x_j over all halves
    const uint32_t* X32 = reinterpret_cast<const uint32_t*>(X);
    uint32_t wi[4 * W];
#pragma unroll
    for (int k = 0; k < 4 * W; ++k) wi[k] = X32[4 * W * min(i, max(s - 1, 0)) + k];
    for (int Wb = 0; Wb <= Rb; ++Wb) {
      uint32_t word = 0u;
      const int jend = min(32 * Wb + 32, i0 + 32);
      for (int j = 32 * Wb; j < jend; ++j) {
        const uint32_t* w = X32 + 4 * W * j;
        uint32_t d = 0u;
#pragma unroll
        for (int h = 0; h < 2 * W; ++h) d ^= (wi[h] & w[2 * W + h]) ^ (wi[2 * W + h] & w[h]);
        if (j < ilim && (__popc(d) & 1u) == 0u) word |= 1u << (j - 32 * Wb);
      }
      if (active) a.rmask[addr + Wb] = word;
      tot += __popc(word);
    }
    if (active) a.rinfo[a.bmem[b0 + i]] = rinfo_pack(addr, i, (int)tot);
    const uint32_t wsum = __reduce_add_sync(0xffffffffu, tot);
    if (lane == 0 && wsum) {
      atomicAdd(reinterpret_cast<unsigned long long*>(a.snnz + set), (unsigned long long)wsum);
      atomicAdd(reinterpret_cast<unsigned long long*>(a.ctl + 3), (unsigned long long)wsum);
    }
  }
  __syncwarp();
}

// W = 1: the same rows by nibble tables (bits_device.cuh).  A warp's items
// in one bucket are the row blocks r0 .. r1; for every column block
// Wb <= r1 it builds the tables of members 32 Wb .. 32 Wb + 31 once and looks
// up each of its rows Rb >= max(Wb, r0) in them: word Wb of row i holds i's
// commutation bits against those members (on the diagonal block, the
// smaller slots only).  wsm: the warp's shared memory (warp_smem_bytes<1>).
__device__ void bucket_bits_tab(const SmallArgs& a, unsigned char* wsm, int lane, int64_t gwarp, int64_t nwarps) {
  uint4* X = reinterpret_cast<uint4*>(wsm);                              // member words x_lo, x_hi, z_lo, z_hi
  int32_t* cnt = reinterpret_cast<int32_t*>(X + kSmallBucketCap);        // run lengths
  uint32_t* colw = reinterpret_cast<uint32_t*>(cnt + kSmallBucketCap);   // [4][32] bit columns
  uint32_t* tab;
  {
    unsigned char* p = reinterpret_cast<unsigned char*>(colw + 128);
    const uint32_t ad = (uint32_t)__cvta_generic_to_shared(p);
    tab = reinterpret_cast<uint32_t*>(p + ((256u - (ad & 255u)) & 255u));
  }
  const uint32_t tab_addr = (uint32_t)__cvta_generic_to_shared(tab);
  const int64_t nitems = __ldcg(a.ctl + 8);
  const int64_t per = (nitems + nwarps - 1) / nwarps;
  const int64_t it0 = min(nitems, gwarp * per), it1 = min(nitems, it0 + per);
  for (int64_t it = it0; it < it1;) {
    const int64_t c = a.ibkt[it];
    const int64_t b0 = a.boff[c], ib0 = a.iboff[c];
    const int s = (int)(a.boff[c + 1] - b0);
    const int r0 = (int)(it - ib0);
    const int r1 = (int)(min(a.iboff[c + 1], it1) - ib0) - 1;
    const int need = min(s, 32 * (r1 + 1));
    __syncwarp();
    for (int i = lane; i < need; i += 32) X[i] = reinterpret_cast<const uint4*>(a.bxz)[b0 + i];
    for (int i = 32 * r0 + lane; i < 32 * (r1 + 1); i += 32) cnt[i] = 0;
    __syncwarp();
    const int64_t m0 = a.moff[c];
    for (int Wb = 0; Wb <= r1; ++Wb) {
      const int jm = 32 * Wb + lane;
      const uint4 wj = jm < s ? X[jm] : make_uint4(0u, 0u, 0u, 0u);
      __syncwarp();  // the warp is done with the previous block's columns
      colw[lane] = transpose32(wj.x, lane);
      colw[32 + lane] = transpose32(wj.y, lane);
      colw[64 + lane] = transpose32(wj.z, lane);
      colw[96 + lane] = transpose32(wj.w, lane);
      build_tables<2>(colw, tab, lane);
      for (int Rb = max(Wb, r0); Rb <= r1; ++Rb) {
        const int i = 32 * Rb + lane;
        const uint4 wi = X[min(i, s - 1)];
        uint32_t word = ~lookup<2>(wi, tab_addr);
        if (Rb == Wb) word &= (1u << lane) - 1u;
        if (i < s) {
          a.rmask[m0 + 16 * (int64_t)Rb * (Rb + 1) + (int64_t)lane * (Rb + 1) + Wb] = word;
          cnt[i] += __popc(word);
        }
      }
    }
    __syncwarp();
    uint32_t tot = 0;
    for (int Rb = r0; Rb <= r1; ++Rb) {
      const int i = 32 * Rb + lane;
      if (i < s) {
        const int64_t addr = m0 + 16 * (int64_t)Rb * (Rb + 1) + (int64_t)lane * (Rb + 1);
        a.rinfo[a.bmem[b0 + i]] = rinfo_pack(addr, i, cnt[i]);
        tot += (uint32_t)cnt[i];
      }
    }
    const uint32_t wsum = __reduce_add_sync(0xffffffffu, tot);
    if (lane == 0 && wsum) {
      const int set = a.nsets > 1 ? find_set(a.scof, a.nsets, c) : 0;
      atomicAdd(reinterpret_cast<unsigned long long*>(a.snnz + set), (unsigned long long)wsum);
      atomicAdd(reinterpret_cast<unsigned long long*>(a.ctl + 3), (unsigned long long)wsum);
    }
    it = ib0 + r1 + 1;
  }
  __syncwarp();
}

// The round's priority keys (priority, global id) in V_l order (gid), the
// buckets and color masks emptied (P bucket colors), the round's counters
// zeroed: what a stage does before its first round (later rounds find it
// done by the round before).
__device__ void round_init(const SmallArgs& a, const int32_t* gid, int64_t n, int32_t round, int64_t P, int64_t gtid,
                           int64_t gthreads) {
  for (int64_t i = gtid; i < n; i += gthreads) {
    const int32_t g = gid[i];
    const int k = a.nsets > 1 ? find_set(a.soff, a.nsets, g) : 0;
    a.key[i] = ((uint64_t)philox_block(a.sseed[k], round, g - a.soff[k], kTagPrio, 0u).x << 32) | (uint32_t)g;
  }
  for (int64_t c = gtid; c < P; c += gthreads) {
    a.bcnt[c] = 0;
    a.bcur[c] = 0;
  }
  for (int64_t t = gtid; t < 32 * P; t += gthreads) a.cmask[t] = 0u;
  for (int64_t k = gtid; k < a.nsets; k += gthreads) a.snnz[k] = 0;
  if (gtid == 0) a.ctl[3] = 0;
}

template <int W, int MODE>
__global__ void __launch_bounds__(kSmallThreads, kSmallBlocksPerSm) k_small_rounds(SmallArgs a) {
  extern __shared__ __align__(16) unsigned char smem_dyn[];
  __shared__ int64_t scan_s[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint64_t* Xw = reinterpret_cast<uint64_t*>(smem_dyn + (size_t)wid * warp_smem_bytes<W>());
  int32_t* Rw = reinterpret_cast<int32_t*>(Xw + 2 * W * kSmallBucketCap);
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t gwarp = gtid >> 5, nwarps = gthreads >> 5;
  const int nsets = a.nsets;

  // a later stage takes over from one that handed off (not from one whose
  // grid barrier timed out)
  if (MODE != kModeGrid && a.err[3] != 0) return;
  if (MODE != kModeGrid && gtid == 0 && a.ctl[2] == kSmallHandoff) a.ctl[2] = kSmallOk;
  if (blockIdx.x == 0) set_prefixes(a, scan_s);
  if (!engine_sync<MODE>(a, __LINE__, 0)) return;
  {
    const int64_t n = __ldcg(a.ctl + 0);
    round_init(a, __ldcg(a.ctl + 4) ? a.gid_b : a.gid_a, n, a.round0 + (int32_t)__ldcg(a.ctl + 1), a.scof[nsets],
               gtid, gthreads);
  }
  if (!engine_sync<MODE>(a, __LINE__, 0)) return;

  while (true) {
    const int64_t n = __ldcg(a.ctl + 0);
    const int64_t done = __ldcg(a.ctl + 1);
    const int32_t round = a.round0 + (int32_t)done;
    if (n == 0 || __ldcg(a.ctl + 2) != kSmallOk) break;
    if (round > a.max_rounds) {
      if (!engine_sync<MODE>(a, __LINE__, round)) return;
      if (gtid == 0) a.ctl[2] = kSmallMaxRounds;
      break;
    }
    if ((MODE == kModeGrid && n <= a.handoff) || (MODE == kModeCluster && n <= a.handoff2)) {
      // small enough for the next stage, whose barriers cost less
      if (!engine_sync<MODE>(a, __LINE__, round)) return;
      if (gtid == 0) a.ctl[2] = kSmallHandoff;
      break;
    }
    const int32_t* gid = __ldcg(a.ctl + 4) ? a.gid_b : a.gid_a;
    int32_t* gid_next = __ldcg(a.ctl + 4) ? a.gid_a : a.gid_b;
    const int64_t P = a.scof[nsets];
    const int64_t E = a.seoff[nsets];

    // rank of vertex i = its set's offset + the number of smaller keys in the
    // set (warp per vertex, lanes over the set); the round's arrays are
    // written at the rank, the rank at i (pos), and the warp draws the
    // vertex's list in rank order (bucket colors: + the set's offset): list
    // offset, entry owners, first candidate, bucket sizes
    for (int64_t i = gwarp; i < n; i += nwarps) {
      const int k = nsets > 1 ? find_set(a.svoff, nsets, i) : 0;
      const int64_t v0 = a.svoff[k], v1 = a.svoff[k + 1];
      const uint64_t ki = a.key[i];
      int r = 0;
      for (int64_t j = v0 + lane; j < v1; j += 32) r += a.key[j] < ki;
      const int64_t rk = v0 + __reduce_add_sync(0xffffffffu, r);
      const int32_t g = (int32_t)(uint32_t)ki;
      if (lane == 0) {
        a.perm[rk] = (int32_t)i;
        a.gid_r[rk] = g;
        a.sid[rk] = k;
        a.pos[i] = rk;
      }
      if (lane < 2 * W) a.xz_r[2 * W * rk + lane] = a.xz[2 * W * (int64_t)g + lane];
      const int2 pl = a.ptab[v1 - v0];
      const int64_t row = a.seoff[k] + (rk - v0) * pl.y;
      const uint32_t first = warp_draw_list(a.sseed[k], round, g - a.soff[k], pl.x, pl.y, a.scof[k], a.lists + row,
                                            a.ent_v + row, (int32_t)rk, a.bcnt, lane);
      if (lane == 0) {
        a.loff[rk] = row;
        a.state[rk] = ((uint64_t)first << 2) | kUndecided;
      }
    }
    if (gtid == 0) a.loff[n] = E;
    if (!engine_sync<MODE>(a, __LINE__, round)) return;

    // bucket offsets, work items (32 members each) and words of the bit rows
    // (the lower blocks, row-major) in one scan; a bucket above the cap stops
    // the engine
    {
      auto get = [&](int64_t c, bool first, int64_t* y) {
        const uint32_t sc = a.bcnt[c];
        const int64_t nwb = (sc + 31) / 32;
        y[0] = sc;
        y[1] = nwb;
        y[2] = 16 * nwb * (nwb + 1);
        if (first && sc > (uint32_t)kSmallBucketCap) a.err[2] = 1;
      };
      auto put = [&](int64_t c, const int64_t* ex) {
        a.boff[c] = ex[0];
        a.iboff[c] = ex[1];
        a.moff[c] = ex[2];
      };
      if (!engine_scan<MODE, 3>(a, round, P, scan_s, get, put)) return;
    }
    if (!engine_sync<MODE>(a, __LINE__, round)) return;
    if (__ldcg(a.err + 2) != 0 || __ldcg(a.moff + P) > a.wcap) {
      if (gtid == 0) a.ctl[2] = kSmallOverflow;
      break;
    }
    // bucket members (list entries) at a slot of the bucket; item -> bucket
    for (int64_t e = gtid; e < E; e += gthreads) {
      const int32_t c = a.lists[e];
      a.bmem[a.boff[c] + atomicAdd(a.bcur + c, 1u)] = (int32_t)e;
    }
    for (int64_t c = gtid; c < P; c += gthreads)
      for (int64_t t = a.iboff[c]; t < a.iboff[c + 1]; ++t) a.ibkt[t] = (int32_t)c;
    if (gtid == 0) a.ctl[8] = a.iboff[P];
    if (!engine_sync<MODE>(a, __LINE__, round)) return;

    // each bucket ascending (entries ascend with the rank), then its
    // members' ranks and words in that order
    for (int64_t c = gwarp; c < P; c += nwarps) {
      const int64_t b0 = a.boff[c];
      const int sc = (int)(a.boff[c + 1] - b0);
      warp_sort_any(a.bmem + b0, sc, lane);
      __syncwarp();
      for (int i = lane; i < sc; i += 32) {
        const int32_t r = a.ent_v[a.bmem[b0 + i]];
        a.brank[b0 + i] = r;
#pragma unroll
        for (int k = 0; k < 2 * W; ++k) a.bxz[2 * W * (b0 + i) + k] = a.xz_r[2 * W * (int64_t)r + k];
      }
    }
    if (!engine_sync<MODE>(a, __LINE__, round)) return;

    if constexpr (W == 1)
      bucket_bits_tab(a, smem_dyn + (size_t)wid * warp_smem_bytes<W>(), lane, gwarp, nwarps);
    else
      bucket_bits<W>(a, Rw, Xw, lane, gwarp, nwarps);
    if (!engine_sync<MODE>(a, __LINE__, round)) return;
    {
      // the round's CSR, counted as the byte budget counts it (8 bytes per
      // row and one, 4 per run entry): over the budget, the round goes back
      const int64_t nnz = __ldcg(a.ctl + 3);
      const int64_t csr_bytes = 8 * (n + 1) + 4 * nnz;
      if (a.budget > 0 && csr_bytes > a.budget) {
        if (!engine_sync<MODE>(a, __LINE__, round)) return;
        if (gtid == 0) a.ctl[2] = kSmallOverflow;
        break;
      }
    }
    if (gtid == 0) a.ctl[6] += __ldcg(a.ctl + 3);

    // ordered first fit in rank order
    {
      ColorArgs ca{};
      ca.n = n;
      ca.lists = a.lists;
      ca.loff = a.loff;
      ca.state = a.state;
      ca.ranked = 1;
      ca.rinfo = a.rinfo;
      ca.rmask = a.rmask;
      ca.cmask = a.cmask;
      ca.Lu = nsets == 1 ? a.ptab[n].y : 0;  // one set: row of rank r = r L
      ca.max_polls = a.max_polls;
      // warp w takes ranks w, w + W, ... (every warp of the launch is
      // resident, so the earliest undecided rank always progresses); the
      // next rank's list entries are loaded while this one is colored
      uint32_t nc = 0u;
      int64_t nrb = 0;
      if (gwarp < n) mask_entry<true>(ca, (int32_t)gwarp, lane, &nc, &nrb);
      for (int64_t t = gwarp; t < n; t += nwarps) {
        const uint32_t c0 = nc;
        const int64_t rb0 = nrb;
        if (t + nwarps < n) mask_entry<true>(ca, (int32_t)(t + nwarps), lane, &nc, &nrb);
        if (__ldcg(a.err) != 0 || !mask_vertex<true>(ca, (int32_t)t, lane, a.err, true, c0, rb0)) break;
      }
    }
    if (!engine_sync<MODE>(a, __LINE__, round)) return;
    if (__ldcg(a.err) != 0) {
      if (gtid == 0) a.ctl[2] = kSmallTimeout;
      break;
    }

    // carry, in the scan of the uncolored flags (V_l order): colors at global
    // ids (final color = the set's base + bucket color - the set's offset)
    // on the summing pass; pos[i] (the rank of i) becomes the number of
    // uncolored vertices before i.  The buckets, masks and counters are
    // emptied for the next round (its P is at most this round's).
    for (int64_t c = gtid; c < P; c += gthreads) {
      a.bcnt[c] = 0;
      a.bcur[c] = 0;
    }
    for (int64_t t = gtid; t < 32 * P; t += gthreads) a.cmask[t] = 0u;
    if (gtid == 0) a.ctl[3] = 0;
    {
      auto get = [&](int64_t i, bool first, int64_t* y) {
        const int64_t r = __ldcg(a.pos + i);
        const uint32_t w = (uint32_t)__ldcg(a.state + r);
        const bool colored = (w & 3u) == kColored;
        if (first && colored) {
          const int k = a.sid[r];
          a.color[gid[i]] = (int32_t)(a.sbase[k] + ((int64_t)(w >> 2) - a.scof[k]));
        }
        y[0] = colored ? 0 : 1;
      };
      auto put = [&](int64_t i, const int64_t* ex) { a.pos[i] = ex[0]; };
      if (!engine_scan<MODE, 1>(a, round, n, scan_s, get, put)) return;
    }
    if (!engine_sync<MODE>(a, __LINE__, round)) return;
    // the uncolored set in ascending global id, with its keys for the next
    // round
    for (int64_t i = gtid; i < n; i += gthreads) {
      const int64_t p0 = a.pos[i];
      if (a.pos[i + 1] != p0) {
        const int32_t g = gid[i];
        gid_next[p0] = g;
        const int k = nsets > 1 ? find_set(a.soff, nsets, g) : 0;
        a.key[p0] = ((uint64_t)philox_block(a.sseed[k], round + 1, g - a.soff[k], kTagPrio, 0u).x << 32) | (uint32_t)g;
      }
    }
    if (blockIdx.x == 0) {
      // per set: next palette base, largest CSR bytes of a round, vertices
      // left; then the next round's offsets
      int64_t pairs = 0;
      for (int k = threadIdx.x; k < nsets; k += blockDim.x) {
        const int64_t v0 = a.svoff[k], v1 = a.svoff[k + 1];
        const int64_t nk = v1 - v0;
        if (nk > 0) {
          const int64_t nnzk = a.snnz[k];
          a.sbase[k] += a.scof[k + 1] - a.scof[k];
          a.speak[k] = max(a.speak[k], 8 * (nk + 1) + 4 * nnzk);
          pairs += nk * (nk - 1) / 2;
        }
        a.snnz[k] = 0;
        a.srem[k] = a.pos[v1] - a.pos[v0];
      }
      pairs = block_sum(pairs, scan_s);
      if (threadIdx.x == 0) {
        a.ctl[0] = a.pos[n];
        a.ctl[1] = done + 1;
        a.ctl[4] = __ldcg(a.ctl + 4) ^ 1;
        a.ctl[7] += pairs;
      }
      __syncthreads();
      set_prefixes(a, scan_s);
    }
    if (!engine_sync<MODE>(a, __LINE__, round)) return;
  }
}

size_t small_smem_bytes(int32_t qw) {
  return (size_t)kSmallWarps * (qw == 2 ? warp_smem_bytes<2>() : warp_smem_bytes<1>());
}

// Up to three stages back to back on s: the grid launch (cooperative, up to
// kSmallBlocksPerSm blocks per SM) runs the rounds above the cluster's and
// the block's thresholds, the cluster launch (one cluster of cluster_blocks
// blocks; a.handoff > 0) the rounds above a.handoff2 vertices, the block
// launch (a.handoff2 > 0) the rest.  A stage with no round left returns at
// once.
cudaError_t launch_small_rounds(const SmallArgs& a, int part_cap, int cluster_blocks, int blocks_per_sm,
                                cudaStream_t s) {
  int dev = 0, sms = 148, per_sm = 0;
  if (a.qw != 1 && a.qw != 2) return cudaErrorInvalidValue;
  // the mask coloring reads the color masks 16 bytes at a time
  if (reinterpret_cast<uintptr_t>(a.cmask) & 15) return cudaErrorMisalignedAddress;
  const size_t smem = small_smem_bytes(a.qw);
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t hb = std::max<int64_t>(a.handoff2, 0);
  const int64_t hc = cluster_blocks > 0 ? std::max<int64_t>(a.handoff, 0) : 0;
  const bool cluster_stage = hc > hb && a.n0 > hb;
  SmallArgs args = a;
  args.handoff = std::max(hc, hb);  // where the grid stage stops
  args.handoff2 = hb;               // where the cluster stage stops
  if (args.handoff == 0 || a.n0 > args.handoff) {
    auto kern = a.qw == 2 ? k_small_rounds<2, kModeGrid> : k_small_rounds<1, kModeGrid>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSmallThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    // fewer resident blocks make each grid barrier cheaper; two per SM keep
    // 16 warps per SM for the latency-bound phases
    int blocks = std::min(per_sm, blocks_per_sm > 0 ? std::min(blocks_per_sm, kSmallBlocksPerSm) : kSmallBlocksPerSm) *
                 sms;
    blocks = std::min(blocks, part_cap / 3);  // the scans' block sums: 3 words a block
    blocks = (int)debug_grid(blocks);
    void* params[] = {(void*)&args};
    e = cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)blocks), dim3(kSmallThreads), params,
                                    smem, s);
    count_launches(1);
    if (e != cudaSuccess) return e;
  }
  if (cluster_stage) {
    auto kern = a.qw == 2 ? k_small_rounds<2, kModeCluster> : k_small_rounds<1, kModeCluster>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && cluster_blocks > 8)
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)std::min(cluster_blocks, part_cap / 3);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(attr[0].val.clusterDim.x);
    cfg.blockDim = dim3(kSmallThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, args);
    count_launches(1);
    if (e != cudaSuccess) return e;
  }
  if (hb > 0) {
    auto kern = a.qw == 2 ? k_small_rounds<2, kModeBlock> : k_small_rounds<1, kModeBlock>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<1, kSmallThreads, smem, s>>>(args);
    count_launches(1);
    e = cudaGetLastError();
  }
  return e;
}

// Largest cluster (16, 8, 4, 2 blocks) the engine's cluster launch can have
// resident on this device, 0 if none.
int small_cluster_blocks(int32_t qw) {
  if (qw != 1 && qw != 2) return 0;
  const size_t smem = small_smem_bytes(qw);
  auto kern = qw == 2 ? k_small_rounds<2, kModeCluster> : k_small_rounds<1, kModeCluster>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) return 0;
  for (int k = 16; k >= 2; k >>= 1) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)k;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(k);
    cfg.blockDim = dim3(kSmallThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) == cudaSuccess && nc >= 1) return k;
    cudaGetLastError();
  }
  return 0;
}

}  // namespace picasso
