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
// part) and ranks
template <int W>
__host__ __device__ constexpr int warp_smem_bytes() { return kSmallBucketCap * (16 * W + 4); }

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

// Barrier of every thread of the launch: the cooperative grid's, or, when
// the launch is one thread-block cluster (CL), the cluster's hardware
// barrier (release / acquire at cluster scope, which covers global memory
// written by the cluster's blocks).
template <bool CL>
__device__ __forceinline__ bool engine_sync(const SmallArgs& a, int site, int64_t round) {
  if constexpr (CL) {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    return true;
  } else {
    // the grid's barrier is bounded in time: a block that gives up records
    // where (first one only) and the launch ends with err[3] set
    int seen = -1;
    if (grid_sync_bounded(a.bar, a.err + 3, kBarrierLimitNs, &seen)) return true;
    if (threadIdx.x == 0 && seen >= 0 && atomicCAS((unsigned long long*)(a.ctl + 9), 0ull, (unsigned long long)site) == 0ull) {
      a.ctl[10] = round;
      a.ctl[11] = seen;
    }
    return false;
  }
}

// Exclusive scan of in[0..m) into out[0..m] (out[m] = the total) by the
// whole grid: block b scans the b-th contiguous chunk after adding the sums
// of the chunks before it (part: one word per block).  Contains a grid
// barrier; every thread of the grid must call it.
template <bool CL, class TI>
__device__ bool grid_scan(const SmallArgs& a, int64_t round, const TI* in, int64_t m, int64_t* out, int64_t* part,
                          int64_t* sm) {
  const int64_t chunk = (m + gridDim.x - 1) / gridDim.x;
  const int64_t lo = min(m, chunk * (int64_t)blockIdx.x), hi = min(m, lo + chunk);
  int64_t x = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) x += (int64_t)in[i];
  x = block_sum(x, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = x;
  if (!engine_sync<CL>(a, __LINE__, round)) return false;
  int64_t pre = 0;
  for (int64_t b = threadIdx.x; b < blockIdx.x; b += blockDim.x) pre += __ldcg(part + b);
  pre = block_sum(pre, sm);
  for (int64_t t0 = lo; t0 < hi; t0 += blockDim.x) {
    const int64_t i = t0 + threadIdx.x;
    const int64_t v = i < hi ? (int64_t)in[i] : 0;
    int64_t tot = 0;
    const int64_t ex = block_excl(v, sm, &tot);
    if (i < hi) out[i] = pre + ex;
    pre += tot;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[m] = pre;
  return true;
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

template <int W, bool CL>
__global__ void __launch_bounds__(kSmallThreads, kSmallBlocksPerSm) k_small_rounds(SmallArgs a) {
  extern __shared__ __align__(16) unsigned char smem_dyn[];
  __shared__ int64_t scan_s[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint64_t* Xw = reinterpret_cast<uint64_t*>(smem_dyn + (size_t)wid * warp_smem_bytes<W>());
  int32_t* Rw = reinterpret_cast<int32_t*>(Xw + 2 * W * kSmallBucketCap);
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t gwarp = gtid >> 5, nwarps = gthreads >> 5;
  // per-vertex loops spread over all blocks: thread t of block b takes t G + b
  const int64_t stid = (int64_t)threadIdx.x * gridDim.x + blockIdx.x;
  const int nsets = a.nsets;

  // the cluster launch takes over from a grid launch that handed off (not
  // from one whose barrier timed out)
  if (CL && a.err[3] != 0) return;
  if (CL && gtid == 0 && a.ctl[2] == kSmallHandoff) a.ctl[2] = kSmallOk;
  if (blockIdx.x == 0) set_prefixes(a, scan_s);
  if (!engine_sync<CL>(a, __LINE__, 0)) return;

  while (true) {
    const int64_t n = __ldcg(a.ctl + 0);
    const int64_t done = __ldcg(a.ctl + 1);
    const int32_t round = a.round0 + (int32_t)done;
    if (n == 0 || __ldcg(a.ctl + 2) != kSmallOk) break;
    if (round > a.max_rounds) {
      if (!engine_sync<CL>(a, __LINE__, round)) return;
      if (gtid == 0) a.ctl[2] = kSmallMaxRounds;
      break;
    }
    if (!CL && n <= a.handoff) {
      // small enough for one cluster: its barriers cost far less
      if (!engine_sync<CL>(a, __LINE__, round)) return;
      if (gtid == 0) a.ctl[2] = kSmallHandoff;
      break;
    }
    const int32_t* gid = __ldcg(a.ctl + 4) ? a.gid_b : a.gid_a;
    int32_t* gid_next = __ldcg(a.ctl + 4) ? a.gid_a : a.gid_b;
    const int64_t P = a.scof[nsets];
    const int64_t E = a.seoff[nsets];

    // (priority, global id) keys in V_l order; empty buckets
    for (int64_t i = stid; i < n; i += gthreads) {
      const int k = nsets > 1 ? find_set(a.svoff, nsets, i) : 0;
      const int32_t g = gid[i];
      a.key[i] = ((uint64_t)philox_block(a.sseed[k], round, g - a.soff[k], kTagPrio, 0u).x << 32) | (uint32_t)g;
    }
    for (int64_t c = gtid; c < P; c += gthreads) {
      a.bcnt[c] = 0;
      a.bcur[c] = 0;
    }
    // the buckets' color masks of the mask coloring start empty; the
    // round's run counts at zero
    for (int64_t t = gtid; t < 32 * P; t += gthreads) a.cmask[t] = 0u;
    for (int64_t k = gtid; k < nsets; k += gthreads) a.snnz[k] = 0;
    if (gtid == 0) a.ctl[3] = 0;
    if (gtid == 0) a.err[1] = 0;
    if (!engine_sync<CL>(a, __LINE__, round)) return;

    // rank of vertex i = its set's offset + the number of smaller keys in the
    // set: warp per vertex, lanes over the set; the round's arrays are
    // written at the rank
    for (int64_t i = gwarp; i < n; i += nwarps) {
      const int k = nsets > 1 ? find_set(a.svoff, nsets, i) : 0;
      const int64_t v0 = a.svoff[k], v1 = a.svoff[k + 1];
      const uint64_t ki = a.key[i];
      int r = 0;
      for (int64_t j = v0 + lane; j < v1; j += 32) r += a.key[j] < ki;
      const int64_t rk = v0 + __reduce_add_sync(0xffffffffu, r);
      if (lane == 0) {
        const int32_t g = (int32_t)(uint32_t)ki;
        a.perm[rk] = (int32_t)i;
        a.gid_r[rk] = g;
        a.sid[rk] = k;
#pragma unroll
        for (int k = 0; k < 2 * W; ++k) a.xz_r[2 * W * rk + k] = a.xz[2 * W * (int64_t)g + k];
      }
    }
    if (!engine_sync<CL>(a, __LINE__, round)) return;

    // lists in rank order (bucket colors: + the set's offset), list offsets,
    // entry owners, first candidates (the ranked coloring reads no priority
    // from the state word), bucket sizes
    for (int64_t r = stid; r < n; r += gthreads) {
      const int k = a.sid[r];
      const int64_t v0 = a.svoff[k], nk = a.svoff[k + 1] - v0;
      const int2 pl = a.ptab[nk];
      const int64_t row = a.seoff[k] + (r - v0) * pl.y;
      int32_t* out = a.lists + row;
      draw_list<kSmallLCap>(a.sseed[k], round, a.gid_r[r] - a.soff[k], pl.x, pl.y, a.scof[k], out);
      a.loff[r] = row;
      a.state[r] = ((uint64_t)(uint32_t)out[0] << 2) | kUndecided;
      for (int t = 0; t < pl.y; ++t) {
        a.ent_v[row + t] = (int32_t)r;
        atomicAdd(a.bcnt + out[t], 1u);
      }
    }
    if (gtid == 0) a.loff[n] = E;
    // bucket work items (32 members each); a bucket above the cap stops the
    // engine
    if (!engine_sync<CL>(a, __LINE__, round)) return;
    for (int64_t c = gtid; c < P; c += gthreads) {
      const uint32_t sc = a.bcnt[c];
      const uint32_t nwb = (sc + 31) / 32;
      a.bitems[c] = nwb;
      a.bwords[c] = 16u * nwb * (nwb + 1u);  // the bucket's lower blocks, row-major
      if (sc > (uint32_t)kSmallBucketCap) a.err[2] = 1;
    }
    if (!grid_scan<CL>(a, round, a.bcnt, P, a.boff, a.part, scan_s)) return;
    if (!engine_sync<CL>(a, __LINE__, round)) return;
    if (!grid_scan<CL>(a, round, a.bitems, P, a.iboff, a.part, scan_s)) return;
    if (!engine_sync<CL>(a, __LINE__, round)) return;
    if (!grid_scan<CL>(a, round, a.bwords, P, a.moff, a.part, scan_s)) return;
    if (!engine_sync<CL>(a, __LINE__, round)) return;
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
    if (!engine_sync<CL>(a, __LINE__, round)) return;

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
    if (!engine_sync<CL>(a, __LINE__, round)) return;

    bucket_bits<W>(a, Rw, Xw, lane, gwarp, nwarps);
    if (!engine_sync<CL>(a, __LINE__, round)) return;
    {
      // the round's CSR, counted as the byte budget counts it (8 bytes per
      // row and one, 4 per run entry): over the budget, the round goes back
      const int64_t nnz = __ldcg(a.ctl + 3);
      const int64_t csr_bytes = 8 * (n + 1) + 4 * nnz;
      if (a.budget > 0 && csr_bytes > a.budget) {
        if (!engine_sync<CL>(a, __LINE__, round)) return;
        if (gtid == 0) a.ctl[2] = kSmallOverflow;
        break;
      }
    }
    if (!engine_sync<CL>(a, __LINE__, round)) return;
    if (gtid == 0) a.ctl[6] += __ldcg(a.ctl + 3);

    // ordered first fit in rank order; warps take ranks from a counter
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
      bool ok = true;
      while (ok) {
        int t = 0;
        if (lane == 0) t = atomicAdd(a.err + 1, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if ((int64_t)t >= n || __ldcg(a.err) != 0) break;
        ok = mask_vertex<true>(ca, t, lane, a.err);
      }
    }
    if (!engine_sync<CL>(a, __LINE__, round)) return;
    if (__ldcg(a.err) != 0) {
      if (gtid == 0) a.ctl[2] = kSmallTimeout;
      break;
    }

    // carry: colors at global ids (final color = the set's base + bucket
    // color - the set's offset), flags in V_l order
    for (int64_t r = gtid; r < n; r += gthreads) {
      const uint32_t w = (uint32_t)__ldcg(a.state + r);
      const bool colored = (w & 3u) == kColored;
      if (colored) {
        const int k = a.sid[r];
        a.color[a.gid_r[r]] = (int32_t)(a.sbase[k] + ((int64_t)(w >> 2) - a.scof[k]));
      }
      a.flag[a.perm[r]] = colored ? 0u : 1u;
    }
    if (!engine_sync<CL>(a, __LINE__, round)) return;
    if (!grid_scan<CL>(a, round, a.flag, n, a.pos, a.part, scan_s)) return;
    if (!engine_sync<CL>(a, __LINE__, round)) return;
    for (int64_t i = gtid; i < n; i += gthreads)
      if (a.flag[i]) gid_next[a.pos[i]] = gid[i];
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
    if (!engine_sync<CL>(a, __LINE__, round)) return;
  }
}

size_t small_smem_bytes(int32_t qw) {
  return (size_t)kSmallWarps * (qw == 2 ? warp_smem_bytes<2>() : warp_smem_bytes<1>());
}

// The grid launch (cooperative, up to kSmallBlocksPerSm blocks per SM) runs
// the rounds above a.handoff vertices; the cluster launch (one cluster of
// cluster_blocks blocks) runs the rest.  `cluster_blocks` 0: no cluster
// launch (the grid launch runs every round).
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
  SmallArgs args = a;
  if (cluster_blocks <= 0) args.handoff = 0;
  const bool grid_rounds = cluster_blocks <= 0 || a.n0 > args.handoff;
  if (grid_rounds) {
    auto kern = a.qw == 2 ? k_small_rounds<2, false> : k_small_rounds<1, false>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSmallThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    // fewer resident blocks make each grid barrier cheaper; two per SM keep
    // 16 warps per SM for the latency-bound phases
    int blocks = std::min(per_sm, blocks_per_sm > 0 ? std::min(blocks_per_sm, kSmallBlocksPerSm) : kSmallBlocksPerSm) *
                 sms;
    blocks = std::min(blocks, part_cap);
    blocks = (int)debug_grid(blocks);
    void* params[] = {(void*)&args};
    e = cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)blocks), dim3(kSmallThreads), params,
                                    smem, s);
    count_launches(1);
    if (e != cudaSuccess) return e;
  }
  if (cluster_blocks <= 0) return cudaSuccess;
  auto kern = a.qw == 2 ? k_small_rounds<2, true> : k_small_rounds<1, true>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && cluster_blocks > 8)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)std::min(cluster_blocks, part_cap);
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
  return e;
}

// Largest cluster (16, 8, 4, 2 blocks) the engine's cluster launch can have
// resident on this device, 0 if none.
int small_cluster_blocks(int32_t qw) {
  if (qw != 1 && qw != 2) return 0;
  const size_t smem = small_smem_bytes(qw);
  auto kern = qw == 2 ? k_small_rounds<2, true> : k_small_rounds<1, true>;
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
