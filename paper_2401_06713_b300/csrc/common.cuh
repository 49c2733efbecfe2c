// common.cuh -- device helpers and internal launcher declarations of
// libpicasso (sm_103a).  Nothing here is part of the C ABI.
//
// A round works on a batch of one or more independent string sets at once,
// as one disjoint-union instance.  Vertices are ordered by set, then by
// global id; every vertex v owns the list entries loff[v] .. loff[v+1]
// (L of its set), and list colors are "bucket colors": the round-local
// color of the set plus the set's color offset cofs, so the color buckets of
// different sets never meet and no pair of vertices of different sets is
// ever tested.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/picasso.h"

namespace picasso {

constexpr uint32_t kTagList = 1u;
constexpr uint32_t kTagPrio = 2u;
constexpr uint32_t kTagDynamic = 4u;  // Alg. 2's color draw
constexpr int kMaxL = 512;           // longest list a round may draw
constexpr int kMaxPolls = 1 << 20;   // default polls of one bounded device wait
constexpr int kBucketCap = 2048;     // largest color bucket of the bucket join
constexpr int kBucketMaxP = 1 << 21; // bucket colors of one round (bucket join)
constexpr int kClistWords = 8;       // colored-list words per color (ordered coloring)
constexpr int64_t kSmallRoundAllPairs = 2048;  // AUTO tests all pairs at or below this n
constexpr uint32_t kFailedColor = 0x3FFFFFFFu;

// Vertex state word of the coloring: bits 31..2 a bucket color, bits 1..0 the
// state.  Undecided: the color is the current candidate.
constexpr uint32_t kUndecided = 0u, kColored = 1u, kFailed = 2u;

// One set's parameters in the current round (device table, one entry per set).
struct SetRound {
  uint64_t seed;  // Philox key of the set
  int64_t P;      // palette size P_l of the set
  int64_t cofs;   // bucket-color offset of the set in this round
  int64_t base;   // the set's palette base: final color = base + (c - cofs)
  int32_t L;      // list size L_l of the set
  int32_t pad;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit products; the key advances by the Weyl constants between
// rounds.
// ---------------------------------------------------------------------------
struct u32x4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = u32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
  }
  return c;
}

// Block b of stream (seed, round, gid, tag).
__device__ __forceinline__ u32x4 philox_block(uint64_t seed, int32_t round, int64_t gid,
                                              uint32_t tag, uint32_t b) {
  u32x4 c{(uint32_t)((uint64_t)gid & 0xffffffffu), (uint32_t)((uint64_t)gid >> 32), (uint32_t)round,
          (tag << 24) | b};
  return philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
}

__device__ __forceinline__ uint32_t pick(const u32x4& v, uint32_t i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// Alg. 1 assign_rand_list_colors for one vertex: Floyd's sampling of L
// distinct values of [0, P) (Bentley & Floyd, CACM 1987): for j = P-L .. P-1
// draw t in [0, j] (x*(j+1) >> 32 of the next Philox word of the LIST stream
// (seed, round, g)); keep t, or j if t was already kept.  Then an insertion
// sort; out[0..L) = cofs + the sorted values.  L <= LCAP.
template <int LCAP>
__device__ __forceinline__ void draw_list(uint64_t seed, int32_t round, int64_t g, int64_t P, int L, int64_t cofs,
                                          int32_t* __restrict__ out) {
  uint32_t sel[LCAP];
  u32x4 blk{0, 0, 0, 0};
  for (int m = 0; m < L; ++m) {
    if ((m & 3) == 0) blk = philox_block(seed, round, g, kTagList, (uint32_t)(m >> 2));
    const uint32_t x = pick(blk, (uint32_t)(m & 3));
    const uint64_t j = (uint64_t)(P - L + m);
    const uint32_t t = (uint32_t)(((uint64_t)x * (j + 1)) >> 32);
    bool seen = false;
    for (int a = 0; a < m; ++a) seen |= (sel[a] == t);
    sel[m] = seen ? (uint32_t)j : t;
  }
  for (int a = 1; a < L; ++a) {
    const uint32_t key = sel[a];
    int b = a - 1;
    while (b >= 0 && sel[b] > key) {
      sel[b + 1] = sel[b];
      --b;
    }
    sel[b + 1] = key;
  }
  for (int a = 0; a < L; ++a) out[a] = (int32_t)(cofs + sel[a]);
}

// draw_list for L <= 32 with the picks in registers: the same draws as
// draw_list (Floyd's sampling on the same Philox words), every loop unrolled
// so no pick leaves registers, then ascending order by a 32-wide bitonic
// network (unused slots hold the maximum and sort last).  With bcount, the
// bucket color of every pick is also counted.
__device__ __forceinline__ void draw_list32(uint64_t seed, int32_t round, int64_t g, int64_t P, int L, int64_t cofs,
                                            int32_t* __restrict__ out, uint32_t* __restrict__ bcount) {
  uint32_t sel[32];
  u32x4 blk{0, 0, 0, 0};
#pragma unroll
  for (int m = 0; m < 32; ++m) {
    sel[m] = 0xFFFFFFFFu;
    if (m < L) {
      if ((m & 3) == 0) blk = philox_block(seed, round, g, kTagList, (uint32_t)(m >> 2));
      const uint32_t x = pick(blk, (uint32_t)(m & 3));
      const uint64_t j = (uint64_t)(P - L + m);
      const uint32_t t = (uint32_t)(((uint64_t)x * (j + 1)) >> 32);
      bool seen = false;
#pragma unroll
      for (int a = 0; a < m; ++a) seen |= (sel[a] == t);
      sel[m] = seen ? (uint32_t)j : t;
    }
  }
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int d = k >> 1; d > 0; d >>= 1) {
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int l = i ^ d;
        if (l > i) {
          const bool up = (i & k) == 0;
          const uint32_t x = sel[i], y = sel[l];
          const bool sw = (x > y) == up;
          sel[i] = sw ? y : x;
          sel[l] = sw ? x : y;
        }
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 32; ++a) {
    if (a < L) {
      const int32_t c = (int32_t)(cofs + sel[a]);
      out[a] = c;
      if (bcount) atomicAdd(bcount + c, 1u);
    }
  }
}

// Symplectic commutation test for one-word strings.
__device__ __forceinline__ bool commute1(uint64_t xu, uint64_t zu, uint64_t xv, uint64_t zv) {
  return (__popcll((xu & zv) ^ (zu & xv)) & 1) == 0;
}

// The same for strings of W words per part (a string is x_0 .. x_{W-1},
// z_0 .. z_{W-1}): the symplectic form is a sum over the words, so the
// words' terms are XORed and one parity taken.
__device__ __forceinline__ bool commuteW(const uint64_t* __restrict__ u, const uint64_t* __restrict__ v, int W) {
  uint64_t acc = 0;
  for (int w = 0; w < W; ++w) acc ^= (u[w] & v[W + w]) ^ (u[W + w] & v[w]);
  return (__popcll(acc) & 1) == 0;
}

constexpr int kMaxQ = 1024;  // qubits of a string: at most 16 words per part
constexpr size_t kWideMaskSmem = 200 * 1024;  // shared memory of the direct wide mask pass
constexpr int kWideTabSlices = 4;             // words per part the table pass serves (q <= 256)
constexpr size_t kWideTabSmem = 225 * 1024;   // shared memory of the table pass
// whether the mask pass for strings of qw > 1 words per part holds a bucket
// of smax members in shared memory
bool wide_mask_fits(int64_t smax, int32_t qw);

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch with a time limit.  bar: one
// word, zero before the launch (two are reserved).  Thread 0 of every block
// adds to it once per call: block 0 adds 2^31 - (blocks - 1), the others
// add 1, so the word's top bit flips exactly when the last block arrives
// and its other bits come back to where they were.  A block waits until the
// top bit differs from the value it found; one that waits longer than
// limit_ns (by the global timer), or sees *abort set, sets *abort, writes
// the arrivals it saw to *seen and returns false: the caller then ends the
// kernel, and every other block leaves at its next barrier.  Writes made
// before the barrier by any block are visible after it (fences on both
// sides).
constexpr uint64_t kBarrierLimitNs = 4000000000ull;
__device__ __forceinline__ bool grid_sync_bounded(unsigned int* bar, int* abort, uint64_t limit_ns, int* seen) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int inc = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
    volatile unsigned int* vb = bar;
    __threadfence();
    const unsigned int old = atomicAdd(bar, inc);
    // spin (an L2 round trip per poll); the clock and the abort flag every
    // 64 polls
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1; ((old ^ *vb) & 0x80000000u) == 0u; ++it) {
      if ((it & 63u) != 0u) continue;
      if (*(volatile int*)abort) {
        ok = 0;
        break;
      }
      if (global_ns() - t0 > limit_ns) {
        *seen = (int)(*vb & 0x7fffffffu);
        atomicExch(abort, 1);
        ok = 0;
        break;
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Set of batch-global vertex id g: the k with soff[k] <= g < soff[k+1].
__device__ __forceinline__ int set_of(const int64_t* __restrict__ soff, int nsets, int64_t g) {
  int lo = 0, hi = nsets - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (soff[mid] <= g)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Process-wide launch counter (capi.cu); every launcher adds its launches.
void count_launches(int k);
// Grid of the persistent and grid-stride kernels: the launcher's choice,
// divided by the PICASSO_GRID_DIVISOR environment variable when it is set
// (a debugging aid: every such kernel gives the same output at any grid
// size, so runs at different divisors must agree bit for bit).
int64_t debug_grid(int64_t blocks);


// ---------------------------------------------------------------------------
// Launchers (host functions defined in the kernel .cu files).
// ---------------------------------------------------------------------------
cudaError_t launch_pack(const uint8_t* codes, int64_t n, int32_t q, uint64_t* xz, cudaStream_t s);
cudaError_t launch_philox_draws(uint64_t seed, int32_t round, int64_t gid, uint32_t tag, uint32_t i0,
                                int32_t count, uint32_t* out, cudaStream_t s);

// Round vertices: gid[v] is the batch-global id (nullptr: identity), soff
// [nsets+1] the batch's set offsets (global ids), sets [nsets] this round's
// set table.  List lengths -> loff (len: [n] scratch, tmp: scan scratch).
cudaError_t launch_list_offsets(const int32_t* gid, int64_t n, const int64_t* soff, int32_t nsets,
                                const SetRound* sets, uint32_t* len, int64_t* loff, void* tmp, cudaStream_t s);
// ent_v[e] = vertex owning list entry e.
// loff[v] = v L for v <= n (every vertex has L entries)
cudaError_t launch_strided_offsets(int64_t* loff, int64_t n, int32_t L, cudaStream_t s);
cudaError_t launch_entry_owner(const int64_t* loff, int64_t n, int32_t* ent_v, cudaStream_t s);
// Alg. 1 list assignment: lists[loff[v] ..] = sorted bucket colors, prio[v].
// Priorities of the round's vertices (draw 0 of the PRIO stream), no lists.
cudaError_t launch_round_prio(int32_t round, const int32_t* gid, int64_t n, const int64_t* soff, int32_t nsets,
                              const SetRound* sets, uint32_t* prio, cudaStream_t s);
// bcount (may be null; used when every list has at most 32 colors): bucket
// sizes, counted as the lists are drawn (zeroed by the caller).
cudaError_t launch_assign_lists(int32_t round, const int32_t* gid, int64_t n, const int64_t* soff, int32_t nsets,
                                const SetRound* sets, int32_t Lmax, const int64_t* loff, int32_t* lists,
                                uint32_t* prio, uint32_t* bcount, cudaStream_t s);

// Exclusive scan of n uint32 counts into out[n+1] (int64); tmp needs
// scan_tmp_bytes(n) bytes.
size_t scan_tmp_bytes(int64_t n);
cudaError_t launch_scan_u32(const uint32_t* in, int64_t n, int64_t* out, void* tmp, cudaStream_t s);
// out[e] = rinfo_len(rinfo[e]): the bit layout's run lengths, e < E.
cudaError_t launch_rinfo_lengths(const int64_t* rinfo, int64_t E, uint32_t* out, cudaStream_t s);

// One word per list entry of the bit layout: row address (bits 0..37, in
// words of the bit rows), bucket slot (bits 38..46) and run length (bits
// 47..55; a run never passes the slot, and slots stay below kFusedMax).
constexpr int kRinfoAddrBits = 38;
__host__ __device__ inline int64_t rinfo_pack(int64_t addr, int slot, int len) {
  return addr | ((int64_t)slot << kRinfoAddrBits) | ((int64_t)len << (kRinfoAddrBits + 9));
}
__host__ __device__ inline int64_t rinfo_addr(int64_t r) { return r & ((int64_t(1) << kRinfoAddrBits) - 1); }
__host__ __device__ inline int rinfo_slot(int64_t r) { return (int)((r >> kRinfoAddrBits) & 511); }
__host__ __device__ inline int rinfo_len(int64_t r) { return (int)((r >> (kRinfoAddrBits + 9)) & 511); }

// Conflict build.  Run k of row v is runoff[loff[v] + k] .. runoff[loff[v]+k+1].
struct ConflictArgs {
  int64_t n;             // vertices of the round
  int64_t E;             // list entries (= loff[n])
  int32_t Lmax;          // longest list of the round
  int32_t Lu;            // L of every vertex when all lists have one length
                         // (loff[v] = v * Lu; ent_v unused), else 0
  int64_t P;             // bucket colors of the round (sum of the sets' P)
  const uint64_t* xz;    // [n][2 qw]: x words, then z words
  int32_t qw;            // 64-bit words per part: ceil(q / 64)
  const int32_t* lists;  // [E] bucket colors, ascending within each vertex
  const int64_t* loff;   // [n+1]
  const int32_t* ent_v;  // [E] vertex of each list entry
  uint32_t* cnt;         // [E] run lengths          (count / mask pass)
  const int64_t* runoff; // [E+1]                    (fill / emit pass)
  int32_t* col;          // [nnz]                    (fill / emit pass)
  int32_t* err;          // device error word
  uint32_t* rmask;       // bucket join: run words (mask pass -> emit)
  int32_t lower;         // 1: rows keep only neighbours with a smaller id
  const uint4* bxz;               // [E] member words in bucket-slot order (x lo, x hi, z lo, z hi)
  const int32_t* bpid;            // [E] member vertex ids in bucket-slot order
  // bit layout (launch_bucket_bits): bucket b's lower blocks are stored
  // row-major at rmask + moff[b]: row i (block R = i / 32) has R + 1 words,
  // word W's bit t = partner slot 32 W + t (< i) commutes with i.  Entry e,
  // member i of bucket b, gets one word rinfo[e] (rinfo_* below): the
  // address of row i, moff[b] + 16 R (R + 1) + (i % 32) (R + 1), the slot i
  // and the run length (the set bits of the row); *nnz gets the sum of the
  // run lengths (one atomic per bucket)
  int64_t* rinfo;                 // [E]
  unsigned long long* nnz;        // one word, zero on entry
  int32_t rowmajor;               // emit pass: a.rmask holds the bit layout's row-major
                                  // rows (row r of block R at 16 R (R + 1) + r (R + 1))
};

// Buckets: members of color c are bmem[boff[c] .. boff[c+1]) ascending; a
// member is stored as its list-entry index e (owner ent_v[e], position
// e - loff[owner]).
cudaError_t launch_bucket_hist(const int32_t* lists, int64_t E, uint32_t* bcount, cudaStream_t s);
// The same sizes, and the members' places, without global atomics (kernels
// in kernels_conflict.cu): entries cut into G = bucket_hist_blocks(E) ranges,
// hist [G][P rounded up to even] 16-bit counts, then per range and color the
// count of the ranges before it; bcount[c] the bucket sizes.  P <= kHistMaxP.
// launch_bucket_place writes bmem[boff[c] + ...] like launch_bucket_fill
// (members in entry order across ranges, in arrival order within one).
constexpr int64_t kHistMaxP = 110000;  // 16-bit counters of P colors in one block's shared memory
int64_t bucket_hist_blocks(int64_t E);
cudaError_t launch_bucket_count(const int32_t* lists, int64_t E, int64_t P, uint16_t* hist, int64_t G,
                                uint32_t* bcount, cudaStream_t s);
cudaError_t launch_bucket_place(const int32_t* lists, int64_t E, int64_t P, const uint16_t* hist, int64_t G,
                                const int64_t* boff, int32_t* bmem, cudaStream_t s);
cudaError_t launch_bucket_fill(const int32_t* lists, int64_t E, const int64_t* boff, uint32_t* bcursor,
                               int32_t* bmem, cudaStream_t s);
// near: every member lies within a few places of its own (the place pass):
// odd-even transposition passes instead of the full network.
cudaError_t launch_bucket_sort(const int64_t* boff, int64_t P, int32_t* bmem, int32_t* err, int32_t smax, bool near,
                               cudaStream_t s);
// out32[0] = max bucket size; out64[0] = sum over buckets of s (s - 1).
cudaError_t launch_bucket_stats(const uint32_t* bcount, int64_t P, uint32_t* out32,
                                unsigned long long* out64, cudaStream_t s);
// Bucket join: mask words per bucket (k_bucket_words + scan -> moff), the
// mask pass (pair tests, counts, words), then the emit pass (CSR writes).
// Mask words of every bucket: nwb^2 blocks of 32 words, or nwb (nwb + 1) / 2 with lower.
cudaError_t launch_bucket_words(const uint32_t* bcount, int64_t P, int32_t lower, uint32_t* words, cudaStream_t s);
cudaError_t launch_bucket_mask(const ConflictArgs& a, const int64_t* boff, const int32_t* bmem,
                               const int64_t* moff, int32_t smax, int32_t q, cudaStream_t s);
// Largest bucket the bit pass handles.
constexpr int kFusedMax = 512;
// The bit pass (EARLIER form, buckets of at most kFusedMax members, one word
// per part): the pair tests of launch_bucket_mask from the gathered members
// (a.bxz), the lower blocks row-major to a.rmask + moff[b], each entry's
// row address, slot and run length to a.rinfo, the run total to *a.nnz.  No
// run is written: the coloring reads the bits, the canonical CSR is made
// from them on request.
// per_sm_cap > 0: at most that many blocks per SM (the schedule's).
cudaError_t launch_bucket_bits(const ConflictArgs& a, const int64_t* boff, const int32_t* bmem, const int64_t* moff,
                               int32_t smax, int32_t q, cudaStream_t s, int per_sm_cap = 0);
// bxz[p], bpid[p]: words and vertex id of the member at bucket slot p < E.
// The warp sort of every bucket (all of at most 512 members) and, by the
// same warp, the members' words and vertex ids in slot order (bit pass).
cudaError_t launch_bucket_sort_gather(const int64_t* boff, int64_t P, int32_t* bmem, int32_t smax, bool near,
                                      const ConflictArgs& a, uint4* bxz, int32_t* bpid, cudaStream_t s);
cudaError_t launch_bucket_jblocks(const uint32_t* bcount, int64_t P, uint32_t* out, cudaStream_t s);
// jboff [P+1]: prefix of ceil(s_c / 32); counter: one device int32 (reset here)
// Rows of vertices in [lo, hi) only (a chunk of the round), written at
// runoff - base.
cudaError_t launch_bucket_emit(const ConflictArgs& a, const int64_t* boff, const int32_t* bmem,
                               const int64_t* moff, const int64_t* jboff, const int32_t* ibkt, int32_t* counter,
                               int64_t lo, int64_t hi, int64_t base, cudaStream_t s);
// ibkt [jboff[P]]: the bucket of every emit work item.
cudaError_t launch_item_bucket(const int64_t* jboff, int64_t P, int32_t* ibkt, cudaStream_t s);
cudaError_t launch_allpairs(const ConflictArgs& a, bool fill, cudaStream_t s);
// off[u] = runoff[loff[u]], u <= n.
cudaError_t launch_row_offsets(const int64_t* runoff, const int64_t* loff, int64_t n, int64_t* off,
                               cudaStream_t s);

// Coloring and carry.
struct ColorArgs {
  int64_t n;
  const int32_t* lists;
  const int64_t* loff;
  const int64_t* runoff;   // [E+1] canonical layout: run of entry e ends at runoff[e+1]
  int64_t cbase;           // canonical layout: run offsets are col indices + cbase
  int64_t v0;              // ordered pass: position t is vertex v0 + t (a chunk of the round)
  // bit layout (rinfo set; ConflictArgs gives the encoding): the run of
  // entry e is the set bits of its row words rmask[rinfo_addr(rinfo[e]) +
  // W], W <= slot / 32, slot = rinfo_slot(rinfo[e]); bit t of word
  // W is the member at slot 32 W + t of bucket c = lists[e], vertex
  // bpid[bboff[c] + 32 W + t]
  const int64_t* rinfo;
  const int64_t* bboff;
  int32_t Lu;           // every list has Lu colors (row of v = v Lu; loff unread), or 0
  const uint32_t* rmask;
  const int32_t* bpid;
  // mask coloring (bit layout; null: off): per bucket color c, 32 words at
  // 32 c, zero at the start of the round: words 0..15 mark the members
  // (by slot) colored c, words 16..31 those that will never take c
  uint32_t* cmask;
  const int32_t* col;
  uint64_t* state;  // [n] priority << 32 | state word
  uint16_t* kcur;   // [n] index of the current candidate in the list
  uint32_t* rcur;   // [n] resolved prefix of the current candidate's run
  int32_t* blk;     // [n] neighbour the vertex waited on last, or -1
  uint32_t* blkw;   // [n] the vertex's candidate color when it started waiting
  int32_t ranked;   // 1: round-local ids are ranks in coloring order, so the
                    // earlier neighbours of a run form its prefix
  // colored lists (ranked coloring only; null: off): per bucket color c,
  // kClistWords words at kClistWords c, zero at the start of the round:
  // word 0 counts the vertices colored c, the others hold rank + 1 of the
  // first of them
  uint32_t* clist;
  const uint64_t* xz;  // [n][2 qw] words in rank order (with clist)
  int32_t qw;          // 64-bit words per part
  int32_t max_polls;   // polls of one bounded wait before the kernel gives up
};
// Work list of all n vertices in ascending (priority, id): a counting sort on
// the top log2(nbins) priority bits, then a sort inside each bin.  hist needs
// nbins uint32, hoff nbins + 1 int64, tmp scan_tmp_bytes(nbins) bytes.
int prio_bins_for(int64_t n);
cudaError_t launch_prio_order(const uint32_t* prio, int64_t n, int nbins, uint32_t* hist, int64_t* hoff,
                              void* tmp, int32_t* work, cudaStream_t s);
cudaError_t launch_color_init(const ColorArgs& a, const uint32_t* prio, int32_t* nwork, cudaStream_t s);
// One sweep = wake (pending -> active or stays pending) + sweep (evaluate
// the active vertices; those still waiting join the pending list again).
cudaError_t launch_color_wake(const ColorArgs& a, const int32_t* work_in, const int32_t* nwork_in, int32_t* active,
                              int32_t* nactive, int32_t* work_out, int32_t* nwork_out, cudaStream_t s);
cudaError_t launch_color_sweep(const ColorArgs& a, const int32_t* work_in, const int32_t* nwork_in,
                               int32_t* work_out, int32_t* nwork_out, cudaStream_t s);
// Ordered persistent coloring of a round: `order` must list the vertices in
// exact (priority, id) order (launch_prio_order gives it).  On return *err
// is 1 if a bounded wait ran out (then recolor with launch_color_all).
cudaError_t launch_color_ordered(const ColorArgs& a, const int32_t* order, int32_t* err, cudaStream_t s,
                                 int per_sm_cap = 0);
// Every sweep of a round in one cooperative launch.  ctl [kCtlWords] int32:
// ctl[0] holds the pending count of wa on entry (launch_color_init writes
// it), the rest must be zero; on exit ctl[3] = sweeps, ctl[4] = 1 if the
// sweep limit (n + 4) ran out.  For the first kSweepLog sweeps the kernel
// logs the pending count (ctl[8 + s]), the globaltimer at the sweep's start
// (uint64 at ctl + 8 + kSweepLog, entry s) and the active count
// (ctl[8 + 3 kSweepLog + s]).
constexpr int kSweepLog = 64;
// after the sweep log: the bounded grid barrier (2 words), its abort flag
// (set when a barrier gave up; the launch ended) and the arrivals it saw
constexpr int kCtlBar = 8 + 4 * kSweepLog, kCtlAbort = kCtlBar + 2, kCtlSeen = kCtlBar + 3;
constexpr int kCtlWords = kCtlBar + 4;
cudaError_t launch_color_all(const ColorArgs& a, int32_t* wa, int32_t* wb, int32_t* wact, int32_t* ctl,
                             cudaStream_t s);
// Colors to the output (final color = base + bucket color - cofs of the
// vertex's set, written at its batch-global id) and flags of the uncolored.
// perm (may be null): flag index of round vertex v is perm[v] (the vertex's
// place in ascending global id) instead of v.
cudaError_t launch_carry_flags(const uint64_t* state, int64_t n, const int32_t* gid, const int32_t* perm,
                               const int64_t* soff, int32_t nsets, const SetRound* sets, int32_t* color,
                               uint32_t* flag, cudaStream_t s);
// Round arrays in coloring order: out[t] = in[perm[t]] for the global ids
// (identity when gid_in is null), packed words and priorities.
cudaError_t launch_rank_gather(const int32_t* perm, int64_t n, const int32_t* gid_in, const uint64_t* xz_in,
                               const uint32_t* prio_in, int32_t* gid_out, uint64_t* xz_out, uint32_t* prio_out,
                               int32_t S, cudaStream_t s);
cudaError_t launch_carry_gather(const uint32_t* flag, const int64_t* pos, int64_t n, const int32_t* gid,
                                const uint64_t* xz, int32_t* gid_out, uint64_t* xz_out, int32_t S, cudaStream_t s);
// Remaining vertices per set after a carry: hist[k] += 1 for each gid.
cudaError_t launch_set_counts(const int32_t* gid, int64_t n, const int64_t* soff, int32_t nsets, uint32_t* hist,
                              cudaStream_t s);
cudaError_t launch_gather_xz(const uint64_t* xz_all, const int32_t* gid, int64_t n, uint64_t* xz_out, int32_t S,
                             cudaStream_t s);
// out[k] (zeroed here) = 8 n_k + 4 * run entries of set k's vertices; the
// entries from runoff (canonical layout) or, if it is null, from cnt.
cudaError_t launch_set_csr_bytes(const int64_t* loff, const int64_t* runoff, const uint32_t* cnt, const int32_t* gid,
                                 int64_t n, const int64_t* soff, int32_t nsets, int64_t* out, cudaStream_t s);
cudaError_t launch_iota(int32_t* out, int64_t n, cudaStream_t s);

// Small-round engine (kernels_small.cu): every remaining round of a context
// (one set or a batch) in one cooperative launch once the round has at most
// kSmallRoundsMax vertices, every set's lists at most kSmallLCap colors and
// small color buckets (mean n_k L_k / P_k at most kSmallMeanBucket; a bucket
// above kSmallBucketCap stops the engine).  ctl[0..4] hold the engine's position between rounds
// (host-initialised); the launch returns with ctl[2] = kSmallOk when no
// vertex is left, or with the reason it stopped at the start of a round it
// did not finish (that round's vertex list intact, none of its colors
// written).
constexpr int64_t kSmallRoundsMax = 16384;
constexpr int kSmallLCap = 64;
constexpr int kSmallBucketCap = 512;  // largest color bucket
constexpr int kSmallMeanBucket = 320; // a set joins only if n L <= this * P
struct SmallArgs {
  int64_t n0;             // vertices when the engine starts
  int32_t round0;         // number of the first round it runs
  int32_t max_rounds;     // last round number it may run
  int32_t qw;             // 64-bit words per part of a string (1 or 2)
  int32_t nsets;          // sets of the context
  const int64_t* soff;    // [nsets + 1] global id offsets of the sets
  const uint64_t* sseed;  // [nsets] Philox keys
  int64_t* sbase;         // [nsets] palette base of the next round (in/out)
  int64_t* srem;          // [nsets] vertices of the set in the round (in/out)
  int64_t* speak;         // [nsets] largest CSR bytes of one round (in/out)
  int64_t* svoff;         // [nsets + 1] the round's offsets: vertices,
  int64_t* scof;          // [nsets + 1]   bucket colors (sum of P),
  int64_t* seoff;         // [nsets + 1]   list entries (sum of n L)
  const int2* ptab;       // [max n_k + 1]: (P, L) of a set with m vertices
  int64_t budget;         // byte budget of one round's CSR (0: none)
  const uint64_t* xz;     // [N][2] all strings
  int32_t* gid_a;         // [n0] V_l in ascending global id (ping-pong)
  int32_t* gid_b;         // [n0]
  int32_t* perm;          // [n0] rank -> place in V_l
  int32_t* gid_r;         // [n0] rank -> global id
  int32_t* sid;           // [n0] rank -> set
  uint64_t* xz_r;         // [2 n0] words in rank order
  int32_t* lists;         // [E0] (E0 = sum of n_k L_k at the start)
  int32_t* ent_v;         // [E0] list entry -> rank
  int64_t* loff;          // [n0 + 1]
  int64_t* rinfo;         // [E0] packed word of every list entry (bit layout)
  uint32_t* rmask;        // [wcap] the buckets' bit rows
  int64_t wcap;           // words rmask holds
  int64_t* moff;          // [P0 + 1] prefix of the words of the buckets' rows
  int64_t* snnz;          // [nsets] run entries of every set in the round
  uint32_t* cmask;        // [32 P0] the buckets' color masks of the mask coloring
  uint64_t* state;        // [n0]
  int64_t* pos;           // [n0 + 1] rank of V_l's i, then the uncolored before i
  int32_t* color;         // [N] global colors
  uint64_t* key;          // [n0] (priority, global id) in V_l order
  uint32_t* bcnt;         // [P0] bucket sizes (P0 = sum of P_k at the start)
  uint32_t* bcur;         // [P0] bucket fill cursors
  int64_t* boff;          // [P0 + 1] bucket offsets
  int64_t* iboff;         // [P0 + 1] prefix of the buckets' work items, ceil(s_c / 32)
  int32_t* ibkt;          // [E0 / 32 + P0 + 1] bucket of every work item
  int32_t* bmem;          // [E0] bucket members: list-entry index,
  int32_t* brank;         // [E0]   rank,
  uint64_t* bxz;          // [2 E0] words
  int64_t* part;          // [3 gridDim.x] block sums of the launch's scans
  int32_t* err;           // [4]: 0 ordered-pass poll timeout, 1 unused, 2 bucket over the cap,
                          //      3 a grid barrier timed out (the launch ended; ctl[9] its site,
                          //      ctl[10] its round, ctl[11] the arrivals it saw)
  int64_t* ctl;           // [kSmallCtlWords]: 0 n, 1 rounds done, 2 stop reason, 4 V_l in gid_b (0..4
                          //      host-initialised), 6 sum of nnz, 7 sum over the sets of
                          //      n_k (n_k - 1) / 2 (6, 7 zero on entry), 3 the round's run
                          //      entries, 5, 8 scratch
  int32_t max_polls;      // polls of one bounded wait before the engine gives up
  unsigned int* bar;      // [2] bounded grid barrier (zero before the grid launch)
  int64_t handoff;        // the cluster launch takes the rounds of at most this many
                          // vertices (0: no cluster launch)
  int64_t handoff2;       // the one-block launch takes the rounds of at most this
                          // many vertices (0: no block launch)
};

// Stop reasons in ctl[2].
constexpr int64_t kSmallOk = 0, kSmallTimeout = 1, kSmallOverflow = 2, kSmallMaxRounds = 3, kSmallHandoff = 4;
constexpr int kSmallCtlWords = 12;
// Rounds of at most this many vertices run in one thread-block cluster (the
// default of picasso_schedule.cluster_max_n).
constexpr int64_t kSmallClusterMaxN = 2048;
// Rounds of at most this many vertices run in one block (the default of
// picasso_schedule.block_max_n).
constexpr int64_t kSmallBlockMaxN = 64;
// part_cap: words of a.part; a launch uses at most part_cap / 3 blocks.  The
// grid launch runs the rounds above the later stages' thresholds, then
// (cluster_blocks > 0, a.handoff > 0) one cluster of cluster_blocks blocks
// the rounds above a.handoff2, then (a.handoff2 > 0) one block the rest,
// back to back on s.
cudaError_t launch_small_rounds(const SmallArgs& a, int part_cap, int cluster_blocks, int blocks_per_sm,
                                cudaStream_t s);
// Blocks of the largest cluster the engine can launch (16, 8, 4 or 2), 0 if none.
int small_cluster_blocks(int32_t qw);

// Alg. 2's dynamic order, parallel rule (kernels_dynamic.cu).  Rows are the
// two-sided canonical ones; lists of at most 64 colors.
struct DynArgs {
  int64_t n;
  int32_t round;
  int32_t nsets;
  const int64_t* soff;
  const SetRound* sets;
  const int32_t* gid;     // [n] global id of each round-local id
  const int64_t* loff;
  const int32_t* lists;
  const int64_t* runoff;  // [E + 1]
  const int32_t* col;
  uint64_t* mask;         // [n] remaining list entries; 0 once finished
  int32_t* state;         // [n] 0 uncolored, 1 colored, 2 left uncolored
  int32_t* color;         // [n] bucket color taken
  int32_t* wa;            // [n] work lists: vertices to examine (by step parity)
  int32_t* wb;            // [n]
  int32_t* sel;           // [n] the step's local minima
  int32_t* fin;           // [n] the step's lists struck empty
  int32_t* blk;           // [n] a smaller uncolored neighbour (blocked vertices)
  int32_t* stamp;         // [n] last step + 1 the vertex was put on a work list
  int32_t* bstep;         // [n] last step + 1 the vertex was found blocked
  int32_t* parts;         // [n] parts of the vertex's examination finished
  int32_t* lng;           // [n] the step's vertices whose row heads decided nothing
  int32_t* ctl;           // [kDynCtlWords] list lengths, sel and fin lengths (by parity), steps,
                          // long list; 8..9 the bounded grid barrier, 10 its abort flag (the
                          // launch ended), 11 the arrivals it saw
};
constexpr int kDynCtlWords = 12;
// masks of full lists, state 0, wa = all vertices, ctl = {n, 0, ...}
cudaError_t launch_dyn_init(const DynArgs& d, cudaStream_t s);
// every step of the round in one cooperative launch; ctl[6] = steps on exit
cudaError_t launch_dyn_all(const DynArgs& d, cudaStream_t s);
// the state words the carry reads (colored: bucket color, else failed)
cudaError_t launch_dyn_finish(const DynArgs& d, uint64_t* words, cudaStream_t s);

// Parameter predictor and instance features (kernels_mlp.cu).
int mlp_param_count();
cudaError_t launch_mlp_forward(const void* w, const float* x, int B, float* y, cudaStream_t s);
cudaError_t launch_mlp_backward(const void* w, const float* x, const float* t, float wo0, float wo1, int B, float* grad,
                                float* loss, cudaStream_t s);
cudaError_t launch_mlp_adamw(float* master, void* w, const float* g, float* m, float* v, float lr, float b1,
                             float b2, float eps, float wd, int step, cudaStream_t s);
cudaError_t launch_to_bf16(const float* a, void* b, int n, cudaStream_t s);
// feat[4] is log2(budget / n) / 4 - 3 (log2_budget given), or 4 beta - 2
// when beta >= 0 (the weighted objective of Eq. ml)
cudaError_t launch_features(const uint64_t* xz, int64_t n, int32_t q, uint64_t seed, int64_t samples,
                            double log2_budget, unsigned long long* counts, float* feat, cudaStream_t s,
                            double beta = -1.0);
cudaError_t launch_fill_i32(int32_t* out, int64_t n, int32_t v, cudaStream_t s);

}  // namespace picasso
