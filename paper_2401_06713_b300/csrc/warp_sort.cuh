// warp_sort.cuh -- ascending sort of up to 512 int32 keys by one warp: a
// bitonic network in registers (lane l holds elements l*E .. l*E+E-1 of the
// padded size m = 32 E); partners closer than E are in the same lane,
// farther ones are exchanged by shuffles.  Internal header of the CUDA
// library (the bucket join of the per-round build and the small-round
// engine).
#pragma once

#include <stdint.h>

namespace picasso {

constexpr int kWarpSortMax = 512;

template <int E>
__device__ __forceinline__ void warp_bitonic(int32_t (&key)[E], int lane) {
  constexpr int m = 32 * E;
#pragma unroll
  for (int k = 2; k <= m; k <<= 1) {
#pragma unroll
    for (int d = k >> 1; d > 0; d >>= 1) {
      if (d < E) {
#pragma unroll
        for (int j = 0; j < E; ++j) {
          if ((j & d) == 0) {
            const int i = lane * E + j;
            const bool up = (i & k) == 0;
            const int32_t x = key[j], y = key[j | d];
            const bool sw = (x > y) == up;
            key[j] = sw ? y : x;
            key[j | d] = sw ? x : y;
          }
        }
      } else {
        const int ld = d / E;
        const bool lower = (lane & ld) == 0;
#pragma unroll
        for (int j = 0; j < E; ++j) {
          const int i = lane * E + j;
          const bool up = (i & k) == 0;
          const int32_t y = __shfl_xor_sync(0xffffffffu, key[j], ld);
          // the lower element keeps the smaller key when ascending
          key[j] = (lower == up) ? min(key[j], y) : max(key[j], y);
        }
      }
    }
  }
}

// Element i of a bucket at p[i], or (PAD: a copy in shared memory with one
// pad word every 16, so that lanes reading 16 consecutive elements each hit
// distinct banks) at p[i + i / 16].
template <bool PAD>
__device__ __forceinline__ int sort_at(int i) { return PAD ? i + (i >> 4) : i; }

template <int E, bool PAD = false>
__device__ __forceinline__ void warp_sort_bucket(int32_t* __restrict__ p, int s, int lane) {
  int32_t key[E];
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int i = lane * E + j;
    key[j] = i < s ? p[sort_at<PAD>(i)] : 0x7fffffff;
  }
  warp_bitonic<E>(key, lane);
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int i = lane * E + j;
    if (i < s) p[sort_at<PAD>(i)] = key[j];
  }
}

// The same for a nearly sorted p (E >= 2): odd-even transposition passes
// (pairs (2i, 2i+1), then (2i+1, 2i+2); the pair across two lanes by
// shuffles) until no pair is out of order.  Each pass pair moves an element
// at least one step towards its place, so a sequence whose elements sit
// within a few places of their own is sorted in a few passes; after
// kFixPasses pass pairs the bitonic network finishes whatever is left.
constexpr int kFixPasses = 12;
template <int E, bool PAD = false>
__device__ __forceinline__ void warp_fix_bucket(int32_t* __restrict__ p, int s, int lane) {
  static_assert(E >= 2 && (E & 1) == 0, "pairs (2i, 2i+1) must lie in one lane");
  int32_t key[E];
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int i = lane * E + j;
    key[j] = i < s ? p[sort_at<PAD>(i)] : 0x7fffffff;
  }
  bool done = false;
  for (int it = 0; it < kFixPasses && !done; ++it) {
#pragma unroll
    for (int j = 0; j + 1 < E; j += 2) {
      const int32_t x = key[j], y = key[j + 1];
      key[j] = min(x, y);
      key[j + 1] = max(x, y);
    }
#pragma unroll
    for (int j = 1; j + 1 < E; j += 2) {
      const int32_t x = key[j], y = key[j + 1];
      key[j] = min(x, y);
      key[j + 1] = max(x, y);
    }
    const int32_t nxt = __shfl_down_sync(0xffffffffu, key[0], 1);
    const int32_t prv = __shfl_up_sync(0xffffffffu, key[E - 1], 1);
    if (lane < 31) key[E - 1] = min(key[E - 1], nxt);
    if (lane > 0) key[0] = max(key[0], prv);
    const int32_t nxt2 = __shfl_down_sync(0xffffffffu, key[0], 1);
    bool ok = lane == 31 || key[E - 1] <= nxt2;
#pragma unroll
    for (int j = 0; j + 1 < E; ++j) ok &= key[j] <= key[j + 1];
    done = __all_sync(0xffffffffu, ok);
  }
  if (!done) warp_bitonic<E>(key, lane);
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int i = lane * E + j;
    if (i < s) p[sort_at<PAD>(i)] = key[j];
  }
}

// Sort p[0..s) in place, s <= 512, by the warp; dispatches on the smallest
// power-of-two E with 32 E >= s.
__device__ __forceinline__ void warp_sort_any(int32_t* __restrict__ p, int s, int lane) {
  if (s <= 1) return;
  if (s <= 32)
    warp_sort_bucket<1>(p, s, lane);
  else if (s <= 64)
    warp_sort_bucket<2>(p, s, lane);
  else if (s <= 128)
    warp_sort_bucket<4>(p, s, lane);
  else if (s <= 256)
    warp_sort_bucket<8>(p, s, lane);
  else
    warp_sort_bucket<16>(p, s, lane);
}

}  // namespace picasso
