// bits_device.cuh -- the nibble-table ("four Russians") commutation test of
// 32 strings against one partner, shared by the bit pass of the per-round
// build and the small-round engine.  Internal header of the CUDA library.
//
// The symplectic form of strings u, v (x | z parts) is
// sum_k x_u[k] z_v[k] + z_u[k] x_v[k] mod 2, a bilinear form over GF(2).  For
// a block of 32 strings the warp transposes their 32-bit words into bit
// columns (bit r of column k = bit k of string r) and, for each 4-bit chunk
// of a part, stores the 16 XOR combinations of the chunk's four columns in
// a per-warp table; a partner then gets the anticommutation bits of the 32
// strings (bit r = string r) with one table lookup per 4-bit chunk of its
// other part, XORed together.
#pragma once

#include <stdint.h>

namespace picasso {

constexpr int kTabWords = 32 * 16;  // one warp's tables: 32 chunks x 16 entries

// 32 x 32 bit transpose across the warp: on entry lane r holds row r (bit k =
// M[r][k]); on exit lane k holds column k (bit r = M[r][k]).  Five butterfly
// stages exchange ever smaller off-diagonal sub-blocks.
__device__ __forceinline__ uint32_t transpose32(uint32_t w, int lane) {
#pragma unroll
  for (int j = 16; j > 0; j >>= 1) {
    const uint32_t m = j == 16 ? 0x0000FFFFu : j == 8 ? 0x00FF00FFu : j == 4 ? 0x0F0F0F0Fu : j == 2 ? 0x33333333u
                                                                                                   : 0x55555555u;
    const uint32_t t = __shfl_xor_sync(0xffffffffu, w, j);
    w = (lane & j) ? ((w & ~m) | ((t >> j) & m)) : ((w & m) | ((t << j) & ~m));
  }
  return w;
}

__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}

template <int QW>
__device__ __forceinline__ uint32_t word_of(const uint4& w, int g) {
  // table word order: x_lo, [x_hi], z_lo, [z_hi]
  if (QW == 2) return g == 0 ? w.x : g == 1 ? w.y : g == 2 ? w.z : w.w;
  return g == 0 ? w.x : w.z;
}

// Build this warp's tables for one row block from the block's bit columns.
template <int QW>
__device__ __forceinline__ void build_tables(const uint32_t* __restrict__ colw, uint32_t* __restrict__ tab, int lane) {
  constexpr int NG = 2 * QW;
  __syncwarp();  // the warp's lookups in the old tables are done
  if (lane < 8 * NG) {
    const int g = lane >> 3, qn = lane & 7;
    const uint4 a = *reinterpret_cast<const uint4*>(colw + g * 32 + 4 * qn);
    const uint32_t t3 = a.x ^ a.y, t5 = a.z ^ a.x, t6 = a.z ^ a.y, t7 = a.z ^ t3;
    uint4* o = reinterpret_cast<uint4*>(tab + lane * 16);
    o[0] = make_uint4(0u, a.x, a.y, t3);
    o[1] = make_uint4(a.z, t5, t6, t7);
    o[2] = make_uint4(a.w, a.w ^ a.x, a.w ^ a.y, a.w ^ t3);
    o[3] = make_uint4(a.w ^ a.z, a.w ^ t5, a.w ^ t6, a.w ^ t7);
  }
  __syncwarp();
}

// Anticommutation bits of partner words `cw` against the 32 rows whose
// tables start at shared address tab_addr (bit r = row r).
template <int QW>
__device__ __forceinline__ uint32_t lookup(const uint4& cw, uint32_t tab_addr) {
  constexpr int NG = 2 * QW;
  uint32_t acc = 0u;
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    // a row's x part meets the partner's z part and vice versa
    const uint32_t idx = word_of<QW>(cw, (g + QW) % NG);
    const uint32_t wl = (idx << 2) & 0x3C3C3C3Cu, wh = (idx >> 2) & 0x3C3C3C3Cu;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      // table base | (nibble * 4) in the low byte, chunk offset added
      const uint32_t lo = lds32(__byte_perm(wl, tab_addr, 0x7650u + k) + (uint32_t)((g * 8 + 2 * k) * 64));
      const uint32_t hi = lds32(__byte_perm(wh, tab_addr, 0x7650u + k) + (uint32_t)((g * 8 + 2 * k + 1) * 64));
      acc ^= lo ^ hi;
    }
  }
  return acc;
}

}  // namespace picasso
