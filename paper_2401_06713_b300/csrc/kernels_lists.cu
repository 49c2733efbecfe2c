// kernels_lists.cu -- string packing and Alg. 1 list assignment (sm_103a).
#include "common.cuh"

namespace picasso {

// Characters -> symplectic words.  One thread per string; the block's rows
// are staged through shared memory so global reads are coalesced.
__global__ void k_pack(const uint8_t* __restrict__ codes, int64_t n, int32_t q, uint64_t* __restrict__ xz) {
  __shared__ uint8_t tile[256 * 64];
  const int64_t row0 = (int64_t)blockIdx.x * blockDim.x;
  const int64_t rows = min((int64_t)blockDim.x, n - row0);
  const int64_t bytes = rows * q;
  const uint8_t* src = codes + row0 * q;
  for (int64_t i = threadIdx.x; i < bytes; i += blockDim.x) tile[i] = src[i];
  __syncthreads();
  if (threadIdx.x >= rows) return;
  uint64_t x = 0, z = 0;
  const uint8_t* s = tile + (int64_t)threadIdx.x * q;
  for (int i = 0; i < q; ++i) {
    const uint32_t c = s[i];
    x |= (uint64_t)(c == 1u || c == 2u) << i;
    z |= (uint64_t)(c == 3u || c == 2u) << i;
  }
  xz[2 * (row0 + threadIdx.x)] = x;
  xz[2 * (row0 + threadIdx.x) + 1] = z;
}

// The same for q a multiple of 16 (rows 16-byte aligned): 16-byte loads,
// four characters a step.  For a code byte c in {0, 1, 2, 3} (I, X, Y, Z) the
// x bit is bit 0 of c ^ (c >> 1) and the z bit is bit 1 of c; any other byte
// gives neither, as above.  The four bytes' bits (at bits 0, 8, 16, 24) go
// to one nibble by a multiply with 1 + 2^7 + 2^14 + 2^21: byte k's bit lands
// at 21 + k (from the term 2^(7 (3 - k))), and every other term lands below
// 21 at a distinct bit (no carry) or above 24.
__global__ void k_pack16(const uint8_t* __restrict__ codes, int64_t n, int32_t q, uint64_t* __restrict__ xz) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const uint4* row = reinterpret_cast<const uint4*>(codes + v * q);
  uint64_t x = 0, z = 0;
  for (int k = 0; k < (q >> 4); ++k) {
    const uint4 w4 = row[k];
    const uint32_t ws[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const uint32_t w = ws[t];
      uint32_t hi = (w >> 2) & 0x3F3F3F3Fu;  // bits 2..7 of each byte
      hi |= hi >> 3;
      hi |= hi >> 1;
      hi |= hi >> 1;
      const uint32_t ok = ~hi & 0x01010101u;  // the byte is a valid code
      const uint32_t xb = (w ^ (w >> 1)) & ok, zb = (w >> 1) & ok;
      const int sh = 16 * k + 4 * t;
      x |= (uint64_t)(((xb * 0x204081u) >> 21) & 0xFu) << sh;
      z |= (uint64_t)(((zb * 0x204081u) >> 21) & 0xFu) << sh;
    }
  }
  xz[2 * v] = x;
  xz[2 * v + 1] = z;
}

// Strings of more than 64 qubits: W = ceil(q / 64) words per part, the
// string's words x_0 .. x_{W-1}, z_0 .. z_{W-1}; word w holds qubits
// 64 w .. 64 w + 63.  One thread per (string, word).
__global__ void k_pack_wide(const uint8_t* __restrict__ codes, int64_t n, int32_t q, uint64_t* __restrict__ xz) {
  const int W = (q + 63) >> 6;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * W) return;
  const int64_t v = t / W;
  const int w = (int)(t - v * W);
  const uint8_t* s = codes + v * q + 64 * w;
  const int m = min(64, q - 64 * w);
  uint64_t x = 0, z = 0;
  for (int i = 0; i < m; ++i) {
    const uint32_t c = s[i];
    x |= (uint64_t)(c == 1u || c == 2u) << i;
    z |= (uint64_t)(c == 3u || c == 2u) << i;
  }
  xz[2 * W * v + w] = x;
  xz[2 * W * v + W + w] = z;
}

cudaError_t launch_pack(const uint8_t* codes, int64_t n, int32_t q, uint64_t* xz, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (q > 64) {
    const int64_t t = n * ((q + 63) / 64);
    k_pack_wide<<<(unsigned)((t + 255) / 256), 256, 0, s>>>(codes, n, q, xz);
    count_launches(1);
    return cudaGetLastError();
  }
  const int64_t blocks = (n + 255) / 256;
  if ((q & 15) == 0 && (reinterpret_cast<uintptr_t>(codes) & 15) == 0)
    k_pack16<<<(unsigned)blocks, 256, 0, s>>>(codes, n, q, xz);
  else
    k_pack<<<(unsigned)blocks, 256, 0, s>>>(codes, n, q, xz);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void k_philox_draws(uint64_t seed, int32_t round, int64_t gid, uint32_t tag, uint32_t i0,
                               int32_t count, uint32_t* out) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const uint32_t d = i0 + (uint32_t)i;
  out[i] = pick(philox_block(seed, round, gid, tag, d / 4u), d % 4u);
}

cudaError_t launch_philox_draws(uint64_t seed, int32_t round, int64_t gid, uint32_t tag, uint32_t i0,
                                int32_t count, uint32_t* out, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_philox_draws<<<(count + 255) / 256, 256, 0, s>>>(seed, round, gid, tag, i0, count, out);
  count_launches(1);
  return cudaGetLastError();
}

// List length of every round vertex (the L of its set), then offsets.
__global__ void k_list_len(const int32_t* __restrict__ gid, int64_t n, const int64_t* __restrict__ soff, int nsets,
                           const SetRound* __restrict__ sets, uint32_t* __restrict__ len) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int64_t g = gid ? (int64_t)gid[v] : v;
  len[v] = (uint32_t)sets[nsets > 1 ? set_of(soff, nsets, g) : 0].L;
}

cudaError_t launch_list_offsets(const int32_t* gid, int64_t n, const int64_t* soff, int32_t nsets,
                                const SetRound* sets, uint32_t* len, int64_t* loff, void* tmp, cudaStream_t s) {
  if (n > 0) {
    k_list_len<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(gid, n, soff, nsets, sets, len);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return launch_scan_u32(len, n, loff, tmp, s);
}

__global__ void k_strided_offsets(int64_t* __restrict__ loff, int64_t n, int32_t L) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v <= n) loff[v] = v * (int64_t)L;
}

cudaError_t launch_strided_offsets(int64_t* loff, int64_t n, int32_t L, cudaStream_t s) {
  k_strided_offsets<<<(unsigned)((n + 1 + 255) / 256), 256, 0, s>>>(loff, n, L);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void k_entry_owner(const int64_t* __restrict__ loff, int64_t n, int32_t* __restrict__ ent_v) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  for (int64_t e = loff[v]; e < loff[v + 1]; ++e) ent_v[e] = (int32_t)v;
}

cudaError_t launch_entry_owner(const int64_t* loff, int64_t n, int32_t* ent_v, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_entry_owner<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(loff, n, ent_v);
  count_launches(1);
  return cudaGetLastError();
}

// Priority of each of the round's vertices: draw 0 of its set's PRIO stream
// at the vertex's id within the set (the static Random order of Sec. III-B).
__global__ void k_round_prio(int32_t round, const int32_t* __restrict__ gid, int64_t n,
                             const int64_t* __restrict__ soff, int nsets, const SetRound* __restrict__ sets,
                             uint32_t* __restrict__ prio) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int64_t gg = gid ? (int64_t)gid[v] : v;
  const int k = nsets > 1 ? set_of(soff, nsets, gg) : 0;
  prio[v] = philox_block(sets[k].seed, round, gg - soff[k], kTagPrio, 0u).x;
}

cudaError_t launch_round_prio(int32_t round, const int32_t* gid, int64_t n, const int64_t* soff, int32_t nsets,
                              const SetRound* sets, uint32_t* prio, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_round_prio<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(round, gid, n, soff, nsets, sets, prio);
  count_launches(1);
  return cudaGetLastError();
}

// Alg. 1 assign_rand_list_colors: one thread per vertex, with the P, L and
// seed of the vertex's set; Philox is keyed by the set's seed and the
// vertex's id within its set (draw_list: Floyd's sampling, sorted); lists
// hold bucket colors (round-local color + the set's offset cofs).  The
// priority is draw 0 of the PRIO stream.
template <int LCAP>
__global__ void k_assign_lists(int32_t round, const int32_t* __restrict__ gid, int64_t n,
                               const int64_t* __restrict__ soff, int nsets, const SetRound* __restrict__ sets,
                               const int64_t* __restrict__ loff, int32_t* __restrict__ lists,
                               uint32_t* __restrict__ prio, uint32_t* __restrict__ bcount) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int64_t gg = gid ? (int64_t)gid[v] : v;
  const int k = nsets > 1 ? set_of(soff, nsets, gg) : 0;
  const SetRound sr = sets[k];
  const int64_t g = gg - soff[k];  // id within the set
  if (LCAP == 32)
    draw_list32(sr.seed, round, g, sr.P, sr.L, sr.cofs, lists + loff[v], bcount);
  else
    draw_list<LCAP>(sr.seed, round, g, sr.P, sr.L, sr.cofs, lists + loff[v]);
  prio[v] = philox_block(sr.seed, round, g, kTagPrio, 0u).x;
}

cudaError_t launch_assign_lists(int32_t round, const int32_t* gid, int64_t n, const int64_t* soff, int32_t nsets,
                                const SetRound* sets, int32_t Lmax, const int64_t* loff, int32_t* lists,
                                uint32_t* prio, uint32_t* bcount, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + 127) / 128);
  if (Lmax <= 32) {
    k_assign_lists<32><<<blocks, 128, 0, s>>>(round, gid, n, soff, nsets, sets, loff, lists, prio, bcount);
  } else if (Lmax <= 128) {
    k_assign_lists<128><<<blocks, 128, 0, s>>>(round, gid, n, soff, nsets, sets, loff, lists, prio, nullptr);
  } else {
    k_assign_lists<kMaxL><<<blocks, 128, 0, s>>>(round, gid, n, soff, nsets, sets, loff, lists, prio, nullptr);
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace picasso
