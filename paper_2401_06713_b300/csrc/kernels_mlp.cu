// kernels_mlp.cu -- the parameter predictor: a 5 -> 64 -> 64 -> 2 MLP (GELU)
// with BF16 weights and FP32 accumulation, trained with MSE and AdamW; and
// the instance features it reads.  Sec. V of the paper predicts (P', alpha)
// from instance features with a learned regressor trained on grid-search
// labels; this is that regressor's B300 form.
//
// Parameter vector (fp32 master copy and bf16 working copy, same layout):
//   W1 [64][5] | b1 [64] | W2 [64][64] | b2 [64] | W3 [2][64] | b3 [2]
// The network is 4.7K parameters and a forward over 2,000 samples is about
// 1.3 MFLOP, so it runs on the FMA pipes (one block of 64 threads -- one per
// hidden unit -- over a chunk of samples); there is no dense contraction
// large enough for the tensor cores.
#include <cuda_bf16.h>

#include "common.cuh"

namespace picasso {

namespace {
constexpr int kIn = 5, kH = 64, kOut = 2;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kOut * kH, kParams = kOffB3 + kOut;
constexpr int kChunk = 32;     // samples per block
constexpr int kPitch = kH + 1;  // W2 row pitch in shared memory: rows and columns both conflict-free

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

// d gelu / dz = Phi(z) + z phi(z)
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

struct MlpSmem {
  float w1[kH * kIn], b1[kH], w2[kH * kPitch], b2[kH], w3[kOut * kH], b3[kOut];
  float x[kIn], z1[kH], h1[kH], z2[kH], h2[kH], dz2[kH], y[kOut], dy[kOut];
};

__device__ void load_weights(MlpSmem& S, const __nv_bfloat16* __restrict__ w) {
  for (int i = threadIdx.x; i < kParams; i += blockDim.x) {
    const float v = __bfloat162float(w[i]);
    if (i < kOffB1) {
      S.w1[i - kOffW1] = v;
    } else if (i < kOffW2) {
      S.b1[i - kOffB1] = v;
    } else if (i < kOffB2) {
      const int r = (i - kOffW2) / kH, cidx = (i - kOffW2) % kH;
      S.w2[r * kPitch + cidx] = v;
    } else if (i < kOffW3) {
      S.b2[i - kOffB2] = v;
    } else if (i < kOffB3) {
      S.w3[i - kOffW3] = v;
    } else {
      S.b3[i - kOffB3] = v;
    }
  }
}

// Forward of one sample by 64 threads (thread j = hidden unit j); ends with
// z1, h1, z2, h2, y of the sample in shared memory.
__device__ void forward_one(MlpSmem& S, const float* __restrict__ x) {
  const int j = threadIdx.x;
  if (j < kIn) S.x[j] = x[j];
  __syncthreads();
  float z = S.b1[j];
#pragma unroll
  for (int i = 0; i < kIn; ++i) z = fmaf(S.w1[j * kIn + i], S.x[i], z);
  S.z1[j] = z;
  S.h1[j] = gelu(z);
  __syncthreads();
  z = S.b2[j];
#pragma unroll 16
  for (int i = 0; i < kH; ++i) z = fmaf(S.w2[j * kPitch + i], S.h1[i], z);
  S.z2[j] = z;
  S.h2[j] = gelu(z);
  __syncthreads();
  {  // warp o computes output o
    const int o = j >> 5, l = j & 31;
    float acc = fmaf(S.w3[o * kH + l], S.h2[l], S.w3[o * kH + l + 32] * S.h2[l + 32]);
    for (int d = 16; d; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    if (l == 0) S.y[o] = acc + S.b3[o];
  }
  __syncthreads();
}
}  // namespace

__global__ void __launch_bounds__(kH) k_mlp_forward(const __nv_bfloat16* __restrict__ w, const float* __restrict__ x,
                                                    int B, float* __restrict__ y) {
  __shared__ MlpSmem S;
  load_weights(S, w);
  __syncthreads();
  const int b0 = blockIdx.x * kChunk;
  for (int b = b0; b < min(B, b0 + kChunk); ++b) {
    forward_one(S, x + (int64_t)b * kIn);
    if (threadIdx.x < kOut) y[(int64_t)b * kOut + threadIdx.x] = S.y[threadIdx.x];
  }
}

// Forward + backward of the loss (1/B) sum_b sum_o wo_o (y_bo - t_bo)^2 / 2.
// Every block accumulates the gradient of its samples in registers (thread j
// owns hidden unit j: row j of W1, column j of W2 and W3) and adds it to grad
// (fp32, zeroed by the launcher); loss (may be null) receives the loss.
__global__ void __launch_bounds__(kH) k_mlp_backward(const __nv_bfloat16* __restrict__ w, const float* __restrict__ x,
                                                     const float* __restrict__ t, float wo0, float wo1, int B,
                                                     float* __restrict__ grad, float* __restrict__ loss) {
  __shared__ MlpSmem S;
  load_weights(S, w);
  __syncthreads();
  const int j = threadIdx.x;
  float gw1[kIn], gw2[kH], gw3[kOut];
#pragma unroll
  for (int k = 0; k < kIn; ++k) gw1[k] = 0.f;
#pragma unroll
  for (int r = 0; r < kH; ++r) gw2[r] = 0.f;
#pragma unroll
  for (int o = 0; o < kOut; ++o) gw3[o] = 0.f;
  float gb1 = 0.f, gb2 = 0.f, gb3 = 0.f, lsum = 0.f;
  const float inv_b = 1.0f / (float)B;
  const int b0 = blockIdx.x * kChunk;
  for (int b = b0; b < min(B, b0 + kChunk); ++b) {
    forward_one(S, x + (int64_t)b * kIn);
    if (j < kOut) {
      const float wo = j == 0 ? wo0 : wo1;
      const float d = S.y[j] - t[(int64_t)b * kOut + j];
      S.dy[j] = wo * d * inv_b;
      lsum += 0.5f * wo * d * d * inv_b;
      gb3 += wo * d * inv_b;
    }
    __syncthreads();
    const float h2 = S.h2[j];
    float dh2 = 0.f;
#pragma unroll
    for (int o = 0; o < kOut; ++o) {
      gw3[o] = fmaf(S.dy[o], h2, gw3[o]);
      dh2 = fmaf(S.w3[o * kH + j], S.dy[o], dh2);
    }
    const float dz2 = dh2 * gelu_grad(S.z2[j]);
    S.dz2[j] = dz2;
    gb2 += dz2;
    __syncthreads();
    // column j of W2 (input unit j of layer 2): dW2[r][j] += dz2_r h1_j and
    // dh1_j = sum_r W2[r][j] dz2_r
    const float h1 = S.h1[j];
    float dh1 = 0.f;
#pragma unroll
    for (int r = 0; r < kH; ++r) {
      const float dr = S.dz2[r];
      gw2[r] = fmaf(dr, h1, gw2[r]);
      dh1 = fmaf(S.w2[r * kPitch + j], dr, dh1);
    }
    const float dz1 = dh1 * gelu_grad(S.z1[j]);
    gb1 += dz1;
#pragma unroll
    for (int k = 0; k < kIn; ++k) gw1[k] = fmaf(dz1, S.x[k], gw1[k]);
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < kIn; ++k) atomicAdd(&grad[kOffW1 + j * kIn + k], gw1[k]);
  atomicAdd(&grad[kOffB1 + j], gb1);
#pragma unroll
  for (int r = 0; r < kH; ++r) atomicAdd(&grad[kOffW2 + r * kH + j], gw2[r]);
  atomicAdd(&grad[kOffB2 + j], gb2);
#pragma unroll
  for (int o = 0; o < kOut; ++o) atomicAdd(&grad[kOffW3 + o * kH + j], gw3[o]);
  if (j < kOut) atomicAdd(&grad[kOffB3 + j], gb3);
  if (loss && j < kOut) atomicAdd(loss, lsum);
}

// AdamW (Loshchilov & Hutter, decoupled weight decay): first and second
// moments, bias correction for step `step` (1-based), update of the fp32
// master weights and refresh of their bf16 copy.
__global__ void k_mlp_adamw(float* __restrict__ master, __nv_bfloat16* __restrict__ w, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, int n, float lr, float b1, float b2,
                            float eps, float wd, int step) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  float p = master[i];
  p -= lr * ((mi / bc1) / (sqrtf(vi / bc2) + eps) + wd * p);
  master[i] = p;
  w[i] = __float2bfloat16_rn(p);
}

__global__ void k_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

// Instance features, counting part: counts[0] = non-identity positions over
// all strings; counts[1] = commuting pairs among `samples` pairs of distinct
// strings drawn by Philox (tag 3, counter = pair index, round 0): first
// string floor(r.x n / 2^32), second floor(r.y (n-1) / 2^32), moved up by one
// when not below the first.  Strings of W words per part.
__global__ void k_feature_counts(const uint64_t* __restrict__ xz, int64_t n, int32_t W, uint64_t seed,
                                 int64_t samples, unsigned long long* __restrict__ counts) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t S = 2 * W;
  unsigned long long wsum = 0, csum = 0;
  for (int64_t v = tid; v < n; v += stride)
    for (int k = 0; k < W; ++k) wsum += __popcll(xz[S * v + k] | xz[S * v + W + k]);
  for (int64_t p = tid; p < samples; p += stride) {
    const u32x4 r = philox_block(seed, 0, p, 3u, 0u);
    const int64_t u = (int64_t)(((uint64_t)r.x * (uint64_t)n) >> 32);
    int64_t w = (int64_t)(((uint64_t)r.y * (uint64_t)(n - 1)) >> 32);
    if (w >= u) ++w;
    csum += commuteW(xz + S * u, xz + S * w, W) ? 1ull : 0ull;
  }
  for (int d = 16; d; d >>= 1) {
    wsum += __shfl_xor_sync(0xffffffffu, wsum, d);
    csum += __shfl_xor_sync(0xffffffffu, csum, d);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&counts[0], wsum);
    atomicAdd(&counts[1], csum);
  }
}

// The five regressor inputs, in double then rounded to float:
//   log2(ln n) - 3, q / 64, mean weight / q, commuting fraction,
//   log2(budget / n) / 4 - 3.
// A round's conflict entries per vertex grow like density * L^2 / (P / n) with
// L = alpha ln n, so size and budget enter on the log scales that count is
// linear in.
__global__ void k_feature_final(const unsigned long long* __restrict__ counts, int64_t n, int32_t q, int64_t samples,
                                double log2_budget, double beta, float* __restrict__ feat) {
  if (threadIdx.x != 0) return;
  const double dn = (double)n;
  feat[0] = (float)(n > 1 ? log2(log(dn)) - 3.0 : -3.0);
  feat[1] = (float)((double)q / 64.0);
  feat[2] = (float)((double)counts[0] / (dn * (double)q));
  feat[3] = samples > 0 ? (float)((double)counts[1] / (double)samples) : 1.0f;
  feat[4] = beta >= 0.0 ? (float)(4.0 * beta - 2.0) : (float)((log2_budget - log2(dn)) / 4.0 - 3.0);
}

int mlp_param_count() { return kParams; }

cudaError_t launch_mlp_forward(const void* w, const float* x, int B, float* y, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  k_mlp_forward<<<(B + kChunk - 1) / kChunk, kH, 0, s>>>((const __nv_bfloat16*)w, x, B, y);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mlp_backward(const void* w, const float* x, const float* t, float wo0, float wo1, int B,
                                float* grad, float* loss, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * kParams, s);
  if (e == cudaSuccess && loss) e = cudaMemsetAsync(loss, 0, sizeof(float), s);
  if (e != cudaSuccess || B <= 0) return e;
  k_mlp_backward<<<(B + kChunk - 1) / kChunk, kH, 0, s>>>((const __nv_bfloat16*)w, x, t, wo0, wo1, B, grad, loss);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adamw(float* master, void* w, const float* g, float* m, float* v, float lr, float b1,
                             float b2, float eps, float wd, int step, cudaStream_t s) {
  k_mlp_adamw<<<(kParams + 255) / 256, 256, 0, s>>>(master, (__nv_bfloat16*)w, g, m, v, kParams, lr, b1, b2, eps, wd,
                                                    step);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* a, void* b, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_to_bf16<<<(n + 255) / 256, 256, 0, s>>>(a, (__nv_bfloat16*)b, n);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_features(const uint64_t* xz, int64_t n, int32_t q, uint64_t seed, int64_t samples,
                            double log2_budget, unsigned long long* counts, float* feat, cudaStream_t s,
                            double beta) {
  cudaError_t e = cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  if (n < 2) samples = 0;
  if (n > 0) {
    k_feature_counts<<<148 * 4, 256, 0, s>>>(xz, n, (q + 63) / 64, seed, samples, counts);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_feature_final<<<1, 32, 0, s>>>(counts, n, q, samples, log2_budget, beta, feat);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace picasso
