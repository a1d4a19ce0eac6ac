// Learned cardinality correction: per-host features and a small MLP trained on the GPU.
//
// Features of a host (k + 2 values, each log(1 + v)): the union SLE's active cells per
// distance a = 0..k-1 (the per-age histogram of Algorithm 8's union SLE), the sum and the
// minimum over the r rows of the host's SRE weights |SRE_i|^k (Section 3.2).
// MLP: n_in -> H -> H -> 1 with ReLU, weights stored in BF16 for the arithmetic and FP32
// for the optimiser, every sum accumulated in FP32. The output is a correction in log space:
// the learned estimate is max(LC, 1) * exp(output), LC being Algorithm 8's estimate.
// Parameter vector layout: W1[H][n_in], b1[H], W2[H][H], b2[H], W3[H], b3.
#pragma once

#include <cuda_bf16.h>

#include "sse_internal.cuh"

namespace sse {

constexpr int kFeatThreads = 128;
constexpr int kMaxHidden = 64;
constexpr int kMaxIn = 64;

// One CTA per host (grid-stride). x: [n][k + 2].
__global__ void __launch_bounds__(kFeatThreads) k_features(const __grid_constant__ KParams p,
                                                           const uint8_t* __restrict__ sre,
                                                           const uint8_t* __restrict__ sle,
                                                           const uint32_t* __restrict__ hosts, uint32_t n,
                                                           const uint32_t* __restrict__ clock,
                                                           float* __restrict__ x) {
  __shared__ uint8_t age_lut[256];
  __shared__ uint32_t hist[256];
  __shared__ uint32_t sre_w[kMaxRows];
  __shared__ const uint8_t* row_base[kMaxRows];
  const uint32_t cs = *clock;
  for (uint32_t s = threadIdx.x; s < 256; s += blockDim.x) {
    const uint32_t a = stamp_age(s, cs);
    age_lut[s] = a < p.k ? (uint8_t)a : 255;
  }
  const uint32_t dim = p.k + 2;
  for (uint32_t h = blockIdx.x; h < n; h += gridDim.x) {
    const uint32_t aip = hosts[h];
    if (threadIdx.x < p.r2) {
      const uint32_t j = mas_top(p.key_a[kLH + threadIdx.x], p.key_b[kLH + threadIdx.x], aip, p.q2);
      row_base[threadIdx.x] = sle + threadIdx.x * p.row_pitch2 + (uint64_t)j * p.delta2;
    }
    for (uint32_t a = threadIdx.x; a < p.k; a += blockDim.x) hist[a] = 0;
    __syncthreads();
    // SRE weights of the host's r estimators (RHFG[i], Eq. 6), one thread per row
    if (threadIdx.x < p.r) {
      const uint32_t i = threadIdx.x;
      const uint32_t r0 = mas_top(p.key_a[kR0], p.key_b[kR0], aip, p.q);
      const uint32_t col =
          i == 0 ? r0 : (uint32_t)((((uint64_t)aip >> (i * p.delta)) ^ r0) & ((1u << p.q) - 1u));
      const uint8_t* cells = sre + (((uint64_t)i << p.q) + col) * 8;
      uint32_t w = 0;
      for (int c = 0; c < 8; ++c) w += age_lut[cells[c]] != 255 ? 1u : 0u;
      sre_w[i] = w;
    }
    // union SLE histogram by largest distance over the rows
    for (uint32_t z = threadIdx.x; z < p.eta2; z += blockDim.x) {
      uint32_t m = 0;
      for (uint32_t i = 0; i < p.r2; ++i) m = max(m, (uint32_t)age_lut[row_base[i][z]]);
      if (m != 255) atomicAdd(&hist[m], 1u);
    }
    __syncthreads();
    float* out = x + (uint64_t)h * dim;
    for (uint32_t a = threadIdx.x; a < p.k; a += blockDim.x) out[a] = log1pf((float)hist[a]);
    if (threadIdx.x == 0) {
      uint32_t sum = 0, mn = 0xFFFFFFFFu;
      for (uint32_t i = 0; i < p.r; ++i) {
        sum += sre_w[i];
        mn = min(mn, sre_w[i]);
      }
      out[p.k] = log1pf((float)sum);
      out[p.k + 1] = log1pf((float)mn);
    }
    __syncthreads();
  }
}

struct MlpShape {
  uint32_t n_in, hidden;
  uint32_t off_w1, off_b1, off_w2, off_b2, off_w3, off_b3, total;
};

__host__ __device__ inline MlpShape mlp_shape(uint32_t n_in, uint32_t hidden) {
  MlpShape s;
  s.n_in = n_in;
  s.hidden = hidden;
  s.off_w1 = 0;
  s.off_b1 = s.off_w1 + hidden * n_in;
  s.off_w2 = s.off_b1 + hidden;
  s.off_b2 = s.off_w2 + hidden * hidden;
  s.off_w3 = s.off_b2 + hidden;
  s.off_b3 = s.off_w3 + hidden;
  s.total = s.off_b3 + 1;
  return s;
}

// Inference: one thread per sample; BF16 weights staged as float in shared memory.
// rows: optional sample indices into x (gather), else sample b is row b.
__global__ void __launch_bounds__(128) k_mlp_forward(MlpShape s, const __nv_bfloat16* __restrict__ wb,
                                                     const float* __restrict__ x, const uint32_t* __restrict__ rows,
                                                     uint32_t n, float* __restrict__ y) {
  extern __shared__ float w[];
  for (uint32_t i = threadIdx.x; i < s.total; i += blockDim.x) w[i] = __bfloat162float(wb[i]);
  __syncthreads();
  const uint32_t H = s.hidden, D = s.n_in;
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
    const float* xb = x + (uint64_t)(rows ? rows[b] : b) * D;
    float xi[kMaxIn];
    for (uint32_t i = 0; i < D; ++i) xi[i] = xb[i];
    float h1[kMaxHidden];
    for (uint32_t o = 0; o < H; ++o) {
      float acc = w[s.off_b1 + o];
      for (uint32_t i = 0; i < D; ++i) acc = fmaf(w[s.off_w1 + o * D + i], xi[i], acc);
      h1[o] = fmaxf(acc, 0.f);
    }
    float out = w[s.off_b3];
    for (uint32_t o = 0; o < H; ++o) {
      float acc = w[s.off_b2 + o];
      for (uint32_t i = 0; i < H; ++i) acc = fmaf(w[s.off_w2 + o * H + i], h1[i], acc);
      out = fmaf(w[s.off_w3 + o], fmaxf(acc, 0.f), out);
    }
    y[b] = out;
  }
}

// Training, per sample: forward, squared-error loss on the target t (mean over the n
// samples) and back-propagation to the pre-activations. Stores per sample: h1 = relu(z1)
// [H], h2 = relu(z2) [H], dz1 [H], dz2 [H], dy; loss partial sums go to loss_acc.
__global__ void __launch_bounds__(128) k_mlp_backward(MlpShape s, const __nv_bfloat16* __restrict__ wb,
                                                      const float* __restrict__ x, const float* __restrict__ t,
                                                      const uint32_t* __restrict__ rows, uint32_t n,
                                                      float* __restrict__ act, float* __restrict__ loss_acc) {
  extern __shared__ float w[];
  for (uint32_t i = threadIdx.x; i < s.total; i += blockDim.x) w[i] = __bfloat162float(wb[i]);
  __syncthreads();
  const uint32_t H = s.hidden, D = s.n_in;
  const float inv_n = 1.f / (float)n;
  float local_loss = 0.f;
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
    const uint32_t row = rows ? rows[b] : b;
    const float* xb = x + (uint64_t)row * D;
    float* a = act + (uint64_t)b * (4 * H + 1);  // h1 | h2 | dz1 | dz2 | dy
    float xi[kMaxIn];
    for (uint32_t i = 0; i < D; ++i) xi[i] = xb[i];
    float h1[kMaxHidden];
    for (uint32_t o = 0; o < H; ++o) {
      float acc = w[s.off_b1 + o];
      for (uint32_t i = 0; i < D; ++i) acc = fmaf(w[s.off_w1 + o * D + i], xi[i], acc);
      h1[o] = fmaxf(acc, 0.f);
      a[o] = h1[o];
    }
    float yv = w[s.off_b3];
    for (uint32_t o = 0; o < H; ++o) {
      float acc = w[s.off_b2 + o];
      for (uint32_t i = 0; i < H; ++i) acc = fmaf(w[s.off_w2 + o * H + i], h1[i], acc);
      const float h2 = fmaxf(acc, 0.f);
      a[H + o] = h2;
      yv = fmaf(w[s.off_w3 + o], h2, yv);
    }
    const float err = yv - t[row];
    local_loss = fmaf(err, err, local_loss);
    const float dy = 2.f * err * inv_n;  // d(mean squared error)/dy
    a[4 * H] = dy;
    // dz2 = dy * W3 * relu'(z2); dz1 = (W2^T dz2) * relu'(z1)
    for (uint32_t o = 0; o < H; ++o) a[3 * H + o] = a[H + o] > 0.f ? dy * w[s.off_w3 + o] : 0.f;
    for (uint32_t i = 0; i < H; ++i) {
      float acc = 0.f;
      if (h1[i] > 0.f)
        for (uint32_t o = 0; o < H; ++o) acc = fmaf(w[s.off_w2 + o * H + i], a[3 * H + o], acc);
      a[2 * H + i] = acc;
    }
  }
  for (int off = 16; off > 0; off >>= 1) local_loss += __shfl_xor_sync(0xFFFFFFFFu, local_loss, off);
  if ((threadIdx.x & 31) == 0 && local_loss != 0.f) atomicAdd(loss_acc, local_loss * inv_n);
}

// Weight gradients, one thread per parameter: sums over the batch in FP32.
__global__ void __launch_bounds__(256) k_mlp_weight_grads(MlpShape s, const float* __restrict__ x,
                                                          const uint32_t* __restrict__ rows, uint32_t n,
                                                          const float* __restrict__ act, float* __restrict__ g) {
  const uint32_t H = s.hidden, D = s.n_in, stride = 4 * H + 1;
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= s.total) return;
  float acc = 0.f;
  if (k < s.off_b1) {  // W1[o][i]: dz1[o] * x[i]
    const uint32_t o = k / D, i = k % D;
    for (uint32_t b = 0; b < n; ++b)
      acc = fmaf(act[(uint64_t)b * stride + 2 * H + o], x[(uint64_t)(rows ? rows[b] : b) * D + i], acc);
  } else if (k < s.off_w2) {  // b1[o]
    const uint32_t o = k - s.off_b1;
    for (uint32_t b = 0; b < n; ++b) acc += act[(uint64_t)b * stride + 2 * H + o];
  } else if (k < s.off_b2) {  // W2[o][i]: dz2[o] * h1[i]
    const uint32_t o = (k - s.off_w2) / H, i = (k - s.off_w2) % H;
    for (uint32_t b = 0; b < n; ++b)
      acc = fmaf(act[(uint64_t)b * stride + 3 * H + o], act[(uint64_t)b * stride + i], acc);
  } else if (k < s.off_w3) {  // b2[o]
    const uint32_t o = k - s.off_b2;
    for (uint32_t b = 0; b < n; ++b) acc += act[(uint64_t)b * stride + 3 * H + o];
  } else if (k < s.off_b3) {  // W3[o]: dy * h2[o]
    const uint32_t o = k - s.off_w3;
    for (uint32_t b = 0; b < n; ++b) acc = fmaf(act[(uint64_t)b * stride + 4 * H], act[(uint64_t)b * stride + H + o], acc);
  } else {  // b3
    for (uint32_t b = 0; b < n; ++b) acc += act[(uint64_t)b * stride + 4 * H];
  }
  g[k] = acc;
}

// Adam (Kingma and Ba 2015) on the FP32 parameters; the BF16 copy is refreshed.
__global__ void k_mlp_adam(uint32_t total, float* __restrict__ wf, __nv_bfloat16* __restrict__ wb,
                           const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v, float lr,
                           float beta1, float beta2, float eps, float bc1, float bc2) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= total) return;
  const float gk = g[k];
  const float mk = beta1 * m[k] + (1.f - beta1) * gk;
  const float vk = beta2 * v[k] + (1.f - beta2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  const float w = wf[k] - lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
  wf[k] = w;
  wb[k] = __float2bfloat16_rn(w);
}

__global__ void k_mlp_to_bf16(uint32_t total, const float* __restrict__ wf, __nv_bfloat16* __restrict__ wb) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < total) wb[k] = __float2bfloat16_rn(wf[k]);
}

// Learned estimate = max(LC, 1) * exp(MLP(features)) for hosts whose union SLE has at least
// min_active active cells (the gate: below it linear counting is kept, being the
// maximum-likelihood estimate where the SLE is far from saturation). The active cells are
// the sum of the per-distance counts, recovered from the features' log(1 + count). When the
// result is not finite, or a feature lies outside the range seen in training
// (feature > x_max), LC is kept as well (fallback).
__global__ void k_learned_select(uint32_t n, uint32_t dim, const float* __restrict__ x, const float* __restrict__ y,
                                 const float* __restrict__ lc, const float* __restrict__ x_max, uint32_t min_active,
                                 float* __restrict__ est) {
  const uint32_t h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= n) return;
  bool inside = true;
  float active = 0.f;
  for (uint32_t i = 0; i < dim; ++i) {
    const float v = x[(uint64_t)h * dim + i];
    inside &= v <= x_max[i];
    if (i + 2 < dim) active += rintf(expm1f(v));
  }
  const float e = fmaxf(lc[h], 1.f) * expf(y[h]);
  est[h] = (inside && active >= (float)min_active && isfinite(e)) ? e : lc[h];
}

}  // namespace sse
