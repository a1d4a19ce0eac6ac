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
      const uint32_t r0 = rhfg0(p, aip);
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

// Training step, part 1: one CTA per kTrainSamples samples of the minibatch. The BF16
// weights (as FP32), the samples' inputs, activations and deltas live in shared memory:
// forward (h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 . h2 + b3), the squared error
// against t (mean over the n samples of the minibatch), back-propagation to the
// pre-activations (dz2 = dy W3 relu'(z2), dz1 = (W2^T dz2) relu'(z1)), and this CTA's share
// of every weight gradient, summed over its samples in a fixed order into partial[cta][k].
// loss_partial[cta] = sum over its samples of (y - t)^2 / n.
constexpr uint32_t kTrainSamples = 4;
constexpr int kTrainThreads = 256;

// Shared memory of k_mlp_grad_partial: the weights, the samples' activations and deltas,
// and W1 and W2 again with rows padded by one word (a warp reading one column of a padded
// matrix hits 32 different banks).
__host__ __device__ inline uint32_t train_smem_floats(const MlpShape& s) {
  const uint32_t wpad = (s.total + 3) & ~3u;
  return wpad + kTrainSamples * (s.n_in + 4 * s.hidden) + 2 * kTrainSamples + s.hidden * (s.n_in + 1) +
         s.hidden * (s.hidden + 1);
}

// HC, DC: the hidden width and input count when known at compile time (loops unroll), else 0.
template <int HC, int DC>
__global__ void __launch_bounds__(kTrainThreads) k_mlp_grad_partial(MlpShape s, const __nv_bfloat16* __restrict__ wb,
                                                                     const float* __restrict__ x,
                                                                     const float* __restrict__ t,
                                                                     const uint32_t* __restrict__ rows, uint32_t n,
                                                                     float* __restrict__ partial,
                                                                     float* __restrict__ loss_partial) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) float train_sm[];
  const uint32_t H = HC ? (uint32_t)HC : s.hidden, D = DC ? (uint32_t)DC : s.n_in;
  constexpr uint32_t S = kTrainSamples;
  float* w = train_sm;
  float* xs = w + ((s.total + 3) & ~3u);  // [S][D]
  float* h1 = xs + S * D;                  // [S][H]
  float* h2 = h1 + S * H;
  float* d2 = h2 + S * H;                  // dz2
  float* d1 = d2 + S * H;                  // dz1
  float* dy = d1 + S * H;                  // [S]
  float* se = dy + S;                      // squared errors [S]
  float* w1p = se + S;                     // W1 rows padded to D + 1
  float* w2p = w1p + H * (D + 1);          // W2 rows padded to H + 1
  const float* W1 = w + s.off_w1;
  const float* B1 = w + s.off_b1;
  const float* W2 = w + s.off_w2;
  const float* B2 = w + s.off_b2;
  const float* W3 = w + s.off_w3;
  const uint32_t b0 = blockIdx.x * S;
  const uint32_t ns = min(S, n - b0);
  const float inv_n = 1.f / (float)n;
  {  // weights: 8 BF16 per 16-byte load (the BF16 array is padded to a multiple of 8)
    const uint32_t nvec = (s.total + 7) / 8;
    const uint4* wv = reinterpret_cast<const uint4*>(wb);
#pragma unroll 4
    for (uint32_t c = threadIdx.x; c < nvec; c += blockDim.x) {
      const uint4 v = __ldg(wv + c);
      const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t idx = c * 8 + 2 * j;
        if (idx < s.total) w[idx] = __uint_as_float(u[j] << 16);
        if (idx + 1 < s.total) w[idx + 1] = __uint_as_float(u[j] & 0xFFFF0000u);
      }
    }
  }
  for (uint32_t i = threadIdx.x; i < S * D; i += blockDim.x) {
    const uint32_t q = i / D, d = i - q * D;
    xs[i] = q < ns ? x[(uint64_t)(rows ? rows[b0 + q] : b0 + q) * D + d] : 0.f;
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < H * D; i += blockDim.x) {
    const uint32_t o = i / D, d = i - o * D;
    w1p[o * (D + 1) + d] = W1[i];
  }
  for (uint32_t i = threadIdx.x; i < H * H; i += blockDim.x) {
    const uint32_t o = i / H, k = i - o * H;
    w2p[o * (H + 1) + k] = W2[i];
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < S * H; i += blockDim.x) {  // layer 1
    const uint32_t q = i / H, o = i - q * H;
    float acc = B1[o];
#pragma unroll
    for (uint32_t d = 0; d < D; ++d) acc = fmaf(w1p[o * (D + 1) + d], xs[q * D + d], acc);
    h1[i] = fmaxf(acc, 0.f);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < S * H; i += blockDim.x) {  // layer 2
    const uint32_t q = i / H, o = i - q * H;
    float acc = B2[o];
#pragma unroll 16
    for (uint32_t k = 0; k < H; ++k) acc = fmaf(w2p[o * (H + 1) + k], h1[q * H + k], acc);
    h2[i] = fmaxf(acc, 0.f);
  }
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (uint32_t q = warp; q < S; q += nwarps) {  // output, error and dy: one warp per sample
    float acc = 0.f;
    for (uint32_t o = lane; o < H; o += 32) acc = fmaf(W3[o], h2[q * H + o], acc);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
    if (lane == 0) {
      const float y = acc + w[s.off_b3];
      const float err = q < ns ? y - t[rows ? rows[b0 + q] : b0 + q] : 0.f;
      dy[q] = 2.f * err * inv_n;
      se[q] = err * err;
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < S * H; i += blockDim.x) {  // dz2
    const uint32_t q = i / H, o = i - q * H;
    d2[i] = h2[i] > 0.f ? dy[q] * W3[o] : 0.f;
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < S * H; i += blockDim.x) {  // dz1
    const uint32_t q = i / H, k = i - q * H;
    float acc = 0.f;
    if (h1[i] > 0.f) {
#pragma unroll 16
      for (uint32_t o = 0; o < H; ++o) acc = fmaf(w2p[o * (H + 1) + k], d2[q * H + o], acc);
    }
    d1[i] = acc;
  }
  __syncthreads();
  float* out = partial + (uint64_t)blockIdx.x * s.total;
  // this CTA's gradient share, region by region (2-D indices without a division per entry)
  for (uint32_t k = threadIdx.x; k < H * D; k += blockDim.x) {  // W1[o][d]: dz1[o] * x[d]
    const uint32_t o = k / D, d = k - o * D;
    float acc = 0.f;
#pragma unroll
    for (uint32_t q = 0; q < S; ++q) acc = fmaf(d1[q * H + o], xs[q * D + d], acc);
    out[s.off_w1 + k] = acc;
  }
  for (uint32_t k = threadIdx.x; k < H * H; k += blockDim.x) {  // W2[o][i]: dz2[o] * h1[i]
    const uint32_t o = k / H, i = k - o * H;
    float acc = 0.f;
#pragma unroll
    for (uint32_t q = 0; q < S; ++q) acc = fmaf(d2[q * H + o], h1[q * H + i], acc);
    out[s.off_w2 + k] = acc;
  }
  for (uint32_t o = threadIdx.x; o < H; o += blockDim.x) {  // b1, b2, W3
    float a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
    for (uint32_t q = 0; q < S; ++q) {
      a1 += d1[q * H + o];
      a2 += d2[q * H + o];
      a3 = fmaf(dy[q], h2[q * H + o], a3);
    }
    out[s.off_b1 + o] = a1;
    out[s.off_b2 + o] = a2;
    out[s.off_w3 + o] = a3;
  }
  if (threadIdx.x == 0) {
    float b3 = 0.f, l = 0.f;
    for (uint32_t q = 0; q < S; ++q) {
      b3 += dy[q];
      l += se[q];
    }
    out[s.off_b3] = b3;
    loss_partial[blockIdx.x] = l * inv_n;
  }
}

// Sum over the CTAs' shares of 32 parameters per block (kSumThreads = 256 threads, blockDim
// fixed): warp j adds the shares c = j, j + 8, j + 16, ... of parameter k0 + lane (four loads
// in flight, coalesced over the lanes), and the eight warps' sums are added in warp order in
// shared memory — a fixed order. Returns the sum in warp 0 (other warps: 0).
constexpr int kSumThreads = 256;
constexpr uint32_t kSumParams = 32;  // parameters per block
__device__ __forceinline__ float sum_parts_block(const float* __restrict__ partial, uint32_t n_parts, uint32_t total,
                                                 uint32_t k) {
  __shared__ float part_sum[kSumThreads / 32][32];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  float acc = 0.f;
  if (k < total) {
    uint32_t c = warp;
    for (; c + 24 < n_parts; c += 32) {  // four shares in flight
      const float x0 = partial[(uint64_t)c * total + k], x1 = partial[(uint64_t)(c + 8) * total + k];
      const float x2 = partial[(uint64_t)(c + 16) * total + k], x3 = partial[(uint64_t)(c + 24) * total + k];
      acc += x0;
      acc += x1;
      acc += x2;
      acc += x3;
    }
    for (; c < n_parts; c += 8) acc += partial[(uint64_t)c * total + k];
  }
  part_sum[warp][lane] = acc;
  __syncthreads();
  float sum = 0.f;
  if (warp == 0)
    for (uint32_t j = 0; j < kSumThreads / 32; ++j) sum += part_sum[j][lane];
  return sum;
}

// The loss of a step: the sum of the CTAs' loss shares, in share order (one thread).
__device__ __forceinline__ float sum_loss(const float* __restrict__ loss_partial, uint32_t n_parts) {
  float l = 0.f;
  for (uint32_t c = 0; c < n_parts; ++c) l += loss_partial[c];
  return l;
}

// Training step, part 2 (gradient only): g[k] = the summed shares (sum_parts_block, 32
// parameters per block); *loss = sum_loss (thread 0 of the last block).
__global__ void __launch_bounds__(kSumThreads) k_mlp_reduce_grads(uint32_t total, uint32_t n_parts,
                                                                  const float* __restrict__ partial,
                                                                  const float* __restrict__ loss_partial,
                                                                  float* __restrict__ g, float* __restrict__ loss) {
  pdl_wait();
  pdl_trigger();
  const uint32_t k = blockIdx.x * kSumParams + (threadIdx.x & 31u);
  const float gk = sum_parts_block(partial, n_parts, total, k);
  if (threadIdx.x < 32 && k < total) g[k] = gk;
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 32) *loss = sum_loss(loss_partial, n_parts);
}

// Adam (Kingma and Ba 2015) on the FP32 parameters; the BF16 copy is refreshed. The step
// number is *step_base + step_off (the base lives on the device so that a captured epoch
// replays correctly; k_mlp_step_add advances it), the learning rate *lr_dev when given,
// else lr. With partial != NULL the gradient is first summed from the CTAs' shares
// (sum_parts_block, as k_mlp_reduce_grads) and stored in g. 32 parameters per block
// (kSumThreads threads); warp 0 updates them.
__global__ void __launch_bounds__(kSumThreads) k_mlp_adam(uint32_t total, float* __restrict__ wf,
                                                          __nv_bfloat16* __restrict__ wb, float* __restrict__ g,
                                                          float* __restrict__ m, float* __restrict__ v,
                                                          const float* __restrict__ lr_dev, float lr_val,
                                                          const uint32_t* __restrict__ step_base, uint32_t step_off,
                                                          float beta1, float beta2, float eps,
                                                          const float* __restrict__ partial, uint32_t n_parts,
                                                          const float* __restrict__ loss_partial,
                                                          float* __restrict__ loss) {
  pdl_wait();
  pdl_trigger();
  const uint32_t k = blockIdx.x * kSumParams + (threadIdx.x & 31u);
  if (partial && loss && blockIdx.x == gridDim.x - 1 && threadIdx.x == 32) *loss = sum_loss(loss_partial, n_parts);
  float gk = 0.f;
  if (partial) gk = sum_parts_block(partial, n_parts, total, k);
  if (threadIdx.x >= 32 || k >= total) return;
  if (partial)
    g[k] = gk;
  else
    gk = g[k];
  const float lr = lr_dev ? *lr_dev : lr_val;
  const float step = (float)(*step_base + step_off);
  const float bc1 = 1.f - powf(beta1, step), bc2 = 1.f - powf(beta2, step);
  const float mk = beta1 * m[k] + (1.f - beta1) * gk;
  const float vk = beta2 * v[k] + (1.f - beta2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  const float w = wf[k] - lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
  wf[k] = w;
  wb[k] = __float2bfloat16_rn(w);
}

__global__ void k_mlp_step_add(uint32_t* step_base, uint32_t n) {
  pdl_wait();
  *step_base += n;
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
