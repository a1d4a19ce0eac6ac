// Roof microbenchmarks for the per-packet update (the memory units its roofline names).
//
// The update is integer scatter work: per pair it reads 8 bytes of the packet stream and
// sets r' + r 2^-tau cells at random addresses. Its two designs meet different units:
//   * stamping every cell directly in the L2-resident estimator: one random one-byte L2
//     store (a partial sector write) per cell;
//   * the tiled design: one random shared-memory atomic OR per pair and SLEA row, plus the
//     pair stream read by every row's CTA through the SM's load pipe (from HBM once, then
//     from L2).
// Each kernel below drives one of those units alone with the same access pattern, so the
// measured rates are the denominators of the update's fractions of its roofs.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sse_microbench.h"

namespace {

// The same streaming 128-bit load as the update kernels: no L1 allocation, L2 evict-first.
__device__ __forceinline__ uint4 mb_load_stream(const uint4* ptr, uint64_t policy) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(ptr), "l"(policy));
  return v;
}

// A 32-bit mixer (xorshift-multiply) for the pseudo-random addresses; each step is a few
// ALU instructions, far below the memory rates measured.
__device__ __forceinline__ uint32_t mb_mix(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7FEB352Du;
  x ^= x >> 15;
  x *= 0x846CA68Bu;
  x ^= x >> 16;
  return x;
}

constexpr int kStoreUnroll = 8;

// Random one-byte stores into an L2-resident buffer of `bytes` bytes: every thread stores
// per_thread bytes (a multiple of kStoreUnroll) at mixed offsets.
__global__ void __launch_bounds__(256) k_mb_l2_stores(uint8_t* __restrict__ buf, uint32_t bytes, uint32_t per_thread,
                                                      uint32_t seed) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  for (uint32_t i = 0; i < per_thread; i += kStoreUnroll) {
#pragma unroll
    for (int u = 0; u < kStoreUnroll; ++u) {
      const uint32_t h = mb_mix((t * per_thread + i + u) ^ seed);
      buf[__umulhi(h, bytes)] = (uint8_t)(h | 1u);
    }
  }
}

constexpr int kAtomThreads = 1024;
constexpr int kAtomUnroll = 8;

// Random shared-memory atomic ORs of one bit into a bitmap of `words` 32-bit words (the
// tiled update's row bitmap), one CTA of 1024 threads per SM. The bitmap's OR is written
// out so that nothing is dead code.
__global__ void __launch_bounds__(kAtomThreads, 1) k_mb_smem_atomics(uint32_t words, uint32_t per_thread, uint32_t seed,
                                                                     uint32_t* __restrict__ sink) {
  extern __shared__ uint32_t bm[];
  for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) bm[w] = 0;
  __syncthreads();
  const uint32_t cells = words * 32u;
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  for (uint32_t i = 0; i < per_thread; i += kAtomUnroll) {
#pragma unroll
    for (int u = 0; u < kAtomUnroll; ++u) {
      const uint32_t cell = __umulhi(mb_mix((t * per_thread + i + u) ^ seed), cells);
      atomicOr(&bm[cell >> 5], 1u << (cell & 31u));
    }
  }
  __syncthreads();
  uint32_t acc = 0;
  for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) acc |= bm[w];
  if (acc == 0xFFFFFFFFu && seed == 0u) sink[blockIdx.x] = acc;  // practically never taken
}

constexpr int kLoadUnroll = 4;

// 128-bit streaming loads over n_vec vectors, `reps` times, grid-stride.
__global__ void __launch_bounds__(1024) k_mb_stream_loads(const uint4* __restrict__ src, uint64_t n_vec, uint32_t reps,
                                                          uint32_t* __restrict__ sink) {
  uint64_t policy;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
  uint32_t acc = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint32_t r = 0; r < reps; ++r) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + (kLoadUnroll - 1) * stride < n_vec; i += kLoadUnroll * stride) {
      uint4 v[kLoadUnroll];
#pragma unroll
      for (int u = 0; u < kLoadUnroll; ++u) v[u] = mb_load_stream(src + i + u * stride, policy);
#pragma unroll
      for (int u = 0; u < kLoadUnroll; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
    }
    for (; i < n_vec; i += stride) {
      const uint4 v = mb_load_stream(src + i, policy);
      acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
  }
  if (acc == 0x9E3779B9u) sink[0] = acc;  // keeps the loads; practically never taken
}

// Pseudo-random 32-bit words over n_vec 16-byte vectors (the skeleton's pairs).
__global__ void __launch_bounds__(256) k_mb_fill(uint4* __restrict__ dst, uint32_t n_vec) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_vec; i += gridDim.x * blockDim.x)
    dst[i] = make_uint4(mb_mix(4 * i), mb_mix(4 * i + 1), mb_mix(4 * i + 2), mb_mix(4 * i + 3));
}

constexpr int kSkelThreads = 1024;
constexpr int kSkelUnroll = 8;
constexpr uint32_t kSkelRows = 5;

// The tiled update's skeleton: the same grid (groups of kSkelRows CTAs, one bitmap of
// `words` 32-bit words per CTA, one CTA per SM), the same aligned 128-bit pair loads and one
// shared atomic OR per pair and CTA at a pseudo-random cell; no hashing of the method, no
// sampling, no flush. Its rate is the floor of the update's design on this device.
__global__ void __launch_bounds__(kSkelThreads, 1) k_mb_tiled_skeleton(const uint4* __restrict__ vec, uint32_t nvec,
                                                                       uint32_t words, uint32_t groups,
                                                                       uint32_t* __restrict__ sink) {
  extern __shared__ uint32_t bm[];
  for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) bm[w] = 0;
  __syncthreads();
  const uint32_t row = blockIdx.x % kSkelRows, group = blockIdx.x / kSkelRows;
  const uint32_t cells = words * 32u;
  const uint32_t key = 0x9E3779B9u * (row + 1u);
  // this group's vectors, in whole 8-vector (128-byte) lines
  const uint32_t lines = nvec >> 3;
  const uint32_t begin = 8u * (uint32_t)((uint64_t)lines * group / groups);
  const uint32_t end = 8u * (uint32_t)((uint64_t)lines * (group + 1) / groups);
  uint64_t policy;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
  auto touch = [&](uint32_t a, uint32_t b) {
    const uint32_t cell = __umulhi((a * key) ^ (b + key), cells);
    atomicOr(&bm[cell >> 5], 1u << (cell & 31u));
  };
  const uint32_t stride = blockDim.x;
  uint32_t i = begin + threadIdx.x;
  for (; i + (kSkelUnroll - 1) * stride < end; i += kSkelUnroll * stride) {
    uint4 v[kSkelUnroll];
#pragma unroll
    for (int u = 0; u < kSkelUnroll; ++u) v[u] = mb_load_stream(vec + i + u * stride, policy);
#pragma unroll
    for (int u = 0; u < kSkelUnroll; ++u) {
      touch(v[u].x, v[u].y);
      touch(v[u].z, v[u].w);
    }
  }
  for (; i < end; i += stride) {
    const uint4 v = mb_load_stream(vec + i, policy);
    touch(v.x, v.y);
    touch(v.z, v.w);
  }
  __syncthreads();
  uint32_t acc = 0;
  for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) acc |= bm[w];
  if (acc == 0x12345678u) sink[blockIdx.x] = acc;  // keeps the atomics; practically never taken
}

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  bool ok = false;
  EventPair() { ok = cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess; }
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// Best (smallest) of `reps` timed launches of fn, after one untimed launch; ms or < 0.
template <typename Launch>
float best_ms(cudaStream_t stream, int reps, Launch fn) {
  EventPair ev;
  if (!ev.ok) return -1.0f;
  fn();
  float best = -1.0f;
  for (int i = 0; i < reps; ++i) {
    if (cudaEventRecord(ev.a, stream) != cudaSuccess) return -1.0f;
    fn();
    if (cudaEventRecord(ev.b, stream) != cudaSuccess || cudaEventSynchronize(ev.b) != cudaSuccess) return -1.0f;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, ev.a, ev.b) != cudaSuccess) return -1.0f;
    if (best < 0.0f || ms < best) best = ms;
  }
  return cudaGetLastError() == cudaSuccess ? best : -1.0f;
}

}  // namespace

extern "C" int sse_microbench(void* d_buf, uint64_t buf_bytes, void* cuda_stream, sse_microbench_result* out) {
  if (!d_buf || !out || buf_bytes < kSseMicrobenchMinBytes || (reinterpret_cast<uintptr_t>(d_buf) & 255u))
    return SSE_ERR_INVALID_PARAM;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0, smem_max = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return SSE_ERR_CUDA;
  }
  *out = sse_microbench_result{};
  out->sms = (uint32_t)sms;
  uint8_t* buf = static_cast<uint8_t*>(d_buf);
  // sink: the last 4 KiB of the buffer (outside every measured region)
  uint32_t* sink = reinterpret_cast<uint32_t*>(buf + buf_bytes - 4096);

  // 1. random one-byte L2 stores into 45 MiB (the core-link estimator's size)
  const uint32_t l2_bytes = kSseMicrobenchL2Bytes;
  const uint32_t store_threads = 256, store_blocks = (uint32_t)sms * 8, store_per_thread = 2048;
  const float ms_st = best_ms(stream, 3, [&] {
    k_mb_l2_stores<<<store_blocks, store_threads, 0, stream>>>(buf, l2_bytes, store_per_thread, 0x1234u);
  });
  if (ms_st <= 0.0f) return SSE_ERR_CUDA;
  out->l2_random_byte_stores_per_s = (double)store_blocks * store_threads * store_per_thread / (ms_st * 1e-3);

  // 2. random shared-memory atomic ORs into a 131,584-byte bitmap per SM (a core-link SLEA
  // row of 1,052,656 cells, rounded to whole 1024-cell pieces)
  const uint32_t words = 1052672u / 32u;
  if ((int)(words * 4u) > smem_max) return SSE_ERR_INVALID_PARAM;
  if (cudaFuncSetAttribute(k_mb_smem_atomics, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(words * 4u)) !=
      cudaSuccess) {
    cudaGetLastError();
    return SSE_ERR_CUDA;
  }
  const uint32_t atom_per_thread = 4096;
  const float ms_at = best_ms(stream, 3, [&] {
    k_mb_smem_atomics<<<(unsigned)sms, kAtomThreads, words * 4u, stream>>>(words, atom_per_thread, 0x9876u, sink);
  });
  if (ms_at <= 0.0f) return SSE_ERR_CUDA;
  out->smem_random_atomics_per_s = (double)sms * kAtomThreads * atom_per_thread / (ms_at * 1e-3);

  // 3. streaming 128-bit loads: 32 MiB read 16 times (L2-resident after the first pass), and
  // the whole buffer (at least 1 GiB, from HBM) once
  const uint64_t l2_vec = (32ull << 20) / 16;
  const uint32_t reps = 16;
  const float ms_l2 = best_ms(stream, 3, [&] {
    k_mb_stream_loads<<<(unsigned)sms * 2, 1024, 0, stream>>>(reinterpret_cast<const uint4*>(buf), l2_vec, reps, sink);
  });
  if (ms_l2 <= 0.0f) return SSE_ERR_CUDA;
  out->l2_stream_load_bytes_per_s = (double)l2_vec * 16 * reps / (ms_l2 * 1e-3);
  const uint64_t hbm_vec = (buf_bytes - 4096) / 16;
  const float ms_hbm = best_ms(stream, 3, [&] {
    k_mb_stream_loads<<<(unsigned)sms * 2, 1024, 0, stream>>>(reinterpret_cast<const uint4*>(buf), hbm_vec, 1, sink);
  });
  if (ms_hbm <= 0.0f) return SSE_ERR_CUDA;
  out->hbm_stream_load_bytes_per_s = (double)hbm_vec * 16 / (ms_hbm * 1e-3);

  // 4. the tiled update's skeleton over 2^25 pseudo-random pairs (the first 256 MiB of the
  // buffer, written first; more than L2 holds, so each launch streams them from HBM)
  const uint32_t skel_vec = (1u << 25) / 2;
  const uint32_t skel_groups = (uint32_t)sms / kSkelRows;
  if (cudaFuncSetAttribute(k_mb_tiled_skeleton, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(words * 4u)) !=
      cudaSuccess) {
    cudaGetLastError();
    return SSE_ERR_CUDA;
  }
  k_mb_fill<<<(unsigned)sms * 8, 256, 0, stream>>>(reinterpret_cast<uint4*>(buf), skel_vec);
  const float ms_sk = best_ms(stream, 3, [&] {
    k_mb_tiled_skeleton<<<skel_groups * kSkelRows, kSkelThreads, words * 4u, stream>>>(
        reinterpret_cast<const uint4*>(buf), skel_vec, words, skel_groups, sink);
  });
  if (ms_sk <= 0.0f) return SSE_ERR_CUDA;
  out->tiled_skeleton_pairs_per_s = (double)skel_vec * 2 / (ms_sk * 1e-3);
  return SSE_OK;
}
