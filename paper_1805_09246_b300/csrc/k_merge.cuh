// Merge of estimators from distributed routers (Algorithm 2 for RSRA, Algorithm 7 for
// SLEA). All estimators share the current stamp; every cell keeps the most recent stamp
// (smallest distance) over dst and the sources, so the result is the estimator of the
// union of the routers' pair streams. 16 cells per thread, coalesced 128-bit accesses.
#pragma once

#include "sse_internal.cuh"

namespace sse {

struct MergeSources {
  const uint8_t* ptr[kMaxMergeSources];
};

// Cells are St (8 or 16 bits): 16 or 8 per 128-bit vector.
template <typename St>
__global__ void __launch_bounds__(256) k_merge(uint8_t* __restrict__ dst, const __grid_constant__ MergeSources src,
                                               int nsrc, uint64_t n16, uint32_t cs_value,
                                               const uint32_t* __restrict__ clock) {
  constexpr int kBits = 8 * sizeof(St);
  constexpr uint32_t kMask = sizeof(St) == 1 ? 0xFFu : 0xFFFFu;
  constexpr uint32_t kMod = sizeof(St) == 1 ? 255u : 65535u;
  __shared__ uint8_t age_lut[256];
  const uint32_t cs = clock ? *clock : cs_value;
  if (sizeof(St) == 1)
    for (uint32_t s = threadIdx.x; s < 256; s += blockDim.x) age_lut[s] = (uint8_t)stamp_age(s, cs);
  __syncthreads();
  // distance of stamp s, unset cells the farthest
  auto age = [&](uint32_t s) -> uint32_t {
    if (sizeof(St) == 1) return age_lut[s];
    return s == 0 ? kMod : (cs >= s ? cs - s : cs + kMod - s);
  };
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n16; x += (uint64_t)gridDim.x * blockDim.x) {
    uint4 d = reinterpret_cast<const uint4*>(dst)[x];
    uint32_t w[4] = {d.x, d.y, d.z, d.w};
    for (int j = 0; j < nsrc; ++j) {
      const uint4 v = reinterpret_cast<const uint4*>(src.ptr[j])[x];
      const uint32_t o[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        uint32_t out = 0;
#pragma unroll
        for (int b = 0; b < 32 / kBits; ++b) {
          const uint32_t s0 = (w[a] >> (kBits * b)) & kMask, s1 = (o[a] >> (kBits * b)) & kMask;
          out |= (age(s1) < age(s0) ? s1 : s0) << (kBits * b);
        }
        w[a] = out;
      }
    }
    reinterpret_cast<uint4*>(dst)[x] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

}  // namespace sse
