// Seeded synthetic traffic generated on the device, for learned-correction training runs
// (inputs only; no estimator arithmetic). synth_cpu_hosts / synth_cpu_noise below produce
// the same streams on the host, and tests check the two agree bit for bit.
//
// Host h (address ip[h]) contacts card[h] distinct opposite hosts, spread evenly over the
// slices first[h]..last[h]: in slice s it sends destinations j in
// [card*(s-first)/L, card*(s-first+1)/L), L = last - first + 1, and destination j is
// mix(seed, ip, j), a bijection of j for a fixed (seed, ip), so all are distinct.
// Background noise pair i of slice s of router r is (mix(seed', r, s, i, 1), mix(seed', r, s, i, 2)),
// its source with the top bit clear: hosts given addresses with the top bit set receive no
// noise pair, so their exact cardinality is known by construction.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__host__ __device__ inline uint32_t perm32(uint32_t x) {  // bijective 32-bit mix
  x ^= x >> 16; x *= 0x7FEB352Du;
  x ^= x >> 15; x *= 0x846CA68Bu;
  x ^= x >> 16;
  return x;
}

__host__ __device__ inline uint32_t dst_of(uint64_t seed, uint32_t ip, uint32_t j) {
  const uint32_t key = perm32(ip ^ (uint32_t)seed) ^ (uint32_t)(seed >> 32);
  return perm32(j ^ key) ^ perm32(key + 0x9E3779B9u);
}

__global__ void k_hosts(const uint32_t* ip, const uint32_t* card, const uint32_t* first, const uint32_t* last,
                        const uint64_t* offset, uint32_t n, uint32_t slice, uint64_t seed, uint32_t* out) {
  for (uint32_t h = blockIdx.x; h < n; h += gridDim.x) {
    if (slice < first[h] || slice > last[h]) continue;
    const uint64_t L = last[h] - first[h] + 1, c = card[h], s = slice - first[h];
    const uint32_t j0 = (uint32_t)(c * s / L), j1 = (uint32_t)(c * (s + 1) / L);
    uint32_t* o = out + 2 * offset[h];
    for (uint32_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
      o[2 * (j - j0)] = ip[h];
      o[2 * (j - j0) + 1] = dst_of(seed, ip[h], j);
    }
  }
}

// blockIdx.y = router: its noise pairs go to out + 2 * offset[router]; each router has its
// own stream of noise (the router index is mixed into the key).
__global__ void k_noise(const uint64_t* offset, uint64_t n, uint32_t slice, uint64_t seed, uint32_t* out) {
  const uint32_t router = blockIdx.y;
  const uint32_t k0 = perm32((uint32_t)seed ^ 0xA5A5A5A5u ^ perm32(router + 0x51ED270Bu)) ^ slice * 0x9E3779B9u;
  uint32_t* o = out + 2 * offset[router];
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    o[2 * i] = perm32(perm32((uint32_t)i ^ k0) + 1u) & 0x7FFFFFFFu;
    o[2 * i + 1] = perm32(perm32((uint32_t)i ^ k0) + 2u);
  }
}

}  // namespace

extern "C" {

// Pairs of slice `slice` for n hosts; host h's pairs start at pair offset[h] of out.
int synth_gpu_hosts(const uint32_t* d_ip, const uint32_t* d_card, const uint32_t* d_first, const uint32_t* d_last,
                    const uint64_t* d_offset, uint32_t n, uint32_t slice, uint64_t seed, uint32_t* d_out,
                    void* stream) {
  if (!n) return 0;
  k_hosts<<<n < 4096 ? n : 4096, 256, 0, (cudaStream_t)stream>>>(d_ip, d_card, d_first, d_last, d_offset, n, slice,
                                                                  seed, d_out);
  return cudaGetLastError() == cudaSuccess ? 0 : -5;
}

// n noise pairs for each of `routers` routers, router r's at pair offset[r] of out.
int synth_gpu_noise(const uint64_t* d_offset, uint32_t routers, uint64_t n, uint32_t slice, uint64_t seed,
                    uint32_t* d_out, void* stream) {
  if (!n || !routers) return 0;
  const dim3 grid((unsigned)((n + 255) / 256 < 64 ? (n + 255) / 256 : 64), routers);
  k_noise<<<grid, 256, 0, (cudaStream_t)stream>>>(d_offset, n, slice, seed, d_out);
  return cudaGetLastError() == cudaSuccess ? 0 : -5;
}

// Host versions of the same streams (for the oracle side of tests).
void synth_cpu_hosts(const uint32_t* ip, const uint32_t* card, const uint32_t* first, const uint32_t* last,
                     const uint64_t* offset, uint32_t n, uint32_t slice, uint64_t seed, uint32_t* out) {
  for (uint32_t h = 0; h < n; ++h) {
    if (slice < first[h] || slice > last[h]) continue;
    const uint64_t L = last[h] - first[h] + 1, c = card[h], s = slice - first[h];
    const uint32_t j0 = (uint32_t)(c * s / L), j1 = (uint32_t)(c * (s + 1) / L);
    uint32_t* o = out + 2 * offset[h];
    for (uint32_t j = j0; j < j1; ++j) {
      o[2 * (j - j0)] = ip[h];
      o[2 * (j - j0) + 1] = dst_of(seed, ip[h], j);
    }
  }
}

void synth_cpu_noise(const uint64_t* offset, uint32_t routers, uint64_t n, uint32_t slice, uint64_t seed,
                     uint32_t* out) {
  for (uint32_t router = 0; router < routers; ++router) {
    const uint32_t k0 = perm32((uint32_t)seed ^ 0xA5A5A5A5u ^ perm32(router + 0x51ED270Bu)) ^ slice * 0x9E3779B9u;
    uint32_t* o = out + 2 * offset[router];
    for (uint64_t i = 0; i < n; ++i) {
      o[2 * i] = perm32(perm32((uint32_t)i ^ k0) + 1u) & 0x7FFFFFFFu;
      o[2 * i + 1] = perm32(perm32((uint32_t)i ^ k0) + 2u);
    }
  }
}

}  // extern "C"
