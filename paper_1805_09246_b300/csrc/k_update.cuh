// Per-packet update of RSRA (Algorithm 3) and SLEA (Algorithm 6): direct stamping.
//
// One thread handles two IP pairs per 128-bit load; the hash functions are evaluated in
// registers and every touched cell is written with the current stamp. Cells written by
// several threads in the same slice all receive the same value, so the writes need no
// atomics and the final state is independent of order and grid shape (Section 3.2:
// a cell may be set to zero many times, which needs no synchronisation).
#pragma once

#include "sse_internal.cuh"

namespace sse {

// Streaming 128-bit load of packet data: read once per SM, so keep it out of L1 and mark it
// first to be evicted from L2, where the estimator should stay resident.
__device__ __forceinline__ uint64_t stream_policy() {
  uint64_t policy;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
  return policy;
}
__device__ __forceinline__ uint4 load_stream(const uint4* ptr, uint64_t policy) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(ptr), "l"(policy));
  return v;
}
__device__ __forceinline__ uint4 load_stream(const uint4* ptr) { return load_stream(ptr, stream_policy()); }

// Exchanges the two ends of n pairs (src <-> dst), for hosts counted as destinations.
__global__ void k_swap_pairs(const uint2* __restrict__ in, uint2* __restrict__ out, uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint2 v = in[i];
    out[i] = make_uint2(v.y, v.x);
  }
}

// Stamps are cells of type St (uint8_t or uint16_t); kernels take byte pointers to the
// estimator and address it in cells.

// Algorithm 6 for one pair: in every row i of SLEA, cell H3(bip) of SLE LH_i(aip); into a
// second SLEA as well when sle2 is set (a serving router's global estimator).
template <typename St, int R2>
__device__ __forceinline__ void stamp_slea(const KParams& p, uint32_t aip, uint32_t bip, St* sle, St stamp,
                                           St* sle2 = nullptr) {
  const uint32_t h3 = mas_top(p.key_a[kH3], p.key_b[kH3], bip, p.lg_eta2);
  const uint32_t rows = R2 > 0 ? (uint32_t)R2 : p.r2;
#pragma unroll
  for (uint32_t i = 0; i < (R2 > 0 ? (uint32_t)R2 : (uint32_t)kMaxRows); ++i) {
    if (R2 == 0 && i >= rows) break;
    const uint32_t j = mas_top(p.key_a[kLH + i], p.key_b[kLH + i], aip, p.q2);
    const uint64_t at = i * p.row_pitch2 + (uint64_t)j * p.delta2 + h3;
    sle[at] = stamp;
    if (sle2) sle2[at] = stamp;
  }
}

// Algorithm 3, sampling test: LSB(H1(bip)) >= tau (the low tau bits of H1 are zero).
__device__ __forceinline__ bool rsra_sampled(const KParams& p, uint32_t bip) {
  return (mas_hi(p.key_a[kH1], p.key_b[kH1], bip) & p.tau_mask) == 0;
}

// Algorithm 3's writes for a sampled pair: cell H2(bip) of SRE RSRA[i, RHFG[i](aip)] in every
// row i, with RHFG[i] from Eq. 6; into a second RSRA as well when sre2 is set (a batch's
// global estimator, which so receives the union of its routers' writes).
template <typename St>
__device__ __forceinline__ void rsra_write(const KParams& p, uint32_t aip, uint32_t bip, St* sre, St stamp,
                                           St* sre2 = nullptr) {
  const uint32_t h2 = mas_top(p.key_a[kH2], p.key_b[kH2], bip, 3);
  const uint32_t r0 = rhfg0(p, aip);
  const uint32_t qmask = (1u << p.q) - 1u;
  uint64_t at = ((uint64_t)r0 << 3) + h2;
  sre[at] = stamp;
  if (sre2) sre2[at] = stamp;
  for (uint32_t i = 1; i < p.r; ++i) {
    const uint32_t col = (uint32_t)((((uint64_t)aip >> (i * p.delta)) ^ r0) & qmask);
    at = ((((uint64_t)i << p.q) + col) << 3) + h2;
    sre[at] = stamp;
    if (sre2) sre2[at] = stamp;
  }
}

// Algorithm 3 for one pair.
template <typename St>
__device__ __forceinline__ void stamp_rsra(const KParams& p, uint32_t aip, uint32_t bip, St* sre, St stamp,
                                           St* sre2 = nullptr) {
  if (p.sre_on && rsra_sampled(p, bip)) rsra_write(p, aip, bip, sre, stamp, sre2);
}

// Warp-cooperative Algorithm 3 for the streaming kernels. Only 2^-tau of the pairs are
// sampled, so a per-pair branch into the write path would be taken by some lane of most
// warps; instead every lane tests its pairs, the sampled ones are appended to the warp's
// queue in shared memory (ballot + prefix count), and each time 32 are queued the whole
// warp writes them, one pair per lane. All 32 lanes must call push() and drain() together.
constexpr uint32_t kRsraQueueEntries = 64;  // per warp: < 32 waiting + up to 32 pushed at once

struct RsraQueue {
  uint2* q;      // this warp's kRsraQueueEntries entries
  uint32_t n;    // entries waiting (the same in every lane)
  uint32_t lane;

  template <typename St>
  __device__ __forceinline__ void push(const KParams& p, bool valid, uint32_t aip, uint32_t bip, St* sre,
                                       St stamp, St* sre2 = nullptr) {
    const bool s = valid && rsra_sampled(p, bip);
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, s);
    if (b == 0) return;
    if (s) q[n + __popc(b & ((1u << lane) - 1u))] = make_uint2(aip, bip);
    n += __popc(b);
    if (n >= 32) {
      __syncwarp();
      const uint2 e = q[lane];
      __syncwarp();
      if (lane + 32 < n) q[lane] = q[lane + 32];
      __syncwarp();
      n -= 32;
      rsra_write(p, e.x, e.y, sre, stamp, sre2);
    }
  }

  template <typename St>
  __device__ __forceinline__ void drain(const KParams& p, St* sre, St stamp, St* sre2 = nullptr) {
    __syncwarp();
    if (lane < n) {
      const uint2 e = q[lane];
      rsra_write(p, e.x, e.y, sre, stamp, sre2);
    }
    __syncwarp();
    n = 0;
  }
};

template <typename St, int R2>
__device__ __forceinline__ void apply_pair(const KParams& p, uint32_t aip, uint32_t bip, St* sre, St* sle,
                                           St stamp, St* sre2, St* sle2) {
  stamp_slea<St, R2>(p, aip, bip, sle, stamp, sle2);
  stamp_rsra(p, aip, bip, sre, stamp, sre2);
}

// pairs: 8-byte aligned {src, dst} pairs. UNROLL 128-bit loads are in flight per thread.
// The stamp is read from the estimator's device clock when `clock` is set, so a captured
// CUDA graph replays correctly in later slices. sre2_bytes / sle2_bytes (may be NULL): a
// second estimator that receives the same stamps (a serving router's global estimator).
template <typename St, int R2, int UNROLL>
__global__ void __launch_bounds__(256) k_update_direct(const __grid_constant__ KParams p,
                                                       const uint2* __restrict__ pairs, uint64_t n,
                                                       uint8_t* __restrict__ sre_bytes, uint8_t* __restrict__ sle_bytes,
                                                       uint32_t stamp_value, const uint32_t* __restrict__ clock,
                                                       uint8_t* __restrict__ sre2_bytes, uint8_t* __restrict__ sle2_bytes) {
  const St stamp = (St)(clock ? *clock : stamp_value);
  St* sre = reinterpret_cast<St*>(sre_bytes);
  St* sle = reinterpret_cast<St*>(sle_bytes);
  St* sre2 = reinterpret_cast<St*>(sre2_bytes);
  St* sle2 = reinterpret_cast<St*>(sle2_bytes);
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint2* base = pairs;
  uint64_t cnt = n;
  if ((reinterpret_cast<uintptr_t>(base) & 15u) != 0 && cnt > 0) {  // peel one pair to reach 16 B
    if (tid == 0) {
      uint2 v = base[0];
      apply_pair<St, R2>(p, v.x, v.y, sre, sle, stamp, sre2, sle2);
    }
    base += 1;
    cnt -= 1;
  }
  const uint4* vec = reinterpret_cast<const uint4*>(base);
  const uint64_t nvec = cnt >> 1;
  for (uint64_t i0 = tid; i0 < nvec; i0 += stride * UNROLL) {
    uint4 buf[UNROLL];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const uint64_t i = i0 + (uint64_t)u * stride;
      if (i < nvec) buf[u] = load_stream(vec + i);
    }
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const uint64_t i = i0 + (uint64_t)u * stride;
      if (i < nvec) {
        apply_pair<St, R2>(p, buf[u].x, buf[u].y, sre, sle, stamp, sre2, sle2);
        apply_pair<St, R2>(p, buf[u].z, buf[u].w, sre, sle, stamp, sre2, sle2);
      }
    }
  }
  if ((cnt & 1) && tid == 0) {
    uint2 v = base[cnt - 1];
    apply_pair<St, R2>(p, v.x, v.y, sre, sle, stamp, sre2, sle2);
  }
}

}  // namespace sse
