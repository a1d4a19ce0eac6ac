// Multi-router batching: one persistent launch updates every router's estimator.
//
// Work items are (router, chunk of item_pairs pairs), ordered router-major. Every tile (a
// piece of one SLEA row, as in k_update_tiled) must see every item once; the CTAs that
// share a tile take items from that tile's counter (atomicAdd, no waiting), so uneven
// router loads balance themselves. A CTA keeps one router's bitmap at a time: when its
// next item belongs to another router it flushes the bitmap into that router's global
// SLEA bitmap and starts a new one. A chunk's RSRA work (Algorithm 3) is done by the
// single tile with index chunk mod tiles.
#pragma once

#include <type_traits>

#include "k_update.cuh"
#include "k_update_tiled.cuh"
#include "sse_internal.cuh"

namespace sse {

constexpr int kMaxRouters = 64;

struct RouterTable {
  uint8_t* state[kMaxRouters];   // RSRA then SLEA of each router
  uint32_t* gbits[kMaxRouters];  // each router's SLEA touched-cell bitmap
};

// Per-step inputs in device memory (refreshed by a copy before every step, so a captured
// graph reads the current pointers and counts).
struct RouterInputs {
  const uint2* pairs[kMaxRouters];
  uint64_t counts[kMaxRouters];
};

template <int UNROLL, bool WHOLE>
__global__ void __launch_bounds__(kTiledThreads, 1)
    k_update_routers(const __grid_constant__ KParams p, TileGeometry g, const __grid_constant__ RouterTable rt,
                     int n_routers, uint64_t sre_bytes, const RouterInputs* __restrict__ in, uint32_t item_pairs,
                     uint32_t* __restrict__ tile_next, const uint32_t* __restrict__ clock,
                     uint8_t* __restrict__ g_sre) {
  const uint64_t* counts = in->counts;
  extern __shared__ __align__(16) uint32_t bm[];
  __shared__ uint64_t first_item[kMaxRouters + 1];
  __shared__ uint32_t sh_item;
  const uint8_t stamp = (uint8_t)*clock;
  const uint32_t tile = blockIdx.x % g.tiles;
  const uint32_t row = tile / g.pieces, piece = tile % g.pieces;
  const uint32_t lo = piece * g.piece_bytes, words = g.piece_bytes >> 5;
  if (threadIdx.x == 0) {
    uint64_t acc = 0;
    for (int r = 0; r < n_routers; ++r) {
      first_item[r] = acc;
      acc += (counts[r] + item_pairs - 1) / item_pairs;
    }
    first_item[n_routers] = acc;
  }
  __syncthreads();
  const uint64_t total = first_item[n_routers];
  const SleTile st(p, row, lo, g.piece_bytes);
  auto touch = [&](uint32_t aip, uint32_t bip) { st.touch<WHOLE, false>(bm, aip, bip); };
  // the bitmap of router r into its global SLEA bitmap (bitmap_or_bulk); with `zero`, the
  // bitmap is cleared for the next router once the reductions have read it
  auto flush = [&](int r, bool zero) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0)
      bitmap_or_bulk(bm, reinterpret_cast<uint8_t*>(rt.gbits[r]) + (((uint64_t)row * p.row_pitch2 + lo) >> 3),
                     tile_flush_bytes(p.row_pitch2, lo, g.piece_bytes), !zero);
    if (zero) {
      __syncthreads();
      for (uint32_t w = threadIdx.x; w < words; w += kTiledThreads) bm[w] = 0;
    }
  };
  for (uint32_t w = threadIdx.x; w < words; w += kTiledThreads) bm[w] = 0;
  RsraQueue rq{reinterpret_cast<uint2*>(bm + words) + (threadIdx.x >> 5) * kRsraQueueEntries, 0u, threadIdx.x & 31u};
  int cur = -1;
  while (true) {
    __syncthreads();  // previous item done; sh_item free
    if (threadIdx.x == 0) sh_item = atomicAdd(&tile_next[tile], 1u);
    __syncthreads();
    const uint64_t it = sh_item;
    if (it >= total) break;
    int r = 0;
    while (r + 1 < n_routers && first_item[r + 1] <= it) ++r;
    if (r != cur) {
      if (cur >= 0) flush(cur, true);
      __syncthreads();
      cur = r;
    }
    const uint64_t chunk = it - first_item[r];
    const uint64_t begin = chunk * item_pairs;
    const uint64_t end = min(begin + item_pairs, counts[r]);
    const bool rsra = (uint32_t)(chunk % g.tiles) == tile;
    const uint2* pairs = in->pairs[r];
    uint8_t* sre = rt.state[r];
    uint64_t j0 = begin;
    if (j0 < end && (reinterpret_cast<uintptr_t>(pairs + j0) & 15u)) {
      if (threadIdx.x == 0) {
        const uint2 v = pairs[j0];
        touch(v.x, v.y);
        if (rsra) stamp_rsra(p, v.x, v.y, sre, stamp, g_sre);
      }
      j0 += 1;
    }
    const uint4* vec = reinterpret_cast<const uint4*>(pairs + j0);
    const uint32_t nvec = (uint32_t)((end - j0) >> 1);
    // the item's RSRA owner runs a separate copy of the loop, so the other tiles execute
    // none of its sampling; iterations are uniform per warp (RsraQueue needs every lane)
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t policy = stream_policy();
    auto scan = [&](auto with_rsra) {
      constexpr bool kRsra = decltype(with_rsra)::value;
      for (uint32_t b0 = threadIdx.x - lane; b0 < nvec; b0 += kTiledThreads * UNROLL) {
        const uint32_t i0 = b0 + lane;
        uint4 buf[UNROLL];
        if (b0 + (UNROLL - 1) * kTiledThreads + 31 < nvec) {  // every load of the warp in range
#pragma unroll
          for (int u = 0; u < UNROLL; ++u) buf[u] = load_stream(vec + i0 + u * kTiledThreads, policy);
#pragma unroll
          for (int u = 0; u < UNROLL; ++u) {
            touch(buf[u].x, buf[u].y);
            touch(buf[u].z, buf[u].w);
          }
          if (kRsra && p.sre_on) {
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
              rq.push(p, true, buf[u].x, buf[u].y, sre, stamp, g_sre);
              rq.push(p, true, buf[u].z, buf[u].w, sre, stamp, g_sre);
            }
          }
          continue;
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
          const uint32_t i = i0 + u * kTiledThreads;
          buf[u] = i < nvec ? load_stream(vec + i, policy) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
          const bool ok = i0 + u * kTiledThreads < nvec;
          if (ok) {
            touch(buf[u].x, buf[u].y);
            touch(buf[u].z, buf[u].w);
          }
          if (kRsra && p.sre_on) {
            rq.push(p, ok, buf[u].x, buf[u].y, sre, stamp, g_sre);
            rq.push(p, ok, buf[u].z, buf[u].w, sre, stamp, g_sre);
          }
        }
      }
      if (kRsra && p.sre_on) rq.drain(p, sre, stamp, g_sre);
    };
    if (rsra)
      scan(std::true_type{});
    else
      scan(std::false_type{});
    if (((end - j0) & 1) && threadIdx.x == 0) {
      const uint2 v = pairs[end - 1];
      touch(v.x, v.y);
      if (rsra) stamp_rsra(p, v.x, v.y, sre, stamp, g_sre);
    }
  }
  if (cur >= 0) flush(cur, false);
  (void)sre_bytes;
}

// k_apply_bits over every router: blockIdx.y is the router. With g_gbits set, every
// router's touched cells are also ORed into the global estimator's bitmap (applied after).
__global__ void __launch_bounds__(256) k_apply_routers(const __grid_constant__ RouterTable rt, uint64_t sre_bytes,
                                                       uint64_t n_words, const uint32_t* __restrict__ clock,
                                                       uint32_t* __restrict__ g_gbits) {
  const uint32_t stamp = *clock;
  uint32_t* gbits = rt.gbits[blockIdx.y];
  uint8_t* sle = rt.state[blockIdx.y] + sre_bytes;
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_words;
       w += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t bits = gbits[w];
    if (!bits) continue;
    if (g_gbits) atomicOr(&g_gbits[w], bits);
    uint4* cells = reinterpret_cast<uint4*>(sle + (w << 5));
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const uint32_t hb = (bits >> (16 * half)) & 0xFFFFu;
      if (!hb) continue;
      uint4 v = cells[half];
      uint32_t x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t nib = (hb >> (4 * q)) & 0xFu;
        const uint32_t mask = ((nib & 1u) ? 0x000000FFu : 0u) | ((nib & 2u) ? 0x0000FF00u : 0u) |
                              ((nib & 4u) ? 0x00FF0000u : 0u) | ((nib & 8u) ? 0xFF000000u : 0u);
        x[q] = (x[q] & ~mask) | (stamp * 0x01010101u & mask);
      }
      cells[half] = make_uint4(x[0], x[1], x[2], x[3]);
    }
    gbits[w] = 0;
  }
}

// Merge of every router into the global estimator (Algorithms 2 and 7: most recent stamp
// per cell) fused with the routers' own expiry: router cells that left the window W(t,k)
// are reset to unset while they are read anyway. 16 cells per thread. With dst == NULL the
// routers are only expired.
__global__ void __launch_bounds__(256) k_merge_routers(uint8_t* __restrict__ dst, const __grid_constant__ RouterTable rt,
                                                       int n_routers, uint64_t n16, uint32_t k,
                                                       const uint32_t* __restrict__ clock) {
  __shared__ uint8_t age_lut[256];
  const uint32_t cs = *clock;
  for (uint32_t s = threadIdx.x; s < 256; s += blockDim.x) age_lut[s] = (uint8_t)stamp_age(s, cs);
  __syncthreads();
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n16; x += (uint64_t)gridDim.x * blockDim.x) {
    const uint4 d = dst ? reinterpret_cast<const uint4*>(dst)[x] : make_uint4(0, 0, 0, 0);
    uint32_t w[4] = {d.x, d.y, d.z, d.w};
    constexpr int kLoads = 4;  // routers' vectors in flight
    for (int r0 = 0; r0 < n_routers; r0 += kLoads) {
      uint4 v[kLoads];
#pragma unroll
      for (int u = 0; u < kLoads; ++u)
        if (r0 + u < n_routers) v[u] = reinterpret_cast<const uint4*>(rt.state[r0 + u])[x];
#pragma unroll
      for (int u = 0; u < kLoads; ++u) {
        if (r0 + u >= n_routers) break;
        const uint32_t o[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
        if ((o[0] | o[1] | o[2] | o[3]) == 0) continue;  // nothing set: no merge, no expiry
        uint32_t keep[4];
        bool expired = false;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          keep[a] = 0;
          if (o[a] == 0) continue;
          uint32_t out = 0, kp = 0;
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const uint32_t s0 = (w[a] >> (8 * b)) & 0xFFu, s1 = (o[a] >> (8 * b)) & 0xFFu;
            out |= (age_lut[s1] < age_lut[s0] ? s1 : s0) << (8 * b);
            kp |= (age_lut[s1] < k ? 0xFFu : 0u) << (8 * b);
          }
          w[a] = out;
          keep[a] = kp;
          expired |= (o[a] & ~kp) != 0;
        }
        if (expired)
          reinterpret_cast<uint4*>(rt.state[r0 + u])[x] =
              make_uint4(o[0] & keep[0], o[1] & keep[1], o[2] & keep[2], o[3] & keep[3]);
      }
    }
    if (dst) reinterpret_cast<uint4*>(dst)[x] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Advances the device clocks of a batch's estimators together.
struct ClockList {
  uint32_t* c[kMaxRouters + 1];
};

__global__ void k_tick_list(const __grid_constant__ ClockList cl, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) cl.c[i][0] = cl.c[i][0] % 255u + 1u;
}

}  // namespace sse
