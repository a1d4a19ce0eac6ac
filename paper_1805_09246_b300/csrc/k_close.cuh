// Slice close, part 1: expire, weigh and count (Sections 3.2-3.3, Definition 4).
//
// One pass over the whole estimator. For every cell the current stamp decides whether it
// is active in the window W(t,k) (distance < k); cells older than the window are reset to
// unset so that the 255-slice stamp cycle never wraps onto a live cell. RSRA: one thread
// per SRE (8 cells = one 64-bit word); the SRE is hot when at least hot_min cells are
// active, and the warp's 32 hot bits form one word of the hot bitmap. SLEA: 16 cells per
// thread; active cells are summed per row (numerators of the setting factors SF(i,k)).
#pragma once

#include <type_traits>

#include "sse_internal.cuh"

namespace sse {

constexpr int kCloseThreads = 256;
constexpr uint32_t kSleBytesPerBlock = kCloseThreads * 16;  // == kPitchAlign

// The window tests of one pass: four 8-bit or two 16-bit cells at a time.
struct CloseWindow {
  Window8 w8;
  Window16 w16;
};

// One 32-bit word of cells: the top bit of every active cell (8-bit cells tested four at a
// time by active_hi8, 16-bit cells two at a time by active_hi16); WRAP = the window wraps
// over stamp 0.
template <typename St, bool WRAP>
__device__ __forceinline__ uint32_t word_active(uint32_t w, const CloseWindow& win) {
  if constexpr (sizeof(St) == 1)
    return active_hi8<WRAP>(w, win.w8);
  else
    return active_hi16<WRAP>(w, win.w16);
}

// The mask that keeps a word's active cells (all ones over them, zero elsewhere) from its
// top bits: one byte permute (PTX prmt.b32, whose selector nibbles with bit 3 set replicate
// the selected byte's top bit over the result byte) that copies each cell's top bit over
// the cell: selectors 8, 9, 10, 11 (byte i from byte i) for 8-bit cells, 9, 9, 11, 11 (both
// bytes of a cell from its upper byte) for 16-bit cells.
template <typename St>
__device__ __forceinline__ uint32_t keep_mask(uint32_t a) {
  uint32_t r;
  asm("prmt.b32 %0, %1, 0, %2;" : "=r"(r) : "r"(a), "n"(sizeof(St) == 1 ? 0xBA98 : 0xBB99));
  return r;
}

// Active cells of four words' top-bit masks with one population count: shifted by 0..3 the
// masks' bits (7, 15, 23, 31, or 15, 31) no longer overlap.
__device__ __forceinline__ uint32_t count4(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3) {
  return __popc(a0 | (a1 >> 1) | (a2 >> 2) | (a3 >> 3));
}

// A word's top-bit mask packed into one bit per cell, in cell order: for 8-bit cells the
// bits at 0, 8, 16, 24 of a >> 7, multiplied by 1 + 2^7 + 2^14 + 2^21, land on bits 21..24
// without carries (every other term of the product falls below bit 21 on a bit of its own,
// or above bit 24); for 16-bit cells bits 0 and 16, times 1 + 2^15, land on bits 15, 16.
template <typename St>
__device__ __forceinline__ uint32_t pack_active(uint32_t a) {
  if constexpr (sizeof(St) == 1)
    return (((a >> 7) * 0x204081u) >> 21) & 0xFu;
  else
    return (((a >> 15) * 0x8001u) >> 15) & 0x3u;
}

// RSRA part of the pass for 8-bit cells: one SRE (8 bytes) per load, four loads in flight,
// 32-bit indices. A warp covers 64 consecutive SREs 64j .. 64j + 63 per step: lane l holds
// SREs 64j + l and 64j + 32 + l, so its two ballots are the two hot-bitmap words of those
// SREs as they are (lane 0 writes both).
template <bool WRAP>
__device__ __forceinline__ void close_rsra8(const KParams& p, uint8_t* __restrict__ sre,
                                           uint32_t* __restrict__ hot_bits, Window8 win, uint32_t mode) {
  const bool expire = (mode & 1u) != 0;
  const uint32_t n_sre = p.r << p.q;         // a multiple of 32 (q >= 5)
  const uint32_t n_pair = (n_sre + 63) >> 6;  // warp steps: 64 SREs each, the last maybe 32
  uint2* words = reinterpret_cast<uint2*>(sre);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;  // blockDim.x is a multiple of 32
  constexpr int kSteps = 2;                               // warp steps in flight (4 loads per lane)
  for (uint32_t j0 = warp; j0 < n_pair; j0 += kSteps * nwarps) {
    uint2 v[kSteps][2];
#pragma unroll
    for (int u = 0; u < kSteps; ++u) {
      const uint32_t j = j0 + u * nwarps;  // warp-uniform
      if (j < n_pair) {
        v[u][0] = words[64 * j + lane];
        v[u][1] = 64 * j + 32 < n_sre ? words[64 * j + 32 + lane] : make_uint2(0u, 0u);
      }
    }
#pragma unroll
    for (int u = 0; u < kSteps; ++u) {
      const uint32_t j = j0 + u * nwarps;
      if (j >= n_pair) break;  // warp-uniform
      uint32_t bal[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t a0 = active_hi8<WRAP>(v[u][h].x, win), a1 = active_hi8<WRAP>(v[u][h].y, win);
        bal[h] = __ballot_sync(0xFFFFFFFFu, (uint32_t)__popc(a0 | (a1 >> 1)) >= p.hot_min);
        if (expire && 64 * j + 32 * h < n_sre) {
          // cells that are set (non-zero) but not active have left the window
          const uint32_t e0 = v[u][h].x & ~keep_mask<uint8_t>(a0), e1 = v[u][h].y & ~keep_mask<uint8_t>(a1);
          if (e0 | e1) words[64 * j + 32 * h + lane] = make_uint2(v[u][h].x ^ e0, v[u][h].y ^ e1);
        }
      }
      if ((mode & 2u) && lane == 0) {
        if (64 * j + 32 < n_sre)
          reinterpret_cast<uint2*>(hot_bits)[j] = make_uint2(bal[0], bal[1]);
        else
          hot_bits[2 * j] = bal[0];  // the ragged last step: SREs 64j .. 64j + 31 only
      }
    }
  }
}

// The pass of k_close for one window shape (WRAP: see word_active).
template <typename St, bool WRAP>
__device__ __forceinline__ void close_body(const KParams& p, uint8_t* __restrict__ sre, uint8_t* __restrict__ sle,
                                          uint32_t* __restrict__ hot_bits, uint32_t* row_sum,
                                          const CloseWindow& win, uint32_t do_sre, uint32_t mode,
                                          uint32_t* __restrict__ sle_act) {
  using SreWord = typename std::conditional<sizeof(St) == 1, uint2, uint4>::type;
  constexpr int kSreInts = sizeof(SreWord) / 4;
  const bool expire = (mode & 1u) != 0;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;  // a multiple of 32
  if (do_sre && sizeof(St) == 1) {
    close_rsra8<WRAP>(p, sre, hot_bits, win.w8, mode);
  } else if (do_sre) {
    // RSRA: SRE index g (row-major over [r][2^q]); r * 2^q is a multiple of 32, so every
    // iteration covers whole warps.
    const uint64_t n_sre = (uint64_t)p.r << p.q;
    SreWord* words = reinterpret_cast<SreWord*>(sre);
    constexpr int kLoads = 4;  // SREs in flight per thread
    for (uint64_t g0 = tid; g0 < n_sre; g0 += kLoads * nthreads) {
      SreWord v[kLoads];
#pragma unroll
      for (int u = 0; u < kLoads; ++u) {
        const uint64_t g = g0 + u * nthreads;
        if (g < n_sre) v[u] = words[g];
      }
#pragma unroll
      for (int u = 0; u < kLoads; ++u) {
        const uint64_t g = g0 + u * nthreads;
        if (g >= n_sre) break;  // whole warps (g0 and nthreads are multiples of 32 apart)
        uint32_t x[kSreInts], keep[kSreInts], a[kSreInts], expired = 0;
        memcpy(x, &v[u], sizeof(SreWord));
#pragma unroll
        for (int i = 0; i < kSreInts; ++i) {
          a[i] = word_active<St, WRAP>(x[i], win);
          keep[i] = keep_mask<St>(a[i]);
          expired |= x[i] & ~keep[i];
        }
        uint32_t weight;
        if constexpr (kSreInts == 4)
          weight = count4(a[0], a[1], a[2], a[3]);
        else
          weight = __popc(a[0] | (a[1] >> 1));
        const unsigned ballot = __ballot_sync(0xFFFFFFFFu, weight >= p.hot_min);
        if ((mode & 2u) && (threadIdx.x & 31) == 0) hot_bits[g >> 5] = ballot;
        if (expire && expired) {
#pragma unroll
          for (int i = 0; i < kSreInts; ++i) x[i] &= keep[i];
          memcpy(&v[u], x, sizeof(SreWord));
          words[g] = v[u];
        }
      }
    }
  }
  // SLEA: 16 bytes per thread; a row pitch is a multiple of 4096 cells, so a warp's
  // 512 bytes lie in one row. With sle_act, the cells' activity also goes to a bitmap (bit c
  // for cell c of the SLEA): a lane's 16 or 8 bits, two or four lanes to a word.
  const uint64_t n_vec = (uint64_t)p.r2 * p.row_pitch2 * sizeof(St) / 16;
  const uint64_t vec_per_row = p.row_pitch2 * sizeof(St) / 16;
  constexpr uint32_t kVecCells = 16 / sizeof(St);  // cells per lane: 16 or 8
  for (uint64_t x0 = tid - (threadIdx.x & 31); x0 < n_vec; x0 += nthreads) {
    const uint64_t x = x0 + (threadIdx.x & 31);
    uint32_t count = 0, act = 0;
    if (x < n_vec) {
      uint4* cell = reinterpret_cast<uint4*>(sle) + x;
      const uint4 v = *cell;
      uint32_t w[4] = {v.x, v.y, v.z, v.w};
      uint32_t a[4], keep[4], expired = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = word_active<St, WRAP>(w[i], win);
        keep[i] = keep_mask<St>(a[i]);
        expired |= w[i] & ~keep[i];
      }
      count += count4(a[0], a[1], a[2], a[3]);
      if (expire && expired) *cell = make_uint4(w[0] & keep[0], w[1] & keep[1], w[2] & keep[2], w[3] & keep[3]);
      constexpr uint32_t kIntCells = kVecCells / 4;
#pragma unroll
      for (int i = 0; i < 4; ++i) act |= pack_active<St>(a[i]) << (kIntCells * i);
    }
    if (sle_act) {  // warp-uniform
      act |= __shfl_down_sync(0xFFFFFFFFu, act, 1) << kVecCells;
      if constexpr (kVecCells == 8) act |= __shfl_down_sync(0xFFFFFFFFu, act, 2) << 16;
      if ((threadIdx.x & (32 / kVecCells - 1)) == 0 && x < n_vec) sle_act[x * kVecCells / 32] = act;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) count += __shfl_xor_sync(0xFFFFFFFFu, count, off);
    if ((threadIdx.x & 31) == 0 && count) atomicAdd(&row_sum[(uint32_t)(x0 / vec_per_row)], count);
  }
}

// mode bit 0: write back expired cells; bit 1: write the hot bitmap. do_sre != 0: the
// RSRA is processed as well as the SLEA. sle_act (may be NULL): the SLEA cells' activity
// bitmap, for the close's estimate. Grid-stride over both arrays (any grid size).
// Cells are St (8 or 16 bits); one SRE is 8 cells (a 64- or 128-bit word).
// 8-bit cells: eight blocks per SM (32 registers), the occupancy of the launch's grid.
template <typename St>
__global__ void __launch_bounds__(kCloseThreads, sizeof(St) == 1 ? 8 : 1) k_close(const __grid_constant__ KParams p,
                                                          uint8_t* __restrict__ sre, uint8_t* __restrict__ sle,
                                                          uint32_t* __restrict__ hot_bits,
                                                          uint32_t* __restrict__ active2, uint32_t cs_value,
                                                          const uint32_t* __restrict__ clock, uint32_t do_sre,
                                                          uint32_t mode, uint32_t* __restrict__ sle_act) {
  pdl_wait();
  pdl_trigger();
  const uint32_t cs = clock ? *clock : cs_value;
  CloseWindow win;
  win.w8 = window8(cs, p.k);    // 8-bit cells
  win.w16 = window16(cs, p.k);  // 16-bit cells
  __shared__ uint32_t row_sum[kMaxRows];
  if (threadIdx.x < kMaxRows) row_sum[threadIdx.x] = 0;
  __syncthreads();
  const bool wrap = sizeof(St) == 1 ? win.w8.wrap != 0 : win.w16.wrap != 0;
  if (wrap)
    close_body<St, true>(p, sre, sle, hot_bits, row_sum, win, do_sre, mode, sle_act);
  else
    close_body<St, false>(p, sre, sle, hot_bits, row_sum, win, do_sre, mode, sle_act);
  __syncthreads();
  if (threadIdx.x < p.r2 && row_sum[threadIdx.x]) atomicAdd(&active2[threadIdx.x], row_sum[threadIdx.x]);
}

// Hot lists HSE(0) and HSE(1) (column indices, any order) and |HSE(i)| for every row.
// One thread per bitmap word; appends are aggregated per block (warp prefix sums, then one
// atomicAdd per block, iteration and list). Run by blocks blk = 0..nblk-1 of a launch (the
// whole block takes the same role; blockDim.x is a multiple of 32, at most 1024).
__device__ __forceinline__ void hot_lists_part(const uint32_t* __restrict__ hot_bits, uint32_t r, uint32_t q,
                                               uint32_t* __restrict__ hot_count, uint32_t* __restrict__ list0,
                                               uint32_t* __restrict__ list1, uint32_t* __restrict__ n_list,
                                               uint32_t blk, uint32_t nblk) {
  __shared__ uint32_t row_sum[kMaxRows];
  __shared__ uint32_t warp_off[2][32];  // per list: this iteration's warp totals, then offsets
  __shared__ uint32_t block_at[2];      // per list: the block's first entry this iteration
  if (threadIdx.x < kMaxRows) row_sum[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t words_per_row = 1u << (q - 5);
  const uint64_t total = (uint64_t)r * words_per_row;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
  for (uint64_t base = (uint64_t)blk * blockDim.x; base < total; base += (uint64_t)nblk * blockDim.x) {
    const uint64_t wi = base + threadIdx.x;
    const uint32_t word = wi < total ? hot_bits[wi] : 0u;
    const uint32_t row = wi < total ? (uint32_t)(wi >> (q - 5)) : 0u;
    const uint32_t bits = __popc(word);
    if (bits) atomicAdd(&row_sum[row], bits);
    // rows 0 and 1: the column of every hot SRE goes to that row's list
    uint32_t incl[2];
#pragma unroll
    for (uint32_t rr = 0; rr < 2; ++rr) {
      incl[rr] = (row == rr) ? bits : 0u;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl[rr], off);
        if (lane >= (uint32_t)off) incl[rr] += t;
      }
      if (lane == 31) warp_off[rr][warp] = incl[rr];
    }
    __syncthreads();
    if (threadIdx.x < 2) {
      const uint32_t rr = threadIdx.x;
      uint32_t run = 0;
      for (uint32_t w = 0; w < n_warps; ++w) {
        const uint32_t t = warp_off[rr][w];
        warp_off[rr][w] = run;
        run += t;
      }
      block_at[rr] = run ? atomicAdd(&n_list[rr], run) : 0u;
    }
    __syncthreads();
    if (row < 2 && bits) {
      uint32_t* list = row == 0 ? list0 : list1;
      uint32_t at = block_at[row] + warp_off[row][warp] + incl[row] - bits;
      const uint32_t col0 = (uint32_t)(wi & (words_per_row - 1)) << 5;
      for (uint32_t m = word; m; m &= m - 1) list[at++] = col0 + (__ffs(m) - 1);
    }
    __syncthreads();  // warp_off and block_at are rewritten by the next iteration
  }
  if (threadIdx.x < r && row_sum[threadIdx.x]) atomicAdd(&hot_count[threadIdx.x], row_sum[threadIdx.x]);
}

}  // namespace sse
