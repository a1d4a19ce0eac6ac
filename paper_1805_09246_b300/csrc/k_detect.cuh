// Slice close, part 2: candidate hosts, ordering and estimation.
//
// Candidates (Section 3.3, Algorithms 4-5). A host aip is a candidate when all r of its
// SREs RSRA[i, RHFG[i](aip)] are hot. For hot he_0 in row 0 and he_1 in row 1,
// B(1) = he_0 XOR he_1 holds aip bits [delta, delta+q) (Eq. 7). Row i >= 2 must hold
// B(i) = he_0 XOR he_i whose low q-delta bits repeat the top q-delta bits of B(i-1),
// so only its top delta bits are free: the 2^delta choices are looked up in row i's hot
// bitmap (the paper's overlap test, applied to all of HSE(i) at once). A complete chain
// fixes bits [delta, 32); the delta low bits are enumerated and a host is kept when
// RHFG[0] maps it back to he_0, which makes all of its r SREs exactly the chain's. Where a
// 32-bit address leaves B(r-1) fewer than q bits, k_join_down finds the same chains from
// rows 0 and r-1 down (see there); k_join_tiled and k_join grow them from rows 0, 1, 2 up.
//
// Estimation (Algorithm 8, Eq. 11-12): one block per host gathers its r' SLEs; a cell of
// the union SLE counts when it is active in every row, with the largest distance over the
// rows; the corrected weight and the estimate are computed in FP64 with explicit
// round-to-nearest operations in a fixed order, so the super point decision is exact.
#pragma once

#include <cstddef>
#include <type_traits>

#include "k_close.cuh"
#include "sse_internal.cuh"

namespace sse {

__device__ __forceinline__ bool hot_bit(const uint32_t* hot_bits, uint32_t q, uint32_t row, uint32_t col) {
  return (hot_bits[((uint64_t)row << (q - 5)) + (col >> 5)] >> (col & 31)) & 1u;
}

// B(i) = (aip >> i*delta) mod 2^q must have no bits at or above address bit 32.
__device__ __forceinline__ bool fits32(uint32_t i, uint32_t delta, uint32_t q, uint32_t b) {
  const uint32_t lo = i * delta;
  if (lo >= 32) return b == 0;
  if (lo + q > 32) return (b >> (32 - lo)) == 0;
  return true;
}

// The top bits t of he_i (i >= 2) that keep B(i) inside 32 address bits, as a mask over
// the 2^delta SREs of a row-i group: B(i)'s top delta bits, (t XOR hi0) with hi0 the top
// delta bits of he_0, sit at address bits [i*delta + q - delta, i*delta + q), so only the
// w = 32 - (i*delta + q - delta) low ones (0 <= w <= delta) may be set: t must agree with hi0
// above bit w, 2^w consecutive values. (Its low q - delta bits come from B(i-1), which fits.)
__device__ __forceinline__ uint32_t fits32_tops(uint32_t i, uint32_t delta, uint32_t q, uint32_t hi0) {
  const int top = (int)(i * delta + q - delta);
  const int w = 32 - top;
  if (w >= (int)delta) return delta == 5 ? 0xFFFFFFFFu : (1u << (1u << delta)) - 1u;
  if (w <= 0) return 1u << hi0;
  const uint32_t base = (hi0 >> w) << w;
  return ((1u << (1u << w)) - 1u) << base;
}

__device__ __forceinline__ void emit_candidate(uint32_t aip, uint32_t* cand, uint32_t* n_cand, uint32_t cap,
                                               uint32_t* overflow) {
  const uint32_t at = atomicAdd(n_cand, 1u);
  if (at < cap)
    cand[at] = aip;
  else
    atomicOr(overflow, 1u);
}

// The 2^delta (<= 32) values a * low (mod 2^64), low < 2^delta, of the multiply-add-shift
// RHFG[0]'s multiplier a, in ascending order with their low bits (a is odd, so they are
// distinct). Built in shared memory by the threads below 2^delta of a block (the caller
// synchronises before use).
struct RegainTable {
  uint64_t d[32];
  uint32_t low[32];
  uint8_t first[65];  // entries below j * 2^58, j = 0..64 (regain_search_bucketed)
};
__device__ __forceinline__ void build_regain_table(const KParams& p, RegainTable* t) {
  const uint32_t n = 1u << p.delta;
  const uint64_t a = p.key_a[kR0];
  if (threadIdx.x < n) {
    const uint64_t d = a * threadIdx.x;
    uint32_t rank = 0;
    for (uint32_t j = 0; j < n; ++j) rank += (a * j < d) ? 1u : 0u;
    t->d[rank] = d;
    t->low[rank] = threadIdx.x;
  }
  if (threadIdx.x <= 64) {
    uint32_t below = 0;
    for (uint32_t j = 0; j < n; ++j) below += ((a * j) >> 58) < threadIdx.x ? 1u : 0u;
    t->first[threadIdx.x] = (uint8_t)below;
  }
}

// Regain the hosts of a complete chain B[1..r-1] (bits [delta, 32) fixed).
// With the multiply-add-shift RHFG[0], the top q bits of a*x + b (mod 2^64) equal he_0
// exactly when v = a*x + b - (he_0 << (64 - q)) (mod 2^64) is below W = 2^(64-q); with
// x = high | low, v = v0 + a*low, i.e. a*low (mod 2^64) lies in the circular interval
// [-v0, -v0 + W). Given the sorted table of a*low (rt), the lows are found by a binary
// search for -v0 and a walk while (a*low + v0) mod 2^64 < W, usually a single test;
// otherwise each low costs a compare and an add (stepping x adds a each time).
// `high`: address bits [delta, 32) of the chain (Eq. 7).
__device__ __forceinline__ void regain_high(const KParams& p, uint32_t he0, uint64_t high, uint32_t* cand,
                                            uint32_t* n_cand, uint32_t cap, uint32_t* overflow,
                                            const RegainTable* rt) {
  if (p.tab) {
    for (uint32_t low = 0; low < (1u << p.delta); ++low) {
      const uint32_t aip = (uint32_t)(high | low);
      if (rhfg0(p, aip) != he0) continue;
      emit_candidate(aip, cand, n_cand, cap, overflow);
    }
    return;
  }
  const uint64_t a = p.key_a[kR0];
  const uint64_t width = 1ull << (64 - p.q);
  uint64_t v = a * (uint32_t)high + p.key_b[kR0] - ((uint64_t)he0 << (64 - p.q));
  if (rt) {
    regain_search_bucketed(rt->d, rt->low, rt->first, 1u << p.delta, v, width,
                           [&](uint32_t low) { emit_candidate((uint32_t)high | low, cand, n_cand, cap, overflow); });
    return;
  }
  for (uint32_t low = 0; low < (1u << p.delta); ++low, v += a)
    if (v < width) emit_candidate((uint32_t)high | low, cand, n_cand, cap, overflow);
}

// The chain B[1..r-1]: B(1) gives address bits [delta, delta + q), each further B(i) its top
// delta bits at [i*delta + q - delta, (i+1)*delta + q - delta) (Eq. 7).
__device__ __forceinline__ void regain(const KParams& p, uint32_t he0, const uint32_t* B, uint32_t* cand,
                                       uint32_t* n_cand, uint32_t cap, uint32_t* overflow,
                                       const RegainTable* rt = nullptr) {
  uint64_t high = (uint64_t)B[1] << p.delta;
  for (uint32_t i = 2; i < p.r; ++i)
    high |= (uint64_t)(B[i] >> (p.q - p.delta)) << (i * p.delta + p.q - p.delta);
  regain_high(p, he0, high, cand, n_cand, cap, overflow, rt);
}

// Rows 3..r-1 of a chain whose rows 0..2 are hot (rare: depth-first, explicit stack).
__device__ __noinline__ void grow_deep(const KParams& p, const uint32_t* hot_bits, uint32_t he0, uint32_t b1,
                                       uint32_t b2, uint32_t* cand, uint32_t* n_cand, uint32_t cap,
                                       uint32_t* overflow) {
  uint32_t B[kMaxRows];
  uint32_t next[kMaxRows];
  B[1] = b1;
  B[2] = b2;
  const uint32_t fan = 1u << p.delta;
  const uint32_t shift_hi = p.q - p.delta;
  int i = 3;
  if (i < (int)p.r) next[i] = 0;
  while (i >= 3) {
    if (i == (int)p.r) {  // chain complete
      regain(p, he0, B, cand, n_cand, cap, overflow);
      i -= 1;
      continue;
    }
    if (next[i] == fan) {  // level exhausted
      i -= 1;
      continue;
    }
    const uint32_t bi = (B[i - 1] >> p.delta) | (next[i] << shift_hi);
    next[i] += 1;
    if (!fits32(i, p.delta, p.q, bi) || !hot_bit(hot_bits, p.q, i, he0 ^ bi)) continue;
    B[i] = bi;
    i += 1;
    if (i < (int)p.r) next[i] = 0;
  }
}

// Hot bitmaps of rows 2..r-1 regrouped for the join: bit (c << delta) + t of table i-2 is
// the hot flag of SRE c | (t << (q - delta)) of row i, so the 2^delta SREs that share their
// low q-delta bits c (the part of B(i) fixed by B(i-1)) are adjacent bits.
// One thread per output word (rows flattened); blocks blk = 0..nblk-1 of a launch.
// With delta <= 5 and q - delta >= 5, output word w = j * 2^delta + m holds c = 32j +
// m * (32 >> delta) + b for b < 32 >> delta, and every t: bits m * (32 >> delta) + b of the
// 2^delta input words j + t * 2^(q-delta-5), one load per t. Otherwise bit by bit.
__device__ __forceinline__ void regroup_part(const uint32_t* __restrict__ hot_bits, uint32_t r, uint32_t q,
                                             uint32_t delta, uint32_t* __restrict__ tables, uint32_t blk,
                                             uint32_t nblk) {
  const uint64_t nwords = (1ull << q) >> 5;
  const uint64_t total = (uint64_t)(r - 2) * nwords;
  const uint32_t tmask = (1u << delta) - 1u;
  const bool fast = delta <= 5 && q - delta >= 5;
  for (uint64_t x = (uint64_t)blk * blockDim.x + threadIdx.x; x < total; x += (uint64_t)nblk * blockDim.x) {
    const uint32_t row = 2 + (uint32_t)(x / nwords);
    const uint64_t w = x % nwords;
    const uint32_t* src = hot_bits + ((uint64_t)row << (q - 5));
    uint32_t out = 0;
    if (fast) {
      const uint32_t per = 32u >> delta;  // c values per output word
      const uint64_t j = w >> delta;
      const uint32_t m = (uint32_t)w & tmask;
      const uint64_t tstride = 1ull << (q - delta - 5);
      for (uint32_t t0 = 0; t0 <= tmask; t0 += 8) {  // 8 loads in flight (2^delta >= 2)
        uint32_t v[8];
#pragma unroll
        for (uint32_t u = 0; u < 8; ++u) v[u] = t0 + u <= tmask ? src[j + (t0 + u) * tstride] : 0u;
#pragma unroll
        for (uint32_t u = 0; u < 8; ++u) {
          if (t0 + u > tmask) break;
          const uint32_t x = v[u] >> (m * per);
          for (uint32_t b = 0; b < per; ++b) out |= ((x >> b) & 1u) << ((b << delta) + t0 + u);
        }
      }
    } else {
      for (uint32_t b = 0; b < 32; ++b) {
        const uint64_t bit = (w << 5) + b;
        const uint32_t c = (uint32_t)(bit >> delta), t = (uint32_t)bit & tmask;
        out |= (hot_bit(hot_bits, q, row, c | (t << (q - delta))) ? 1u : 0u) << b;
      }
    }
    tables[x] = out;
  }
}

// "Any hot" bitmap of one row (delta <= 5): bit c is set when some of the 2^delta SREs
// c | (t << (q - delta)) is hot. With q - delta >= 5, output word j is the OR over t of the
// row's bitmap words j + t * 2^(q-delta-5); otherwise the single word is built bit by bit.
// Blocks blk = 0..nblk-1 of a launch.
__device__ __forceinline__ void any_part(const uint32_t* __restrict__ hot_bits, uint32_t row, uint32_t q,
                                         uint32_t delta, uint32_t* __restrict__ any, uint32_t blk, uint32_t nblk) {
  const uint32_t* src = hot_bits + ((uint64_t)row << (q - 5));
  if (q - delta < 5) {
    if (blk == 0 && threadIdx.x == 0) {
      uint32_t out = 0;
      for (uint32_t c = 0; c < (1u << (q - delta)); ++c)
        for (uint32_t t = 0; t < (1u << delta); ++t)
          if (hot_bit(hot_bits, q, row, c | (t << (q - delta)))) out |= 1u << c;
      any[0] = out;
    }
    return;
  }
  const uint32_t n_words = (1u << (q - delta)) >> 5;
  const uint32_t tstride = 1u << (q - delta - 5);
  for (uint32_t j = blk * blockDim.x + threadIdx.x; j < n_words; j += nblk * blockDim.x) {
    uint32_t out = 0;
    for (uint32_t t0 = 0; t0 < (1u << delta); t0 += 8) {  // 8 loads in flight
      uint32_t v[8];
#pragma unroll
      for (uint32_t u = 0; u < 8; ++u) v[u] = t0 + u < (1u << delta) ? src[j + (t0 + u) * tstride] : 0u;
#pragma unroll
      for (uint32_t u = 0; u < 8; ++u) out |= v[u];
    }
    any[j] = out;
  }
}

// Eq. 12's P = prod_i SF(i,k), SF(i,k) = active2[i] / row_len2 (Definition 4), multiplied
// in row order with round-to-nearest FP64 operations.
__device__ __forceinline__ double setting_product(const uint32_t* active2, uint32_t r2, uint64_t row_len2) {
  double P = 1.0;
  for (uint32_t i = 0; i < r2; ++i) P = __dmul_rn(P, __ddiv_rn((double)active2[i], (double)row_len2));
  return P;
}

struct LcResult {
  double w;       // corrected weight (Eq. 12), clamped to [0, eta' - 1]
  float est;      // Eq. 8 on w
  uint8_t flags;  // SSE_FLAG_SUPER when w >= w_theta; SSE_FLAG_SATURATED when clamped at eta' - 1
};

// Algorithm 8's last steps for a host whose union SLE has U active cells: w from Eq. 12 in
// FP64 with round-to-nearest operations in a fixed order (so the super point decision is
// exact), and the estimate of Eq. 8.
__device__ __forceinline__ LcResult lc_estimate(uint32_t U, double P, double eta2, double w_theta) {
  LcResult res;
  res.flags = 0;
  double w;
  if (P >= 1.0) {
    w = eta2 - 1.0;
    res.flags |= SSE_FLAG_SATURATED;
  } else {
    const double num = __dsub_rn((double)U, __dmul_rn(eta2, P));
    const double den = __dsub_rn(1.0, P);
    w = __ddiv_rn(num, den);
    if (w < 0.0) w = 0.0;
    if (!(w <= eta2 - 1.0)) {
      w = eta2 - 1.0;
      res.flags |= SSE_FLAG_SATURATED;
    }
  }
  // est = -eta' ln(1 - x), x = w / eta' < 1 (eta' is a power of two, so x is exact). The
  // flag is decided on w in FP64; the FP32 estimate is taken in FP32 from an argument that
  // is exact in FP64: log1p(-x) below x = 1/2 (no cancellation), else log(1 - x), where
  // 1 - x is exact (Sterbenz). Either way a few FP32 ulps from the FP64 value.
  const double x = __dmul_rn(w, 1.0 / eta2);
  const float lg = x < 0.5 ? log1pf((float)-x) : logf((float)__dsub_rn(1.0, x));
  res.est = -(float)eta2 * lg;
  if (w >= w_theta) res.flags |= SSE_FLAG_SUPER;
  res.w = w;
  return res;
}

// lc_estimate for every U = 0..eta' under one close's P (the same for all of its hosts),
// built by `blocks` blocks of k_hot_prep; the estimates of that close then look U up. Unused
// (est == nullptr) outside the slice close.
struct EstTable {
  double* w;
  float* est;
  uint8_t* flags;
  const uint32_t* active2;  // SLEA row counts of the close (for P)
  uint64_t row_len2;
  double w_theta;
  uint32_t r2, eta2, blocks;
  uint32_t per_block;  // entries per block (a multiple of 32, at most the block size): the
                       // FP64 work spread over many SMs
};

// The hot SREs of one row grouped by column block: block b (columns [b * 2^s, (b+1) * 2^s),
// 5 <= s < q) lists its hot columns at blist[b * 2^s ...] (any order) and their number in
// bcount[b]. One block of the launch per column block (b = blk, blk + nblk, ...), which
// reads the block's 2^(s-5) bitmap words 8 per thread at a time.
__device__ __forceinline__ void block_list_part(const uint32_t* __restrict__ hot_bits, uint32_t row, uint32_t q,
                                                uint32_t s, uint32_t* __restrict__ blist,
                                                uint32_t* __restrict__ bcount, uint32_t blk, uint32_t nblk) {
  __shared__ uint32_t s_n;
  const uint32_t nb = 1u << (q - s), wpb = 1u << (s - 5);
  const uint32_t* src = hot_bits + ((uint64_t)row << (q - 5));
  for (uint32_t b = blk; b < nb; b += nblk) {
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    uint32_t* out = blist + ((uint64_t)b << s);
    for (uint32_t w0 = 0; w0 < wpb; w0 += 8 * blockDim.x) {
      uint32_t v[8];
#pragma unroll
      for (uint32_t u = 0; u < 8; ++u) {
        const uint32_t w = w0 + u * blockDim.x + threadIdx.x;
        v[u] = w < wpb ? src[b * wpb + w] : 0u;
      }
#pragma unroll
      for (uint32_t u = 0; u < 8; ++u) {
        uint32_t x = v[u];
        if (!x) continue;
        uint32_t at = atomicAdd(&s_n, (uint32_t)__popc(x));
        const uint32_t col0 = (b * wpb + w0 + u * blockDim.x + threadIdx.x) << 5;
        while (x) {
          out[at++] = col0 + (uint32_t)(__ffs(x) - 1);
          x &= x - 1u;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) bcount[b] = s_n;
    __syncthreads();  // s_n is reset for the next column block
  }
}

// Everything the join reads from the hot bitmap, in one launch: blocks [0, n_lists) build
// the hot lists of rows 0-1 and the hot counts, the next n_regroup blocks the regrouped
// tables of rows 2..r-1, the next n_block blocks row r-1's hot SREs by column block of 2^s
// (the join from the top row down), the rest (when any2 != NULL) the "any hot" bitmaps of
// rows 2 and 3 (any3 when r > 3), half of them each.
__global__ void __launch_bounds__(256) k_hot_prep(const uint32_t* __restrict__ hot_bits, uint32_t r, uint32_t q,
                                                  uint32_t delta, uint32_t* __restrict__ hot_count,
                                                  uint32_t* __restrict__ list0, uint32_t* __restrict__ list1,
                                                  uint32_t* __restrict__ n_list, uint32_t* __restrict__ tables,
                                                  uint32_t* __restrict__ any2, uint32_t* __restrict__ any3,
                                                  uint32_t n_lists, uint32_t n_regroup, EstTable tab,
                                                  uint32_t* __restrict__ blist, uint32_t* __restrict__ bcount,
                                                  uint32_t n_block, uint32_t s) {
  pdl_wait();
  pdl_trigger();
  const uint32_t b = blockIdx.x;
  if (b >= gridDim.x - tab.blocks) {  // the last tab.blocks blocks: the estimate table
    // Eq. 12's P as in setting_product (the same quotients, multiplied in row order), with the
    // r' divisions done side by side
    __shared__ double quot[kMaxRows];
    if (threadIdx.x < tab.r2) quot[threadIdx.x] = __ddiv_rn((double)tab.active2[threadIdx.x], (double)tab.row_len2);
    __syncthreads();
    double P = 1.0;
    for (uint32_t i = 0; i < tab.r2; ++i) P = __dmul_rn(P, quot[i]);
    const uint32_t U = (b - (gridDim.x - tab.blocks)) * tab.per_block + threadIdx.x;
    if (threadIdx.x < tab.per_block && U <= tab.eta2) {
      const LcResult res = lc_estimate(U, P, (double)tab.eta2, tab.w_theta);
      tab.w[U] = res.w;
      tab.est[U] = res.est;
      tab.flags[U] = res.flags;
    }
    return;
  }
  if (b < n_lists) {
    hot_lists_part(hot_bits, r, q, hot_count, list0, list1, n_list, b, n_lists);
  } else if (b < n_lists + n_regroup) {
    regroup_part(hot_bits, r, q, delta, tables, b - n_lists, n_regroup);
  } else if (b < n_lists + n_regroup + n_block) {
    block_list_part(hot_bits, r - 1, q, s, blist, bcount, b - n_lists - n_regroup, n_block);
  } else if (any2) {
    const uint32_t first_any = n_lists + n_regroup + n_block;
    const uint32_t rest = gridDim.x - first_any - tab.blocks, x = b - first_any;
    const uint32_t half = (rest + 1) / 2;
    if (x < half)
      any_part(hot_bits, 2, q, delta, any2, x, half);
    else if (any3)
      any_part(hot_bits, 3, q, delta, any3, x - half, rest - half);
  }
}

// The 2^delta (<= 32) hot flags, indexed by the top delta bits of he_i, of the row whose
// regrouped table is `table`, for the SREs whose low q-delta bits are c.
__device__ __forceinline__ uint32_t hot_group(const uint32_t* table, uint32_t c, uint32_t delta) {
  const uint32_t first = c << delta;
  const uint32_t span = 1u << delta;
  const uint32_t w = table[first >> 5];
  return span == 32 ? w : (w >> (first & 31)) & ((1u << span) - 1u);
}

// Rows 3..r-1 for delta <= 5: depth-first over the set bits of each row's hot group.
__device__ __forceinline__ void grow_grouped(const KParams& p, const uint32_t* tables, uint32_t he0, uint32_t b1,
                                          uint32_t b2, uint32_t* cand, uint32_t* n_cand, uint32_t cap,
                                          uint32_t* overflow, const RegainTable* rt = nullptr) {
  const uint32_t delta = p.delta, q = p.q, shift_hi = q - delta;
  const uint32_t cmask = (1u << shift_hi) - 1u, hi0 = he0 >> shift_hi;
  const uint64_t nwords = (1ull << q) >> 5;
  uint32_t B[kMaxRows], M[kMaxRows];
  B[1] = b1;
  B[2] = b2;
  int i = 3;
  if (i < (int)p.r) M[i] = hot_group(tables + (uint64_t)(i - 2) * nwords, (he0 ^ (b2 >> delta)) & cmask, delta);
  while (i >= 3) {
    if (i == (int)p.r) {  // chain complete
      regain(p, he0, B, cand, n_cand, cap, overflow, rt);
      i -= 1;
      continue;
    }
    if (M[i] == 0) {  // level exhausted
      i -= 1;
      continue;
    }
    const uint32_t tp = __ffs(M[i]) - 1;  // top bits of he_i
    M[i] &= M[i] - 1;
    const uint32_t bi = (B[i - 1] >> delta) | ((tp ^ hi0) << shift_hi);
    if (!fits32(i, delta, q, bi)) continue;
    B[i] = bi;
    i += 1;
    if (i < (int)p.r) M[i] = hot_group(tables + (uint64_t)(i - 2) * nwords, (he0 ^ (bi >> delta)) & cmask, delta);
  }
}

// grow_grouped for r = 5: rows 3 and 4 as two nested loops over their hot groups, the chain
// in registers.
__device__ __forceinline__ void grow_grouped5(const KParams& p, const uint32_t* tables, uint32_t he0, uint32_t b1,
                                           uint32_t b2, uint32_t* cand, uint32_t* n_cand, uint32_t cap,
                                           uint32_t* overflow, const RegainTable* rt) {
  const uint32_t delta = p.delta, q = p.q, shift_hi = q - delta;
  const uint32_t cmask = (1u << shift_hi) - 1u, hi0 = he0 >> shift_hi;
  const uint64_t nwords = (1ull << q) >> 5;
  const uint64_t high12 = ((uint64_t)b1 << delta) | ((uint64_t)(b2 >> shift_hi) << (2 * delta + shift_hi));
  uint32_t m3 = hot_group(tables + nwords, (he0 ^ (b2 >> delta)) & cmask, delta);
  while (m3) {
    const uint32_t b3 = (b2 >> delta) | (((uint32_t)(__ffs(m3) - 1) ^ hi0) << shift_hi);
    m3 &= m3 - 1u;
    if (!fits32(3, delta, q, b3)) continue;
    const uint64_t high123 = high12 | ((uint64_t)(b3 >> shift_hi) << (3 * delta + shift_hi));
    uint32_t m4 = hot_group(tables + 2 * nwords, (he0 ^ (b3 >> delta)) & cmask, delta);
    while (m4) {
      const uint32_t b4 = (b3 >> delta) | (((uint32_t)(__ffs(m4) - 1) ^ hi0) << shift_hi);
      m4 &= m4 - 1u;
      if (!fits32(4, delta, q, b4)) continue;
      regain_high(p, he0, high123 | ((uint64_t)(b4 >> shift_hi) << (4 * delta + shift_hi)), cand, n_cand, cap,
                  overflow, rt);
    }
  }
}

// Rows 3..r-1 of one queued chain: the r = 5 loops, else the general depth-first walk.
__device__ __forceinline__ void grow_chain(const KParams& p, const uint32_t* tables, uint32_t he0, uint32_t b1,
                                        uint32_t b2, uint32_t* cand, uint32_t* n_cand, uint32_t cap,
                                        uint32_t* overflow, const RegainTable* rt) {
  if (p.r == 5)
    grow_grouped5(p, tables, he0, b1, b2, cand, n_cand, cap, overflow, rt);
  else
    grow_grouped(p, tables, he0, b1, b2, cand, n_cand, cap, overflow, rt);
}

constexpr int kJoinThreads = 1024;

// Blocks stride over HSE(0), threads over HSE(1). For a pair (he_0, he_1), B(1) fixes the
// low q-delta bits c of every admissible he_2 (he_2 = he_0 XOR B(2)); the regrouped row-2
// table gives all 2^delta hot flags of those he_2 at once. A chain through rows 0-2 then
// needs some hot SRE in row 3 among the 2^delta its B(2) admits: that is one bit of row 3's
// "any hot" bitmap (any3, when given), checked in shared memory before the chain is grown
// from the global tables. Shared memory holds, when they fit: the row-2 table (smem_t2),
// any3, and HSE(1) (up to list1_cap entries).
__global__ void __launch_bounds__(kJoinThreads) k_join(const __grid_constant__ KParams p,
                                                       const uint32_t* __restrict__ hot_bits,
                                                       const uint32_t* __restrict__ tables,
                                                       const uint32_t* __restrict__ any3,
                                                       const uint32_t* __restrict__ list0,
                                                       const uint32_t* __restrict__ list1,
                                                       const uint32_t* __restrict__ n_list, uint32_t* __restrict__ cand,
                                                       uint32_t* __restrict__ n_cand, uint32_t cap,
                                                       uint32_t* __restrict__ overflow, uint32_t smem_t2,
                                                       uint32_t list1_cap) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ uint32_t sm[];
  const uint32_t n0 = n_list[0], n1 = n_list[1];
  if (n0 == 0 || n1 == 0) return;
  const uint32_t delta = p.delta, q = p.q;
  const uint32_t shift_hi = q - delta;
  const uint32_t cmask = (1u << shift_hi) - 1u;
  const uint32_t span = 1u << delta;  // flags per c
  const bool grouped = span <= 32;
  const bool row2_fits_all = 2 * delta + q <= 32;
  const uint32_t nwords = (1u << q) >> 5;
  const uint32_t* t2 = tables;
  uint32_t* sm_next = sm;
  if (smem_t2) {
    for (uint32_t w = threadIdx.x; w < nwords; w += blockDim.x) sm[w] = tables[w];
    t2 = sm;
    sm_next = sm + nwords;
  }
  const uint32_t* a3 = nullptr;
  if (any3) {
    const uint32_t any_words = (1u << shift_hi) >> 5;
    for (uint32_t w = threadIdx.x; w < any_words; w += blockDim.x) sm_next[w] = any3[w];
    a3 = sm_next;
    sm_next += any_words;
  }
  const uint32_t* l1 = list1;
  if (n1 <= list1_cap) {
    for (uint32_t x = threadIdx.x; x < n1; x += blockDim.x) sm_next[x] = list1[x];
    l1 = sm_next;
  }
  __syncthreads();
  for (uint32_t a = blockIdx.x; a < n0; a += gridDim.x) {
    const uint32_t he0 = list0[a];
    const uint32_t hi0 = he0 >> shift_hi;  // top delta bits of he_0
    for (uint32_t b = threadIdx.x; b < n1; b += blockDim.x) {
      const uint32_t b1 = he0 ^ l1[b];
      if (!fits32(1, delta, q, b1)) continue;
      const uint32_t low2 = b1 >> delta;
      const uint32_t first = ((he0 ^ low2) & cmask) << delta;
      for (uint32_t base = 0; base < span; base += 32) {
        uint32_t m = t2[(first + base) >> 5];
        if (span < 32) m = (m >> (first & 31)) & ((1u << span) - 1u);
        while (m) {
          const uint32_t tp = base + (__ffs(m) - 1);  // top bits of he_2
          m &= m - 1;
          const uint32_t b2 = low2 | ((tp ^ hi0) << shift_hi);
          if (!row2_fits_all && !fits32(2, delta, q, b2)) continue;
          if (a3) {
            const uint32_t c3 = (he0 ^ (b2 >> delta)) & cmask;
            if (!((a3[c3 >> 5] >> (c3 & 31)) & 1u)) continue;
          }
          if (grouped)
            grow_grouped(p, tables, he0, b1, b2, cand, n_cand, cap, overflow);
          else
            grow_deep(p, hot_bits, he0, b1, b2, cand, n_cand, cap, overflow);
        }
      }
    }
  }
}

// The close's report written straight into page-locked, device-mapped host memory (one
// kernel instead of copy-engine transfers): the counters, then the first min(n_cand, cap,
// n_stage) hosts, estimates and flags. Layout: CloseScratch | hosts[n_stage] |
// est[n_stage] | flags[n_stage]. When tick_clock is set, the last step of the close — the
// clock moving to the next slice's stamp (1..tick_mod) — is done here too (nothing in this
// kernel reads the clock). The last block to finish sets the stage's report_done after
// every block's writes are visible to the host (system-scope fences), so the host can wait
// on that word instead of on the stream.
__global__ void __launch_bounds__(256) k_report(CloseScratch* __restrict__ sc, const uint32_t* __restrict__ hosts,
                                                const float* __restrict__ est, const uint8_t* __restrict__ flags,
                                                uint32_t cap, uint32_t n_stage, uint8_t* __restrict__ out,
                                                uint32_t* __restrict__ tick_clock, uint32_t tick_mod) {
  pdl_wait();
  pdl_trigger();
  if (tick_clock && blockIdx.x == 0 && threadIdx.x == 0) *tick_clock = *tick_clock % tick_mod + 1u;
  const uint32_t n = min(min(sc->n_cand, cap), n_stage);
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  constexpr uint32_t kWords = offsetof(CloseScratch, report_blocks) / 4;  // the counters before the flags
  for (uint32_t i = tid; i < kWords; i += stride)
    reinterpret_cast<uint32_t*>(out)[i] = reinterpret_cast<const uint32_t*>(sc)[i];
  uint32_t* oh = reinterpret_cast<uint32_t*>(out + sizeof(CloseScratch));
  float* oe = reinterpret_cast<float*>(oh + n_stage);
  uint8_t* of = reinterpret_cast<uint8_t*>(oe + n_stage);
  for (uint32_t i = tid; i < n; i += stride) {
    oh[i] = hosts[i];
    oe[i] = est[i];
    of[i] = flags[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence_system();  // this block's writes (and, via the barrier, its threads') first
    if (atomicAdd(&sc->report_blocks, 1u) == gridDim.x - 1) {
      __threadfence_system();
      *reinterpret_cast<volatile uint32_t*>(out + offsetof(CloseScratch, report_done)) = 1u;
    }
  }
}

// Join for delta <= 5, tiled over (HSE(1) x HSE(0)): each thread keeps one he_1 in registers
// and probes it against a chunk of HSE(0) staged in shared memory. With
// g_1 = (he_1 >> delta) mod 2^(q-delta) and K(he_0) = (he_0 XOR (he_0 >> delta)) mod 2^(q-delta),
// the low bits c of every admissible B(2) XOR he_0 are K(he_0) XOR g_1 (Eq. 7 and the overlap
// of B(1) and B(2)), so a probe is one XOR and one bit of row 2's "any hot" bitmap (some of
// the 2^delta SREs with low bits c is hot). Probes run 16 he_0 at a time; the (lane, he_0)
// pairs that hit are pushed on a per-warp stack (warp prefix sum), and whenever 32 wait, every
// lane expands one: the hot SREs of the group come from the regrouped row-2 table, and each
// chain must pass row 3's "any hot" bit before it is queued. Each warp works as a pipeline of
// stages, all 32 lanes in every stage: expanded chains go to the warp's partial-chain queue;
// whenever 32 wait, each lane walks one chain's row-3 hot SREs (a warp-uniform loop) and
// queues every B(3) whose row-4 group holds a hot SRE; whenever 32 of those wait, each lane
// walks one's row-4 hot SREs into the warp's complete-chain queue; whenever 32 complete
// chains wait, each lane regains the hosts of one. So the divergent depth-first walk of a lone
// lane never runs, a loop waits only for the lane with the most hot SREs of one row, and
// the regain search, a large part of the work when hot SREs are common, runs on full warps. The
// two "any hot" bitmaps are staged in shared memory when `stage` is set; the blocks are small
// (kJoinTiledThreads) so that several share an SM.
constexpr int kJoinTiledThreads = 256;
constexpr uint32_t kJoinWarpQueue = 64;    // entries of each per-warp chain queue (< 32 waiting + 32 pushed)
constexpr uint32_t kJoinQueueWords = 9;    // words per entry over a warp's three queues (3 + 4 + 2)
constexpr uint32_t kJoinChunkMax = 256;    // he_0 per work unit
constexpr uint32_t kJoinProbeBlock = 16;   // he_0 probed before a compaction
constexpr uint32_t kJoinListWords = (32 + 32 * kJoinProbeBlock) / 2;  // per warp hit stack: 16-bit entries
// dynamic shared memory after the optional bitmaps: per-warp chain queues (partial: 3 words,
// waiting for row 4: 4 words, complete: 2 words per entry), he_0 chunk, K chunk, he_1, hit
// stacks
constexpr size_t kJoinTiledFixedBytes =
    ((kJoinTiledThreads / 32) * kJoinQueueWords * (size_t)kJoinWarpQueue + 2 * kJoinChunkMax + kJoinTiledThreads +
     (kJoinTiledThreads / 32) * kJoinListWords) * 4;

// Words of an "any hot" bitmap over the 2^(q-delta) values of c, and the shared-memory words
// that hold one (a multiple of 4, so that what follows stays 16-byte aligned).
__host__ __device__ __forceinline__ uint32_t any_words(uint32_t q, uint32_t delta) {
  const uint32_t w = (1u << (q - delta)) >> 5;
  return w ? w : 1u;
}
__host__ __device__ __forceinline__ uint32_t any_words_staged(uint32_t q, uint32_t delta) {
  return (any_words(q, delta) + 3u) & ~3u;
}

// STAGE: both "any hot" bitmaps are copied to shared memory first, so that the probes are
// shared-memory loads with 32-bit addresses (else they read the global bitmaps).
template <bool STAGE>
__global__ void __launch_bounds__(kJoinTiledThreads) k_join_tiled(
    const __grid_constant__ KParams p, const uint32_t* __restrict__ tables, const uint32_t* __restrict__ any2,
    const uint32_t* __restrict__ any3, const uint32_t* __restrict__ list0, const uint32_t* __restrict__ list1,
    const uint32_t* __restrict__ n_list, uint32_t* __restrict__ cand, uint32_t* __restrict__ n_cand, uint32_t cap,
    uint32_t* __restrict__ overflow) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ uint32_t sm[];
  const uint32_t n0 = n_list[0], n1 = n_list[1];
  if (n0 == 0 || n1 == 0) return;
  const uint32_t delta = p.delta, q = p.q;
  const uint32_t shift_hi = q - delta;
  const uint32_t cmask = (1u << shift_hi) - 1u;
  const uint32_t span_mask = delta == 5 ? 0xFFFFFFFFu : (1u << (1u << delta)) - 1u;
  const bool row2_fits_all = 2 * delta + q <= 32;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  // shared memory: [any2] [any3] [queue: he0 | b1 | b2] [he_0 chunk] [K chunk] [he_1] [lists]
  const uint32_t aw = any_words(q, delta);
  const uint32_t* a2 = any2;
  const uint32_t* a3 = any3;
  uint32_t* next = sm;
  if constexpr (STAGE) {
    // both bitmaps with 16-byte loads, all of a thread's loads issued before its stores
    // (the word counts are multiples of 4 from 2^(q-delta) >= 128; smaller ones word by word)
    uint32_t* d2 = next;
    uint32_t* d3 = next + any_words_staged(q, delta);
    if ((aw & 3u) == 0) {
      const uint32_t n4 = aw >> 2;
      for (uint32_t w0 = threadIdx.x; w0 < n4; w0 += 2 * blockDim.x) {
        uint4 v2[2], v3[2];
#pragma unroll
        for (uint32_t u = 0; u < 2; ++u) {
          const uint32_t w = w0 + u * blockDim.x;
          if (w < n4) {
            v2[u] = reinterpret_cast<const uint4*>(any2)[w];
            if (any3) v3[u] = reinterpret_cast<const uint4*>(any3)[w];
          }
        }
#pragma unroll
        for (uint32_t u = 0; u < 2; ++u) {
          const uint32_t w = w0 + u * blockDim.x;
          if (w < n4) {
            reinterpret_cast<uint4*>(d2)[w] = v2[u];
            if (any3) reinterpret_cast<uint4*>(d3)[w] = v3[u];
          }
        }
      }
    } else {
      for (uint32_t w = threadIdx.x; w < aw; w += blockDim.x) {
        d2[w] = any2[w];
        if (any3) d3[w] = any3[w];
      }
    }
    a2 = d2;
    if (any3) a3 = d3;
    next = d3 + any_words_staged(q, delta);
  }
  // per-warp queues of kJoinWarpQueue entries: partial chains (he_0, B(1), B(2)), chains
  // waiting for row 4 (he_0, address bits so far, B(3), row 4's hot SREs) and complete
  // chains (he_0, address bits [delta, 32))
  uint32_t* wq_he0 = next + warp * (kJoinQueueWords * kJoinWarpQueue);
  uint32_t* wq_b1 = wq_he0 + kJoinWarpQueue;
  uint32_t* wq_b2 = wq_b1 + kJoinWarpQueue;
  uint32_t* wf_he0 = wq_b2 + kJoinWarpQueue;
  uint32_t* wf_high = wf_he0 + kJoinWarpQueue;
  uint32_t* wf_b3 = wf_high + kJoinWarpQueue;
  uint32_t* wf_m4 = wf_b3 + kJoinWarpQueue;
  uint32_t* wc_he0 = wf_m4 + kJoinWarpQueue;
  uint32_t* wc_high = wc_he0 + kJoinWarpQueue;
  uint32_t* s_he0 = next + (kJoinTiledThreads / 32) * (kJoinQueueWords * kJoinWarpQueue);
  uint32_t* s_k = s_he0 + kJoinChunkMax;
  uint32_t* s_he1 = s_k + kJoinChunkMax;
  uint16_t* my_list = reinterpret_cast<uint16_t*>(s_he1 + kJoinTiledThreads) + warp * (2 * kJoinListWords);
  static_assert(kJoinChunkMax <= 256, "hit entries hold 8-bit chunk indices");
  // the sorted a*low table of regain (multiply-add-shift RHFG[0]; first used after the
  // barrier that opens every work unit)
  __shared__ RegainTable s_rt;
  if (!p.tab) build_regain_table(p, &s_rt);
  const RegainTable* rt = p.tab ? nullptr : &s_rt;

  // Work rows (tile of HSE(1), he_0), tile-major, split evenly over the blocks; a block's
  // range is cut into units of at most kJoinChunkMax he_0 of one tile.
  const uint32_t tiles1 = (n1 + blockDim.x - 1) / blockDim.x;
  const uint32_t width1 = (n1 + tiles1 - 1) / tiles1;
  const uint64_t rows = (uint64_t)tiles1 * n0;
  const uint64_t r_begin = rows * blockIdx.x / gridDim.x, r_end = rows * (blockIdx.x + 1) / gridDim.x;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint64_t nwords = (1ull << q) >> 5;

  // Every stage below is entered by all 32 lanes of the warp together, each lane holding
  // one item or none (`ok`), and loops while any lane has work; items flow to the next stage
  // through the warp's queues, which hand the next stage 32 at a time.
  uint32_t cn = 0;  // complete chains queued (the same in every lane)
  // Regain (Eq. 7 plus the delta low bits): one complete chain per lane.
  auto push_complete = [&](bool ok, uint32_t he0, uint32_t high) {
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, ok);
    if (ok) {
      const uint32_t at = cn + __popc(b & lt_mask);
      wc_he0[at] = he0;
      wc_high[at] = high;
    }
    cn += __popc(b);
    if (cn >= 32) {
      cn -= 32;
      __syncwarp();
      const uint32_t e0 = wc_he0[cn + lane], eh = wc_high[cn + lane];
      __syncwarp();
      regain_high(p, e0, eh, cand, n_cand, cap, overflow, rt);
    }
  };
  // Row 4 (Algorithm 5, r = 5): one chain (he_0, address bits so far, B(3), row 4's hot
  // SREs of its group) per lane; every hot SRE that keeps B(4) inside 32 address bits
  // completes the chain.
  auto grow4 = [&](bool ok, uint32_t he0, uint32_t high123, uint32_t b3, uint32_t m4) {
    const uint32_t hi0 = he0 >> shift_hi;
    if (!ok) m4 = 0;
    while (__any_sync(0xFFFFFFFFu, m4 != 0u)) {
      bool done = false;
      uint32_t high = 0;
      if (m4) {
        const uint32_t b4 = (b3 >> delta) | (((uint32_t)(__ffs(m4) - 1) ^ hi0) << shift_hi);
        m4 &= m4 - 1u;
        // with B(4) inside 32 address bits (fits32), bits [delta, 32) hold the whole chain
        done = fits32(4, delta, q, b4);
        high = (uint32_t)((uint64_t)high123 | ((uint64_t)(b4 >> shift_hi) << (4 * delta + shift_hi)));
      }
      push_complete(done, he0, high);
    }
  };
  uint32_t fn = 0;  // chains waiting for row 4 (the same in every lane)
  auto push_four = [&](bool ok, uint32_t he0, uint32_t high123, uint32_t b3, uint32_t m4) {
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, ok);
    if (ok) {
      const uint32_t at = fn + __popc(b & lt_mask);
      wf_he0[at] = he0;
      wf_high[at] = high123;
      wf_b3[at] = b3;
      wf_m4[at] = m4;
    }
    fn += __popc(b);
    if (fn >= 32) {
      fn -= 32;
      __syncwarp();
      const uint32_t e0 = wf_he0[fn + lane], eh = wf_high[fn + lane], e3 = wf_b3[fn + lane], em = wf_m4[fn + lane];
      __syncwarp();
      grow4(true, e0, eh, e3, em);
    }
  };
  // Rows 3 .. r-1 of a chain (Algorithm 5). For r = 5, row 3's hot SREs are walked one per
  // lane and every B(3) whose row-4 group holds a hot SRE is queued for row 4, so that each
  // stage loops over one row's hot SREs only; other r grow their chains lane by lane (depth
  // first, regaining inline).
  auto grow = [&](bool ok, uint32_t he0, uint32_t b1, uint32_t b2) {
    if (p.r != 5) {
      if (ok) grow_chain(p, tables, he0, b1, b2, cand, n_cand, cap, overflow, rt);
      return;
    }
    const uint32_t hi0 = he0 >> shift_hi;
    const uint64_t high12 = ((uint64_t)b1 << delta) | ((uint64_t)(b2 >> shift_hi) << (2 * delta + shift_hi));
    uint32_t m3 = ok ? hot_group(tables + nwords, (he0 ^ (b2 >> delta)) & cmask, delta) & fits32_tops(3, delta, q, hi0)
                     : 0u;
    const uint32_t tops4 = fits32_tops(4, delta, q, hi0);
    while (__any_sync(0xFFFFFFFFu, m3 != 0u)) {
      uint32_t m4 = 0, b3 = 0;
      if (m3) {
        b3 = (b2 >> delta) | (((uint32_t)(__ffs(m3) - 1) ^ hi0) << shift_hi);
        m3 &= m3 - 1u;
        if (fits32(3, delta, q, b3))
          m4 = hot_group(tables + 2 * nwords, (he0 ^ (b3 >> delta)) & cmask, delta) & tops4;
      }
      // with B(3) inside 32 address bits, so are the bits fixed so far
      const uint32_t high123 = (uint32_t)(high12 | ((uint64_t)(b3 >> shift_hi) << (3 * delta + shift_hi)));
      push_four(m4 != 0u, he0, high123, b3, m4);
    }
  };
  uint32_t pn = 0;  // partial chains queued (the same in every lane)
  auto push_partial = [&](bool ok, uint32_t he0, uint32_t b1, uint32_t b2) {
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, ok);
    if (ok) {
      const uint32_t at = pn + __popc(b & lt_mask);
      wq_he0[at] = he0;
      wq_b1[at] = b1;
      wq_b2[at] = b2;
    }
    pn += __popc(b);
    if (pn >= 32) {
      pn -= 32;
      __syncwarp();
      const uint32_t e0 = wq_he0[pn + lane], e1 = wq_b1[pn + lane], e2 = wq_b2[pn + lane];
      __syncwarp();
      grow(true, e0, e1, e2);
    }
  };
  // One hit (he_0, he_1) per lane: every hot row-2 SRE of the group gives B(2); chains whose
  // row-3 group has a hot SRE are queued.
  auto expand = [&](bool ok, uint32_t e) {
    uint32_t he0 = 0, b1 = 0, m = 0;
    if (ok) {
      he0 = s_he0[e & 255u];
      b1 = he0 ^ s_he1[warp * 32 + (e >> 8)];
    }
    const uint32_t low2 = b1 >> delta;
    const uint32_t hi0 = he0 >> shift_hi;
    if (ok && fits32(1, delta, q, b1)) {
      const uint32_t first = ((he0 ^ low2) & cmask) << delta;  // row-2 group of c
      m = (tables[first >> 5] >> (first & 31)) & span_mask & fits32_tops(2, delta, q, hi0);
    }
    while (__any_sync(0xFFFFFFFFu, m != 0u)) {
      bool keep = false;
      uint32_t b2 = 0;
      if (m) {
        const uint32_t tp = __ffs(m) - 1;  // top bits of he_2
        m &= m - 1;
        b2 = low2 | ((tp ^ hi0) << shift_hi);
        keep = row2_fits_all || fits32(2, delta, q, b2);
        if (keep && a3) {
          const uint32_t c3 = (he0 ^ (b2 >> delta)) & cmask;
          keep = (a3[c3 >> 5] >> (c3 & 31)) & 1u;
        }
      }
      push_partial(keep, he0, b1, b2);
    }
  };
  uint32_t hn = 0;  // entries on this warp's hit stack (the same in every lane)

  for (uint64_t r0 = r_begin; r0 < r_end;) {
    const uint32_t tile = (uint32_t)(r0 / n0), c0 = (uint32_t)(r0 % n0);
    uint64_t mm = n0 - c0;  // he_0 left in this tile
    if (mm > kJoinChunkMax) mm = kJoinChunkMax;
    if (mm > r_end - r0) mm = r_end - r0;
    const uint32_t m0 = (uint32_t)mm;
    r0 += m0;
    __syncthreads();  // previous unit's chunk is done with
    for (uint32_t j = threadIdx.x; j < ((m0 + kJoinProbeBlock - 1) & ~(kJoinProbeBlock - 1)); j += blockDim.x) {
      if (j < m0) {
        const uint32_t he0 = list0[c0 + j];
        s_he0[j] = he0;
        s_k[j] = ((he0 ^ (he0 >> delta)) & cmask) ^ 31u;  // K(he_0) with its 5 low bits flipped
      } else {
        s_k[j] = 0;  // the probe block's padding: an in-range c, masked off after the probes
      }
    }
    const uint32_t b = tile * width1 + threadIdx.x;
    const bool valid = threadIdx.x < width1 && b < n1;
    const uint32_t he1 = valid ? list1[b] : 0u;
    const uint32_t g1 = (he1 >> delta) & cmask;
    s_he1[threadIdx.x] = he1;
    __syncthreads();
    for (uint32_t j0 = 0; j0 < m0; j0 += kJoinProbeBlock) {  // uniform over the block
      const uint32_t jn = min(kJoinProbeBlock, m0 - j0);
      uint32_t hits = 0;
      if (valid) {
        // 16 probes from four broadcast vector loads; entries past the chunk (inside the
        // kJoinChunkMax-entry array, which is a multiple of 16) are masked off below.
        // With c' = c ^ 31 the word is c' >> 5 and rotating it left by c' (mod 32) brings bit
        // c mod 32 to the top; the bits are gathered first probe highest, then reversed.
        const uint4* k4 = reinterpret_cast<const uint4*>(s_k + j0);
#pragma unroll
        for (uint32_t v = 0; v < kJoinProbeBlock / 4; ++v) {
          const uint4 kk = k4[v];
          const uint32_t c[4] = {kk.x ^ g1, kk.y ^ g1, kk.z ^ g1, kk.w ^ g1};
#pragma unroll
          for (uint32_t u = 0; u < 4; ++u) {
            const uint32_t x = a2[c[u] >> 5];
            // (hits << 1) | top bit of the rotated word, as one funnel shift
            hits = __funnelshift_l(__funnelshift_l(x, x, c[u]), hits, 1);
          }
        }
        hits = __brev(hits) >> (32 - kJoinProbeBlock);
        if (jn < kJoinProbeBlock) hits &= (1u << jn) - 1u;
      }
      // append this warp's hits to its hit stack (exclusive prefix sum of the per-lane
      // counts); each entry is (lane << 8) | index of he_0 in the chunk
      const uint32_t cnt = __popc(hits);
      uint32_t incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= (uint32_t)o) incl += v;
      }
      const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
      uint32_t at = hn + incl - cnt;
      while (hits) {
        const uint32_t j = __ffs(hits) - 1;
        hits &= hits - 1;
        my_list[at++] = (uint16_t)((lane << 8) | (j0 + j));
      }
      hn += total;
      __syncwarp();
      while (hn >= 32) {  // every lane expands one hit, from the top of the stack
        hn -= 32;
        expand(true, my_list[hn + lane]);
        __syncwarp();  // those entries are overwritten by the next append
      }
    }
    // the rest of the hits, before the chunk is replaced (the chain queues carry over)
    expand(lane < hn, lane < hn ? my_list[lane] : 0u);
    hn = 0;
    __syncwarp();
  }
  // the chains still queued: partial ones grown, then those waiting for row 4, then the
  // complete ones regained
  grow(lane < pn, wq_he0[lane], wq_b1[lane], wq_b2[lane]);
  pn = 0;
  __syncwarp();
  grow4(lane < fn, wf_he0[lane], wf_high[lane], wf_b3[lane], wf_m4[lane]);
  fn = 0;
  __syncwarp();
  if (lane < cn) regain_high(p, wc_he0[lane], wc_high[lane], cand, n_cand, cap, overflow, rt);
}

// Join from the top row down, for r = R (4..6), delta <= 5 and s = 32 - (R-1)*delta with
// 5 <= s < q. B(R-1) = aip >> (R-1)*delta has only s bits inside a 32-bit address, so
// he_{R-1} = he_0 XOR B(R-1) agrees with he_0 above bit s: the hot SREs of row R-1 that can
// share a host with he_0 are those of he_0's column block of 2^s (listed by k_hot_prep).
// Each such pair fixes address bits [(R-1)*delta, 32). Then every row L = R-2 .. 1 adds bits
// [L*delta, (L+1)*delta): B(L)'s upper q-delta bits repeat B(L+1)'s lower ones (the overlap
// of Algorithm 5), so he_L's upper q-delta bits are known, and its delta low bits are the
// set bits of one 2^delta-bit group of row L's hot bitmap. A chain through row 1 fixes bits
// [delta, 32) and is regained as in the join from row 0 up (Eq. 7). The chains are those of
// Algorithms 4-5 that stay inside 32 address bits, found from the other end: the top row's
// 2^(q-s) blocks cut the pairs to start from by that factor against HSE(0) x HSE(1).
// Every stage runs on whole warps: each lane holds one chain, and the children of a row
// wait in the warp's queue for that row until 32 are there.
constexpr int kJoinDownThreads = 256;
constexpr uint32_t kJoinDownQueue = 64;   // entries per queue (< 32 waiting + 32 pushed)
constexpr uint32_t kJoinDownUnroll = 4;   // row R-1 entries per lane in flight

template <int R>
struct DownWalk {
  const KParams& p;
  const uint32_t* hot;   // hot bitmaps of all rows
  uint32_t* qs;          // this warp's queues: level L holds he_0 [kJoinDownQueue], then bits
  uint32_t cnt[R - 2];   // entries waiting at level L (the same in every lane); level 0: complete
  uint32_t delta, qbits, gmask, span_mask, lane, lt_mask;
  uint32_t* cand;
  uint32_t* n_cand;
  uint32_t cap;
  uint32_t* overflow;
  const RegainTable* rt;

  __device__ __forceinline__ DownWalk(const KParams& p_, const uint32_t* hot_, uint32_t* qs_, uint32_t lane_,
                                      uint32_t* cand_, uint32_t* n_cand_, uint32_t cap_, uint32_t* overflow_,
                                      const RegainTable* rt_)
      : p(p_), hot(hot_), qs(qs_), delta(p_.delta), qbits(p_.q), gmask((1u << (p_.q - p_.delta)) - 1u),
        span_mask(p_.delta == 5 ? 0xFFFFFFFFu : (1u << (1u << p_.delta)) - 1u), lane(lane_),
        lt_mask((1u << lane_) - 1u), cand(cand_), n_cand(n_cand_), cap(cap_), overflow(overflow_), rt(rt_) {
#pragma unroll
    for (int L = 0; L < R - 2; ++L) cnt[L] = 0;
  }

  // Row L's hot flags for the chain (he_0, bits [(L+1)*delta, 32) of the address): the
  // 2^delta SREs whose upper q-delta bits are those of he_0 XOR B(L), adjacent in the bitmap.
  template <int L>
  __device__ __forceinline__ uint32_t group(uint32_t he0, uint32_t a) const {
    const uint32_t first = (((he0 >> delta) ^ (a >> ((L + 1) * delta))) & gmask) << delta;
    return (__ldg(hot + ((uint64_t)L << (qbits - 5)) + (first >> 5)) >> (first & 31)) & span_mask;
  }

  // Every hot SRE t of row L's group (m) extends the chain by bits [L*delta, (L+1)*delta):
  // the low delta bits of B(L) = he_0 XOR he_L are t XOR the low delta bits of he_0.
  template <int L>
  __device__ __forceinline__ void walk(uint32_t m, uint32_t he0, uint32_t a) {
    const uint32_t xl = he0 & ((1u << delta) - 1u);
    while (__any_sync(0xFFFFFFFFu, m != 0u)) {
      const bool has = m != 0u;
      uint32_t child = 0;
      if (has) {
        const uint32_t t = (uint32_t)(__ffs(m) - 1);
        m &= m - 1u;
        child = a | ((t ^ xl) << (L * delta));
      }
      push<L - 1>(has, he0, child);
    }
  }

  // Queue a chain for row L (L >= 1) or, at L = 0, a complete chain for regain; whenever
  // 32 wait, every lane takes one.
  template <int L>
  __device__ __forceinline__ void push(bool ok, uint32_t he0, uint32_t a) {
    uint32_t* qh = qs + L * 2 * kJoinDownQueue;
    uint32_t* qa = qh + kJoinDownQueue;
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, ok);
    if (ok) {
      const uint32_t at = cnt[L] + __popc(b & lt_mask);
      qh[at] = he0;
      qa[at] = a;
    }
    cnt[L] += __popc(b);
    if (cnt[L] >= 32) {
      cnt[L] -= 32;
      __syncwarp();
      const uint32_t e0 = qh[cnt[L] + lane], ea = qa[cnt[L] + lane];
      __syncwarp();  // those entries are overwritten by the next push
      if constexpr (L == 0)
        regain_high(p, e0, ea, cand, n_cand, cap, overflow, rt);
      else
        walk<L>(group<L>(e0, ea), e0, ea);
    }
  }

  // The chains still queued at level L and below, the highest level first.
  template <int L>
  __device__ __forceinline__ void flush() {
    uint32_t* qh = qs + L * 2 * kJoinDownQueue;
    const bool ok = lane < cnt[L];
    const uint32_t e0 = ok ? qh[lane] : 0u, ea = ok ? qh[kJoinDownQueue + lane] : 0u;
    cnt[L] = 0;
    __syncwarp();
    if constexpr (L == 0) {
      if (ok) regain_high(p, e0, ea, cand, n_cand, cap, overflow, rt);
    } else {
      walk<L>(ok ? group<L>(e0, ea) : 0u, e0, ea);
      flush<L - 1>();
    }
  }
};

// One warp per he_0 of HSE(0) (list0, striding over the grid's warps); its lanes take the
// row R-1 hot SREs of he_0's block, kJoinDownUnroll each at a time.
template <int R>
__global__ void __launch_bounds__(kJoinDownThreads) k_join_down(
    const __grid_constant__ KParams p, const uint32_t* __restrict__ hot_bits, const uint32_t* __restrict__ list0,
    const uint32_t* __restrict__ n_list, const uint32_t* __restrict__ blist, const uint32_t* __restrict__ bcount,
    uint32_t* __restrict__ cand, uint32_t* __restrict__ n_cand, uint32_t cap, uint32_t* __restrict__ overflow,
    unsigned long long* __restrict__ n_pairs) {
  pdl_wait();
  pdl_trigger();
  static_assert(R >= 4 && R <= 6, "rows");
  __shared__ uint32_t s_queue[kJoinDownThreads / 32][(R - 2) * 2 * kJoinDownQueue];
  __shared__ RegainTable s_rt;
  if (!p.tab) build_regain_table(p, &s_rt);
  __syncthreads();
  const uint32_t n0 = n_list[0];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  DownWalk<R> w(p, hot_bits, s_queue[warp], lane, cand, n_cand, cap, overflow, p.tab ? nullptr : &s_rt);
  const uint32_t top = (R - 1) * p.delta;  // B(R-1) is address bits [top, 32)
  const uint32_t s = 32u - top;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  uint64_t pairs = 0;
  for (uint32_t i = blockIdx.x * (blockDim.x >> 5) + warp; i < n0; i += warps) {
    const uint32_t he0 = list0[i];
    const uint32_t b = he0 >> s;
    const uint32_t n4 = bcount[b];
    const uint32_t* l4 = blist + ((uint64_t)b << s);
    pairs += n4;
    for (uint32_t k0 = 0; k0 < n4; k0 += 32 * kJoinDownUnroll) {  // uniform over the warp
      uint32_t a[kJoinDownUnroll], m[kJoinDownUnroll];
#pragma unroll
      for (uint32_t u = 0; u < kJoinDownUnroll; ++u) {
        const uint32_t k = k0 + u * 32 + lane;
        a[u] = k < n4 ? (he0 ^ l4[k]) << top : 0u;
      }
#pragma unroll
      for (uint32_t u = 0; u < kJoinDownUnroll; ++u)
        m[u] = k0 + u * 32 + lane < n4 ? w.template group<R - 2>(he0, a[u]) : 0u;
#pragma unroll
      for (uint32_t u = 0; u < kJoinDownUnroll; ++u) w.template walk<R - 2>(m[u], he0, a[u]);
    }
  }
  w.template flush<R - 3>();
  if (lane == 0 && pairs) atomicAdd(n_pairs, (unsigned long long)pairs);
}

// ---------------------------------------------------------------- ordering
// The report lists the candidates in ascending order. One cooperative launch of kSortBlocks
// blocks (all resident at once) sorts them:
// * up to kSortChunk keys (the usual report): each key is placed at its rank, the number of
//   smaller keys (ties, which a candidate set does not have, are broken by index); every
//   block reads all keys into shared memory and kRankSplit neighbouring threads count one
//   key's rank over interleaved parts of the keys, adding their counts with shuffles. With
//   small_by_estimate set the launch leaves these to k_estimate, whose block for a host
//   counts that host's rank while it gathers the SLEs, and returns at once;
// * more: every kSortChunk-key chunk is sorted in shared memory (bitonic network, tail
//   padded with 0xFFFFFFFF, which sorts last), then sorted runs are merged pairwise (each key
//   placed by a binary search in the partner run), pass after pass, with a grid-wide
//   barrier between passes; the last pass writes `out`.
constexpr int kSortThreads = 256;
constexpr uint32_t kRankSplit = 8;
constexpr uint32_t kSortBlocks = kSortChunk / (kSortThreads / kRankSplit);  // 128
constexpr uint32_t kBarrierSpins = 1u << 22;  // polls (64 ns apart) before a barrier gives up

// Grid-wide barrier of a cooperative launch. bar[0] counts arrivals, bar[1] is the
// generation; both are zero before the launch (the close's scratch is cleared). The block
// whose arrival is number `last` (gridDim.x - 1 normally) releases the others. A wait that
// outlasts `spins` polls sets *error and returns false; the caller then returns.
__device__ __forceinline__ bool grid_barrier(uint32_t* bar, uint32_t* error, uint32_t spins_max, uint32_t last) {
  __shared__ uint32_t ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile uint32_t* gen = bar + 1;
    const uint32_t g = *gen;  // this barrier's generation: it cannot move before we arrive
    ok = 1u;
    __threadfence();
    if (atomicAdd(bar, 1u) == last) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      uint32_t spins = 0;
      while (*gen == g) {
        if (++spins > spins_max) {
          atomicOr(error, 1u);
          ok = 0u;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0u;
}

// keys: the n = min(*n_ptr, cap) unsorted candidates (reordered in place when n > kSortChunk);
// alt: a second buffer of cap entries; out: the sorted candidates. bar: two zeroed words.
// ctl (may be NULL): ctl[0] the barrier's poll limit (0: kBarrierSpins), ctl[1] arrivals the
// barrier waits for beyond the grid's blocks (0; a failure-detection test sets 1, so that
// every barrier wait runs out and the launch reports the timeout in *error).
__global__ void __launch_bounds__(kSortThreads) k_sort_candidates(uint32_t* __restrict__ keys,
                                                                  uint32_t* __restrict__ alt,
                                                                  uint32_t* __restrict__ out,
                                                                  const uint32_t* __restrict__ n_ptr, uint32_t cap,
                                                                  uint32_t* __restrict__ bar,
                                                                  uint32_t* __restrict__ error,
                                                                  uint32_t small_by_estimate,
                                                                  const uint32_t* __restrict__ ctl) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t s[kSortChunk];
  const uint32_t n = min(*n_ptr, cap);
  if (n <= kSortChunk) {
    if (small_by_estimate) return;
    const uint32_t per_block = kSortThreads / kRankSplit;
    if (blockIdx.x * per_block >= n) return;
    for (uint32_t x = threadIdx.x; x < n; x += blockDim.x) s[x] = keys[x];
    __syncthreads();
    const uint32_t i = blockIdx.x * per_block + threadIdx.x / kRankSplit;
    const uint32_t part = threadIdx.x % kRankSplit;
    const uint32_t v = i < n ? s[i] : 0u;
    uint32_t rank = 0;
    if (i < n)
      for (uint32_t y = part; y < n; y += kRankSplit) rank += (s[y] < v || (s[y] == v && y < i)) ? 1u : 0u;
#pragma unroll
    for (uint32_t o = kRankSplit / 2; o > 0; o >>= 1) rank += __shfl_xor_sync(0xFFFFFFFFu, rank, o);
    if (i < n && part == 0) out[rank] = v;
    return;
  }
  // chunk sorts (keys written back in place)
  const uint32_t chunks = (n + kSortChunk - 1) / kSortChunk;
  for (uint32_t c = blockIdx.x; c < chunks; c += gridDim.x) {
    const uint32_t start = c * kSortChunk;
    const uint32_t m = min(n - start, (uint32_t)kSortChunk);
    for (uint32_t x = threadIdx.x; x < kSortChunk; x += blockDim.x) s[x] = x < m ? __ldcg(keys + start + x) : 0xFFFFFFFFu;
    __syncthreads();
    for (uint32_t size = 2; size <= kSortChunk; size <<= 1) {
      for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
        for (uint32_t x = threadIdx.x; x < kSortChunk / 2; x += blockDim.x) {
          const uint32_t lo = 2 * x - (x & (stride - 1));
          const uint32_t hi = lo + stride;
          const bool up = (lo & size) == 0;
          const uint32_t a = s[lo], b = s[hi];
          if ((a > b) == up) {
            s[lo] = b;
            s[hi] = a;
          }
        }
        __syncthreads();
      }
    }
    for (uint32_t x = threadIdx.x; x < m; x += blockDim.x) keys[start + x] = s[x];
    __syncthreads();  // s is refilled by the next chunk
  }
  // merge passes: runs of `width` pairwise, keys -> alt -> keys ... -> out (reads bypass L1,
  // which other blocks' writes do not update)
  const uint32_t spins = ctl && ctl[0] ? ctl[0] : kBarrierSpins;
  const uint32_t last = gridDim.x - 1 + (ctl ? ctl[1] : 0u);
  const uint32_t* src = keys;
  for (uint64_t width = kSortChunk; width < n; width *= 2) {
    if (!grid_barrier(bar, error, spins, last)) return;
    uint32_t* dst = 2 * width >= n ? out : (src == keys ? alt : keys);
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
      const uint64_t pair_start = (x / (2 * width)) * (2 * width);
      const uint64_t mid = pair_start + width < n ? pair_start + width : n;
      const uint64_t end = pair_start + 2 * width < n ? pair_start + 2 * width : n;
      const uint32_t v = __ldcg(src + x);
      uint64_t lo, hi, pos;
      if (x < mid) {  // left run: count right-run keys < v
        lo = mid;
        hi = end;
        while (lo < hi) {
          const uint64_t md = (lo + hi) >> 1;
          if (__ldcg(src + md) < v) lo = md + 1; else hi = md;
        }
        pos = x + (lo - mid);
      } else {  // right run: count left-run keys <= v
        lo = pair_start;
        hi = mid;
        while (lo < hi) {
          const uint64_t md = (lo + hi) >> 1;
          if (__ldcg(src + md) <= v) lo = md + 1; else hi = md;
        }
        pos = pair_start + (x - mid) + (lo - pair_start);
      }
      dst[pos] = v;
    }
    src = dst;
  }
}

// ---------------------------------------------------------------- estimation
constexpr int kEstThreads = 128;      // threads per host, for SLE rows below 16 KiB
constexpr int kEstThreadsWide = 512;  // for rows of 16 KiB and more (the launch bound below)

// Threads per host of k_estimate: a host's r' rows are gathered in rounds of one 16-byte
// vector per thread and row, so wide rows (eta' cells of 2 bytes at the paper's
// eta' = 2^14: 32 KiB) take 4 rounds at 512 threads where they would take 16 at 128.
__host__ __device__ __forceinline__ int est_threads(uint32_t eta2, uint32_t cell_bytes) {
  return (uint64_t)eta2 * cell_bytes >= 16384u ? kEstThreadsWide : kEstThreads;
}

// One CTA per host (grid-stride). hosts: n_ptr ? min(*n_ptr, n) hosts : n hosts. active2:
// active cells per SLEA row. Outputs (any may be NULL except est): est, flags, w (FP64
// corrected weight), U, hist[n][k]. vec16: every SLE starts on a 16-byte boundary
// (delta' % 16 == 0), so cells are gathered 16 at a time.
// Distance of a stamp from the current stamp cs, or kInactive<St> when unset or outside the
// window (8-bit stamps: a 256-entry table with 255 for inactive, windows being at most 254
// slices; 16-bit stamps: computed, mod 65535). The sentinel exceeds every active distance,
// so the largest distance over a host's rows is inactive as soon as one row is.
template <typename St>
constexpr uint32_t kInactive = sizeof(St) == 1 ? 255u : 0xFFFFFFFFu;

template <typename St>
__device__ __forceinline__ uint32_t cell_age(uint32_t s, const uint8_t* age_lut, uint32_t cs, uint32_t k) {
  if constexpr (sizeof(St) == 1) {
    return age_lut[s];
  } else {
    const uint32_t age = cs >= s ? cs - s : cs + 65535u - s;
    return (s != 0 && age < k) ? age : kInactive<St>;
  }
}

// ACT: U from the close pass's activity bitmap (sle_act), the close's own estimate;
// otherwise from the stamps (queries, features, histograms).
template <typename St, bool ACT = false>
__global__ void __launch_bounds__(kEstThreadsWide, ACT ? 2 : 1) k_estimate(
    const __grid_constant__ KParams p, const uint8_t* __restrict__ sle_bytes, const uint32_t* __restrict__ hosts,
    const uint32_t* __restrict__ n_ptr, uint32_t n, const uint32_t* __restrict__ active2, EstTable tab,
    const uint32_t* __restrict__ unsorted, uint32_t* __restrict__ hosts_out, double w_theta,
    uint32_t cs_value, const uint32_t* __restrict__ clock, float* __restrict__ est, uint8_t* __restrict__ flags,
    double* __restrict__ w_out,
    uint32_t* __restrict__ u_out, uint32_t* __restrict__ hist, uint32_t* __restrict__ n_super,
    const uint32_t* __restrict__ sle_act) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint8_t age_lut[256];
  __shared__ uint32_t sh_hist[256];
  __shared__ uint32_t warp_u[kEstThreadsWide / 32];
  __shared__ const St* row_base[kMaxRows];
  __shared__ uint64_t row_cell[kMaxRows];  // the host's SLE start in each row, as an SLEA cell index
  const St* sle = reinterpret_cast<const St*>(sle_bytes);
  // the count, the stamp and the first host are loaded together (the grid is never larger
  // than the host buffers, so index blockIdx.x is in bounds even past the count)
  const uint32_t first_aip = (unsorted ? unsorted : hosts)[blockIdx.x];
  const uint32_t count = n_ptr ? min(*n_ptr, n) : n;
  const uint32_t cs = clock ? *clock : cs_value;
  if (blockIdx.x >= count) return;  // the grid is sized for the capacity
  // rank mode (unsorted given, at most kSortChunk hosts): the hosts come unsorted, and the
  // outputs of each go to its rank in ascending order (the number of smaller hosts; ties,
  // which a candidate set does not have, broken by index), hosts_out included; otherwise
  // `hosts` is already sorted and the outputs go to the host's own index
  const bool rank_mode = unsorted != nullptr && count <= kSortChunk && hist == nullptr;
  const bool vec16 = (p.delta2 & 15u) == 0;
  // U alone: from the close pass's activity bitmap when given, else from byte-wise or
  // half-word-wise activity masks of the stamps
  const bool u_only = ACT || (vec16 && !hist);
  if (sizeof(St) == 1 && !u_only)
    for (uint32_t s = threadIdx.x; s < 256; s += blockDim.x) {
      const uint32_t a = stamp_age(s, cs);
      age_lut[s] = a < p.k ? (uint8_t)a : 255;
    }
  const double eta2 = (double)p.eta2;
  // Eq. 12's P: the same for every host (and already applied in the table when there is one)
  __shared__ double s_P;
  if (threadIdx.x == 0 && !tab.est) s_P = setting_product(active2, p.r2, p.row_len2);
  __shared__ uint32_t warp_rank[kEstThreadsWide / 32];
  for (uint32_t h = blockIdx.x; h < count; h += gridDim.x) {
    const uint32_t aip = rank_mode ? (h == blockIdx.x ? first_aip : unsorted[h])
                                   : (h == blockIdx.x && !unsorted ? first_aip : hosts[h]);
    // rank mode: this thread's share of the host's rank, over keys y = threadIdx.x + i *
    // blockDim.x; the first eight are loaded here and compared after the SLE gathers, so that
    // both sets of loads are in flight together
    uint32_t rank = 0;
    uint32_t kk[8];
    auto rank_batch = [&](uint32_t y0, bool load) {
#pragma unroll
      for (uint32_t u = 0; u < 8; ++u) {
        const uint32_t y = y0 + u * blockDim.x + threadIdx.x;
        if (load) kk[u] = y < count ? unsorted[y] : 0u;
      }
#pragma unroll
      for (uint32_t u = 0; u < 8; ++u) {
        const uint32_t y = y0 + u * blockDim.x + threadIdx.x;
        rank += (y < count && (kk[u] < aip || (kk[u] == aip && y < h))) ? 1u : 0u;
      }
    };
    if (rank_mode)
#pragma unroll
      for (uint32_t u = 0; u < 8; ++u) {
        const uint32_t y = u * blockDim.x + threadIdx.x;
        kk[u] = y < count ? unsorted[y] : 0u;
      }
    if (threadIdx.x < p.r2) {
      const uint32_t j = mas_top(p.key_a[kLH + threadIdx.x], p.key_b[kLH + threadIdx.x], aip, p.q2);
      row_cell[threadIdx.x] = threadIdx.x * p.row_pitch2 + (uint64_t)j * p.delta2;
      row_base[threadIdx.x] = sle + row_cell[threadIdx.x];
    }
    // per-distance counts: in shared memory for windows up to 256 slices, else straight
    // into this host's output row (zeroed first)
    const bool hist_smem = p.k <= 256;
    uint32_t* hist_row = hist ? hist + (uint64_t)h * p.k : nullptr;
    if (hist)
      for (uint32_t a = threadIdx.x; a < p.k; a += blockDim.x) {
        if (hist_smem)
          sh_hist[a] = 0;
        else
          hist_row[a] = 0;
      }
    __syncthreads();
    uint32_t u = 0;
    constexpr int kVecCells = 16 / sizeof(St);  // cells per 16-byte load
    constexpr int kIntCells = 4 / sizeof(St);
    constexpr uint32_t kMask = sizeof(St) == 1 ? 0xFFu : 0xFFFFu;
    if constexpr (ACT) {
      // U only, from the activity bitmap of this close (bit c: SLEA cell c is active): a union
      // cell counts when it is active in every row, so the rows' bits are ANDed. Row i's eta'
      // bits start at bit row_cell[i], at any alignment: each 32-bit piece is a funnel shift
      // of two words (the bitmap has a word of padding after the last row)
      const uint32_t n_words = p.eta2 >> 5;
      for (uint32_t k = threadIdx.x; k < n_words; k += blockDim.x) {
        uint32_t m = 0xFFFFFFFFu;
        for (uint32_t i0 = 0; i0 < p.r2; i0 += 4) {  // 4 rows' loads in flight
          uint32_t lo[4], hi[4], sh[4];
#pragma unroll
          for (uint32_t j = 0; j < 4; ++j)
            if (i0 + j < p.r2) {
              const uint64_t b = row_cell[i0 + j] + ((uint64_t)k << 5);
              sh[j] = (uint32_t)b & 31u;
              lo[j] = sle_act[b >> 5];
              hi[j] = sle_act[(b >> 5) + 1];
            }
#pragma unroll
          for (uint32_t j = 0; j < 4; ++j)
            if (i0 + j < p.r2) m &= __funnelshift_r(lo[j], hi[j], sh[j]);
        }
        u += __popc(m);
      }
    } else {  // from the stamps
    if (u_only) {
      // U only: a union cell counts when it is active in every row, so the rows' activity
      // masks (active_hi8 for 8-bit cells, active_hi16 for 16-bit ones: the top bit of every
      // active cell) are ANDed; up to 8 rows' loads are in flight at once
      constexpr uint32_t kAll = sizeof(St) == 1 ? 0x80808080u : 0x80008000u;
      auto rows_and = [&](auto wrap, auto win) {  // wrap: std::true_type when the window wraps over 0
        constexpr bool W = decltype(wrap)::value;
        auto active = [&](uint32_t x) {
          if constexpr (sizeof(St) == 1)
            return active_hi8<W>(x, win);
          else
            return active_hi16<W>(x, win);
        };
        uint32_t c = 0;
        for (uint32_t z = threadIdx.x * kVecCells; z < p.eta2; z += blockDim.x * kVecCells) {
          uint32_t a0 = kAll, a1 = a0, a2 = a0, a3 = a0;
          for (uint32_t i0 = 0; i0 < p.r2; i0 += 8) {
            uint4 v[8];
#pragma unroll
            for (uint32_t j = 0; j < 8; ++j)
              if (i0 + j < p.r2) v[j] = *reinterpret_cast<const uint4*>(row_base[i0 + j] + z);
#pragma unroll
            for (uint32_t j = 0; j < 8; ++j)
              if (i0 + j < p.r2) {
                a0 &= active(v[j].x);
                a1 &= active(v[j].y);
                a2 &= active(v[j].z);
                a3 &= active(v[j].w);
              }
          }
          c += count4(a0, a1, a2, a3);
        }
        return c;
      };
      if constexpr (sizeof(St) == 1) {
        const Window8 win = window8(cs, p.k);
        u = win.wrap ? rows_and(std::true_type{}, win) : rows_and(std::false_type{}, win);
      } else {
        const Window16 win = window16(cs, p.k);
        u = win.wrap ? rows_and(std::true_type{}, win) : rows_and(std::false_type{}, win);
      }
    } else if (vec16) {
      for (uint32_t z = threadIdx.x * kVecCells; z < p.eta2; z += blockDim.x * kVecCells) {
        uint32_t m[kVecCells];
#pragma unroll
        for (int b = 0; b < kVecCells; ++b) m[b] = 0;
        // several rows' loads in flight at once (8 for 16-bit cells, 4 for 8-bit, whose 16
        // per-cell maxima take the registers), then their distances
        constexpr uint32_t kRowBatch = sizeof(St) == 1 ? 4 : 8;
        for (uint32_t i0 = 0; i0 < p.r2; i0 += kRowBatch) {
          uint4 v[kRowBatch];
#pragma unroll
          for (uint32_t j = 0; j < kRowBatch; ++j)
            if (i0 + j < p.r2) v[j] = *reinterpret_cast<const uint4*>(row_base[i0 + j] + z);
#pragma unroll
          for (uint32_t j = 0; j < kRowBatch; ++j) {
            if (i0 + j >= p.r2) break;
            const uint32_t x[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
#pragma unroll
            for (int b = 0; b < kVecCells; ++b)
              m[b] = max(m[b], cell_age<St>((x[b / kIntCells] >> (8 * sizeof(St) * (b % kIntCells))) & kMask,
                                            age_lut, cs, p.k));
          }
        }
#pragma unroll
        for (int b = 0; b < kVecCells; ++b)
          if (m[b] != kInactive<St>) {
            u += 1;
            if (hist) atomicAdd(hist_smem ? &sh_hist[m[b]] : &hist_row[m[b]], 1u);
          }
      }
    } else {
      for (uint32_t z = threadIdx.x; z < p.eta2; z += blockDim.x) {
        uint32_t m = 0;
        for (uint32_t i = 0; i < p.r2; ++i) m = max(m, cell_age<St>(row_base[i][z], age_lut, cs, p.k));
        if (m != kInactive<St>) {
          u += 1;
          if (hist) atomicAdd(hist_smem ? &sh_hist[m] : &hist_row[m], 1u);
        }
      }
    }
    }
    if (rank_mode) {
      rank_batch(0, false);  // the keys loaded before the gathers
      for (uint32_t y0 = 8 * blockDim.x; y0 < count; y0 += 8 * blockDim.x) rank_batch(y0, true);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      u += __shfl_xor_sync(0xFFFFFFFFu, u, off);
      rank += __shfl_xor_sync(0xFFFFFFFFu, rank, off);
    }
    if ((threadIdx.x & 31) == 0) {
      warp_u[threadIdx.x >> 5] = u;
      warp_rank[threadIdx.x >> 5] = rank;
    }
    __syncthreads();
    if (hist && hist_smem)
      for (uint32_t a = threadIdx.x; a < p.k; a += blockDim.x) hist_row[a] = sh_hist[a];
    if (threadIdx.x == 0) {
      uint32_t U = 0, at = 0;
#pragma unroll
      for (uint32_t x = 0; x < kEstThreadsWide / 32; ++x)
        if (x < (blockDim.x >> 5)) {
          U += warp_u[x];
          at += warp_rank[x];
        }
      const uint32_t slot = rank_mode ? at : h;  // where this host's outputs go
      LcResult res;
      if (tab.est) {  // this close's table
        res.est = tab.est[U];
        res.flags = tab.flags[U];
        res.w = w_out ? tab.w[U] : 0.0;
      } else {
        res = lc_estimate(U, s_P, eta2, w_theta);
      }
      if ((res.flags & SSE_FLAG_SUPER) && n_super) atomicAdd(n_super, 1u);
      est[slot] = res.est;
      if (flags) flags[slot] = res.flags;
      if (w_out) w_out[slot] = res.w;
      if (u_out) u_out[slot] = U;
      if (rank_mode) hosts_out[slot] = aip;
    }
    __syncthreads();
  }
}

}  // namespace sse
