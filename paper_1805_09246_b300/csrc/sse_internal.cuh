// Internal definitions shared by the kernels and the host runtime of libsse.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sse.h"

namespace sse {

constexpr int kMaxRows = 16;            // r and r' are at most 16
constexpr int kEta = 8;                 // cells per SRE (one 64-bit word)
constexpr uint32_t kPitchAlign = 4096;  // SLEA row pitch: whole close-kernel blocks per row
constexpr int kSortChunk = 4096;        // elements sorted per CTA before merge passes
constexpr int kMaxMergeSources = 64;

// Key order: 0 = H1, 1 = H2, 2 = H3, 3 = RHFG[0], 4 + i = LH_i.
enum { kH1 = 0, kH2 = 1, kH3 = 2, kR0 = 3, kLH = 4 };

// Everything a kernel needs to evaluate the method's hash functions and addresses.
struct KParams {
  uint64_t key_a[kLH + kMaxRows];
  uint64_t key_b[kLH + kMaxRows];
  uint32_t r, q, delta, r2;
  uint32_t q2, delta2, lg_eta2, eta2;
  uint32_t k, tau_mask, sre_on, hot_min;
  uint64_t row_pitch2;  // cells between SLEA rows
  uint64_t row_len2;    // cells per SLEA row
  const uint32_t* tab;  // RHFG[0] tabulation tables [4][256] (device), or NULL: multiply-add-shift
};

// Multiply-add-shift hash: the top m bits (0 <= m <= 32) of (a*x + b) mod 2^64.
// With x < 2^32 the high word is hi32(lo32(a)*x + b) + hi32(a)*x (mod 2^32): one widening
// multiply-add and one 32-bit multiply-add.
__host__ __device__ __forceinline__ uint32_t mas_hi(uint64_t a, uint64_t b, uint32_t x) {
  const uint64_t t = (uint64_t)(uint32_t)a * x + b;
  return (uint32_t)(t >> 32) + (uint32_t)(a >> 32) * x;
}
__host__ __device__ __forceinline__ uint32_t mas_top(uint64_t a, uint64_t b, uint32_t x, uint32_t m) {
  return (uint32_t)((uint64_t)mas_hi(a, b, x) >> (32 - m));
}

// RHFG[0](aip) (Eq. 6): simple tabulation over the four address bytes when the tables are
// set, else multiply-add-shift; the top q bits.
__device__ __forceinline__ uint32_t rhfg0(const KParams& p, uint32_t aip) {
  if (p.tab)
    return (p.tab[aip & 255u] ^ p.tab[256 + ((aip >> 8) & 255u)] ^ p.tab[512 + ((aip >> 16) & 255u)] ^
            p.tab[768 + (aip >> 24)]) >> (32 - p.q);
  return mas_top(p.key_a[kR0], p.key_b[kR0], aip, p.q);
}

// The lows of regain's interval test by search: emit(low) for every entry of the table d
// (n values a*low mod 2^64, ascending, a power of two of them, with their lows) whose
// (d + v) mod 2^64 is below width. A binary search finds the first entry at or above -v;
// from there (d + v) mod 2^64 ascends around the table, so the walk stops at the first
// miss.
template <typename Emit>
__host__ __device__ __forceinline__ void regain_search(const uint64_t* d, const uint32_t* low, uint32_t n, uint64_t v,
                                                       uint64_t width, Emit emit) {
  const uint64_t s = 0ull - v;  // the interval's start
  uint32_t at = 0;              // entries of the table below s
  for (uint32_t step = n >> 1; step > 0; step >>= 1)
    if (d[at + step - 1] < s) at += step;
  if (d[at] < s) at += 1;
  for (uint32_t k = 0; k < n; ++k) {
    const uint32_t i = (at + k) & (n - 1u);
    if (d[i] + v >= width) break;
    emit(low[i]);
  }
}

// regain_search with the binary search replaced by a bucket lookup: first[j] (j = 0..64) is
// the number of table entries below j * 2^58, so the entries below the interval's start s are
// first[s >> 58] plus those of s's bucket below s (about n / 64 of them: a few at most).
template <typename Emit>
__host__ __device__ __forceinline__ void regain_search_bucketed(const uint64_t* d, const uint32_t* low,
                                                                const uint8_t* first, uint32_t n, uint64_t v,
                                                                uint64_t width, Emit emit) {
  const uint64_t s = 0ull - v;  // the interval's start
  uint32_t at = first[s >> 58];
  while (at < n && d[at] < s) ++at;
  for (uint32_t k = 0; k < n; ++k) {
    const uint32_t i = (at + k) & (n - 1u);
    if (d[i] + v >= width) break;
    emit(low[i]);
  }
}

// Cyclic stamp arithmetic: slice t has stamp 1 + (t mod 255); 0 marks an unset cell.
__host__ __device__ __forceinline__ uint8_t stamp_of(uint64_t slice) { return (uint8_t)(1 + slice % 255); }

// Age in slices of stamp s seen from current stamp cs (both 1..255), or 255 when unset.
__host__ __device__ __forceinline__ uint32_t stamp_age(uint32_t s, uint32_t cs) {
  if (s == 0) return 255;
  return (cs + 255 - s) % 255;
}

// Stamps of w-bit cells cycle through 1..2^w - 1 (slice t: 1 + t mod (2^w - 1)); 0 is unset.
__host__ __device__ __forceinline__ uint32_t stamp_mod(uint32_t stamp_bits) { return (1u << stamp_bits) - 1u; }
__host__ __device__ __forceinline__ uint32_t stamp_of(uint64_t slice, uint32_t mod) {
  return (uint32_t)(1 + slice % mod);
}

// Activity of four 8-bit stamps at once (SWAR on a 32-bit word). A stamp s is active for a
// window of k slices at current stamp cs when s != 0 and (cs - s) mod 255 < k. The active
// stamps form one cyclic interval, so with L = cs - k + 1, K = k when cs >= k, and
// L = cs + 256 - k, K = k + 1 otherwise (the interval then wraps over 0, which s != 0
// removes), s is active exactly when s != 0 and (s - L) mod 256 < K. The byte-wise
// subtraction, addition and carry formulas are the standard ones (Hacker's Delight,
// Section 2-18): no carry crosses a byte. Returns 0x80 in every active byte, 0 elsewhere.
struct Window8 {
  uint32_t L4;    // L in every byte
  uint32_t C4;    // 256 - K in every byte (t < K exactly when t + (256 - K) does not carry)
  uint32_t wrap;  // cs < k: the interval wraps over 0, so s != 0 must be tested too
};
__host__ __device__ __forceinline__ Window8 window8(uint32_t cs, uint32_t k) {
  const uint32_t L = cs >= k ? cs - k + 1 : cs + 256 - k;
  const uint32_t K = cs >= k ? k : k + 1;
  return Window8{(L & 255u) * 0x01010101u, (256u - K) * 0x01010101u, cs < k ? 1u : 0u};
}
// WRAP = win.wrap. Without the wrap, s = 0 gives (0 - L) mod 256 = 256 - L >= K, so the
// interval test alone decides.
template <bool WRAP>
__host__ __device__ __forceinline__ uint32_t active_hi8(uint32_t w, Window8 win) {
  constexpr uint32_t H = 0x80808080u, Lo = 0x7F7F7F7Fu;
  const uint32_t t = ((w | H) - (win.L4 & Lo)) ^ ((w ^ ~win.L4) & H);  // (s - L) mod 256 per byte
  const uint32_t low = (t & Lo) + (win.C4 & Lo);                       // carry into bit 7
  const uint32_t carry = (t & win.C4) | ((t | win.C4) & low);           // bit 7: t + C >= 256
  if (!WRAP) return ~carry & H;
  const uint32_t nz = ((w & Lo) + Lo) | w;  // bit 7: s != 0
  return ~carry & nz & H;
}
__host__ __device__ __forceinline__ uint32_t active_hi8(uint32_t w, Window8 win) {
  return win.wrap ? active_hi8<true>(w, win) : active_hi8<false>(w, win);
}

// The same test for two 16-bit stamps in a 32-bit word (cycle 1..65535, windows k <= 65534):
// the active stamps form the cyclic interval from L = cs - k + 1 (mod 65535, in 1..65535) to
// cs; with K = k when cs >= k and L = cs + 65536 - k, K = k + 1 otherwise (the interval then
// wraps over 0, which s != 0 removes), s is active exactly when s != 0 and
// (s - L) mod 65536 < K. Returns 0x8000 in every active half, 0 elsewhere.
struct Window16 {
  uint32_t L2;    // L in both halves
  uint32_t C2;    // 65536 - K in both halves
  uint32_t wrap;  // cs < k
};
__host__ __device__ __forceinline__ Window16 window16(uint32_t cs, uint32_t k) {
  const uint32_t L = cs >= k ? cs - k + 1 : cs + 65536 - k;
  const uint32_t K = cs >= k ? k : k + 1;
  return Window16{(L & 0xFFFFu) * 0x00010001u, (65536u - K) * 0x00010001u, cs < k ? 1u : 0u};
}
template <bool WRAP>
__host__ __device__ __forceinline__ uint32_t active_hi16(uint32_t w, Window16 win) {
  constexpr uint32_t H = 0x80008000u, Lo = 0x7FFF7FFFu;
  const uint32_t t = ((w | H) - (win.L2 & Lo)) ^ ((w ^ ~win.L2) & H);  // (s - L) mod 65536 per half
  const uint32_t low = (t & Lo) + (win.C2 & Lo);                       // carry into bit 15
  const uint32_t carry = (t & win.C2) | ((t | win.C2) & low);           // bit 15: t + C >= 65536
  if (!WRAP) return ~carry & H;
  const uint32_t nz = ((w & Lo) + Lo) | w;  // bit 15: s != 0
  return ~carry & nz & H;
}
__host__ __device__ __forceinline__ uint32_t active_hi16(uint32_t w, Window16 win) {
  return win.wrap ? active_hi16<true>(w, win) : active_hi16<false>(w, win);
}

// Programmatic dependent launch. A kernel launched with programmatic stream serialization
// may be scheduled before the previous kernel on its stream has finished; pdl_wait(), called
// before the kernel touches memory, returns once that kernel has completed and its writes
// are visible (for an ordinary launch it returns at once). pdl_trigger() lets the next
// kernel be scheduled once every block of this one has called it (so no block of this
// kernel can be kept waiting for room by the next one's blocks).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// The estimator's device clock holds the current stamp; advancing a slice moves it along the
// 1..mod cycle on the device, so launches read the right stamp even when replayed.
__global__ void k_tick(uint32_t* clock, uint32_t n, uint32_t mod = 255u) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    for (uint32_t i = 0; i < n; ++i) clock[i] = clock[i] % mod + 1u;
}

// Scratch counters of one close, zeroed before it (one cudaMemsetAsync).
struct CloseScratch {
  uint32_t active2[kMaxRows];  // active cells of each SLEA row
  uint32_t hot[kMaxRows];      // hot SREs of each RSRA row
  uint32_t n_list[2];          // entries of the hot lists of rows 0 and 1
  unsigned long long down_pairs;  // (he_0, he_{r-1}) pairs the join from the top row down started from
  uint32_t n_cand;             // candidate hosts found (may exceed capacity)
  uint32_t n_super;            // candidates flagged super
  uint32_t overflow;           // nonzero when a buffer was too small
  uint32_t error;              // nonzero when a bounded device-side wait gave up
  uint32_t barrier[2];         // grid barrier of the candidate sort (arrivals, generation)
  uint32_t report_blocks;      // blocks of the report kernel that have written their part
  uint32_t report_done;        // in the report stage: set last, once the whole report is there
};

}  // namespace sse
