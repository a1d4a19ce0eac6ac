// Per-packet update, tiled strategy: SLEA writes are collected on chip.
//
// Within one slice every write stores the same stamp, so a slice's SLEA update is fully
// described by the set of cells touched (Algorithm 6 writes are idempotent). Each CTA owns
// one tile: a piece of one SLEA row, kept as a bitmap in shared memory (one bit per cell).
// The CTAs of a group together own every tile and share one contiguous range of the pairs:
// each CTA hashes each pair for its own row (LH_row and H3), and sets the bit when the cell
// falls in its piece — an on-chip atomic OR instead of a scattered one-byte L2 write. At the
// end every CTA ORs its non-zero bitmap words into a global bitmap of the SLEA, and
// k_apply_bits turns each set bit into the stamp (and clears the bitmap for the next call).
// RSRA writes (Algorithm 3, only a 2^-tau fraction of pairs) stay direct global stores;
// each pair's RSRA work is done by exactly one CTA of its group.
#pragma once

#include "k_update.cuh"
#include "sse_internal.cuh"

namespace sse {

constexpr int kTiledThreads = 1024;
// Shared memory behind the tile's bitmap: one RSRA queue per warp.
constexpr uint32_t kRsraQueueBytes = (kTiledThreads / 32) * kRsraQueueEntries * sizeof(uint2);

// Hashing and marking for one tile: cell H3(bip) of SLE LH_row(aip) (Algorithm 6) as a bit
// of the tile's shared-memory bitmap. Keys are split into 32-bit halves once, so each hash
// is one widening multiply-add and one multiply-add. WHOLE: the tile is the whole row
// (lo = 0, every cell of the row is inside the bitmap), so no range test is needed.
struct SleTile {
  uint32_t a3lo, a3hi, alo, ahi;
  uint64_t b3, bl;
  uint32_t sh3, shl, d2, lo, span;

  __device__ __forceinline__ SleTile(const KParams& p, uint32_t row, uint32_t lo_, uint32_t span_)
      : a3lo((uint32_t)p.key_a[kH3]), a3hi((uint32_t)(p.key_a[kH3] >> 32)), alo((uint32_t)p.key_a[kLH + row]),
        ahi((uint32_t)(p.key_a[kLH + row] >> 32)), b3(p.key_b[kH3]), bl(p.key_b[kLH + row]),
        sh3(32 - p.lg_eta2), shl(32 - p.q2), d2(p.delta2), lo(lo_), span(span_) {}

  static __device__ __forceinline__ uint32_t hash_hi(uint32_t alo_, uint32_t ahi_, uint64_t b, uint32_t x) {
    const uint64_t t = (uint64_t)alo_ * x + b;
    return (uint32_t)(t >> 32) + ahi_ * x;
  }

  template <bool WHOLE, bool CHECK>
  __device__ __forceinline__ void touch(uint32_t* bm, uint32_t aip, uint32_t bip) const {
    const uint32_t h3 = hash_hi(a3lo, a3hi, b3, bip) >> sh3;  // sh3, shl <= 31: eta', 2^q' >= 2
    const uint32_t lh = hash_hi(alo, ahi, bl, aip) >> shl;
    uint32_t cell = lh * d2 + h3;
    if (!WHOLE) {
      cell -= lo;  // wraps to a large value below lo
      if (cell >= span) return;
    }
    uint32_t bit;  // 1 << (cell mod 32): funnel shift of {1:0}
    asm("shf.l.wrap.b32 %0, %1, %2, %3;" : "=r"(bit) : "r"(0u), "r"(1u), "r"(cell));
    uint32_t* w = bm + (cell >> 5);
    if (CHECK && (*w & bit)) return;
    atomicOr(w, bit);
  }
};

// ORs `bytes` of a shared-memory bitmap into global memory with bulk reductions done in L2 by
// the Tensor Memory Accelerator (cp.reduce.async.bulk .or.b32), not one atomic per word from
// the SM. Called by one thread, after every thread's writes to the bitmap were followed by
// fence.proxy.async.shared::cta and a barrier. Both addresses are 16-byte aligned and bytes
// is a multiple of 16. Returns once the bitmap has been read (it may then be rewritten) or,
// with `done`, once the reductions are complete.
__device__ __forceinline__ void bitmap_or_bulk(const uint32_t* bm, uint8_t* dst, uint32_t bytes, bool done) {
  const uint32_t src = (uint32_t)__cvta_generic_to_shared(bm);
  constexpr uint32_t kChunk = 32768u;
  for (uint32_t off = 0; off < bytes; off += kChunk) {
    const uint32_t n = bytes - off < kChunk ? bytes - off : kChunk;
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.or.b32 [%0], [%1], %2;" ::"l"(dst + off),
                 "r"(src + off), "r"(n)
                 : "memory");
  }
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  if (done)
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  else
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Bytes of a tile's bitmap to reduce into the row: the last piece of a row may reach past
// the row pitch (pieces are rounded up to 1024 cells), and cells beyond it are never set.
__device__ __forceinline__ uint32_t tile_flush_bytes(uint64_t row_pitch2, uint32_t lo, uint32_t piece_bytes) {
  const uint64_t left = row_pitch2 - lo;
  return (uint32_t)((left < piece_bytes ? left : piece_bytes) >> 3);
}

struct TileGeometry {
  uint32_t tiles;         // tiles per group (r' * pieces)
  uint32_t pieces;        // pieces per SLEA row
  uint32_t piece_bytes;   // cells per piece (multiple of 1024)
  uint32_t groups;        // groups of CTAs; the pairs are split evenly between groups
};

// grid = groups * tiles CTAs; dynamic shared memory = piece_bytes / 8 + kRsraQueueBytes. UNROLL 128-bit loads
// are in flight per thread; CHECK reads the bitmap word first and skips the atomic when the
// bit is already set (repeated pairs are common in real traffic). PIPE issues the next block
// iteration's loads before the current iteration's pairs are hashed (two register buffers),
// so each thread's loads overlap its own atomics.
template <typename St, int UNROLL, bool CHECK, bool WHOLE, bool PIPE = false>
__global__ void __launch_bounds__(kTiledThreads, 1) k_update_tiled(const __grid_constant__ KParams p, TileGeometry g,
                                                                   const uint2* __restrict__ pairs, uint64_t n,
                                                                   uint8_t* __restrict__ sre_bytes,
                                                                   uint32_t* __restrict__ gbits, uint32_t stamp_value,
                                                                   const uint32_t* __restrict__ clock,
                                                                   uint8_t* __restrict__ sre2_bytes,
                                                                   uint32_t* __restrict__ gbits2) {
  pdl_wait();
  pdl_trigger();
  const St stamp = (St)(clock ? *clock : stamp_value);
  St* sre = reinterpret_cast<St*>(sre_bytes);
  St* sre2 = reinterpret_cast<St*>(sre2_bytes);  // may be NULL: see the flush
  extern __shared__ __align__(16) uint32_t bm[];
  const uint32_t tile = blockIdx.x % g.tiles;
  const uint32_t group = blockIdx.x / g.tiles;
  const uint32_t row = tile / g.pieces;
  const uint32_t piece = tile % g.pieces;
  const uint32_t lo = piece * g.piece_bytes;  // cell range [lo, lo + piece_bytes) of the row
  const uint32_t words = g.piece_bytes >> 5;
  for (uint32_t w = threadIdx.x; w < words; w += kTiledThreads) bm[w] = 0;
  RsraQueue rq{reinterpret_cast<uint2*>(bm + words) + (threadIdx.x >> 5) * kRsraQueueEntries, 0u, threadIdx.x & 31u};
  __syncthreads();

  // this group's pairs: [begin, end). The pairs before the first 128-byte boundary (the
  // head, at most 15) belong to group 0; the rest is cut at multiples of 16 pairs, so every
  // group starts on a 128-byte line and a warp's 512-byte load covers four whole lines (an
  // unaligned one spans five, and the load pipe moves one line per wavefront). The head's
  // and the odd last pair's RSRA work belongs to tile 0.
  const uint64_t head = min((uint64_t)(((128u - (reinterpret_cast<uintptr_t>(pairs) & 127u)) & 127u) >> 3), n);
  const uint64_t lines = (n - head) >> 4;
  const uint64_t begin = head + 16 * (lines * group / g.groups);
  const uint64_t end = group + 1 == g.groups ? n : head + 16 * (lines * (group + 1) / g.groups);
  const SleTile st(p, row, lo, g.piece_bytes);
  auto touch = [&](uint32_t aip, uint32_t bip) { st.touch<WHOLE, CHECK>(bm, aip, bip); };
  if (group == 0 && threadIdx.x < head) {
    const uint2 v = pairs[threadIdx.x];
    touch(v.x, v.y);
    if (tile == 0) stamp_rsra(p, v.x, v.y, sre, stamp, sre2);
  }
  const uint64_t j0 = begin;
  const uint4* vec = reinterpret_cast<const uint4*>(pairs + j0);
  const uint32_t nvec = (uint32_t)((end - j0) >> 1);
  constexpr uint32_t stride = kTiledThreads;  // the launch's block size: load offsets fold into immediates
  const uint64_t policy = stream_policy();
  // Block iteration k covers vectors [k*stride*UNROLL, (k+1)*stride*UNROLL); its RSRA work
  // belongs to tile k mod tiles. The test is uniform across the block and taken once per
  // 2*UNROLL pairs, so the RSRA code is a real branch, skipped by the other tiles (per-pair
  // ownership let the compiler predicate the hashing of H1 into every tile).
  const uint32_t full = nvec / (stride * UNROLL);
  uint32_t owner = 0;
  auto block_iteration = [&](const uint4 (&buf)[UNROLL]) {
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      touch(buf[u].x, buf[u].y);
      touch(buf[u].z, buf[u].w);
    }
    if (owner == tile && p.sre_on) {
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) {
        rq.push(p, true, buf[u].x, buf[u].y, sre, stamp, sre2);
        rq.push(p, true, buf[u].z, buf[u].w, sre, stamp, sre2);
      }
    }
    owner = owner + 1 == g.tiles ? 0 : owner + 1;
  };
  if (PIPE) {
    uint4 cur[UNROLL];
    if (full > 0) {
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) cur[u] = load_stream(vec + threadIdx.x + u * stride, policy);
    }
    for (uint32_t k = 0; k < full; ++k) {
      uint4 nxt[UNROLL];
      if (k + 1 < full) {  // uniform
        const uint32_t base = (k + 1) * stride * UNROLL + threadIdx.x;
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) nxt[u] = load_stream(vec + base + u * stride, policy);
      } else {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) nxt[u] = make_uint4(0, 0, 0, 0);
      }
      block_iteration(cur);
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) cur[u] = nxt[u];
    }
  } else {
    for (uint32_t k = 0; k < full; ++k) {
      const uint32_t base = k * stride * UNROLL + threadIdx.x;
      uint4 buf[UNROLL];
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) buf[u] = load_stream(vec + base + u * stride, policy);
      block_iteration(buf);
    }
  }
  const bool mine = owner == tile && p.sre_on;  // remainder: the last, partial iteration
  for (uint32_t u = 0; u < UNROLL; ++u) {
    const uint32_t i = full * stride * UNROLL + u * stride + threadIdx.x;
    const bool ok = i < nvec;
    const uint4 v = ok ? load_stream(vec + i, policy) : make_uint4(0, 0, 0, 0);
    if (ok) {
      touch(v.x, v.y);
      touch(v.z, v.w);
    }
    if (mine) {
      rq.push(p, ok, v.x, v.y, sre, stamp, sre2);
      rq.push(p, ok, v.z, v.w, sre, stamp, sre2);
    }
  }
  if (p.sre_on) rq.drain(p, sre, stamp, sre2);
  if (((end - j0) & 1) && threadIdx.x == 0) {
    const uint2 v = pairs[end - 1];
    touch(v.x, v.y);
    if (tile == 0) stamp_rsra(p, v.x, v.y, sre, stamp, sre2);
  }
  // flush: OR the piece's bitmap into the global SLEA bitmap (bitmap_or_bulk). Byte offsets
  // are cells / 8: the row pitch is a multiple of 4096 cells, a piece and its start
  // multiples of 1024, so both ends are 16-byte aligned.
  // With gbits2 (a second estimator's SLEA bitmap, e.g. a serving router's global
  // estimator: sre2 above received the RSRA stamps) the piece is ORed into both.
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint64_t at = ((uint64_t)row * p.row_pitch2 + lo) >> 3;
    const uint32_t bytes = tile_flush_bytes(p.row_pitch2, lo, g.piece_bytes);
    if (gbits2) bitmap_or_bulk(bm, reinterpret_cast<uint8_t*>(gbits2) + at, bytes, false);
    bitmap_or_bulk(bm, reinterpret_cast<uint8_t*>(gbits) + at, bytes, true);
  }
}

// Stamp every SLEA cell whose bit is set and clear the bitmap. One thread per 16-byte vector
// of cells (16 8-bit or 8 16-bit stamps), so a warp reads and writes 512 contiguous bytes;
// the 2 or 4 lanes that share a bitmap word read it together, and the first of them clears
// it after the warp has read it.
template <typename St>
__global__ void __launch_bounds__(256) k_apply_bits(uint32_t* __restrict__ gbits, uint8_t* __restrict__ sle,
                                                    uint64_t n_words, uint32_t stamp_value,
                                                    const uint32_t* __restrict__ clock) {
  pdl_wait();
  pdl_trigger();
  constexpr int kCellsPerVec = 16 / sizeof(St);  // 16 or 8
  constexpr int kVecs = 32 / kCellsPerVec;       // vectors per bitmap word: 2 or 4
  constexpr int kCellsPerInt = 4 / sizeof(St);   // 4 or 2
  constexpr uint32_t kCellMask = sizeof(St) == 1 ? 0xFFu : 0xFFFFu;
  const uint32_t stamp = clock ? *clock : stamp_value;
  const uint32_t fill = sizeof(St) == 1 ? stamp * 0x01010101u : stamp * 0x00010001u;
  const uint64_t n_vecs = n_words * kVecs;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;  // a multiple of 32
  // warp-uniform loop: every lane of a warp takes the same number of steps
  for (uint64_t v0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); v0 < n_vecs; v0 += stride) {
    const uint64_t v = v0 + (threadIdx.x & 31u);
    const bool ok = v < n_vecs;
    const uint32_t bits = ok ? gbits[v / kVecs] : 0u;
    __syncwarp();  // every lane sharing the word has read it
    if (ok && bits && v % kVecs == 0) gbits[v / kVecs] = 0;
    const uint32_t hb = (bits >> (kCellsPerVec * (uint32_t)(v % kVecs))) & ((1u << kCellsPerVec) - 1u);
    if (!hb) continue;
    uint4* cells = reinterpret_cast<uint4*>(sle) + v;
    const uint4 c = *cells;
    uint32_t x[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t nib = (hb >> (kCellsPerInt * q)) & ((1u << kCellsPerInt) - 1u);
      uint32_t mask = 0;  // all ones in the cells whose bit is set
#pragma unroll
      for (int b = 0; b < kCellsPerInt; ++b) mask |= ((nib >> b) & 1u) ? kCellMask << (8 * sizeof(St) * b) : 0u;
      x[q] = (x[q] & ~mask) | (fill & mask);
    }
    *cells = make_uint4(x[0], x[1], x[2], x[3]);
  }
}

}  // namespace sse
