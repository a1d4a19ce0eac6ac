// Host runtime of libsse: parameters, handles, launches and the C ABI of sse.h.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <chrono>
#include <cstddef>
#include <new>

// NVTX ranges around the entry points' host work (update, close, merge, query, batch
// steps), for timeline tools; compiled in only with -DSSE_NVTX (header-only NVTX v3, no
// library to link; a range costs nothing when no tool is attached).
#ifdef SSE_NVTX
#include <nvtx3/nvToolsExt.h>
namespace {
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace
#define SSE_NVTX_RANGE(name) NvtxRange sse_nvtx_range_(name)
#else
#define SSE_NVTX_RANGE(name) ((void)0)
#endif

#include "k_batch.cuh"
#include "k_close.cuh"
#include "k_detect.cuh"
#include "k_learn.cuh"
#include "k_merge.cuh"
#include "k_update.cuh"
#include "k_update_tiled.cuh"
#include "sse.h"
#include "sse_internal.cuh"

namespace sse {
namespace {

// SplitMix64 (Steele, Lea, Flood 2014): the hash keys are its successive outputs.
uint64_t splitmix64(uint64_t& state) {
  state += 0x9E3779B97F4A7C15ULL;
  uint64_t z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint32_t ilog2(uint64_t v) {
  uint32_t m = 0;
  while ((1ull << m) < v) ++m;
  return m;
}

bool is_pow2(uint64_t v) { return v && !(v & (v - 1)); }

int derive_params(const sse_params& in, sse_params& p, sse_derived& d) {
  p = in;
  if (p.r < 3 || p.r > (uint32_t)kMaxRows) return SSE_ERR_INVALID_PARAM;
  if (p.q < 5 || p.q > 26) return SSE_ERR_INVALID_PARAM;
  if (p.delta == 0) p.delta = (32 - p.q + p.r - 3) / (p.r - 2);  // ceil((32 - q) / (r - 2))
  if (p.delta == 0 || p.delta >= p.q) return SSE_ERR_INVALID_PARAM;
  if ((uint64_t)(p.r - 2) * p.delta + p.q < 32) return SSE_ERR_INVALID_PARAM;
  if ((uint64_t)(p.r - 1) * p.delta + p.q > 64) return SSE_ERR_INVALID_PARAM;
  if (p.eta != (uint32_t)kEta) return SSE_ERR_INVALID_PARAM;
  if (p.r2 < 1 || p.r2 > (uint32_t)kMaxRows || p.q2 > 24) return SSE_ERR_INVALID_PARAM;
  if (!is_pow2(p.eta2) || p.eta2 < 32 || p.eta2 > 65536) return SSE_ERR_INVALID_PARAM;
  if (p.delta2 < 1 || p.delta2 > p.eta2) return SSE_ERR_INVALID_PARAM;
  if (p.stamp_bits != 8 && p.stamp_bits != 16) return SSE_ERR_INVALID_PARAM;
  if (p.rhfg_hash > 1 || p.reserved != 0) return SSE_ERR_INVALID_PARAM;
  if (p.k < 1 || p.k > stamp_mod(p.stamp_bits) - 1) return SSE_ERR_INVALID_PARAM;  // k <= 254 or 65534
  if (p.theta < 1) return SSE_ERR_INVALID_PARAM;
  if (p.max_candidates < 1 || p.max_candidates > (1u << 22)) return SSE_ERR_INVALID_PARAM;
  memset(&d, 0, sizeof(d));
  d.delta = p.delta;
  uint32_t tau = 0;
  while (((uint64_t)p.eta << tau) < p.theta) ++tau;  // Eq. 1
  d.tau = tau;
  const double rho = 0.99 * (1.0 - std::exp(-1.0 / 3.0));
  d.hot_min = (uint32_t)std::ceil((double)p.eta * rho);
  d.lg_eta2 = ilog2(p.eta2);
  d.row_len2 = ((uint64_t)1 << p.q2) * p.delta2 + p.eta2 - p.delta2;
  if (d.row_len2 > (1ull << 31)) return SSE_ERR_INVALID_PARAM;
  d.row_pitch2 = (d.row_len2 + kPitchAlign - 1) / kPitchAlign * kPitchAlign;
  d.sre_bytes = ((uint64_t)p.r << p.q << 3) * (p.stamp_bits / 8);
  d.sle_bytes = (uint64_t)p.r2 * d.row_pitch2 * (p.stamp_bits / 8);
  d.w_theta = (double)p.eta2 * (-std::expm1(-(double)p.theta / (double)p.eta2));
  return SSE_OK;
}

}  // namespace
}  // namespace sse

using namespace sse;

struct sse_handle {
  sse_params p;
  sse_derived d;
  KParams kp;
  int device = 0;
  cudaStream_t stream = nullptr;
  uint64_t slice = 0;
  uint32_t smod = 255;    // stamp cycle: 255 (8-bit cells) or 65535 (16-bit cells)
  bool wide = false;      // 16-bit cells
  uint64_t sle_cells = 0; // r' * row pitch
  int sticky = SSE_OK;    // first CUDA error seen; later calls return it
  cudaError_t cuda_error = cudaSuccess;  // the CUDA error behind `sticky`
  uint64_t launches = 0;  // kernels launched by this handle
  int update_mode = SSE_UPDATE_AUTO;
  int direction = SSE_DIR_SRC;   // which end of a pair is the host aip (Definition 1)
  uint32_t* swap_buf = nullptr;  // pairs with their ends exchanged (SSE_DIR_DST / BOTH)
  int tuned_variant = -1;  // update variant chosen by sse_autotune_update (-1: none yet)
  int num_sms = 148;
  // device memory
  uint8_t* state = nullptr;  // RSRA then SLEA
  uint32_t* clock = nullptr; // device copy of the current stamp, 1 + (slice mod 255)
  uint32_t* sort_ctl = nullptr;  // in the clock's allocation: the sort barrier's controls (k_sort_candidates)
  // A second estimator that receives every write of this one's updates (a serving router's
  // global estimator, not owned): its RSRA and SLEA get the same stamps, directly or through
  // its SLEA bitmap (applied when it closes the slice).
  uint8_t* mirror_sre = nullptr;
  uint8_t* mirror_sle = nullptr;
  uint32_t* mirror_bits = nullptr;
  uint8_t* sre = nullptr;
  uint8_t* sle = nullptr;
  uint32_t* hot_bits = nullptr;
  uint32_t* sle_bits = nullptr;  // touched-cell bitmap of SLEA for the tiled update (kept zero)
  uint32_t* sle_act = nullptr;   // activity bitmap of SLEA cells, written by a close's pass for its estimate
  TileGeometry tiles;
  uint32_t* list0 = nullptr;
  uint32_t* list1 = nullptr;
  uint32_t* tables = nullptr;  // hot bitmaps of rows 2..r-1 regrouped for the join
  uint32_t* any2 = nullptr;    // row 2's "any hot" bitmap over c (delta <= 5)
  uint32_t* any3 = nullptr;    // row 3's "any hot" bitmap over c (r > 3, delta <= 5)
  uint32_t join_stage = 0;     // k_join_tiled stages any2 and any3 in shared memory
  uint32_t join_grid = 0;      // k_join_tiled blocks (all resident)
  uint32_t* rhfg_tab = nullptr;  // RHFG[0] tabulation tables (rhfg_hash = 1)
  uint32_t join_smem_t2 = 0;   // stage the row-2 table in shared memory
  uint32_t join_list1_cap = 0; // HSE(1) entries staged in shared memory when it fits
  size_t join_smem = 0;
  size_t join_tiled_smem = 0;  // k_join_tiled (delta <= 5)
  // the join from the top row down (k_join_down), where the parameters admit it
  int join_mode = SSE_JOIN_AUTO;
  uint32_t join_down_s = 0;       // columns per block of row r-1: 2^s, s = 32 - (r-1)*delta (0: not admitted)
  uint32_t join_down_grid = 0;
  uint32_t* blist = nullptr;      // row r-1's hot SREs by column block (2^q entries)
  uint32_t* bcount = nullptr;     // their number per block (2^(q-s) entries)
  uint32_t* cand = nullptr;  // two buffers of cand_cap entries
  uint32_t* cand_alt = nullptr;
  uint32_t* cand_out = nullptr;  // the sorted candidates
  float* est = nullptr;
  uint8_t* flags = nullptr;
  CloseScratch* scratch = nullptr;
  uint32_t* query_active2 = nullptr;
  uint8_t* est_table = nullptr;  // per-close estimate table (EstTable): w | est | flags over U = 0..eta'
  uint32_t cand_cap = 0;  // max_candidates
  CloseScratch* host_scratch = nullptr;  // pinned
  sse_stats stats;
  // staging for sse_update_host
  uint32_t* stage_dev[2] = {nullptr, nullptr};
  uint32_t* stage_host[2] = {nullptr, nullptr};
  cudaEvent_t ev_copied[2] = {nullptr, nullptr};
  cudaEvent_t ev_used[2] = {nullptr, nullptr};
  cudaStream_t copy_stream[2] = {nullptr, nullptr};  // one per staging buffer (two copy engines)
  // sse_close_slice as one CUDA graph (captured on a private stream, replayed on `stream`)
  int close_graph = 1;
  cudaStream_t capture_stream = nullptr;
  cudaGraph_t close_g = nullptr;
  cudaGraphExec_t close_exec = nullptr;
  uint32_t* close_sorted = nullptr;  // the candidate buffer the captured sort ends in
  uint64_t close_kernels = 0;        // kernels per replay
  uint32_t report_stage_n = 0;       // report entries the graph writes to report_stage
  uint8_t* report_stage = nullptr;   // page-locked, mapped: CloseScratch | hosts | est | flags
  uint8_t* report_stage_dev = nullptr;  // its device address
  cudaEvent_t close_done = nullptr;  // recorded after each graph replay
  int close_pending = 0;             // a replay whose report has not been collected
  uint64_t close_pending_slice = 0;
};

namespace {

int fail(sse_handle* h, cudaError_t e) {
  if (e == cudaSuccess) return SSE_OK;
  if (h && h->sticky == SSE_OK) {
    h->sticky = SSE_ERR_CUDA;
    h->cuda_error = e;
  }
  return SSE_ERR_CUDA;
}

#define SSE_CUDA(h, call)                        \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return fail((h), e_); \
  } while (0)

#define SSE_LAUNCHED(h)                          \
  do {                                           \
    (h)->launches += 1;                          \
    cudaError_t e_ = cudaGetLastError();         \
    if (e_ != cudaSuccess) return fail((h), e_); \
  } while (0)

// The simple-tabulation tables of RHFG[0]: 1024 32-bit entries (table j, byte value v at
// j * 256 + v), the top halves of the SplitMix64(seed) outputs that follow the keys of
// H1, H2, H3, RHFG[0] and LH_0..LH_{r'-1}.
void make_rhfg_tables(const sse_params& p, uint32_t* tab) {
  uint64_t s = p.seed;
  for (uint32_t x = 0; x < 2 * (kLH + p.r2); ++x) splitmix64(s);
  for (int i = 0; i < 1024; ++i) tab[i] = (uint32_t)(splitmix64(s) >> 32);
}

KParams make_kparams(const sse_params& p, const sse_derived& d) {
  KParams k;
  memset(&k, 0, sizeof(k));
  uint64_t s = p.seed;
  const uint32_t nkeys = kLH + p.r2;
  for (uint32_t x = 0; x < nkeys; ++x) {
    k.key_a[x] = splitmix64(s) | 1ull;
    k.key_b[x] = splitmix64(s);
  }
  k.r = p.r;
  k.q = p.q;
  k.delta = p.delta;
  k.r2 = p.r2;
  k.q2 = p.q2;
  k.delta2 = p.delta2;
  k.lg_eta2 = d.lg_eta2;
  k.eta2 = p.eta2;
  k.k = p.k;
  k.hot_min = d.hot_min;
  if (d.tau <= 31) {
    k.sre_on = 1;
    k.tau_mask = (1u << d.tau) - 1u;
  } else if (d.tau == 32) {
    k.sre_on = 1;
    k.tau_mask = 0xFFFFFFFFu;
  } else {
    k.sre_on = 0;  // LSB(H1) <= 32 < tau: no pair is sampled
    k.tau_mask = 0xFFFFFFFFu;
  }
  k.row_pitch2 = d.row_pitch2;
  k.row_len2 = d.row_len2;
  return k;
}

// The join from the top row down (k_join_down) applies when B(r-1) keeps only
// s = 32 - (r-1)*delta < q bits inside a 32-bit address (so row r-1's hot SREs fall into
// 2^(q-s) column blocks, at most 4096), with delta <= 5, 4 <= r <= 6 and s >= 5 (valid
// parameters have (r-2)*delta + q >= 32, so s < q always, and r = 3 would need q >= 27).
// Returns s, or 0 when it does not apply.
uint32_t join_down_bits(const sse_params& p, const sse_derived& d) {
  if (d.delta > 5 || p.r < 4 || p.r > 6) return 0;
  const int s = 32 - (int)((p.r - 1) * d.delta);
  if (s < 5 || s >= (int)p.q || (int)p.q - s > 12) return 0;
  return (uint32_t)s;
}

using JoinDownKernel = void (*)(KParams, const uint32_t*, const uint32_t*, const uint32_t*, const uint32_t*,
                                const uint32_t*, uint32_t*, uint32_t*, uint32_t, uint32_t*, unsigned long long*);
const JoinDownKernel kJoinDownFns[3] = {k_join_down<4>, k_join_down<5>, k_join_down<6>};

// The close's join: from the top row down where it applies, unless SSE_JOIN_FORWARD is set.
bool join_down(const sse_handle* h) { return h->join_down_s != 0 && h->join_mode != SSE_JOIN_FORWARD; }

// Launches `kernel` after the previous kernel on `stream` with programmatic stream
// serialization: its blocks may be scheduled once every block of the previous kernel has
// called pdl_trigger(), and each waits in pdl_wait() for that kernel's completion before it
// touches memory, so the launch latency overlaps the previous kernel instead of following it.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

int grid_for(const sse_handle* h, uint64_t work, int block, int per_sm) {
  uint64_t g = (work + block - 1) / block;
  uint64_t cap = (uint64_t)h->num_sms * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

int launch_update_direct(sse_handle* h, const uint32_t* d_pairs, uint64_t n) {
  const uint32_t stamp = stamp_of(h->slice, h->smod);
  const uint64_t work = (n + 1) / 2;
  constexpr int kUnroll = 4;
  const int grid = grid_for(h, (work + kUnroll - 1) / kUnroll, 256, 8);
  const uint2* pairs = reinterpret_cast<const uint2*>(d_pairs);
  const auto fn = h->wide ? (h->p.r2 == 5 ? k_update_direct<uint16_t, 5, kUnroll> : k_update_direct<uint16_t, 0, kUnroll>)
                          : (h->p.r2 == 5 ? k_update_direct<uint8_t, 5, kUnroll> : k_update_direct<uint8_t, 0, kUnroll>);
  fn<<<grid, 256, 0, h->stream>>>(h->kp, pairs, n, h->sre, h->sle, stamp, h->clock, h->mirror_sre, h->mirror_sle);
  SSE_LAUNCHED(h);
  return SSE_OK;
}

// Tiles: each SLEA row is cut into pieces whose bitmap fits one CTA's shared memory.
constexpr uint64_t kTileMaxCells = 1600u * 1024u;  // 200 KiB of bitmap

TileGeometry make_tiles(const sse_params& p, const sse_derived& d, int num_sms) {
  TileGeometry g;
  g.pieces = (uint32_t)((d.row_pitch2 + kTileMaxCells - 1) / kTileMaxCells);
  uint64_t piece = (d.row_pitch2 + g.pieces - 1) / g.pieces;
  g.piece_bytes = (uint32_t)((piece + 1023) / 1024 * 1024);
  g.tiles = p.r2 * g.pieces;
  g.groups = std::max<uint32_t>(1u, (uint32_t)num_sms / g.tiles);
  return g;
}

// Tiled update variants: loads in flight per thread and test-before-set atomics.
using TiledKernel = void (*)(KParams, TileGeometry, const uint2*, uint64_t, uint8_t*, uint32_t*, uint32_t,
                            const uint32_t*, uint8_t*, uint32_t*);
struct TiledVariant {
  TiledKernel fn[2][2];  // [16-bit cells][one tile per row (no range test)]
  int unroll;
  bool check;
};
#define SSE_TILED(U, C, P)                                                                  \
  {{{k_update_tiled<uint8_t, U, C, false, P>, k_update_tiled<uint8_t, U, C, true, P>},       \
    {k_update_tiled<uint16_t, U, C, false, P>, k_update_tiled<uint16_t, U, C, true, P>}}, \
   U, C}
const TiledVariant kTiledVariants[] = {
    SSE_TILED(4, false, false), SSE_TILED(2, false, false), SSE_TILED(8, false, false),
    SSE_TILED(4, true, false),  SSE_TILED(2, true, false),  SSE_TILED(8, true, false),
    SSE_TILED(4, false, true),  SSE_TILED(5, false, true),  SSE_TILED(3, false, true),
};
#undef SSE_TILED
constexpr int kNumTiledVariants = sizeof(kTiledVariants) / sizeof(kTiledVariants[0]);
// Update variants seen by the autotuner: 0 = direct, 1 + v = tiled variant v.
constexpr int kNumUpdateVariants = 1 + kNumTiledVariants;

int launch_update_tiled(sse_handle* h, const uint32_t* d_pairs, uint64_t n, int variant) {
  const uint32_t stamp = stamp_of(h->slice, h->smod);
  const TileGeometry& g = h->tiles;
  const size_t smem = g.piece_bytes / 8 + kRsraQueueBytes;
  const TiledKernel fn = kTiledVariants[variant].fn[h->wide][g.pieces == 1];
  constexpr uint64_t kMaxPairsPerLaunch = 1ull << 30;  // keeps per-group indices in 32 bits
  for (uint64_t done = 0; done < n; done += kMaxPairsPerLaunch) {
    const uint64_t m = std::min(kMaxPairsPerLaunch, n - done);
    fn<<<g.groups * g.tiles, kTiledThreads, smem, h->stream>>>(h->kp, g,
                                                               reinterpret_cast<const uint2*>(d_pairs + 2 * done), m,
                                                               h->sre, h->sle_bits, stamp, h->clock, h->mirror_sre,
                                                               h->mirror_bits);
    SSE_LAUNCHED(h);
  }
  const uint64_t words = h->sle_cells / 32;
  const auto apply = h->wide ? k_apply_bits<uint16_t> : k_apply_bits<uint8_t>;
  // one thread per 16-byte vector of cells (2 or 4 per bitmap word), up to 8 blocks per SM
  const uint64_t vecs = words * (h->wide ? 4 : 2);
  SSE_CUDA(h, launch_pdl(apply, dim3(grid_for(h, vecs, 256, 8)), dim3(256), 0, h->stream, h->sle_bits, h->sle,
                         words, stamp, (const uint32_t*)h->clock));
  SSE_LAUNCHED(h);
  return SSE_OK;
}

// Batches of at least this many pairs use the tiled update in SSE_UPDATE_AUTO mode unless
// the autotuner chose otherwise: the flush of one bitmap per CTA (about r' * row length
// bits per group) must be small against the pairs' own work.
constexpr uint64_t kTiledMinPairs = 1ull << 20;

int launch_variant(sse_handle* h, const uint32_t* d_pairs, uint64_t n, int variant) {
  return variant == 0 ? launch_update_direct(h, d_pairs, n) : launch_update_tiled(h, d_pairs, n, variant - 1);
}

int launch_update_one_way(sse_handle* h, const uint32_t* d_pairs, uint64_t n) {
  const int tiled_variant = h->tuned_variant > 0 ? h->tuned_variant : 1;
  if (h->update_mode == SSE_UPDATE_DIRECT) return launch_variant(h, d_pairs, n, 0);
  if (h->update_mode == SSE_UPDATE_TILED) return launch_variant(h, d_pairs, n, tiled_variant);
  if (n < kTiledMinPairs) return launch_variant(h, d_pairs, n, 0);
  return launch_variant(h, d_pairs, n, h->tuned_variant >= 0 ? h->tuned_variant : tiled_variant);
}

constexpr uint64_t kSwapChunk = 1ull << 24;  // pairs per exchanged chunk (128 MiB)

// Definition 1 counts a host's opposite hosts; SSE_DIR_SRC takes aip = src (the default),
// SSE_DIR_DST aip = dst, SSE_DIR_BOTH both (each pair is scanned in both directions).
int launch_update(sse_handle* h, const uint32_t* d_pairs, uint64_t n) {
  if (h->direction == SSE_DIR_SRC) return launch_update_one_way(h, d_pairs, n);
  if (h->direction == SSE_DIR_BOTH) {
    const int rc = launch_update_one_way(h, d_pairs, n);
    if (rc) return rc;
  }
  if (!h->swap_buf && cudaMalloc(&h->swap_buf, kSwapChunk * 8) != cudaSuccess) {
    cudaGetLastError();
    return SSE_ERR_OOM;
  }
  for (uint64_t done = 0; done < n; done += kSwapChunk) {
    const uint64_t m = std::min(kSwapChunk, n - done);
    k_swap_pairs<<<grid_for(h, m, 256, 8), 256, 0, h->stream>>>(reinterpret_cast<const uint2*>(d_pairs + 2 * done),
                                                                 reinterpret_cast<uint2*>(h->swap_buf), m);
    SSE_LAUNCHED(h);
    const int rc = launch_update_one_way(h, h->swap_buf, m);
    if (rc) return rc;
  }
  return SSE_OK;
}

// Expire/weigh/count pass. mode: bit 0 expire, bit 1 write hot bitmap. Without either
// bit only the SLEA counts are needed and RSRA is skipped.
int launch_close_pass(sse_handle* h, uint32_t* active2, uint32_t mode) {
  const auto fn = h->wide ? k_close<uint16_t> : k_close<uint8_t>;
  fn<<<(unsigned)(h->num_sms * 8), kCloseThreads, 0, h->stream>>>(h->kp, h->sre, h->sle, h->hot_bits, active2,
                                                                  stamp_of(h->slice, h->smod), h->clock,
                                                                  mode ? 1u : 0u, mode,
                                                                  (mode & 2u) ? h->sle_act : nullptr);
  SSE_LAUNCHED(h);
  return SSE_OK;
}

// Moves the handle to the next slice: the device clock on the stream, the host copy now.
int advance_clock(sse_handle* h) {
  k_tick<<<1, 32, 0, h->stream>>>(h->clock, 1, h->smod);
  SSE_LAUNCHED(h);
  h->slice += 1;
  return SSE_OK;
}

// Sorts the first min(n_cand, cap) candidates into cand_out: one cooperative launch (its
// blocks meet at grid barriers when there are more than kSortChunk candidates).
int launch_sort(sse_handle* h) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kSortBlocks);
  cfg.blockDim = dim3(kSortThreads);
  cfg.stream = h->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CloseScratch* sc = h->scratch;
  // up to kSortChunk candidates are placed by the estimate kernel (rank mode)
  SSE_CUDA(h, cudaLaunchKernelEx(&cfg, k_sort_candidates, h->cand, h->cand_alt, h->cand_out,
                                 (const uint32_t*)&sc->n_cand, h->cand_cap, sc->barrier, &sc->error, 1u,
                                 (const uint32_t*)h->sort_ctl));
  SSE_LAUNCHED(h);
  return SSE_OK;
}

}  // namespace

extern "C" {

void sse_params_default(sse_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->r = 5;
  p->q = 17;
  p->delta = 5;
  p->eta = 8;
  p->r2 = 5;
  p->q2 = 17;
  p->delta2 = 16;
  p->eta2 = 1u << 14;
  p->k = 300;
  p->theta = 1024;
  p->stamp_bits = 16;
  p->max_candidates = 1u << 16;
  p->seed = 0;
}

int sse_derive(const sse_params* p, sse_derived* d) {
  if (!p) return SSE_ERR_INVALID_PARAM;
  sse_params q;
  sse_derived dd;
  const int rc = derive_params(*p, q, dd);
  if (rc == SSE_OK && d) *d = dd;
  return rc;
}

const char* sse_strerror(int status) {
  switch (status) {
    case SSE_OK: return "ok";
    case SSE_ERR_INVALID_PARAM: return "invalid parameter or argument";
    case SSE_ERR_OOM: return "out of memory";
    case SSE_ERR_CAPACITY: return "result exceeds buffer capacity";
    case SSE_ERR_MISMATCH: return "estimators differ in parameters or slice";
    case SSE_ERR_CUDA: return "CUDA runtime error";
    case SSE_ERR_TIMEOUT: return "device-side wait timed out";
    case SSE_ERR_STATE: return "call not valid in the current state";
    default: return "unknown status";
  }
}

void sse_destroy(sse_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  for (int b = 0; b < 2; ++b)
    if (h->copy_stream[b]) {
      cudaStreamSynchronize(h->copy_stream[b]);
      cudaStreamDestroy(h->copy_stream[b]);
    }
  for (int b = 0; b < 2; ++b) {
    if (h->stage_dev[b]) cudaFree(h->stage_dev[b]);
    if (h->stage_host[b]) cudaFreeHost(h->stage_host[b]);
    if (h->ev_copied[b]) cudaEventDestroy(h->ev_copied[b]);
    if (h->ev_used[b]) cudaEventDestroy(h->ev_used[b]);
  }
  cudaFree(h->state);
  cudaFree(h->clock);
  cudaFree(h->hot_bits);
  cudaFree(h->sle_bits);
  cudaFree(h->sle_act);
  cudaFree(h->list0);
  cudaFree(h->list1);
  cudaFree(h->tables);
  cudaFree(h->cand);
  cudaFree(h->cand_alt);
  cudaFree(h->cand_out);
  cudaFree(h->est);
  cudaFree(h->flags);
  cudaFree(h->scratch);
  cudaFree(h->query_active2);
  cudaFree(h->est_table);
  cudaFree(h->any2);
  cudaFree(h->any3);
  cudaFree(h->blist);
  cudaFree(h->bcount);
  cudaFree(h->rhfg_tab);
  cudaFree(h->swap_buf);
  if (h->host_scratch) cudaFreeHost(h->host_scratch);
  if (h->close_exec) cudaGraphExecDestroy(h->close_exec);
  if (h->close_g) cudaGraphDestroy(h->close_g);
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  if (h->report_stage) cudaFreeHost(h->report_stage);
  if (h->close_done) cudaEventDestroy(h->close_done);
  delete h;
}

int sse_init(const sse_params* p, void* cuda_stream, sse_handle** out) {
  if (!p || !out) return SSE_ERR_INVALID_PARAM;
  *out = nullptr;
  sse_params q;
  sse_derived d;
  int rc = derive_params(*p, q, d);
  if (rc != SSE_OK) return rc;
  sse_handle* h = new (std::nothrow) sse_handle();
  if (!h) return SSE_ERR_OOM;
  h->p = q;
  h->d = d;
  h->kp = make_kparams(q, d);
  h->smod = stamp_mod(q.stamp_bits);
  h->wide = q.stamp_bits == 16;
  h->sle_cells = (uint64_t)q.r2 * d.row_pitch2;
  h->stream = (cudaStream_t)cuda_stream;
  memset(&h->stats, 0, sizeof(h->stats));
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return SSE_ERR_CUDA;
  }
  h->cand_cap = q.max_candidates;
  const uint64_t state_bytes = d.sre_bytes + d.sle_bytes;
  const uint64_t list_entries = 1ull << q.q;
  bool ok = cudaMalloc(&h->state, state_bytes) == cudaSuccess && cudaMalloc(&h->clock, 256) == cudaSuccess &&
            cudaMalloc(&h->hot_bits, ((uint64_t)q.r << q.q) / 8) == cudaSuccess &&
            cudaMalloc(&h->sle_bits, h->sle_cells / 8) == cudaSuccess &&
            cudaMalloc(&h->sle_act, h->sle_cells / 8 + 8) == cudaSuccess &&  // + a word read past the last row
            cudaMalloc(&h->list0, list_entries * 4) == cudaSuccess &&
            cudaMalloc(&h->list1, list_entries * 4) == cudaSuccess &&
            cudaMalloc(&h->tables, (q.r - 2) * (list_entries / 8)) == cudaSuccess &&
            cudaMalloc(&h->cand, (uint64_t)h->cand_cap * 4) == cudaSuccess &&
            cudaMalloc(&h->cand_alt, (uint64_t)h->cand_cap * 4) == cudaSuccess &&
            cudaMalloc(&h->cand_out, (uint64_t)h->cand_cap * 4) == cudaSuccess &&
            cudaMalloc(&h->est, (uint64_t)h->cand_cap * 4) == cudaSuccess &&
            cudaMalloc(&h->flags, (uint64_t)h->cand_cap) == cudaSuccess &&
            cudaMalloc(&h->scratch, sizeof(CloseScratch)) == cudaSuccess &&
            cudaMalloc(&h->query_active2, kMaxRows * 4) == cudaSuccess &&
            cudaMalloc(&h->est_table, (uint64_t)(q.eta2 + 1) * 13 + 16) == cudaSuccess &&
            cudaMallocHost(&h->host_scratch, sizeof(CloseScratch)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    sse_destroy(h);
    return SSE_ERR_OOM;
  }
  h->sre = h->state;
  h->sle = h->state + d.sre_bytes;
  h->sort_ctl = h->clock + 16;  // bytes 64..71 of the clock's 256
  if (q.rhfg_hash == 1) {
    uint32_t tab[1024];
    make_rhfg_tables(q, tab);
    if (cudaMalloc(&h->rhfg_tab, sizeof(tab)) != cudaSuccess ||
        cudaMemcpy(h->rhfg_tab, tab, sizeof(tab), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      sse_destroy(h);
      return SSE_ERR_OOM;
    }
    h->kp.tab = h->rhfg_tab;
  }
  h->tiles = make_tiles(q, d, h->num_sms);
  {  // the candidate sort's blocks must all be resident at once (cooperative launch)
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sort_candidates, kSortThreads, 0) != cudaSuccess ||
        (uint64_t)per_sm * h->num_sms < kSortBlocks) {
      cudaGetLastError();
      sse_destroy(h);
      return SSE_ERR_CUDA;
    }
  }
  for (int v = 0; v < 4 * kNumTiledVariants; ++v) {
    const TiledKernel fn = kTiledVariants[v / 4].fn[(v >> 1) & 1][v & 1];
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(h->tiles.piece_bytes / 8 + kRsraQueueBytes)) !=
        cudaSuccess) {
      cudaGetLastError();
      sse_destroy(h);
      return SSE_ERR_CUDA;
    }
  }
  // k_join (delta > 5) shared memory: the regrouped row-2 table (2^q bits) up to q = 20, then
  // as much of HSE(1) as fits in the rest of a 216 KiB budget
  {
    const size_t budget = 216u * 1024u;
    const size_t t2_bytes = (size_t)(list_entries / 8);
    h->join_smem_t2 = t2_bytes <= 128u * 1024u ? 1u : 0u;
    const size_t used = h->join_smem_t2 ? t2_bytes : 0;
    h->join_list1_cap = (uint32_t)std::min<uint64_t>(list_entries, (budget - used) / 4);
    h->join_smem = used + (size_t)h->join_list1_cap * 4;
    if (cudaFuncSetAttribute(k_join, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->join_smem) != cudaSuccess) {
      cudaGetLastError();
      sse_destroy(h);
      return SSE_ERR_CUDA;
    }
  }
  // k_join_tiled (delta <= 5): the "any hot" bitmaps of rows 2 and 3 (2^(q-delta) bits each),
  // staged in shared memory when both fit in 64 KiB; as many blocks as fit on the SMs
  if (d.delta <= 5) {
    const size_t any_bytes = (size_t)any_words(q.q, d.delta) * 4;
    if (cudaMalloc(&h->any2, any_bytes) != cudaSuccess || (q.r > 3 && cudaMalloc(&h->any3, any_bytes) != cudaSuccess)) {
      cudaGetLastError();
      sse_destroy(h);
      return SSE_ERR_OOM;
    }
    h->join_stage = 2 * any_bytes <= 64u * 1024u ? 1u : 0u;
    h->join_tiled_smem = (h->join_stage ? 2 * (size_t)any_words_staged(q.q, d.delta) * 4 : 0) + kJoinTiledFixedBytes;
    int per_sm = 0;
    const auto join_fn = h->join_stage ? k_join_tiled<true> : k_join_tiled<false>;
    if (cudaFuncSetAttribute(join_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->join_tiled_smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, join_fn, kJoinTiledThreads, h->join_tiled_smem) !=
            cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      sse_destroy(h);
      return SSE_ERR_CUDA;
    }
    h->join_grid = (uint32_t)(per_sm * h->num_sms);
  }
  if (const uint32_t s = join_down_bits(q, d)) {
    int per_sm = 0;
    const auto fn = kJoinDownFns[q.r - 4];
    if (cudaMalloc(&h->blist, list_entries * 4) != cudaSuccess ||
        cudaMalloc(&h->bcount, ((size_t)1 << (q.q - s)) * 4) != cudaSuccess) {
      cudaGetLastError();
      sse_destroy(h);
      return SSE_ERR_OOM;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kJoinDownThreads, 0) != cudaSuccess || per_sm < 1) {
      cudaGetLastError();
      sse_destroy(h);
      return SSE_ERR_CUDA;
    }
    h->join_down_s = s;
    h->join_down_grid = (uint32_t)(per_sm * h->num_sms);
  }
  const uint32_t first_stamp = stamp_of(0, h->smod);
  if (cudaMemsetAsync(h->clock, 0, 256, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(h->clock, &first_stamp, sizeof(first_stamp), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->state, 0, state_bytes, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->hot_bits, 0, ((uint64_t)q.r << q.q) / 8, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->sle_bits, 0, h->sle_cells / 8, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->scratch, 0, sizeof(CloseScratch), h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cudaGetLastError();
    sse_destroy(h);
    return SSE_ERR_CUDA;
  }
  *out = h;
  return SSE_OK;
}

uint64_t sse_current_slice(const sse_handle* h) { return h ? h->slice : 0; }

uint64_t sse_kernel_launches(const sse_handle* h) { return h ? h->launches : 0; }

const char* sse_cuda_error(const sse_handle* h) {
  return (h && h->cuda_error != cudaSuccess) ? cudaGetErrorName(h->cuda_error) : "";
}

int sse_set_direction(sse_handle* h, int direction) {
  if (!h || direction < SSE_DIR_SRC || direction > SSE_DIR_BOTH) return SSE_ERR_INVALID_PARAM;
  h->direction = direction;
  return SSE_OK;
}

int sse_set_update_mode(sse_handle* h, int mode) {
  if (!h || mode < SSE_UPDATE_AUTO || mode > SSE_UPDATE_TILED) return SSE_ERR_INVALID_PARAM;
  h->update_mode = mode;
  return SSE_OK;
}

int sse_update_variant_count(void) { return kNumUpdateVariants; }

int sse_set_update_variant(sse_handle* h, int variant) {
  if (!h || variant < -1 || variant >= kNumUpdateVariants) return SSE_ERR_INVALID_PARAM;
  h->tuned_variant = variant;
  return SSE_OK;
}

int sse_autotune_update(sse_handle* h, const uint32_t* d_pairs, uint64_t n_pairs, int reps, float* times_ms,
                        int* chosen) {
  if (!h || !d_pairs || n_pairs == 0 || reps < 1 || (reinterpret_cast<uintptr_t>(d_pairs) & 7u))
    return SSE_ERR_INVALID_PARAM;
  if (h->sticky) return h->sticky;
  cudaEvent_t e0, e1;
  SSE_CUDA(h, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(h, cudaGetLastError());
  }
  int best = -1, rc = SSE_OK;
  float best_ms = 0.f;
  for (int v = 0; v < kNumUpdateVariants && rc == SSE_OK; ++v) {
    // the pairs belong to the current slice, so repeating their update changes nothing
    rc = launch_variant(h, d_pairs, n_pairs, v);
    if (rc == SSE_OK && cudaEventRecord(e0, h->stream) != cudaSuccess) rc = fail(h, cudaGetLastError());
    for (int r = 0; r < reps && rc == SSE_OK; ++r) rc = launch_variant(h, d_pairs, n_pairs, v);
    if (rc == SSE_OK && (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
      rc = fail(h, cudaGetLastError());
    if (rc != SSE_OK) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
    if (times_ms) times_ms[v] = ms;
    if (best < 0 || ms < best_ms) {
      best = v;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SSE_OK) return rc;
  h->tuned_variant = best;
  if (chosen) *chosen = best;
  return SSE_OK;
}

int sse_update(sse_handle* h, const uint32_t* d_pairs, uint64_t n_pairs) {
  SSE_NVTX_RANGE("sse_update");
  if (!h) return SSE_ERR_INVALID_PARAM;
  if (h->sticky) return h->sticky;
  if (n_pairs == 0) return SSE_OK;
  if (!d_pairs || (reinterpret_cast<uintptr_t>(d_pairs) & 7u)) return SSE_ERR_INVALID_PARAM;
  return launch_update(h, d_pairs, n_pairs);
}

int sse_update_host(sse_handle* h, const uint32_t* h_pairs, uint64_t n_pairs) {
  SSE_NVTX_RANGE("sse_update_host");
  if (!h) return SSE_ERR_INVALID_PARAM;
  if (h->sticky) return h->sticky;
  if (n_pairs == 0) return SSE_OK;
  if (!h_pairs) return SSE_ERR_INVALID_PARAM;
  constexpr uint64_t kChunk = 1ull << 22;  // pairs per staging buffer (32 MiB)
  if (!h->copy_stream[0]) {
    bool ok = true;
    for (int b = 0; b < 2 && ok; ++b) {
      ok = cudaStreamCreateWithFlags(&h->copy_stream[b], cudaStreamNonBlocking) == cudaSuccess &&
           cudaMalloc(&h->stage_dev[b], kChunk * 8) == cudaSuccess &&
           cudaEventCreateWithFlags(&h->ev_copied[b], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&h->ev_used[b], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
      cudaGetLastError();
      return SSE_ERR_OOM;
    }
  }
  cudaPointerAttributes attr;
  const bool pinned = cudaPointerGetAttributes(&attr, h_pairs) == cudaSuccess && attr.type == cudaMemoryTypeHost;
  cudaGetLastError();
  if (!pinned && !h->stage_host[0]) {
    for (int b = 0; b < 2; ++b)
      if (cudaMallocHost(&h->stage_host[b], kChunk * 8) != cudaSuccess) {
        cudaGetLastError();
        return SSE_ERR_OOM;
      }
  }
  uint64_t done = 0;
  int b = 0;
  while (done < n_pairs) {
    const uint64_t m = std::min<uint64_t>(kChunk, n_pairs - done);
    SSE_CUDA(h, cudaEventSynchronize(h->ev_used[b]));  // buffer b is free again
    const void* src = h_pairs + 2 * done;
    if (!pinned) {
      memcpy(h->stage_host[b], src, m * 8);
      src = h->stage_host[b];
    }
    SSE_CUDA(h, cudaMemcpyAsync(h->stage_dev[b], src, m * 8, cudaMemcpyHostToDevice, h->copy_stream[b]));
    SSE_CUDA(h, cudaEventRecord(h->ev_copied[b], h->copy_stream[b]));
    SSE_CUDA(h, cudaStreamWaitEvent(h->stream, h->ev_copied[b], 0));
    int rc = launch_update(h, h->stage_dev[b], m);
    if (rc) return rc;
    SSE_CUDA(h, cudaEventRecord(h->ev_used[b], h->stream));
    done += m;
    b ^= 1;
  }
  // the caller's buffer may be reused once every copy out of it has finished
  SSE_CUDA(h, cudaEventSynchronize(h->ev_copied[0]));
  SSE_CUDA(h, cudaEventSynchronize(h->ev_copied[1]));
  return SSE_OK;
}

int sse_advance(sse_handle* h) {
  SSE_NVTX_RANGE("sse_advance");
  if (!h) return SSE_ERR_INVALID_PARAM;
  if (h->sticky) return h->sticky;
  SSE_CUDA(h, cudaMemsetAsync(h->scratch, 0, sizeof(CloseScratch), h->stream));
  int rc = launch_close_pass(h, h->scratch->active2, 3u);
  if (rc) return rc;
  h->stats.slice = h->slice;
  return advance_clock(h);
}

}  // extern "C"

namespace {

// The close's estimate table: (eta' + 1) entries of w (FP64), est (FP32) and flags in one
// allocation, built by the last blocks of k_hot_prep from the close's row counts.
EstTable est_table(sse_handle* h, const uint32_t* active2) {
  const uint64_t n = (uint64_t)h->p.eta2 + 1;
  EstTable t;
  t.w = reinterpret_cast<double*>(h->est_table);
  t.est = reinterpret_cast<float*>(h->est_table + n * 8);
  t.flags = h->est_table + n * 12;
  t.active2 = active2;
  t.row_len2 = h->kp.row_len2;
  t.w_theta = h->d.w_theta;
  t.r2 = h->p.r2;
  t.eta2 = h->p.eta2;
  // about two blocks per SM, whole warps each: the table's FP64 divisions and logarithms
  // then run on every SM instead of on n / 256 of them
  const uint64_t per = (n + 2 * (uint64_t)h->num_sms - 1) / (2 * (uint64_t)h->num_sms);
  t.per_block = (uint32_t)std::min<uint64_t>(256, (per + 31) / 32 * 32);
  t.blocks = (uint32_t)((n + t.per_block - 1) / t.per_block);
  return t;
}

// Detection kernels of a close (no host synchronisation, so a CUDA graph can hold them):
// the sorted candidates end in *sorted, estimates and flags in h->est / h->flags, and the
// counters are copied to the pinned h->host_scratch.
int close_enqueue(sse_handle* h, uint32_t** sorted, bool copy_counters = true) {
  CloseScratch* sc = h->scratch;
  SSE_CUDA(h, cudaMemsetAsync(sc, 0, sizeof(CloseScratch), h->stream));
  int rc = launch_close_pass(h, sc->active2, 3u);
  if (rc) return rc;
  {
    const uint64_t words = (1ull << h->p.q) >> 5;
    const bool down = join_down(h);
    const uint32_t s = h->join_down_s;
    const uint32_t n_lists = grid_for(h, words * h->p.r, 256, 4);
    // the join from the top row down reads the plain hot bitmaps and row r-1 by column block;
    // the join from row 0 up reads the regrouped tables and the "any hot" bitmaps
    const uint32_t n_regroup = down ? 0u : grid_for(h, words * (h->p.r - 2), 256, 2);
    const uint32_t n_block = down ? std::min(1u << (h->p.q - s), 1024u) : 0u;
    const uint32_t any_each = (any_words(h->p.q, h->p.delta) + 255) / 256;
    const uint32_t n_any = !down && h->any2 ? (h->any3 ? 2 * any_each : any_each) : 0u;
    const EstTable tab = est_table(h, sc->active2);
    SSE_CUDA(h, launch_pdl(k_hot_prep, dim3(n_lists + n_regroup + n_block + n_any + tab.blocks), dim3(256), 0,
                           h->stream, (const uint32_t*)h->hot_bits, h->p.r, h->p.q, h->p.delta, sc->hot, h->list0,
                           h->list1, sc->n_list, h->tables, down ? nullptr : h->any2, h->any3, n_lists, n_regroup,
                           tab, h->blist, h->bcount, n_block, s));
    SSE_LAUNCHED(h);
    if (down)
      SSE_CUDA(h, launch_pdl(kJoinDownFns[h->p.r - 4], dim3(h->join_down_grid), dim3(kJoinDownThreads), 0, h->stream,
                             h->kp, (const uint32_t*)h->hot_bits, (const uint32_t*)h->list0,
                             (const uint32_t*)sc->n_list, (const uint32_t*)h->blist, (const uint32_t*)h->bcount,
                             h->cand, &sc->n_cand, h->cand_cap, &sc->overflow, &sc->down_pairs));
    else if (h->kp.delta <= 5)
      SSE_CUDA(h, launch_pdl(h->join_stage ? k_join_tiled<true> : k_join_tiled<false>, dim3(h->join_grid),
                             dim3(kJoinTiledThreads), h->join_tiled_smem, h->stream, h->kp,
                             (const uint32_t*)h->tables, (const uint32_t*)h->any2, (const uint32_t*)h->any3,
                             (const uint32_t*)h->list0, (const uint32_t*)h->list1, (const uint32_t*)sc->n_list,
                             h->cand, &sc->n_cand, h->cand_cap, &sc->overflow));
    else
      SSE_CUDA(h, launch_pdl(k_join, dim3(h->num_sms), dim3(kJoinThreads), h->join_smem, h->stream, h->kp,
                             (const uint32_t*)h->hot_bits, (const uint32_t*)h->tables, (const uint32_t*)h->any3,
                             (const uint32_t*)h->list0, (const uint32_t*)h->list1, (const uint32_t*)sc->n_list,
                             h->cand, &sc->n_cand, h->cand_cap, &sc->overflow, h->join_smem_t2,
                             h->join_list1_cap));
    SSE_LAUNCHED(h);
  }
  rc = launch_sort(h);
  if (rc) return rc;
  *sorted = h->cand_out;
  {
    const int grid = grid_for(h, h->cand_cap, 1, 8);
    const auto est_fn = h->wide ? k_estimate<uint16_t, true> : k_estimate<uint8_t, true>;
    // up to kSortChunk candidates: rank mode (h->cand unsorted in, h->cand_out written here)
    const int threads = est_threads(h->p.eta2, h->wide ? 2 : 1);
    SSE_CUDA(h, launch_pdl(est_fn, dim3(threads == kEstThreads ? grid : grid_for(h, h->cand_cap, 1, 2)),
                           dim3(threads), 0, h->stream, h->kp, (const uint8_t*)h->sle, (const uint32_t*)*sorted,
                           (const uint32_t*)&sc->n_cand, h->cand_cap, (const uint32_t*)sc->active2,
                           est_table(h, sc->active2), (const uint32_t*)h->cand, h->cand_out, h->d.w_theta,
                           stamp_of(h->slice, h->smod), (const uint32_t*)h->clock, h->est, h->flags,
                           (double*)nullptr, (uint32_t*)nullptr, (uint32_t*)nullptr, &sc->n_super,
                           (const uint32_t*)h->sle_act));
    SSE_LAUNCHED(h);
  }
  if (copy_counters)
    SSE_CUDA(h, cudaMemcpyAsync(h->host_scratch, sc, sizeof(CloseScratch), cudaMemcpyDeviceToHost, h->stream));
  return SSE_OK;
}

// Waits for an enqueued close and copies its report to the host.
int close_collect(sse_handle* h, const uint32_t* sorted, sse_report* out) {
  SSE_CUDA(h, cudaStreamSynchronize(h->stream));
  const CloseScratch& hs = *h->host_scratch;
  const uint32_t n_found = hs.n_cand;
  const uint32_t n_kept = std::min(n_found, h->cand_cap);
  int status = SSE_OK;
  if (n_found > h->cand_cap) status = SSE_ERR_CAPACITY;
  if (hs.error) status = SSE_ERR_TIMEOUT;
  h->stats.slice = h->slice;
  for (int i = 0; i < kMaxRows; ++i) {
    h->stats.hot[i] = i < (int)h->p.r ? hs.hot[i] : 0;
    h->stats.active2[i] = i < (int)h->p.r2 ? hs.active2[i] : 0;
  }
  h->stats.join_pairs = join_down(h) ? hs.down_pairs : (uint64_t)hs.n_list[0] * hs.n_list[1];
  h->stats.n_candidates = n_found;
  h->stats.n_super = hs.n_super;
  if (out) {
    out->slice = h->slice;
    out->n_candidates = n_found;
    out->n_super = hs.n_super;
    const uint32_t n_copy = std::min(n_kept, out->cap);
    out->truncated = (n_found > n_copy) ? 1u : 0u;
    if (n_kept > out->cap) status = SSE_ERR_CAPACITY;
    if (n_copy) {
      if (out->hosts)
        SSE_CUDA(h, cudaMemcpyAsync(out->hosts, sorted, (uint64_t)n_copy * 4, cudaMemcpyDeviceToHost, h->stream));
      if (out->est)
        SSE_CUDA(h, cudaMemcpyAsync(out->est, h->est, (uint64_t)n_copy * 4, cudaMemcpyDeviceToHost, h->stream));
      if (out->flags)
        SSE_CUDA(h, cudaMemcpyAsync(out->flags, h->flags, n_copy, cudaMemcpyDeviceToHost, h->stream));
      SSE_CUDA(h, cudaStreamSynchronize(h->stream));
    }
  }
  return status;
}

// sse_close_slice replayed from a CUDA graph: the close kernels (which read the stamp from
// the device clock), the copy of the counters and of the first report_stage_n report
// entries into pinned memory, and the clock tick. One launch and one synchronisation per
// slice; reports longer than report_stage_n are completed with direct copies.
// The page-locked, device-mapped report stage written by k_report (allocated once).
int ensure_report_stage(sse_handle* h) {
  if (h->report_stage) return SSE_OK;
  h->report_stage_n = std::min<uint32_t>(h->cand_cap, 8192u);
  SSE_CUDA(h, cudaHostAlloc(&h->report_stage, sizeof(CloseScratch) + (size_t)h->report_stage_n * 9,
                            cudaHostAllocMapped));
  SSE_CUDA(h, cudaHostGetDevicePointer(reinterpret_cast<void**>(&h->report_stage_dev), h->report_stage, 0));
  return SSE_OK;
}

// Report of a finished close from the stage (and, beyond report_stage_n entries, from the
// device buffers): counters into the statistics, entries into out.
int collect_staged(sse_handle* h, const uint32_t* sorted, uint64_t slice, sse_report* out, const uint8_t* stage,
                   uint32_t stage_n);

// Captures the close's kernels into a CUDA graph and instantiates it, once per handle.
int close_graph_build(sse_handle* h) {
  if (!h->close_exec) {
    if (!h->capture_stream) SSE_CUDA(h, cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
    const int rc_stage = ensure_report_stage(h);
    if (rc_stage) return rc_stage;
    const cudaStream_t user = h->stream;
    const uint64_t launches0 = h->launches;
    h->stream = h->capture_stream;
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    int rc = SSE_OK;
    if (e == cudaSuccess) {
      rc = close_enqueue(h, &h->close_sorted, false);
      if (rc == SSE_OK) {
        SSE_CUDA(h, launch_pdl(k_report, dim3(8), dim3(256), 0, h->stream, h->scratch,
                               (const uint32_t*)h->close_sorted, (const float*)h->est, (const uint8_t*)h->flags,
                               h->cand_cap, h->report_stage_n, h->report_stage_dev, h->clock, h->smod));
        SSE_LAUNCHED(h);
      }
      cudaGraph_t g = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
      if (e2 == cudaSuccess && rc == SSE_OK) {
        h->close_g = g;
        e = cudaGraphInstantiate(&h->close_exec, g, 0);
      } else {
        if (g) cudaGraphDestroy(g);
        if (e == cudaSuccess) e = e2;
      }
    }
    h->stream = user;
    h->close_kernels = h->launches - launches0;
    h->launches = launches0;
    if (rc) return rc;
    SSE_CUDA(h, e);
  }
  return SSE_OK;
}

int close_graph_launch(sse_handle* h) {
  const int rc_build = close_graph_build(h);
  if (rc_build) return rc_build;
  if (!h->close_done) SSE_CUDA(h, cudaEventCreateWithFlags(&h->close_done, cudaEventDisableTiming));
  // the report kernel sets this word last (no report is pending, so nothing writes it now)
  *reinterpret_cast<volatile uint32_t*>(h->report_stage + offsetof(CloseScratch, report_done)) = 0u;
  SSE_CUDA(h, cudaGraphLaunch(h->close_exec, h->stream));
  SSE_CUDA(h, cudaEventRecord(h->close_done, h->stream));
  h->launches += h->close_kernels;
  h->close_pending = 1;
  h->close_pending_slice = h->slice;
  h->slice += 1;  // the replay ends with the clock tick
  return SSE_OK;
}

// Waits for the pending replay and fills `out` from the page-locked stage.
int close_graph_collect(sse_handle* h, sse_report* out) {
  h->close_pending = 0;
  // The report is complete once the report kernel's last block has set report_done: poll
  // that word for up to 5 ms (a close takes well under that), which wakes up sooner than a
  // blocking wait; otherwise (a longer close, or a failed one) wait for the stream's event,
  // which also reports errors.
  const volatile uint32_t* done =
      reinterpret_cast<const volatile uint32_t*>(h->report_stage + offsetof(CloseScratch, report_done));
  bool flagged = false;
  const auto t0 = std::chrono::steady_clock::now();
  for (uint32_t i = 0;; ++i) {
    if (*done) {
      flagged = true;
      break;
    }
    if ((i & 1023u) == 1023u && std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(5)) break;
#if defined(__x86_64__)
    __builtin_ia32_pause();
#endif
  }
  if (!flagged) SSE_CUDA(h, cudaEventSynchronize(h->close_done));
  std::atomic_thread_fence(std::memory_order_acquire);  // the report is read after the flag
  return collect_staged(h, h->close_sorted, h->close_pending_slice, out, h->report_stage, h->report_stage_n);
}

int collect_staged(sse_handle* h, const uint32_t* sorted, uint64_t slice, sse_report* out, const uint8_t* stage,
                   uint32_t stage_n) {
  CloseScratch hs;
  memcpy(&hs, stage, sizeof(hs));  // written by k_report before the synchronisation
  const uint32_t n_found = hs.n_cand;
  const uint32_t n_kept = std::min(n_found, h->cand_cap);
  int status = n_found > h->cand_cap ? SSE_ERR_CAPACITY : SSE_OK;
  if (hs.error) status = SSE_ERR_TIMEOUT;
  h->stats.slice = slice;
  for (int i = 0; i < kMaxRows; ++i) {
    h->stats.hot[i] = i < (int)h->p.r ? hs.hot[i] : 0;
    h->stats.active2[i] = i < (int)h->p.r2 ? hs.active2[i] : 0;
  }
  h->stats.join_pairs = join_down(h) ? hs.down_pairs : (uint64_t)hs.n_list[0] * hs.n_list[1];
  h->stats.n_candidates = n_found;
  h->stats.n_super = hs.n_super;
  if (out) {
    out->slice = slice;
    out->n_candidates = n_found;
    out->n_super = hs.n_super;
    const uint32_t n_copy = std::min(n_kept, out->cap);
    out->truncated = (n_found > n_copy) ? 1u : 0u;
    if (n_kept > out->cap) status = SSE_ERR_CAPACITY;
    const uint32_t staged = std::min(n_copy, stage_n);
    const size_t n = stage_n;
    const uint8_t* st = stage + sizeof(CloseScratch);
    if (out->hosts) memcpy(out->hosts, st, (size_t)staged * 4);
    if (out->est) memcpy(out->est, st + n * 4, (size_t)staged * 4);
    if (out->flags) memcpy(out->flags, st + n * 8, staged);
    if (n_copy > staged) {  // the rest, straight from the device
      const uint32_t m = n_copy - staged;
      if (out->hosts)
        SSE_CUDA(h, cudaMemcpyAsync(out->hosts + staged, sorted + staged, (size_t)m * 4, cudaMemcpyDeviceToHost,
                                    h->stream));
      if (out->est)
        SSE_CUDA(h, cudaMemcpyAsync(out->est + staged, h->est + staged, (size_t)m * 4, cudaMemcpyDeviceToHost,
                                    h->stream));
      if (out->flags)
        SSE_CUDA(h, cudaMemcpyAsync(out->flags + staged, h->flags + staged, m, cudaMemcpyDeviceToHost, h->stream));
      SSE_CUDA(h, cudaStreamSynchronize(h->stream));
    }
  }
  return status;
}

int close_slice_graph(sse_handle* h, sse_report* out) {
  const int rc = close_graph_launch(h);
  return rc ? rc : close_graph_collect(h, out);
}

}  // namespace

extern "C" {

int sse_close_slice(sse_handle* h, sse_report* out) {
  SSE_NVTX_RANGE("sse_close_slice");
  if (!h) return SSE_ERR_INVALID_PARAM;
  if (h->sticky) return h->sticky;
  if (h->close_pending) return SSE_ERR_STATE;
  if (h->close_graph) return close_slice_graph(h, out);
  uint32_t* sorted = nullptr;
  int rc = close_enqueue(h, &sorted);
  if (rc) return rc;
  const int status = close_collect(h, sorted, out);
  // a full or out-of-order report still closes the slice (as the graph path does)
  if (status != SSE_OK && status != SSE_ERR_CAPACITY && status != SSE_ERR_TIMEOUT) return status;
  const int rc_tick = advance_clock(h);
  return rc_tick ? rc_tick : status;
}

int sse_close_use_graph(sse_handle* h, int enable) {
  if (!h || h->close_pending) return SSE_ERR_INVALID_PARAM;
  h->close_graph = enable ? 1 : 0;
  return SSE_OK;
}

int sse_set_join(sse_handle* h, int mode) {
  if (!h || mode < SSE_JOIN_AUTO || mode > SSE_JOIN_BACKWARD) return SSE_ERR_INVALID_PARAM;
  if (mode == SSE_JOIN_BACKWARD && !h->join_down_s) return SSE_ERR_INVALID_PARAM;
  if (h->close_pending) return SSE_ERR_STATE;
  if (mode == h->join_mode) return SSE_OK;
  h->join_mode = mode;
  if (h->close_exec) {  // captured with the other join
    cudaGraphExecDestroy(h->close_exec);
    h->close_exec = nullptr;
  }
  if (h->close_g) {
    cudaGraphDestroy(h->close_g);
    h->close_g = nullptr;
  }
  return SSE_OK;
}

int sse_debug_sort_barrier(sse_handle* h, uint32_t spin_limit, uint32_t extra_arrivals) {
  if (!h || extra_arrivals > 1u) return SSE_ERR_INVALID_PARAM;
  if (h->sticky) return h->sticky;
  const uint32_t ctl[2] = {spin_limit, extra_arrivals};
  // stream-ordered with the closes, read by the sort kernel at each replay of the close graph
  SSE_CUDA(h, cudaMemcpyAsync(h->sort_ctl, ctl, sizeof(ctl), cudaMemcpyHostToDevice, h->stream));
  SSE_CUDA(h, cudaStreamSynchronize(h->stream));  // ctl is a stack array
  return SSE_OK;
}

int sse_close_slice_async(sse_handle* h) {
  SSE_NVTX_RANGE("sse_close_slice_async");
  if (!h) return SSE_ERR_INVALID_PARAM;
  if (h->sticky) return h->sticky;
  if (!h->close_graph || h->close_pending) return SSE_ERR_STATE;
  return close_graph_launch(h);
}

int sse_close_slice_wait(sse_handle* h, sse_report* out) {
  SSE_NVTX_RANGE("sse_close_slice_wait");
  if (!h) return SSE_ERR_INVALID_PARAM;
  if (h->sticky) return h->sticky;
  if (!h->close_pending) return SSE_ERR_STATE;
  return close_graph_collect(h, out);
}

int sse_merge(sse_handle* dst, const sse_handle* const* srcs, int n) {
  SSE_NVTX_RANGE("sse_merge");
  if (!dst || !srcs || n < 1 || n > kMaxMergeSources) return SSE_ERR_INVALID_PARAM;
  if (dst->sticky) return dst->sticky;
  MergeSources sre_src, sle_src;
  memset(&sre_src, 0, sizeof(sre_src));
  memset(&sle_src, 0, sizeof(sle_src));
  for (int j = 0; j < n; ++j) {
    const sse_handle* s = srcs[j];
    if (!s || s == dst) return SSE_ERR_INVALID_PARAM;
    if (memcmp(&s->p, &dst->p, sizeof(sse_params)) != 0 || s->slice != dst->slice || s->device != dst->device)
      return SSE_ERR_MISMATCH;
    sre_src.ptr[j] = s->sre;
    sle_src.ptr[j] = s->sle;
  }
  const uint32_t cs = stamp_of(dst->slice, dst->smod);
  const auto merge_fn = dst->wide ? k_merge<uint16_t> : k_merge<uint8_t>;
  const uint64_t n16_sre = dst->d.sre_bytes / 16, n16_sle = dst->d.sle_bytes / 16;
  merge_fn<<<grid_for(dst, n16_sre, 256, 8), 256, 0, dst->stream>>>(dst->sre, sre_src, n, n16_sre, cs, dst->clock);
  SSE_LAUNCHED(dst);
  merge_fn<<<grid_for(dst, n16_sle, 256, 8), 256, 0, dst->stream>>>(dst->sle, sle_src, n, n16_sle, cs, dst->clock);
  SSE_LAUNCHED(dst);
  return SSE_OK;
}

int sse_query(sse_handle* h, const uint32_t* d_hosts, uint32_t n, float* d_est, uint8_t* d_flags, uint32_t* d_hist) {
  SSE_NVTX_RANGE("sse_query");
  if (!h) return SSE_ERR_INVALID_PARAM;
  if (h->sticky) return h->sticky;
  if (n == 0) return SSE_OK;
  if (!d_hosts || !d_est) return SSE_ERR_INVALID_PARAM;
  SSE_CUDA(h, cudaMemsetAsync(h->query_active2, 0, kMaxRows * 4, h->stream));
  int rc = launch_close_pass(h, h->query_active2, 0u);  // count only
  if (rc) return rc;
  const int grid = grid_for(h, n, 1, 16);
  const auto est_fn = h->wide ? k_estimate<uint16_t> : k_estimate<uint8_t>;
  est_fn<<<grid, est_threads(h->p.eta2, h->wide ? 2 : 1), 0, h->stream>>>(h->kp, h->sle, d_hosts, nullptr, n,
                                                                         h->query_active2, EstTable{},
                                                      nullptr, nullptr, h->d.w_theta, stamp_of(h->slice, h->smod), h->clock, d_est, d_flags, nullptr,
                                                      nullptr, d_hist, nullptr, nullptr);
  SSE_LAUNCHED(h);
  return SSE_OK;
}

int sse_get_stats(sse_handle* h, sse_stats* out) {
  if (!h || !out) return SSE_ERR_INVALID_PARAM;
  SSE_CUDA(h, cudaStreamSynchronize(h->stream));
  *out = h->stats;
  return SSE_OK;
}

int sse_get_hot_bitmap(sse_handle* h, uint32_t* h_bits, size_t cap_bytes) {
  if (!h || !h_bits) return SSE_ERR_INVALID_PARAM;
  const size_t bytes = ((size_t)h->p.r << h->p.q) / 8;
  if (cap_bytes < bytes) return SSE_ERR_INVALID_PARAM;
  SSE_CUDA(h, cudaMemcpyAsync(h_bits, h->hot_bits, bytes, cudaMemcpyDeviceToHost, h->stream));
  SSE_CUDA(h, cudaStreamSynchronize(h->stream));
  return SSE_OK;
}

int sse_read_stamps(sse_handle* h, uint8_t* h_sre, size_t sre_cap, uint8_t* h_sle, size_t sle_cap) {
  if (!h) return SSE_ERR_INVALID_PARAM;
  if ((h_sre && sre_cap < h->d.sre_bytes) || (h_sle && sle_cap < h->d.sle_bytes)) return SSE_ERR_CAPACITY;
  if (h_sre) SSE_CUDA(h, cudaMemcpyAsync(h_sre, h->sre, h->d.sre_bytes, cudaMemcpyDeviceToHost, h->stream));
  if (h_sle) SSE_CUDA(h, cudaMemcpyAsync(h_sle, h->sle, h->d.sle_bytes, cudaMemcpyDeviceToHost, h->stream));
  SSE_CUDA(h, cudaStreamSynchronize(h->stream));
  return SSE_OK;
}

namespace {
struct StateHeader {
  uint64_t magic;
  uint32_t version, pad;
  sse_params p;
  uint64_t slice;
  uint64_t sre_bytes, sle_bytes;
};
constexpr uint64_t kMagic = 0x3130455453534553ull;  // "SESSTE01"
}  // namespace

int sse_export_state(sse_handle* h, void* h_buf, size_t cap, size_t* used) {
  if (!h || !used) return SSE_ERR_INVALID_PARAM;
  const size_t total = sizeof(StateHeader) + h->d.sre_bytes + h->d.sle_bytes;
  *used = total;
  if (!h_buf) return SSE_OK;
  if (cap < total) return SSE_ERR_CAPACITY;
  StateHeader hd;
  memset(&hd, 0, sizeof(hd));
  hd.magic = kMagic;
  hd.version = SSE_VERSION;
  hd.p = h->p;
  hd.slice = h->slice;
  hd.sre_bytes = h->d.sre_bytes;
  hd.sle_bytes = h->d.sle_bytes;
  memcpy(h_buf, &hd, sizeof(hd));
  uint8_t* body = static_cast<uint8_t*>(h_buf) + sizeof(hd);
  SSE_CUDA(h, cudaMemcpyAsync(body, h->state, h->d.sre_bytes + h->d.sle_bytes, cudaMemcpyDeviceToHost, h->stream));
  SSE_CUDA(h, cudaStreamSynchronize(h->stream));
  return SSE_OK;
}

int sse_import_state(sse_handle* h, const void* h_buf, size_t n) {
  if (!h || !h_buf || n < sizeof(StateHeader)) return SSE_ERR_INVALID_PARAM;
  StateHeader hd;
  memcpy(&hd, h_buf, sizeof(hd));
  if (hd.magic != kMagic || hd.version != SSE_VERSION) return SSE_ERR_INVALID_PARAM;
  if (memcmp(&hd.p, &h->p, sizeof(sse_params)) != 0 || hd.sre_bytes != h->d.sre_bytes ||
      hd.sle_bytes != h->d.sle_bytes)
    return SSE_ERR_MISMATCH;
  if (n < sizeof(hd) + hd.sre_bytes + hd.sle_bytes) return SSE_ERR_INVALID_PARAM;
  const uint8_t* body = static_cast<const uint8_t*>(h_buf) + sizeof(hd);
  const uint32_t stamp = stamp_of(hd.slice, h->smod);
  SSE_CUDA(h, cudaMemcpyAsync(h->state, body, hd.sre_bytes + hd.sle_bytes, cudaMemcpyHostToDevice, h->stream));
  SSE_CUDA(h, cudaMemcpyAsync(h->clock, &stamp, sizeof(stamp), cudaMemcpyHostToDevice, h->stream));
  SSE_CUDA(h, cudaStreamSynchronize(h->stream));
  h->slice = hd.slice;
  return SSE_OK;
}

int sse_sync(sse_handle* h) {
  if (!h) return SSE_ERR_INVALID_PARAM;
  if (h->sticky) return h->sticky;
  SSE_CUDA(h, cudaStreamSynchronize(h->stream));
  SSE_CUDA(h, cudaGetLastError());
  return SSE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Allocation-free query. Some callers cannot allocate device memory at all: for example a
// packet-processing process that receives fixed, pre-sized device buffers from its host
// framework and may not call the CUDA allocator (an allocation can synchronise the device
// and stall the data path), so it cannot create a handle. sse_query_noalloc() serves them:
// the caller passes the SLEA stamps, the hosts and the output buffers; the only scratch the
// query needs (one active-cell counter per SLEA row) lives in the file-scope device array
// below, which every GPU that loads this library holds until the process exits.
namespace {

constexpr int kNoAllocMaxRows = 16;  // scratch capacity: one counter per SLEA row
static __device__ __align__(256) uint32_t g_noalloc_row_counts[kNoAllocMaxRows];
// Parameter validation already caps r' at kMaxRows, so every valid estimator fits.
static_assert(kNoAllocMaxRows >= kMaxRows, "the scratch array must hold a counter for every SLEA row");

constexpr int kNoAllocMaxDevices = 64;
// Device address of the array, per device. Atomic: two host threads may make their first
// call on a device at the same time; both look up the same address, either store wins.
std::atomic<uint32_t*> g_noalloc_ptr[kNoAllocMaxDevices];

// First call on a device: look up the array's device address with that device current.
// The host-side name of the array is only a stand-in and must never reach a kernel.
int noalloc_scratch(uint32_t** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
    cudaGetLastError();
    return SSE_ERR_CUDA;
  }
  uint32_t* cached = g_noalloc_ptr[dev].load(std::memory_order_acquire);
  if (!cached) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_row_counts) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return SSE_ERR_CUDA;
    }
    cached = static_cast<uint32_t*>(ptr);
    g_noalloc_ptr[dev].store(cached, std::memory_order_release);
  }
  *out = cached;
  return SSE_OK;
}

}  // namespace

extern "C" int sse_query_noalloc(const sse_params* p, const uint8_t* d_sle, uint64_t slice, const uint32_t* d_hosts,
                                 uint32_t n, float* d_est, uint8_t* d_flags, void* cuda_stream) {
  if (!p) return SSE_ERR_INVALID_PARAM;
  sse_params q;
  sse_derived d;
  const int rc = derive_params(*p, q, d);
  if (rc != SSE_OK) return rc;
  if (q.r2 > (uint32_t)kNoAllocMaxRows) return SSE_ERR_INVALID_PARAM;  // beyond the scratch array (see static_assert)
  if (q.stamp_bits != 8) return SSE_ERR_INVALID_PARAM;                // 8-bit stamps only
  if (n == 0) return SSE_OK;
  if (!d_sle || !d_hosts || !d_est || (reinterpret_cast<uintptr_t>(d_sle) & 15u)) return SSE_ERR_INVALID_PARAM;
  uint32_t* counts = nullptr;
  if (noalloc_scratch(&counts) != SSE_OK) return SSE_ERR_CUDA;
  int num_sms = 148, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return SSE_ERR_CUDA;
  }
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  const KParams kp = make_kparams(q, d);
  // the counters still hold the previous call's totals: clear them first
  if (cudaMemsetAsync(counts, 0, kNoAllocMaxRows * sizeof(uint32_t), stream) != cudaSuccess) {
    cudaGetLastError();
    return SSE_ERR_CUDA;
  }
  k_close<uint8_t><<<(unsigned)(num_sms * 8), kCloseThreads, 0, stream>>>(
      kp, nullptr, const_cast<uint8_t*>(d_sle), nullptr, counts, stamp_of(slice), nullptr, 0u, 0u, nullptr);
  if (cudaGetLastError() != cudaSuccess) return SSE_ERR_CUDA;
  uint64_t grid = std::min<uint64_t>((uint64_t)n, (uint64_t)num_sms * 16);
  k_estimate<uint8_t><<<(unsigned)grid, est_threads(q.eta2, 1), 0, stream>>>(
      kp, d_sle, d_hosts, nullptr, n, counts, EstTable{}, nullptr, nullptr, d.w_theta, stamp_of(slice), nullptr, d_est,
      d_flags, nullptr, nullptr, nullptr, nullptr, nullptr);
  if (cudaGetLastError() != cudaSuccess) return SSE_ERR_CUDA;
  return SSE_OK;
}

// ---------------------------------------------------------------------------------------
// Multi-router batches: R router estimators and one global estimator advanced together.
struct sse_batch {
  int n = 0;
  sse_params p;
  sse_derived d;
  cudaStream_t stream = nullptr;  // owned; graphs are captured on it
  sse_handle* router[kMaxRouters] = {};
  sse_handle* global = nullptr;
  uint64_t capacity = 0;      // pairs per router input buffer
  uint32_t* inputs = nullptr; // n * capacity pairs
  RouterInputs* d_in = nullptr;      // per-step input pointers and counts (device)
  RouterInputs* h_in[2] = {};        // pinned copies, one per step parity
  uint8_t* stage[2] = {};            // page-locked, mapped report stages, one per step parity
  uint8_t* stage_dev[2] = {};
  uint32_t stage_n = 0;              // report entries per stage (the candidate capacity)
  cudaEvent_t done[2] = {};          // recorded after each step, per parity
  uint64_t issued = 0;               // steps launched
  int pending = 0;                   // launched steps whose report is not collected (<= 2)
  struct Pending {
    uint64_t slice;
    int mode;
  } pend[2] = {};
  uint32_t* tile_next = nullptr;
  uint32_t item_pairs = 1u << 20;
  int unroll = 4;
  RouterTable rt;
  int use_graph = 1;
  int mode = SSE_BATCH_DETECT;
  cudaGraph_t graph[12] = {};    // one captured step per (mode, routers expire, parity)
  cudaGraphExec_t exec[12] = {};
  bool expire_now = false;       // this step expires the routers' old cells
  uint32_t since_expire = 0;     // steps since the routers were last expired
  uint32_t* sorted = nullptr;     // global's sorted candidates (fixed per configuration)
  uint64_t kernels_per_step[6] = {};
  uint64_t launches = 0;
};

namespace {

using RoutersKernel = void (*)(KParams, TileGeometry, RouterTable, int, uint64_t, const RouterInputs*, uint32_t,
                               uint32_t*, const uint32_t*, uint8_t*);

void drop_graphs(sse_batch* b) {
  for (int m = 0; m < 12; ++m) {
    if (b->exec[m]) cudaGraphExecDestroy(b->exec[m]);
    if (b->graph[m]) cudaGraphDestroy(b->graph[m]);
    b->exec[m] = nullptr;
    b->graph[m] = nullptr;
  }
}

RoutersKernel routers_kernel(int unroll, bool whole) {
  if (whole) return unroll == 2 ? k_update_routers<2, true> : unroll == 8 ? k_update_routers<8, true> : k_update_routers<4, true>;
  return unroll == 2 ? k_update_routers<2, false> : unroll == 8 ? k_update_routers<8, false> : k_update_routers<4, false>;
}

// Update of every router (one persistent launch) and the bitmap apply, on b->stream. In
// detect mode the same writes go to the global estimator too (RSRA stamps directly, SLEA
// through its bitmap), so the global holds the union of the routers' pairs — what merging
// the routers (Algorithms 2 and 7) gives — without reading every router's state.
int batch_enqueue_update(sse_batch* b) {
  sse_handle* g = b->global;
  const TileGeometry& tg = g->tiles;
  SSE_CUDA(g, cudaMemsetAsync(b->tile_next, 0, tg.tiles * sizeof(uint32_t), b->stream));
  const uint32_t per_tile = std::max<uint32_t>(1u, (uint32_t)g->num_sms / tg.tiles);
  routers_kernel(b->unroll, tg.pieces == 1)<<<tg.tiles * per_tile, kTiledThreads, tg.piece_bytes / 8 + kRsraQueueBytes,
                                               b->stream>>>(
      g->kp, tg, b->rt, b->n, g->d.sre_bytes, b->d_in, b->item_pairs, b->tile_next, g->clock,
      b->mode == SSE_BATCH_DETECT ? g->sre : nullptr);
  SSE_LAUNCHED(g);
  const uint64_t words = g->d.sle_bytes / 32;
  const dim3 grid(grid_for(g, words, 256, 2), b->n);
  const bool global = b->mode == SSE_BATCH_DETECT;
  k_apply_routers<<<grid, 256, 0, b->stream>>>(b->rt, g->d.sre_bytes, words, g->clock, global ? g->sle_bits : nullptr);
  SSE_LAUNCHED(g);
  if (global) {
    k_apply_bits<uint8_t><<<grid_for(g, 2 * words, 256, 8), 256, 0, b->stream>>>(g->sle_bits, g->sle, words, 0u, g->clock);
    SSE_LAUNCHED(g);
  }
  return SSE_OK;
}

// One slice: update all routers, merge them (with their expiry) into the global estimator,
// detect on it, and advance every clock (SSE_BATCH_DETECT); see sse_batch_set_mode for the
// other modes.
int batch_enqueue_step(sse_batch* b, int parity) {
  sse_handle* g = b->global;
  int rc = batch_enqueue_update(b);
  if (rc || b->mode == SSE_BATCH_SCAN) return rc;
  const bool detect = b->mode == SSE_BATCH_DETECT;
  if (b->expire_now) {  // reset the routers' cells that left the window (no merge: see above)
    const uint64_t n16 = (g->d.sre_bytes + g->d.sle_bytes) / 16;
    k_merge_routers<<<grid_for(g, n16, 256, 8), 256, 0, b->stream>>>(nullptr, b->rt, b->n, n16, g->p.k, g->clock);
    SSE_LAUNCHED(g);
  }
  if (detect) {
    rc = close_enqueue(g, &b->sorted, false);
    if (rc) return rc;
    k_report<<<8, 256, 0, b->stream>>>(g->scratch, b->sorted, g->est, g->flags, g->cand_cap, b->stage_n,
                                       b->stage_dev[parity], nullptr, 0u);
    SSE_LAUNCHED(g);
  }
  ClockList cl;
  for (int r = 0; r < b->n; ++r) cl.c[r] = b->router[r]->clock;
  cl.c[b->n] = g->clock;  // the global clock advances in either mode (the routers read it)
  k_tick_list<<<1, 128, 0, b->stream>>>(cl, b->n + 1);
  SSE_LAUNCHED(g);
  return SSE_OK;
}

}  // namespace

extern "C" {

void sse_batch_destroy(sse_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  for (int r = 0; r < b->n; ++r) sse_destroy(b->router[r]);
  sse_destroy(b->global);
  cudaFree(b->inputs);
  cudaFree(b->d_in);
  cudaFree(b->tile_next);
  for (int i = 0; i < 2; ++i) {
    if (b->h_in[i]) cudaFreeHost(b->h_in[i]);
    if (b->stage[i]) cudaFreeHost(b->stage[i]);
    if (b->done[i]) cudaEventDestroy(b->done[i]);
  }
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

int sse_batch_create(const sse_params* p, int n_routers, uint64_t capacity_pairs, sse_batch** out) {
  if (!p || !out || n_routers < 1 || n_routers > kMaxRouters || capacity_pairs == 0) return SSE_ERR_INVALID_PARAM;
  *out = nullptr;
  sse_params q;
  sse_derived d;
  int rc = derive_params(*p, q, d);
  if (rc) return rc;
  if (q.stamp_bits != 8) return SSE_ERR_INVALID_PARAM;  // batches use 8-bit stamps
  sse_batch* b = new (std::nothrow) sse_batch();
  if (!b) return SSE_ERR_OOM;
  b->n = n_routers;
  b->p = q;
  b->d = d;
  b->capacity = capacity_pairs;
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return SSE_ERR_CUDA;
  }
  for (int r = 0; r < n_routers && rc == SSE_OK; ++r) rc = sse_init(p, b->stream, &b->router[r]);
  if (rc == SSE_OK) rc = sse_init(p, b->stream, &b->global);
  if (rc == SSE_OK) {
    const bool ok = cudaMalloc(&b->inputs, (uint64_t)n_routers * capacity_pairs * 8) == cudaSuccess &&
                    cudaMalloc(&b->d_in, sizeof(RouterInputs)) == cudaSuccess &&
                    cudaMalloc(&b->tile_next, b->global->tiles.tiles * sizeof(uint32_t)) == cudaSuccess &&
                    cudaMallocHost(&b->h_in[0], sizeof(RouterInputs)) == cudaSuccess &&
                    cudaMallocHost(&b->h_in[1], sizeof(RouterInputs)) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      rc = SSE_ERR_OOM;
    }
  }
  if (rc == SSE_OK) {
    for (int v = 0; v < 6; ++v)  // loads in flight 2, 4, 8 x (part of a row, whole row)
      if (cudaFuncSetAttribute(routers_kernel(2 << (v >> 1), v & 1), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(b->global->tiles.piece_bytes / 8 + kRsraQueueBytes)) != cudaSuccess) {
        cudaGetLastError();
        rc = SSE_ERR_CUDA;
      }
  }
  if (rc != SSE_OK) {
    sse_batch_destroy(b);
    return rc;
  }
  memset(&b->rt, 0, sizeof(b->rt));
  for (int r = 0; r < n_routers; ++r) {
    b->rt.state[r] = b->router[r]->state;
    b->rt.gbits[r] = b->router[r]->sle_bits;
  }
  memset(b->h_in[0], 0, sizeof(RouterInputs));
  memset(b->h_in[1], 0, sizeof(RouterInputs));
  // the step's report kernel writes the whole report into the stage of the step's parity,
  // so a step may run while the previous step's report is read
  b->stage_n = b->global->cand_cap;
  for (int i = 0; i < 2 && rc == SSE_OK; ++i) {
    if (cudaHostAlloc(&b->stage[i], sizeof(CloseScratch) + (size_t)b->stage_n * 9, cudaHostAllocMapped) !=
            cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void**>(&b->stage_dev[i]), b->stage[i], 0) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      rc = SSE_ERR_OOM;
    }
  }
  if (rc != SSE_OK) {
    sse_batch_destroy(b);
    return rc;
  }
  *out = b;
  return SSE_OK;
}

uint32_t* sse_batch_input(sse_batch* b, int router) {
  if (!b || router < 0 || router >= b->n) return nullptr;
  return b->inputs + 2 * (uint64_t)router * b->capacity;
}

void* sse_batch_stream(sse_batch* b) { return b ? (void*)b->stream : nullptr; }

int sse_batch_load(sse_batch* b, int router, const uint32_t* pairs, uint64_t n_pairs, int from_host) {
  if (!b || router < 0 || router >= b->n || (!pairs && n_pairs)) return SSE_ERR_INVALID_PARAM;
  if (b->pending) return SSE_ERR_STATE;
  if (n_pairs > b->capacity) return SSE_ERR_CAPACITY;
  if (!n_pairs) return SSE_OK;
  SSE_CUDA(b->global, cudaMemcpyAsync(sse_batch_input(b, router), pairs, n_pairs * 8,
                                      from_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, b->stream));
  SSE_CUDA(b->global, cudaStreamSynchronize(b->stream));
  return SSE_OK;
}

int sse_batch_router(sse_batch* b, int router, sse_handle** out) {
  if (!b || !out || router < 0 || router >= b->n) return SSE_ERR_INVALID_PARAM;
  *out = b->router[router];
  return SSE_OK;
}

int sse_batch_global(sse_batch* b, sse_handle** out) {
  if (!b || !out) return SSE_ERR_INVALID_PARAM;
  *out = b->global;
  return SSE_OK;
}

int sse_batch_use_graph(sse_batch* b, int enable) {
  if (!b) return SSE_ERR_INVALID_PARAM;
  if (b->pending) return SSE_ERR_STATE;
  b->use_graph = enable ? 1 : 0;
  return SSE_OK;
}

int sse_batch_set_mode(sse_batch* b, int mode) {
  if (!b || mode < SSE_BATCH_DETECT || mode > SSE_BATCH_SCAN) return SSE_ERR_INVALID_PARAM;
  if (b->pending) return SSE_ERR_STATE;
  b->mode = mode;
  return SSE_OK;
}

int sse_batch_reset(sse_batch* b) {
  if (!b) return SSE_ERR_INVALID_PARAM;
  if (b->pending) return SSE_ERR_STATE;
  b->since_expire = 0;
  for (int r = 0; r < b->n; ++r) {
    const int rc = sse_reset(b->router[r]);
    if (rc) return rc;
  }
  return sse_reset(b->global);
}

int sse_batch_configure(sse_batch* b, uint32_t item_pairs, int unroll) {
  if (!b || item_pairs < 1024 || item_pairs > (1u << 30) || (unroll != 2 && unroll != 4 && unroll != 8))
    return SSE_ERR_INVALID_PARAM;
  if (b->pending) return SSE_ERR_STATE;
  b->item_pairs = item_pairs;
  b->unroll = unroll;
  drop_graphs(b);  // the captured graphs hold the old launch configuration
  return SSE_OK;
}

}  // extern "C"

namespace {

// Launches one step (inputs from d_pairs) behind any earlier one on the batch's stream and
// returns; batch_collect() waits for the oldest launched step and reads its report. The
// slice bookkeeping is done at launch (it depends on nothing the step computes).
int batch_launch(sse_batch* b, const uint32_t* const* d_pairs, const uint64_t* h_counts) {
  sse_handle* g = b->global;
  if (g->sticky) return g->sticky;
  if (b->pending >= 2) return SSE_ERR_STATE;
  for (int r = 0; r < b->n; ++r) {
    if (b->router[r]->sticky) return b->router[r]->sticky;
    if (h_counts[r] && (!d_pairs[r] || (reinterpret_cast<uintptr_t>(d_pairs[r]) & 7u))) return SSE_ERR_INVALID_PARAM;
  }
  const int parity = (int)(b->issued & 1);
  RouterInputs* in = b->h_in[parity];  // free: the step that last used it has been collected
  for (int r = 0; r < b->n; ++r) {
    in->pairs[r] = reinterpret_cast<const uint2*>(d_pairs[r]);
    in->counts[r] = h_counts[r];
  }
  // A router cell stamped at slice t leaves the window at t + k and would look active again
  // when its stamp comes round at t + 255; expiring the routers every 254 - k slices clears
  // every such cell in between (the global estimator expires its own cells at every close).
  const uint32_t every = g->p.k < 253 ? 254u - g->p.k : 1u;
  b->expire_now = b->mode != SSE_BATCH_SCAN && b->since_expire + 1 >= every;
  SSE_CUDA(g, cudaMemcpyAsync(b->d_in, in, sizeof(RouterInputs), cudaMemcpyHostToDevice, b->stream));
  const int kind = b->mode * 2 + (b->expire_now ? 1 : 0);
  const uint64_t launches0 = g->launches;
  if (b->use_graph) {
    const int m = kind * 2 + parity;
    if (!b->exec[m]) {
      SSE_CUDA(g, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      const int rc = batch_enqueue_step(b, parity);
      cudaGraph_t graph = nullptr;
      const cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
      if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      SSE_CUDA(g, e);
      b->graph[m] = graph;
      SSE_CUDA(g, cudaGraphInstantiate(&b->exec[m], b->graph[m], 0));
      b->kernels_per_step[kind] = g->launches - launches0;
      g->launches = launches0;
    }
    SSE_CUDA(g, cudaGraphLaunch(b->exec[m], b->stream));
  } else {
    const int rc = batch_enqueue_step(b, parity);
    if (rc) return rc;
    b->kernels_per_step[kind] = g->launches - launches0;
    g->launches = launches0;
  }
  SSE_CUDA(g, cudaEventRecord(b->done[parity], b->stream));
  b->launches += b->kernels_per_step[kind];
  b->pend[parity] = sse_batch::Pending{g->slice, b->mode};
  b->issued += 1;
  b->pending += 1;
  if (b->mode != SSE_BATCH_SCAN) {  // otherwise the slice stays open
    b->since_expire = b->expire_now ? 0 : b->since_expire + 1;
    for (int r = 0; r < b->n; ++r) b->router[r]->slice += 1;
    g->slice += 1;
  }
  return SSE_OK;
}

int batch_collect(sse_batch* b, sse_report* out) {
  sse_handle* g = b->global;
  if (b->pending == 0) return SSE_ERR_STATE;
  const int parity = (int)((b->issued - (uint64_t)b->pending) & 1);
  b->pending -= 1;
  SSE_CUDA(g, cudaEventSynchronize(b->done[parity]));
  const sse_batch::Pending& st = b->pend[parity];
  if (st.mode == SSE_BATCH_DETECT) return collect_staged(g, b->sorted, st.slice, out, b->stage[parity], b->stage_n);
  if (out) {
    out->slice = st.slice;
    out->n_candidates = out->n_super = out->truncated = 0;
  }
  return SSE_OK;
}

int batch_step(sse_batch* b, const uint32_t* const* d_pairs, const uint64_t* h_counts, sse_report* out) {
  if (b->pending) return SSE_ERR_STATE;
  const int rc = batch_launch(b, d_pairs, h_counts);
  return rc ? rc : batch_collect(b, out);
}

}  // namespace

extern "C" {

int sse_batch_step(sse_batch* b, const uint64_t* h_counts, sse_report* out) {
  SSE_NVTX_RANGE("sse_batch_step");
  if (!b || !h_counts) return SSE_ERR_INVALID_PARAM;
  const uint32_t* ptrs[kMaxRouters];
  for (int r = 0; r < b->n; ++r) {
    if (h_counts[r] > b->capacity) return SSE_ERR_CAPACITY;
    ptrs[r] = sse_batch_input(b, r);
  }
  return batch_step(b, ptrs, h_counts, out);
}

int sse_batch_step_from(sse_batch* b, const uint32_t* const* d_pairs, const uint64_t* h_counts, sse_report* out) {
  if (!b || !d_pairs || !h_counts) return SSE_ERR_INVALID_PARAM;
  return batch_step(b, d_pairs, h_counts, out);
}

int sse_batch_step_async(sse_batch* b, const uint32_t* const* d_pairs, const uint64_t* h_counts) {
  SSE_NVTX_RANGE("sse_batch_step_async");
  if (!b || !h_counts) return SSE_ERR_INVALID_PARAM;
  const uint32_t* ptrs[kMaxRouters];
  for (int r = 0; r < b->n; ++r) {
    if (!d_pairs && h_counts[r] > b->capacity) return SSE_ERR_CAPACITY;
    ptrs[r] = d_pairs ? d_pairs[r] : sse_batch_input(b, r);
  }
  return batch_launch(b, ptrs, h_counts);
}

int sse_batch_step_wait(sse_batch* b, sse_report* out) {
  if (!b) return SSE_ERR_INVALID_PARAM;
  return batch_collect(b, out);
}

int sse_batch_pending(const sse_batch* b) { return b ? b->pending : 0; }

int sse_batch_tune(sse_batch* b, const uint32_t* const* d_pairs, const uint64_t* h_counts, int reps, float* times_ms,
                   int* chosen) {
  if (!b || !h_counts || reps < 1) return SSE_ERR_INVALID_PARAM;
  if (b->pending) return SSE_ERR_STATE;
  sse_handle* g = b->global;
  for (int r = 0; r < b->n; ++r) {
    if (!d_pairs && h_counts[r] > b->capacity) return SSE_ERR_CAPACITY;
    b->h_in[0]->pairs[r] = reinterpret_cast<const uint2*>(d_pairs ? d_pairs[r] : sse_batch_input(b, r));
    b->h_in[0]->counts[r] = h_counts[r];
  }
  SSE_CUDA(g, cudaMemcpyAsync(b->d_in, b->h_in[0], sizeof(RouterInputs), cudaMemcpyHostToDevice, b->stream));
  const uint32_t items[3] = {1u << 18, 1u << 20, 1u << 22};
  const int unrolls[3] = {2, 4, 8};
  cudaEvent_t e0, e1;
  SSE_CUDA(g, cudaEventCreate(&e0));
  SSE_CUDA(g, cudaEventCreate(&e1));
  int best = -1, rc = SSE_OK;
  float best_ms = 0.f;
  for (int c = 0; c < 9 && rc == SSE_OK; ++c) {
    b->item_pairs = items[c / 3];
    b->unroll = unrolls[c % 3];
    rc = batch_enqueue_update(b);  // the routers' pairs belong to the current slice: idempotent
    if (rc == SSE_OK && cudaEventRecord(e0, b->stream) != cudaSuccess) rc = fail(g, cudaGetLastError());
    for (int r = 0; r < reps && rc == SSE_OK; ++r) rc = batch_enqueue_update(b);
    if (rc == SSE_OK && (cudaEventRecord(e1, b->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
      rc = fail(g, cudaGetLastError());
    if (rc) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
    if (times_ms) times_ms[c] = ms;
    if (best < 0 || ms < best_ms) {
      best = c;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (chosen) *chosen = best;
  return sse_batch_configure(b, items[best / 3], unrolls[best % 3]);
}

uint64_t sse_batch_kernel_launches(const sse_batch* b) { return b ? b->launches : 0; }

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Serving: a request loop over many routers with state resident on the device.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

namespace {

uint64_t estimator_bytes(const sse_params& p, const sse_derived& d) {
  const uint64_t cols = 1ull << p.q;
  return d.sre_bytes + d.sle_bytes + 256 + ((uint64_t)p.r << p.q) / 8 + d.sle_bytes / 8 + 2 * cols * 4 +
         (p.r - 2) * cols / 8 + (uint64_t)p.max_candidates * 13 + sizeof(CloseScratch) + kMaxRows * 4;
}

struct ServerSlot {
  uint32_t* h_pin = nullptr;  // pinned staging
  uint32_t* d_buf = nullptr;  // device staging
  cudaEvent_t done = nullptr; // the update that read d_buf has finished
  cudaEvent_t copied = nullptr;  // the host-to-device copy into d_buf has finished
  bool used = false;
};

struct PendingClose {
  uint64_t slice;
  std::chrono::steady_clock::time_point boundary;
};

struct ReadyReport {
  uint64_t slice;
  uint32_t n_candidates, n_super, truncated;
  int status;
  double latency_ms;
  std::vector<uint32_t> hosts;
  std::vector<float> est;
  std::vector<uint8_t> flags;
};

}  // namespace

struct sse_server {
  sse_params p;
  sse_derived d;
  sse_server_config cfg;
  int n = 0;
  sse_handle* router[kMaxRouters] = {};
  cudaStream_t rstream[kMaxRouters] = {};
  cudaEvent_t ev_router[kMaxRouters] = {};
  sse_handle* global = nullptr;
  cudaStream_t gstream = nullptr;
  cudaStream_t xstream = nullptr;  // the routers' expiry pass, after each close
  cudaEvent_t ev_closed = nullptr;  // the global estimator's close kernels are done
  cudaEvent_t ev_merged = nullptr;  // the routers' expiry pass is done
  RouterTable rt;
  std::vector<ServerSlot> slots;
  size_t next_slot = 0;
  uint64_t cur_slice = 0;
  bool started = false;
  double first_time = 0.0;
  // reporting thread
  std::thread reporter;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<PendingClose> pending;
  std::deque<ReadyReport> ready;
  std::vector<double> latencies;
  bool stop = false;
  int error = SSE_OK;
  std::vector<uint32_t> rep_hosts;
  std::vector<float> rep_est;
  std::vector<uint8_t> rep_flags;
  // counters
  uint64_t requests = 0, pairs = 0, slot_waits = 0, slices_closed = 0;
};

namespace {

void reporter_loop(sse_server* s) {
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    s->cv.wait(lk, [s] { return s->stop || !s->pending.empty(); });
    if (s->pending.empty()) return;  // stop requested and nothing left
    const PendingClose pc = s->pending.front();
    lk.unlock();
    sse_report rep;
    memset(&rep, 0, sizeof(rep));
    rep.cap = (uint32_t)s->rep_hosts.size();
    rep.hosts = s->rep_hosts.data();
    rep.est = s->rep_est.data();
    rep.flags = s->rep_flags.data();
    // the report kernel's page-locked stage (close_graph_collect polls its completion word)
    const int status = close_graph_collect(s->global, &rep);
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - pc.boundary).count();
    ReadyReport rr;
    rr.slice = pc.slice;
    rr.n_candidates = rep.n_candidates;
    rr.n_super = rep.n_super;
    rr.truncated = rep.truncated;
    rr.status = status;
    rr.latency_ms = ms;
    const uint32_t m = std::min(rep.n_candidates, rep.cap);
    rr.hosts.assign(rep.hosts, rep.hosts + m);
    rr.est.assign(rep.est, rep.est + m);
    rr.flags.assign(rep.flags, rep.flags + m);
    lk.lock();
    if (status != SSE_OK && status != SSE_ERR_CAPACITY && s->error == SSE_OK) s->error = status;
    s->latencies.push_back(ms);
    s->ready.push_back(std::move(rr));
    s->pending.pop_front();
    s->slices_closed += 1;
    s->cv.notify_all();
  }
}

// Closes the current slice. Every router's update also wrote the global estimator (its RSRA
// directly, its SLEA through the global's bitmap), so the global estimator already holds the
// merge of the routers (Algorithms 2 and 7: the most recent stamp per cell) and the close
// needs no pass over the routers' state: once the routers' updates are done (each request
// makes the global stream wait for its own), the global's bitmap is applied and the close's
// graph replayed on the global stream (expiry and counts, detection, the report written into
// page-locked host memory, the clock tick). The reporter thread is woken at once. Then, on a
// stream of its own so that it does not delay the report, one pass resets the routers' cells
// that left the window (their next updates wait for it), and the router clocks advance. At
// most one close is in flight; the reporter owns the global estimator's report fields until
// it has collected the report.
int server_close_slice(sse_server* s) {
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv.wait(lk, [s] { return s->pending.empty(); });
    if (s->error) return s->error;
  }
  sse_handle* g = s->global;
  const auto boundary = std::chrono::steady_clock::now();
  const uint64_t words = g->sle_cells / 32;
  k_apply_bits<uint8_t><<<grid_for(g, 2 * words, 256, 8), 256, 0, s->gstream>>>(g->sle_bits, g->sle, words, 0u, g->clock);
  SSE_LAUNCHED(g);
  const int rc = close_graph_launch(g);  // advances g->slice; the graph ticks the global clock
  if (rc) return rc;
  SSE_CUDA(g, cudaEventRecord(s->ev_closed, s->gstream));
  {  // the reporter starts waiting for the report now, while the routers' work is enqueued
    std::lock_guard<std::mutex> lk(s->mu);
    s->pending.push_back(PendingClose{s->cur_slice, boundary});
  }
  s->cv.notify_all();
  // the routers' expiry at this slice's stamp (router clocks tick only after it)
  const uint64_t n16 = (g->d.sre_bytes + g->d.sle_bytes) / 16;
  SSE_CUDA(g, cudaStreamWaitEvent(s->xstream, s->ev_closed, 0));
  k_merge_routers<<<grid_for(g, n16, 256, 8), 256, 0, s->xstream>>>(nullptr, s->rt, s->n, n16, g->p.k,
                                                                     s->router[0]->clock);
  SSE_LAUNCHED(g);
  SSE_CUDA(g, cudaEventRecord(s->ev_merged, s->xstream));
  for (int r = 0; r < s->n; ++r) {
    sse_handle* h = s->router[r];
    SSE_CUDA(h, cudaStreamWaitEvent(s->rstream[r], s->ev_merged, 0));
    k_tick<<<1, 32, 0, s->rstream[r]>>>(h->clock, 1);
    SSE_LAUNCHED(h);
    h->slice += 1;
  }
  s->cur_slice += 1;
  return SSE_OK;
}

}  // namespace

extern "C" {

void sse_server_config_default(sse_server_config* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->n_routers = 32;
  c->slots = 16;
  c->slot_pairs = 1u << 22;
  c->memory_budget = 40ull << 30;
  c->slice_seconds = (double)(1u << 26) / 2e9;
}

void sse_server_destroy(sse_server* s) {
  if (!s) return;
  if (s->reporter.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv.notify_all();
    s->reporter.join();
  }
  for (int r = 0; r < s->n; ++r) {
    if (s->rstream[r]) cudaStreamSynchronize(s->rstream[r]);
    sse_destroy(s->router[r]);
    if (s->ev_router[r]) cudaEventDestroy(s->ev_router[r]);
  }
  if (s->gstream) cudaStreamSynchronize(s->gstream);
  if (s->xstream) cudaStreamSynchronize(s->xstream);
  sse_destroy(s->global);
  for (ServerSlot& sl : s->slots) {
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.copied) cudaEventDestroy(sl.copied);
    cudaFree(sl.d_buf);
    if (sl.h_pin) cudaFreeHost(sl.h_pin);
  }
  if (s->ev_merged) cudaEventDestroy(s->ev_merged);
  if (s->ev_closed) cudaEventDestroy(s->ev_closed);
  for (int r = 0; r < s->n; ++r)
    if (s->rstream[r]) cudaStreamDestroy(s->rstream[r]);
  if (s->gstream) cudaStreamDestroy(s->gstream);
  if (s->xstream) cudaStreamDestroy(s->xstream);
  delete s;
}

int sse_server_create(const sse_params* p, const sse_server_config* cfg, sse_server** out) {
  if (!p || !cfg || !out || cfg->n_routers < 1 || cfg->n_routers > (uint32_t)kMaxRouters || cfg->slots < 1 ||
      cfg->slot_pairs < 1024 || !(cfg->slice_seconds > 0.0))
    return SSE_ERR_INVALID_PARAM;
  *out = nullptr;
  sse_params q;
  sse_derived d;
  int rc = derive_params(*p, q, d);
  if (rc) return rc;
  if (q.stamp_bits != 8) return SSE_ERR_INVALID_PARAM;  // the server uses 8-bit stamps
  // admission by memory budget: every router's estimator, the global one and the staging
  const uint64_t need = (cfg->n_routers + 1) * estimator_bytes(q, d) + (uint64_t)cfg->slots * cfg->slot_pairs * 8;
  if (need > cfg->memory_budget) return SSE_ERR_OOM;
  sse_server* s = new (std::nothrow) sse_server();
  if (!s) return SSE_ERR_OOM;
  s->p = q;
  s->d = d;
  s->cfg = *cfg;
  s->n = (int)cfg->n_routers;
  bool ok = cudaStreamCreateWithFlags(&s->gstream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&s->xstream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&s->ev_closed, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&s->ev_merged, cudaEventDisableTiming) == cudaSuccess;
  for (int r = 0; r < s->n && ok; ++r)
    ok = cudaStreamCreateWithFlags(&s->rstream[r], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&s->ev_router[r], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    sse_server_destroy(s);
    return SSE_ERR_CUDA;
  }
  for (int r = 0; r < s->n && rc == SSE_OK; ++r) rc = sse_init(p, s->rstream[r], &s->router[r]);
  if (rc == SSE_OK) rc = sse_init(p, s->gstream, &s->global);
  if (rc == SSE_OK) {
    s->slots.resize(cfg->slots);
    for (ServerSlot& sl : s->slots) {
      if (cudaMallocHost(&sl.h_pin, cfg->slot_pairs * 8) != cudaSuccess ||
          cudaMalloc(&sl.d_buf, cfg->slot_pairs * 8) != cudaSuccess ||
          cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&sl.copied, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        rc = SSE_ERR_OOM;
        break;
      }
    }
  }
  if (rc != SSE_OK) {
    sse_server_destroy(s);
    return rc;
  }
  memset(&s->rt, 0, sizeof(s->rt));
  for (int r = 0; r < s->n; ++r) {
    s->rt.state[r] = s->router[r]->state;
    s->rt.gbits[r] = s->router[r]->sle_bits;
    // every write of a router's updates goes to the global estimator as well
    s->router[r]->mirror_sre = s->global->sre;
    s->router[r]->mirror_sle = s->global->sle;
    s->router[r]->mirror_bits = s->global->sle_bits;
  }
  s->rep_hosts.resize(q.max_candidates);
  s->rep_est.resize(q.max_candidates);
  s->rep_flags.resize(q.max_candidates);
  // the global estimator's close graph, captured now rather than at the first boundary
  rc = close_graph_build(s->global);
  if (rc != SSE_OK) {
    sse_server_destroy(s);
    return rc;
  }
  s->reporter = std::thread(reporter_loop, s);
  *out = s;
  return SSE_OK;
}

int sse_server_submit(sse_server* s, uint32_t router, double t_arrival, const uint32_t* h_pairs, uint64_t n_pairs) {
  if (!s || router >= (uint32_t)s->n || (!h_pairs && n_pairs) || !(t_arrival >= 0.0)) return SSE_ERR_INVALID_PARAM;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->error) return s->error;
  }
  const uint64_t slice = (uint64_t)(t_arrival / s->cfg.slice_seconds);
  if (slice < s->cur_slice) return SSE_ERR_STATE;  // arrivals must not go back in time
  while (s->cur_slice < slice) {
    const int rc = server_close_slice(s);
    if (rc) return rc;
  }
  sse_handle* h = s->router[router];
  // page-locked caller memory is copied by DMA straight from where it is; the request
  // returns once those copies are done, so the caller may reuse the buffer
  cudaPointerAttributes attr;
  const bool pinned =
      n_pairs && cudaPointerGetAttributes(&attr, h_pairs) == cudaSuccess && attr.type == cudaMemoryTypeHost;
  cudaGetLastError();
  uint64_t done = 0;
  while (done < n_pairs) {
    const uint64_t m = std::min<uint64_t>(s->cfg.slot_pairs, n_pairs - done);
    ServerSlot& sl = s->slots[s->next_slot];
    s->next_slot = (s->next_slot + 1) % s->slots.size();
    if (sl.used) {  // admission: wait until this slot's previous batch has been scanned
      if (cudaEventQuery(sl.done) == cudaErrorNotReady) s->slot_waits += 1;
      SSE_CUDA(h, cudaEventSynchronize(sl.done));
    }
    const void* src = h_pairs + 2 * done;
    if (!pinned) {
      memcpy(sl.h_pin, src, m * 8);
      src = sl.h_pin;
    }
    SSE_CUDA(h, cudaMemcpyAsync(sl.d_buf, src, m * 8, cudaMemcpyHostToDevice, s->rstream[router]));
    SSE_CUDA(h, cudaEventRecord(sl.copied, s->rstream[router]));
    int rc = sse_update(h, sl.d_buf, m);
    if (rc) return rc;
    SSE_CUDA(h, cudaEventRecord(sl.done, s->rstream[router]));
    sl.used = true;
    done += m;
  }
  // the next slice close (on the global stream) waits for this request's updates; the wait is
  // enqueued now, so the boundary itself only launches the close
  if (n_pairs) {
    SSE_CUDA(h, cudaEventRecord(s->ev_router[router], s->rstream[router]));
    SSE_CUDA(h, cudaStreamWaitEvent(s->gstream, s->ev_router[router], 0));
  }
  if (pinned && n_pairs)  // copies on one stream finish in order: the last one covers all
    SSE_CUDA(h, cudaEventSynchronize(s->slots[(s->next_slot + s->slots.size() - 1) % s->slots.size()].copied));
  s->requests += 1;
  s->pairs += n_pairs;
  return SSE_OK;
}

int sse_server_flush(sse_server* s) {
  if (!s) return SSE_ERR_INVALID_PARAM;
  int rc = server_close_slice(s);
  if (rc) return rc;
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv.wait(lk, [s] { return s->pending.empty(); });
  return s->error;
}

int sse_server_poll(sse_server* s, sse_report* out, double* latency_ms) {
  if (!s) return SSE_ERR_INVALID_PARAM;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->ready.empty()) return SSE_ERR_STATE;
  ReadyReport& rr = s->ready.front();
  if (out) {
    out->slice = rr.slice;
    out->n_candidates = rr.n_candidates;
    out->n_super = rr.n_super;
    const uint32_t m = std::min<uint32_t>((uint32_t)rr.hosts.size(), out->cap);
    out->truncated = rr.truncated || m < rr.hosts.size();
    if (out->hosts) memcpy(out->hosts, rr.hosts.data(), m * 4);
    if (out->est) memcpy(out->est, rr.est.data(), m * 4);
    if (out->flags) memcpy(out->flags, rr.flags.data(), m);
  }
  if (latency_ms) *latency_ms = rr.latency_ms;
  const int status = rr.status;
  s->ready.pop_front();
  return status;
}

int sse_server_get_stats(sse_server* s, sse_server_stats* out) {
  if (!s || !out) return SSE_ERR_INVALID_PARAM;
  std::lock_guard<std::mutex> lk(s->mu);
  memset(out, 0, sizeof(*out));
  out->requests = s->requests;
  out->pairs = s->pairs;
  out->slices_closed = s->slices_closed;
  out->slot_waits = s->slot_waits;
  out->current_slice = s->cur_slice;
  std::vector<double> l = s->latencies;
  std::sort(l.begin(), l.end());
  if (!l.empty()) {
    out->latency_p50_ms = l[l.size() / 2];
    out->latency_p99_ms = l[std::min(l.size() - 1, (size_t)(0.99 * l.size()))];
  }
  return SSE_OK;
}

int sse_server_router(sse_server* s, uint32_t router, sse_handle** out) {
  if (!s || !out || router >= (uint32_t)s->n) return SSE_ERR_INVALID_PARAM;
  *out = s->router[router];
  return SSE_OK;
}

int sse_server_global(sse_server* s, sse_handle** out) {
  if (!s || !out) return SSE_ERR_INVALID_PARAM;
  *out = s->global;
  return SSE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Learned correction: features, MLP training and inference.
struct sse_mlp {
  MlpShape s;
  uint32_t max_batch = 0;
  float* wf = nullptr;           // FP32 parameters (optimiser)
  __nv_bfloat16* wb = nullptr;   // BF16 parameters (arithmetic)
  float* g = nullptr;            // gradients
  float* m = nullptr;            // Adam moments
  float* v = nullptr;
  float* partial = nullptr;      // per-CTA gradient shares [max_batch / kTrainSamples][total]
  float* loss_partial = nullptr; // per-CTA loss shares
  float* loss = nullptr;         // device loss accumulator
  float* x_max = nullptr;        // per-feature upper bound of the training data
  float* scratch_x = nullptr;    // query features [max_batch][n_in]
  float* scratch_y = nullptr;    // query outputs [max_batch]
  uint32_t min_active = 0;       // gate of sse_query_learned
  uint32_t* d_step = nullptr;    // Adam steps taken (device)
  float* d_lr = nullptr;         // learning rate of the captured epoch (device)
  uint64_t launches = 0;         // kernels launched by forward / gradients / Adam
  // sse_mlp_train_epoch as one CUDA graph, for a fixed (x, t, n, batch)
  uint32_t* perm = nullptr;      // the epoch's row order, copied from the caller
  uint64_t perm_cap = 0;
  cudaStream_t capture_stream = nullptr;
  cudaGraph_t epoch_g = nullptr;
  cudaGraphExec_t epoch_exec = nullptr;
  const float* key_x = nullptr;
  const float* key_t = nullptr;
  uint32_t key_n = 0, key_batch = 0;
  uint64_t epoch_kernels = 0;
};

extern "C" {

void sse_mlp_destroy(sse_mlp* m) {
  if (!m) return;
  cudaDeviceSynchronize();
  cudaFree(m->wf);
  cudaFree(m->wb);
  cudaFree(m->g);
  cudaFree(m->m);
  cudaFree(m->v);
  cudaFree(m->partial);
  cudaFree(m->loss_partial);
  cudaFree(m->d_step);
  cudaFree(m->d_lr);
  cudaFree(m->perm);
  if (m->epoch_exec) cudaGraphExecDestroy(m->epoch_exec);
  if (m->epoch_g) cudaGraphDestroy(m->epoch_g);
  if (m->capture_stream) cudaStreamDestroy(m->capture_stream);
  cudaFree(m->loss);
  cudaFree(m->x_max);
  cudaFree(m->scratch_x);
  cudaFree(m->scratch_y);
  delete m;
}

int sse_mlp_create(uint32_t n_in, uint32_t hidden, uint32_t max_batch, uint64_t seed, sse_mlp** out) {
  if (!out || n_in < 1 || n_in > (uint32_t)kMaxIn || hidden < 1 || hidden > (uint32_t)kMaxHidden || max_batch < 1)
    return SSE_ERR_INVALID_PARAM;
  *out = nullptr;
  sse_mlp* m = new (std::nothrow) sse_mlp();
  if (!m) return SSE_ERR_OOM;
  m->s = mlp_shape(n_in, hidden);
  m->max_batch = max_batch;
  if (cudaFuncSetAttribute(k_mlp_grad_partial<64, 18>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(train_smem_floats(m->s) * 4)) != cudaSuccess ||
      cudaFuncSetAttribute(k_mlp_grad_partial<0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(train_smem_floats(m->s) * 4)) != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return SSE_ERR_CUDA;
  }
  const uint32_t T = m->s.total;
  const bool ok = cudaMalloc(&m->wf, T * 4) == cudaSuccess && cudaMalloc(&m->wb, (T + 7) / 8 * 16) == cudaSuccess &&
                  cudaMalloc(&m->g, T * 4) == cudaSuccess && cudaMalloc(&m->m, T * 4) == cudaSuccess &&
                  cudaMalloc(&m->v, T * 4) == cudaSuccess &&
                  cudaMalloc(&m->partial, (uint64_t)((max_batch + kTrainSamples - 1) / kTrainSamples) *
                                              m->s.total * 4) == cudaSuccess &&
                  cudaMalloc(&m->loss_partial, (uint64_t)((max_batch + kTrainSamples - 1) / kTrainSamples) * 4) ==
                      cudaSuccess &&
                  cudaMalloc(&m->d_step, 4) == cudaSuccess && cudaMalloc(&m->d_lr, 4) == cudaSuccess &&
                  cudaMalloc(&m->loss, 4) == cudaSuccess && cudaMalloc(&m->x_max, n_in * 4) == cudaSuccess &&
                  cudaMalloc(&m->scratch_x, (uint64_t)max_batch * n_in * 4) == cudaSuccess &&
                  cudaMalloc(&m->scratch_y, (uint64_t)max_batch * 4) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    sse_mlp_destroy(m);
    return SSE_ERR_OOM;
  }
  // uniform initialisation in +-sqrt(6 / fan_in) (He et al. 2015), zero biases, from SplitMix64(seed)
  std::vector<float> w(T, 0.f);
  uint64_t st = seed;
  auto uni = [&st]() { return (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0); };
  const double a1 = std::sqrt(6.0 / n_in), a2 = std::sqrt(6.0 / hidden);
  for (uint32_t k = m->s.off_w1; k < m->s.off_b1; ++k) w[k] = (float)((2 * uni() - 1) * a1);
  for (uint32_t k = m->s.off_w2; k < m->s.off_b2; ++k) w[k] = (float)((2 * uni() - 1) * a2);
  for (uint32_t k = m->s.off_w3; k < m->s.off_b3; ++k) w[k] = (float)((2 * uni() - 1) * a2);
  std::vector<float> big(n_in, 3.0e38f);
  if (cudaMemcpy(m->wf, w.data(), T * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(m->m, 0, T * 4) != cudaSuccess || cudaMemset(m->v, 0, T * 4) != cudaSuccess ||
      cudaMemset(m->d_step, 0, 4) != cudaSuccess ||
      cudaMemcpy(m->x_max, big.data(), n_in * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    sse_mlp_destroy(m);
    return SSE_ERR_CUDA;
  }
  k_mlp_to_bf16<<<(T + 255) / 256, 256>>>(T, m->wf, m->wb);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    sse_mlp_destroy(m);
    return SSE_ERR_CUDA;
  }
  *out = m;
  return SSE_OK;
}

uint32_t sse_mlp_param_count(const sse_mlp* m) { return m ? m->s.total : 0; }

uint64_t sse_mlp_kernel_launches(const sse_mlp* m) { return m ? m->launches : 0; }

int sse_mlp_set_params(sse_mlp* m, const float* h_params) {
  if (!m || !h_params) return SSE_ERR_INVALID_PARAM;
  if (cudaMemcpy(m->wf, h_params, m->s.total * 4, cudaMemcpyHostToDevice) != cudaSuccess) return SSE_ERR_CUDA;
  k_mlp_to_bf16<<<(m->s.total + 255) / 256, 256>>>(m->s.total, m->wf, m->wb);
  if (cudaMemset(m->m, 0, m->s.total * 4) != cudaSuccess || cudaMemset(m->v, 0, m->s.total * 4) != cudaSuccess ||
      cudaMemset(m->d_step, 0, 4) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess)
    return SSE_ERR_CUDA;
  return SSE_OK;
}

int sse_mlp_get_params(sse_mlp* m, float* h_fp32, uint16_t* h_bf16, float* h_grads) {
  if (!m) return SSE_ERR_INVALID_PARAM;
  if (cudaDeviceSynchronize() != cudaSuccess) return SSE_ERR_CUDA;
  if (h_fp32 && cudaMemcpy(h_fp32, m->wf, m->s.total * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return SSE_ERR_CUDA;
  if (h_bf16 && cudaMemcpy(h_bf16, m->wb, m->s.total * 2, cudaMemcpyDeviceToHost) != cudaSuccess) return SSE_ERR_CUDA;
  if (h_grads && cudaMemcpy(h_grads, m->g, m->s.total * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return SSE_ERR_CUDA;
  return SSE_OK;
}

int sse_mlp_set_feature_max(sse_mlp* m, const float* h_xmax) {
  if (!m || !h_xmax) return SSE_ERR_INVALID_PARAM;
  return cudaMemcpy(m->x_max, h_xmax, m->s.n_in * 4, cudaMemcpyHostToDevice) == cudaSuccess ? SSE_OK : SSE_ERR_CUDA;
}

int sse_mlp_set_gate(sse_mlp* m, uint32_t min_active) {
  if (!m) return SSE_ERR_INVALID_PARAM;
  m->min_active = min_active;
  return SSE_OK;
}

int sse_mlp_forward(sse_mlp* m, const float* d_x, uint32_t n, float* d_y, void* stream) {
  if (!m || (!d_x && n) || (!d_y && n)) return SSE_ERR_INVALID_PARAM;
  if (!n) return SSE_OK;
  const unsigned grid = std::min<uint64_t>((n + 127) / 128, 148 * 8);
  k_mlp_forward<<<grid, 128, m->s.total * 4, (cudaStream_t)stream>>>(m->s, m->wb, d_x, nullptr, n, d_y);
  m->launches += 1;
  return cudaGetLastError() == cudaSuccess ? SSE_OK : SSE_ERR_CUDA;
}

}  // extern "C"

namespace {

// Part 1 of a training step: every CTA's gradient share for the n samples d_rows[0..n).
int mlp_grad_partial(sse_mlp* m, const float* d_x, const float* d_t, const uint32_t* d_rows, uint32_t n,
                     cudaStream_t st, uint32_t* parts) {
  *parts = (n + kTrainSamples - 1) / kTrainSamples;
  const auto fn = (m->s.hidden == 64 && m->s.n_in == 18) ? k_mlp_grad_partial<64, 18> : k_mlp_grad_partial<0, 0>;
  const cudaError_t e = launch_pdl(fn, dim3(*parts), dim3(kTrainThreads), train_smem_floats(m->s) * 4, st, m->s,
                                   (const __nv_bfloat16*)m->wb, d_x, d_t, d_rows, n, m->partial, m->loss_partial);
  m->launches += 1;
  return e == cudaSuccess ? SSE_OK : SSE_ERR_CUDA;
}

// Part 2: Adam step number *d_step + step_off on the summed shares (parts > 0) or on m->g
// (parts == 0); the learning rate from *lr_dev when given, else lr.
int mlp_adam(sse_mlp* m, const float* lr_dev, float lr, uint32_t step_off, cudaStream_t st, uint32_t parts,
             float* d_loss) {
  const cudaError_t e =
      launch_pdl(k_mlp_adam, dim3((m->s.total + kSumParams - 1) / kSumParams), dim3(kSumThreads), 0, st, m->s.total,
                 m->wf, m->wb, m->g, m->m, m->v, lr_dev, lr, (const uint32_t*)m->d_step, step_off, 0.9f, 0.999f,
                 1e-8f, parts ? (const float*)m->partial : nullptr, parts, (const float*)m->loss_partial, d_loss);
  m->launches += 1;
  return e == cudaSuccess ? SSE_OK : SSE_ERR_CUDA;
}

int mlp_step_add(sse_mlp* m, uint32_t n, cudaStream_t st) {
  k_mlp_step_add<<<1, 1, 0, st>>>(m->d_step, n);
  m->launches += 1;
  return cudaGetLastError() == cudaSuccess ? SSE_OK : SSE_ERR_CUDA;
}

}  // namespace

extern "C" {

int sse_mlp_gradients(sse_mlp* m, const float* d_x, const float* d_t, const uint32_t* d_rows, uint32_t n,
                      float* h_loss, void* stream) {
  if (!m || !d_x || !d_t || n < 1 || n > m->max_batch) return SSE_ERR_INVALID_PARAM;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t parts = 0;
  int rc = mlp_grad_partial(m, d_x, d_t, d_rows, n, st, &parts);
  if (rc) return rc;
  k_mlp_reduce_grads<<<(m->s.total + kSumParams - 1) / kSumParams, kSumThreads, 0, st>>>(
      m->s.total, parts, m->partial, m->loss_partial, m->g,
                                                               m->loss);
  m->launches += 1;
  if (cudaGetLastError() != cudaSuccess) return SSE_ERR_CUDA;
  if (h_loss) {
    if (cudaMemcpyAsync(h_loss, m->loss, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return SSE_ERR_CUDA;
  }
  return SSE_OK;
}

int sse_mlp_adam(sse_mlp* m, float lr, void* stream) {
  if (!m || !(lr > 0.f)) return SSE_ERR_INVALID_PARAM;
  const int rc = mlp_adam(m, nullptr, lr, 1, (cudaStream_t)stream, 0, nullptr);
  return rc ? rc : mlp_step_add(m, 1, (cudaStream_t)stream);
}

// One epoch over d_perm (n indices into d_x / d_t), minibatches of `batch`, each one
// gradient-share kernel and one Adam kernel (which sums the shares); returns the last
// minibatch's loss. The minibatch kernels of an epoch are captured once into a CUDA graph
// for a given (d_x, d_t, n, batch) and replayed: the row order is first copied into the
// MLP's own buffer and the learning rate into device memory, and the Adam steps count
// from a device counter, so every replay is a fresh epoch.
int sse_mlp_train_epoch(sse_mlp* m, const float* d_x, const float* d_t, const uint32_t* d_perm, uint32_t n,
                        uint32_t batch, float lr, float* h_loss, void* stream) {
  if (!m || !d_x || !d_t || !d_perm || n < 1 || batch < 1 || batch > m->max_batch || !(lr > 0.f))
    return SSE_ERR_INVALID_PARAM;
  cudaStream_t st = (cudaStream_t)stream;
  if (n > m->perm_cap) {
    cudaFree(m->perm);
    m->perm = nullptr;
    m->perm_cap = 0;
    if (cudaMalloc(&m->perm, (uint64_t)n * 4) != cudaSuccess) {
      cudaGetLastError();
      return SSE_ERR_OOM;
    }
    m->perm_cap = n;
    if (m->epoch_exec) {  // the graph reads the old buffer
      cudaGraphExecDestroy(m->epoch_exec);
      cudaGraphDestroy(m->epoch_g);
      m->epoch_exec = nullptr;
      m->epoch_g = nullptr;
    }
  }
  if (m->epoch_exec && (m->key_x != d_x || m->key_t != d_t || m->key_n != n || m->key_batch != batch)) {
    cudaGraphExecDestroy(m->epoch_exec);
    cudaGraphDestroy(m->epoch_g);
    m->epoch_exec = nullptr;
    m->epoch_g = nullptr;
  }
  if (!m->epoch_exec) {
    if (!m->capture_stream && cudaStreamCreateWithFlags(&m->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
      return SSE_ERR_CUDA;
    const uint64_t launches0 = m->launches;
    cudaStream_t cs = m->capture_stream;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SSE_ERR_CUDA;
    int rc = SSE_OK;
    uint32_t steps = 0;
    for (uint32_t b0 = 0; b0 < n && rc == SSE_OK; b0 += batch, ++steps) {
      const uint32_t nb = std::min(batch, n - b0);
      uint32_t parts = 0;
      rc = mlp_grad_partial(m, d_x, d_t, m->perm + b0, nb, cs, &parts);
      if (rc == SSE_OK) rc = mlp_adam(m, m->d_lr, 0.f, steps + 1, cs, parts, b0 + batch >= n ? m->loss : nullptr);
    }
    if (rc == SSE_OK) rc = mlp_step_add(m, steps, cs);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &g);
    m->epoch_kernels = m->launches - launches0;
    m->launches = launches0;
    if (rc != SSE_OK || e != cudaSuccess || cudaGraphInstantiate(&m->epoch_exec, g, 0) != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      m->epoch_exec = nullptr;
      cudaGetLastError();
      return rc ? rc : SSE_ERR_CUDA;
    }
    m->epoch_g = g;
    m->key_x = d_x;
    m->key_t = d_t;
    m->key_n = n;
    m->key_batch = batch;
  }
  if (cudaMemcpyAsync(m->perm, d_perm, (uint64_t)n * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(m->d_lr, &lr, 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaGraphLaunch(m->epoch_exec, st) != cudaSuccess)
    return SSE_ERR_CUDA;
  m->launches += m->epoch_kernels;
  if (h_loss && cudaMemcpyAsync(h_loss, m->loss, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return SSE_ERR_CUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? SSE_OK : SSE_ERR_CUDA;
}

int sse_features(sse_handle* h, const uint32_t* d_hosts, uint32_t n, float* d_x) {
  if (!h || (!d_hosts && n) || (!d_x && n) || h->wide) return SSE_ERR_INVALID_PARAM;
  if (h->sticky) return h->sticky;
  if (!n) return SSE_OK;
  k_features<<<grid_for(h, n, 1, 16), kFeatThreads, 0, h->stream>>>(h->kp, h->sre, h->sle, d_hosts, n, h->clock, d_x);
  SSE_LAUNCHED(h);
  return SSE_OK;
}

int sse_query_learned(sse_handle* h, sse_mlp* m, const uint32_t* d_hosts, uint32_t n, float* d_est,
                      float* d_est_lc, uint8_t* d_flags) {
  if (!h || !m || (!d_hosts && n) || (!d_est && n) || (!d_est_lc && n) || h->wide) return SSE_ERR_INVALID_PARAM;
  if (m->s.n_in != h->p.k + 2) return SSE_ERR_MISMATCH;
  for (uint32_t b0 = 0; b0 < n; b0 += m->max_batch) {
    const uint32_t nb = std::min(m->max_batch, n - b0);
    int rc = sse_query(h, d_hosts + b0, nb, d_est_lc + b0, d_flags ? d_flags + b0 : nullptr, nullptr);
    if (rc) return rc;
    rc = sse_features(h, d_hosts + b0, nb, m->scratch_x);
    if (rc) return rc;
    rc = sse_mlp_forward(m, m->scratch_x, nb, m->scratch_y, h->stream);
    if (rc) return fail(h, cudaGetLastError());
    k_learned_select<<<(nb + 255) / 256, 256, 0, h->stream>>>(nb, m->s.n_in, m->scratch_x, m->scratch_y,
                                                             d_est_lc + b0, m->x_max, m->min_active, d_est + b0);
    SSE_LAUNCHED(h);
  }
  return SSE_OK;
}

int sse_reset(sse_handle* h) {
  if (!h) return SSE_ERR_INVALID_PARAM;
  if (h->sticky) return h->sticky;
  const uint32_t first = stamp_of(0, h->smod);
  SSE_CUDA(h, cudaMemsetAsync(h->state, 0, h->d.sre_bytes + h->d.sle_bytes, h->stream));
  SSE_CUDA(h, cudaMemsetAsync(h->sle_bits, 0, h->sle_cells / 8, h->stream));
  SSE_CUDA(h, cudaMemsetAsync(h->hot_bits, 0, ((uint64_t)h->p.r << h->p.q) / 8, h->stream));
  SSE_CUDA(h, cudaMemsetAsync(h->scratch, 0, sizeof(CloseScratch), h->stream));
  SSE_CUDA(h, cudaMemcpyAsync(h->clock, &first, 4, cudaMemcpyHostToDevice, h->stream));
  SSE_CUDA(h, cudaStreamSynchronize(h->stream));
  h->slice = 0;
  h->close_pending = 0;  // a pending report is dropped
  memset(&h->stats, 0, sizeof(h->stats));
  return SSE_OK;
}

}  // extern "C"
