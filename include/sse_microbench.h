/*
 * Roof microbenchmarks of the per-packet update's memory units (part of libsse.so).
 *
 * The update of the sliding estimators (Algorithm 3 for the RSRA, Algorithm 6 for the
 * SLEA; Section 3.3 and Section 4 of "Memory efficient distributed sliding super point
 * cardinality estimation by GPU") is integer scatter work: per IP pair it reads 8 bytes and
 * sets r' + r 2^-tau cells at hashed addresses. sse_microbench() measures, on the current
 * device, the peak rate of each unit that work can be bound by, with the update's own
 * access pattern, so that a measured update rate can be stated as a fraction of each roof.
 */
#ifndef SSE_MICROBENCH_H
#define SSE_MICROBENCH_H

#include <stdint.h>

#include "sse.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Bytes of the caller's scratch buffer that sse_microbench() needs at least (1 GiB + 4 KiB). */
#define kSseMicrobenchMinBytes ((uint64_t)(1ull << 30) + 4096ull)
/* Size of the L2-resident region the random stores go to (45 MiB: a core-link estimator). */
#define kSseMicrobenchL2Bytes (45u << 20)

typedef struct sse_microbench_result {
  /* random one-byte stores into a 45 MiB L2-resident region per second: each is one partial
   * L2 sector write, the unit that stamping every cell directly is bound by */
  double l2_random_byte_stores_per_s;
  /* random one-bit atomic ORs into a 128.5 KiB shared-memory bitmap per SM (one CTA of 1024
   * threads per SM), summed over the SMs: the tiled update's row-bitmap writes */
  double smem_random_atomics_per_s;
  /* 128-bit streaming loads (no L1 allocation, L2 evict-first) of a 32 MiB L2-resident
   * region, bytes per second: the pair stream as the tiled update's row CTAs re-read it */
  double l2_stream_load_bytes_per_s;
  /* the same loads over the whole buffer (>= 1 GiB, from HBM), bytes per second */
  double hbm_stream_load_bytes_per_s;
  /* the tiled update's skeleton, pairs per second: 2^25 pairs streamed from HBM by groups of
   * 5 CTAs (one per SLEA row, a 128.5 KiB bitmap each, one CTA per SM), each CTA loading
   * every pair of its group and setting one pseudo-random bit per pair with a shared atomic
   * OR; the method's hashing and sampling left out. The floor of the update's design. */
  double tiled_skeleton_pairs_per_s;
  uint32_t sms;  /* streaming multiprocessors of the device */
  uint32_t reserved;
} sse_microbench_result;

/*
 * Runs the five measurements on cuda_stream (each the best of three timed launches after
 * one untimed launch; about 0.1 s in all) and fills *out. d_buf: caller-owned device
 * scratch of buf_bytes >= kSseMicrobenchMinBytes, 256-byte aligned; its contents are
 * overwritten. Blocks until done. Errors: INVALID_PARAM, CUDA.
 */
SSE_API int sse_microbench(void* d_buf, uint64_t buf_bytes, void* cuda_stream, sse_microbench_result* out);

#ifdef __cplusplus
}
#endif

#endif /* SSE_MICROBENCH_H */
