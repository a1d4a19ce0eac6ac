/*
 * sse.h — C ABI of the B300 sliding super point estimator.
 *
 * Method: "Memory efficient distributed sliding super point cardinality estimation by
 * GPU" (Jie Xu). A host aip is a sliding super point of window W(t,k) (k consecutive
 * time slices, Section 3.1) when it contacted at least theta distinct opposite hosts bip
 * in that window (Definitions 1 and 2). Each estimator keeps
 *   - RSRA, r rows of 2^q sliding rough estimators (SRE) of eta cells (Section 3.3), used
 *     to find candidate super points through the reversible hash group RHFG (Eq. 6-7);
 *   - SLEA, r' rows of 2^q' overlapping sliding linear estimators (SLE) of eta' cells,
 *     adjacent SLEs offset by delta' (Section 4), used to estimate cardinalities.
 * The paper's cells are 16-bit distances incremented every slice; here every cell is an
 * 8-bit time stamp 1 + (slice mod 255) (0 = never set), which needs no per-slice pass:
 * a cell's distance is (current stamp - stamp) mod 255, and a cell is active in the
 * window when that distance is < k. Both encodings give the same active cells and ages.
 *
 * Conventions for every call:
 *   - Return SSE_OK (0) or a negative SSE_ERR_* code; sse_strerror() names it. Nothing
 *     aborts, traps or asserts on the device; an invalid argument changes no state.
 *   - Device pointers ("d_") are caller-owned CUDA global memory, borrowed for the call
 *     and, for asynchronous calls, until the handle's stream reaches the call. Host
 *     pointers ("h_") are caller-owned host memory.
 *   - All device work of a handle is ordered on the CUDA stream given to sse_init().
 *   - An IP pair is two uint32 in host byte order, {src, dst}: src is aip (the host whose
 *     cardinality is measured), dst is bip (its opposite host); n pairs are 2n uint32.
 *   - Handles are not thread-safe; use one handle per thread or serialise calls.
 */
#ifndef SSE_H
#define SSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SSE_VERSION 2

#if defined(__GNUC__)
#define SSE_API __attribute__((visibility("default")))
#else
#define SSE_API
#endif

enum sse_status {
  SSE_OK = 0,
  SSE_ERR_INVALID_PARAM = -1, /* argument or parameter out of its documented range */
  SSE_ERR_OOM = -2,           /* device or pinned host allocation failed */
  SSE_ERR_CAPACITY = -3,      /* a result did not fit its buffer; see the call */
  SSE_ERR_MISMATCH = -4,      /* estimators differ in parameters, seed or slice */
  SSE_ERR_CUDA = -5,          /* a CUDA runtime call failed (sticky for the handle) */
  SSE_ERR_TIMEOUT = -6,       /* a bounded device-side wait gave up */
  SSE_ERR_STATE = -7          /* call not valid in the handle's current state */
};

/* Per-host flags of a report or query. */
enum sse_host_flags {
  SSE_FLAG_SUPER = 1,    /* corrected weight >= w_theta, i.e. estimate >= theta */
  SSE_FLAG_SATURATED = 2 /* SLE full or noise correction undefined; estimate capped */
};

/* Update strategies (sse_set_update_mode). Both give bit-identical estimator state. */
enum sse_update_mode {
  SSE_UPDATE_AUTO = 0,   /* choose per call from the batch size and the parameters */
  SSE_UPDATE_DIRECT = 1, /* every cell write goes straight to the L2-resident estimator */
  SSE_UPDATE_TILED = 2   /* SLEA writes collect in on-chip bitmaps, then merge into it */
};

/* Joins of a slice close (sse_set_join): both find the same candidate hosts. */
enum sse_join_mode {
  SSE_JOIN_AUTO = 0,     /* from the top row down where it applies, else from row 0 up */
  SSE_JOIN_FORWARD = 1,  /* from rows 0, 1, 2 up (Algorithms 4-5) */
  SSE_JOIN_BACKWARD = 2  /* from rows 0 and r-1 down (see sse_set_join) */
};

/*
 * Parameters (symbols of the paper). sse_params_default() fills the values of the
 * paper's experiment (Section 5): r=r'=5, q=q'=17, delta=5, eta=8, delta'=16,
 * eta'=2^14, theta=1024, with k=8.
 *   r      rows of RSRA, 3..16 (candidate tuples start from rows 0, 1, 2: Alg. 4)
 *   q      log2 of SREs per RSRA row, 5..26
 *   delta  RHFG shift (Eq. 6); 0 derives ceil((32-q)/(r-2)). Needs delta < q and
 *          (r-2)*delta + q >= 32 (Section 3.3)
 *   eta    cells per SRE; must be 8 (the paper's eta, one 64-bit word per SRE)
 *   r2     rows of SLEA (r'), 1..16
 *   q2     log2 of SLEs per SLEA row (q'), 0..24
 *   delta2 offset between adjacent SLEs (delta'), 1..eta2 (Section 4, Eq. 10)
 *   eta2   cells per SLE (eta'), a power of two, 32..65536
 *   k      window length in slices, 1..254 (8-bit stamps) or 1..65534 (16-bit stamps)
 *   theta  super point threshold (Definition 2), >= 1
 *   stamp_bits  cell width, 8 or 16: a cell holds the stamp 1 + (t mod (2^w - 1)) of the last
 *          slice t that touched it (0: never), so the window k must be < 2^w - 1. 16-bit cells
 *          double the state; batches, the server, sse_features and sse_query_learned take
 *          8-bit cells only
 *   max_candidates  capacity for candidate hosts per close, 1..2^22
 *   rhfg_hash  hash of RHFG[0] (Eq. 6): 0 = multiply-add-shift like the other functions,
 *          1 = simple tabulation (the family the paper cites for RHFG[0]): four tables of 256
 *          32-bit entries indexed by the address bytes and XORed, entries drawn from
 *          SplitMix64(seed) after the other keys; the top q bits are used
 *   reserved  must be 0
 *   seed   every hash key derives from it (SplitMix64)
 */
typedef struct sse_params {
  uint32_t r, q, delta, eta;
  uint32_t r2, q2, delta2, eta2;
  uint32_t k, theta;
  uint32_t stamp_bits;
  uint32_t max_candidates;
  uint32_t rhfg_hash;
  uint32_t reserved;
  uint64_t seed;
} sse_params;

/* Values derived from sse_params by sse_derive(). */
typedef struct sse_derived {
  uint32_t delta;      /* after derivation */
  uint32_t tau;        /* Eq. 1: smallest tau >= 0 with eta * 2^tau >= theta */
  uint32_t hot_min;    /* an SRE is hot when >= ceil(eta * rho) cells are active, rho = 0.99(1-e^-1/3) */
  uint32_t lg_eta2;    /* log2(eta') */
  uint64_t row_len2;   /* cells of one SLEA row: 2^q' * delta' + eta' - delta' (Section 4) */
  uint64_t row_pitch2; /* bytes between SLEA rows in device memory (row_len2 rounded up) */
  uint64_t sre_bytes;  /* r * 2^q * eta */
  uint64_t sle_bytes;  /* r' * row_pitch2 */
  double w_theta;      /* eta' * (1 - exp(-theta/eta')): est >= theta <=> w^ >= w_theta (Eq. 8) */
} sse_derived;

typedef struct sse_handle sse_handle; /* opaque; owns the estimator's device memory */

/*
 * Result of closing a slice. The caller sets cap and the three array pointers (host
 * memory, each of cap entries, any may be NULL to skip it); the library fills the rest.
 * Candidates are all hosts whose r SREs are hot (Section 3.3), ascending; est is the
 * Algorithm 8 estimate of each (Eq. 8 applied to the corrected weight of Eq. 12), as
 * float; flags are SSE_FLAG_* bits. Super points are the candidates with
 * SSE_FLAG_SUPER (the paper drops candidates whose estimate is below theta).
 */
typedef struct sse_report {
  uint64_t slice;        /* index t of the slice that was closed (window ends at t) */
  uint32_t n_candidates; /* total candidates found (may exceed cap) */
  uint32_t n_super;      /* candidates flagged SSE_FLAG_SUPER */
  uint32_t cap;          /* in: capacity of the arrays below */
  uint32_t truncated;    /* 1 if n_candidates > cap or > max_candidates */
  uint32_t* hosts;       /* in: [cap] host memory, or NULL */
  float* est;            /* in: [cap] host memory, or NULL */
  uint8_t* flags;        /* in: [cap] host memory, or NULL */
} sse_report;

/* Slice statistics of the most recent close or advance. */
typedef struct sse_stats {
  uint64_t slice;          /* index of the slice that was closed */
  uint32_t hot[16];        /* |HSE(i)|: hot SREs of RSRA row i (Section 3.3) */
  uint32_t active2[16];    /* active cells of SLEA row i; SF(i,k) = active2[i] / row_len2 (Definition 4) */
  uint64_t join_pairs;     /* pairs the last close's join grew tuples from: (he_0, he_1) from
                              row 0 up, (he_0, he_{r-1}) of one column block from the top down */
  uint32_t n_candidates;
  uint32_t n_super;
} sse_stats;

/* Fills *p with the paper's experiment parameters (Section 5: q = q' = 17, delta = 5,
 * delta' = 16, eta' = 2^14, r = r' = 5) and its sliding-window length k = 300, which needs
 * 16-bit stamps. */
SSE_API void sse_params_default(sse_params* p);

/* Validates *p and computes derived values (d may be NULL). SSE_ERR_INVALID_PARAM if
 * any field is outside the ranges above. No device work. */
SSE_API int sse_derive(const sse_params* p, sse_derived* d);

/* Creates an estimator for slice 0 with every cell unset (the paper's initialisation of
 * every short integer to its largest value, Section 3.2). cuda_stream is a cudaStream_t
 * (NULL = legacy default stream) on which all of the handle's work is ordered. The device
 * is the current CUDA device. Errors: INVALID_PARAM, OOM, CUDA. */
SSE_API int sse_init(const sse_params* p, void* cuda_stream, sse_handle** out);

/* Releases the handle and its device memory after its stream has drained. NULL is a no-op. */
SSE_API void sse_destroy(sse_handle* h);

/*
 * Scans n_pairs IP pairs of the current slice (Algorithm 3 for RSRA: the pair updates
 * the r SREs RSRA[i, RHFG[i](aip)], cell H2(bip), only if LSB(H1(bip)) >= tau;
 * Algorithm 6 for SLEA: cell H3(bip) of SLE LH_i(aip) in every row i). Every touched cell
 * is stamped with the current slice; repeated and concurrent writes are idempotent.
 * d_pairs: device memory, 2*n_pairs uint32 {src, dst, src, dst, ...}, 8-byte aligned.
 * Asynchronous on the handle's stream. n_pairs == 0 is a no-op.
 * Errors: INVALID_PARAM (NULL with n_pairs > 0, misaligned), CUDA.
 */
SSE_API int sse_update(sse_handle* h, const uint32_t* d_pairs, uint64_t n_pairs);

/*
 * sse_update() for pairs in host memory: the library copies them to the device in
 * chunks through its own staging buffers, overlapping copies with the update kernels.
 * Page-locked host memory is copied directly; pageable memory is staged through pinned
 * buffers. Returns when h_pairs may be reused (all its bytes have reached the device).
 * Errors: INVALID_PARAM, OOM, CUDA.
 */
SSE_API int sse_update_host(sse_handle* h, const uint32_t* h_pairs, uint64_t n_pairs);

/*
 * Which end of a pair is the host aip whose opposite hosts are counted (Definition 1 lets a
 * host be either end): SSE_DIR_SRC (default) scans (src, dst) as (aip, bip), SSE_DIR_DST as
 * (bip, aip), SSE_DIR_BOTH scans every pair both ways (a host's opposite hosts in either
 * direction). DST and BOTH exchange the ends into a 128 MiB device buffer owned by the
 * handle, allocated at first use. Errors: INVALID_PARAM.
 */
enum { SSE_DIR_SRC = 0, SSE_DIR_DST = 1, SSE_DIR_BOTH = 2 };
SSE_API int sse_set_direction(sse_handle* h, int direction);

/* Selects how sse_update() writes cells (enum sse_update_mode). Results never depend on
 * it. Errors: INVALID_PARAM. */
SSE_API int sse_set_update_mode(sse_handle* h, int mode);

/* Number of update variants the autotuner chooses from (variant 0 is the direct update,
 * the others are tiled updates with different loads in flight and atomic policies). */
SSE_API int sse_update_variant_count(void);

/* Fixes the update variant used by SSE_UPDATE_AUTO for large batches (and, if tiled, by
 * SSE_UPDATE_TILED); -1 restores the built-in rule. Errors: INVALID_PARAM. */
SSE_API int sse_set_update_variant(sse_handle* h, int variant);

/*
 * Autotuner: times every update variant on d_pairs (device pairs of the current slice;
 * rescanning them changes nothing, since a slice's writes are idempotent), reps timed
 * launches each after one warm-up, on the handle's stream, and keeps the fastest for
 * batches of this size in SSE_UPDATE_AUTO mode (and the fastest tiled one for
 * SSE_UPDATE_TILED). times_ms: NULL or sse_update_variant_count() floats (mean ms per
 * update); *chosen: the chosen variant. Synchronous. Errors: INVALID_PARAM, CUDA.
 */
SSE_API int sse_autotune_update(sse_handle* h, const uint32_t* d_pairs, uint64_t n_pairs, int reps,
                                float* times_ms, int* chosen);

/*
 * Closes the current slice t: expires cells older than the window W(t,k), finds the
 * hot SREs of every row, grows candidate tuples and regains candidate hosts (Algorithms
 * 4-5: every 32-bit aip whose r SREs are all hot), estimates each candidate (Algorithm 8,
 * Eq. 11-12) and flags those reaching theta; then the handle moves to slice t+1 (the
 * paper's "slice updating", Section 3.2). Blocks until the report is in host memory.
 * out may be NULL (statistics are still kept, see sse_get_stats()).
 * Errors: CAPACITY when candidates exceed max_candidates or out->cap (the report then
 * holds the first entries, truncated = 1, and the slice still advances); TIMEOUT when the
 * ordering of more than 4096 candidates, whose blocks meet at bounded device-side
 * barriers, gave up waiting (the report's hosts and order are then not valid; the slice
 * still advances and the handle stays usable); CUDA.
 */
SSE_API int sse_close_slice(sse_handle* h, sse_report* out);

/* 1 (default): sse_close_slice replays its device work (close kernels, counter and report
 * copies, clock tick) from a CUDA graph captured at the first call; 0: launches the same
 * kernels one by one. Results are identical. Errors: INVALID_PARAM. */
SSE_API int sse_close_use_graph(sse_handle* h, int enable);

/*
 * Chooses how a close grows candidate tuples (Section 3.3, Algorithms 4-5; Eq. 7). Both ways
 * list every chain of hot SREs, one per row, that one 32-bit address maps to, and regain the
 * hosts of each from RHFG[0]; the candidate sets are identical. SSE_JOIN_FORWARD grows the
 * chains from HSE(0) x HSE(1) upwards, as the paper does. SSE_JOIN_BACKWARD starts from
 * HSE(0) and HSE(r-1): B(r-1) = aip >> (r-1)*delta keeps only s = 32 - (r-1)*delta bits of
 * an address, so he_{r-1} agrees with he_0 above bit s and only pairs inside one of the
 * 2^(q-s) column blocks can meet; rows r-2 .. 1 then each add delta address bits. It applies
 * when delta <= 5, 4 <= r <= 6 and q - s <= 12 (the paper's q = 17,
 * delta = 5, r = 5 has s = 12: 32 blocks). SSE_JOIN_AUTO (the default) takes it wherever it
 * applies. Takes effect at the next close (a captured close graph is dropped and captured
 * again). Errors: INVALID_PARAM (unknown mode, or BACKWARD where it does not apply), STATE
 * (a close is pending).
 */
SSE_API int sse_set_join(sse_handle* h, int mode);

/*
 * Failure-detection hook (the paper has no counterpart; for tests of the bounded device-side
 * waits). When a close finds more than 4096 candidates, their ordering runs as one
 * cooperative launch whose blocks meet at grid-wide barriers; each wait polls at most
 * spin_limit times (0 restores the default of 2^22 polls, about a quarter of a second)
 * and then gives up. extra_arrivals = 1 makes every barrier wait for one block that does
 * not exist, so every wait runs out: that close returns SSE_ERR_TIMEOUT, its report order
 * is not valid, and the handle stays usable (no sticky error); set 0 again and the next
 * close is correct. Applies to closes enqueued after the call (stream-ordered); blocks
 * until the setting is on the device. Errors: INVALID_PARAM (extra_arrivals > 1), CUDA.
 */
SSE_API int sse_debug_sort_barrier(sse_handle* h, uint32_t spin_limit, uint32_t extra_arrivals);

/* sse_close_slice in two halves, so that the next slice's updates can be enqueued while the
 * report is produced: _async enqueues the close (graph mode only) and moves the handle to
 * the next slice; _wait blocks until that close's report is in host memory and fills out
 * (as sse_close_slice). One close may be pending; sse_close_slice, a second _async and
 * sse_close_use_graph are refused meanwhile. Errors: STATE (no graph mode, a close already
 * pending, or none pending for _wait), CAPACITY, CUDA. */
SSE_API int sse_close_slice_async(sse_handle* h);
SSE_API int sse_close_slice_wait(sse_handle* h, sse_report* out);

/* Moves to the next slice without detection: expires old cells and advances, so a router
 * whose super points are detected elsewhere (after a merge) keeps a valid window.
 * Asynchronous. Errors: CUDA. */
SSE_API int sse_advance(sse_handle* h);

/*
 * Merges estimators of distributed routers (Algorithm 2 for RSRA, Algorithm 7 for SLEA):
 * every cell of dst becomes the most recent of dst's and the sources' stamps (the
 * smallest distance), so dst then describes the union of all their traffic. All handles
 * need identical parameters and seed and the same current slice, and must live on the
 * same device; sources are read on dst's stream (the caller orders their own streams
 * before it, e.g. with sse_sync()). n in 1..64; dst may not be among srcs.
 * Errors: INVALID_PARAM, MISMATCH, CUDA.
 */
SSE_API int sse_merge(sse_handle* dst, const sse_handle* const* srcs, int n);

/*
 * Estimates the cardinality of n arbitrary hosts in the current window, as if the
 * current slice were closed now (Algorithm 8 with Eq. 11-12), without changing state.
 * d_hosts: [n] device uint32; d_est: [n] device float; d_flags: [n] device uint8 or NULL;
 * d_hist: [n][k] device uint32 or NULL, the number of union-SLE cells whose (largest)
 * distance is a, for a = 0..k-1. Asynchronous. Errors: INVALID_PARAM, CUDA.
 */
SSE_API int sse_query(sse_handle* h, const uint32_t* d_hosts, uint32_t n, float* d_est, uint8_t* d_flags,
                      uint32_t* d_hist);

/*
 * sse_query() for callers that cannot allocate device memory. The paper has no
 * counterpart: this entry point exists for processes that are handed pre-sized device
 * buffers by their host framework and may not call the CUDA allocator themselves (an
 * allocation can synchronise the device and stall their data path), so they cannot create
 * a handle. The caller owns everything: p (the estimator's parameters), d_sle (its SLEA
 * stamps, [r'][row_pitch2] bytes as sse_read_stamps() lays them out, 16-byte aligned),
 * slice (the index t of the slice being scanned), d_hosts [n], d_est [n], d_flags [n] or
 * NULL; results equal sse_query() on an estimator holding those stamps. The only scratch,
 * one active-cell counter per SLEA row, is a 64-byte array inside the library that every
 * GPU which loads the library keeps until the process exits; it holds a counter for every
 * r' that parameter validation accepts (at most 16). Only 8-bit stamps are served:
 * p->stamp_bits = 16 is rejected with SSE_ERR_INVALID_PARAM. The first call on a device
 * looks up that array's device address for the device current on the calling thread (make
 * it before any stream capture); cuda_stream must belong to that same device. Each call
 * clears the counters and then runs asynchronously on cuda_stream. All calls share the one
 * array, so calls whose GPU work overlaps (different streams or threads) race and must be
 * serialised by the caller. Allocates nothing. Errors: INVALID_PARAM, CUDA.
 */
SSE_API int sse_query_noalloc(const sse_params* p, const uint8_t* d_sle, uint64_t slice, const uint32_t* d_hosts,
                              uint32_t n, float* d_est, uint8_t* d_flags, void* cuda_stream);

/* Statistics of the last close (hot SREs per row, active SLEA cells per row, candidate
 * and super point counts). Synchronises the stream. Errors: CUDA. */
SSE_API int sse_get_stats(sse_handle* h, sse_stats* out);

/* Copies the hot-SRE bitmap of the last close into h_bits (r * 2^q bits, row-major,
 * bit j of row i at bit i*2^q + j, little-endian uint32 words). Synchronous.
 * Errors: INVALID_PARAM (cap_bytes too small), CUDA. */
SSE_API int sse_get_hot_bitmap(sse_handle* h, uint32_t* h_bits, size_t cap_bytes);

/*
 * Checkpoint: writes the estimator (parameters, current slice, RSRA and SLEA stamps) into
 * h_buf; *used receives the size. With h_buf == NULL only *used is set. Synchronous.
 * sse_import_state() restores it into a handle with identical parameters; the result is
 * bit-identical to the exported estimator. Errors: CAPACITY, MISMATCH, INVALID_PARAM, CUDA.
 */
SSE_API int sse_export_state(sse_handle* h, void* h_buf, size_t cap, size_t* used);
SSE_API int sse_import_state(sse_handle* h, const void* h_buf, size_t n);

/* Raw stamp arrays, for inspection: RSRA as [r][2^q][eta] bytes and SLEA as
 * [r'][row_pitch2] bytes (cells beyond row_len2 are padding). Stamps are 1+(slice mod 255),
 * 0 = unset. Synchronous. Either pointer may be NULL. Errors: CAPACITY, CUDA. */
SSE_API int sse_read_stamps(sse_handle* h, uint8_t* h_sre, size_t sre_cap, uint8_t* h_sle, size_t sle_cap);

/* Index t of the slice currently being scanned. */
SSE_API uint64_t sse_current_slice(const sse_handle* h);

/* Number of CUDA kernels this handle has launched since sse_init (for accounting). */
SSE_API uint64_t sse_kernel_launches(const sse_handle* h);

/* Waits for the handle's stream and reports deferred errors (CUDA faults, device-side
 * error flags). Errors: CUDA, TIMEOUT. */
SSE_API int sse_sync(sse_handle* h);

/*
 * Batches: R edge routers (1..64) whose estimators advance slice by slice together, plus a
 * global estimator that merges them (the distributed setting of Section 3.3 and Alg. 7,
 * with all routers' estimators on one device). Each step scans every router's pairs of
 * the current slice in ONE persistent kernel launch (work items = (router, chunk), taken
 * from per-tile counters, so uneven router loads balance) whose cell writes go both to the
 * router and to the global estimator, so the global estimator always equals the merge of
 * the routers (Algorithms 2 and 7: merge(A, B) is the estimator of A's and B's pairs) without
 * a pass over the routers' state; it closes the slice on the global estimator (candidates,
 * estimates, flags, as sse_close_slice) and advances every estimator. The routers' cells
 * that left the window are reset every 254 - k slices (before their stamp comes round).
 * The step's device work is captured once into a CUDA graph and replayed.
 * The batch owns a non-blocking CUDA stream (sse_batch_stream) and its estimators; the
 * handles from sse_batch_router / sse_batch_global stay owned by the batch (do not
 * destroy them, and call only read-only functions on them between steps).
 */
typedef struct sse_batch sse_batch;

/* capacity_pairs: size of each router's input buffer. Errors: INVALID_PARAM, OOM, CUDA. */
SSE_API int sse_batch_create(const sse_params* p, int n_routers, uint64_t capacity_pairs, sse_batch** out);
SSE_API void sse_batch_destroy(sse_batch* b);

/* Device input buffer of a router (capacity_pairs pairs {src, dst}); fill it, on the
 * batch's stream or before the step, with the router's pairs of the current slice. */
SSE_API uint32_t* sse_batch_input(sse_batch* b, int router);
SSE_API void* sse_batch_stream(sse_batch* b);

/* Copies n_pairs pairs (device memory, or host memory when from_host) into a router's
 * input buffer and returns when the copy is done (device sources must be ready: the copy
 * runs on the batch's own stream). Errors: INVALID_PARAM, CAPACITY, CUDA. */
SSE_API int sse_batch_load(sse_batch* b, int router, const uint32_t* pairs, uint64_t n_pairs, int from_host);
SSE_API int sse_batch_router(sse_batch* b, int router, sse_handle** out);
SSE_API int sse_batch_global(sse_batch* b, sse_handle** out);

/* 1 (default): capture the step into a CUDA graph on first use and replay it; 0: launch
 * the same kernels directly each step. Results are identical. */
SSE_API int sse_batch_use_graph(sse_batch* b, int enable);

/* Work-item size (pairs, >= 1024) and loads in flight per thread (2, 4 or 8) of the
 * persistent update. Errors: INVALID_PARAM. */
SSE_API int sse_batch_configure(sse_batch* b, uint32_t item_pairs, int unroll);

/* Autotuner for the persistent update: times 9 configurations (item 2^18, 2^20, 2^22 x
 * loads 2, 4, 8) on the routers' current inputs (idempotent within the slice) and keeps
 * the fastest. d_pairs: NULL (the routers' input buffers) or one device pointer per router;
 * times_ms: NULL or 9 floats; *chosen: index item*3 + load. Synchronous. */
SSE_API int sse_batch_tune(sse_batch* b, const uint32_t* const* d_pairs, const uint64_t* h_counts, int reps,
                           float* times_ms, int* chosen);

/* One slice (see above). h_counts[r] pairs of router r's input buffer are scanned; out
 * receives the global estimator's report (may be NULL). Blocks until the report is on the
 * host. Errors: CAPACITY (a count above capacity_pairs, or report truncated), CUDA. */
SSE_API int sse_batch_step(sse_batch* b, const uint64_t* h_counts, sse_report* out);

/* sse_batch_step() reading router r's h_counts[r] pairs from the caller's device buffer
 * d_pairs[r] (8-byte aligned; written before the call, since the batch runs on its own
 * stream) instead of the batch's input buffers. Errors: INVALID_PARAM, CAPACITY, CUDA. */
SSE_API int sse_batch_step_from(sse_batch* b, const uint32_t* const* d_pairs, const uint64_t* h_counts,
                                sse_report* out);

/* The step of sse_batch_step_from() split in two, so that the device runs steps back to
 * back while the host reads reports. sse_batch_step_async() enqueues one step behind any
 * earlier one on the batch's stream and returns at once; d_pairs: one device pointer per
 * router (8-byte aligned; their pairs must stay unchanged until the step is collected) or
 * NULL for the batch's input buffers. sse_batch_step_wait() blocks until the oldest
 * enqueued step is done and fills out (may be NULL) with its report, as sse_batch_step()
 * does. At most two steps may be enqueued and not yet collected: a third
 * sse_batch_step_async(), a wait with none enqueued, and sse_batch_step, _load, _tune,
 * _configure, _set_mode, _use_graph or _reset while any is, return SSE_ERR_STATE.
 * Errors: INVALID_PARAM, CAPACITY, STATE, CUDA (step_async); CAPACITY, STATE, TIMEOUT, CUDA
 * (step_wait). */
SSE_API int sse_batch_step_async(sse_batch* b, const uint32_t* const* d_pairs, const uint64_t* h_counts);
SSE_API int sse_batch_step_wait(sse_batch* b, sse_report* out);

/* Steps enqueued by sse_batch_step_async() and not yet collected (0, 1 or 2). */
SSE_API int sse_batch_pending(const sse_batch* b);

/* Kernels executed by the batch's steps so far. */
SSE_API uint64_t sse_batch_kernel_launches(const sse_batch* b);

/* What a step does. SSE_BATCH_DETECT (default): as described above. SSE_BATCH_ROUTERS: the
 * routers scan their pairs and close the slice (their old cells expire, every clock
 * advances); the global estimator is not merged into and the report is empty
 * (n_candidates = 0): for independent routers, e.g. training episodes queried one by one.
 * SSE_BATCH_SCAN: the routers scan their pairs and the slice stays open (sse_query on a
 * router then sees it); a later step continues the same slice. Errors: INVALID_PARAM. */
enum { SSE_BATCH_DETECT = 0, SSE_BATCH_ROUTERS = 1, SSE_BATCH_SCAN = 2 };
SSE_API int sse_batch_set_mode(sse_batch* b, int mode);

/* Resets every router and the global estimator to slice 0 (sse_reset). Synchronous. */
SSE_API int sse_batch_reset(sse_batch* b);

/*
 * Serving: a request loop over many routers with all estimator state on the device (the
 * paper's deployment: edge routers stream IP pairs, the detector reports sliding super
 * points at every slice end, Sections 3.1 and 3.3). Requests are batches of one router's
 * pairs with a virtual arrival time; the slice of a request is floor(t / slice_seconds),
 * fixed at admission, so results never depend on GPU timing. Each router has its own
 * estimator and stream: requests of different routers run concurrently, those of one router
 * in order. A request is copied into one of `slots` pinned staging buffers and scanned from
 * its device twin; when every slot is busy, admission waits for the oldest one (the only
 * backpressure). Every update of a router writes the global estimator as well (its RSRA
 * and SLEA stamps, or its SLEA bitmap), so the global estimator always holds the merge of the
 * routers (Algorithm 7: the most recent stamp per cell). A request in a later slice first
 * closes the current slice: detection runs on the global estimator while the next slice's
 * requests proceed, then one pass resets the routers' cells that left the window (the
 * routers' next updates wait for it), and a reporter thread collects the report (the
 * close's last kernel writes it into page-locked host memory); its latency runs from the
 * slice boundary to the report being on the host. Arrival times must
 * not decrease. One thread submits.
 */
typedef struct sse_server sse_server;

typedef struct sse_server_config {
  uint32_t n_routers;      /* routers served, 1..64 */
  uint32_t slots;          /* staging buffers (batches in flight) */
  uint64_t slot_pairs;     /* capacity of one staging buffer; larger requests are split */
  uint64_t memory_budget;  /* device bytes the server may use: (routers + 1) estimators + staging */
  double slice_seconds;    /* virtual-time length of one slice */
} sse_server_config;

typedef struct sse_server_stats {
  uint64_t requests, pairs, slices_closed, slot_waits, current_slice;
  double latency_p50_ms, latency_p99_ms; /* slice boundary to report on the host */
} sse_server_stats;

/* Defaults: 32 routers, 16 slots of 2^22 pairs, a 40 GiB budget, slices of 2^26 packets at
 * an aggregate 2e9 packets/s (33.6 ms). */
SSE_API void sse_server_config_default(sse_server_config* c);

/* Errors: INVALID_PARAM; OOM when the estimators and staging exceed memory_budget (nothing
 * is allocated then) or an allocation fails; CUDA. */
SSE_API int sse_server_create(const sse_params* p, const sse_server_config* cfg, sse_server** out);
SSE_API void sse_server_destroy(sse_server* s);

/* Admits n_pairs host pairs of `router` arriving at virtual time t_arrival (seconds);
 * returns once they are copied to staging (h_pairs may then be reused). Errors:
 * INVALID_PARAM, STATE (t_arrival in an already closed slice), CUDA. */
SSE_API int sse_server_submit(sse_server* s, uint32_t router, double t_arrival, const uint32_t* h_pairs,
                              uint64_t n_pairs);

/* Closes the current slice and waits until every report is ready. */
SSE_API int sse_server_flush(sse_server* s);

/* Takes the oldest ready report (out may be NULL; out->cap and arrays as for
 * sse_close_slice) and its latency. Returns SSE_ERR_STATE when no report is ready. */
SSE_API int sse_server_poll(sse_server* s, sse_report* out, double* latency_ms);

SSE_API int sse_server_get_stats(sse_server* s, sse_server_stats* out);

/* The estimators (owned by the server; read-only use after sse_server_flush: an update
 * through a router's handle would also write the global estimator). */
SSE_API int sse_server_router(sse_server* s, uint32_t router, sse_handle** out);
SSE_API int sse_server_global(sse_server* s, sse_handle** out);

/* Clears the estimator to its initial state at slice 0 (as sse_init). Synchronous. */
SSE_API int sse_reset(sse_handle* h);

/*
 * Learned cardinality correction (an extension beside the paper's method; Algorithm 8's
 * linear-counting estimate stays the fallback). Features of a host, as in Algorithm 8 at
 * the current slice: the union SLE's active cells per distance a = 0..k-1 (the largest
 * distance over the host's r' SLEs), then the sum and the minimum over rows of the host's
 * SRE weights |SRE_i|^k; each value v is given as log(1 + v). d_x: [n][k + 2] device floats.
 * Asynchronous on the handle's stream. Errors: INVALID_PARAM, CUDA.
 */
SSE_API int sse_features(sse_handle* h, const uint32_t* d_hosts, uint32_t n, float* d_x);

/*
 * A multilayer perceptron n_in -> hidden -> hidden -> 1 with ReLU, mapping a host's features
 * to a correction in log space: the learned estimate is max(LC, 1) * exp(output), LC being
 * linear counting's estimate (Algorithm 8), so the training target is log(cardinality) -
 * log(max(LC, 1)). Parameters are kept in FP32 for the optimiser and in BF16 for the
 * arithmetic; all sums accumulate in FP32. Flat parameter layout: W1[hidden][n_in],
 * b1[hidden], W2[hidden][hidden], b2[hidden], W3[hidden], b3. Weights start uniform in
 * +-sqrt(6 / fan_in) from SplitMix64(seed), biases at 0. max_batch bounds the samples of one
 * gradient call and of one chunk of sse_query_learned. Calls run on the given stream (NULL:
 * legacy default); functions that return host values synchronise it.
 */
typedef struct sse_mlp sse_mlp;
SSE_API int sse_mlp_create(uint32_t n_in, uint32_t hidden, uint32_t max_batch, uint64_t seed, sse_mlp** out);
SSE_API void sse_mlp_destroy(sse_mlp* m);
SSE_API uint32_t sse_mlp_param_count(const sse_mlp* m);
/* Kernels launched by the MLP's forward, gradient and Adam calls so far. */
SSE_API uint64_t sse_mlp_kernel_launches(const sse_mlp* m);
/* Replaces the FP32 parameters (and their BF16 copy) and resets the optimiser. */
SSE_API int sse_mlp_set_params(sse_mlp* m, const float* h_params);
/* Host copies of the FP32 parameters, the BF16 parameters (raw bits) and the last
 * gradients; any pointer may be NULL. */
SSE_API int sse_mlp_get_params(sse_mlp* m, float* h_fp32, uint16_t* h_bf16, float* h_grads);
/* Per-feature upper bounds of the training data: inputs beyond them fall back to linear
 * counting in sse_query_learned. */
SSE_API int sse_mlp_set_feature_max(sse_mlp* m, const float* h_xmax);
/* Gate of sse_query_learned: the network's estimate is used only for hosts whose union SLE
 * has at least min_active active cells; below, linear counting is kept (default 0: all). */
SSE_API int sse_mlp_set_gate(sse_mlp* m, uint32_t min_active);
/* d_y[b] = network output for d_x[b] ([n][n_in]). */
SSE_API int sse_mlp_forward(sse_mlp* m, const float* d_x, uint32_t n, float* d_y, void* stream);
/* Gradients of the mean squared error between the output and d_t over the n samples
 * d_rows[0..n) of d_x / d_t (d_rows NULL: rows 0..n-1), n <= max_batch; *h_loss (may be
 * NULL) receives the loss. The gradients stay in the MLP for sse_mlp_adam. */
SSE_API int sse_mlp_gradients(sse_mlp* m, const float* d_x, const float* d_t, const uint32_t* d_rows, uint32_t n,
                              float* h_loss, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr. */
SSE_API int sse_mlp_adam(sse_mlp* m, float lr, void* stream);
/* One epoch: minibatches of `batch` consecutive entries of d_perm (a permutation of the n
 * training rows), each a gradient call and an Adam step; *h_loss: the last minibatch's loss. */
SSE_API int sse_mlp_train_epoch(sse_mlp* m, const float* d_x, const float* d_t, const uint32_t* d_perm, uint32_t n,
                                uint32_t batch, float lr, float* h_loss, void* stream);

/* Estimates n hosts with the network: d_est[b] = max(LC, 1) * exp(output) for the host's
 * features, or LC itself when the host is below the gate (sse_mlp_set_gate), a feature
 * exceeds the training range or the result is not finite; d_est_lc and d_flags receive sse_query's estimate and flags. The network must
 * take k + 2 inputs. Asynchronous on the handle's stream. Errors: INVALID_PARAM, MISMATCH,
 * CUDA. */
SSE_API int sse_query_learned(sse_handle* h, sse_mlp* m, const uint32_t* d_hosts, uint32_t n, float* d_est,
                              float* d_est_lc, uint8_t* d_flags);

/* Name of the CUDA error behind a handle's SSE_ERR_CUDA ("" if none). */
SSE_API const char* sse_cuda_error(const sse_handle* h);

/* Static string for a status code. */
SSE_API const char* sse_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* SSE_H */
