/*
 * bolt.h -- C ABI of a B300-native BOLT oblivious map.
 *
 * BOLT (Guo et al., CCS '25) is an oblivious key-value map: records live in
 * fixed-size encrypted pages in host memory (V_host), a position map, an HBM
 * value store and an eviction stash live in device HBM, which the paper treats
 * as unobservable memory.  Every access reads the two random logical bins a
 * key is mapped to and writes the pages back, so the host sees a trace whose
 * distribution does not depend on the keys or operations (Claim 3.1).
 *
 * Operation definitions and where the paper fixes them:
 *   Get / Put / Delete ............ Sec. 2.1 (deletion = Put of a tombstone)
 *   bins, pages, stash, remap ..... Alg. 1 and Sec. 3.1
 *   sizing (lmax, V_hbm, stash) ... Claims 3.2-3.4, Sec. 3.3
 *   position map, value store,
 *   free ring, reverse index ...... Sec. 4.2
 *   initial load .................. Sec. 4.2 "Fast data initialization"
 *
 * Conventions for every entry point:
 *   - return value: 0 on success, a negative BOLT_E_* code otherwise; nothing
 *     is thrown and no call aborts the process;
 *   - BOLT_E_OVERFLOW (a bin, position-map row or value store ran over its
 *     bound, probability 1/O(N) per Sec. 3.3) poisons the handle: later
 *     bolt_access calls return BOLT_E_STATE until bolt_init succeeds again;
 *   - the caller owns every array it passes; the library copies what it needs
 *     before returning (host-pointer calls) or before the stream work it
 *     enqueues completes (device-pointer calls);
 *   - the handle owns all device memory and the pinned host pages it
 *     allocates, and bolt_destroy releases them;
 *   - a handle is not re-entrant: calls on one handle must not overlap;
 *     distinct handles are independent.
 */
#ifndef BOLT_H
#define BOLT_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bolt bolt_t;

#if defined(__GNUC__)
#define BOLT_API __attribute__((visibility("default")))
#else
#define BOLT_API
#endif

/* error codes */
#define BOLT_OK 0
#define BOLT_E_ARG -1      /* bad argument (null pointer, size out of range) */
#define BOLT_E_NOMEM -2    /* device or pinned host allocation failed, or the
                              HBM budget cannot hold even alpha = 0 */
#define BOLT_E_OVERFLOW -3 /* a capacity bound was exceeded; handle poisoned */
#define BOLT_E_STATE -4    /* not initialised, or poisoned by an overflow */
#define BOLT_E_DUPKEY -5   /* bolt_init keys are not unique (Sec. 2.1) */
#define BOLT_E_CUDA -6     /* a CUDA runtime call failed */
#define BOLT_E_TIMEOUT -7  /* a bounded device wait gave up */
#define BOLT_E_INTEGRITY -8 /* a host page failed its tag (BOLT_PARAM_INTEGRITY):
                               altered or replayed; handle poisoned */
#define BOLT_E_INTERNAL -9 /* an internal consistency check failed */

/* operation codes (Sec. 2.1; Delete is the paper's tombstone Put) */
#define BOLT_GET 0
#define BOLT_PUT 1
#define BOLT_DEL 2

/* largest batch one call processes in one go; longer calls are split into
 * consecutive batches of this many operations */
#define BOLT_MAX_BATCH 65536

/* bolt_set_param ids */
#define BOLT_PARAM_ALPHA 1  /* HBM-bin ratio alpha in [0,1) overriding the
                               budget policy; before bolt_init */
#define BOLT_PARAM_C 2      /* average bin load c in [1, 32] (default 8, Sec. 5.1);
                               before bolt_init; the plan must give lmax <= 32
                               (one warp lane per page slot) */
#define BOLT_PARAM_TRACE 4  /* 1 = record the host-access trace (parity runs) */
#define BOLT_PARAM_BATCH 5  /* operations per batch, 1..BOLT_MAX_BATCH */
#define BOLT_PARAM_TRACE_CAP 6 /* trace capacity in entries (default 1<<22) */
#define BOLT_PARAM_CHECK_KEYS 7 /* 1 = bolt_init verifies key uniqueness (default) */
#define BOLT_PARAM_PROFILE 8 /* 1 = time kernel classes with CUDA events */
#define BOLT_PARAM_BATCH_CAP 9 /* capacity of the device batch buffers, 1..BOLT_MAX_BATCH
                                  (default BOLT_MAX_BATCH); reallocates, drops contents */
#define BOLT_PARAM_LOOKAHEAD 10 /* share in [0, 1] of each batch's predicted host pages
                                   that bolt_access_device_batches reads ahead, while
                                   the previous batch finishes (default 0 = off);
                                   results are the same for every value */
#define BOLT_PARAM_DEFER_FLUSH 11 /* 1 = between the batches of one call, a batch's host
                                     write-back starts once the next batch's page reads
                                     are done; 2 = the same with twice the write-back
                                     warps; 0 = right after its eviction (default: the
                                     fastest here); results, pages and trace are the
                                     same for all */
#define BOLT_PARAM_FUSED 13 /* 1 = a batch of at most 32 operations runs as one
                               single-CTA launch that also writes its pages to
                               the host (default); 0 = the multi-kernel chain
                               of larger batches for every batch.  Results,
                               pages and trace are the same for both */
#define BOLT_PARAM_INTEGRITY 14 /* 1 = seal every host page with ChaCha20-Poly1305
                                    (RFC 8439 Sec. 2.8; the per-chunk authenticated
                                    encryption of the paper's appendix on TEE
                                    integrity): ciphertext from key-stream block 1,
                                    a 16-byte tag over it and its length in the
                                    page's last 16 bytes, nonce (page, version).
                                    The versions stay in HBM, so a replayed older
                                    page fails its tag as an altered one does.  A
                                    page that fails is read as empty and the call
                                    returns BOLT_E_INTEGRITY (handle poisoned until
                                    bolt_init).  page_bytes grows by 16 (before the
                                    64-byte rounding); re-plans the map (like
                                    BOLT_PARAM_C).  Not with BOLT_PARAM_LOOKAHEAD
                                    (BOLT_E_ARG): pages read ahead are not checked.
                                    Default 0. */
#define BOLT_PARAM_ROUNDS_PRF 15 /* where the build computes the records' PRF (their
                                    INIT pairs and position-map rows): 0 = automatic
                                    (default): inside the persistent P2C rounds, in the
                                    blocks' barrier waits, when the round's grid has a
                                    block on every SM, else in a pass before them; 1 =
                                    inside the rounds wherever the co-resident grid
                                    has a thread for every 4 records of a round; 2 =
                                    always a pass before them.  The map built is the
                                    same either way */
#define BOLT_PARAM_SPIN_LIMIT 12 /* iterations (of a ~256 ns sleep) a bounded device wait
                                    spins before it gives up, 0..2^22 (default 2^22,
                                    about one second): the build's grid barrier between
                                    P2C rounds.  A wait that gives up makes bolt_init
                                    return BOLT_E_TIMEOUT with nothing placed; the
                                    context stays usable and the next bolt_init
                                    rebuilds the map.  Small values exist to test that
                                    path. */

/* derived parameters (Sec. 3.3 sizing, Sec. 4.2 position map) */
typedef struct {
  uint64_t N, B, K, M, rows;   /* capacity, bins, HBM bins, host pages, pm rows */
  uint32_t key_bytes, val_bytes;
  uint32_t c, d, lmax, R;      /* avg bin load, pm choices, max bin load, pm row cap */
  uint32_t page_bytes, rec_bytes;
  uint64_t round_width;        /* P2C round width W_r = max(1, floor(B/256)) */
  uint64_t vs_cap;             /* value-store slots = ceil(beta1 + beta2) + min(N, 65536):
                                  the paper's bounds plus one batch of headroom */
  double alpha, beta1, beta2;  /* Claim 3.3 and Claim 3.4 bounds */
} bolt_info_t;

typedef struct {
  uint64_t ops;                /* operations processed since bolt_init */
  uint64_t n_hbm, n_stash;     /* live items in the HBM store and the stash */
  uint64_t batches;            /* batches processed since bolt_init */
  uint64_t trace_len;          /* recorded trace entries */
  uint32_t max_load, max_row;  /* largest bin load / position-map row count now */
  /* peaks since bolt_init, the quantities Claims 3.2-3.4 bound (Sec. 3.3
   * "Dimensions in practice"): the largest HBM-store and stash occupancy at
   * the end of the build or of any batch, and the largest bin load reached */
  uint64_t peak_hbm, peak_stash;
  uint32_t peak_load, pad;
} bolt_stats_t;

/*
 * bolt_create -- plan a map of capacity N records (Sec. 3.3 sizing) and
 * allocate its device state and its M pinned, device-mapped host pages.
 *   N           capacity in records, 64 <= N <= 2^31;
 *   key_bytes   8 (keys are uint64) or 4 (keys are uint32): the width of the
 *               keys the host-pointer calls (bolt_init, bolt_access,
 *               bolt_autotune) take; the map zero-extends 4-byte keys and
 *               holds every key as a uint64 (an 8-byte little-endian key
 *               field in each page slot, so page_bytes does not depend on
 *               it); the device-pointer calls and the server take uint64
 *               keys for either width;
 *   val_bytes   value size, a multiple of 8 in [8, 504];
 *   hbm_budget  bytes the value store (HBM bins + stash, Claims 3.3/3.4) may
 *               use; alpha is the largest of {0.2, 0.1, 0.05, 0.01, 0} that
 *               fits (Sec. 3.3 "Parameters selection"); the position map,
 *               reverse index and load counters are metadata outside it;
 *   out         receives the handle.
 * Errors: BOLT_E_ARG, BOLT_E_NOMEM, BOLT_E_CUDA.
 */
BOLT_API int bolt_create(uint64_t N, uint32_t key_bytes, uint32_t val_bytes, uint64_t hbm_budget,
                bolt_t** out);

/* bolt_plan -- the sizing of bolt_create without allocating anything (host
 * only, needs no GPU): alpha < 0 applies the budget policy, otherwise that
 * alpha is used; c is the average bin load.  Fills *out. */
BOLT_API int bolt_plan(uint64_t N, uint32_t key_bytes, uint32_t val_bytes, uint64_t hbm_budget,
                       double alpha, uint32_t c, bolt_info_t* out);

/* bolt_set_param -- change a parameter (ids above).  Sizing parameters
 * (ALPHA, C) re-plan and reallocate the map and drop its contents. */
BOLT_API int bolt_set_param(bolt_t* h, int which, double value);

/*
 * bolt_init -- the oblivious build (Sec. 4.2 "Fast data initialization", run
 * on the device): keys[i] gets the pair PRF(INIT, i), P2C places it in the
 * less-loaded bin in rounds of W_r records, the position map takes it by
 * d-choice, HBM-bin records enter the value store, and the remaining records
 * are grouped per page by a bitonic sorting network, padded with dummies to
 * lmax slots, encrypted and written to the pinned host pages.
 *   keys  HOST pointer, n uint64 keys, all distinct;
 *   vals  HOST pointer, n * val_bytes bytes, record i at i * val_bytes;
 *   n     0 <= n <= N;  seed  derives the PRF and page-cipher keys.
 * Synchronous.  Errors: BOLT_E_ARG, BOLT_E_DUPKEY, BOLT_E_OVERFLOW, BOLT_E_CUDA.
 */
BOLT_API int bolt_init(bolt_t* h, const void* keys, const void* vals, uint64_t n, uint64_t seed);

/* bolt_init_device -- bolt_init with DEVICE pointers for keys and vals, the
 * work enqueued on `stream` (a cudaStream_t, NULL = legacy default stream);
 * returns after the stream work completes. */
BOLT_API int bolt_init_device(bolt_t* h, const void* d_keys, const void* d_vals, uint64_t n,
                     uint64_t seed, void* stream);

/*
 * bolt_init_device_noalloc -- bolt_init_device that allocates no memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory while they (re)build a map -- for example a
 * serving loop that re-keys maps in place and must not stall other streams
 * (cudaMalloc/cudaFree can synchronize the device), or a process whose device
 * memory is owned by another allocator or a fixed arena.  bolt_init_device
 * grows its build scratch with cudaMalloc when n exceeds what it holds; this
 * variant instead uses one fixed scratch array compiled into the library
 * (about 7 MB, held on every GPU that loads the library until the process
 * exits), so it calls no cudaMalloc, cudaFree or other allocating routine.
 *   limits   n <= 2^18 records and a map of at most 2^18 host pages (M);
 *            larger sizes return BOLT_E_ARG before any work is enqueued;
 *   set-up   the first call on each device looks up the array's device
 *            address (cudaGetSymbolAddress) with that device current; make
 *            that first call before any stream capture;
 *   sharing  every call on a device, from any handle, uses the same array:
 *            the call clears what must start at zero, but calls whose work
 *            overlaps on the GPU race on it, so serialise them (one stream,
 *            or wait for the previous call to return);
 *   profile  the call records no BOLT_PARAM_PROFILE spans (recording one
 *            creates CUDA events and grows a host list);
 *   memory   the array (BOLT_NOALLOC_SCRATCH_BYTES) is not part of any
 *            handle's bolt_footprint; the server counts it once against its
 *            HBM budget;
 * Arguments, results and errors are those of bolt_init_device. */
#define BOLT_NOALLOC_SCRATCH_BYTES 7340800ull
BOLT_API int bolt_init_device_noalloc(bolt_t* h, const void* d_keys, const void* d_vals,
                                      uint64_t n, uint64_t seed, void* stream);

/*
 * Owner-side build (Sec. 4.2 "Fast data initialization").  The paper's data
 * owner pre-organizes the records offline -- each record's random bin pair,
 * its power-of-two-choices bin, its position-map row -- and the device only
 * loads that layout with sequential reads and writes.  An image holds n
 * records in bin-major order: bin 0's records, then bin 1's, ... (bins
 * 0..K-1 are the HBM bins, bin K + q is host page q), ascending record index
 * within a bin; all arrays on the DEVICE, 8-byte aligned:
 */
typedef struct {
  uint64_t* keys;   /* [n] the records' keys, bin-major */
  void* vals;       /* [n * val_bytes] their values, the same order */
  uint64_t* pairs;  /* [n] each record's bin pair b1 | b2 << 32 */
  uint32_t* rows;   /* [n] its position-map row, bit 31 set when it sits in b2 */
  uint8_t* counts;  /* [B] records per bin (the bin loads) */
} bolt_image_t;

/* bolt_prepare_device -- the data owner's preprocessing on a device: builds
 * the map from n records exactly as bolt_init_device does (same arguments,
 * results and errors) and writes the placement it made as an image into the
 * arrays of *out, which the caller allocated on the device (keys n * 8,
 * vals n * val_bytes, pairs n * 8, rows n * 4, counts B bytes).  The image
 * depends only on the records, the map's sizing and the seed. */
BOLT_API int bolt_prepare_device(bolt_t* h, const void* d_keys, const void* d_vals, uint64_t n,
                                 uint64_t seed, const bolt_image_t* out, void* stream);

/* bolt_init_prepared -- load an image of n records prepared for this map's
 * sizing under the same seed (by bolt_prepare_device, or by the data owner's
 * own program): bin loads from the counts, position-map entries and HBM
 * residents from the records in order, each host page built from its
 * contiguous run, encrypted (version 0) and stored.  The result is the map
 * bolt_init builds from the same records and seed (same pages, loads, rows
 * and later behaviour).  The image is trusted as the paper's data owner is:
 * the loader checks what keeps it in bounds -- bins and rows in range, counts
 * covering exactly n records, no count above lmax (BOLT_E_OVERFLOW), no row
 * above R (BOLT_E_OVERFLOW), HBM-bin records first -- not the keys'
 * uniqueness.  Synchronous.  Errors: BOLT_E_ARG, BOLT_E_OVERFLOW, BOLT_E_CUDA. */
BOLT_API int bolt_init_prepared(bolt_t* h, const bolt_image_t* img, uint64_t n, uint64_t seed,
                                void* stream);

/*
 * bolt_access -- a batch of n oblivious Get/Put/Delete operations (Alg. 1,
 * applied to a batch; a batch of one is Alg. 1).  Per batch every operation
 * reads the host pages of both bins of its pair (stored pair for the first
 * operation on a present key, a fresh random pair otherwise), every distinct
 * page read is written back once with its stash items evicted into it, and
 * every key present afterwards is remapped by P2C.
 *   ops        HOST, n bytes: BOLT_GET, BOLT_PUT or BOLT_DEL;
 *   keys       HOST, n uint64 keys (repeats allowed, applied in order);
 *   vals_in    HOST, n * val_bytes, read for Put;
 *   vals_out   HOST, n * val_bytes, written: the value for a Get on a
 *              present key, zeros otherwise;
 *   status_out HOST, n bytes or NULL: 1 if the key was present before the op;
 * n may exceed BOLT_MAX_BATCH: the call is split into batches of the
 * configured width.  Results never depend on the batch partition; page
 * ciphertexts and the trace do.  Synchronous.  Copies: the call moves chunks
 * of up to the batch capacity; a chunk of pageable (or, up to 64 KiB, any)
 * arrays is packed into the handle's pinned staging and crosses the link in
 * one copy each way, larger pinned arrays are copied directly.
 * Errors: BOLT_E_ARG, BOLT_E_STATE, BOLT_E_OVERFLOW, BOLT_E_CUDA.
 */
BOLT_API int bolt_access(bolt_t* h, const uint8_t* ops, const void* keys, const void* vals_in,
                void* vals_out, uint8_t* status_out, uint64_t n);

/* bolt_access_device -- bolt_access with DEVICE pointers (status may be
 * NULL), enqueued on `stream`; n <= the batch capacity is one batch.  Returns
 * after enqueueing; the overflow check of this batch is reported by the next
 * call on the handle or by bolt_sync. */
BOLT_API int bolt_access_device(bolt_t* h, const uint8_t* d_ops, const void* d_keys,
                       const void* d_vals_in, void* d_vals_out, uint8_t* d_status,
                       uint64_t n, void* stream);

/* bolt_access_device_batches -- ceil(n / width) consecutive access batches
 * (Alg. 1 applied to each batch) over DEVICE arrays of n ops: batch j takes
 * ops [j*width, min(n, (j+1)*width)); the result equals one
 * bolt_access_device call per slice, in order.  width 0 means the handle's
 * batch width (BOLT_PARAM_BATCH); width <= the batch capacity.  All five
 * arrays are required (d_status holds n bytes).  Each batch's preparation
 * (grouping, DUMMY/REMAP pairs, position-map rows) runs on an internal stream
 * ahead of the previous batch's main part.  Enqueued on `stream`; the inputs
 * must be ready in `stream` order at the call; errors are reported as for
 * bolt_access_device. */
BOLT_API int bolt_access_device_batches(bolt_t* h, const uint8_t* d_ops, const void* d_keys,
                                        const void* d_vals_in, void* d_vals_out,
                                        uint8_t* d_status, uint64_t n, uint32_t width,
                                        void* stream);

/* bolt_sync -- wait for the handle's enqueued work and report its error. */
BOLT_API int bolt_sync(bolt_t* h);

/* bolt_destroy -- release every allocation of the handle (NULL is a no-op). */
BOLT_API int bolt_destroy(bolt_t* h);

/* bolt_get_info / bolt_get_stats -- derived parameters and counters.  The
 * occupancy figures come from counters the kernels keep on the device;
 * bolt_get_stats recounts n_hbm and n_stash from the bin loads and the
 * reverse index and returns BOLT_E_INTERNAL if the two disagree (not checked
 * on a poisoned map). */
BOLT_API int bolt_get_info(const bolt_t* h, bolt_info_t* out);
BOLT_API int bolt_get_stats(bolt_t* h, bolt_stats_t* out);

/* bolt_read_pages -- copy `count` host pages starting at page `first`
 * (ciphertext, page_bytes each) into dst (host). */
BOLT_API int bolt_read_pages(bolt_t* h, uint64_t first, uint64_t count, void* dst);

/* bolt_write_pages -- overwrite `count` host pages starting at page `first`
 * with src (host, page_bytes each), after the handle's work in flight ends.
 * The page store is the untrusted host's memory (Sec. 2.2 threat model):
 * this is the host's own move, not a trusted update -- a page changed or
 * replayed here decrypts to garbage, or, with BOLT_PARAM_INTEGRITY, fails
 * its tag on its next read (BOLT_E_INTEGRITY).  Errors: BOLT_E_ARG,
 * BOLT_E_CUDA. */
BOLT_API int bolt_write_pages(bolt_t* h, uint64_t first, uint64_t count, const void* src);

/* bolt_read_trace -- copy up to `cap` trace entries into dst (host) and
 * clear the trace; *len receives the number copied.  Entry encoding: page
 * number in bits 0-30, bit 31 set for a write. */
BOLT_API int bolt_read_trace(bolt_t* h, uint32_t* dst, uint64_t cap, uint64_t* len);

/* bolt_read_loads -- copy the B bin loads (one byte each) into dst (host);
 * bolt_read_rowcounts -- copy the position-map row counts (one byte each). */
BOLT_API int bolt_read_loads(bolt_t* h, uint8_t* dst);
BOLT_API int bolt_read_rowcounts(bolt_t* h, uint8_t* dst);

/* Kernel-class profile (BOLT_PARAM_PROFILE): index = class
 *   0 bitonic global steps (HBM passes)   1 bitonic in-tile steps
 *   2 build page gather/encrypt/store     3 build P2C + position-map rounds
 *   4 build key-uniqueness check          5 whole access batch
 *   6 access position-map search + page read + decrypt
 *   7 access write-back + eviction (with exec)
 *   8 whole build                         9 access grouping sort + scans
 *  10 key check: bitonic global steps    11 key check: bitonic in-tile steps
 *  12 access: written pages copied to the host (side stream)
 *  13 access: lookahead position-map search + page reads (side stream)
 *  14 build: host records grouped by page  15 access: distinct pages + trace
 *  16 access: find_remove + semantics    17 access: P2C remap
 *  18 access: PRF pairs, rows, grouping keys
 * ms[c] sums the event-timed durations of the spans[c] launches (or phases)
 * of class c; launches counts every kernel the library launched. */
#define BOLT_PROF_CLASSES 19
typedef struct {
  uint64_t launches;
  uint64_t spans[BOLT_PROF_CLASSES];
  double ms[BOLT_PROF_CLASSES];
} bolt_profile_t;

/* bolt_read_profile -- wait for the handle's stream, fold the recorded
 * events into *out; reset != 0 clears the accumulated profile. */
BOLT_API int bolt_read_profile(bolt_t* h, bolt_profile_t* out, int reset);

/* Autotuner results (bolt_autotune). */
#define BOLT_TUNE_WIDTHS 6
typedef struct {
  uint32_t sort_log_tile;      /* bitonic tile picked: 2^12 or 2^13 elements */
  uint32_t batch_width;        /* access batch width picked for bolt_access */
  double sort_ms[2];           /* sort time of a tag-sized array, tile 2^12 / 2^13 */
  uint32_t widths[BOLT_TUNE_WIDTHS];
  double width_us[BOLT_TUNE_WIDTHS];  /* device time per batch at each width
                                         (0: not measured, above the capacity) */
} bolt_tune_t;

/* bolt_autotune -- pick performance knobs by measuring them on this device:
 * the bitonic tile of later builds (a tag-sized scratch array is sorted with
 * each tile; allocates it) and, when a sample of present keys is given, the
 * batch width bolt_access splits host calls into: Get batches of 64..65536
 * ops over the sample, the highest accesses/s whose device time per batch is
 * at most max_batch_us (<= 0: no bound).  The knobs change no result.  The
 * tuning Gets are real accesses: they remap their keys (contents unchanged,
 * layout and trace advanced).  Errors as bolt_access. */
BOLT_API int bolt_autotune(bolt_t* h, const void* sample_keys, uint64_t n_sample,
                           double max_batch_us, bolt_tune_t* out);

/* bolt_trim -- release the build scratch (tags, PRF tables, staging); the
 * next bolt_init allocates it again. */
BOLT_API int bolt_trim(bolt_t* h);

/* bolt_footprint -- device bytes the handle holds: resident state and batch
 * buffers, and build scratch (including the host-pointer staging copy). */
BOLT_API int bolt_footprint(const bolt_t* h, uint64_t* resident_bytes, uint64_t* scratch_bytes);

/* bolt_probe_link -- measure the host link as the access path uses it, on
 * this map's own pinned page store, through zero-copy 16-byte loads and
 * stores (warp per 512-byte page, full width), CUDA-event timed on the
 * handle's stream over `launches` launches of `pages` random pages each:
 *   *read_pages_per_s       random pages read per second;
 *   *pipelined_pages_per_s  pages per second when each launch reads a random
 *                           set and writes back the set the previous launch
 *                           read (one page read + one page written each) --
 *                           the access path's batch reads beside the
 *                           previous batch's write-back, with no compute.
 * Written pages get their own bytes back, so the map is unchanged; waits for
 * the handle's work first and allocates 2 * pages * page_bytes of device
 * scratch for the call.  pages <= 2^22.  No counterpart in the paper: it is
 * the access path's roofline denominator.  BOLT_E_STATE before bolt_init. */
BOLT_API int bolt_probe_link(bolt_t* h, uint32_t pages, uint32_t launches,
                             double* read_pages_per_s, double* pipelined_pages_per_s);

/* bolt_plan_bytes -- host-only estimate of the same two figures for a map of
 * capacity N (budget policy for alpha, c = 8, default trace capacity) with
 * batch buffers for batch_cap ops and a build of n_init records. */
BOLT_API int bolt_plan_bytes(uint64_t N, uint32_t val_bytes, uint64_t hbm_budget,
                             uint32_t batch_cap, uint64_t n_init, uint64_t* resident_bytes,
                             uint64_t* build_bytes);

/* ------------------------------------------------------------------------
 * Serving many maps (continuous batching).  The paper serves one command
 * stream on one device; this layer keeps many maps resident and batches
 * their requests as they arrive.
 *
 * A server owns a set of maps and a scheduler thread.  Maps are admitted, in
 * the order they were added, while their planned device footprint (state,
 * batch buffers, build scratch) fits `hbm_budget` less the library's fixed
 * BOLT_NOALLOC_SCRATCH_BYTES array; the rest wait until a removed map frees
 * memory.  A request is up to `max_batch` Get/Put/Delete
 * ops on one map; requests queue per map, and whenever a map has no batch on
 * the GPU the scheduler packs its queued requests (arrival order, at most
 * max_batch ops) into one access batch on the map's stream, so batches of
 * different maps overlap on the device.  Each batch is one bolt access batch:
 * a request's values and status do not depend on the requests it shares a
 * batch with; the per-map batch log reproduces ciphertexts and the trace.
 * All server calls are thread-safe; results are returned by bolt_server_wait.
 * ------------------------------------------------------------------------ */
typedef struct bolt_server bolt_server_t;

typedef struct {
  uint64_t id;
  uint32_t map, n;
  int rc;                      /* BOLT_OK or the batch's error */
  double submit_us, start_us, done_us;  /* microseconds since server creation:
                                           arrival, batch enqueue, batch done */
} bolt_req_info_t;

typedef struct {
  uint64_t budget, used;       /* HBM budget and planned bytes of admitted maps */
  uint64_t batches, ops;       /* completed batches and operations */
  uint32_t maps_pending, maps_ready;
  uint64_t queued;             /* requests waiting for a batch */
} bolt_server_stats_t;

BOLT_API int bolt_server_create(uint64_t hbm_budget, uint32_t max_batch, bolt_server_t** out);
/* add a map of capacity N built from n (key, value) records (HOST pointers,
 * copied); BOLT_E_NOMEM if its footprint alone exceeds the budget */
BOLT_API int bolt_server_add_map(bolt_server_t* s, uint64_t N, uint32_t val_bytes,
                                 const void* keys, const void* vals, uint64_t n, uint64_t seed,
                                 uint32_t* map_id);
/* 0 pending admission, 1 ready, 2 removed, or the map's error code */
BOLT_API int bolt_server_map_state(bolt_server_t* s, uint32_t map_id);
/* remove once its queued requests are served; frees its memory */
BOLT_API int bolt_server_remove_map(bolt_server_t* s, uint32_t map_id);
/* bolt_server_submit_many -- queue `count` requests at once: request j is
 * ns[j] ops on map map_ids[j] with HOST arrays ops[j], keys[j], vals_in[j]
 * (each as bolt_server_submit takes them, copied); req_ids[j] receives its
 * id.  All requests are checked first: on any error (BOLT_E_ARG, BOLT_E_STATE
 * for a removed map, BOLT_E_NOMEM) none is queued.  Queued in array order,
 * under one lock, with one wake-up of the scheduler: a client with many
 * requests ready pays one call instead of one per request. */
BOLT_API int bolt_server_submit_many(bolt_server_t* s, uint32_t count, const uint32_t* map_ids,
                                     const uint8_t* const* ops, const void* const* keys,
                                     const void* const* vals_in, const uint32_t* ns,
                                     uint64_t* req_ids);
/* queue a request (HOST pointers, copied): n <= max_batch ops */
BOLT_API int bolt_server_submit(bolt_server_t* s, uint32_t map_id, const uint8_t* ops,
                                const void* keys, const void* vals_in, uint32_t n,
                                uint64_t* req_id);
/* wait for a request (timeout_ms < 0: forever), copy its outputs (HOST,
 * n * val_bytes and n bytes, either may be NULL) and its timestamps, and
 * release it; returns its result code or BOLT_E_TIMEOUT */
BOLT_API int bolt_server_wait(bolt_server_t* s, uint64_t req_id, void* vals_out,
                              uint8_t* status_out, bolt_req_info_t* info, int timeout_ms);
/* sizes of the batches run on a map so far (copy up to cap, *count = all) */
BOLT_API int bolt_server_map_batches(bolt_server_t* s, uint32_t map_id, uint32_t* sizes,
                                     uint64_t cap, uint64_t* count);
/* the handle of a ready map, for inspection while the server is quiescent */
BOLT_API int bolt_server_map_handle(bolt_server_t* s, uint32_t map_id, bolt_t** out);
BOLT_API int bolt_server_stats(bolt_server_t* s, bolt_server_stats_t* out);
BOLT_API int bolt_server_destroy(bolt_server_t* s);

/* bolt_strerror -- static description of an error code. */
BOLT_API const char* bolt_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif
