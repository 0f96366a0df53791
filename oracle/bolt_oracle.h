/*
 * bolt_oracle.h -- plain single-threaded CPU oracle of the BOLT oblivious map.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this library: only tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or helper with the
 * CUDA path.
 *
 * What it computes (paper section / algorithm / claim each step follows):
 *   - Alg. 1 (logical BOLT algorithm, Sec. 3.1) generalised to a batch of
 *     operations; a batch of one operation is Alg. 1.
 *   - Power-of-two-choices placement (Sec. 3.1, Claim 3.2) and the d-choice
 *     position map (Sec. 4.2 "Decomposed HBM storage"), both processed in
 *     round-synchronous groups of a fixed public width.
 *   - The eviction stash and reverse index (Sec. 3.1, Sec. 4.2 "Fast eviction
 *     with reverse index"), the free-slot ring (Sec. 4.2 "Dynamic HBM
 *     management"), sizing by Claims 3.2-3.4 and the parameter policy of
 *     Sec. 3.3 "Parameters selection".
 *   - Initial placement = "Fast data initialization" (Sec. 4.2): records are
 *     mapped to two random bins and placed by P2C, then loaded into pages.
 *   - The page cipher is ChaCha20 (the paper delegates encryption to the TEE,
 *     Sec. 2.3); it is written here from the published block-function
 *     definition (RFC 8439, Sec. 2.3 of that document).
 *
 * Parity status: results are pinned by a plain dictionary, ChaCha20 by an
 * independent library, sizing by the paper's slack table (Fig. 5 table) and the
 * load / stash dynamics by the paper's validation experiment.  Page ciphertexts
 * and the host-access trace beyond those pins are "parity unpinned": they are
 * fixed by this file's definition only.
 */
#ifndef BOLT_ORACLE_H
#define BOLT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct omap omap_t;

typedef struct {
  uint64_t N, B, K, M, rows;      /* capacity, bins, HBM bins, host pages, pm rows */
  uint32_t key_bytes, val_bytes;
  uint32_t c, d, lmax, R;         /* avg bin load, pm choices, max bin load, pm row cap */
  uint32_t page_bytes, rec_bytes;
  uint64_t round_width;           /* P2C round width W_r */
  uint64_t vs_cap;                /* ceil(beta1 + beta2) + min(N, 65536) */
  double alpha, beta1, beta2;
} oracle_info_t;

typedef struct {
  uint64_t ops;                   /* global op counter t */
  uint64_t n_hbm, n_stash, n_host;/* live items by location */
  uint64_t peak_stash, peak_hbm;  /* maxima seen after each batch */
  uint32_t max_load, peak_load;   /* current / peak max bin load */
  uint32_t max_row, pad;          /* current max pm row count */
} oracle_stats_t;

/* error codes (same numbering as the product library's public header) */
#define ORC_OK 0
#define ORC_E_ARG -1
#define ORC_E_NOMEM -2
#define ORC_E_OVERFLOW -3
#define ORC_E_STATE -4
#define ORC_E_DUPKEY -5
#define ORC_E_INTEGRITY -8   /* a page read from the host failed its tag */

/* parameter ids for oracle_set_param */
#define ORC_PARAM_ALPHA 1      /* override the alpha policy (before init) */
#define ORC_PARAM_C 2          /* average bin load c (before init) */
#define ORC_PARAM_NOCRYPT 3    /* 1 = skip the page cipher (long simulations only) */
#define ORC_PARAM_TRACE 4      /* 1 = record the host-access trace (default 1) */
#define ORC_PARAM_BATCH 5      /* operations per batch, 1..65536 (default 65536) */
#define ORC_PARAM_INTEGRITY 6  /* 1 = pages sealed by ChaCha20-Poly1305 (before init) */

int oracle_create(uint64_t N, uint32_t key_bytes, uint32_t val_bytes,
                  uint64_t hbm_budget, omap_t** out);
int oracle_set_param(omap_t*, int which, double v);
int oracle_init(omap_t*, const uint64_t* keys, const uint8_t* vals, uint64_t n,
                uint64_t seed);
/* the data owner's image of the placement oracle_init makes (Sec. 4.2 "Fast
 * data initialization"): records in bin-major order (HBM bins first, then
 * host pages; ascending record index within a bin) with their keys, values,
 * pairs (b1 | b2 << 32) and position-map rows (bit 31 set: in b2), and the B
 * per-bin counts; builds the map as oracle_init does */
int oracle_prepare(omap_t*, const uint64_t* keys, const uint8_t* vals, uint64_t n,
                   uint64_t seed, uint64_t* img_keys, uint8_t* img_vals, uint64_t* img_pairs,
                   uint32_t* img_rows, uint8_t* counts);
int oracle_access(omap_t*, const uint8_t* ops, const uint64_t* keys,
                  const uint8_t* vals_in, uint8_t* vals_out, uint8_t* status_out,
                  uint64_t n);
void oracle_destroy(omap_t*);

int oracle_info(const omap_t*, oracle_info_t* out);
/* threads of the OpenMP build (n > 0 sets them); 1 for the plain build */
int oracle_threads(int n);
int oracle_stats(const omap_t*, oracle_stats_t* out);
/* host-resident encrypted pages, M * page_bytes bytes (read only) */
const uint8_t* oracle_pages(const omap_t*);
/* copy of the bin-load array (B bytes) and page versions (M u64) */
int oracle_loads(const omap_t*, uint8_t* out);
int oracle_versions(const omap_t*, uint64_t* out);
/* position-map row occupancies (rows u32) */
int oracle_rowcounts(const omap_t*, uint32_t* out);
/* trace entries since the last clear: bit 31 set = write, low 31 bits = page */
uint64_t oracle_trace_len(const omap_t*);
uint64_t oracle_trace_copy(const omap_t*, uint32_t* out, uint64_t cap);
void oracle_trace_clear(omap_t*);
/* decrypt page q with the map's key and current version into out (page_bytes) */
int oracle_decrypt_page(const omap_t*, uint64_t q, uint8_t* out);
/* the two derived 256-bit keys (K_prf, K_enc) after init, 8 words each */
int oracle_keys(const omap_t*, uint32_t* kprf, uint32_t* kenc);

/* primitives exposed for pins */
void oracle_chacha20_block(const uint32_t key[8], uint32_t counter,
                           const uint32_t nonce[3], uint32_t out[16]);
void oracle_chacha20_xor(const uint32_t key[8], uint32_t counter,
                         const uint32_t nonce[3], uint8_t* buf, uint64_t len);
int oracle_sizing(uint64_t N, uint32_t c, double alpha, uint32_t val_bytes,
                  oracle_info_t* out);
int oracle_pair(const uint32_t kprf[8], uint32_t dom, uint64_t x, uint64_t B,
                uint32_t* b1, uint32_t* b2);
/* Poly1305 tag of len bytes under a 32-byte one-time key (RFC 8439) */
void oracle_poly1305(const uint8_t key[32], const uint8_t* msg, uint64_t len, uint8_t tag[16]);
/* the two working keys derived from a seed, as bolt_init derives them */
void oracle_kdf(uint64_t seed, uint32_t kprf[8], uint32_t kenc[8]);
/* decrypt one page ciphertext of page_bytes taken from page q at `version`
 * under K_enc (in and out may alias) -- for checking sampled pages of maps
 * too large to rebuild here */
void oracle_page_decrypt(const uint32_t kenc[8], uint64_t q, uint64_t version,
                         const uint8_t* in, uint8_t* out, uint64_t page_bytes);

#ifdef __cplusplus
}
#endif
#endif
