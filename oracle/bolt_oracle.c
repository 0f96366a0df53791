/*
 * bolt_oracle.c -- plain single-threaded CPU oracle of the BOLT oblivious map.
 *
 * TEST INFRASTRUCTURE ONLY (see bolt_oracle.h): never linked into, imported
 * by or called from the product path.  Written for readability, not speed:
 * every step is a direct loop over plain arrays, in the order the paper's
 * Alg. 1 (Sec. 3.1) and architecture walk-through (Sec. 4.1, steps 2-6) give.
 *
 * Conventions fixed here (the paper leaves them open; each is a reading):
 *   - bins 0..K-1 live in HBM, bins K..B-1 are host pages q = bin - K;
 *   - P2C picks the first choice on ties; the d-choice position map picks the
 *     lowest choice index on ties;
 *   - placement decisions are taken in rounds of W_r = max(1, floor(B/256))
 *     consecutive items against the loads at the start of the round; W_r = 1
 *     is the paper's sequential greedy rule;
 *   - a batch reads every host bin of every operation's pair (operation order,
 *     first bin then second), writes every distinct page it read once, in
 *     first-read order, and evicts before it remaps (Alg. 1 order);
 *   - a page holds its real tuples in ascending key order in the first slots,
 *     a bitmap of occupied slots in its 16-byte header and zero dummies.
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include "bolt_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_E_INTERNAL -9
#define ORC_E_INTEGRITY -8

enum { LOC_EMPTY = 0, LOC_HOST = 1, LOC_HBM = 2, LOC_STASH = 3 };
enum { OP_GET = 0, OP_PUT = 1, OP_DEL = 2 };
enum { DOM_INIT = 1, DOM_PM = 2, DOM_REMAP = 3, DOM_DUMMY = 4 };
#define NO_INDEX UINT64_MAX

struct omap {
  oracle_info_t p;
  uint64_t hbm_budget;
  double alpha_override; /* < 0: use the budget policy */
  uint32_t c_param;
  int nocrypt, trace_on;
  int integrity; /* pages are ChaCha20-Poly1305 sealed (tag in the last 16 bytes) */
  uint64_t batch_width;

  int allocated, initialized, poisoned;
  uint32_t kprf[8], kenc[8];
  uint64_t t; /* global operation counter */

  uint32_t* load;    /* [B] logical bin loads */
  uint32_t* rowcnt;  /* [rows] position-map row occupancy */
  uint64_t* pm_key;  /* [rows*R] */
  uint32_t* pm_b1;   /* [rows*R] */
  uint32_t* pm_b2;   /* [rows*R] */
  uint8_t* pm_which; /* [rows*R] 0: item sits in b1, 1: in b2 */
  uint8_t* pm_loc;   /* [rows*R] LOC_* */
  uint64_t* pm_ptr;  /* [rows*R] value-store slot for LOC_HBM / LOC_STASH */

  uint64_t* vs_key;  /* [vs_cap] value store = HBM bins + stash (Sec. 4.2) */
  uint8_t* vs_val;   /* [vs_cap*val_bytes] */
  uint64_t* vs_pm;   /* [vs_cap] owning position-map slot */
  uint8_t* vs_live;  /* [vs_cap] */
  uint64_t* ring;    /* [vs_cap] free-slot ring (Sec. 4.2, Fig. ring) */
  uint64_t ring_head, ring_count;

  uint64_t* rev;     /* [M*lmax] reverse index: stash slots bound for page q */
  uint32_t* revcnt;  /* [M] */

  int64_t* dindex;   /* [M] batch-local: distinct-page index or -1 */
  uint8_t* pages;    /* [M*page_bytes] host store, ciphertext */
  uint64_t* version; /* [M] */

  uint32_t* trace;
  uint64_t trace_len, trace_cap;

  uint64_t n_hbm, n_stash, n_host, peak_stash, peak_hbm;
  uint32_t peak_load;
};

/* ------------------------------------------------------------------------ */
/* ChaCha20 block function, from the published definition (RFC 8439 Sec. 2.1 */
/* quarter round, Sec. 2.3 block function: 20 rounds = 10 column/diagonal    */
/* double rounds, then the input state is added word-wise).                  */

static uint32_t rotl32(uint32_t v, int n) { return (v << n) | (v >> (32 - n)); }

static void quarter(uint32_t* s, int a, int b, int c, int d) {
  s[a] += s[b]; s[d] ^= s[a]; s[d] = rotl32(s[d], 16);
  s[c] += s[d]; s[b] ^= s[c]; s[b] = rotl32(s[b], 12);
  s[a] += s[b]; s[d] ^= s[a]; s[d] = rotl32(s[d], 8);
  s[c] += s[d]; s[b] ^= s[c]; s[b] = rotl32(s[b], 7);
}

void oracle_chacha20_block(const uint32_t key[8], uint32_t counter,
                           const uint32_t nonce[3], uint32_t out[16]) {
  uint32_t init[16], s[16];
  init[0] = 0x61707865u; /* "expa" */
  init[1] = 0x3320646eu; /* "nd 3" */
  init[2] = 0x79622d32u; /* "2-by" */
  init[3] = 0x6b206574u; /* "te k" */
  for (int i = 0; i < 8; i++) init[4 + i] = key[i];
  init[12] = counter;
  init[13] = nonce[0];
  init[14] = nonce[1];
  init[15] = nonce[2];
  memcpy(s, init, sizeof s);
  for (int r = 0; r < 10; r++) {
    quarter(s, 0, 4, 8, 12);
    quarter(s, 1, 5, 9, 13);
    quarter(s, 2, 6, 10, 14);
    quarter(s, 3, 7, 11, 15);
    quarter(s, 0, 5, 10, 15);
    quarter(s, 1, 6, 11, 12);
    quarter(s, 2, 7, 8, 13);
    quarter(s, 3, 4, 9, 14);
  }
  for (int i = 0; i < 16; i++) out[i] = s[i] + init[i];
}

/* XOR buf with the key stream starting at block `counter` (little-endian
 * serialisation of each output word). */
void oracle_chacha20_xor(const uint32_t key[8], uint32_t counter,
                         const uint32_t nonce[3], uint8_t* buf, uint64_t len) {
  uint32_t blk[16];
  for (uint64_t off = 0; off < len; off += 64, counter++) {
    oracle_chacha20_block(key, counter, nonce, blk);
    for (uint64_t j = 0; j < 64 && off + j < len; j++)
      buf[off + j] ^= (uint8_t)(blk[j / 4] >> (8 * (j % 4)));
  }
}

/* ------------------------------------------------------------------------ */
/* Keys and PRF.  The paper only says a secret key is provisioned (Sec. 1.2); */
/* the two working keys are derived from a 64-bit seed as follows.           */

static void derive_keys(uint64_t seed, uint32_t kprf[8], uint32_t kenc[8]) {
  uint32_t master[8] = {(uint32_t)seed, (uint32_t)(seed >> 32), 0, 0, 0, 0, 0, 0};
  uint32_t nonce[3] = {0x544c4f42u /* bytes "BOLT" */, 0, 0};
  uint32_t blk[16];
  oracle_chacha20_block(master, 0, nonce, blk);
  for (int i = 0; i < 8; i++) {
    kprf[i] = blk[i];
    kenc[i] = blk[8 + i];
  }
}

static void prf(const uint32_t kprf[8], uint32_t dom, uint64_t x, uint32_t w[16]) {
  uint32_t nonce[3] = {dom, (uint32_t)x, (uint32_t)(x >> 32)};
  oracle_chacha20_block(kprf, 0, nonce, w);
}

static uint64_t mulhi64(uint64_t a, uint64_t b) {
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
}

/* An ordered pair of distinct bins, uniform over all such pairs up to a
 * 2^-64 rounding bias (the pi mapping of Sec. 3.2). */
int oracle_pair(const uint32_t kprf[8], uint32_t dom, uint64_t x, uint64_t B,
                uint32_t* b1, uint32_t* b2) {
  if (B < 2) return ORC_E_ARG;
  uint32_t w[16];
  prf(kprf, dom, x, w);
  uint64_t r0 = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
  uint64_t r1 = (uint64_t)w[2] | ((uint64_t)w[3] << 32);
  uint64_t first = mulhi64(r0, B);
  uint64_t second = mulhi64(r1, B - 1);
  if (second >= first) second += 1;
  *b1 = (uint32_t)first;
  *b2 = (uint32_t)second;
  return ORC_OK;
}

/* The d = 4 candidate position-map rows of a key (Sec. 4.2). */
static void pm_rows(const omap_t* m, uint64_t key, uint64_t rows[4]) {
  uint32_t w[16];
  prf(m->kprf, DOM_PM, key, w);
  for (int j = 0; j < 4; j++)
    rows[j] = mulhi64((uint64_t)w[2 * j] | ((uint64_t)w[2 * j + 1] << 32), m->p.rows);
}

/* ------------------------------------------------------------------------ */
/* Sizing: Claim 3.2 (bin load), Claim 3.3 (sum of HBM bin loads), Claim 3.4 */
/* (stash), with every O(.) replaced by its argument times 1 as in Sec. 3.3  */
/* "Dimensions in practice"; position-map rows per Sec. 4.2 (d = 4,          */
/* N/16 rows, row capacity N/B_pm + loglogN / log d).                        */

int oracle_sizing(uint64_t N, uint32_t c, double alpha, uint32_t val_bytes,
                  oracle_info_t* o) {
  if (N < 64 || c < 1 || alpha < 0.0 || alpha >= 1.0) return ORC_E_ARG;
  memset(o, 0, sizeof *o);
  double lg = log2((double)N);
  double llg = log2(lg);
  o->N = N;
  o->c = c;
  o->d = 4;
  o->key_bytes = 8;
  o->val_bytes = val_bytes;
  o->lmax = c + (uint32_t)ceil(llg) + 1;
  o->R = 16 + (uint32_t)ceil(llg / log2((double)o->d));
  o->rows = (N + 15) / 16;
  o->B = (N + c - 1) / c;
  o->alpha = alpha;
  o->K = (uint64_t)floor(alpha * (double)o->B);
  o->M = o->B - o->K;
  if (o->M < 2 || o->lmax > 64) return ORC_E_ARG;
  double lnN = log((double)N);
  o->beta1 = (double)o->K * c + o->lmax * sqrt((double)o->K * lnN);
  o->beta2 = (1.0 + alpha) * (double)o->M / 2.0 + o->lmax * sqrt((double)o->M * lnN);
  /* Claims 3.3/3.4 bound one-at-a-time access; a batch can push up to one
   * batch of remapped keys into the stash before their pages are next read,
   * so the store gets min(N, 65536) slots of batch headroom. */
  o->vs_cap = (uint64_t)ceil(o->beta1 + o->beta2) + (N < 65536 ? N : 65536);
  o->round_width = o->B / 256 > 0 ? o->B / 256 : 1;
  o->rec_bytes = 8 + val_bytes;
  o->page_bytes = (16 + o->lmax * o->rec_bytes + 63) / 64 * 64;
  return ORC_OK;
}

/* alpha policy (Sec. 3.3 "Parameters selection"): the largest alpha of a
 * fixed grid whose value store (V_hbm + stash) fits the HBM budget. */
static int choose_alpha_plain(omap_t* m, oracle_info_t* o);

/* the sizing policy, then room for the tag when pages are sealed */
static int choose_alpha(omap_t* m, oracle_info_t* o) {
  int rc = choose_alpha_plain(m, o);
  if (rc == ORC_OK && m->integrity)
    o->page_bytes = (16 + o->lmax * o->rec_bytes + 16 + 63) / 64 * 64;
  return rc;
}

static int choose_alpha_plain(omap_t* m, oracle_info_t* o) {
  if (m->alpha_override >= 0.0)
    return oracle_sizing(m->p.N, m->c_param, m->alpha_override, m->p.val_bytes, o);
  static const double grid[] = {0.2, 0.1, 0.05, 0.01, 0.0};
  for (int i = 0; i < 5; i++) {
    int rc = oracle_sizing(m->p.N, m->c_param, grid[i], m->p.val_bytes, o);
    if (rc) return rc;
    double bytes = (double)o->vs_cap * (double)(8 + m->p.val_bytes);
    if (bytes <= (double)m->hbm_budget) return ORC_OK;
  }
  return ORC_E_NOMEM;
}

/* ------------------------------------------------------------------------ */

int oracle_create(uint64_t N, uint32_t key_bytes, uint32_t val_bytes,
                  uint64_t hbm_budget, omap_t** out) {
  if (!out || key_bytes != 8 || val_bytes < 8 || val_bytes % 8 || val_bytes > 504 ||
      N < 64 || N > (1ull << 32))
    return ORC_E_ARG;
  omap_t* m = (omap_t*)calloc(1, sizeof *m);
  if (!m) return ORC_E_NOMEM;
  m->p.N = N;
  m->p.val_bytes = val_bytes;
  m->p.key_bytes = key_bytes;
  m->hbm_budget = hbm_budget;
  m->alpha_override = -1.0;
  m->c_param = 8;
  m->trace_on = 1;
  m->batch_width = 65536;
  oracle_info_t o;
  int rc = choose_alpha(m, &o);
  if (rc) {
    free(m);
    return rc;
  }
  m->p = o;
  *out = m;
  return ORC_OK;
}

static void free_state(omap_t* m) {
  free(m->load); free(m->rowcnt);
  free(m->pm_key); free(m->pm_b1); free(m->pm_b2); free(m->pm_which);
  free(m->pm_loc); free(m->pm_ptr);
  free(m->vs_key); free(m->vs_val); free(m->vs_pm); free(m->vs_live); free(m->ring);
  free(m->rev); free(m->revcnt); free(m->pages); free(m->version); free(m->dindex);
  m->load = NULL; m->rowcnt = NULL; m->pm_key = NULL; m->pm_b1 = m->pm_b2 = NULL;
  m->pm_which = m->pm_loc = NULL; m->pm_ptr = NULL; m->vs_key = NULL; m->vs_val = NULL;
  m->vs_pm = NULL; m->vs_live = NULL; m->ring = NULL; m->rev = NULL; m->revcnt = NULL;
  m->pages = NULL; m->version = NULL; m->dindex = NULL;
  m->allocated = 0;
}

void oracle_destroy(omap_t* m) {
  if (!m) return;
  free_state(m);
  free(m->trace);
  free(m);
}

int oracle_set_param(omap_t* m, int which, double v) {
  if (!m) return ORC_E_ARG;
  switch (which) {
    case ORC_PARAM_ALPHA:
      if (v < 0.0 || v >= 1.0) return ORC_E_ARG;
      m->alpha_override = v;
      break;
    case ORC_PARAM_C:
      if (v < 1.0 || v > 32.0) return ORC_E_ARG;
      m->c_param = (uint32_t)v;
      break;
    case ORC_PARAM_NOCRYPT: m->nocrypt = v != 0.0; return ORC_OK;
    case ORC_PARAM_INTEGRITY:
      m->integrity = v != 0.0;
      break;
    case ORC_PARAM_TRACE: m->trace_on = v != 0.0; return ORC_OK;
    case ORC_PARAM_BATCH:
      if (v < 1.0 || v > 65536.0) return ORC_E_ARG;
      m->batch_width = (uint64_t)v;
      return ORC_OK;
    default: return ORC_E_ARG;
  }
  /* sizing parameters changed: recompute, state is rebuilt by the next init */
  oracle_info_t o;
  int rc = choose_alpha(m, &o);
  if (rc) return rc;
  free_state(m);
  m->p = o;
  m->initialized = 0;
  return ORC_OK;
}

static int alloc_state(omap_t* m) {
  const oracle_info_t* p = &m->p;
  uint64_t slots = p->rows * p->R;
  m->load = calloc(p->B, sizeof *m->load);
  m->rowcnt = calloc(p->rows, sizeof *m->rowcnt);
  m->pm_key = calloc(slots, sizeof *m->pm_key);
  m->pm_b1 = calloc(slots, sizeof *m->pm_b1);
  m->pm_b2 = calloc(slots, sizeof *m->pm_b2);
  m->pm_which = calloc(slots, 1);
  m->pm_loc = calloc(slots, 1);
  m->pm_ptr = calloc(slots, sizeof *m->pm_ptr);
  m->vs_key = calloc(p->vs_cap, sizeof *m->vs_key);
  m->vs_val = calloc(p->vs_cap, p->val_bytes);
  m->vs_pm = calloc(p->vs_cap, sizeof *m->vs_pm);
  m->vs_live = calloc(p->vs_cap, 1);
  m->ring = calloc(p->vs_cap, sizeof *m->ring);
  m->rev = calloc(p->M * p->lmax, sizeof *m->rev);
  m->revcnt = calloc(p->M, sizeof *m->revcnt);
  m->pages = calloc(p->M, p->page_bytes);
  m->version = calloc(p->M, sizeof *m->version);
  m->dindex = malloc(p->M * sizeof *m->dindex);
  if (!m->dindex || !m->load || !m->rowcnt || !m->pm_key || !m->pm_b1 || !m->pm_b2 || !m->pm_which ||
      !m->pm_loc || !m->pm_ptr || !m->vs_key || !m->vs_val || !m->vs_pm || !m->vs_live ||
      !m->ring || !m->rev || !m->revcnt || !m->pages || !m->version) {
    free_state(m);
    return ORC_E_NOMEM;
  }
  m->allocated = 1;
  return ORC_OK;
}

static void reset_state(omap_t* m) {
  const oracle_info_t* p = &m->p;
  uint64_t slots = p->rows * p->R;
  memset(m->load, 0, p->B * sizeof *m->load);
  memset(m->rowcnt, 0, p->rows * sizeof *m->rowcnt);
  memset(m->pm_loc, 0, slots);
  memset(m->vs_live, 0, p->vs_cap);
  memset(m->revcnt, 0, p->M * sizeof *m->revcnt);
  memset(m->version, 0, p->M * sizeof *m->version);
  for (uint64_t q = 0; q < p->M; q++) m->dindex[q] = -1;
  for (uint64_t s = 0; s < p->vs_cap; s++) m->ring[s] = s; /* all slots free */
  m->ring_head = 0;
  m->ring_count = p->vs_cap;
  m->t = 0;
  m->n_hbm = m->n_stash = m->n_host = 0;
  m->peak_stash = m->peak_hbm = 0;
  m->peak_load = 0;
  m->trace_len = 0;
  m->poisoned = 0;
}

/* free-slot ring: pop from the head, push at the tail */
static int ring_pop(omap_t* m, uint64_t* slot) {
  if (m->ring_count == 0) return ORC_E_OVERFLOW;
  *slot = m->ring[m->ring_head];
  m->ring_head = (m->ring_head + 1) % m->p.vs_cap;
  m->ring_count--;
  return ORC_OK;
}

static void ring_push(omap_t* m, uint64_t slot) {
  m->ring[(m->ring_head + m->ring_count) % m->p.vs_cap] = slot;
  m->ring_count++;
}

static void trace_add(omap_t* m, uint32_t e) {
  if (!m->trace_on) return;
  if (m->trace_len == m->trace_cap) {
    uint64_t cap = m->trace_cap ? 2 * m->trace_cap : 4096;
    uint32_t* t = realloc(m->trace, cap * sizeof *t);
    if (!t) return;
    m->trace = t;
    m->trace_cap = cap;
  }
  m->trace[m->trace_len++] = e;
}

/* ------------------------------------------------------------------------ */
/* Page encoding (Sec. 4.2 "Decomposed HBM storage": each page holds tuples  */
/* with a dummy flag, a key and a value) and encryption.                     */

typedef struct {
  uint64_t key;
  const uint8_t* val;
} tuple_t;

static int cmp_tuple(const void* a, const void* b) {
  uint64_t x = ((const tuple_t*)a)->key, y = ((const tuple_t*)b)->key;
  return x < y ? -1 : x > y;
}

/* Poly1305 one-time authenticator (RFC 8439, Sec. 2.5), written from its
 * definition: r = key[0..15] with the specified bits cleared, s =
 * key[16..31]; each 16-byte block of the message (the last one may be short)
 * with a 1 byte appended is added to the accumulator, which is then
 * multiplied by r modulo p = 2^130 - 5; the tag is (h + s) mod 2^128.  The
 * accumulator is kept in three 64-bit limbs, products in 128-bit integers. */
void oracle_poly1305(const uint8_t key[32], const uint8_t* msg, uint64_t len, uint8_t tag[16]) {
  typedef unsigned __int128 u128;
  uint64_t r0, r1, s0, s1;
  memcpy(&r0, key, 8);
  memcpy(&r1, key + 8, 8);
  memcpy(&s0, key + 16, 8);
  memcpy(&s1, key + 24, 8);
  r0 &= 0x0ffffffc0fffffffull;
  r1 &= 0x0ffffffc0ffffffcull;
  uint64_t h0 = 0, h1 = 0, h2 = 0; /* h = h0 + h1 2^64 + h2 2^128 */
  for (uint64_t off = 0; off < len; off += 16) {
    uint8_t blk[17] = {0};
    const uint64_t n = len - off < 16 ? len - off : 16;
    memcpy(blk, msg + off, n);
    blk[n] = 1;
    uint64_t m0, m1;
    memcpy(&m0, blk, 8);
    memcpy(&m1, blk + 8, 8);
    /* h += block */
    u128 t = (u128)h0 + m0;
    h0 = (uint64_t)t;
    t = (u128)h1 + m1 + (uint64_t)(t >> 64);
    h1 = (uint64_t)t;
    h2 += blk[16] + (uint64_t)(t >> 64);
    /* h *= r: the four 128-bit partial sums of the product */
    const u128 d0 = (u128)h0 * r0;
    const u128 d1 = (u128)h0 * r1 + (u128)h1 * r0;
    const u128 d2 = (u128)h1 * r1 + (u128)h2 * r0;
    const u128 d3 = (u128)h2 * r1;
    uint64_t p0 = (uint64_t)d0;
    u128 c = (d0 >> 64) + d1;
    uint64_t p1 = (uint64_t)c;
    c = (c >> 64) + d2;
    uint64_t p2 = (uint64_t)c;
    uint64_t p3 = (uint64_t)((c >> 64) + d3);
    /* mod p: the bits from 2^130 up fold back times 5 (2^130 = 5 mod p) */
    const u128 hi = ((u128)p3 << 62) | (p2 >> 2);
    const u128 hi5 = hi * 5;
    t = (u128)p0 + (uint64_t)hi5;
    h0 = (uint64_t)t;
    t = (u128)p1 + (uint64_t)(hi5 >> 64) + (uint64_t)(t >> 64);
    h1 = (uint64_t)t;
    h2 = (p2 & 3) + (uint64_t)(t >> 64);
  }
  /* full reduction: subtract p while h >= p (h + 5 reaches 2^130) */
  for (int k = 0; k < 2; k++) {
    u128 t = (u128)h0 + 5;
    const uint64_t g0 = (uint64_t)t;
    t = (u128)h1 + (uint64_t)(t >> 64);
    const uint64_t g1 = (uint64_t)t;
    const uint64_t g2 = h2 + (uint64_t)(t >> 64);
    if (g2 >> 2) {
      h0 = g0;
      h1 = g1;
      h2 = g2 & 3;
    }
  }
  u128 t = (u128)h0 + s0;
  const uint64_t t0 = (uint64_t)t;
  const uint64_t t1 = h1 + s1 + (uint64_t)(t >> 64);
  memcpy(tag, &t0, 8);
  memcpy(tag + 8, &t1, 8);
}

/* The page cipher.  Without integrity: ChaCha20 under K_enc, nonce = page q
 * (u32) || version (u64), counter from 0, over the whole page.  With
 * integrity (NEXT-4: per-page authentication bound to (page, version)): the
 * ChaCha20-Poly1305 AEAD of RFC 8439 Sec. 2.8 with the same key and nonce and
 * no additional data -- the one-time Poly1305 key is the first 32 bytes of
 * block 0, the page's first page_bytes - 16 bytes are encrypted from block 1,
 * and the tag over them and their length fills the last 16 bytes. */
static void aead_tag(const omap_t* m, const uint32_t nonce[3], const uint8_t* ct, uint64_t len,
                     uint8_t tag[16]) {
  uint32_t blk[16];
  oracle_chacha20_block(m->kenc, 0, nonce, blk);
  uint8_t otk[32];
  memcpy(otk, blk, 32);
  uint8_t* mac = malloc(len + 16);
  memcpy(mac, ct, len);
  const uint64_t lens[2] = {0, len}; /* no additional data; len is a multiple of 16 */
  memcpy(mac + len, lens, 16);
  oracle_poly1305(otk, mac, len + 16, tag);
  free(mac);
}

static void page_seal(const omap_t* m, uint64_t q, uint64_t version, uint8_t* buf) {
  if (m->nocrypt) return;
  uint32_t nonce[3] = {(uint32_t)q, (uint32_t)version, (uint32_t)(version >> 32)};
  if (!m->integrity) {
    oracle_chacha20_xor(m->kenc, 0, nonce, buf, m->p.page_bytes);
    return;
  }
  const uint64_t len = m->p.page_bytes - 16;
  oracle_chacha20_xor(m->kenc, 1, nonce, buf, len);
  aead_tag(m, nonce, buf, len, buf + len);
}

/* decrypt a page read from the host; with integrity its tag is checked
 * first (ORC_E_INTEGRITY when it does not match: the host changed the page,
 * or replayed an older version of it) */
static int page_open(const omap_t* m, uint64_t q, uint64_t version, uint8_t* buf) {
  if (m->nocrypt) return ORC_OK;
  uint32_t nonce[3] = {(uint32_t)q, (uint32_t)version, (uint32_t)(version >> 32)};
  if (!m->integrity) {
    oracle_chacha20_xor(m->kenc, 0, nonce, buf, m->p.page_bytes);
    return ORC_OK;
  }
  const uint64_t len = m->p.page_bytes - 16;
  uint8_t tag[16];
  aead_tag(m, nonce, buf, len, tag);
  if (memcmp(tag, buf + len, 16)) return ORC_E_INTEGRITY;
  oracle_chacha20_xor(m->kenc, 1, nonce, buf, len);
  memset(buf + len, 0, 16);
  return ORC_OK;
}

/* Build the plaintext of a page holding `cnt` tuples (sorted here), encrypt
 * it under (q, version) and store it in the host store. */
static void page_store(omap_t* m, uint64_t q, tuple_t* t, uint32_t cnt, uint64_t version) {
  const oracle_info_t* p = &m->p;
  uint8_t* buf = calloc(1, p->page_bytes);
  qsort(t, cnt, sizeof *t, cmp_tuple);
  uint64_t bitmap = cnt == 64 ? ~0ull : ((1ull << cnt) - 1);
  memcpy(buf, &bitmap, 8);
  for (uint32_t s = 0; s < cnt; s++) {
    uint8_t* slot = buf + 16 + (uint64_t)s * p->rec_bytes;
    memcpy(slot, &t[s].key, 8);
    memcpy(slot + 8, t[s].val, p->val_bytes);
  }
  page_seal(m, q, version, buf);
  memcpy(m->pages + q * p->page_bytes, buf, p->page_bytes);
  free(buf);
}

void oracle_kdf(uint64_t seed, uint32_t kprf[8], uint32_t kenc[8]) {
  derive_keys(seed, kprf, kenc);
}

void oracle_page_decrypt(const uint32_t kenc[8], uint64_t q, uint64_t version,
                         const uint8_t* in, uint8_t* out, uint64_t page_bytes) {
  uint32_t nonce[3] = {(uint32_t)q, (uint32_t)version, (uint32_t)(version >> 32)};
  if (out != in) memmove(out, in, page_bytes);
  oracle_chacha20_xor(kenc, 0, nonce, out, page_bytes);
}

int oracle_decrypt_page(const omap_t* m, uint64_t q, uint8_t* out) {
  if (!m || !m->initialized || q >= m->p.M) return ORC_E_ARG;
  memcpy(out, m->pages + q * m->p.page_bytes, m->p.page_bytes);
  return page_open(m, q, m->version[q], out);
}

/* ------------------------------------------------------------------------ */
/* Initialisation ("Fast data initialization", Sec. 4.2): two random bins per */
/* record, P2C placement, position-map insertion, HBM residents into the     */
/* value store, every host page written once (dummy-padded, version 0).      */

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return x < y ? -1 : x > y;
}

/* lowest-index candidate row with the smallest occupancy */
static uint64_t pick_row(const omap_t* m, const uint64_t rows[4]) {
  uint64_t best = rows[0];
  for (int j = 1; j < 4; j++)
    if (m->rowcnt[rows[j]] < m->rowcnt[best]) best = rows[j];
  return best;
}

/* lowest free slot of a position-map row */
static int claim_pm_slot(omap_t* m, uint64_t row, uint64_t* slot) {
  for (uint32_t s = 0; s < m->p.R; s++) {
    uint64_t idx = row * m->p.R + s;
    if (m->pm_loc[idx] == LOC_EMPTY) {
      *slot = idx;
      return ORC_OK;
    }
  }
  return ORC_E_OVERFLOW;
}

/* where oracle_init put each record: its pair, its P2C bin, its
 * position-map row (arrays of n, filled when non-NULL) */
typedef struct {
  uint32_t *b1, *b2, *dest;
  uint64_t* prow;
} placement_t;

static int init_impl(omap_t* m, const uint64_t* keys, const uint8_t* vals, uint64_t n,
                     uint64_t seed, placement_t* out);

int oracle_init(omap_t* m, const uint64_t* keys, const uint8_t* vals, uint64_t n,
                uint64_t seed) {
  return init_impl(m, keys, vals, n, seed, NULL);
}

static int init_impl(omap_t* m, const uint64_t* keys, const uint8_t* vals, uint64_t n,
                     uint64_t seed, placement_t* out) {
  if (!m || n > m->p.N || (n && (!keys || !vals))) return ORC_E_ARG;
  const oracle_info_t* p = &m->p;
  /* keys must be unique (Sec. 2.1) */
  if (n) {
    uint64_t* sorted = malloc(n * sizeof *sorted);
    if (!sorted) return ORC_E_NOMEM;
    memcpy(sorted, keys, n * sizeof *sorted);
    qsort(sorted, n, sizeof *sorted, cmp_u64);
    for (uint64_t i = 1; i < n; i++)
      if (sorted[i] == sorted[i - 1]) {
        free(sorted);
        return ORC_E_DUPKEY;
      }
    free(sorted);
  }
  if (!m->allocated) {
    int rc = alloc_state(m);
    if (rc) return rc;
  }
  reset_state(m);
  m->initialized = 0;
  derive_keys(seed, m->kprf, m->kenc);

  uint32_t* b1 = malloc((n + 1) * sizeof *b1);
  uint32_t* b2 = malloc((n + 1) * sizeof *b2);
  uint32_t* dest = malloc((n + 1) * sizeof *dest);
  uint64_t* prow = malloc((n + 1) * sizeof *prow);
  int rc = ORC_OK;
  if (!b1 || !b2 || !dest || !prow) { rc = ORC_E_NOMEM; goto out; }

#pragma omp parallel for schedule(static)
  for (uint64_t i = 0; i < n; i++) oracle_pair(m->kprf, DOM_INIT, i, p->B, &b1[i], &b2[i]);

  /* P2C and d-choice in rounds of W_r records against round-start loads */
  for (uint64_t lo = 0; lo < n; lo += p->round_width) {
    uint64_t hi = lo + p->round_width < n ? lo + p->round_width : n;
#pragma omp parallel for schedule(static) if (hi - lo >= 512)
    for (uint64_t i = lo; i < hi; i++) {
      dest[i] = m->load[b1[i]] <= m->load[b2[i]] ? b1[i] : b2[i];
      uint64_t rows[4];
      pm_rows(m, keys[i], rows);
      prow[i] = pick_row(m, rows);
    }
    for (uint64_t i = lo; i < hi; i++) {
      m->load[dest[i]]++;
      if (m->load[dest[i]] > p->lmax) { rc = ORC_E_OVERFLOW; goto out; }
      uint64_t slot;
      if (claim_pm_slot(m, prow[i], &slot)) { rc = ORC_E_OVERFLOW; goto out; }
      m->rowcnt[prow[i]]++;
      m->pm_key[slot] = keys[i];
      m->pm_b1[slot] = b1[i];
      m->pm_b2[slot] = b2[i];
      m->pm_which[slot] = dest[i] == b2[i];
      if (dest[i] < p->K) {
        uint64_t vs;
        if (ring_pop(m, &vs)) { rc = ORC_E_OVERFLOW; goto out; }
        m->vs_key[vs] = keys[i];
        memcpy(m->vs_val + vs * p->val_bytes, vals + i * p->val_bytes, p->val_bytes);
        m->vs_pm[vs] = slot;
        m->vs_live[vs] = 1;
        m->pm_loc[slot] = LOC_HBM;
        m->pm_ptr[slot] = vs;
        m->n_hbm++;
      } else {
        m->pm_loc[slot] = LOC_HOST;
        m->pm_ptr[slot] = 0;
        m->n_host++;
      }
    }
  }
  for (uint64_t b = 0; b < p->B; b++)
    if (m->load[b] > m->peak_load) m->peak_load = m->load[b];

  /* every host page: its records (by P2C destination), sorted, padded */
  {
    uint64_t* start = calloc(p->M + 1, sizeof *start);
    tuple_t* all = malloc((n + 1) * sizeof *all);
    uint64_t* fill = calloc(p->M, sizeof *fill);
    if (!start || !all || !fill) {
      free(start); free(all); free(fill);
      rc = ORC_E_NOMEM;
      goto out;
    }
    for (uint64_t q = 0; q < p->M; q++) start[q + 1] = start[q] + m->load[p->K + q];
    for (uint64_t i = 0; i < n; i++)
      if (dest[i] >= p->K) {
        uint64_t q = dest[i] - p->K;
        all[start[q] + fill[q]].key = keys[i];
        all[start[q] + fill[q]].val = vals + i * p->val_bytes;
        fill[q]++;
      }
#pragma omp parallel for schedule(static)
    for (uint64_t q = 0; q < p->M; q++)
      page_store(m, q, all + start[q], (uint32_t)(start[q + 1] - start[q]), 0);
    free(start); free(all); free(fill);
  }
  m->peak_hbm = m->n_hbm;
  m->initialized = 1;
  if (out && n) {
    memcpy(out->b1, b1, n * sizeof *b1);
    memcpy(out->b2, b2, n * sizeof *b2);
    memcpy(out->dest, dest, n * sizeof *dest);
    memcpy(out->prow, prow, n * sizeof *prow);
  }
out:
  free(b1); free(b2); free(dest); free(prow);
  if (rc) m->poisoned = 1;
  return rc;
}

/* The data owner's preprocessing (Sec. 4.2 "Fast data initialization"): the
 * placement oracle_init makes for these records and this seed, as an image
 * in bin-major order -- bin 0's records, then bin 1's, ... (bins 0..K-1 are
 * the HBM bins, bin K + q is host page q), ascending record index within a
 * bin -- with each record's key and value, its pair b1 | b2 << 32, its
 * position-map row with bit 31 set when it sits in b2, and every bin's
 * record count.  The map is built as by oracle_init. */
int oracle_prepare(omap_t* m, const uint64_t* keys, const uint8_t* vals, uint64_t n,
                   uint64_t seed, uint64_t* img_keys, uint8_t* img_vals, uint64_t* img_pairs,
                   uint32_t* img_rows, uint8_t* counts) {
  if (!m || n > m->p.N || (n && (!keys || !vals || !img_keys || !img_vals || !img_pairs ||
                                 !img_rows)) || !counts)
    return ORC_E_ARG;
  placement_t pl = {malloc((n + 1) * 4), malloc((n + 1) * 4), malloc((n + 1) * 4),
                    malloc((n + 1) * 8)};
  uint64_t* start = calloc(m->p.B + 1, sizeof *start);
  int rc = (!pl.b1 || !pl.b2 || !pl.dest || !pl.prow || !start) ? ORC_E_NOMEM
                                                                 : init_impl(m, keys, vals, n, seed, &pl);
  if (rc == ORC_OK) {
    const oracle_info_t* p = &m->p;
    const uint32_t vb = p->val_bytes;
    for (uint64_t b = 0; b < p->B; b++) {
      counts[b] = (uint8_t)m->load[b];
      start[b + 1] = start[b] + m->load[b];
    }
    for (uint64_t i = 0; i < n; i++) {
      const uint64_t at = start[pl.dest[i]]++;
      img_keys[at] = keys[i];
      memcpy(img_vals + at * vb, vals + i * vb, vb);
      img_pairs[at] = (uint64_t)pl.b1[i] | ((uint64_t)pl.b2[i] << 32);
      img_rows[at] = (uint32_t)pl.prow[i] | (pl.dest[i] == pl.b2[i] ? 0x80000000u : 0u);
    }
  }
  free(pl.b1); free(pl.b2); free(pl.dest); free(pl.prow); free(start);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Batched access: Alg. 1 applied to a batch of operations (Sec. 3.1), with  */
/* the module order of Sec. 4.1 (KS -> VAC -> exec -> write-back -> RMP).    */

typedef struct {
  uint64_t key;
  uint64_t idx;
} keyidx_t;

static int cmp_keyidx(const void* a, const void* b) {
  const keyidx_t* x = a;
  const keyidx_t* y = b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->idx < y->idx ? -1 : x->idx > y->idx;
}

/* find a key in the position map: scan all slots of its d rows */
static uint64_t pm_find(const omap_t* m, uint64_t key) {
  uint64_t rows[4];
  pm_rows(m, key, rows);
  for (int j = 0; j < 4; j++)
    for (uint32_t s = 0; s < m->p.R; s++) {
      uint64_t idx = rows[j] * m->p.R + s;
      if (m->pm_loc[idx] != LOC_EMPTY && m->pm_key[idx] == key) return idx;
    }
  return NO_INDEX;
}

typedef struct {
  uint64_t q;        /* page number */
  uint8_t* plain;    /* decrypted page */
  uint32_t cnt;      /* real tuples in the page as read */
  uint64_t removed;  /* bitmap of slots removed by find_remove */
} dpage_t;

static int access_batch(omap_t* m, const uint8_t* ops, const uint64_t* keys,
                        const uint8_t* vin, uint8_t* vout, uint8_t* status, uint64_t n) {
  const oracle_info_t* p = &m->p;
  const uint32_t vb = p->val_bytes;
  int rc = ORC_OK;
  uint64_t t0 = m->t;

  keyidx_t* ki = malloc(n * sizeof *ki);
  uint64_t* leader = malloc(n * sizeof *leader);
  uint64_t* prevw = malloc(n * sizeof *prevw);  /* last PUT/DEL before i, same key */
  uint64_t* lastw = malloc(n * sizeof *lastw);  /* for leaders: last PUT/DEL of group */
  uint64_t* hit = malloc(n * sizeof *hit);      /* for leaders: pm slot or NO_INDEX */
  uint32_t* p1 = malloc(n * sizeof *p1);
  uint32_t* p2 = malloc(n * sizeof *p2);
  uint8_t* init_present = calloc(n, 1);
  uint8_t* init_val = calloc(n, vb);
  int64_t* dindex = m->dindex;
  dpage_t* dp = calloc(2 * n, sizeof *dp);
  uint64_t nd = 0;
  if (!ki || !leader || !prevw || !lastw || !hit || !p1 || !p2 || !init_present ||
      !init_val || !dp) {
    rc = ORC_E_NOMEM;
    goto out;
  }

  /* 1. group operations by key: leader = first operation on the key; for each
   *    operation the previous writer on the same key (batch semantics). */
  for (uint64_t i = 0; i < n; i++) {
    ki[i].key = keys[i];
    ki[i].idx = i;
  }
  qsort(ki, n, sizeof *ki, cmp_keyidx);
  for (uint64_t a = 0; a < n;) {
    uint64_t b = a;
    while (b < n && ki[b].key == ki[a].key) b++;
    uint64_t lead = ki[a].idx, writer = NO_INDEX;
    for (uint64_t j = a; j < b; j++) {
      uint64_t i = ki[j].idx;
      leader[i] = lead;
      prevw[i] = writer;
      if (ops[i] != OP_GET) writer = i;
    }
    lastw[lead] = writer;
    a = b;
  }

  /* 2. key search (KS): leaders look up the position map; a hit yields the
   *    stored pair, every other operation (miss, duplicate) a fresh random
   *    pair (Alg. 1 line 3, Sec. 4.1 step 3). */
#pragma omp parallel for schedule(static) if (n >= 64)
  for (uint64_t i = 0; i < n; i++) {
    hit[i] = NO_INDEX;
    if (leader[i] == i) hit[i] = pm_find(m, keys[i]);
    if (hit[i] != NO_INDEX) {
      p1[i] = m->pm_b1[hit[i]];
      p2[i] = m->pm_b2[hit[i]];
    } else {
      oracle_pair(m->kprf, DOM_DUMMY, t0 + i, p->B, &p1[i], &p2[i]);
    }
  }

  /* 3. value access (VAC): read every host bin of every pair, in operation
   *    order, first bin then second (Alg. 1 lines 5-8); decrypt each distinct
   *    page once (the decryptions are independent of one another). */
  for (uint64_t i = 0; i < n; i++) {
    uint32_t pair[2] = {p1[i], p2[i]};
    for (int j = 0; j < 2; j++) {
      if (pair[j] < p->K) continue; /* HBM bin: no host access (Sec. 3.2) */
      uint64_t q = pair[j] - p->K;
      trace_add(m, (uint32_t)q);
      if (dindex[q] >= 0) continue;
      dindex[q] = (int64_t)nd;
      dp[nd].q = q;
      dp[nd].plain = malloc(p->page_bytes);
      if (!dp[nd].plain) { rc = ORC_E_NOMEM; goto out; }
      memcpy(dp[nd].plain, m->pages + q * p->page_bytes, p->page_bytes);
      nd++;
    }
  }
  int open_rc = ORC_OK;
#pragma omp parallel for schedule(static) if (nd >= 64)
  for (uint64_t d = 0; d < nd; d++) {
    if (page_open(m, dp[d].q, m->version[dp[d].q], dp[d].plain) != ORC_OK) {
#pragma omp critical
      open_rc = ORC_E_INTEGRITY;
    }
    uint64_t bitmap;
    memcpy(&bitmap, dp[d].plain, 8);
    uint32_t cnt = 0;
    while (cnt < 64 && (bitmap >> cnt) & 1) cnt++;
    dp[d].cnt = cnt;
  }
  if (open_rc) { rc = open_rc; goto out; }

  /* 4. find_remove (Alg. 1 lines 6 and 9): take each hit key out of the HBM
   *    store, the stash or its page; its bin's load drops by one. */
  for (uint64_t i = 0; i < n; i++) {
    if (hit[i] == NO_INDEX) continue;
    uint64_t s = hit[i];
    uint32_t bin = m->pm_which[s] ? m->pm_b2[s] : m->pm_b1[s];
    init_present[i] = 1;
    if (m->pm_loc[s] == LOC_HOST) {
      uint64_t q = bin - p->K;
      if (dindex[q] < 0) { rc = ORC_E_INTERNAL; goto out; }
      dpage_t* d = &dp[dindex[q]];
      uint32_t found = UINT32_MAX;
      for (uint32_t k = 0; k < d->cnt; k++) {
        uint64_t key;
        memcpy(&key, d->plain + 16 + (uint64_t)k * p->rec_bytes, 8);
        if (key == keys[i] && !((d->removed >> k) & 1)) found = k;
      }
      if (found == UINT32_MAX) { rc = ORC_E_INTERNAL; goto out; }
      memcpy(init_val + i * vb, d->plain + 16 + (uint64_t)found * p->rec_bytes + 8, vb);
      d->removed |= 1ull << found;
      m->n_host--;
    } else {
      uint64_t vs = m->pm_ptr[s];
      memcpy(init_val + i * vb, m->vs_val + vs * vb, vb);
      m->vs_live[vs] = 0;
      ring_push(m, vs);
      if (m->pm_loc[s] == LOC_HBM) m->n_hbm--; else m->n_stash--;
    }
    m->load[bin]--;
  }

  /* 5. exec_cmd (Alg. 1 line 12): each operation sees the state left by the
   *    previous writer on its key, else the state found above. */
  for (uint64_t i = 0; i < n; i++) {
    uint64_t w = prevw[i], l = leader[i];
    int present;
    const uint8_t* val;
    if (w != NO_INDEX) {
      present = ops[w] == OP_PUT;
      val = vin + w * vb;
    } else {
      present = init_present[l];
      val = init_val + l * vb;
    }
    if (status) status[i] = (uint8_t)present;
    if (ops[i] == OP_GET && present) memcpy(vout + i * vb, val, vb);
    else memset(vout + i * vb, 0, vb);
  }

  /* 6. deleted keys leave the position map before any insertion */
  for (uint64_t i = 0; i < n; i++) {
    if (hit[i] == NO_INDEX) continue;
    uint64_t w = lastw[i];
    if (w != NO_INDEX && ops[w] == OP_DEL) {
      uint64_t s = hit[i];
      m->pm_loc[s] = LOC_EMPTY;
      m->rowcnt[s / p->R]--;
    }
  }

  /* 7. write-back with eviction (Alg. 1 line 10): every distinct page read,
   *    in first-read order, gets its remaining tuples plus every stash item
   *    bound for it, under a fresh version.  A page's new content depends on
   *    its own tuples and stash items only, so the pages are built and
   *    encrypted independently; the bookkeeping that follows (stash items
   *    leave, slots return to the free ring, trace) runs in page order. */
  int wb_rc = ORC_OK;
#pragma omp parallel for schedule(static) if (nd >= 64)
  for (uint64_t d = 0; d < nd; d++) {
    dpage_t* pg = &dp[d];
    uint64_t q = pg->q;
    tuple_t* t = malloc((pg->cnt + p->lmax + 1) * sizeof *t);
    uint32_t cnt = 0;
    const int nomem = !t;
    int bad = nomem;
    for (uint32_t k = 0; !bad && k < pg->cnt; k++) {
      if ((pg->removed >> k) & 1) continue;
      uint8_t* slot = pg->plain + 16 + (uint64_t)k * p->rec_bytes;
      memcpy(&t[cnt].key, slot, 8);
      t[cnt].val = slot + 8;
      cnt++;
    }
    for (uint32_t r = 0; !bad && r < m->revcnt[q]; r++) {
      uint64_t vs = m->rev[q * p->lmax + r];
      if (!m->vs_live[vs]) continue; /* taken out by find_remove above */
      if (cnt >= p->lmax) { bad = 1; break; }
      t[cnt].key = m->vs_key[vs];
      t[cnt].val = m->vs_val + vs * vb;
      cnt++;
    }
    if (!bad) {
      m->version[q]++;
      page_store(m, q, t, cnt, m->version[q]);
    }
    free(t);
    if (bad) {
#pragma omp critical
      wb_rc = nomem ? ORC_E_NOMEM : ORC_E_INTERNAL;
    }
  }
  if (wb_rc) { rc = wb_rc; goto out; }
  for (uint64_t d = 0; d < nd; d++) {
    uint64_t q = dp[d].q;
    for (uint32_t r = 0; r < m->revcnt[q]; r++) {
      uint64_t vs = m->rev[q * p->lmax + r];
      if (!m->vs_live[vs]) continue;
      m->pm_loc[m->vs_pm[vs]] = LOC_HOST;
      m->vs_live[vs] = 0;
      ring_push(m, vs);
      m->n_stash--;
      m->n_host++;
    }
    m->revcnt[q] = 0;
    trace_add(m, (uint32_t)q | 0x80000000u);
  }

  /* 8. remap + P2C (Alg. 1 lines 13-14, Sec. 4.1 step 5): every key present
   *    after the batch gets a fresh pair and goes to the less-loaded bin; HBM
   *    bins take it directly, host bins through the stash.  Rounds of W_r
   *    operation slots decide on round-start loads. */
  for (uint64_t lo = 0; lo < n; lo += p->round_width) {
    uint64_t hi = lo + p->round_width < n ? lo + p->round_width : n;
    uint64_t cnt = 0;
    for (uint64_t i = lo; i < hi; i++) cnt++;
    uint32_t* nb1 = malloc(cnt * sizeof *nb1);
    uint32_t* nb2 = malloc(cnt * sizeof *nb2);
    uint32_t* nd_ = malloc(cnt * sizeof *nd_);
    uint64_t* nrow = malloc(cnt * sizeof *nrow);
    uint8_t* live = calloc(cnt, 1);
    if (!nb1 || !nb2 || !nd_ || !nrow || !live) {
      free(nb1); free(nb2); free(nd_); free(nrow); free(live);
      rc = ORC_E_NOMEM;
      goto out;
    }
    /* decide */
#pragma omp parallel for schedule(static) if (hi - lo >= 64)
    for (uint64_t i = lo; i < hi; i++) {
      uint64_t k = i - lo;
      if (leader[i] != i) continue;
      uint64_t w = lastw[i];
      int final_present = w != NO_INDEX ? ops[w] == OP_PUT : init_present[i];
      if (!final_present) continue;
      live[k] = 1;
      oracle_pair(m->kprf, DOM_REMAP, t0 + i, p->B, &nb1[k], &nb2[k]);
      nd_[k] = m->load[nb1[k]] <= m->load[nb2[k]] ? nb1[k] : nb2[k];
      if (hit[i] == NO_INDEX) {
        uint64_t rows[4];
        pm_rows(m, keys[i], rows);
        nrow[k] = pick_row(m, rows);
      }
    }
    /* apply */
    for (uint64_t i = lo; i < hi && rc == ORC_OK; i++) {
      uint64_t k = i - lo;
      if (!live[k]) continue;
      uint64_t w = lastw[i];
      const uint8_t* val = w != NO_INDEX ? vin + w * vb : init_val + i * vb;
      m->load[nd_[k]]++;
      if (m->load[nd_[k]] > m->peak_load) m->peak_load = m->load[nd_[k]];
      if (m->load[nd_[k]] > p->lmax) { rc = ORC_E_OVERFLOW; break; }
      uint64_t s = hit[i];
      if (s == NO_INDEX) {
        if (claim_pm_slot(m, nrow[k], &s)) { rc = ORC_E_OVERFLOW; break; }
        m->rowcnt[nrow[k]]++;
        m->pm_key[s] = keys[i];
      }
      uint64_t vs;
      if (ring_pop(m, &vs)) { rc = ORC_E_OVERFLOW; break; }
      m->vs_key[vs] = keys[i];
      memcpy(m->vs_val + vs * vb, val, vb);
      m->vs_pm[vs] = s;
      m->vs_live[vs] = 1;
      m->pm_b1[s] = nb1[k];
      m->pm_b2[s] = nb2[k];
      m->pm_which[s] = nd_[k] == nb2[k];
      m->pm_ptr[s] = vs;
      if (nd_[k] < p->K) {
        m->pm_loc[s] = LOC_HBM;
        m->n_hbm++;
      } else {
        uint64_t q = nd_[k] - p->K;
        if (m->revcnt[q] >= p->lmax) { rc = ORC_E_INTERNAL; break; }
        m->rev[q * p->lmax + m->revcnt[q]++] = vs;
        m->pm_loc[s] = LOC_STASH;
        m->n_stash++;
      }
    }
    free(nb1); free(nb2); free(nd_); free(nrow); free(live);
    if (rc) goto out;
  }
  if (m->n_stash > m->peak_stash) m->peak_stash = m->n_stash;
  if (m->n_hbm > m->peak_hbm) m->peak_hbm = m->n_hbm;
  m->t = t0 + n;

out:
  if (dp)
    for (uint64_t d = 0; d < nd; d++) {
      dindex[dp[d].q] = -1;
      free(dp[d].plain);
    }
  free(ki); free(leader); free(prevw); free(lastw); free(hit); free(p1); free(p2);
  free(init_present); free(init_val); free(dp);
  return rc;
}

int oracle_access(omap_t* m, const uint8_t* ops, const uint64_t* keys,
                  const uint8_t* vals_in, uint8_t* vals_out, uint8_t* status_out,
                  uint64_t n) {
  if (!m) return ORC_E_ARG;
  if (!m->initialized || m->poisoned) return ORC_E_STATE;
  if (n == 0) return ORC_OK;
  if (!ops || !keys || !vals_in || !vals_out) return ORC_E_ARG;
  for (uint64_t i = 0; i < n; i++)
    if (ops[i] > OP_DEL) return ORC_E_ARG;
  const uint32_t vb = m->p.val_bytes;
  for (uint64_t lo = 0; lo < n; lo += m->batch_width) {
    uint64_t cnt = n - lo < m->batch_width ? n - lo : m->batch_width;
    int rc = access_batch(m, ops + lo, keys + lo, vals_in + lo * vb, vals_out + lo * vb,
                          status_out ? status_out + lo : NULL, cnt);
    if (rc) {
      m->poisoned = 1;
      return rc;
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */

/* Host threads the loops above may use: the library built with OpenMP runs
 * its independent loops (PRF draws, per-round decisions, page decryption and
 * encryption) on up to `n` threads; built without it, it is single-threaded
 * and this returns 1.  Results do not depend on the thread count. */
int oracle_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

int oracle_info(const omap_t* m, oracle_info_t* out) {
  if (!m || !out) return ORC_E_ARG;
  *out = m->p;
  return ORC_OK;
}

int oracle_stats(const omap_t* m, oracle_stats_t* out) {
  if (!m || !out) return ORC_E_ARG;
  memset(out, 0, sizeof *out);
  out->ops = m->t;
  out->n_hbm = m->n_hbm;
  out->n_stash = m->n_stash;
  out->n_host = m->n_host;
  out->peak_stash = m->peak_stash;
  out->peak_hbm = m->peak_hbm;
  out->peak_load = m->peak_load;
  if (m->allocated) {
    for (uint64_t b = 0; b < m->p.B; b++)
      if (m->load[b] > out->max_load) out->max_load = m->load[b];
    for (uint64_t r = 0; r < m->p.rows; r++)
      if (m->rowcnt[r] > out->max_row) out->max_row = m->rowcnt[r];
  }
  return ORC_OK;
}

const uint8_t* oracle_pages(const omap_t* m) { return m ? m->pages : NULL; }

int oracle_loads(const omap_t* m, uint8_t* out) {
  if (!m || !m->allocated) return ORC_E_STATE;
  for (uint64_t b = 0; b < m->p.B; b++) out[b] = (uint8_t)m->load[b];
  return ORC_OK;
}

int oracle_rowcounts(const omap_t* m, uint32_t* out) {
  if (!m || !m->allocated) return ORC_E_STATE;
  memcpy(out, m->rowcnt, m->p.rows * sizeof *out);
  return ORC_OK;
}

int oracle_versions(const omap_t* m, uint64_t* out) {
  if (!m || !m->allocated) return ORC_E_STATE;
  memcpy(out, m->version, m->p.M * sizeof *out);
  return ORC_OK;
}

uint64_t oracle_trace_len(const omap_t* m) { return m ? m->trace_len : 0; }

uint64_t oracle_trace_copy(const omap_t* m, uint32_t* out, uint64_t cap) {
  if (!m) return 0;
  uint64_t n = m->trace_len < cap ? m->trace_len : cap;
  memcpy(out, m->trace, n * sizeof *out);
  return n;
}

void oracle_trace_clear(omap_t* m) {
  if (m) m->trace_len = 0;
}

int oracle_keys(const omap_t* m, uint32_t* kprf, uint32_t* kenc) {
  if (!m || !m->initialized) return ORC_E_STATE;
  memcpy(kprf, m->kprf, sizeof m->kprf);
  memcpy(kenc, m->kenc, sizeof m->kenc);
  return ORC_OK;
}
