// bolt_internal.cuh -- device-side types and primitives of the B300 BOLT map.
//
// Shared by the build, sort and access translation units.  Nothing here is
// shared with the CPU oracle: every primitive is written afresh for the GPU.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/bolt.h"

namespace bdev {

// ---------------------------------------------------------------------------
// Error bits set by kernels in the device error word (Sec. 3.3: a capacity
// bound may be exceeded with probability 1/O(N); that is reported, not
// silently absorbed).
enum : uint32_t {
  ERR_LOAD = 1u << 0,      // a bin load went above lmax (Claim 3.2)
  ERR_ROW = 1u << 1,       // a position-map row went above R (Sec. 4.2)
  ERR_VS = 1u << 2,        // value store (HBM bins + stash) full (Claims 3.3/3.4)
  ERR_REV = 1u << 3,       // reverse-index list over lmax entries
  ERR_NOTFOUND = 1u << 4,  // a position-map hit was not found where it points
  ERR_PAGE = 1u << 5,      // a page held more than lmax tuples
  ERR_TIMEOUT = 1u << 6,   // a bounded device wait gave up
  ERR_INTEGRITY = 1u << 7, // a page read from the host failed its tag
  ERR_OVERFLOW_MASK = ERR_LOAD | ERR_ROW | ERR_VS | ERR_REV | ERR_PAGE,
};

// position-map slot metadata: bits 0-1 location, bit 2 which-bin, bits 3-31
// value-store slot (Sec. 4.2: flag bit for HBM vs stash, index pointer)
enum : uint32_t { LOC_EMPTY = 0, LOC_HOST = 1, LOC_HBM = 2, LOC_STASH = 3 };
__host__ __device__ __forceinline__ uint32_t meta_make(uint32_t loc, uint32_t which,
                                                       uint32_t ptr) {
  return loc | (which << 2) | (ptr << 3);
}
__host__ __device__ __forceinline__ uint32_t meta_loc(uint32_t m) { return m & 3u; }
__host__ __device__ __forceinline__ uint32_t meta_which(uint32_t m) { return (m >> 2) & 1u; }
__host__ __device__ __forceinline__ uint32_t meta_ptr(uint32_t m) { return m >> 3; }

enum : uint32_t { DOM_INIT = 1, DOM_PM = 2, DOM_REMAP = 3, DOM_DUMMY = 4 };
enum : uint8_t { OP_GET = 0, OP_PUT = 1, OP_DEL = 2 };
constexpr uint32_t NONE32 = 0xffffffffu;

// Map parameters and device pointers, passed by value to every kernel.
struct MapDev {
  // sizing (Sec. 3.3, Sec. 4.2)
  uint64_t N, B, K, M, rows, Wr, vs_cap;
  uint32_t R, lmax, vb, rec, page_bytes;
  uint32_t spin_limit;  // iterations a bounded device wait spins before it gives up
  uint32_t kprf[8], kenc[8];
  // state in HBM
  uint32_t* load;      // packed u8 bin loads, B bytes (4 per word)
  uint32_t* rowcnt;    // packed u8 position-map row counts
  uint64_t* pm_key;    // [rows*R]
  uint64_t* pm_bins;   // [rows*R] b1 | b2 << 32
  uint32_t* pm_meta;   // [rows*R]
  uint64_t* vs_key;    // [vs_cap] value store = HBM bins + stash
  uint8_t* vs_val;     // [vs_cap * vb]
  uint32_t* vs_pm;     // [vs_cap] owning position-map slot
  uint8_t* vs_live;    // [vs_cap]
  uint32_t* ring;      // [vs_cap] free value-store slots
  unsigned long long* ring_ctr;  // [0] head (pops), [1] tail (pushes)
  uint32_t* rev;       // [M * lmax] reverse index: stash slots bound for page q
  uint32_t* revcnt;    // packed u8 counts, M bytes
  uint64_t* version;   // [M] page write counters (cipher nonces)
  uint8_t* pages;      // device alias of the pinned host pages [M * page_bytes]
  uint32_t* err;       // error word
  unsigned long long* stat;  // [ST_WORDS] occupancy counters and their peaks (below)
  uint32_t* trace;     // host-access trace (optional)
  unsigned long long* trace_len;
  uint64_t trace_cap;
  uint32_t trace_on;
  uint32_t integrity;  // 1: pages are ChaCha20-Poly1305 sealed (tag in the last 16 bytes)
};

// ---------------------------------------------------------------------------
// Packed byte counters: 4 counters per 32-bit word, updated with word atomics.
__device__ __forceinline__ uint32_t byte_get(const uint32_t* w, uint64_t i) {
  return reinterpret_cast<const uint8_t*>(w)[i];
}
__device__ __forceinline__ uint32_t byte_inc(uint32_t* w, uint64_t i) {
  uint32_t sh = (uint32_t)(i & 3) * 8;
  return (atomicAdd(w + (i >> 2), 1u << sh) >> sh) & 0xffu;  // old value
}
// the increment alone (no result: nothing waits for the atomic)
__device__ __forceinline__ void byte_add(uint32_t* w, uint64_t i) {
  uint32_t sh = (uint32_t)(i & 3) * 8;
  atomicAdd(w + (i >> 2), 1u << sh);
}
__device__ __forceinline__ void byte_dec(uint32_t* w, uint64_t i) {
  uint32_t sh = (uint32_t)(i & 3) * 8;
  atomicSub(w + (i >> 2), 1u << sh);
}

__device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) { return __umul64hi(a, b); }

// ---------------------------------------------------------------------------
// ChaCha20 block function (RFC 8439): 16-word state = 4 constant words,
// 8 key words, block counter, 3 nonce words; 10 double rounds of column then
// diagonal quarter rounds; output = final state + input state.

#define BOLT_QR(a, b, c, d)             \
  a += b; d ^= a; d = __funnelshift_l(d, d, 16); \
  c += d; b ^= c; b = __funnelshift_l(b, b, 12); \
  a += b; d ^= a; d = __funnelshift_l(d, d, 8);  \
  c += d; b ^= c; b = __funnelshift_l(b, b, 7);

__device__ __forceinline__ void chacha_block(const uint32_t* key, uint32_t counter, uint32_t n0,
                                             uint32_t n1, uint32_t n2, uint32_t out[16]) {
  uint32_t x0 = 0x61707865u, x1 = 0x3320646eu, x2 = 0x79622d32u, x3 = 0x6b206574u;
  uint32_t x4 = key[0], x5 = key[1], x6 = key[2], x7 = key[3];
  uint32_t x8 = key[4], x9 = key[5], x10 = key[6], x11 = key[7];
  uint32_t x12 = counter, x13 = n0, x14 = n1, x15 = n2;
  // the 10 double rounds stay a loop: unrolled, the block is ~1000
  // instructions of straight-line code, and in the latency-bound kernels
  // (one CTA per batch) fetching it costs more than the loop's branches
#pragma unroll 1
  for (int r = 0; r < 10; r++) {
    BOLT_QR(x0, x4, x8, x12);
    BOLT_QR(x1, x5, x9, x13);
    BOLT_QR(x2, x6, x10, x14);
    BOLT_QR(x3, x7, x11, x15);
    BOLT_QR(x0, x5, x10, x15);
    BOLT_QR(x1, x6, x11, x12);
    BOLT_QR(x2, x7, x8, x13);
    BOLT_QR(x3, x4, x9, x14);
  }
  out[0] = x0 + 0x61707865u; out[1] = x1 + 0x3320646eu;
  out[2] = x2 + 0x79622d32u; out[3] = x3 + 0x6b206574u;
  out[4] = x4 + key[0]; out[5] = x5 + key[1]; out[6] = x6 + key[2]; out[7] = x7 + key[3];
  out[8] = x8 + key[4]; out[9] = x9 + key[5]; out[10] = x10 + key[6]; out[11] = x11 + key[7];
  out[12] = x12 + counter; out[13] = x13 + n0; out[14] = x14 + n1; out[15] = x15 + n2;
}

// Four lanes compute one block together: lane g (= lane & 3) holds column g
// of the state (words g, 4+g, 8+g, 12+g).  Column rounds are lane-local;
// diagonal rounds rotate rows 1-3 across the quad with shuffles.  Returns
// words 4g..4g+3 of the block, i.e. key-stream bytes [16g, 16g+16).  All 32
// lanes of the warp must call it (full-mask shuffles).
__device__ __forceinline__ uint4 chacha_quad(const uint32_t* key, uint32_t counter, uint32_t n0,
                                             uint32_t n1, uint32_t n2) {
  const int lane = threadIdx.x & 31;
  const int g = lane & 3;
  const int base = lane & ~3;
  const uint32_t c_const = g == 0 ? 0x61707865u : g == 1 ? 0x3320646eu
                         : g == 2 ? 0x79622d32u : 0x6b206574u;
  const uint32_t ib = g == 0 ? key[0] : g == 1 ? key[1] : g == 2 ? key[2] : key[3];
  const uint32_t ic = g == 0 ? key[4] : g == 1 ? key[5] : g == 2 ? key[6] : key[7];
  const uint32_t id = g == 0 ? counter : g == 1 ? n0 : g == 2 ? n1 : n2;
  uint32_t a = c_const, b = ib, c = ic, d = id;
  const int s1 = base | ((g + 1) & 3), s2 = base | ((g + 2) & 3), s3 = base | ((g + 3) & 3);
#pragma unroll 1
  for (int r = 0; r < 10; r++) {
    BOLT_QR(a, b, c, d);
    b = __shfl_sync(0xffffffffu, b, s1);
    c = __shfl_sync(0xffffffffu, c, s2);
    d = __shfl_sync(0xffffffffu, d, s3);
    BOLT_QR(a, b, c, d);
    b = __shfl_sync(0xffffffffu, b, s3);
    c = __shfl_sync(0xffffffffu, c, s2);
    d = __shfl_sync(0xffffffffu, d, s1);
  }
  a += c_const; b += ib; c += ic; d += id;
  // Transpose the quad: this lane needs row g of every column k (word 4g+k).
  // In round r it receives from lane (g + r) & 3 that lane's row g, which the
  // sender selects as its row (own index - r) & 3.
  uint32_t v[4];
#pragma unroll
  for (int r = 0; r < 4; r++) {
    const int want = (g - r) & 3;
    const uint32_t send = want == 0 ? a : want == 1 ? b : want == 2 ? c : d;
    v[r] = __shfl_sync(0xffffffffu, send, base | ((g + r) & 3));
  }
  // v[r] is column (g + r) & 3, i.e. word 4g + ((g + r) & 3); word 4g + k is
  // v[(k - g) & 3]
  const int r0 = (0 - g) & 3, r1 = (1 - g) & 3, r2 = (2 - g) & 3, r3 = (3 - g) & 3;
  auto pick = [&](int r) { return r == 0 ? v[0] : r == 1 ? v[1] : r == 2 ? v[2] : v[3]; };
  return make_uint4(pick(r0), pick(r1), pick(r2), pick(r3));
}

// Two chacha_quad blocks at once (same key, their own counters and nonces):
// the two blocks' quarter-rounds and shuffles are independent, so they
// overlap and a warp that needs both waits for about one.
__device__ __forceinline__ void chacha_quad2(const uint32_t* key, uint32_t ctr0, uint32_t n00,
                                             uint32_t n01, uint32_t n02, uint32_t ctr1,
                                             uint32_t n10, uint32_t n11, uint32_t n12,
                                             uint4& out0, uint4& out1) {
  const int lane = threadIdx.x & 31;
  const int g = lane & 3;
  const int base = lane & ~3;
  const uint32_t c_const = g == 0 ? 0x61707865u : g == 1 ? 0x3320646eu
                         : g == 2 ? 0x79622d32u : 0x6b206574u;
  const uint32_t ib = g == 0 ? key[0] : g == 1 ? key[1] : g == 2 ? key[2] : key[3];
  const uint32_t ic = g == 0 ? key[4] : g == 1 ? key[5] : g == 2 ? key[6] : key[7];
  const uint32_t id0 = g == 0 ? ctr0 : g == 1 ? n00 : g == 2 ? n01 : n02;
  const uint32_t id1 = g == 0 ? ctr1 : g == 1 ? n10 : g == 2 ? n11 : n12;
  uint32_t a0 = c_const, b0 = ib, c0 = ic, d0 = id0;
  uint32_t a1 = c_const, b1 = ib, c1 = ic, d1 = id1;
  const int s1 = base | ((g + 1) & 3), s2 = base | ((g + 2) & 3), s3 = base | ((g + 3) & 3);
#pragma unroll 1
  for (int r = 0; r < 10; r++) {
    BOLT_QR(a0, b0, c0, d0);
    BOLT_QR(a1, b1, c1, d1);
    b0 = __shfl_sync(0xffffffffu, b0, s1);
    b1 = __shfl_sync(0xffffffffu, b1, s1);
    c0 = __shfl_sync(0xffffffffu, c0, s2);
    c1 = __shfl_sync(0xffffffffu, c1, s2);
    d0 = __shfl_sync(0xffffffffu, d0, s3);
    d1 = __shfl_sync(0xffffffffu, d1, s3);
    BOLT_QR(a0, b0, c0, d0);
    BOLT_QR(a1, b1, c1, d1);
    b0 = __shfl_sync(0xffffffffu, b0, s3);
    b1 = __shfl_sync(0xffffffffu, b1, s3);
    c0 = __shfl_sync(0xffffffffu, c0, s2);
    c1 = __shfl_sync(0xffffffffu, c1, s2);
    d0 = __shfl_sync(0xffffffffu, d0, s1);
    d1 = __shfl_sync(0xffffffffu, d1, s1);
  }
  a0 += c_const; b0 += ib; c0 += ic; d0 += id0;
  a1 += c_const; b1 += ib; c1 += ic; d1 += id1;
  // the quad's transpose, as in chacha_quad
  auto transpose = [&](uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    uint32_t v[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const int want = (g - r) & 3;
      const uint32_t send = want == 0 ? a : want == 1 ? b : want == 2 ? c : d;
      v[r] = __shfl_sync(0xffffffffu, send, base | ((g + r) & 3));
    }
    const int r0 = (0 - g) & 3, r1 = (1 - g) & 3, r2 = (2 - g) & 3, r3 = (3 - g) & 3;
    auto pick = [&](int r) { return r == 0 ? v[0] : r == 1 ? v[1] : r == 2 ? v[2] : v[3]; };
    return make_uint4(pick(r0), pick(r1), pick(r2), pick(r3));
  };
  out0 = transpose(a0, b0, c0, d0);
  out1 = transpose(a1, b1, c1, d1);
}

// The 16 key-stream bytes chacha_quad gives this lane (words 4g..4g+3 of
// block `counter`, g = lane & 3), from the whole block computed by this lane
// alone: the four lanes of a quad compute the same block, four times
// chacha_quad's arithmetic, but no shuffle sits in the rounds' dependency
// chain, so the bytes come about twice as soon.  For the single-CTA fused
// batch, whose warps wait on them; the batched kernels, bound by
// throughput, keep chacha_quad.
__device__ __forceinline__ uint4 chacha_lane16(const uint32_t* key, uint32_t counter,
                                               uint32_t n0, uint32_t n1, uint32_t n2) {
  uint32_t x[16];
  chacha_block(key, counter, n0, n1, n2, x);
  const int g = threadIdx.x & 3;
  auto pick = [&](int k) {
    return g == 0 ? x[k] : g == 1 ? x[4 + k] : g == 2 ? x[8 + k] : x[12 + k];
  };
  return make_uint4(pick(0), pick(1), pick(2), pick(3));
}

// PRF(dom, x) = ChaCha20(K_prf, counter 0, nonce = dom || x)
__device__ __forceinline__ void prf(const MapDev& m, uint32_t dom, uint64_t x, uint32_t w[16]) {
  chacha_block(m.kprf, 0, dom, (uint32_t)x, (uint32_t)(x >> 32), w);
}

// ordered pair of distinct bins (the random remap of Sec. 3.2)
__device__ __forceinline__ void prf_pair(const MapDev& m, uint32_t dom, uint64_t x, uint32_t& b1,
                                         uint32_t& b2) {
  uint32_t w[16];
  prf(m, dom, x, w);
  uint64_t r0 = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
  uint64_t r1 = (uint64_t)w[2] | ((uint64_t)w[3] << 32);
  uint64_t f = mulhi64(r0, m.B);
  uint64_t s = mulhi64(r1, m.B - 1);
  s += (s >= f);
  b1 = (uint32_t)f;
  b2 = (uint32_t)s;
}

// d = 4 candidate position-map rows of a key (Sec. 4.2)
__device__ __forceinline__ void prf_rows(const MapDev& m, uint64_t key, uint32_t rows[4]) {
  uint32_t w[16];
  prf(m, DOM_PM, key, w);
#pragma unroll
  for (int j = 0; j < 4; j++)
    rows[j] = (uint32_t)mulhi64((uint64_t)w[2 * j] | ((uint64_t)w[2 * j + 1] << 32), m.rows);
}

// first choice with the fewest occupants, lowest index on ties
__device__ __forceinline__ uint32_t pick_row(const MapDev& m, const uint32_t rows[4]) {
  uint32_t best = rows[0], bc = byte_get(m.rowcnt, rows[0]);
#pragma unroll
  for (int j = 1; j < 4; j++) {
    uint32_t c = byte_get(m.rowcnt, rows[j]);
    if (c < bc) { best = rows[j]; bc = c; }
  }
  return best;
}

__device__ __forceinline__ void set_err(const MapDev& m, uint32_t bits) { atomicOr(m.err, bits); }

// Occupancy statistics (the quantities Claims 3.2-3.4 bound): live items in
// the HBM store and in the stash, and the largest values seen since the build.
// The stash and the HBM store only shrink before a batch's remap phase
// (find_remove, eviction) and only grow in it, so the running maximum taken
// at every increment of the remap phase is the maximum over end-of-batch
// values; a bin load only grows by a placement, so its running maximum at
// every increment is the peak load.
enum : int { ST_HBM = 0, ST_STASH = 1, ST_PEAK_HBM = 2, ST_PEAK_STASH = 3, ST_PEAK_LOAD = 4,
             ST_WORDS = 8 };

// A warp's placements of the remap phase: `placed` lanes put one item into
// the HBM store (hbm) or the stash, a bin reaching `new_load`.  All 32 lanes
// call; one lane per warp updates the counters.
// (peaks = false: only the counts move, by atomics nothing waits for; the
// store and stash peaks are then the counts a batch ends with, which
// stat_end_peaks records when the next batch starts)
__device__ __forceinline__ void stat_place(const MapDev& m, bool placed, bool hbm,
                                           uint32_t new_load, bool peaks = true) {
  const uint32_t hm = __ballot_sync(0xffffffffu, placed && hbm);
  const uint32_t sm = __ballot_sync(0xffffffffu, placed && !hbm);
  const uint32_t top = __reduce_max_sync(0xffffffffu, placed ? new_load : 0u);
  if ((threadIdx.x & 31) == 0) {
    if (hm) {
      const unsigned long long c = __popc(hm);
      if (peaks)
        atomicMax(m.stat + ST_PEAK_HBM, atomicAdd(m.stat + ST_HBM, c) + c);
      else
        atomicAdd(m.stat + ST_HBM, c);
    }
    if (sm) {
      const unsigned long long c = __popc(sm);
      if (peaks)
        atomicMax(m.stat + ST_PEAK_STASH, atomicAdd(m.stat + ST_STASH, c) + c);
      else
        atomicAdd(m.stat + ST_STASH, c);
    }
    if (top) atomicMax(m.stat + ST_PEAK_LOAD, (unsigned long long)top);
  }
}

// The counts the previous batch ended with, into the peaks: one thread of a
// batch calls it before the batch changes a count, and the host takes the
// current counts into the peaks it reads.  A batch whose placements took no
// peaks (stat_place with peaks = false) is covered so: its largest counts
// are the ones it ends with (see above).
__device__ __forceinline__ void stat_end_peaks(const MapDev& m) {
  const unsigned long long h = __ldcg(m.stat + ST_HBM), s = __ldcg(m.stat + ST_STASH);
  atomicMax(m.stat + ST_PEAK_HBM, h);
  atomicMax(m.stat + ST_PEAK_STASH, s);
}

// items leaving the HBM store (hbm) or the stash
__device__ __forceinline__ void stat_leave(const MapDev& m, bool hbm, unsigned long long count) {
  atomicAdd(m.stat + (hbm ? ST_HBM : ST_STASH), 0ull - count);
}

// Block-wide exclusive sum (blockDim.x a multiple of 32, <= 1024); `sh`
// holds 32 words of shared memory; `total` receives the block total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* sh, uint32_t& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sh[lane] = w;
  }
  __syncthreads();
  total = sh[(blockDim.x >> 5) - 1];
  uint32_t excl = x - v + (wid > 0 ? sh[wid - 1] : 0);
  __syncthreads();
  return excl;
}

// --- warp-level ordering of up to 32 (key, source) items ------------------
// ascending on (key, src): lanes without an item carry src NONE32 (and key
// ~0) and sort after every item, an item whose key is ~0 included; equal
// keys (only with duplicate keys) go in source order, so the result never
// depends on the order the items arrived in
__device__ __forceinline__ void warp_sort_by_key(uint64_t& key, uint32_t& src) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      uint64_t ok = __shfl_xor_sync(0xffffffffu, key, j);
      uint32_t os = __shfl_xor_sync(0xffffffffu, src, j);
      bool asc = (lane & k) == 0;
      bool lower = (lane & j) == 0;
      const bool o_less = ok < key || (ok == key && os < src);
      const bool o_greater = ok > key || (ok == key && os > src);
      bool take = lower == asc ? o_less : o_greater;
      if (take) {
        key = ok;
        src = os;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Poly1305 (RFC 8439 Sec. 2.5) over a sealed page, computed by a warp.
// Numbers mod p = 2^130 - 5 are held in five 26-bit limbs; a product is
// formed with 64-bit accumulators, the limbs past 2^130 folding back times 5.
// The page's message blocks are the 16-byte pieces a lane already holds when
// it encrypts or decrypts (block j = bytes [16j, 16j + 16) sits in lane
// j mod 32, chunk j / 32), then one block of lengths; the tag
//   sum_j m_j r^(K - j)  (+ s, mod 2^128),  K blocks,
// is split per lane: Horner over the lane's own blocks with r^32, times
// r^(K - last block of the lane), summed over the warp.
struct P130 {
  uint32_t l[5];
};

__device__ __forceinline__ P130 p130_norm(uint64_t d0, uint64_t d1, uint64_t d2, uint64_t d3,
                                          uint64_t d4) {
  const uint32_t M26 = (1u << 26) - 1;
  P130 h;
  uint64_t c;
  c = d0 >> 26; h.l[0] = (uint32_t)d0 & M26; d1 += c;
  c = d1 >> 26; h.l[1] = (uint32_t)d1 & M26; d2 += c;
  c = d2 >> 26; h.l[2] = (uint32_t)d2 & M26; d3 += c;
  c = d3 >> 26; h.l[3] = (uint32_t)d3 & M26; d4 += c;
  c = d4 >> 26; h.l[4] = (uint32_t)d4 & M26;
  uint64_t t = (uint64_t)h.l[0] + c * 5;
  h.l[0] = (uint32_t)t & M26;
  h.l[1] += (uint32_t)(t >> 26);
  return h;
}

// a * b mod p, limbs of both below 2^27
__device__ __forceinline__ P130 p130_mul(const P130& a, const P130& b) {
  const uint64_t b0 = b.l[0], b1 = b.l[1], b2 = b.l[2], b3 = b.l[3], b4 = b.l[4];
  const uint64_t s1 = b1 * 5, s2 = b2 * 5, s3 = b3 * 5, s4 = b4 * 5;
  const uint64_t a0 = a.l[0], a1 = a.l[1], a2 = a.l[2], a3 = a.l[3], a4 = a.l[4];
  return p130_norm(a0 * b0 + a1 * s4 + a2 * s3 + a3 * s2 + a4 * s1,
                   a0 * b1 + a1 * b0 + a2 * s4 + a3 * s3 + a4 * s2,
                   a0 * b2 + a1 * b1 + a2 * b0 + a3 * s4 + a4 * s3,
                   a0 * b3 + a1 * b2 + a2 * b1 + a3 * b0 + a4 * s4,
                   a0 * b4 + a1 * b3 + a2 * b2 + a3 * b1 + a4 * b0);
}

__device__ __forceinline__ P130 p130_add(const P130& a, const P130& b) {
  return p130_norm((uint64_t)a.l[0] + b.l[0], (uint64_t)a.l[1] + b.l[1],
                   (uint64_t)a.l[2] + b.l[2], (uint64_t)a.l[3] + b.l[3],
                   (uint64_t)a.l[4] + b.l[4]);
}

// a 16-byte message block with the 2^128 bit set
__device__ __forceinline__ P130 p130_block(uint4 w) {
  const uint32_t M26 = (1u << 26) - 1;
  P130 h;
  h.l[0] = w.x & M26;
  h.l[1] = ((w.x >> 26) | (w.y << 6)) & M26;
  h.l[2] = ((w.y >> 20) | (w.z << 12)) & M26;
  h.l[3] = ((w.z >> 14) | (w.w << 18)) & M26;
  h.l[4] = (w.w >> 8) | (1u << 24);
  return h;
}

__device__ __forceinline__ P130 p130_shfl(const P130& a, int src) {
  P130 r;
#pragma unroll
  for (int i = 0; i < 5; i++) r.l[i] = __shfl_sync(0xffffffffu, a.l[i], src);
  return r;
}

// The running state of a warp's Poly1305 over one page (see above).
struct PolyWarp {
  P130 acc;     // this lane's Horner sum
  P130 rpow;    // r^(lane + 1)
  P130 r32;     // r^32
  uint4 s;      // the key's second half
  int last;     // this lane's last block so far, -1 for none
};

// r and s from the one-time key: the first 32 bytes of the ChaCha20 block 0
// of (K_enc, page, version); all 32 lanes call
// (LAT: the block from chacha_lane16, for the latency-bound fused batch)
template <bool LAT = false>
__device__ __forceinline__ PolyWarp poly_begin(const MapDev& m, uint64_t q, uint64_t version) {
  const int lane = threadIdx.x & 31;
  const uint4 ks = (LAT ? chacha_lane16 : chacha_quad)(m.kenc, 0, (uint32_t)q, (uint32_t)version,
                               (uint32_t)(version >> 32));
  uint4 r, s;
  r.x = __shfl_sync(0xffffffffu, ks.x, 0); r.y = __shfl_sync(0xffffffffu, ks.y, 0);
  r.z = __shfl_sync(0xffffffffu, ks.z, 0); r.w = __shfl_sync(0xffffffffu, ks.w, 0);
  s.x = __shfl_sync(0xffffffffu, ks.x, 1); s.y = __shfl_sync(0xffffffffu, ks.y, 1);
  s.z = __shfl_sync(0xffffffffu, ks.z, 1); s.w = __shfl_sync(0xffffffffu, ks.w, 1);
  r.x &= 0x0fffffffu; r.y &= 0x0ffffffcu; r.z &= 0x0ffffffcu; r.w &= 0x0ffffffcu;
  P130 rr = p130_block(r);
  rr.l[4] &= (1u << 24) - 1;  // no 2^128 bit: r < 2^124
  // r^(lane + 1) by an inclusive product scan over the warp
  P130 x = rr;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const P130 y = p130_shfl(x, lane >= d ? lane - d : lane);
    if (lane >= d) x = p130_mul(x, y);
  }
  PolyWarp w;
  w.rpow = x;
  w.r32 = p130_shfl(x, 31);
  w.s = s;
  w.last = -1;
  for (int i = 0; i < 5; i++) w.acc.l[i] = 0;
  return w;
}

// block j of the message, held by lane j % 32 (the caller passes only its own)
// A warp's start state (after poly_begin) kept in shared memory: lane L's
// r^(L + 1) in words 5L..5L+4, then r^32 and s.  All 32 lanes call.
constexpr uint32_t POLY_WORDS = 32 * 5 + 5 + 4;
__device__ __forceinline__ void poly_store(const PolyWarp& w, uint32_t* sm) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < 5; i++) sm[5 * lane + i] = w.rpow.l[i];
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < 5; i++) sm[160 + i] = w.r32.l[i];
    sm[165] = w.s.x; sm[166] = w.s.y; sm[167] = w.s.z; sm[168] = w.s.w;
  }
}
__device__ __forceinline__ PolyWarp poly_load(const uint32_t* sm) {
  const int lane = threadIdx.x & 31;
  PolyWarp w;
#pragma unroll
  for (int i = 0; i < 5; i++) {
    w.rpow.l[i] = sm[5 * lane + i];
    w.r32.l[i] = sm[160 + i];
    w.acc.l[i] = 0;
  }
  w.s = make_uint4(sm[165], sm[166], sm[167], sm[168]);
  w.last = -1;
  return w;
}
__device__ __forceinline__ void poly_block(PolyWarp& w, int j, uint4 blk) {
  w.acc = w.last < 0 ? p130_block(blk) : p130_add(p130_mul(w.acc, w.r32), p130_block(blk));
  w.last = j;
}

// the tag after the K blocks (all lanes call); every lane gets it
__device__ __forceinline__ uint4 poly_finish(const PolyWarp& w, int K) {
  // this lane's part: acc * r^(K - last), r^e held by lane e - 1
  const int e = w.last < 0 ? 1 : K - w.last;
  const P130 re = p130_shfl(w.rpow, e - 1);
  P130 part = p130_mul(w.acc, re);
  if (w.last < 0)
    for (int i = 0; i < 5; i++) part.l[i] = 0;
  // the warp's sum: raw limb sums (32 limbs below 2^26 stay below 2^31),
  // then one normalisation
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const P130 o = p130_shfl(part, (threadIdx.x & 31) ^ d);
#pragma unroll
    for (int i = 0; i < 5; i++) part.l[i] += o.l[i];
  }
  part = p130_norm(part.l[0], part.l[1], part.l[2], part.l[3], part.l[4]);
  // the sum as an exact integer in 32-bit words (limbs below 2^27: value
  // below 2^131), bits from 2^130 up folded back times 5, then p subtracted
  // once if still reached (the value is then below 2^130 + 5)
  uint64_t acc = (uint64_t)part.l[0] + ((uint64_t)part.l[1] << 26);
  uint32_t v0 = (uint32_t)acc; acc >>= 32;
  acc += (uint64_t)part.l[2] << 20;
  uint32_t v1 = (uint32_t)acc; acc >>= 32;
  acc += (uint64_t)part.l[3] << 14;
  uint32_t v2 = (uint32_t)acc; acc >>= 32;
  acc += (uint64_t)part.l[4] << 8;
  uint32_t v3 = (uint32_t)acc; acc >>= 32;
  uint32_t v4 = (uint32_t)acc;
  {
    uint64_t t = (uint64_t)v0 + 5ull * (v4 >> 2);
    v4 &= 3;
    v0 = (uint32_t)t; t >>= 32;
    t += v1; v1 = (uint32_t)t; t >>= 32;
    t += v2; v2 = (uint32_t)t; t >>= 32;
    t += v3; v3 = (uint32_t)t; t >>= 32;
    v4 += (uint32_t)t;
  }
  {
    // v >= p iff v + 5 reaches 2^130; then v - p = (v + 5) mod 2^130
    uint64_t t = (uint64_t)v0 + 5;
    const uint32_t u0 = (uint32_t)t; t >>= 32;
    t += v1; const uint32_t u1 = (uint32_t)t; t >>= 32;
    t += v2; const uint32_t u2 = (uint32_t)t; t >>= 32;
    t += v3; const uint32_t u3 = (uint32_t)t; t >>= 32;
    const uint32_t u4 = v4 + (uint32_t)t;
    if (u4 >> 2) {
      v0 = u0; v1 = u1; v2 = u2; v3 = u3;
    }
  }
  // tag = (v + s) mod 2^128
  uint64_t t = (uint64_t)v0 + w.s.x;
  const uint32_t f0 = (uint32_t)t; t >>= 32;
  t += (uint64_t)v1 + w.s.y;
  const uint32_t f1 = (uint32_t)t; t >>= 32;
  t += (uint64_t)v2 + w.s.z;
  const uint32_t f2 = (uint32_t)t; t >>= 32;
  t += (uint64_t)v3 + w.s.w;
  return make_uint4(f0, f1, f2, (uint32_t)t);
}

// the lengths block of a sealed page: no additional data, L bytes of ciphertext
__device__ __forceinline__ uint4 poly_lengths(uint32_t L) { return make_uint4(0, 0, L, 0); }

// Encrypt a plaintext page (shared memory) into dst (page_bytes): lane L
// handles bytes [16L, 16L+16) of each 512-byte chunk; the four lanes of a
// quad compute the chunk's ChaCha20 block together.  Sealed pages (integrity
// on) are the ChaCha20-Poly1305 AEAD of RFC 8439 Sec. 2.8: the first
// page_bytes - 16 bytes encrypted from block 1, the tag over them and their
// length in the last 16 bytes.  SEALED = m.integrity (kernels are compiled
// for both, so the sealing's registers do not weigh on plain pages).  With
// ks_pre the page's key stream (the same bytes, offset by offset) was
// computed ahead into shared memory and is only XORed here; with poly_pre
// (sealed) the tag's start state was too (poly_store).
template <bool SEALED, bool LAT = false>
__device__ __forceinline__ void page_encrypt_to(const MapDev& m, const uint8_t* plain,
                                                uint8_t* dst, uint64_t q, uint64_t version,
                                                const uint8_t* ks_pre = nullptr,
                                                const uint32_t* poly_pre = nullptr) {
  const int lane = threadIdx.x & 31;
  constexpr uint32_t sealed = SEALED ? 1u : 0u;
  const uint32_t L = m.page_bytes - 16 * sealed;
  PolyWarp pw;
  if (SEALED) pw = poly_pre ? poly_load(poly_pre) : poly_begin<LAT>(m, q, version);
  for (uint32_t c = 0; c < m.page_bytes; c += 512) {
    uint32_t off = c + 16 * lane;
    uint4 ks;
    if (ks_pre)
      ks = off < L ? *reinterpret_cast<const uint4*>(ks_pre + off) : make_uint4(0, 0, 0, 0);
    else
      ks = (LAT ? chacha_lane16 : chacha_quad)(m.kenc, c / 64 + (lane >> 2) + sealed, (uint32_t)q,
                                               (uint32_t)version,
                       (uint32_t)(version >> 32));
    uint4 blk = SEALED ? poly_lengths(L) : make_uint4(0, 0, 0, 0);
    if (off < L) {
      uint4 p = *reinterpret_cast<const uint4*>(plain + off);
      p.x ^= ks.x; p.y ^= ks.y; p.z ^= ks.z; p.w ^= ks.w;
      *reinterpret_cast<uint4*>(dst + off) = p;
      blk = p;
    }
    // (the ciphertext's blocks and, at L, the lengths block: one call)
    if (SEALED && off <= L) poly_block(pw, off / 16, blk);
  }
  if (SEALED) {
    const uint4 tag = poly_finish(pw, L / 16 + 1);
    if (lane == (int)((L / 16) & 31)) *reinterpret_cast<uint4*>(dst + L) = tag;
  }
}

// ---------------------------------------------------------------------------
// Profiling: per-kernel-class durations from CUDA events recorded on the
// launching stream, and a count of every kernel launch.  The runtime points
// g_prof at the handle's profiler for the duration of an ABI call.
enum ProfClass : int {
  P_SORT_GLOBAL = 0,  // bitonic steps with stride >= tile (HBM passes)
  P_SORT_TILE = 1,    // bitonic in-tile steps (shared memory)
  P_PAGE_BUILD = 2,   // build: page gather + encrypt + host store
  P_P2C = 3,          // build: all P2C / position-map rounds
  P_KEYCHECK = 4,     // build: key-uniqueness check
  P_ACCESS = 5,       // one whole access batch
  P_GATHER = 6,       // access: position-map search + page reads + decrypt
  P_EVICT = 7,        // access: write-back with eviction
  P_BUILD = 8,        // one whole build
  P_GROUP = 9,        // access: batch grouping sort + scans
  P_KSORT_GLOBAL = 10,  // key-uniqueness check: bitonic global steps
  P_KSORT_TILE = 11,    // key-uniqueness check: bitonic in-tile steps
  P_FLUSH = 12,         // access: written pages copied to the host
  P_AHEAD = 13,         // access: lookahead search + page reads (side stream)
  P_PAGE_GROUP = 14,    // build: host records grouped by page (two bucket passes)
  P_PAGES = 15,         // access: distinct pages, trace
  P_FINDEXEC = 16,      // access: find_remove + Get/Put/Delete semantics
  P_REMAP = 17,         // access: P2C remap
  P_STAGE = 18,         // access: PRF pairs, rows, grouping keys
  P_NCLASS = 19
};

struct Prof {
  bool on = false;
  uint64_t launches = 0;
  struct Span { int cls; cudaEvent_t a, b; };
  std::vector<Span> pending;
  double ms[P_NCLASS] = {};
  uint64_t count[P_NCLASS] = {};
};
extern thread_local Prof* g_prof;

// Raise a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device.  The limit is a per-kernel attribute shared by every host
// thread, so it is only ever raised (under a lock): a launch of the same
// kernel for another map, enqueued by another thread, never finds its size
// above a limit that was lowered meanwhile.
cudaError_t raise_smem_limit(const void* kernel, size_t bytes);

inline void count_launch(uint64_t n = 1) {
  if (g_prof) g_prof->launches += n;
}

struct ProfSpan {
  int cls;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  ProfSpan(int c, cudaStream_t s) : cls(c), st(s) {
    if (g_prof && g_prof->on && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, st);
  }
  ~ProfSpan() {
    if (!a) return;
    cudaEvent_t b = nullptr;
    if (cudaEventCreate(&b) == cudaSuccess) {
      cudaEventRecord(b, st);
      g_prof->pending.push_back({cls, a, b});
    } else {
      cudaEventDestroy(a);
    }
  }
};

// ---------------------------------------------------------------------------
// host-side launchers (defined in the .cu files)

// build.cu
cudaError_t launch_build(const MapDev& m, const uint64_t* keys, const uint8_t* vals, uint64_t n,
                         struct BuildScratch& s, cudaStream_t st,
                         cudaEvent_t vals_wait,  // the values are on the device (or null);
                                                 // `side` is already ordered after them
                         cudaStream_t side, cudaEvent_t side_fork, cudaEvent_t side_join,
                         // pages built in HBM chunks and copied to the host on
                         // copy_st (null: straight to the host); two events each
                         cudaStream_t copy_st, cudaEvent_t* ev_built, cudaEvent_t* ev_copied);

// build.cu, the data owner's image (Sec. 4.2 "Fast data initialization"):
// export the placement the last build (still in `s`) made as a bin-major
// image; load an image into the map (loads, position map, HBM residents,
// pages, free ring)
cudaError_t launch_image_export(const MapDev& m, const uint64_t* keys, const uint8_t* vals,
                                uint64_t n, struct BuildScratch& s, cudaStream_t st,
                                uint64_t* img_keys, uint8_t* img_vals, uint64_t* img_pairs,
                                uint32_t* img_rows, uint8_t* img_counts);
cudaError_t launch_image_load(const MapDev& m, const uint64_t* keys, const uint8_t* vals,
                              const uint64_t* pairs, const uint32_t* rows, const uint8_t* counts,
                              uint64_t n, struct BuildScratch& s, cudaStream_t st,
                              cudaStream_t side, cudaEvent_t side_fork, cudaEvent_t side_join,
                              cudaStream_t copy_st, cudaEvent_t* ev_built, cudaEvent_t* ev_copied);

// sort.cu: ascending bitonic sort of n_pow2 uint64 tags in place; the
// passes are profiled under the given classes
cudaError_t sort_tags_u64(uint64_t* tags, uint64_t n_pow2, int log_tile, cudaStream_t st,
                          int cls_global = P_SORT_GLOBAL, int cls_tile = P_SORT_TILE);

struct BuildScratch {
  uint64_t cap = 0;        // records the buffers hold
  uint64_t tag_cap = 0;    // tag buffer elements (power of two)
  int prf_rounds = 0;      // BOLT_PARAM_ROUNDS_PRF: 0 automatic, 1 the PRF inside
                           // the P2C rounds where the grid allows, 2 a PRF pass
  uint64_t* tags = nullptr;
  uint64_t* bins = nullptr;   // per record b1 | b2 << 32
  uint32_t* dest = nullptr;   // per record destination bin
  uint32_t* prow = nullptr;   // per record chosen position-map row
  uint4* rows4 = nullptr;     // per record position-map candidate rows, then (after
                              // the rounds) the two staging halves of the page build
                              // (optional: without it the rounds compute the rows
                              // inline and pages are stored straight to the host)
  uint64_t* keysort = nullptr;  // [2 tag_cap] the key-uniqueness hash table (optional:
                                // without it the check sorts a copy of the keys in
                                // `tags`, in line)
  uint32_t* page_off = nullptr;  // [M + 1] exclusive prefix of page loads
  uint32_t* block_sums = nullptr;
  uint64_t block_cap = 0;
  int log_tile = 13;          // bitonic tile (2^log_tile elements), chosen by the autotuner
  unsigned long long* counters = nullptr;  // [0] value-store fill
};

}  // namespace bdev
