// build.cu -- the oblivious build (Sec. 4.2 "Fast data initialization",
// performed on the device instead of by the data owner).
//
// Steps (all on the launching stream):
//   1. rounds of W_r records: record i draws the pair PRF(INIT, i) and its
//      d = 4 position-map rows PRF(PM, key); it picks the less-loaded bin
//      (P2C, first choice on ties) and the least-occupied row (lowest index on
//      ties) against the counts at the start of the round (decide kernel);
//      then the counts are bumped with atomics, the position-map entry is
//      written and HBM-bin records take a value-store slot (apply kernel);
//   2. exclusive prefix sum of the host-page loads -> each page's run start;
//   3. tag = (page << 32 | record) for host-bin records, all-ones otherwise;
//      the tags are sorted by the bitonic network (sort.cu), which groups the
//      records page by page;
//   4. one warp per page gathers its run, orders it by key, pads it with zero
//      dummy slots to lmax, encrypts it (ChaCha20, nonce = page || version 0)
//      and writes it to the pinned host page with 16-byte coalesced stores;
//   5. the free-slot ring receives every value-store slot not taken in 1.
#include "bolt_internal.cuh"

namespace bdev {

// every record's pair PRF(INIT, i) and candidate rows PRF(PM, key), computed
// once at full occupancy so the rounds only touch counters
__global__ void k_build_prf(MapDev m, const uint64_t* __restrict__ keys, uint64_t n,
                            uint64_t* __restrict__ bins, uint4* __restrict__ rows4) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t b1, b2;
    prf_pair(m, DOM_INIT, i, b1, b2);
    bins[i] = (uint64_t)b1 | ((uint64_t)b2 << 32);
    uint32_t rows[4];
    prf_rows(m, keys[i], rows);
    rows4[i] = make_uint4(rows[0], rows[1], rows[2], rows[3]);
  }
}

// decide on round-start counts: P2C bin (first choice on ties) and d-choice
// row (lowest index on ties)
__global__ void k_build_decide(MapDev m, const uint64_t* __restrict__ keys, uint64_t lo,
                               uint64_t hi, uint64_t* __restrict__ bins,
                               const uint4* __restrict__ rows4, uint32_t* __restrict__ dest,
                               uint32_t* __restrict__ prow) {
  uint64_t i = lo + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= hi) return;
  uint32_t b1, b2, rows[4];
  if (rows4) {
    const uint64_t bb = bins[i];
    b1 = (uint32_t)bb;
    b2 = (uint32_t)(bb >> 32);
    const uint4 r4 = rows4[i];
    rows[0] = r4.x; rows[1] = r4.y; rows[2] = r4.z; rows[3] = r4.w;
  } else {
    prf_pair(m, DOM_INIT, i, b1, b2);
    bins[i] = (uint64_t)b1 | ((uint64_t)b2 << 32);
    prf_rows(m, keys[i], rows);
  }
  const uint32_t l1 = byte_get(m.load, b1), l2 = byte_get(m.load, b2);
  dest[i] = l1 <= l2 ? b1 : b2;
  prow[i] = pick_row(m, rows);
}

// bump the counts of record i's choices, write its position-map entry, give
// an HBM-bin record a value-store slot
__device__ __forceinline__ void build_apply_one(const MapDev& m, const uint64_t* __restrict__ keys,
                                                const uint8_t* __restrict__ vals, uint64_t i,
                                                const uint64_t* __restrict__ bins, uint32_t d,
                                                uint32_t row, unsigned long long* vs_fill) {
  if (byte_inc(m.load, d) + 1 > m.lmax) {
    set_err(m, ERR_LOAD);
    return;
  }
  const uint32_t slot = byte_inc(m.rowcnt, row);
  if (slot >= m.R) {
    set_err(m, ERR_ROW);
    return;
  }
  const uint64_t pmi = (uint64_t)row * m.R + slot;
  const uint64_t bb = bins[i];
  const uint32_t which = d == (uint32_t)(bb >> 32) ? 1u : 0u;
  uint32_t meta = meta_make(LOC_HOST, which, 0);
  if (d < m.K) {
    unsigned long long vs = atomicAdd(vs_fill, 1ull);
    if (vs >= m.vs_cap) {
      set_err(m, ERR_VS);
      return;
    }
    m.vs_key[vs] = keys[i];
    const uint64_t* src = reinterpret_cast<const uint64_t*>(vals + i * m.vb);
    uint64_t* dst = reinterpret_cast<uint64_t*>(m.vs_val + vs * m.vb);
    for (uint32_t w = 0; w < m.vb / 8; w++) dst[w] = src[w];
    m.vs_pm[vs] = (uint32_t)pmi;
    m.vs_live[vs] = 1;
    meta = meta_make(LOC_HBM, which, (uint32_t)vs);
  }
  m.pm_key[pmi] = keys[i];
  m.pm_bins[pmi] = bb;
  m.pm_meta[pmi] = meta;
}

__global__ void k_build_apply(MapDev m, const uint64_t* __restrict__ keys,
                              const uint8_t* __restrict__ vals, uint64_t lo, uint64_t hi,
                              const uint64_t* __restrict__ bins, const uint32_t* __restrict__ dest,
                              const uint32_t* __restrict__ prow, unsigned long long* vs_fill) {
  uint64_t i = lo + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= hi) return;
  build_apply_one(m, keys, vals, i, bins, dest[i], prow[i], vs_fill);
}

// --- all rounds in one persistent kernel ------------------------------------
// A software grid barrier separates the decide and apply phases of every
// round.  All blocks are co-resident (cooperative launch).  Every wait is
// bounded (m.spin_limit iterations of a ~256 ns sleep; the default 2^22 is
// about one second): a block that gives up sets ERR_TIMEOUT and leaves the
// kernel, so the others give up at their next barrier too and the kernel
// always ends.  The steps after the rounds then skip their work (they would
// read a half-decided placement), and the build returns BOLT_E_TIMEOUT.

// a record's claimed position-map row and slot packed in one word (rows <
// 2^27 for N <= 2^31, slots < R <= 32); NONE32 marks a record that overflowed
constexpr uint32_t PROW_SLOT_SHIFT = 27;
constexpr uint32_t PROW_ROW_MASK = (1u << PROW_SLOT_SHIFT) - 1;

__device__ __forceinline__ bool grid_barrier(const MapDev& m, unsigned int* bar) {
  // bar[0]: arrivals, bar[1]: generation
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = bar + 1;
    const unsigned int g = *gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(bar, 1u);
    ok = 1;
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      uint32_t it = 0;
      while (*gen == g) {
        if (++it > m.spin_limit) {
          ok = 0;
          set_err(m, ERR_TIMEOUT);
          break;
        }
        __nanosleep(256);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// round-start counts must come from L2, not from a line this SM cached in an
// earlier round of the same kernel
__device__ __forceinline__ uint32_t byte_get_l2(const uint32_t* w, uint64_t i) {
  return (__ldcg(w + (i >> 2)) >> ((uint32_t)(i & 3) * 8)) & 0xffu;
}

__global__ void __launch_bounds__(256) k_build_rounds(MapDev m, const uint64_t* __restrict__ keys,
                                                      const uint8_t* __restrict__ vals, uint64_t n,
                                                      const uint64_t* __restrict__ bins,
                                                      const uint4* __restrict__ rows4,
                                                      uint32_t* __restrict__ dest,
                                                      uint32_t* __restrict__ prow,
                                                      unsigned long long* vs_fill,
                                                      unsigned int* bar) {
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (uint64_t lo = 0; lo < n; lo += m.Wr) {
    const uint64_t hi = lo + m.Wr < n ? lo + m.Wr : n;
    for (uint64_t i = lo + tid; i < hi; i += nthreads) {
      const uint64_t bb = bins[i];
      const uint32_t b1 = (uint32_t)bb, b2 = (uint32_t)(bb >> 32);
      const uint32_t l1 = byte_get_l2(m.load, b1), l2 = byte_get_l2(m.load, b2);
      dest[i] = l1 <= l2 ? b1 : b2;
      const uint4 r4 = rows4[i];
      const uint32_t rows[4] = {r4.x, r4.y, r4.z, r4.w};
      uint32_t best = rows[0], bc = byte_get_l2(m.rowcnt, rows[0]);
#pragma unroll
      for (int j = 1; j < 4; j++) {
        const uint32_t c = byte_get_l2(m.rowcnt, rows[j]);
        if (c < bc) {
          best = rows[j];
          bc = c;
        }
      }
      prow[i] = best;
    }
    if (!grid_barrier(m, bar)) return;
    // only the order-dependent part happens between the barriers: the
    // counts; the entry is written later by k_build_place
    for (uint64_t i = lo + tid; i < hi; i += nthreads) {
      const uint32_t row = prow[i];
      uint32_t tag = NONE32;
      if (byte_inc(m.load, dest[i]) + 1 > m.lmax) {
        set_err(m, ERR_LOAD);
      } else {
        const uint32_t slot = byte_inc(m.rowcnt, row);
        if (slot >= m.R) set_err(m, ERR_ROW);
        else tag = row | (slot << PROW_SLOT_SHIFT);
      }
      prow[i] = tag;
    }
    if (!grid_barrier(m, bar)) return;
  }
}

// The same barrier in two halves, so a block can work between its arrival
// and its wait: grid_arrive after the block's writes of the phase (returns
// the generation to wait on), grid_wait before reading what the other blocks
// wrote.  The wait is bounded like grid_barrier's.
__device__ __forceinline__ unsigned int grid_arrive(unsigned int* bar) {
  __shared__ unsigned int s_gen;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = bar + 1;
    const unsigned int g = *gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    }
    s_gen = g;
  }
  __syncthreads();
  return s_gen;
}
__device__ __forceinline__ bool grid_wait(const MapDev& m, unsigned int* bar, unsigned int g) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = bar + 1;
    ok = 1;
    uint32_t it = 0;
    while (*gen == g) {
      if (++it > m.spin_limit) {
        ok = 0;
        set_err(m, ERR_TIMEOUT);
        break;
      }
      __nanosleep(256);
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// The rounds with each record's PRF computed inside them, for grids of at
// least W_r / ROUNDS_KPT threads (each thread owns at most ROUNDS_KPT records
// of a round, records lo + tid + k * nthreads): while a block waits at the
// decide barrier it computes its records' pairs PRF(INIT, i) for the next
// round, and while it waits at the apply barrier their rows PRF(PM, key), so
// the PRF costs no pass of its own.  Pairs still go to `bins` (the placement
// reads them); decisions, counts and claims are those of k_build_rounds.
constexpr uint32_t ROUNDS_KPT = 4;

__global__ void __launch_bounds__(256) k_build_rounds_prf(MapDev m,
                                                          const uint64_t* __restrict__ keys,
                                                          uint64_t n, uint64_t* __restrict__ bins,
                                                          uint32_t* __restrict__ dest,
                                                          uint32_t* __restrict__ prow,
                                                          unsigned int* bar) {
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t pr[ROUNDS_KPT];
  uint32_t rw[ROUNDS_KPT][4], dst[ROUNDS_KPT], row[ROUNDS_KPT];
  auto pairs = [&](uint64_t lo) {
    const uint64_t hi = lo + m.Wr < n ? lo + m.Wr : n;
#pragma unroll
    for (uint32_t k = 0; k < ROUNDS_KPT; k++) {
      const uint64_t i = lo + tid + k * nthreads;
      if (i < hi) {
        uint32_t b1, b2;
        prf_pair(m, DOM_INIT, i, b1, b2);
        pr[k] = (uint64_t)b1 | ((uint64_t)b2 << 32);
        bins[i] = pr[k];
      }
    }
  };
  auto rows = [&](uint64_t lo) {
    const uint64_t hi = lo + m.Wr < n ? lo + m.Wr : n;
#pragma unroll
    for (uint32_t k = 0; k < ROUNDS_KPT; k++) {
      const uint64_t i = lo + tid + k * nthreads;
      if (i < hi) prf_rows(m, keys[i], rw[k]);
    }
  };
  if (n == 0) return;
  pairs(0);
  rows(0);
  for (uint64_t lo = 0; lo < n; lo += m.Wr) {
    const uint64_t hi = lo + m.Wr < n ? lo + m.Wr : n;
    // decide on round-start counts (read from L2)
#pragma unroll
    for (uint32_t k = 0; k < ROUNDS_KPT; k++) {
      const uint64_t i = lo + tid + k * nthreads;
      if (i >= hi) continue;
      const uint32_t b1 = (uint32_t)pr[k], b2 = (uint32_t)(pr[k] >> 32);
      const uint32_t l1 = byte_get_l2(m.load, b1), l2 = byte_get_l2(m.load, b2);
      dst[k] = l1 <= l2 ? b1 : b2;
      dest[i] = dst[k];
      uint32_t best = rw[k][0], bc = byte_get_l2(m.rowcnt, rw[k][0]);
#pragma unroll
      for (int j = 1; j < 4; j++) {
        const uint32_t c = byte_get_l2(m.rowcnt, rw[k][j]);
        if (c < bc) {
          best = rw[k][j];
          bc = c;
        }
      }
      row[k] = best;
    }
    const uint64_t next = lo + m.Wr;
    unsigned int g = grid_arrive(bar);
    if (next < n) pairs(next);
    if (!grid_wait(m, bar, g)) return;
    // the counts, in round order: the order-dependent part
#pragma unroll
    for (uint32_t k = 0; k < ROUNDS_KPT; k++) {
      const uint64_t i = lo + tid + k * nthreads;
      if (i >= hi) continue;
      uint32_t tag = NONE32;
      if (byte_inc(m.load, dst[k]) + 1 > m.lmax) {
        set_err(m, ERR_LOAD);
      } else {
        const uint32_t slot = byte_inc(m.rowcnt, row[k]);
        if (slot >= m.R) set_err(m, ERR_ROW);
        else tag = row[k] | (slot << PROW_SLOT_SHIFT);
      }
      prow[i] = tag;
    }
    g = grid_arrive(bar);
    if (next < n) rows(next);
    if (!grid_wait(m, bar, g)) return;
  }
}

// write every record's position-map entry (row and slot claimed in the
// rounds) and give HBM-bin records a value-store slot.  The slots come from
// one counter, taken once per warp for all its HBM-bin records (which slot a
// record gets is never observable: the value store lives in HBM).
__global__ void k_build_place(MapDev m, const uint64_t* __restrict__ keys,
                              const uint8_t* __restrict__ vals, uint64_t n,
                              const uint64_t* __restrict__ bins, const uint32_t* __restrict__ dest,
                              const uint32_t* __restrict__ prow, unsigned long long* vs_fill) {
  const int lane = threadIdx.x & 31;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  // rounds that gave up at a barrier leave rows and slots unclaimed (and the
  // claim words of later rounds unwritten): nothing is placed then
  if (*(volatile uint32_t*)m.err & ERR_TIMEOUT) return;
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n;
       base += stride) {
    const uint64_t i = base + lane;
    uint32_t tag = NONE32, d = 0;
    if (i < n) {
      tag = prow[i];
      d = dest[i];
    }
    const bool hbm = tag != NONE32 && d < m.K;
    const uint32_t hmask = __ballot_sync(0xffffffffu, hbm);
    unsigned long long vbase = 0;
    if (lane == 0 && hmask) vbase = atomicAdd(vs_fill, (unsigned long long)__popc(hmask));
    vbase = __shfl_sync(0xffffffffu, vbase, 0);
    if (tag == NONE32) continue;
    if ((tag & PROW_ROW_MASK) >= m.rows || (tag >> PROW_SLOT_SHIFT) >= m.R) {
      set_err(m, ERR_ROW);  // not a claim the rounds wrote
      continue;
    }
    const uint64_t pmi = (uint64_t)(tag & PROW_ROW_MASK) * m.R + (tag >> PROW_SLOT_SHIFT);
    const uint64_t bb = bins[i];
    const uint32_t which = d == (uint32_t)(bb >> 32) ? 1u : 0u;
    uint32_t meta = meta_make(LOC_HOST, which, 0);
    const uint64_t key = keys[i];
    if (hbm) {
      const unsigned long long vs = vbase + __popc(hmask & ((1u << lane) - 1u));
      if (vs >= m.vs_cap) {
        set_err(m, ERR_VS);
        continue;
      }
      m.vs_key[vs] = key;
      const uint64_t* src = reinterpret_cast<const uint64_t*>(vals + i * m.vb);
      uint64_t* dst = reinterpret_cast<uint64_t*>(m.vs_val + vs * m.vb);
      for (uint32_t w = 0; w < m.vb / 8; w++) dst[w] = src[w];
      m.vs_pm[vs] = (uint32_t)pmi;
      m.vs_live[vs] = 1;
      meta = meta_make(LOC_HBM, which, (uint32_t)vs);
    }
    m.pm_key[pmi] = key;
    m.pm_bins[pmi] = bb;
    m.pm_meta[pmi] = meta;
  }
}

// tags: host-bin records -> (page << 32 | i); HBM-bin records and padding -> ~0
__global__ void k_build_tags(MapDev m, const uint32_t* __restrict__ dest, uint64_t n,
                             uint64_t n_pow2, uint64_t* __restrict__ tags) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pow2;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t t = ~0ull;
    if (i < n) {
      uint32_t d = dest[i];
      if (d >= m.K) t = ((uint64_t)(d - m.K) << 32) | i;
    }
    tags[i] = t;
  }
}

// Host-bin records grouped by page without a sort, in two passes.  Page q's
// run starts at page_off[q] (the prefix of the page loads the rounds left),
// so a bucket of GROUP_PAGES consecutive pages owns one contiguous run too.
//   k_group_buckets: each record takes the next position of its bucket's run
//     from the bucket's cursor (one counter per bucket: they stay in L2, and
//     each bucket's writes advance sequentially, so L2 merges them into full
//     lines) and writes its tag (page << 32 | record) there;
//   k_group_pages: a CTA per bucket moves each tag of the bucket's run to the
//     next position of its page's run (cursors in shared memory; all writes
//     within the bucket's run).
// The order inside a page's run is the atomics' order; the page build orders
// every run by (key, record), so no page depends on it.  A record whose bin is
// out of range (rounds that gave up leave `dest` unwritten) or whose run is
// already full (loads and destinations disagree) is not written and raises
// ERR_PAGE.
constexpr uint32_t GROUP_PAGE_BITS = 9;
constexpr uint32_t GROUP_PAGES = 1u << GROUP_PAGE_BITS;

// bucket b's cursor and run end: page_off[b * GROUP_PAGES], page_off[min(..., M)]
__global__ void k_group_init(MapDev m, const uint32_t* __restrict__ page_off, uint32_t nb,
                             uint32_t* __restrict__ bcur, uint32_t* __restrict__ bend) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
    const uint64_t q0 = (uint64_t)b << GROUP_PAGE_BITS, q1 = q0 + GROUP_PAGES;
    bcur[b] = page_off[q0];
    bend[b] = page_off[q1 < m.M ? q1 : m.M];
  }
}

__global__ void __launch_bounds__(256) k_group_buckets(MapDev m, const uint32_t* __restrict__ dest,
                                                       uint64_t n, uint32_t* __restrict__ bcur,
                                                       const uint32_t* __restrict__ bend,
                                                       uint64_t* __restrict__ tmp) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t d = dest[i];
    if (d < m.K) continue;  // an HBM bin: no page
    if (d >= m.B) {
      set_err(m, ERR_PAGE);
      continue;
    }
    const uint32_t q = d - (uint32_t)m.K, b = q >> GROUP_PAGE_BITS;
    const uint32_t pos = atomicAdd(bcur + b, 1u);
    if (pos >= bend[b]) {
      set_err(m, ERR_PAGE);
      continue;
    }
    tmp[pos] = ((uint64_t)q << 32) | i;
  }
}

__global__ void __launch_bounds__(256) k_group_pages(MapDev m, const uint32_t* __restrict__ page_off,
                                                     uint32_t nb, const uint64_t* __restrict__ tmp,
                                                     uint64_t* __restrict__ tags) {
  __shared__ uint32_t cur[GROUP_PAGES], end[GROUP_PAGES];
  for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
    const uint64_t q0 = (uint64_t)b << GROUP_PAGE_BITS;
    const uint64_t q1 = q0 + GROUP_PAGES < m.M ? q0 + GROUP_PAGES : m.M;
    for (uint64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
      cur[q - q0] = page_off[q];
      end[q - q0] = page_off[q + 1];
    }
    __syncthreads();
    const uint32_t lo = page_off[q0], hi = page_off[q1];
    for (uint32_t k = lo + threadIdx.x; k < hi; k += blockDim.x) {
      const uint64_t t = tmp[k];
      const uint64_t q = t >> 32;
      if (q < q0 || q >= q1) {  // a slot pass one left unwritten
        set_err(m, ERR_PAGE);
        continue;
      }
      const uint32_t pos = atomicAdd(&cur[q - q0], 1u);
      if (pos >= end[q - q0]) {
        set_err(m, ERR_PAGE);
        continue;
      }
      tags[pos] = t;
    }
    __syncthreads();
  }
}

// --- exclusive prefix sum of the M page loads (u8) -> u32 run starts ------
constexpr int SCAN_BLOCK = 1024;
constexpr int SCAN_ITEMS = 8;  // 8192 pages per block

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_sums(MapDev m, uint32_t* block_sums) {
  __shared__ uint32_t sh[32];
  const uint64_t base = (uint64_t)blockIdx.x * SCAN_BLOCK * SCAN_ITEMS;
  uint32_t s = 0;
  for (int k = 0; k < SCAN_ITEMS; k++) {
    uint64_t q = base + (uint64_t)threadIdx.x * SCAN_ITEMS + k;
    if (q < m.M) s += byte_get(m.load, m.K + q);
  }
  uint32_t total;
  block_excl_scan(s, sh, total);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// single CTA: exclusive scan of the block sums in place
__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_top(uint32_t* block_sums, uint32_t nb) {
  __shared__ uint32_t sh[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t lo = 0; lo < nb; lo += SCAN_BLOCK) {
    uint32_t i = lo + threadIdx.x;
    uint32_t v = i < nb ? block_sums[i] : 0;
    uint32_t total;
    uint32_t e = block_excl_scan(v, sh, total);
    if (i < nb) block_sums[i] = carry + e;
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_fill(MapDev m, const uint32_t* block_sums,
                                                          uint32_t* page_off) {
  __shared__ uint32_t sh[32];
  const uint64_t base = (uint64_t)blockIdx.x * SCAN_BLOCK * SCAN_ITEMS;
  uint32_t v[SCAN_ITEMS], s = 0;
  for (int k = 0; k < SCAN_ITEMS; k++) {
    uint64_t q = base + (uint64_t)threadIdx.x * SCAN_ITEMS + k;
    v[k] = q < m.M ? byte_get(m.load, m.K + q) : 0;
    s += v[k];
  }
  uint32_t total;
  uint32_t e = block_excl_scan(s, sh, total) + block_sums[blockIdx.x];
  for (int k = 0; k < SCAN_ITEMS; k++) {
    uint64_t q = base + (uint64_t)threadIdx.x * SCAN_ITEMS + k;
    if (q <= m.M) page_off[q] = e;  // page_off[M] = total host records
    e += v[k];
  }
}

// One warp per host page: gather its run of sorted tags, order by key, pad
// with zero dummies, encrypt under version 0, store.
// Pages [q0, q1); each ciphertext goes to out + (q - q0) * page_bytes in HBM
// when `out` is given (the copy engine moves the chunk to the host), else
// straight to the host page.
// Without tags (a data owner's image, records already in bin-major order)
// page q's run is records run_base[0] + page_off[q] ... of keys / vals, the
// first n_rec of them being valid.  SEALED = m.integrity.
template <bool SEALED>
__global__ void k_page_build(MapDev m, const uint64_t* __restrict__ keys,
                             const uint8_t* __restrict__ vals, const uint64_t* __restrict__ tags,
                             const uint32_t* __restrict__ page_off, uint32_t warps_per_block,
                             uint64_t q0, uint64_t q1, uint8_t* out,
                             const unsigned long long* run_base, uint64_t n_rec) {
  extern __shared__ __align__(16) uint8_t sbuf[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint8_t* plain = sbuf + (size_t)wid * m.page_bytes;
  const uint64_t stride = (uint64_t)gridDim.x * warps_per_block;
  for (uint64_t q = q0 + (uint64_t)blockIdx.x * warps_per_block + wid; q < q1; q += stride) {
    const uint32_t cnt = byte_get(m.load, m.K + q);
    const uint32_t off = page_off[q];
    uint64_t key = ~0ull;
    uint32_t src = NONE32;
    if (lane < (int)cnt) {
      if (tags) {
        uint64_t t = tags[off + lane];
        if ((t >> 32) != q) {
          set_err(m, ERR_PAGE);  // counts and sorted tags disagree
        } else {
          src = (uint32_t)t;
          key = keys[src];
        }
      } else {
        const uint64_t r = *run_base + off + lane;
        if (r < n_rec && lane < (int)m.lmax) {
          src = (uint32_t)r;
          key = keys[src];
        } else {
          set_err(m, ERR_PAGE);  // counts do not fit the image
        }
      }
    }
    if (cnt > 32 || cnt > m.lmax) set_err(m, ERR_PAGE);
    warp_sort_by_key(key, src);
    for (uint32_t o = 16 * lane; o < m.page_bytes; o += 512)
      *reinterpret_cast<uint4*>(plain + o) = make_uint4(0, 0, 0, 0);
    __syncwarp();
    if (lane == 0) {
      uint64_t bitmap = cnt >= 64 ? ~0ull : ((1ull << cnt) - 1);
      *reinterpret_cast<uint64_t*>(plain) = bitmap;
    }
    if (lane < (int)cnt && lane < (int)m.lmax && src != NONE32) {
      uint8_t* slot = plain + 16 + (size_t)lane * m.rec;
      *reinterpret_cast<uint64_t*>(slot) = key;
      const uint64_t* vsrc = reinterpret_cast<const uint64_t*>(vals + (uint64_t)src * m.vb);
      for (uint32_t w = 0; w < m.vb / 8; w++)
        reinterpret_cast<uint64_t*>(slot + 8)[w] = vsrc[w];
    }
    __syncwarp();
    page_encrypt_to<SEALED>(m, plain,
                            out ? out + (q - q0) * m.page_bytes : m.pages + q * m.page_bytes, q, 0);
    __syncwarp();
  }
}

// The free ring gets every value-store slot the placement left; the
// occupancy counters start from the build's HBM residents (an empty stash),
// and the peak bin load from the largest load the build left (blockDim a
// multiple of 32).
__global__ void k_ring_fill(MapDev m, const unsigned long long* vs_fill) {
  const uint64_t used = *vs_fill < m.vs_cap ? *vs_fill : m.vs_cap;
  const uint64_t nfree = m.vs_cap - used;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nfree;
       j += (uint64_t)gridDim.x * blockDim.x)
    m.ring[j] = (uint32_t)(used + j);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    m.ring_ctr[0] = 0;
    m.ring_ctr[1] = nfree;
    m.stat[ST_HBM] = used;
    m.stat[ST_PEAK_HBM] = used;
    m.stat[ST_STASH] = 0;
    m.stat[ST_PEAK_STASH] = 0;
  }
  uint32_t top = 0;
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < m.B;
       b += (uint64_t)gridDim.x * blockDim.x)
    top = max(top, byte_get(m.load, b));
  top = __reduce_max_sync(0xffffffffu, top);
  if ((threadIdx.x & 31) == 0 && top) atomicMax(m.stat + ST_PEAK_LOAD, (unsigned long long)top);
}

// --- the data owner's image (Sec. 4.2 "Fast data initialization") ---------
// export: every record tagged (bin << 32 | record) so that sorting groups the
// records bin by bin, ascending record index within a bin
__global__ void k_image_tags(const uint32_t* __restrict__ dest, uint64_t n, uint64_t n_pow2,
                             uint64_t* __restrict__ tags) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pow2;
       i += (uint64_t)gridDim.x * blockDim.x)
    tags[i] = i < n ? ((uint64_t)dest[i] << 32) | i : ~0ull;
}

// export: the sorted records' keys, values, pairs and rows (bit 31: in b2)
__global__ void k_image_gather(MapDev m, const uint64_t* __restrict__ keys,
                               const uint8_t* __restrict__ vals, const uint64_t* __restrict__ tags,
                               const uint64_t* __restrict__ bins, const uint32_t* __restrict__ dest,
                               const uint32_t* __restrict__ prow, uint64_t n, uint64_t* img_keys,
                               uint8_t* img_vals, uint64_t* img_pairs, uint32_t* img_rows) {
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)tags[p];
    const uint64_t bb = bins[i];
    img_keys[p] = keys[i];
    const uint64_t* s = reinterpret_cast<const uint64_t*>(vals + (uint64_t)i * m.vb);
    uint64_t* d = reinterpret_cast<uint64_t*>(img_vals + p * m.vb);
    for (uint32_t w = 0; w < m.vb / 8; w++) d[w] = s[w];
    img_pairs[p] = bb;
    const uint32_t in_b2 = dest[i] == (uint32_t)(bb >> 32) ? 0x80000000u : 0u;
    img_rows[p] = (prow[i] & PROW_ROW_MASK) | in_b2;
  }
}

// load: bin counts above lmax, and the records of the HBM bins (the first of
// the image) counted into *n_hbm (blockDim a multiple of 32)
__global__ void k_image_counts(MapDev m, unsigned long long* n_hbm) {
  uint32_t s = 0;
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < m.B;
       b += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t c = byte_get(m.load, b);
    if (c > m.lmax) set_err(m, ERR_LOAD);
    if (b < m.K) s += c;
  }
  s = __reduce_add_sync(0xffffffffu, s);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(n_hbm, (unsigned long long)s);
}

// load: the counts must cover the n records exactly
__global__ void k_image_total(MapDev m, const uint32_t* page_off, const unsigned long long* n_hbm,
                              uint64_t n) {
  if (*n_hbm + page_off[m.M] != n) set_err(m, ERR_PAGE);
}

// load: every record's position-map entry (a slot of its row, claimed in any
// order: which slot holds a key is never observable) and, for the HBM bins'
// records (the first n_hbm of the image), value-store slot p
__global__ void k_image_place(MapDev m, const uint64_t* __restrict__ keys,
                              const uint8_t* __restrict__ vals, const uint64_t* __restrict__ pairs,
                              const uint32_t* __restrict__ rows, uint64_t n,
                              const unsigned long long* n_hbm_p) {
  if (*(volatile uint32_t*)m.err) return;  // counts already wrong
  const uint64_t n_hbm = *n_hbm_p;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t rw = rows[p];
    const uint32_t row = rw & 0x7fffffffu, which = rw >> 31;
    const uint64_t bb = pairs[p];
    const uint32_t bin = which ? (uint32_t)(bb >> 32) : (uint32_t)bb;
    const bool hbm = p < n_hbm;
    if (row >= m.rows || (uint32_t)bb >= m.B || (uint32_t)(bb >> 32) >= m.B ||
        (bin < m.K) != hbm || (hbm && p >= m.vs_cap)) {
      set_err(m, ERR_PAGE);  // not an image of this map's sizing
      continue;
    }
    const uint32_t slot = byte_inc(m.rowcnt, row);
    if (slot >= m.R) {
      set_err(m, ERR_ROW);
      continue;
    }
    const uint64_t pmi = (uint64_t)row * m.R + slot;
    uint32_t meta = meta_make(LOC_HOST, which, 0);
    if (hbm) {
      m.vs_key[p] = keys[p];
      const uint64_t* s = reinterpret_cast<const uint64_t*>(vals + p * m.vb);
      uint64_t* d = reinterpret_cast<uint64_t*>(m.vs_val + p * m.vb);
      for (uint32_t w = 0; w < m.vb / 8; w++) d[w] = s[w];
      m.vs_pm[p] = (uint32_t)pmi;
      m.vs_live[p] = 1;
      meta = meta_make(LOC_HBM, which, (uint32_t)p);
    }
    m.pm_key[pmi] = keys[p];
    m.pm_bins[pmi] = bb;
    m.pm_meta[pmi] = meta;
  }
}

static int sm_count() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

// Every host page: one warp gathers the page's run (from the sorted tags, or
// a contiguous run of an owner's image when tags is null), orders it by key,
// pads it, encrypts it under version 0.  With the candidate-row buffer free
// (it is read only by the rounds), pages are built into two halves of it in
// chunks and the copy engine moves each chunk to the host (pinned copies run
// faster than zero-copy stores, and hold no SM-side requests in flight);
// otherwise straight to the host.
static cudaError_t build_pages(const MapDev& m, const uint64_t* keys, const uint8_t* vals,
                               const uint64_t* tags, const unsigned long long* run_base,
                               uint64_t n_rec, BuildScratch& s, cudaStream_t st,
                               cudaStream_t copy_st, cudaEvent_t* ev_built, cudaEvent_t* ev_copied) {
  const int sms = sm_count();
  uint32_t wpb = (uint32_t)(65536 / m.page_bytes);
  wpb = wpb < 1 ? 1 : wpb > 8 ? 8 : wpb;
  size_t smem = (size_t)wpb * m.page_bytes;
  auto kp = m.integrity ? k_page_build<true> : k_page_build<false>;
  cudaError_t e = raise_smem_limit((const void*)kp, smem);
  if (e != cudaSuccess) return e;
  const uint64_t cap = (uint64_t)sms * 32;
  const uint64_t stage_bytes = s.rows4 ? s.cap * sizeof(uint4) : 0;
  const uint64_t chunk = stage_bytes / 2 / m.page_bytes;
  const bool staged = copy_st && chunk >= (1u << 14);
  ProfSpan ps(P_PAGE_BUILD, st);
  if (!staged) {
    const uint64_t blocks = (m.M + wpb - 1) / wpb;
    kp<<<(unsigned)(blocks < cap ? blocks : cap), wpb * 32, smem, st>>>(
        m, keys, vals, tags, s.page_off, wpb, 0, m.M, nullptr, run_base, n_rec);
    count_launch();
    return cudaGetLastError();
  }
  uint8_t* stage = reinterpret_cast<uint8_t*>(s.rows4);
  uint64_t c = 0;
  for (uint64_t q0 = 0; q0 < m.M; q0 += chunk, c++) {
    const uint64_t q1 = q0 + chunk < m.M ? q0 + chunk : m.M;
    const int k = (int)(c & 1);
    uint8_t* buf = stage + (uint64_t)k * chunk * m.page_bytes;
    if (c >= 2) cudaStreamWaitEvent(st, ev_copied[k], 0);
    const uint64_t blocks = (q1 - q0 + wpb - 1) / wpb;
    kp<<<(unsigned)(blocks < cap ? blocks : cap), wpb * 32, smem, st>>>(
        m, keys, vals, tags, s.page_off, wpb, q0, q1, buf, run_base, n_rec);
    count_launch();
    cudaEventRecord(ev_built[k], st);
    cudaStreamWaitEvent(copy_st, ev_built[k], 0);
    e = cudaMemcpyAsync(m.pages + q0 * m.page_bytes, buf, (q1 - q0) * m.page_bytes,
                        cudaMemcpyDefault, copy_st);
    if (e != cudaSuccess) return e;
    cudaEventRecord(ev_copied[k], copy_st);
  }
  // every chunk is on the host once the last copy on copy_st is done
  if (c) cudaStreamWaitEvent(st, ev_copied[(c - 1) & 1], 0);
  return cudaGetLastError();
}

// the page run starts: exclusive prefix sum of the host pages' loads
static void scan_page_runs(const MapDev& m, BuildScratch& s, cudaStream_t st) {
  const uint32_t nblocks = (uint32_t)((m.M + 1 + SCAN_BLOCK * SCAN_ITEMS - 1) /
                                      (SCAN_BLOCK * SCAN_ITEMS));
  k_scan_sums<<<nblocks, SCAN_BLOCK, 0, st>>>(m, s.block_sums);
  k_scan_top<<<1, SCAN_BLOCK, 0, st>>>(s.block_sums, nblocks);
  k_scan_fill<<<nblocks, SCAN_BLOCK, 0, st>>>(m, s.block_sums, s.page_off);
  count_launch(3);
}

cudaError_t launch_build(const MapDev& m, const uint64_t* keys, const uint8_t* vals, uint64_t n,
                         BuildScratch& s, cudaStream_t st, cudaEvent_t vals_wait,
                         cudaStream_t side, cudaEvent_t side_fork, cudaEvent_t side_join,
                         cudaStream_t copy_st, cudaEvent_t* ev_built, cudaEvent_t* ev_copied) {
  const int sms = sm_count();
  cudaMemsetAsync(s.counters, 0, 2 * sizeof(unsigned long long), st);
  // 1. P2C + position map, round by round
  bool deferred_place = false;
  {
    ProfSpan ps(P_P2C, st);
    bool done = false;
    int per_sm_prf = 0;
    if (s.rows4 && n && s.prf_rounds != 2 &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_prf, k_build_rounds_prf, 256, 0) ==
            cudaSuccess && per_sm_prf > 0) {
      // the rounds with the PRF inside them, when the co-resident grid has a
      // thread for every ROUNDS_KPT records of a round and a block on every
      // SM: the PRF then fills the barrier waits of a full grid (with a few
      // blocks a round has no wait to hide it in, and a PRF pass is faster)
      unsigned int* bar = reinterpret_cast<unsigned int*>(s.counters + 1);
      const uint64_t want = (m.Wr + 255) / 256;
      const uint64_t cap = (uint64_t)sms * (per_sm_prf < 4 ? per_sm_prf : 4);
      const unsigned int blocks = (unsigned int)(want < cap ? want : cap);
      if ((uint64_t)blocks * 256 * ROUNDS_KPT >= m.Wr &&
          (blocks >= (unsigned int)sms || s.prf_rounds == 1)) {
        cudaMemsetAsync(bar, 0, 8, st);
        const uint64_t* kp = keys;
        uint64_t nn = n;
        uint64_t* bp = s.bins;
        uint32_t* dp = s.dest;
        uint32_t* pp = s.prow;
        MapDev mm = m;
        void* args[] = {&mm, &kp, &nn, &bp, &dp, &pp, &bar};
        if (cudaLaunchCooperativeKernel((const void*)k_build_rounds_prf, dim3(blocks), dim3(256),
                                        args, 0, st) == cudaSuccess) {
          count_launch();
          done = true;
          deferred_place = true;
        } else {
          cudaGetLastError();  // clear; the PRF pass and the rounds kernel follow
        }
      }
    }
    if (!done && s.rows4 && n) {
      k_build_prf<<<sms * 16, 256, 0, st>>>(m, keys, n, s.bins, s.rows4);
      count_launch();
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_build_rounds, 256, 0) ==
              cudaSuccess && per_sm > 0) {
        unsigned int* bar = reinterpret_cast<unsigned int*>(s.counters + 1);
        cudaMemsetAsync(bar, 0, 8, st);
        // about one record per thread per round; a small round needs few blocks
        const uint64_t want = (m.Wr + 255) / 256;
        const uint64_t cap = (uint64_t)sms * (per_sm < 4 ? per_sm : 4);
        const unsigned int blocks = (unsigned int)(want < cap ? want : cap);
        const uint64_t* kp = keys;
        const uint8_t* vp = vals;
        uint64_t nn = n;
        const uint64_t* bp = s.bins;
        const uint4* rp = s.rows4;
        uint32_t* dp = s.dest;
        uint32_t* pp = s.prow;
        unsigned long long* fp = s.counters;
        MapDev mm = m;
        void* args[] = {&mm, &kp, &vp, &nn, &bp, &rp, &dp, &pp, &fp, &bar};
        if (cudaLaunchCooperativeKernel((const void*)k_build_rounds, dim3(blocks), dim3(256), args,
                                        0, st) == cudaSuccess) {
          count_launch();
          done = true;
          deferred_place = true;
        } else {
          cudaGetLastError();  // clear; fall back to one launch pair per round
        }
      }
    }
    if (!done && vals_wait) cudaStreamWaitEvent(st, vals_wait, 0);
    for (uint64_t lo = 0; !done && lo < n; lo += m.Wr) {
      uint64_t hi = lo + m.Wr < n ? lo + m.Wr : n;
      unsigned g = (unsigned)((hi - lo + 255) / 256);
      k_build_decide<<<g, 256, 0, st>>>(m, keys, lo, hi, s.bins, s.rows4, s.dest, s.prow);
      k_build_apply<<<g, 256, 0, st>>>(m, keys, vals, lo, hi, s.bins, s.dest, s.prow,
                                        s.counters);
      count_launch(2);
    }
  }
  // 2. page run starts
  scan_page_runs(m, s, st);
  // 3. host records grouped by page: two bucket passes with the bucket
  // tags and cursors in the rows4 buffer (free between the rounds and the
  // page staging); without it, tags + bitonic sort
  cudaError_t e;
  const uint32_t nbk = (uint32_t)((m.M + GROUP_PAGES - 1) >> GROUP_PAGE_BITS);
  if (s.rows4 && s.cap * sizeof(uint4) >= n * sizeof(uint64_t) + 2ull * nbk * sizeof(uint32_t)) {
    ProfSpan ps(P_PAGE_GROUP, st);
    uint64_t* tmp = reinterpret_cast<uint64_t*>(s.rows4);
    uint32_t* bcur = reinterpret_cast<uint32_t*>(tmp + n);
    uint32_t* bend = bcur + nbk;
    k_group_init<<<(nbk + 255) / 256, 256, 0, st>>>(m, s.page_off, nbk, bcur, bend);
    k_group_buckets<<<sms * 8, 256, 0, st>>>(m, s.dest, n, bcur, bend, tmp);
    k_group_pages<<<nbk < (uint32_t)sms * 16 ? nbk : (uint32_t)sms * 16, 256, 0, st>>>(
        m, s.page_off, nbk, tmp, s.tags);
    count_launch(3);
  } else {
    k_build_tags<<<sms * 8, 256, 0, st>>>(m, s.dest, n, s.tag_cap, s.tags);
    count_launch();
    e = sort_tags_u64(s.tags, s.tag_cap, s.log_tile, st);
    if (e != cudaSuccess) return e;
  }
  // The position-map entries and HBM residents (k_build_place) are read by
  // none of the steps that follow, so after the rounds kernel they are
  // written on the side stream beside the page build, which is bound by the
  // host link; the free ring needs their count and follows them.
  if (deferred_place) {
    cudaEventRecord(side_fork, st);
    cudaStreamWaitEvent(side, side_fork, 0);
    {
      ProfSpan ps(P_P2C, side);
      k_build_place<<<sms * 16, 256, 0, side>>>(m, keys, vals, n, s.bins, s.dest, s.prow,
                                                 s.counters);
      count_launch();
    }
    k_ring_fill<<<sms * 4, 256, 0, side>>>(m, s.counters);
    count_launch();
    cudaEventRecord(side_join, side);
  }
  // 4. pages (they read the values)
  if (vals_wait) cudaStreamWaitEvent(st, vals_wait, 0);
  e = build_pages(m, keys, vals, s.tags, nullptr, n, s, st, copy_st, ev_built, ev_copied);
  if (e != cudaSuccess) return e;
  // 5. free ring
  if (deferred_place) {
    cudaStreamWaitEvent(st, side_join, 0);
  } else {
    k_ring_fill<<<sms * 4, 256, 0, st>>>(m, s.counters);
    count_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_image_export(const MapDev& m, const uint64_t* keys, const uint8_t* vals,
                                uint64_t n, BuildScratch& s, cudaStream_t st, uint64_t* img_keys,
                                uint8_t* img_vals, uint64_t* img_pairs, uint32_t* img_rows,
                                uint8_t* img_counts) {
  const int sms = sm_count();
  cudaError_t e = cudaMemcpyAsync(img_counts, m.load, m.B, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess || n == 0) return e;
  k_image_tags<<<sms * 8, 256, 0, st>>>(s.dest, n, s.tag_cap, s.tags);
  count_launch();
  e = sort_tags_u64(s.tags, s.tag_cap, s.log_tile, st);
  if (e != cudaSuccess) return e;
  k_image_gather<<<sms * 8, 256, 0, st>>>(m, keys, vals, s.tags, s.bins, s.dest, s.prow, n,
                                          img_keys, img_vals, img_pairs, img_rows);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_image_load(const MapDev& m, const uint64_t* keys, const uint8_t* vals,
                              const uint64_t* pairs, const uint32_t* rows, const uint8_t* counts,
                              uint64_t n, BuildScratch& s, cudaStream_t st, cudaStream_t side,
                              cudaEvent_t side_fork, cudaEvent_t side_join, cudaStream_t copy_st,
                              cudaEvent_t* ev_built, cudaEvent_t* ev_copied) {
  const int sms = sm_count();
  // bin loads straight from the counts (one byte per bin, as the map packs them)
  cudaError_t e = cudaMemcpyAsync(m.load, counts, m.B, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  unsigned long long* n_hbm = s.counters;
  cudaMemsetAsync(s.counters, 0, 2 * sizeof(unsigned long long), st);
  k_image_counts<<<sms * 4, 256, 0, st>>>(m, n_hbm);
  scan_page_runs(m, s, st);
  k_image_total<<<1, 1, 0, st>>>(m, s.page_off, n_hbm, n);
  count_launch(2);
  // the position-map entries, HBM residents and free ring are read by no
  // step of the page build: they are written on the side stream beside it
  cudaEventRecord(side_fork, st);
  cudaStreamWaitEvent(side, side_fork, 0);
  {
    ProfSpan ps(P_P2C, side);
    k_image_place<<<sms * 16, 256, 0, side>>>(m, keys, vals, pairs, rows, n, n_hbm);
    count_launch();
  }
  k_ring_fill<<<sms * 4, 256, 0, side>>>(m, s.counters);
  count_launch();
  cudaEventRecord(side_join, side);
  e = build_pages(m, keys, vals, nullptr, n_hbm, n, s, st, copy_st, ev_built, ev_copied);
  if (e != cudaSuccess) return e;
  cudaStreamWaitEvent(st, side_join, 0);
  return cudaGetLastError();
}

}  // namespace bdev
