// access.cu -- batched oblivious access (Alg. 1 over a batch of operations,
// with the module order of Sec. 4.1: KS -> VAC -> exec -> write-back -> RMP).
//
// One batch of n <= BOLT_MAX_BATCH operations, operation i with global
// sequence number t0 + i:
//   k_stage     per op: sort element (key, i); PRF pairs for DUMMY and REMAP,
//               position-map rows PRF(PM, key)
//   sort        (key, i) ascending (bitonic, sort.cu)
//   k_group     one CTA: leader (first op on the key), previous writer of each
//               op, last writer of each key group, by prefix-max scans
//   k_lookup    warp per op: leaders scan their d rows of the position map
//               (ballot over the R slots of each row); hit -> stored pair,
//               otherwise the DUMMY pair; host bins enter a page hash table,
//               and the position claiming a page's slot reads it (zero-copy
//               16-byte loads of the pinned host page) and decrypts it
//               (quad-cooperative ChaCha20 key stream) into the slot's buffer
//   k_pages     (trace on) read/write trace, distinct pages in first-read
//               order
//   k_find      warp per op: find_remove of each hit (page scan by ballot, or
//               the value store), load and position-map bookkeeping
//   k_exec_evict  blocks of warps per page: write-back (below); other blocks
//               per op: Get/Put/Delete semantics in op order per key, and the
//               P2C decision when the remap is one round
//   (evict)     warp per distinct page: remaining tuples + stash items bound
//               for the page, ordered by key, dummy-padded, version + 1,
//               encrypted, written back to the host page
//   k_remap_*   P2C remap of every key present after the batch, in rounds of
//               W_r operation slots decided on round-start loads
// A batch of at most FUSED_MAX_OPS operations runs all of these steps in one
// CTA instead (k_fused, below).
#include "bolt_internal.cuh"
#include "batch.cuh"

namespace bdev {

__device__ __forceinline__ uint32_t key_hash(uint64_t k, uint32_t mask) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  return (uint32_t)k & mask;
}

// SMs of the current device (queried once per device)
static int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cached[dev]) {
    int v = 148;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 148;
  }
  return cached[dev];
}

// Programmatic dependent launch for the batch's main chain: a kernel
// launched with launch_dependent() may be scheduled while its predecessor on
// the stream finishes; it must pass dep_wait() before touching anything the
// predecessor wrote (a no-op when launched normally).  dep_trigger() lets the
// successor be scheduled once every block of this kernel has reached it.
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void dep_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... Params, typename... Args>
static cudaError_t launch_dependent(void (*kernel)(Params...), unsigned grid, unsigned block,
                                    size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Params>(args)...);
}

// per op: PRF pairs and rows, and the op's grouping key.  Equal keys share a
// hash-table slot (claimed by the first op to reach it), so sorting
// (slot << 16 | op) lists every key's ops together, in op order.
// Batches of at most 4096 ops pack (slot << 12 | op) into 32 bits (slot <
// 8192); larger ones use (slot << 16 | op) in 64 bits.
__global__ void k_stage(MapDev m, BatchDev b, uint32_t n, uint32_t n_sort, uint64_t t0,
                        int keys32) {
  // three threads per op: 0 = grouping key + DUMMY pair, 1 = REMAP pair,
  // 2 = position-map rows (one ChaCha20 block each)
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t i = tid / 3, kind = tid % 3;
  if (i >= n_sort) return;
  if (i >= n) {
    if (kind == 0) {
      if (keys32) reinterpret_cast<uint32_t*>(b.skeys)[i] = ~0u;
      else b.skeys[i] = ~0ull;
    }
    return;
  }
  const uint64_t key = b.keys[i];
  uint32_t p1, p2;
  if (kind == 0) {
    uint32_t h = key_hash(key, b.kt_mask);
    for (uint32_t probe = 0; probe <= b.kt_mask; probe++) {
      const uint32_t old = atomicCAS(b.kt_own + h, 0u, i + 1);
      if (old == 0 || b.keys[old - 1] == key) break;
      h = (h + 1) & b.kt_mask;
    }
    if (keys32) reinterpret_cast<uint32_t*>(b.skeys)[i] = (h << 12) | i;
    else b.skeys[i] = ((uint64_t)h << 16) | i;
    prf_pair(m, DOM_DUMMY, t0 + i, p1, p2);
    b.pair[i] = (uint64_t)p1 | ((uint64_t)p2 << 32);
  } else if (kind == 1) {
    prf_pair(m, DOM_REMAP, t0 + i, p1, p2);
    b.rpair[i] = (uint64_t)p1 | ((uint64_t)p2 << 32);
  } else {
    uint32_t rows[4];
    prf_rows(m, key, rows);
    *reinterpret_cast<uint4*>(b.rows + 4 * (uint64_t)i) =
        make_uint4(rows[0], rows[1], rows[2], rows[3]);
  }
}

// ---------------------------------------------------------------------------
// grouping: prefix-max scans over the sorted (key, op) sequence
__device__ __forceinline__ int32_t block_excl_max(int32_t v, int32_t* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x = max(x, y);
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int32_t w = lane < (int)(blockDim.x >> 5) ? sh[lane] : -1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w = max(w, y);
    }
    sh[lane] = w;
  }
  __syncthreads();
  int32_t prev_warps = wid > 0 ? sh[wid - 1] : -1;
  int32_t excl = __shfl_up_sync(0xffffffffu, x, 1);
  if (lane == 0) excl = -1;
  excl = max(excl, prev_warps);
  __syncthreads();
  return excl;
}

constexpr int GROUP_THREADS = 1024;

// grouping keys sort as (slot << SHIFT | op): a group is a run of equal slots
template <typename K>
struct GroupKey {
  static constexpr int SHIFT = sizeof(K) == 4 ? 12 : 16;
  static __device__ __forceinline__ uint32_t slot(K k) { return (uint32_t)(k >> SHIFT); }
  static __device__ __forceinline__ uint32_t op(K k) {
    return (uint32_t)(k & (((K)1 << SHIFT) - 1));
  }
};

template <typename K>
__global__ void __launch_bounds__(GROUP_THREADS) k_group(BatchDev b, uint32_t n) {
  using G = GroupKey<K>;
  const K* sk = reinterpret_cast<const K*>(b.skeys);
  __shared__ int32_t sh[32];
  const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
  const uint32_t lo = threadIdx.x * per;
  const uint32_t hi = min(n, lo + per);
  // local maxima of group-head positions and writer positions
  int32_t hmax = -1, wmax = -1;
  for (uint32_t s = lo; s < hi; s++) {
    const K e = sk[s];
    const bool head = s == 0 || G::slot(sk[s - 1]) != G::slot(e);
    if (head) hmax = (int32_t)s;
    if (b.ops[G::op(e)] != OP_GET) wmax = (int32_t)s;
  }
  int32_t hcar = block_excl_max(hmax, sh);
  int32_t wcar = block_excl_max(wmax, sh);
  for (uint32_t s = lo; s < hi; s++) {
    const K e = sk[s];
    const uint32_t i = G::op(e);
    const bool head = s == 0 || G::slot(sk[s - 1]) != G::slot(e);
    if (head) hcar = (int32_t)s;
    const uint32_t lead = G::op(sk[hcar]);
    // previous writer in the same group (strictly before s)
    b.prevw[i] = wcar >= hcar ? G::op(sk[wcar]) : NONE32;
    b.leader[i] = lead;
    if (b.ops[i] != OP_GET) wcar = (int32_t)s;
    const bool last = s + 1 == n || G::slot(sk[s + 1]) != G::slot(e);
    if (last) b.lastw[lead] = wcar >= hcar ? G::op(sk[wcar]) : NONE32;
  }
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ht_hash(uint32_t page, uint32_t mask) {
  return (page * 0x9E3779B1u) & mask;
}

// page into the batch's page table; returns the slot if this call claimed
// it (the caller then reads the page), NONE32 if the page was already there
__device__ __forceinline__ uint32_t ht_insert(const BatchDev& b, uint32_t page, uint32_t pos) {
  uint32_t h = ht_hash(page, b.ht_mask);
  for (uint32_t probe = 0; probe <= b.ht_mask; probe++) {
    uint32_t old = atomicCAS(b.ht_key + h, NONE32, page);
    if (old == NONE32 || old == page) {
      atomicMin(b.ht_min + h, pos);
      b.pos_slot[pos] = h;
      return old == NONE32 ? h : NONE32;
    }
    h = (h + 1) & b.ht_mask;
  }
  return NONE32;
}

// The warp scans the key's d = 4 rows, R slots each (a ballot per row; the
// first row with a match, then its first matching slot).  Every slot's
// metadata, key and bin pair of all four rows are loaded at once -- one
// memory round trip instead of two per row -- and *bins receives the pair
// of the matching slot (all lanes), *hmeta (if given) its metadata.
__device__ __forceinline__ uint32_t pm_search(const MapDev& m, const BatchDev& b, uint32_t i,
                                              uint64_t key, int lane, uint64_t* bins,
                                              uint32_t* hmeta = nullptr) {
  const uint4 rows = *reinterpret_cast<const uint4*>(b.rows + 4 * (uint64_t)i);
  const uint32_t rr[4] = {rows.x, rows.y, rows.z, rows.w};
  const bool in = lane < (int)m.R;
  uint32_t meta[4];
  uint64_t k[4], pb[4];
#pragma unroll
  for (int j = 0; j < 4; j++) {
    const uint64_t idx = (uint64_t)rr[j] * m.R + lane;
    meta[j] = in ? m.pm_meta[idx] : 0u;
    k[j] = in ? m.pm_key[idx] : 0ull;
    pb[j] = in ? m.pm_bins[idx] : 0ull;
  }
  uint32_t found = NONE32, fm = 0;
  uint64_t fb = 0;
#pragma unroll
  for (int j = 3; j >= 0; j--) {  // the lowest matching row wins
    const uint32_t bal = __ballot_sync(0xffffffffu, meta_loc(meta[j]) != LOC_EMPTY && k[j] == key);
    if (bal) {
      const int s = __ffs(bal) - 1;
      found = (uint32_t)((uint64_t)rr[j] * m.R + s);
      fb = __shfl_sync(0xffffffffu, pb[j], s);
      fm = __shfl_sync(0xffffffffu, meta[j], s);
    }
  }
  *bins = fb;
  if (hmeta) *hmeta = fm;
  return found;
}

// ---------------------------------------------------------------------------
// lookahead
constexpr uint32_t PREV_UNKNOWN = 0xFFFFFFFEu;

// the previous batch's op owning the key's slot in its key table; NONE32 if
// the key is not in the previous batch
__device__ __forceinline__ uint32_t prev_owner(const BatchDev& b, uint64_t key) {
  uint32_t h = key_hash(key, b.prev_kt_mask);
  for (uint32_t probe = 0; probe <= b.prev_kt_mask; probe++) {
    const uint32_t own = b.prev_kt_own[h];
    if (own == 0) return NONE32;
    if (b.prev_keys[own - 1] == key) return own - 1;
    h = (h + 1) & b.prev_kt_mask;
  }
  return PREV_UNKNOWN;
}

__device__ __forceinline__ void la_insert(const BatchDev& b, uint32_t q) {
  uint32_t h = ht_hash(q, b.ht_mask);
  for (uint32_t probe = 0; probe <= b.ht_mask; probe++) {
    const uint32_t old = atomicCAS(b.la_key + h, NONE32, q);
    if (old == NONE32) {
      const uint32_t e = atomicAdd(b.la_count, 1u);
      b.la_idx[h] = e;
      b.la_list[e] = q;
      return;
    }
    if (old == q) return;
    h = (h + 1) & b.ht_mask;
  }
}

__device__ __forceinline__ uint32_t la_find(const BatchDev& b, uint32_t q) {
  uint32_t h = ht_hash(q, b.ht_mask);
  for (uint32_t probe = 0; probe <= b.ht_mask; probe++) {
    const uint32_t k = b.la_key[h];
    if (k == q) {
      const uint32_t e = b.la_idx[h];
      return e < b.la_limit ? e : NONE32;  // queued beyond the limit: not read
    }
    if (k == NONE32) return NONE32;
    h = (h + 1) & b.ht_mask;
  }
  return NONE32;
}

__global__ void k_clear_la(BatchDev b) {
  for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h <= b.ht_mask;
       h += gridDim.x * blockDim.x)
    b.la_key[h] = NONE32;
  if (blockIdx.x == 0 && threadIdx.x == 0) *b.la_count = 0;
}

// warp per op: leaders whose key the previous batch does not touch search the
// position map now (the previous batch changes no slot of such a key: it
// removes, deletes and re-places only its own keys, and its eviction changes
// only the location field of an occupied slot).  A leader whose key the
// previous batch touches gets the bins that batch re-maps it to (its
// leader's REMAP pair) if the key is present after it, else its DUMMY pair.
// Then the page of every read position whose bin is known is queued for
// reading ahead.  What is found here only decides which pages are read
// ahead: the main lookup re-checks hits and searches for the other leaders.
__global__ void k_ahead_lookup(MapDev m, BatchDev b, uint32_t n) {
  const uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  bool known = true;
  uint64_t pr = b.pair[i];
  if (b.leader[i] == i) {
    const uint64_t key = b.keys[i];
    const uint32_t o = prev_owner(b, key);
    if (o == NONE32) {
      uint64_t fb;
      const uint32_t found = pm_search(m, b, i, key, lane, &fb);
      if (found != NONE32) pr = fb;
      if (lane == 0) {
        b.hit[i] = found;
        b.done[i] = 1;
        b.pres[i] = found != NONE32 ? 1 : 0;
      }
    } else {
      uint32_t after = 2;
      uint32_t lead = 0;
      if (o != PREV_UNKNOWN) {
        lead = b.prev_leader[o];
        const uint32_t lw = b.prev_lastw[lead];
        after = lw != NONE32 ? (b.prev_ops[lw] == OP_PUT ? 1u : 0u) : b.prev_pres[lead];
      }
      if (after == 1) pr = b.prev_rpair[lead];
      known = after != 2;
      if (lane == 0) {
        b.done[i] = 0;
        b.pres[i] = (uint8_t)after;
      }
    }
  }
  if (known && lane < 2) {
    const uint32_t p = lane == 0 ? (uint32_t)pr : (uint32_t)(pr >> 32);
    if (p >= m.K) la_insert(b, (uint32_t)(p - m.K));
  }
}

// Host-page copies that run while other kernels of the access path run use
// few warps, one 512-byte chunk in flight per warp: pending host reads and
// writes slow down every random HBM access on the device roughly in
// proportion to how many are outstanding, while a few hundred in flight
// already keep the host link near its random-page rate.
constexpr uint32_t LINK_WARPS = 192;
constexpr uint32_t COPY_BLOCK = 128;
constexpr uint32_t LINK_BLOCKS = LINK_WARPS * 32 / COPY_BLOCK;
// The write-back of batch k has until batch k + 2 starts and runs beside
// batch k + 1, whose random HBM accesses and page reads it slows in
// proportion to its writes in flight: as few warps as keep it inside about
// one batch time.  A warp writes a page per ~1.2 us, a 4096-op batch (~6.5 k
// host pages at N = 2^28) takes ~220 us, so about one warp per 160 read
// positions (2 per op), between 16 and 192 warps.
__host__ __device__ __forceinline__ uint32_t flush_blocks(uint32_t n, int fast) {
  uint32_t w = 2 * n / (fast ? 80 : 160);
  w = w < 16 ? 16 : (w > 192 ? 192 : w);
  return (w * 32 + COPY_BLOCK - 1) / COPY_BLOCK;
}

// the pages queued ahead, one 512-byte chunk per warp step: host read +
// decryption into la_buf.  Pages the previous batch rewrites may be read torn
// here; the main gather takes those from the previous batch's ciphertexts.
__global__ void __launch_bounds__(COPY_BLOCK) k_ahead_gather(MapDev m, BatchDev b,
                                                             uint32_t limit) {
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t nch = (m.page_bytes + 511) / 512;
  const uint32_t cnt = *b.la_count;
  const uint32_t items = (cnt < limit ? cnt : limit) * nch;
  for (uint32_t it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < items; it += nw) {
    const uint32_t e = it / nch, c = (it % nch) * 512, off = c + 16 * lane;
    const uint64_t q = b.la_list[e];
    uint4 x = make_uint4(0, 0, 0, 0);
    if (off < m.page_bytes) x = *reinterpret_cast<const uint4*>(m.pages + q * m.page_bytes + off);
    const uint64_t v = m.version[q];
    const uint4 ks = chacha_quad(m.kenc, c / 64 + (lane >> 2), (uint32_t)q, (uint32_t)v,
                                 (uint32_t)(v >> 32));
    if (off < m.page_bytes) {
      x.x ^= ks.x; x.y ^= ks.y; x.z ^= ks.z; x.w ^= ks.w;
      *reinterpret_cast<uint4*>(b.la_buf + (uint64_t)e * m.page_bytes + off) = x;
    }
  }
}

// The host-access trace (parity runs): every read position's page in
// position order, then each distinct page once, in first-read order, as a
// write.  Three passes over the 2n read positions: per-block counts of valid
// reads and of first reads, one scan of the block counts, then ranks and
// outputs.
constexpr int PAGES_BLOCK = 256;

__device__ __forceinline__ void pos_flags(const BatchDev& b, uint32_t p, uint32_t np, bool& valid,
                                          bool& first, uint32_t& q, uint32_t& slot) {
  valid = first = false;
  q = NONE32;
  slot = 0;
  if (p >= np) return;
  q = b.pos_page[p];
  if (q == NONE32) return;
  valid = true;
  slot = b.pos_slot[p];
  first = b.ht_min[slot] == p;
}

__global__ void __launch_bounds__(PAGES_BLOCK) k_pages_count(BatchDev b, uint32_t np,
                                                             uint32_t* block_cnt) {
  __shared__ uint32_t sh[32];
  const uint32_t p = blockIdx.x * PAGES_BLOCK + threadIdx.x;
  bool valid, first;
  uint32_t q, slot;
  pos_flags(b, p, np, valid, first, q, slot);
  uint32_t tv, tf;
  block_excl_scan(valid ? 1u : 0u, sh, tv);
  block_excl_scan(first ? 1u : 0u, sh, tf);
  if (threadIdx.x == 0) {
    block_cnt[2 * blockIdx.x] = tv;
    block_cnt[2 * blockIdx.x + 1] = tf;
  }
}

// one block: exclusive scan of the per-block (valid, first) counts in place
__global__ void __launch_bounds__(1024) k_pages_scan(MapDev m, BatchDev b, uint32_t nblocks,
                                                     uint32_t* block_cnt) {
  __shared__ uint32_t sh[32];
  __shared__ uint32_t carry_v, carry_f;
  if (threadIdx.x == 0) carry_v = carry_f = 0;
  __syncthreads();
  for (uint32_t lo = 0; lo < nblocks; lo += 1024) {
    const uint32_t i = lo + threadIdx.x;
    const uint32_t v = i < nblocks ? block_cnt[2 * i] : 0;
    const uint32_t f = i < nblocks ? block_cnt[2 * i + 1] : 0;
    uint32_t tv, tf;
    const uint32_t ev = block_excl_scan(v, sh, tv);
    const uint32_t ef = block_excl_scan(f, sh, tf);
    if (i < nblocks) {
      block_cnt[2 * i] = carry_v + ev;
      block_cnt[2 * i + 1] = carry_f + ef;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      carry_v += tv;
      carry_f += tf;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const uint64_t tbase = m.trace_on ? *m.trace_len : 0;
    b.trace_base[0] = tbase;
    b.trace_base[1] = carry_v;
    if (m.trace_on) *m.trace_len = tbase + carry_v + carry_f;
  }
}

__global__ void __launch_bounds__(PAGES_BLOCK) k_pages_emit(MapDev m, BatchDev b, uint32_t np,
                                                            const uint32_t* block_cnt) {
  __shared__ uint32_t sh[32];
  const uint32_t p = blockIdx.x * PAGES_BLOCK + threadIdx.x;
  bool valid, first;
  uint32_t q, slot;
  pos_flags(b, p, np, valid, first, q, slot);
  uint32_t tv, tf;
  const uint32_t rv = block_excl_scan(valid ? 1u : 0u, sh, tv) + block_cnt[2 * blockIdx.x];
  const uint32_t d = block_excl_scan(first ? 1u : 0u, sh, tf) + block_cnt[2 * blockIdx.x + 1];
  if (!valid) return;
  const uint64_t tbase = b.trace_base[0], tot_valid = b.trace_base[1];
  if (m.trace_on && tbase + rv < m.trace_cap) m.trace[tbase + rv] = q;
  if (first) {
    const uint64_t w = tbase + tot_valid + d;
    if (m.trace_on && w < m.trace_cap) m.trace[w] = q | 0x80000000u;
  }
}

// Batches of up to 4096 ops (8192 read positions): the three passes in one
// CTA, each thread over 8 consecutive positions.
constexpr uint32_t PAGES_SMALL_MAX = 8192;

__global__ void __launch_bounds__(1024) k_pages_small(MapDev m, BatchDev b, uint32_t np) {
  __shared__ uint32_t sh[32];
  __shared__ unsigned long long s_tbase;
  const uint32_t per = (np + 1023) / 1024;
  const uint32_t lo = threadIdx.x * per;
  uint32_t qs[8], slots[8], flags = 0, cv = 0, cf = 0;
#pragma unroll
  for (uint32_t k = 0; k < 8; k++) {
    bool valid = false, first = false;
    qs[k] = NONE32;
    slots[k] = 0;
    if (k < per) pos_flags(b, lo + k, np, valid, first, qs[k], slots[k]);
    cv += valid;
    cf += first;
    flags |= (valid ? 1u : 0u) << (2 * k);
    flags |= (first ? 1u : 0u) << (2 * k + 1);
  }
  uint32_t tv, tf;
  uint32_t rv = block_excl_scan(cv, sh, tv);
  uint32_t d = block_excl_scan(cf, sh, tf);
  if (threadIdx.x == 0) {
    const uint64_t tbase = m.trace_on ? *m.trace_len : 0;
    s_tbase = tbase;
    b.trace_base[0] = tbase;
    b.trace_base[1] = tv;
    if (m.trace_on) *m.trace_len = tbase + tv + tf;
  }
  __syncthreads();
  const uint64_t tbase = s_tbase;
#pragma unroll
  for (uint32_t k = 0; k < 8; k++) {
    if (!((flags >> (2 * k)) & 1u)) continue;
    if (m.trace_on && tbase + rv < m.trace_cap) m.trace[tbase + rv] = qs[k];
    rv++;
    if ((flags >> (2 * k + 1)) & 1u) {
      const uint64_t w = tbase + tv + d;
      if (m.trace_on && w < m.trace_cap) m.trace[w] = qs[k] | 0x80000000u;
      d++;
    }
  }
}

// page q in the previous batch's write set? -> its slot there, else NONE
__device__ __forceinline__ uint32_t prev_written(const BatchDev& b, uint32_t q) {
  if (!b.prev_valid) return NONE32;
  uint32_t h = ht_hash(q, b.prev_ht_mask);
  for (uint32_t probe = 0; probe <= b.prev_ht_mask; probe++) {
    const uint32_t k = b.prev_ht_key[h];
    if (k == q) return h;
    if (k == NONE32) return NONE32;
    h = (h + 1) & b.prev_ht_mask;
  }
  return NONE32;
}

// Where a claimed page comes from: the host page (ciphertext), the previous
// batch's not-yet-flushed ciphertext, or a plaintext read ahead.
enum : int { SRC_NONE = 0, SRC_HOST = 1, SRC_PREV = 2, SRC_PLAIN = 3 };

// the rest of a page whose first 16 bytes per lane are in `first`: decrypt
// (unless already plaintext) into the slot's buffer.  A sealed page (integrity
// on) is opened as the AEAD of RFC 8439 Sec. 2.8: Poly1305 over its
// ciphertext and lengths block, checked against the tag in its last 16
// bytes; on a mismatch (the host altered or replayed the page) the slot gets
// an empty page and ERR_INTEGRITY is raised, so nothing of the altered page
// enters the map.  All 32 lanes call; SEALED = m.integrity.
template <bool SEALED>
__device__ __forceinline__ void page_in(const MapDev& m, const BatchDev& b, uint32_t slot,
                                        uint64_t q, int kind, const uint8_t* src, uint4 first,
                                        int lane) {
  uint8_t* dst = b.dbuf + (uint64_t)slot * m.page_bytes;
  const uint64_t v = kind == SRC_PLAIN ? 0 : m.version[q];
  const uint32_t L = m.page_bytes - (SEALED ? 16u : 0u);
  const uint32_t sealed = (SEALED && kind != SRC_PLAIN) ? 1u : 0u;
  PolyWarp pw;
  if (SEALED && sealed) pw = poly_begin(m, q, v);
  uint4 stored = make_uint4(0, 0, 0, 0);
  for (uint32_t c = 0; c < m.page_bytes; c += 512) {
    const uint32_t off = c + 16 * lane;
    uint4 x = first;
    if (c > 0 && off < m.page_bytes) x = *reinterpret_cast<const uint4*>(src + off);
    if (kind != SRC_PLAIN) {
      if (SEALED && sealed) {
        if (off == L) stored = x;
        if (off <= L) poly_block(pw, off / 16, off < L ? x : poly_lengths(L));
      }
      const uint4 ks = chacha_quad(m.kenc, c / 64 + (lane >> 2) + sealed, (uint32_t)q,
                                   (uint32_t)v, (uint32_t)(v >> 32));
      x.x ^= ks.x; x.y ^= ks.y; x.z ^= ks.z; x.w ^= ks.w;
    }
    if (off < L) *reinterpret_cast<uint4*>(dst + off) = x;
    else if (off < m.page_bytes) *reinterpret_cast<uint4*>(dst + off) = make_uint4(0, 0, 0, 0);
  }
  if (SEALED && sealed) {
    const uint4 tag = poly_finish(pw, L / 16 + 1);
    const bool bad = lane == (int)((L / 16) & 31) &&
                     (tag.x != stored.x || tag.y != stored.y || tag.z != stored.z ||
                      tag.w != stored.w);
    if (__any_sync(0xffffffffu, bad)) {
      if (lane == 0) set_err(m, ERR_INTEGRITY);
      for (uint32_t off = 16 * lane; off < m.page_bytes; off += 512)
        *reinterpret_cast<uint4*>(dst + off) = make_uint4(0, 0, 0, 0);
    }
  }
  if (lane == 0) b.removed[slot] = 0;
}

// the rest of a page whose first 16 bytes per lane are in `first`, copied as
// it is (sealed ciphertext) into the slot's buffer.  All 32 lanes call.
__device__ __forceinline__ void page_copy(const MapDev& m, const BatchDev& b, uint32_t slot,
                                          const uint8_t* src, uint4 first, int lane) {
  uint8_t* dst = b.dbuf + (uint64_t)slot * m.page_bytes;
  for (uint32_t c = 0; c < m.page_bytes; c += 512) {
    const uint32_t off = c + 16 * lane;
    uint4 x = first;
    if (c > 0 && off < m.page_bytes) x = *reinterpret_cast<const uint4*>(src + off);
    if (off < m.page_bytes) *reinterpret_cast<uint4*>(dst + off) = x;
  }
  if (lane == 0) b.removed[slot] = 0;
}

// Sealed pages of a batch, a warp per page (claim order): the ciphertext
// k_lookup left in the slot's buffer is checked against its tag and
// decrypted in place (page_in; a page that fails reads as empty and raises
// ERR_INTEGRITY).  Separate from k_lookup, whose warps wait on host reads, so
// that the Poly1305 work runs on every warp of the GPU at once.
__global__ void __launch_bounds__(256) k_open(MapDev m, BatchDev b) {
  dep_wait();
  const int lane = threadIdx.x & 31;
  const uint32_t nd = *b.dcount;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t d = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; d < nd; d += nw) {
    const uint32_t slot = b.dslot[d];
    const uint64_t q = b.dpage[d];
    const uint8_t* pg = b.dbuf + (uint64_t)slot * m.page_bytes;
    uint4 x = make_uint4(0, 0, 0, 0);
    if (16 * lane < m.page_bytes) x = *reinterpret_cast<const uint4*>(pg + 16 * lane);
    page_in<true>(m, b, slot, q, SRC_HOST, pg, x, lane);
  }
}

// warp per op (Alg. 1 lines 2-5 over a batch): leaders search the position
// map -- a hit reads the stored pair, a miss and every non-leader the DUMMY
// pair -- and the two bins' host pages enter the batch's page table.  The
// position that claims a page's slot reads the page at once into the slot's
// buffer: from the previous batch's ciphertext if that batch wrote it
// (its host copy may still be in flight), from the plaintext read ahead
// (lookahead), else from the host.  With lookahead, a leader searched ahead
// keeps a miss and re-checks a hit (a slot the previous batch was re-using
// could have looked like a match), the others search now.
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
// every 128-byte line of [p, p + bytes) into L2
__device__ __forceinline__ void prefetch_range_l2(const void* p, uint32_t bytes) {
  const uintptr_t e = (uintptr_t)p + bytes;
  for (uintptr_t a = (uintptr_t)p & ~(uintptr_t)127; a < e; a += 128)
    prefetch_l2(reinterpret_cast<const void*>(a));
}
// [p, p + bytes) into L2 by the bulk-copy unit: p 16-byte aligned, bytes a
// multiple of 16; exactly these bytes are read
__device__ __forceinline__ void prefetch_bulk_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// While a claimed page's host read is in flight: bring what its eviction will
// read into L2 -- the reverse-index count and list, then each listed stash
// item's live flag, key, map slot and value (only entries below the count:
// those past it are stale).  All 32 lanes call.
__device__ __forceinline__ void prefetch_eviction(const MapDev& m, uint32_t q, bool claimed,
                                                  int lane) {
  uint32_t vs = NONE32;
  if (claimed && lane < (int)m.lmax) {
    const uint32_t e = m.rev[(uint64_t)q * m.lmax + lane];
    if (lane < (int)byte_get(m.revcnt, q)) vs = e;
  }
  if (vs != NONE32) {
    prefetch_l2(m.vs_live + vs);
    prefetch_l2(m.vs_key + vs);
    prefetch_l2(m.vs_pm + vs);
    prefetch_l2(m.vs_val + (uint64_t)vs * m.vb);
  }
}

template <bool SEALED>
__device__ __forceinline__ void lookup_op(const MapDev& m, const BatchDev& b, uint32_t i,
                                          int lane) {
  uint32_t found = NONE32;
  uint64_t fb = 0;
  if (b.leader[i] == i) {
    const uint64_t key = b.keys[i];
    bool scan = true;
    if (b.la_on && b.done[i]) {
      const uint32_t hs = b.hit[i];
      if (hs == NONE32) {
        scan = false;
      } else if (meta_loc(m.pm_meta[hs]) != LOC_EMPTY && m.pm_key[hs] == key) {
        found = hs;
        fb = m.pm_bins[hs];
        scan = false;
      }
    }
    if (scan) found = pm_search(m, b, i, key, lane, &fb);
  }
  // a hit reads its stored pair, everything else the DUMMY pair
  const uint64_t pr = found != NONE32 ? fb : b.pair[i];
  if (lane == 0) {
    b.hit[i] = found;
    if (found != NONE32) b.pair[i] = pr;
  }
  uint32_t q = NONE32, claim = NONE32;
  if (lane < 2) {
    const uint32_t p = lane == 0 ? (uint32_t)pr : (uint32_t)(pr >> 32);
    const uint32_t pos = 2 * i + lane;
    if (p >= m.K) {
      q = (uint32_t)(p - m.K);
      b.pos_page[pos] = q;
      claim = ht_insert(b, q, pos);
      if (claim != NONE32) {
        const uint32_t e = atomicAdd(b.dcount, 1u);
        b.dslot[e] = claim;
        b.dpage[e] = q;
      }
    } else {
      b.pos_page[pos] = NONE32;
    }
  }
  uint32_t sl[2], qs[2];
  int kind[2];
  const uint8_t* src[2];
  uint4 x[2];
#pragma unroll
  for (int k = 0; k < 2; k++) {
    sl[k] = __shfl_sync(0xffffffffu, claim, k);
    qs[k] = __shfl_sync(0xffffffffu, q, k);
    kind[k] = sl[k] == NONE32 ? SRC_NONE : SRC_HOST;
    src[k] = m.pages + (uint64_t)qs[k] * m.page_bytes;
    if (kind[k] != SRC_NONE && b.la_on) {
      const uint32_t pd = prev_written(b, qs[k]);
      if (pd != NONE32) {
        kind[k] = SRC_PREV;
        src[k] = b.prev_dbuf + (uint64_t)pd * m.page_bytes;
      } else {
        const uint32_t e = la_find(b, qs[k]);
        if (e != NONE32) {
          kind[k] = SRC_PLAIN;
          src[k] = b.la_buf + (uint64_t)e * m.page_bytes;
        }
      }
    }
  }
  // first 16 bytes per lane of both pages in flight before either is used;
  // without lookahead the host reads are issued before the previous-batch
  // check resolves (a page the previous batch wrote is rare)
#pragma unroll
  for (int k = 0; k < 2; k++) {
    x[k] = make_uint4(0, 0, 0, 0);
    if (kind[k] != SRC_NONE && 16 * lane < m.page_bytes)
      x[k] = *reinterpret_cast<const uint4*>(src[k] + 16 * lane);
  }
  if (!b.la_on) {
#pragma unroll
    for (int k = 0; k < 2; k++) {
      if (kind[k] == SRC_NONE) continue;
      const uint32_t pd = prev_written(b, qs[k]);
      if (pd != NONE32) {
        kind[k] = SRC_PREV;
        src[k] = b.prev_dbuf + (uint64_t)pd * m.page_bytes;
        if (16 * lane < m.page_bytes) x[k] = *reinterpret_cast<const uint4*>(src[k] + 16 * lane);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 2; k++) {
    if (kind[k] == SRC_NONE) continue;
    if (SEALED)  // k_open checks and decrypts it, a warp per page
      page_copy(m, b, sl[k], src[k], x[k], lane);
    else
      page_in<false>(m, b, sl[k], qs[k], kind[k], src[k], x[k], lane);
  }
}

// ops over at most LOOKUP_BLOCKS_PER_SM blocks per SM: a warp waiting on host
// reads holds its registers, and the next batch's preparation (one-CTA
// kernels on another stream) must still find room beside it
constexpr uint32_t LOOKUP_BLOCKS_PER_SM = 2;

template <bool SEALED>
__global__ void __launch_bounds__(256) k_lookup(MapDev m, BatchDev b, uint32_t n) {
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  // the previous batch's end counts into the peaks (a fused batch takes none
  // while it places); nothing changes a count while this kernel runs
  if (blockIdx.x == 0 && threadIdx.x == 0) stat_end_peaks(m);
  for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw)
    lookup_op<SEALED>(m, b, i, lane);
  dep_trigger();
}

// the written pages (the batch's page list), one 512-byte chunk per warp
// step: copy the ciphertexts from dbuf to the host pages (few warps: runs
// beside the next batch)
__global__ void __launch_bounds__(COPY_BLOCK) k_flush(MapDev m, BatchDev b) {
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t nch = (m.page_bytes + 511) / 512;
  const uint32_t items = *b.dcount * nch;
  for (uint32_t it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < items; it += nw) {
    const uint32_t e = it / nch, off = (it % nch) * 512 + 16 * lane;
    const uint32_t slot = b.dslot[e];
    const uint64_t q = b.dpage[e];
    if (off < m.page_bytes)
      *reinterpret_cast<uint4*>(m.pages + q * m.page_bytes + off) =
          *reinterpret_cast<const uint4*>(b.dbuf + (uint64_t)slot * m.page_bytes + off);
  }
}

__device__ __forceinline__ void ring_push(const MapDev& m, uint32_t slot) {
  unsigned long long pos = atomicAdd(m.ring_ctr + 1, 1ull);
  m.ring[pos % m.vs_cap] = slot;
}

// find_remove of op i's hit (Alg. 1 lines 6 and 9), one warp; a no-op for
// non-leaders
__device__ __forceinline__ void find_op(const MapDev& m, const BatchDev& b, uint32_t i,
                                        int lane) {
  if (b.leader[i] != i) return;
  const uint32_t slot = b.hit[i];
  if (slot == NONE32) {
    if (lane == 0) b.init_present[i] = 0;
    return;
  }
  const uint32_t meta = b.hit_meta ? b.hit_meta[i] : m.pm_meta[slot];
  const uint64_t pr = b.pair[i];
  const uint32_t which = meta_which(meta);
  const uint32_t bin = which ? (uint32_t)(pr >> 32) : (uint32_t)pr;
  uint8_t* out = b.init_val + (uint64_t)i * m.vb;
  const uint32_t nw = m.vb / 8;
  if (meta_loc(meta) == LOC_HOST) {
    const uint32_t pos = 2 * i + which;
    const uint32_t d = b.pos_page[pos] == NONE32 ? NONE32 : b.pos_slot[pos];
    if (d == NONE32) {
      if (lane == 0) set_err(m, ERR_NOTFOUND);
      return;
    }
    const uint8_t* pg = b.dbuf + (uint64_t)d * m.page_bytes;
    const uint64_t bitmap = *reinterpret_cast<const uint64_t*>(pg);
    const uint64_t key = b.keys[i];
    bool match = false;
    if (lane < (int)m.lmax && ((bitmap >> lane) & 1))
      match = *reinterpret_cast<const uint64_t*>(pg + 16 + (size_t)lane * m.rec) == key;
    const uint32_t bal = __ballot_sync(0xffffffffu, match);
    if (!bal) {
      if (lane == 0) set_err(m, ERR_NOTFOUND);
      return;
    }
    const int s = __ffs(bal) - 1;
    const uint64_t* val = reinterpret_cast<const uint64_t*>(pg + 16 + (size_t)s * m.rec + 8);
    for (uint32_t w = lane; w < nw; w += 32) reinterpret_cast<uint64_t*>(out)[w] = val[w];
    if (lane == 0) atomicOr(reinterpret_cast<unsigned long long*>(b.removed + d), 1ull << s);
  } else {
    const uint32_t vs = meta_ptr(meta);
    const uint64_t* val = reinterpret_cast<const uint64_t*>(m.vs_val + (uint64_t)vs * m.vb);
    for (uint32_t w = lane; w < nw; w += 32) reinterpret_cast<uint64_t*>(out)[w] = val[w];
    __syncwarp();
    if (lane == 0) {
      m.vs_live[vs] = 0;
      ring_push(m, vs);
      stat_leave(m, meta_loc(meta) == LOC_HBM, 1);
    }
  }
  if (lane == 0) {
    b.init_present[i] = 1;
    byte_dec(m.load, bin);
    const uint32_t lw = b.lastw[i];
    if (lw != NONE32 && b.ops[lw] == OP_DEL) {  // deleted: free the map slot
      m.pm_meta[slot] = 0;
      byte_dec(m.rowcnt, slot / m.R);
    }
  }
}

// the previous batch's page table was last read by this batch's gather:
// return the entries it used to NONE for the batch after this one
__device__ __forceinline__ void clear_prev_table(const BatchDev& b, uint32_t tid,
                                                 uint32_t nthreads) {
  if (b.clr_ht_key)
    for (uint32_t h = tid; h <= b.clr_mask; h += nthreads) {
      b.clr_ht_key[h] = NONE32;
      b.clr_ht_min[h] = NONE32;
    }
}

// warp per op: find_remove for hits
__global__ void k_find(MapDev m, BatchDev b, uint32_t n) {
  dep_wait();
  clear_prev_table(b, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
  const uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i < n) find_op(m, b, i, threadIdx.x & 31);
}

// thread per op: Get/Put/Delete semantics (Alg. 1 line 12)
// P2C decision for leader i on the round-start loads (Alg. 1 lines 13-14):
// the less loaded of its REMAP pair, and for a new key the position-map row
__device__ __forceinline__ void decide_op(const MapDev& m, const BatchDev& b, uint32_t i) {
  const uint64_t pr = b.rpair[i];
  const uint32_t p1 = (uint32_t)pr, p2 = (uint32_t)(pr >> 32);
  b.rdest[i] = byte_get(m.load, p1) <= byte_get(m.load, p2) ? p1 : p2;
  if (b.hit[i] == NONE32) {
    const uint4 rows = *reinterpret_cast<const uint4*>(b.rows + 4 * (uint64_t)i);
    const uint32_t rr[4] = {rows.x, rows.y, rows.z, rows.w};
    b.rrow[i] = pick_row(m, rr);
  }
}

__device__ __forceinline__ void exec_op(const MapDev& m, const BatchDev& b, uint32_t i) {
  const uint32_t nw = m.vb / 8;
  const uint32_t w = b.prevw[i];
  bool present;
  const uint64_t* src;
  if (w != NONE32) {
    present = b.ops[w] == OP_PUT;
    src = reinterpret_cast<const uint64_t*>(b.vin + (uint64_t)w * m.vb);
  } else {
    const uint32_t l = b.leader[i];
    present = b.init_present[l] != 0;
    src = reinterpret_cast<const uint64_t*>(b.init_val + (uint64_t)l * m.vb);
  }
  b.status[i] = present;
  uint64_t* out = reinterpret_cast<uint64_t*>(b.vout + (uint64_t)i * m.vb);
  const bool give = b.ops[i] == OP_GET && present;
  for (uint32_t k = 0; k < nw; k++) out[k] = give ? src[k] : 0;
  if (b.leader[i] == i) {
    const uint32_t lw = b.lastw[i];
    bool fp;
    const uint64_t* fs;
    if (lw != NONE32) {
      fp = b.ops[lw] == OP_PUT;
      fs = reinterpret_cast<const uint64_t*>(b.vin + (uint64_t)lw * m.vb);
    } else {
      fp = b.init_present[i] != 0;
      fs = reinterpret_cast<const uint64_t*>(b.init_val + (uint64_t)i * m.vb);
    }
    b.fpres[i] = fp;
    uint64_t* rv = reinterpret_cast<uint64_t*>(b.rval + (uint64_t)i * m.vb);
    if (fp)
      for (uint32_t k = 0; k < nw; k++) rv[k] = fs[k];
  }
}

// One warp writes back page e of the batch's page list with eviction (Alg. 1
// line 10): `plain` is this warp's page_bytes + 512 bytes of shared memory.
// The ciphertext goes to the page's slot in dbuf (the next batch reads it
// there while the host copy is in flight) and, with to_host, also straight
// to the host page.  `ks` (or null): the page's new key stream, computed
// ahead in shared memory; `poly` (or null, sealed pages): its tag's start
// state, likewise.
// (LAT: the key streams from chacha_lane16, for the latency-bound fused
// batch)
template <bool SEALED, bool LAT = false>
__device__ __forceinline__ void evict_one(const MapDev& m, const BatchDev& b, uint32_t e,
                                          uint8_t* plain, bool to_host,
                                          const uint8_t* ks = nullptr,
                                          const uint32_t* poly = nullptr) {
  const int lane = threadIdx.x & 31;
  ulonglong2* items = reinterpret_cast<ulonglong2*>(plain + m.page_bytes);
  const uint32_t d = b.dslot[e];
  const uint64_t q = b.dpage[e];
  // loads whose results are needed only later are issued first (the stores
  // below go through generic pointers, so the compiler keeps reads after them)
  const uint64_t ver = m.version[q] + 1;
  const uint8_t* old = b.dbuf + (uint64_t)d * m.page_bytes;
  const uint64_t bitmap = *reinterpret_cast<const uint64_t*>(old);
  const uint64_t removed = b.removed[d];
  // remaining page tuples (source tag: slot index) and live stash items bound
  // for this page (source tag: 1 << 31 | value-store slot)
  const bool pv = lane < (int)m.lmax && ((bitmap >> lane) & 1) && !((removed >> lane) & 1);
  // the reverse-index list is read with its count (entries past the count
  // are not used), then each listed item's live flag and key together
  const uint32_t rev_e = lane < (int)m.lmax ? m.rev[q * m.lmax + lane] : NONE32;
  const uint32_t rc = byte_get(m.revcnt, q);
  const bool listed = lane < (int)rc && lane < (int)m.lmax;
  const uint32_t vs = listed ? rev_e : NONE32;
  uint64_t skey = 0;
  uint32_t spm = 0;
  bool sv = false;
  if (listed) {
    sv = m.vs_live[vs] != 0;
    skey = m.vs_key[vs];
    spm = m.vs_pm[vs];
  }
  const uint32_t pmask = __ballot_sync(0xffffffffu, pv);
  const uint32_t smask = __ballot_sync(0xffffffffu, sv);
  const uint32_t below = (1u << lane) - 1u;
  const uint32_t np = __popc(pmask), tot = np + __popc(smask);
  if (tot > m.lmax) {  // cannot happen while every load is <= lmax
    if (lane == 0) set_err(m, ERR_PAGE);
    return;
  }
  // an evicted stash item's map entry (kept but for its location) and the
  // free ring's tail for the items' value-store slots, ahead of the page
  // build and encryption (one tail bump per warp)
  const uint32_t smeta = sv ? m.pm_meta[spm] : 0u;
  unsigned long long tail = 0;
  if (smask && lane == __ffs(smask) - 1) {
    tail = atomicAdd(m.ring_ctr + 1, (unsigned long long)__popc(smask));
    stat_leave(m, false, __popc(smask));
  }
  if (pv)
    items[__popc(pmask & below)] =
        make_ulonglong2(*reinterpret_cast<const uint64_t*>(old + 16 + (size_t)lane * m.rec), lane);
  if (sv) items[np + __popc(smask & below)] = make_ulonglong2(skey, (1ull << 31) | vs);
  __syncwarp();
  uint64_t key = ~0ull;
  uint32_t src = NONE32;
  if (lane < (int)tot) {
    key = items[lane].x;
    src = (uint32_t)items[lane].y;
  }
  warp_sort_by_key(key, src);
  for (uint32_t o = 16 * lane; o < m.page_bytes; o += 512)
    *reinterpret_cast<uint4*>(plain + o) = make_uint4(0, 0, 0, 0);
  __syncwarp();
  if (lane == 0) *reinterpret_cast<uint64_t*>(plain) = tot >= 64 ? ~0ull : ((1ull << tot) - 1);
  if (lane < (int)tot) {
    uint8_t* slot = plain + 16 + (size_t)lane * m.rec;
    *reinterpret_cast<uint64_t*>(slot) = key;
    const uint64_t* val =
        (src >> 31) ? reinterpret_cast<const uint64_t*>(m.vs_val + (uint64_t)(src & 0x7fffffffu) * m.vb)
                    : reinterpret_cast<const uint64_t*>(old + 16 + (size_t)src * m.rec + 8);
    for (uint32_t w = 0; w < m.vb / 8; w++) reinterpret_cast<uint64_t*>(slot + 8)[w] = val[w];
  }
  __syncwarp();
  // the old plaintext in dbuf is no longer read: the ciphertext replaces it
  // and k_flush copies it to the host page (or this warp does, below)
  uint8_t* cipher = b.dbuf + (uint64_t)d * m.page_bytes;
  page_encrypt_to<SEALED, LAT>(m, plain, cipher, q, ver, ks, poly);
  if (to_host)  // each lane stores the 16-byte pieces it encrypted
    for (uint32_t o = 16 * lane; o < m.page_bytes; o += 512)
      *reinterpret_cast<uint4*>(m.pages + q * m.page_bytes + o) =
          *reinterpret_cast<const uint4*>(cipher + o);
  __syncwarp();
  if (lane == 0) {
    m.version[q] = ver;
    const uint32_t sh = (uint32_t)(q & 3) * 8;
    atomicAnd(m.revcnt + (q >> 2), ~(0xffu << sh));
  }
  // evicted stash items now live in the page; their value-store slots go
  // back to the free ring
  tail = __shfl_sync(0xffffffffu, tail, smask ? __ffs(smask) - 1 : 0);
  if (sv) {
    m.pm_meta[spm] = meta_make(LOC_HOST, meta_which(smeta), 0);
    m.vs_live[vs] = 0;
    m.ring[(tail + __popc(smask & below)) % m.vs_cap] = vs;
  }
}

// warp per page of the batch (block `block` of the eviction blocks)
template <bool SEALED>
__device__ __forceinline__ void evict_page(const MapDev& m, const BatchDev& b, uint32_t block,
                                           uint8_t* sbuf) {
  const int wid = threadIdx.x >> 5;
  const uint32_t e = block * (blockDim.x >> 5) + wid;
  if (e >= *b.dcount) return;
  evict_one<SEALED>(m, b, e, sbuf + (size_t)wid * (m.page_bytes + 32 * 16), false);
}

// The first blocks run the ops' semantics (thread per op) and, when the
// batch's remap is one round, the leaders' P2C decisions; the last
// evict_blocks write the pages back (warp per page).  Exec and the decisions
// need only find_remove's results, and eviction changes no bin load or row
// count, so the two run side by side.
constexpr uint32_t EVICT_WARPS_PER_BLOCK = 4;

template <bool SEALED>
__global__ void __launch_bounds__(EVICT_WARPS_PER_BLOCK * 32)
    k_exec_evict(MapDev m, BatchDev b, uint32_t n, uint32_t evict_blocks, int decide) {
  extern __shared__ __align__(16) uint8_t sbuf[];
  dep_wait();
  const uint32_t exec_blocks = gridDim.x - evict_blocks;
  if (blockIdx.x >= exec_blocks) {
    evict_page<SEALED>(m, b, blockIdx.x - exec_blocks, sbuf);
    return;
  }
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  exec_op(m, b, i);
  if (decide && b.leader[i] == i && b.fpres[i]) decide_op(m, b, i);
}

// P2C remap, decide on round-start loads (Alg. 1 lines 13-14)
__global__ void k_remap_decide(MapDev m, BatchDev b, uint32_t lo, uint32_t hi) {
  const uint32_t i = lo + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= hi || b.leader[i] != i || !b.fpres[i]) return;
  decide_op(m, b, i);
}

// place leader i in its new bin: a value-store slot from the ring, the
// position-map entry (a free slot of the chosen row for a new key), and the
// reverse-index entry for a stash item; the counts are already bumped
// One counter hands out ring positions to every lane of the warp that places
// an item (one atomic per warp): returns this lane's position, or ~0 when the
// lane does not take one.  All 32 lanes must call it.
// A fused batch's view of its map's free ring: the head and tail as the
// batch found them and the entries from the head on, read while its host
// pages are in flight.  Only the batch's own remap takes from the ring while
// it runs (one warp, round after round) and its find_remove and eviction only
// append past the tail, so the head moves only by the takes counted here and
// the entries in the window do not change.
constexpr uint32_t RING_WIN = 32;
struct RingWin {
  unsigned long long head, tail, taken;
  uint32_t v[RING_WIN];
};

__device__ __forceinline__ unsigned long long ring_take(const MapDev& m, bool take,
                                                        RingWin* w = nullptr) {
  const uint32_t mask = __ballot_sync(0xffffffffu, take);
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (w) {
    // positions from the window's count; the shared head still moves (its
    // result is not waited for: an atomic at the end of the batch would
    // hold up the kernel's completion instead)
    base = w->head + w->taken;
    __syncwarp();
    if (mask && lane == __ffs(mask) - 1) {
      w->taken += __popc(mask);
      atomicAdd(m.ring_ctr, (unsigned long long)__popc(mask));
    }
    __syncwarp();
  } else {
    if (mask && lane == __ffs(mask) - 1)
      base = atomicAdd(m.ring_ctr, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, mask ? __ffs(mask) - 1 : 0);
  }
  return take ? base + __popc(mask & ((1u << lane) - 1u)) : ~0ull;
}

// (rev_slot: the entry of the destination page's reverse-index list this
// item takes, already counted; NONE32 to count it here)
__device__ __forceinline__ void remap_place(const MapDev& m, const BatchDev& b, uint32_t i,
                                            uint32_t dest, unsigned long long pos,
                                            uint32_t rev_slot = NONE32,
                                            const RingWin* w = nullptr) {
  const uint64_t pr = b.rpair[i];
  const uint32_t which = dest == (uint32_t)(pr >> 32) ? 1u : 0u;
  uint32_t vs;
  if (w && pos < w->tail && pos - w->head < RING_WIN) {
    vs = w->v[pos - w->head];
  } else {
    if (pos >= m.ring_ctr[1]) {
      set_err(m, ERR_VS);
      return;
    }
    vs = m.ring[pos % m.vs_cap];
  }
  const bool hbm = dest < m.K;
  const uint32_t meta = meta_make(hbm ? LOC_HBM : LOC_STASH, which, vs);
  uint32_t slot = b.hit[i];
  const uint64_t key = b.keys[i];
  if (slot == NONE32) {
    const uint32_t row = b.rrow[i];
    for (uint32_t s = 0; s < m.R; s++) {
      const uint64_t idx = (uint64_t)row * m.R + s;
      if (atomicCAS(m.pm_meta + idx, 0u, meta) == 0u) {
        slot = (uint32_t)idx;
        break;
      }
    }
    if (slot == NONE32) {
      set_err(m, ERR_ROW);
      return;
    }
    m.pm_key[slot] = key;
  } else {
    m.pm_meta[slot] = meta;
  }
  m.pm_bins[slot] = pr;
  m.vs_key[vs] = key;
  const uint64_t* src = reinterpret_cast<const uint64_t*>(b.rval + (uint64_t)i * m.vb);
  uint64_t* dst = reinterpret_cast<uint64_t*>(m.vs_val + (uint64_t)vs * m.vb);
  for (uint32_t w = 0; w < m.vb / 8; w++) dst[w] = src[w];
  m.vs_pm[vs] = slot;
  m.vs_live[vs] = 1;
  if (!hbm) {
    const uint64_t q = dest - m.K;
    const uint32_t r = rev_slot != NONE32 ? rev_slot : byte_inc(m.revcnt, q);
    if (r >= m.lmax) {
      set_err(m, ERR_REV);
      return;
    }
    m.rev[q * m.lmax + r] = vs;
  }
}

// What a placement's counter atomics would return, known beforehand: the
// bin's new load, the row's count before it (a new key) and the reverse-index
// entry it takes (a host bin).
struct PlaceCounts {
  uint32_t load, row, rev;
};

// place op i if `go` (a leader whose key is present after the batch, in the
// current round): bump the counts of its decided bin (and row, for a new
// key), take a ring slot, write its entries.  All 32 lanes of the warp call.
// With `known`, the counts are bumped by atomics nothing waits for.
__device__ __forceinline__ void remap_apply_op(const MapDev& m, const BatchDev& b, uint32_t i,
                                               bool go, RingWin* w = nullptr,
                                               bool peaks = true,
                                               const PlaceCounts* known = nullptr) {
  // the bin's load, the row's count (a new key), the destination page's
  // reverse-index count (a host bin) and the free-ring position are taken
  // together (independent atomics in flight at once), then checked; a count
  // that ran over poisons the map (Sec. 3.3), so what else was taken then no
  // longer matters
  uint32_t dest = 0, new_load = 0, row_old = 0, rev_slot = NONE32;
  bool fresh = false;
  if (go) {
    dest = b.rdest[i];
    fresh = b.hit[i] == NONE32;
    if (known) {
      byte_add(m.load, dest);
      new_load = known->load;
      if (fresh) {
        byte_add(m.rowcnt, b.rrow[i]);
        row_old = known->row;
      }
      if (dest >= m.K) {
        byte_add(m.revcnt, dest - m.K);
        rev_slot = known->rev;
      }
    } else {
      new_load = byte_inc(m.load, dest) + 1;
      if (fresh) row_old = byte_inc(m.rowcnt, b.rrow[i]);
      if (dest >= m.K) rev_slot = byte_inc(m.revcnt, dest - m.K);
    }
  }
  const unsigned long long pos = ring_take(m, go, w);
  if (go) {
    if (new_load > m.lmax) {
      set_err(m, ERR_LOAD);
      go = false;
    } else if (fresh && row_old + 1 > m.R) {
      set_err(m, ERR_ROW);
      go = false;
    }
  }
  if (go) remap_place(m, b, i, dest, pos, rev_slot, w);
  stat_place(m, go, dest < m.K, new_load, peaks);
}

__global__ void k_remap_apply(MapDev m, BatchDev b, uint32_t lo, uint32_t hi) {
  dep_wait();
  const uint32_t i = lo + blockIdx.x * blockDim.x + threadIdx.x;
  remap_apply_op(m, b, i, i < hi && b.leader[i] == i && b.fpres[i]);
}

// Small maps (B <= 2^17 bins, <= 2^16 rows): every P2C round of the batch in
// one CTA, on shared-memory copies of the bin loads and row counts (same
// round-start decisions and counts as the launch-per-round path); the
// placement work then runs in parallel in k_remap_rest.
constexpr uint32_t REMAP_SMEM_MAX_BINS = 1u << 17;
constexpr uint32_t REMAP_SMEM_MAX_ROWS = 1u << 16;

__device__ __forceinline__ uint32_t sbyte_get(const uint32_t* w, uint32_t i) {
  return (w[i >> 2] >> ((i & 3) * 8)) & 0xffu;
}
__device__ __forceinline__ uint32_t sbyte_inc(uint32_t* w, uint32_t i) {
  const uint32_t sh = (i & 3) * 8;
  return (atomicAdd(w + (i >> 2), 1u << sh) >> sh) & 0xffu;
}

__global__ void __launch_bounds__(1024) k_remap_smem(MapDev m, BatchDev b, uint32_t n) {
  extern __shared__ uint32_t rsm[];
  const uint32_t lw = (uint32_t)(m.B + 3) / 4, rw = (uint32_t)(m.rows + 3) / 4;
  uint32_t* sload = rsm;
  uint32_t* srow = rsm + lw;
  for (uint32_t w = threadIdx.x; w < lw; w += blockDim.x) sload[w] = m.load[w];
  for (uint32_t w = threadIdx.x; w < rw; w += blockDim.x) srow[w] = m.rowcnt[w];
  __syncthreads();
  uint32_t err = 0;
  for (uint64_t lo = 0; lo < n; lo += m.Wr) {
    const uint32_t hi = (uint32_t)(lo + m.Wr < n ? lo + m.Wr : n);
    for (uint32_t i = (uint32_t)lo + threadIdx.x; i < hi; i += blockDim.x) {
      if (b.leader[i] != i || !b.fpres[i]) continue;
      const uint64_t pr = b.rpair[i];
      const uint32_t p1 = (uint32_t)pr, p2 = (uint32_t)(pr >> 32);
      b.rdest[i] = sbyte_get(sload, p1) <= sbyte_get(sload, p2) ? p1 : p2;
      if (b.hit[i] == NONE32) {
        const uint4 r4 = *reinterpret_cast<const uint4*>(b.rows + 4 * (uint64_t)i);
        const uint32_t rows[4] = {r4.x, r4.y, r4.z, r4.w};
        uint32_t best = rows[0], bc = sbyte_get(srow, rows[0]);
#pragma unroll
        for (int j = 1; j < 4; j++) {
          const uint32_t c = sbyte_get(srow, rows[j]);
          if (c < bc) {
            best = rows[j];
            bc = c;
          }
        }
        b.rrow[i] = best;
      }
    }
    __syncthreads();
    for (uint32_t i = (uint32_t)lo + threadIdx.x; i < hi; i += blockDim.x) {
      if (b.leader[i] != i || !b.fpres[i]) continue;
      if (sbyte_inc(sload, b.rdest[i]) + 1 > m.lmax) err |= ERR_LOAD;
      if (b.hit[i] == NONE32 && sbyte_inc(srow, b.rrow[i]) + 1 > m.R) err |= ERR_ROW;
    }
    __syncthreads();
  }
  if (err) set_err(m, err);
  // peak load: a bin's final load is the value its last placement reached
  uint32_t top = 0;
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x)
    if (b.leader[i] == i && b.fpres[i]) top = max(top, sbyte_get(sload, b.rdest[i]));
  top = __reduce_max_sync(0xffffffffu, top);
  if ((threadIdx.x & 31) == 0 && top) atomicMax(m.stat + ST_PEAK_LOAD, (unsigned long long)top);
  for (uint32_t w = threadIdx.x; w < lw; w += blockDim.x) m.load[w] = sload[w];
  for (uint32_t w = threadIdx.x; w < rw; w += blockDim.x) m.rowcnt[w] = srow[w];
}

// Batches of at most 4 x 1024 ops: every thread loads its (up to) four ops
// into registers once, so a round costs two barriers and shared-memory work
// only (the rounds of a small map are many and short).
constexpr int REMAP_REG_OPS = 4;

__global__ void __launch_bounds__(1024) k_remap_smem_reg(MapDev m, BatchDev b, uint32_t n) {
  extern __shared__ uint32_t rsm[];
  const uint32_t lw = (uint32_t)(m.B + 3) / 4, rw = (uint32_t)(m.rows + 3) / 4;
  uint32_t* sload = rsm;
  uint32_t* srow = rsm + lw;
  for (uint32_t w = threadIdx.x; w < lw; w += blockDim.x) sload[w] = m.load[w];
  for (uint32_t w = threadIdx.x; w < rw; w += blockDim.x) srow[w] = m.rowcnt[w];
  uint32_t op[REMAP_REG_OPS], p1[REMAP_REG_OPS], p2[REMAP_REG_OPS], dest[REMAP_REG_OPS];
  uint4 rows[REMAP_REG_OPS];
  uint32_t row[REMAP_REG_OPS];
  bool act[REMAP_REG_OPS], fresh[REMAP_REG_OPS];
#pragma unroll
  for (int k = 0; k < REMAP_REG_OPS; k++) {
    op[k] = threadIdx.x + k * blockDim.x;
    act[k] = op[k] < n && b.leader[op[k]] == op[k] && b.fpres[op[k]];
    fresh[k] = false;
    dest[k] = row[k] = 0;
    if (act[k]) {
      const uint64_t pr = b.rpair[op[k]];
      p1[k] = (uint32_t)pr;
      p2[k] = (uint32_t)(pr >> 32);
      fresh[k] = b.hit[op[k]] == NONE32;
      if (fresh[k]) rows[k] = *reinterpret_cast<const uint4*>(b.rows + 4 * (uint64_t)op[k]);
    }
  }
  __syncthreads();
  uint32_t err = 0;
  for (uint64_t lo = 0; lo < n; lo += m.Wr) {
    const uint64_t hi = lo + m.Wr;
#pragma unroll
    for (int k = 0; k < REMAP_REG_OPS; k++) {
      if (!act[k] || op[k] < lo || op[k] >= hi) continue;
      dest[k] = sbyte_get(sload, p1[k]) <= sbyte_get(sload, p2[k]) ? p1[k] : p2[k];
      if (fresh[k]) {
        const uint32_t rr[4] = {rows[k].x, rows[k].y, rows[k].z, rows[k].w};
        uint32_t best = rr[0], bc = sbyte_get(srow, rr[0]);
#pragma unroll
        for (int j = 1; j < 4; j++) {
          const uint32_t c = sbyte_get(srow, rr[j]);
          if (c < bc) {
            best = rr[j];
            bc = c;
          }
        }
        row[k] = best;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < REMAP_REG_OPS; k++) {
      if (!act[k] || op[k] < lo || op[k] >= hi) continue;
      if (sbyte_inc(sload, dest[k]) + 1 > m.lmax) err |= ERR_LOAD;
      if (fresh[k] && sbyte_inc(srow, row[k]) + 1 > m.R) err |= ERR_ROW;
    }
    __syncthreads();
  }
  if (err) set_err(m, err);
  uint32_t top = 0;
#pragma unroll
  for (int k = 0; k < REMAP_REG_OPS; k++)
    if (act[k]) {
      b.rdest[op[k]] = dest[k];
      if (fresh[k]) b.rrow[op[k]] = row[k];
      top = max(top, sbyte_get(sload, dest[k]));  // final load of the bin (peak)
    }
  top = __reduce_max_sync(0xffffffffu, top);
  if ((threadIdx.x & 31) == 0 && top) atomicMax(m.stat + ST_PEAK_LOAD, (unsigned long long)top);
  for (uint32_t w = threadIdx.x; w < lw; w += blockDim.x) m.load[w] = sload[w];
  for (uint32_t w = threadIdx.x; w < rw; w += blockDim.x) m.rowcnt[w] = srow[w];
}

__global__ void k_remap_rest(MapDev m, BatchDev b, uint32_t n) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool go = i < n && b.leader[i] == i && b.fpres[i];
  const uint32_t dest = go ? b.rdest[i] : 0;
  const unsigned long long pos = ring_take(m, go);
  if (go) remap_place(m, b, i, dest, pos);
  // the loads were raised in k_remap_smem(_reg), which took their peak
  stat_place(m, go, dest < m.K, 0);
}

__global__ void k_clear_keys(BatchDev b, uint32_t n) {
  for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h <= b.kt_mask;
       h += gridDim.x * blockDim.x) {
    b.kt_own[h] = 0;
    if (h < n) b.pres[h] = 2;
  }
}


// ---------------------------------------------------------------------------
// Small batches in one CTA.  A batch of at most FUSED_MAX_OPS operations (a
// batch of one is Alg. 1 for one command) runs every step of the chain above
// in a single launch, with block barriers where the chain has kernel
// boundaries: the same device functions on the same tables and buffers, so
// the same results, pages and trace.  Its written pages go to the host from
// this kernel (no separate write-back launch): a caller issuing one
// operation at a time pays one launch per operation.  The kernel is bound by
// dependent round trips (the host page, the position map and counters in
// L2), so it starts everything it can early: the host pages' prefetch as
// soon as the search has a pair, the write-back's key streams and tag keys
// and the remap's counts in spare warps during the host read.
constexpr uint32_t FUSED_THREADS = 512;
// the page table of a batch of <= FUSED_MAX_OPS ops: 4 x 2^ceil(log2 n)
// entries, at least 256 (the runtime's sizing)
constexpr uint32_t FUSED_TABLE = 256;
static_assert(4 * FUSED_MAX_OPS <= FUSED_TABLE, "a small batch's page table fits the shared copy");

// the P2C decision of op i on round-start counts read from L2: the counts
// change by atomics between the rounds of this one launch
// (every count it needs is read at once: one round trip)
__device__ __forceinline__ void decide_op_l2(const MapDev& m, const BatchDev& b, uint32_t i) {
  auto get = [](const uint32_t* w, uint64_t k) {
    return (__ldcg(w + (k >> 2)) >> ((uint32_t)(k & 3) * 8)) & 0xffu;
  };
  const uint64_t pr = b.rpair[i];
  const uint32_t p1 = (uint32_t)pr, p2 = (uint32_t)(pr >> 32);
  const bool fresh = b.hit[i] == NONE32;
  const uint4 r4 = *reinterpret_cast<const uint4*>(b.rows + 4 * (uint64_t)i);
  const uint32_t rr[4] = {r4.x, r4.y, r4.z, r4.w};
  const uint32_t l1 = get(m.load, p1), l2 = get(m.load, p2);
  uint32_t rc[4] = {0, 0, 0, 0};
  if (fresh) {
#pragma unroll
    for (int j = 0; j < 4; j++) rc[j] = get(m.rowcnt, rr[j]);
  }
  b.rdest[i] = l1 <= l2 ? p1 : p2;
  if (fresh) {
    uint32_t best = rr[0], bc = rc[0];
#pragma unroll
    for (int j = 1; j < 4; j++)
      if (rc[j] < bc) {
        best = rr[j];
        bc = rc[j];
      }
    b.rrow[i] = best;
  }
}

// largest value the fused launch stages in shared memory (the ABI's limit)
constexpr uint32_t FUSED_VB_MAX = 504;

// ONE: compiled for batches of a single op (n = 1 folded into the code,
// which shrinks what a cold SM fetches)
template <bool SEALED, bool ONE>
__global__ void __launch_bounds__(FUSED_THREADS, 1)
    k_fused(MapDev m, BatchDev b, uint32_t n_arg, uint64_t t0, uint32_t evict_warps,
            uint32_t early_in, uint32_t ks_slots, const __grid_constant__ FusedInline inl) {
  const uint32_t n = ONE ? 1u : n_arg;
  extern __shared__ __align__(16) uint8_t sbuf[];
  // Everything the batch reads back within itself lives in shared memory:
  // the inputs, the grouping, pairs, rows, hits, the page table and its read
  // positions, the found and re-placed values.  The shared helpers reach it
  // through `L`, a copy of the batch descriptor whose pointers address these
  // arrays (generic addressing), so a batch pays a memory round trip only for
  // map state, pages and outputs.  The page buffers (dbuf), the global page
  // table keys (read by the next batch) and the outputs stay in global memory.
  __shared__ __align__(16) uint8_t s_in[FUSED_MAX_OPS * (9 + FUSED_VB_MAX) + 16];
  __shared__ __align__(16) uint8_t s_vals[2 * FUSED_MAX_OPS * FUSED_VB_MAX];
  __shared__ uint64_t s_pair[FUSED_MAX_OPS], s_rpair[FUSED_MAX_OPS], s_removed[FUSED_TABLE];
  __shared__ __align__(16) uint32_t s_rows[4 * FUSED_MAX_OPS];
  __shared__ uint32_t s_hit[FUSED_MAX_OPS], s_hmeta[FUSED_MAX_OPS], s_leader[FUSED_MAX_OPS],
      s_prevw[FUSED_MAX_OPS], s_lastw[FUSED_MAX_OPS], s_rdest[FUSED_MAX_OPS],
      s_rrow[FUSED_MAX_OPS];
  __shared__ uint32_t s_posq[2 * FUSED_MAX_OPS], s_slot[2 * FUSED_MAX_OPS],
      s_dslot[2 * FUSED_MAX_OPS], s_dpage[2 * FUSED_MAX_OPS];
  __shared__ uint32_t s_ht[FUSED_TABLE], s_htmin[FUSED_TABLE], s_dcount;
  __shared__ uint8_t s_initp[FUSED_MAX_OPS], s_fpres[FUSED_MAX_OPS], s_defer[FUSED_MAX_OPS];
  // a one-round remap's counts as read during the page reads: the REMAP
  // pair's two loads and two reverse-index counts, a new key's four row counts
  __shared__ uint8_t s_cnt[8][FUSED_MAX_OPS];
  // (sealed) the write-back tags' start states (batches of at most 7 pages;
  // wider ones derive them in the eviction) and the pages whose tag failed
  __shared__ uint32_t s_poly[SEALED ? 7 : 1][POLY_WORDS];
  __shared__ unsigned long long s_bad;
  __shared__ RingWin s_ring;
  static_assert(RING_WIN >= FUSED_MAX_OPS, "the remap's takes fit the ring window");
  const int lane = threadIdx.x & 31;
  const uint32_t wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  BatchDev L = b;
  L.keys = reinterpret_cast<uint64_t*>(s_in);
  L.vin = s_in + 8 * n;
  L.ops = s_in + (8 + m.vb) * n;
  L.pair = s_pair; L.rpair = s_rpair; L.rows = s_rows;
  L.hit = s_hit; L.hit_meta = s_hmeta;
  L.leader = s_leader; L.prevw = s_prevw; L.lastw = s_lastw;
  L.pos_page = s_posq; L.pos_slot = s_slot; L.ht_min = s_htmin;
  L.removed = s_removed; L.dslot = s_dslot; L.dpage = s_dpage; L.dcount = &s_dcount;
  L.init_val = s_vals; L.rval = s_vals + FUSED_MAX_OPS * FUSED_VB_MAX;
  L.init_present = s_initp; L.fpres = s_fpres; L.rdest = s_rdest; L.rrow = s_rrow;
  // Launched as a programmatic dependent of the previous kernel on the
  // stream: it may start while that kernel runs, and passes dep_wait() before
  // it touches anything another kernel writes.  Before the wait it computes
  // what depends only on its own parameters (the DUMMY and REMAP pairs) and,
  // with early_in, also stages its inputs, the position-map rows and the
  // grouping (the caller guarantees the inputs are complete: host staging
  // written before the launch, or a batch whose predecessor is an earlier
  // batch of the same call).  It lets its successor start only after its own
  // wait, so a successor never runs ahead of this kernel's predecessor.
  for (uint32_t h = threadIdx.x; h < FUSED_TABLE; h += blockDim.x) {
    s_ht[h] = NONE32;
    s_htmin[h] = NONE32;
  }
  if (threadIdx.x == 0) {
    s_dcount = 0;
    s_bad = 0;
  }
  // 1a. per op the DUMMY pair and the REMAP pair (one ChaCha20 block each,
  //     each kind in a warp of its own, lane = op)
  auto pairs = [&]() {
    if (wid < 2 && (uint32_t)lane < n) {
      const uint32_t i = lane;
      uint32_t p1, p2;
      prf_pair(m, wid == 0 ? DOM_DUMMY : DOM_REMAP, t0 + i, p1, p2);
      const uint64_t pr = (uint64_t)p1 | ((uint64_t)p2 << 32);
      if (wid == 0) {
        s_pair[i] = pr;
      } else {
        s_rpair[i] = pr;
        // the remap will read these loads (an address only: nothing is read)
        prefetch_l2(m.load + (p1 >> 2));
        prefetch_l2(m.load + (p2 >> 2));
      }
    }
  };
  // 0. the inputs, laid out keys | vin | ops: from the launch's parameters,
  //    straight from the caller's pinned staging (16-byte reads over the
  //    link; the staging holds the rounded-up tail), or from the device
  //    arrays; then (1b) per op the position-map rows (one ChaCha20 block,
  //    warp 2, lane = op) and the grouping (warp 3, n^2 compares: leader =
  //    first op on the key, previous writer of each op, last writer of each
  //    key group)
  auto inputs = [&]() {
    if (inl.bytes) {
      for (uint32_t w = threadIdx.x; w < (inl.bytes + 15) / 16; w += blockDim.x)
        reinterpret_cast<uint4*>(s_in)[w] = inl.d[w];
    } else if (b.h_in) {
      const uint32_t words = (n * (9 + m.vb) + 15) / 16;
      for (uint32_t w = threadIdx.x; w < words; w += blockDim.x)
        reinterpret_cast<uint4*>(s_in)[w] = reinterpret_cast<const uint4*>(b.h_in)[w];
    } else {
      const uint32_t vw = n * m.vb / 8;
      for (uint32_t w = threadIdx.x; w < n + vw + n; w += blockDim.x) {
        if (w < n)
          L.keys[w] = b.keys[w];
        else if (w < n + vw)
          reinterpret_cast<uint64_t*>(L.vin)[w - n] =
              reinterpret_cast<const uint64_t*>(b.vin)[w - n];
        else
          L.ops[w - n - vw] = b.ops[w - n - vw];
      }
    }
  };
  auto rows_group = [&]() {
    if (wid == 2 && (uint32_t)lane < n) {
      const uint32_t i = lane;
      uint32_t rows[4];
      prf_rows(m, L.keys[i], rows);
      *reinterpret_cast<uint4*>(s_rows + 4 * i) = make_uint4(rows[0], rows[1], rows[2], rows[3]);
#pragma unroll
      for (int j = 0; j < 4; j++) {
        prefetch_l2(m.rowcnt + (rows[j] >> 2));
        // the rows the search reads (before the wait too: a line the
        // previous kernel then writes is updated in L2 like any other)
        const uint64_t at = (uint64_t)rows[j] * m.R;
        prefetch_range_l2(m.pm_meta + at, 4 * m.R);
        prefetch_range_l2(m.pm_key + at, 8 * m.R);
        prefetch_range_l2(m.pm_bins + at, 8 * m.R);
      }
    }
    if (wid == 3) {
      const bool mine = (uint32_t)lane < n;
      const uint64_t key = mine ? L.keys[lane] : 0;
      const uint32_t op = mine ? L.ops[lane] : OP_GET;
      uint32_t lead = lane, prevw = NONE32, lastw = NONE32;
      for (uint32_t j = 0; j < n; j++) {
        const uint64_t kj = __shfl_sync(0xffffffffu, key, j);
        const uint32_t oj = __shfl_sync(0xffffffffu, op, j);
        if (!mine || kj != key) continue;
        if (j < (uint32_t)lane) {
          lead = min(lead, j);
          if (oj != OP_GET) prevw = j;
        } else if (oj != OP_GET) {
          lastw = j;
        }
      }
      if (mine) {
        s_leader[lane] = lead;
        s_prevw[lane] = prevw;
        s_lastw[lane] = lastw;
      }
    }
  };
  // (with early_in the pairs, the rows and the grouping run side by side,
  // after the inputs)
  if (early_in) {
    inputs();
    __syncthreads();
    pairs();
    rows_group();
  } else {
    pairs();
  }
  dep_wait();
  dep_trigger();
  if (!early_in) {
    inputs();
    __syncthreads();
    rows_group();
  }
  __syncthreads();
  // 2. position-map search (warp per op): a hit reads its stored pair, every
  //    other op its DUMMY pair; the host bins of each read position.  A hit
  //    in the HBM store or the stash has its value brought into L2 for
  //    find_remove.
  for (uint32_t i = wid; i < n; i += nwarps) {
    uint32_t found = NONE32, fm = 0;
    uint64_t fb = 0;
    if (s_leader[i] == i) found = pm_search(m, L, i, L.keys[i], lane, &fb, &fm);
    const uint64_t pr = found != NONE32 ? fb : s_pair[i];
    if (lane < 2) {
      // the op's host pages into L2 now, exactly their bytes: the reads in
      // 2c start only after the page table is built
      const uint32_t p = lane == 0 ? (uint32_t)pr : (uint32_t)(pr >> 32);
      if (p >= m.K) prefetch_bulk_l2(m.pages + (uint64_t)(p - m.K) * m.page_bytes, m.page_bytes);
    }
    if (lane == 0) {
      s_hit[i] = found;
      s_hmeta[i] = fm;
      s_pair[i] = pr;
      if (found != NONE32 && meta_loc(fm) != LOC_HOST)
        prefetch_l2(m.vs_val + (uint64_t)meta_ptr(fm) * m.vb);
    }
    if (lane < 2) {
      const uint32_t p = lane == 0 ? (uint32_t)pr : (uint32_t)(pr >> 32);
      s_posq[2 * i + lane] = p >= m.K ? (uint32_t)(p - m.K) : NONE32;
    }
  }
  __syncthreads();
  // 2b. warp 0: the batch's page table -- each distinct page once, at the
  //     slot linear probing gives it, its first read position, the page
  //     list in claim order; the table's keys also go to the global table,
  //     where the next batch looks for pages this one wrote.  Every read
  //     position finds or claims its page's slot at once (lane per
  //     position), and the smallest position on a slot is the page's first.
  if (wid == 0) {
    const uint32_t np = 2 * n;
    uint32_t q[2], hs[2];
    bool valid[2];
#pragma unroll
    for (int k = 0; k < 2; k++) {
      const uint32_t p = lane + 32 * k;
      q[k] = p < np ? s_posq[p] : NONE32;
      valid[k] = q[k] != NONE32;
      hs[k] = 0;
      if (valid[k]) {
        uint32_t h = ht_hash(q[k], b.ht_mask);
        for (uint32_t probe = 0; probe <= b.ht_mask; probe++) {
          const uint32_t prev = atomicCAS(&s_ht[h], NONE32, q[k]);
          if (prev == NONE32 || prev == q[k]) break;
          h = (h + 1) & b.ht_mask;
        }
        hs[k] = h;
        s_slot[p] = h;
        atomicMin(&s_htmin[h], p);
      }
    }
    __syncwarp();
    bool first[2];
#pragma unroll
    for (int k = 0; k < 2; k++) first[k] = valid[k] && s_htmin[hs[k]] == lane + 32u * k;
    const uint32_t below = (1u << lane) - 1u;
    const uint32_t bf0 = __ballot_sync(0xffffffffu, first[0]);
    const uint32_t bf1 = __ballot_sync(0xffffffffu, first[1]);
#pragma unroll
    for (int k = 0; k < 2; k++)
      if (first[k]) {
        const uint32_t d = k == 0 ? __popc(bf0 & below) : __popc(bf0) + __popc(bf1 & below);
        b.ht_key[hs[k]] = q[k];
        s_dslot[d] = hs[k];
        s_dpage[d] = q[k];
      }
    if (lane == 0) s_dcount = __popc(bf0) + __popc(bf1);
  }
  __syncthreads();
  // 2c. read each distinct page (the previous batch's ciphertext if that
  //     batch wrote it, else the host page) and decrypt it into its slot's
  //     buffer, a warp per 512-byte chunk (the chunks' ChaCha20 blocks side
  //     by side; a one-op batch, whose few warps wait on them, takes each
  //     block from chacha_lane16); meanwhile bring each page's eviction data
  //     into L2.  A
  //     sealed page's tag is checked beside its decryption by a warp of its
  //     own (one Poly1305 over the page); a page that fails it is emptied
  //     after the phase.  The last warp first reads the free ring's window
  //     for the remap.
  if (wid == nwarps - 1) {
    // (the previous batch's end counts into the peaks: this batch's
    // placements take none)
    if (lane == 1) stat_end_peaks(m);
    const unsigned long long hd = m.ring_ctr[0], tl = m.ring_ctr[1];
    if (lane < (int)RING_WIN && hd + lane < tl) s_ring.v[lane] = m.ring[(hd + lane) % m.vs_cap];
    if (lane == 0) {
      s_ring.head = hd;
      s_ring.tail = tl;
      s_ring.taken = 0;
    }
  }
  {
    const uint32_t nd = s_dcount, nch = (m.page_bytes + 511) / 512, reads = nd * nch;
    const uint32_t Lc = m.page_bytes - (SEALED ? 16u : 0u);  // the ciphertext's bytes
    // where page d's bytes come from: the previous batch's ciphertext if that
    // batch wrote it (its host copy may still be in flight), else the host page
    auto source = [&](uint32_t q) {
      const uint32_t pd = prev_written(b, q);
      return pd != NONE32 ? b.prev_dbuf + (uint64_t)pd * m.page_bytes
                          : m.pages + (uint64_t)q * m.page_bytes;
    };
    // (a warp's items in groups of up to 4: every item's host load and page
    // version are issued before the first one is decrypted; a one-op batch's
    // reads fit one item per warp)
    constexpr uint32_t GRP = ONE ? 1 : 4;
    for (uint32_t base = wid; base < reads; base += GRP * nwarps) {
      uint4 xs[GRP];
      uint64_t vs[GRP];
#pragma unroll
      for (uint32_t g = 0; g < GRP; g++) {
        const uint32_t it = base + g * nwarps;
        xs[g] = make_uint4(0, 0, 0, 0);
        vs[g] = 0;
        if (it < reads) {
          const uint32_t d = it / nch, c = it % nch, off = 512 * c + 16 * lane;
          const uint32_t q = s_dpage[d];
          if (off < m.page_bytes)
            xs[g] = *reinterpret_cast<const uint4*>(m.pages + (uint64_t)q * m.page_bytes + off);
          vs[g] = m.version[q];
          if (c == 0) prefetch_eviction(m, q, true, lane);
        }
      }
      // each item: its bytes (the previous batch's ciphertext instead when
      // that batch wrote the page), decrypted into its slot's buffer; a
      // warp's items two by two, their ChaCha20 blocks side by side
      auto bytes_of = [&](uint32_t g) {
        const uint32_t it = base + g * nwarps, d = it / nch, c = it % nch;
        const uint32_t off = 512 * c + 16 * lane, q = s_dpage[d];
        uint4 x = xs[g];
        const uint8_t* at = source(q);
        if (at != m.pages + (uint64_t)q * m.page_bytes && off < m.page_bytes)
          x = *reinterpret_cast<const uint4*>(at + off);
        return x;
      };
      auto put = [&](uint32_t g, uint4 x, uint4 k4) {
        const uint32_t it = base + g * nwarps, d = it / nch, c = it % nch;
        const uint32_t off = 512 * c + 16 * lane, h = s_dslot[d];
        x.x ^= k4.x; x.y ^= k4.y; x.z ^= k4.z; x.w ^= k4.w;
        if (off < Lc)
          *reinterpret_cast<uint4*>(L.dbuf + (uint64_t)h * m.page_bytes + off) = x;
        else if (off < m.page_bytes)
          *reinterpret_cast<uint4*>(L.dbuf + (uint64_t)h * m.page_bytes + off) =
              make_uint4(0, 0, 0, 0);
        if (c == 0 && lane == 0) L.removed[h] = 0;
      };
      auto ctr_of = [&](uint32_t g) {
        return 8 * ((base + g * nwarps) % nch) + (lane >> 2) + (SEALED ? 1u : 0u);
      };
      auto page_of = [&](uint32_t g) { return s_dpage[(base + g * nwarps) / nch]; };
#pragma unroll
      for (uint32_t g = 0; g < GRP; g += 2) {
        if (base + g * nwarps >= reads) break;
        const uint4 x0 = bytes_of(g);
        const uint64_t v0 = vs[g];
        if (GRP > 1 && base + (g + 1) * nwarps < reads) {
          const uint4 x1 = bytes_of(g + 1);
          const uint64_t v1 = vs[g + 1];
          uint4 k0, k1;
          chacha_quad2(m.kenc, ctr_of(g), page_of(g), (uint32_t)v0, (uint32_t)(v0 >> 32),
                       ctr_of(g + 1), page_of(g + 1), (uint32_t)v1, (uint32_t)(v1 >> 32), k0,
                       k1);
          put(g, x0, k0);
          put(g + 1, x1, k1);
        } else {
          put(g, x0, (ONE ? chacha_lane16 : chacha_quad)(m.kenc, ctr_of(g), page_of(g),
                                                          (uint32_t)v0, (uint32_t)(v0 >> 32)));
        }
      }
    }
    // meanwhile the warps after those: (sealed) a warp per page checks its
    // tag; each page's key stream for its write-back (version + 1), a warp
    // per chunk, into the key-stream region after the eviction buffers (room
    // for ks_slots pages), which the eviction of page d then only XORs;
    // (sealed, at most 7 pages) a warp per page computes that write-back's
    // tag start state.  The write-back's ChaCha20 (and Poly1305 key) leave
    // the eviction's path.
    const bool ks_pre = nd <= ks_slots;
    uint8_t* const ks_base = sbuf + (size_t)evict_warps * (m.page_bytes + 32 * 16);
    const uint32_t n_chk = SEALED ? nd : 0u, n_ks = ks_pre ? nd * nch : 0u;
    const uint32_t n_pk = SEALED && ks_pre && nd <= 7 ? nd : 0u;
    for (uint32_t t = (wid + nwarps - reads % nwarps) % nwarps; t < n_chk + n_ks + n_pk;
         t += nwarps) {
      if (SEALED && t < n_chk) {
        const uint32_t d = t, q = s_dpage[d];
        const uint8_t* at = source(q);
        uint4 x = make_uint4(0, 0, 0, 0);
        if (16 * lane < m.page_bytes) x = *reinterpret_cast<const uint4*>(at + 16 * lane);
        PolyWarp pw = poly_begin<ONE>(m, q, m.version[q]);
        uint4 stored = make_uint4(0, 0, 0, 0);
        for (uint32_t c = 0; c < m.page_bytes; c += 512) {
          const uint32_t off = c + 16 * lane;
          if (c > 0 && off < m.page_bytes) x = *reinterpret_cast<const uint4*>(at + off);
          if (off == Lc) stored = x;
          if (off <= Lc) poly_block(pw, off / 16, off < Lc ? x : poly_lengths(Lc));
        }
        const uint4 tag = poly_finish(pw, Lc / 16 + 1);
        const bool bad = lane == (int)((Lc / 16) & 31) &&
                         (tag.x != stored.x || tag.y != stored.y || tag.z != stored.z ||
                          tag.w != stored.w);
        if (__any_sync(0xffffffffu, bad) && lane == 0) {
          set_err(m, ERR_INTEGRITY);
          atomicOr(&s_bad, 1ull << d);
        }
      } else if (t < n_chk + n_ks) {
        // (this warp's next key-stream item too, when it has one: the two
        // blocks side by side)
        const bool two = !ONE && t + nwarps < n_chk + n_ks;
        const uint32_t j0 = t - n_chk, j1 = two ? j0 + nwarps : j0;
        const uint32_t d0 = j0 / nch, c0 = j0 % nch, d1 = j1 / nch, c1 = j1 % nch;
        const uint64_t q0 = s_dpage[d0], v0 = m.version[q0] + 1;
        const uint64_t q1 = s_dpage[d1], v1 = m.version[q1] + 1;
        const uint32_t sc = (lane >> 2) + (SEALED ? 1u : 0u);
        uint4 k0, k1;
        if (two)
          chacha_quad2(m.kenc, 8 * c0 + sc, (uint32_t)q0, (uint32_t)v0, (uint32_t)(v0 >> 32),
                       8 * c1 + sc, (uint32_t)q1, (uint32_t)v1, (uint32_t)(v1 >> 32), k0, k1);
        else
          k0 = (ONE ? chacha_lane16 : chacha_quad)(m.kenc, 8 * c0 + sc, (uint32_t)q0,
                                                    (uint32_t)v0, (uint32_t)(v0 >> 32));
        if (512 * c0 + 16 * lane < m.page_bytes)
          *reinterpret_cast<uint4*>(ks_base + (size_t)d0 * m.page_bytes + 512 * c0 + 16 * lane) =
              k0;
        if (two) {
          if (512 * c1 + 16 * lane < m.page_bytes)
            *reinterpret_cast<uint4*>(ks_base + (size_t)d1 * m.page_bytes + 512 * c1 +
                                      16 * lane) = k1;
          t += nwarps;  // (taken)
        }
      } else {
        const uint32_t d = t - n_chk - n_ks;
        const uint64_t q = s_dpage[d];
        poly_store(poly_begin<ONE>(m, q, m.version[q] + 1), s_poly[d]);
      }
    }
    // the counts a one-round remap decides on, read now (nothing but
    // find_remove changes them before the remap, and phase 5 takes its
    // removals out)
    if (wid == nwarps - 2 && (uint32_t)lane < n && n <= m.Wr) {
      auto get = [](const uint32_t* w, uint64_t k) {
        return (__ldcg(w + (k >> 2)) >> ((uint32_t)(k & 3) * 8)) & 0xffu;
      };
      const uint64_t pr = s_rpair[lane];
      const uint32_t p1 = (uint32_t)pr, p2 = (uint32_t)(pr >> 32);
      const bool fresh = s_hit[lane] == NONE32;
      uint32_t c[8];
      c[0] = get(m.load, p1);
      c[1] = get(m.load, p2);
      c[2] = p1 >= m.K ? get(m.revcnt, p1 - m.K) : 0u;
      c[3] = p2 >= m.K ? get(m.revcnt, p2 - m.K) : 0u;
#pragma unroll
      for (int j = 0; j < 4; j++) c[4 + j] = fresh ? get(m.rowcnt, s_rows[4 * lane + j]) : 0u;
#pragma unroll
      for (int k = 0; k < 8; k++) s_cnt[k][lane] = (uint8_t)c[k];
    }
  }
  __syncthreads();
  // (sealed) a page that failed its tag reads as empty: nothing of it enters
  // the map, and the batch ends with ERR_INTEGRITY
  if (SEALED && s_bad) {
    for (uint32_t d = 0; d < s_dcount; d++)
      if ((s_bad >> d) & 1)
        for (uint32_t off = 16 * threadIdx.x; off < m.page_bytes; off += 16 * blockDim.x)
          *reinterpret_cast<uint4*>(L.dbuf + (uint64_t)s_dslot[d] * m.page_bytes + off) =
              make_uint4(0, 0, 0, 0);
    __syncthreads();
  }
  // 3. the host-access trace (every read position in order, then each
  //    distinct page once as a write); the previous batch's table is cleared
  if (m.trace_on && wid == 0) {
    const uint32_t np = 2 * n;
    bool v0, f0, v1, f1;
    uint32_t q0, q1, s0, s1;
    pos_flags(L, lane, np, v0, f0, q0, s0);
    pos_flags(L, lane + 32, np, v1, f1, q1, s1);
    const uint32_t bv0 = __ballot_sync(0xffffffffu, v0), bv1 = __ballot_sync(0xffffffffu, v1);
    const uint32_t bf0 = __ballot_sync(0xffffffffu, f0), bf1 = __ballot_sync(0xffffffffu, f1);
    const uint32_t below = (1u << lane) - 1u;
    const uint32_t tv = __popc(bv0) + __popc(bv1), tf = __popc(bf0) + __popc(bf1);
    unsigned long long tbase = 0;
    if (lane == 0) {
      tbase = *m.trace_len;
      *m.trace_len = tbase + tv + tf;
    }
    tbase = __shfl_sync(0xffffffffu, tbase, 0);
    auto put = [&](uint64_t at, uint32_t e) {
      if (at < m.trace_cap) m.trace[at] = e;
    };
    if (v0) put(tbase + __popc(bv0 & below), q0);
    if (v1) put(tbase + __popc(bv0) + __popc(bv1 & below), q1);
    if (f0) put(tbase + tv + __popc(bf0 & below), q0 | 0x80000000u);
    if (f1) put(tbase + tv + __popc(bf0) + __popc(bf1 & below), q1 | 0x80000000u);
  }
  clear_prev_table(b, threadIdx.x, blockDim.x);
  // 4. find_remove (warp per op)
  for (uint32_t i = wid; i < n; i += nwarps) find_op(m, L, i, lane);
  __syncthreads();
  // 5. Get/Put/Delete semantics (the last warp, lane per op) beside the
  //    write-back with eviction (the other warps, warp per page, straight to
  //    the host as well).  A remap of one round also decides its bins here
  //    (eviction changes no load or row count) and, when the ring window
  //    holds a slot for every take, places every key whose bin is not a page
  //    of this batch: such a placement touches none of the pages, stash lists
  //    or ring slots the eviction reads.  The others wait for the eviction.
  const bool one_round = ONE || n <= m.Wr;  // (W_r >= 1)
  const bool early = one_round && s_ring.tail - s_ring.head >= n;
  if (wid == nwarps - 1) {
    if ((uint32_t)lane < n) exec_op(m, L, lane);
    __syncwarp();
    const bool act =
        one_round && (uint32_t)lane < n && s_leader[lane] == (uint32_t)lane && s_fpres[lane];
    PlaceCounts pc{0, 0, 0};
    if (one_round) {
      // the counts read in 2c less find_remove's removals: a leader's hit
      // left its bin and, deleted, its row; then the lower load wins (the
      // first bin on a tie), a new key takes its least-filled row
      uint32_t rbin = NONE32, rrow = NONE32;
      if ((uint32_t)lane < n && s_leader[lane] == (uint32_t)lane && s_hit[lane] != NONE32) {
        const uint64_t pr = s_pair[lane];
        rbin = meta_which(s_hmeta[lane]) ? (uint32_t)(pr >> 32) : (uint32_t)pr;
        const uint32_t lw = s_lastw[lane];
        if (lw != NONE32 && L.ops[lw] == OP_DEL) rrow = s_hit[lane] / m.R;
      }
      const uint64_t rp = s_rpair[lane];
      const uint32_t p1 = (uint32_t)rp, p2 = (uint32_t)(rp >> 32);
      const uint4 r4 = *reinterpret_cast<const uint4*>(s_rows + 4 * lane);
      const uint32_t rr[4] = {r4.x, r4.y, r4.z, r4.w};
      uint32_t l1 = s_cnt[0][lane], l2 = s_cnt[1][lane];
      uint32_t rc[4] = {s_cnt[4][lane], s_cnt[5][lane], s_cnt[6][lane], s_cnt[7][lane]};
      for (uint32_t j = 0; j < n; j++) {
        const uint32_t bj = __shfl_sync(0xffffffffu, rbin, j);
        const uint32_t wj = __shfl_sync(0xffffffffu, rrow, j);
        l1 -= bj == p1 ? 1u : 0u;
        l2 -= bj == p2 ? 1u : 0u;
#pragma unroll
        for (int k = 0; k < 4; k++) rc[k] -= wj == rr[k] ? 1u : 0u;
      }
      if (act) {
        const bool first = l1 <= l2;
        s_rdest[lane] = first ? p1 : p2;
        pc.load = first ? l1 : l2;
        pc.rev = first ? s_cnt[2][lane] : s_cnt[3][lane];
        if (s_hit[lane] == NONE32) {
          uint32_t best = rr[0], bc = rc[0];
#pragma unroll
          for (int k = 1; k < 4; k++)
            if (rc[k] < bc) {
              best = rr[k];
              bc = rc[k];
            }
          s_rrow[lane] = best;
          pc.row = bc;
        }
      }
    }
    __syncwarp();
    if (early) {
      // (a page of this batch: a probe of its page table)
      bool in_batch = false;
      if (act && s_rdest[lane] >= m.K) {
        const uint32_t q = s_rdest[lane] - (uint32_t)m.K;
        uint32_t h = ht_hash(q, b.ht_mask);
        for (uint32_t probe = 0; probe <= b.ht_mask; probe++) {
          const uint32_t k = s_ht[h];
          if (k == q) in_batch = true;
          if (k == q || k == NONE32) break;
          h = (h + 1) & b.ht_mask;
        }
      }
      if ((uint32_t)lane < FUSED_MAX_OPS) s_defer[lane] = act && in_batch;
      // what each placement's counter atomics would return: the counts read
      // for the decision (nothing else changes them before these
      // placements) plus the placements of lower lanes on the same bin or
      // row
      const bool go = act && !in_batch, fresh = go && s_hit[lane] == NONE32;
      uint32_t rb = 0, rw = 0;  // (a single op has no lower lanes)
      if (!ONE) {
        const uint32_t below = (1u << lane) - 1u;
        const uint32_t gm = __ballot_sync(0xffffffffu, go), fm = __ballot_sync(0xffffffffu, fresh);
        rb = __popc(__match_any_sync(0xffffffffu, go ? s_rdest[lane] : NONE32) & gm & below);
        rw = __popc(__match_any_sync(0xffffffffu, fresh ? s_rrow[lane] : NONE32) & fm & below);
      }
      pc.load += rb + 1;
      pc.rev += rb;
      pc.row += rw;
      remap_apply_op(m, L, lane, go, &s_ring, false, &pc);
    }
  } else if (wid < evict_warps) {
    const uint32_t nd = s_dcount, per_warp = m.page_bytes + 32 * 16;
    const bool ks_pre = nd <= ks_slots;
    uint8_t* const ks_base = sbuf + (size_t)evict_warps * per_warp;
    for (uint32_t e = wid; e < nd; e += evict_warps)
      evict_one<SEALED, ONE>(m, L, e, sbuf + (size_t)wid * per_warp, true,
                             ks_pre ? ks_base + (size_t)e * m.page_bytes : nullptr,
                             SEALED && ks_pre && nd <= 7 ? s_poly[e] : nullptr);
  }
  __syncthreads();
  // 6. P2C remap in rounds of W_r op slots (warp 0, lane per op): decide on
  //    round-start counts (a single round decided above), then place; with
  //    the early placements above, only the ones that waited for the eviction
  if (wid == 0 && early) {
    remap_apply_op(m, L, lane, s_defer[lane] != 0, &s_ring, false);
  } else if (wid == 0) {
    for (uint64_t lo = 0; lo < n; lo += m.Wr) {
      const uint64_t hi = lo + m.Wr < n ? lo + m.Wr : n;
      const uint32_t i = lane;
      const bool act = i >= lo && i < hi && s_leader[i] == i && s_fpres[i];
      if (act && !one_round) decide_op_l2(m, L, i);
      __syncwarp();
      remap_apply_op(m, L, i, act, &s_ring);
      __syncwarp();
    }
  }
  __syncthreads();

  if (b.h_res) {
    // results vout | status (packed in the device buffer) and the error word
    // to the caller's pinned staging as 8-byte words of 7 stream bytes and
    // the call's tag: each is one store the host sees whole, so the host
    // takes the results once every word is tagged, with no system-scope
    // fence here and no completion word after it
    const uint32_t nb = n * (m.vb + 1), total = nb + 4;
    for (uint32_t w = threadIdx.x; w < (total + 6) / 7; w += blockDim.x) {
      uint64_t v = (uint64_t)b.res_tag << 56;
      for (uint32_t k = 0; k < 7; k++) {
        const uint32_t at = 7 * w + k;
        uint32_t byte = 0;
        if (at < nb) byte = b.vout[at];
        else if (at < total) byte = (*(volatile uint32_t*)m.err >> (8 * (at - nb))) & 0xffu;
        v |= (uint64_t)byte << (8 * k);
      }
      *(volatile uint64_t*)(b.h_res + w) = v;
    }
  }
}

cudaError_t launch_fused(const MapDev& m, const BatchDev& b, uint32_t n, uint64_t t0,
                         cudaStream_t st, bool early_in, const FusedInline* inl) {
  if (n == 0) return cudaSuccess;
  if (n > FUSED_MAX_OPS || b.ht_mask + 1 != FUSED_TABLE) return cudaErrorInvalidValue;
  if (inl && inl->bytes != n * (9 + m.vb)) return cudaErrorInvalidValue;
  ProfSpan whole(P_ACCESS, st);
  if (m.vb > FUSED_VB_MAX) return cudaErrorInvalidValue;
  using Kf = void (*)(MapDev, BatchDev, uint32_t, uint64_t, uint32_t, uint32_t, uint32_t,
                      FusedInline);
  static const Kf kfs[4] = {k_fused<false, false>, k_fused<false, true>, k_fused<true, false>,
                            k_fused<true, true>};
  const int which = (m.integrity ? 2 : 0) + (n == 1 ? 1 : 0);
  const Kf kf = kfs[which];
  // the eviction warps' page buffers take what the kernel's own shared
  // arrays leave of the 227 KB a block may use
  static const size_t static_bytes[4] = {
      [] { cudaFuncAttributes a{}; return cudaFuncGetAttributes(&a, kfs[0]) == cudaSuccess
                                              ? a.sharedSizeBytes : (size_t)(64u << 10); }(),
      [] { cudaFuncAttributes a{}; return cudaFuncGetAttributes(&a, kfs[1]) == cudaSuccess
                                              ? a.sharedSizeBytes : (size_t)(64u << 10); }(),
      [] { cudaFuncAttributes a{}; return cudaFuncGetAttributes(&a, kfs[2]) == cudaSuccess
                                              ? a.sharedSizeBytes : (size_t)(64u << 10); }(),
      [] { cudaFuncAttributes a{}; return cudaFuncGetAttributes(&a, kfs[3]) == cudaSuccess
                                              ? a.sharedSizeBytes : (size_t)(64u << 10); }()};
  const size_t budget = (227u << 10) - static_bytes[which];
  const uint32_t per_warp = m.page_bytes + 32 * 16;
  uint32_t ew = (uint32_t)(budget / per_warp);
  // (the last warp runs the ops' semantics meanwhile)
  ew = ew < 1 ? 1 : (ew > FUSED_THREADS / 32 - 1 ? FUSED_THREADS / 32 - 1 : ew);
  size_t smem = (size_t)ew * per_warp;
  if (smem > budget) return cudaErrorInvalidValue;
  // then the write-back key streams of up to 2n pages, as many as fit
  uint64_t ks_slots = (budget - smem) / m.page_bytes;
  if (ks_slots > 2ull * n) ks_slots = 2ull * n;
  smem += ks_slots * m.page_bytes;
  cudaError_t e = raise_smem_limit((const void*)kf, smem);
  if (e != cudaSuccess) return e;
  FusedInline none;
  none.bytes = 0;
  e = launch_dependent(kf, 1, FUSED_THREADS, smem, st, m, b, n, t0, ew, early_in ? 1u : 0u,
                       (uint32_t)ks_slots, inl ? *inl : none);
  if (e != cudaSuccess) return e;
  count_launch();
  return cudaSuccess;
}

// The batch's preparation depends only on its own inputs: the grouping keys
// (key hash table), the DUMMY / REMAP pairs and position-map rows, the
// grouping sort and scan.  It may run on its own stream, ahead of the
// previous batch's main part.
cudaError_t launch_prep(const MapDev& m, const BatchDev& b, uint32_t n, uint64_t t0,
                        cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  uint32_t n_sort = 512;
  while (n_sort < n) n_sort <<= 1;
  if (n_sort > 512 && n_sort < 4096) n_sort = 4096;
  const int keys32 = n_sort <= 4096;
  {
    ProfSpan ps(P_STAGE, st);
    k_clear_keys<<<32, 256, 0, st>>>(b, n);
    k_stage<<<(3 * n_sort + 255) / 256, 256, 0, st>>>(m, b, n, n_sort, t0, keys32);
    count_launch(2);
  }
  cudaError_t e;
  {
    ProfSpan ps(P_GROUP, st);
    if (keys32) {
      e = sort_batch_keys32(reinterpret_cast<uint32_t*>(b.skeys), n_sort, st);
      if (e != cudaSuccess) return e;
      k_group<uint32_t><<<1, n <= 8192 ? 256 : GROUP_THREADS, 0, st>>>(b, n);
    } else {
      e = sort_batch_keys(b.skeys, n_sort, st);
      if (e != cudaSuccess) return e;
      k_group<uint64_t><<<1, n <= 8192 ? 256 : GROUP_THREADS, 0, st>>>(b, n);
    }
    count_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_ahead_lookup(const MapDev& m, const BatchDev& b, uint32_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  ProfSpan ps(P_AHEAD, st);
  k_clear_la<<<64, 256, 0, st>>>(b);
  const uint32_t warp_blocks = (n * 32 + 255) / 256;
  k_ahead_lookup<<<warp_blocks, 256, 0, st>>>(m, b, n);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_ahead_gather(const MapDev& m, const BatchDev& b, uint32_t limit,
                                cudaStream_t st) {
  if (limit == 0) return cudaSuccess;
  ProfSpan ps(P_AHEAD, st);
  k_ahead_gather<<<LINK_BLOCKS, COPY_BLOCK, 0, st>>>(m, b, limit);
  count_launch();
  return cudaGetLastError();
}

// The part that reads and changes the map: lookup, page reads, find_remove,
// exec, write-back, remap.
cudaError_t launch_main(const MapDev& m, const BatchDev& b, uint32_t n, cudaStream_t st,
                        const FlushCtx& fc) {
  if (n == 0) return cudaSuccess;
  cudaError_t e;
  ProfSpan whole(P_ACCESS, st);
  const uint32_t warp_blocks = (n * 32 + 255) / 256;
  e = cudaMemsetAsync(b.dcount, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  {
    // position-map search fused with the page reads
    ProfSpan ps(P_GATHER, st);
    const uint32_t lb = LOOKUP_BLOCKS_PER_SM * (uint32_t)num_sms();
    auto kl = m.integrity ? k_lookup<true> : k_lookup<false>;
    kl<<<warp_blocks < lb ? warp_blocks : lb, 256, 0, st>>>(m, b, n);
    count_launch();
  }
  if (m.trace_on) {
    ProfSpan ps(P_PAGES, st);
    const uint32_t np = 2 * n;
    if (np <= PAGES_SMALL_MAX) {
      k_pages_small<<<1, 1024, 0, st>>>(m, b, np);
      count_launch();
    } else {
      const uint32_t nblk = (np + PAGES_BLOCK - 1) / PAGES_BLOCK;
      k_pages_count<<<nblk, PAGES_BLOCK, 0, st>>>(b, np, b.block_cnt);
      k_pages_scan<<<1, 1024, 0, st>>>(m, b, nblk, b.block_cnt);
      k_pages_emit<<<nblk, PAGES_BLOCK, 0, st>>>(m, b, np, b.block_cnt);
      count_launch(3);
    }
  }
  if (fc.ev_looked) cudaEventRecord(fc.ev_looked, st);
  if (fc.prev) {
    // the previous batch's write-back, now that this batch's page reads
    // (which took the pages it rewrote from its ciphertexts) are done
    e = cudaEventRecord(fc.ev_reads_done, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(fc.flush_st, fc.ev_reads_done, 0);
    if (e != cudaSuccess) return e;
    ProfSpan ps(P_FLUSH, fc.flush_st);
    k_flush<<<flush_blocks(fc.prev_n, fc.prev_fast), COPY_BLOCK, 0, fc.flush_st>>>(m, *fc.prev);
    count_launch();
    e = cudaEventRecord(fc.prev_flushed, fc.flush_st);
    if (e != cudaSuccess) return e;
  }
  if (m.integrity) {
    // the sealed pages' tags and decryption (warp per page)
    ProfSpan ps(P_GATHER, st);
    const uint32_t want = (2 * n * 32 + 255) / 256, cap = 8 * (uint32_t)num_sms();
    e = launch_dependent(k_open, want < cap ? want : cap, 256, 0, st, m, b);
    if (e != cudaSuccess) return e;
    count_launch();
  }
  {
    ProfSpan ps(P_FINDEXEC, st);
    e = launch_dependent(k_find, warp_blocks, 256, 0, st, m, b, n);
    if (e != cudaSuccess) return e;
    count_launch();
  }
  // P2C remap: one round -> the decisions run with exec, then one apply
  // launch; many rounds on a small map -> all rounds in one CTA on
  // shared-memory counts; otherwise a decide and an apply launch per round
  const uint64_t rounds = (n + m.Wr - 1) / m.Wr;
  const bool smem_remap = rounds > 1 && m.B <= REMAP_SMEM_MAX_BINS && m.rows <= REMAP_SMEM_MAX_ROWS;
  const int fused_decide = rounds == 1 ? 1 : 0;
  {
    ProfSpan ps(P_EVICT, st);
    const uint32_t wpb = EVICT_WARPS_PER_BLOCK;
    const size_t smem = (size_t)wpb * (m.page_bytes + 32 * 16);
    auto kx = m.integrity ? k_exec_evict<true> : k_exec_evict<false>;
    e = raise_smem_limit((const void*)kx, smem);
    if (e != cudaSuccess) return e;
    const uint32_t evict_blocks = (2 * n + wpb - 1) / wpb;
    const uint32_t exec_blocks = (n + wpb * 32 - 1) / (wpb * 32);
    e = launch_dependent(kx, evict_blocks + exec_blocks, wpb * 32, smem, st, m, b, n,
                         evict_blocks, fused_decide);
    if (e != cudaSuccess) return e;
    count_launch();
  }
  // the host write-back overlaps the rest of this batch and the next one
  cudaEventRecord(fc.ev_evicted, st);
  if (!fc.defer_own) {
    cudaStreamWaitEvent(fc.flush_st, fc.ev_evicted, 0);
    {
      ProfSpan ps(P_FLUSH, fc.flush_st);
      k_flush<<<flush_blocks(n, fc.fast_flush), COPY_BLOCK, 0, fc.flush_st>>>(m, b);
      count_launch();
    }
    cudaEventRecord(fc.ev_flushed, fc.flush_st);
  }
  ProfSpan prs(P_REMAP, st);
  const size_t rsmem = ((m.B + 3) / 4 + (m.rows + 3) / 4) * 4;
  if (fused_decide) {
    e = launch_dependent(k_remap_apply, (n + 255) / 256, 256, 0, st, m, b, 0u, n);
    if (e != cudaSuccess) return e;
    count_launch();
  } else if (smem_remap) {
    const bool reg = n <= REMAP_REG_OPS * 1024;
    e = raise_smem_limit(reg ? (const void*)k_remap_smem_reg : (const void*)k_remap_smem, rsmem);
    if (e != cudaSuccess) return e;
    if (reg) k_remap_smem_reg<<<1, 1024, rsmem, st>>>(m, b, n);
    else k_remap_smem<<<1, 1024, rsmem, st>>>(m, b, n);
    k_remap_rest<<<(n + 255) / 256, 256, 0, st>>>(m, b, n);
    count_launch(2);
  } else {
    for (uint64_t lo = 0; lo < n; lo += m.Wr) {
      const uint32_t hi = (uint32_t)(lo + m.Wr < n ? lo + m.Wr : n);
      const uint32_t g = (hi - (uint32_t)lo + 255) / 256;
      k_remap_decide<<<g, 256, 0, st>>>(m, b, (uint32_t)lo, hi);
      k_remap_apply<<<g, 256, 0, st>>>(m, b, (uint32_t)lo, hi);
      count_launch(2);
    }
  }
  return cudaGetLastError();
}

}  // namespace bdev
