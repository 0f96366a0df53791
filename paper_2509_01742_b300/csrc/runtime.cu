// runtime.cu -- host runtime behind the C ABI of include/bolt.h.
//
// Owns the planner (Sec. 3.3 sizing and the alpha policy of "Parameters
// selection"), every device allocation, the pinned device-mapped host pages
// (Sec. 4.1 step 1: the host provisions pinned memory the accelerator reaches
// directly), the batch staging buffers, and the error / poison state.  All
// arithmetic of the method runs in the kernels of build.cu, sort.cu and
// access.cu; this file only plans, allocates, copies and launches.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "handle.h"

using namespace bdev;

namespace bdev {
thread_local Prof* g_prof = nullptr;

cudaError_t raise_smem_limit(const void* kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  // a fixed table (no host allocation: the allocation-free build uses this)
  struct Limit {
    const void* kernel;
    int device;
    size_t bytes;
  };
  constexpr int MAX_LIMITS = 256;
  static std::mutex mu;
  static Limit limits[MAX_LIMITS];
  static int n_limits = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  for (int i = 0; i < n_limits; i++) {
    Limit& l = limits[i];
    if (l.kernel == kernel && l.device == dev) {
      if (l.bytes >= bytes) return cudaSuccess;
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e == cudaSuccess) l.bytes = bytes;
      return e;
    }
  }
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  // past the table's end the attribute is still set (under the lock) each time
  if (e == cudaSuccess && n_limits < MAX_LIMITS) limits[n_limits++] = {kernel, dev, bytes};
  return e;
}
}  // namespace bdev

namespace {


struct Plan {
  bolt_info_t info;
};

// Claim 3.2: lmax = c + ceil(log2 log2 N) + 1 (constant 1 in the O-term, as
// in Sec. 3.3); Claims 3.3 / 3.4 with constant 1; position map of
// ceil(N/16) rows holding 16 + ceil(log2 log2 N / log2 d) keys (Sec. 4.2).
// A sealed page (integrity on) carries a 16-byte Poly1305 tag after them.
int plan_sizes(uint64_t N, uint32_t c, double alpha, uint32_t vb, bolt_info_t* o,
               bool integrity = false) {
  if (N < 64 || c < 1 || alpha < 0.0 || alpha >= 1.0) return BOLT_E_ARG;
  std::memset(o, 0, sizeof *o);
  const double llg = std::log2(std::log2((double)N));
  o->N = N;
  o->c = c;
  o->d = 4;
  o->key_bytes = 8;
  o->val_bytes = vb;
  o->lmax = c + (uint32_t)std::ceil(llg) + 1;
  o->R = 16 + (uint32_t)std::ceil(llg / 2.0);
  o->rows = (N + 15) / 16;
  o->B = (N + c - 1) / c;
  o->alpha = alpha;
  o->K = (uint64_t)std::floor(alpha * (double)o->B);
  o->M = o->B - o->K;
  if (o->M < 2 || o->lmax > 32 || o->R > 32) return BOLT_E_ARG;
  const double lnN = std::log((double)N);
  o->beta1 = (double)o->K * c + o->lmax * std::sqrt((double)o->K * lnN);
  o->beta2 = (1.0 + alpha) * (double)o->M / 2.0 + o->lmax * std::sqrt((double)o->M * lnN);
  // Claims 3.3/3.4 bound one-at-a-time access; one batch can add up to a
  // batch of remapped keys to the stash before their pages are read again.
  o->vs_cap = (uint64_t)std::ceil(o->beta1 + o->beta2) + (N < MAXB ? N : MAXB);
  o->round_width = o->B / 256 > 0 ? o->B / 256 : 1;
  o->rec_bytes = 8 + vb;
  o->page_bytes = (16 + o->lmax * o->rec_bytes + (integrity ? 16 : 0) + 63) / 64 * 64;
  if (o->vs_cap >= (1ull << 29) || o->rows * o->R >= (1ull << 32)) return BOLT_E_ARG;
  return BOLT_OK;
}

}  // namespace


namespace {

int cuda_fail(cudaError_t e) {
  if (e == cudaSuccess) return BOLT_OK;
  if (e == cudaErrorMemoryAllocation) return BOLT_E_NOMEM;
  return BOLT_E_CUDA;
}

// wait for the handle's own stream and for the caller stream it last used
cudaError_t sync_all(bolt* h) {
  cudaError_t e = cudaSuccess;
  if (h->last_st && h->last_st != h->st) e = cudaStreamSynchronize(h->last_st);
  for (cudaStream_t s : {h->st, h->st2, h->st_fl, h->st_prep, h->st_out}) {
    if (!s) continue;
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
  }
  return e;
}

template <typename T>
int dalloc(bolt* h, T** p, uint64_t count) {
  void* ptr = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(&ptr, count * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(e);
  h->dev_allocs.push_back(ptr);
  h->dev_bytes += count * sizeof(T);
  *p = static_cast<T*>(ptr);
  return BOLT_OK;
}

void free_build_scratch(bolt* h) {
  BuildScratch& s = h->bs;
  cudaFree(s.tags); cudaFree(s.bins); cudaFree(s.dest); cudaFree(s.prow);
  cudaFree(s.page_off); cudaFree(s.block_sums); cudaFree(s.counters);
  cudaFree(s.rows4); cudaFree(s.keysort);
  s = BuildScratch{};
  cudaFree(h->in_keys); cudaFree(h->in_vals);
  h->in_keys = nullptr; h->in_vals = nullptr; h->in_cap = 0;
  h->scratch_bytes = 0;
}

void free_state(bolt* h) {
  sync_all(h);
  h->last_st = nullptr;
  for (void* p : h->dev_allocs) cudaFree(p);
  h->dev_allocs.clear();
  h->dev_bytes = 0;
  if (h->pages_host) cudaFreeHost(h->pages_host);
  h->pages_host = nullptr;
  free_build_scratch(h);
  h->m = MapDev{};
  h->b = BatchDev{};
  for (int s = 0; s < 2; s++) {
    h->flush_pending[s] = false;
    h->s_ht_key[s] = h->s_ht_min[s] = h->s_dslot[s] = h->s_dpage[s] = h->s_dcount[s] = nullptr;
    h->s_dbuf[s] = nullptr;
  }
  h->prev_valid = false;
  h->deferred = false;
  h->slot = 0;
  h->allocated = false;
  h->initialized = false;
}

// streams and events of a handle (any of them may be null)
void destroy_streams(bolt* h) {
  for (cudaEvent_t* ev : {&h->ev_fork, &h->ev_join, &h->ev_evicted[0], &h->ev_evicted[1],
                          &h->ev_flushed[0], &h->ev_flushed[1], &h->ev_in, &h->ev_prep[0],
                          &h->ev_prep[1], &h->ev_pfree[0], &h->ev_pfree[1], &h->ev_h2d[0],
                          &h->ev_h2d[1], &h->ev_d2h[0], &h->ev_d2h[1], &h->ev_looked[0],
                          &h->ev_looked[1], &h->ev_ioready[0], &h->ev_ioready[1],
                          &h->ev_pfork, &h->ev_pjoin, &h->ev_reads_done})
    if (*ev) {
      cudaEventDestroy(*ev);
      *ev = nullptr;
    }
  for (cudaStream_t* s : {&h->st_out, &h->st_prep, &h->st_fl, &h->st2, &h->st})
    if (*s) {
      cudaStreamDestroy(*s);
      *s = nullptr;
    }
}

int choose_plan(bolt* h, bolt_info_t* o) {
  if (h->alpha_override >= 0.0)
    return plan_sizes(h->N, h->c, h->alpha_override, h->vb, o, h->integrity);
  static const double grid[] = {0.2, 0.1, 0.05, 0.01, 0.0};
  for (double a : grid) {
    int rc = plan_sizes(h->N, h->c, a, h->vb, o, h->integrity);
    if (rc) return rc;
    if ((double)o->vs_cap * (double)(8 + h->vb) <= (double)h->hbm_budget) return BOLT_OK;
  }
  return BOLT_E_NOMEM;
}

int alloc_state(bolt* h) {
  int rc = choose_plan(h, &h->info);
  if (rc) return rc;
  h->info.key_bytes = h->kb;
  const bolt_info_t& I = h->info;
  MapDev& m = h->m;
  m.N = I.N; m.B = I.B; m.K = I.K; m.M = I.M; m.rows = I.rows; m.Wr = I.round_width;
  m.vs_cap = I.vs_cap; m.R = I.R; m.lmax = I.lmax; m.vb = I.val_bytes; m.rec = I.rec_bytes;
  m.page_bytes = I.page_bytes;
  const uint64_t slots = I.rows * I.R;
#define TRY(x) do { int r_ = (x); if (r_) { free_state(h); return r_; } } while (0)
  TRY(dalloc(h, &m.load, I.B / 4 + 2));
  TRY(dalloc(h, &m.rowcnt, I.rows / 4 + 2));
  TRY(dalloc(h, &m.pm_key, slots));
  TRY(dalloc(h, &m.pm_bins, slots));
  TRY(dalloc(h, &m.pm_meta, slots));
  TRY(dalloc(h, &m.vs_key, I.vs_cap));
  TRY(dalloc(h, &m.vs_val, I.vs_cap * I.val_bytes));
  TRY(dalloc(h, &m.vs_pm, I.vs_cap));
  TRY(dalloc(h, &m.vs_live, I.vs_cap));
  TRY(dalloc(h, &m.ring, I.vs_cap));
  TRY(dalloc(h, &m.ring_ctr, 2));
  TRY(dalloc(h, &m.rev, I.M * I.lmax));
  TRY(dalloc(h, &m.revcnt, I.M / 4 + 2));
  TRY(dalloc(h, &m.version, I.M));
  TRY(dalloc(h, &m.err, 1));
  TRY(dalloc(h, &m.stat, ST_WORDS));
  TRY(dalloc(h, &m.trace, h->trace_cap));
  TRY(dalloc(h, &m.trace_len, 1));
  m.trace_cap = h->trace_cap;
  m.trace_on = h->trace_on ? 1 : 0;
  m.spin_limit = h->spin_limit;
  m.integrity = h->integrity ? 1 : 0;
  void* hp = nullptr;
  cudaError_t e = cudaHostAlloc(&hp, I.M * I.page_bytes, cudaHostAllocMapped | cudaHostAllocPortable);
  if (e != cudaSuccess) { free_state(h); return BOLT_E_NOMEM; }
  h->pages_host = static_cast<uint8_t*>(hp);
  void* dp = nullptr;
  e = cudaHostGetDevicePointer(&dp, hp, 0);
  if (e != cudaSuccess) { free_state(h); return BOLT_E_CUDA; }
  m.pages = static_cast<uint8_t*>(dp);
  // batch buffers, for batches of up to cap_batch operations
  BatchDev& b = h->b;
  const uint64_t vb = I.val_bytes;
  const uint64_t cap = h->cap_batch;
  uint64_t cap2 = 1;
  while (cap2 < cap) cap2 <<= 1;
  const uint64_t sort_cap = cap2 <= 512 ? 512 : (cap2 < 4096 ? 4096 : cap2);
  // two I/O sets, one block each: inputs keys | vin | ops, then (from a
  // 256-byte boundary) outputs vout | status; set 0 is the batch's own
  const uint64_t io_in = (cap * (9 + vb) + 255) / 256 * 256;
  for (int s = 0; s < 2; s++) {
    uint8_t* blk = nullptr;
    TRY(dalloc(h, &blk, io_in + cap * (vb + 1)));
    bolt::IoSet& d = h->d_io[s];
    d.keys = reinterpret_cast<uint64_t*>(blk);
    d.vin = blk + cap * 8;
    d.ops = blk + cap * (8 + vb);
    d.vout = blk + io_in;
    d.status = blk + io_in + cap * vb;
  }
  b.ops = h->d_io[0].ops;
  b.keys = h->d_io[0].keys;
  b.vin = h->d_io[0].vin;
  b.vout = h->d_io[0].vout;
  b.status = h->d_io[0].status;
  b.kt_mask = (uint32_t)(2 * cap2 < 128 ? 127 : 2 * cap2 - 1);
  const uint32_t ht = (uint32_t)(4 * cap2 < 256 ? 256 : 4 * cap2);
  b.ht_mask = ht - 1;
  for (int s = 0; s < 2; s++) {
    bolt::PrepSet& ps = h->s_prep[s];
    TRY(dalloc(h, &ps.skeys, sort_cap));
    TRY(dalloc(h, &ps.kt_own, (uint64_t)b.kt_mask + 1));
    TRY(dalloc(h, &ps.leader, cap));
    TRY(dalloc(h, &ps.prevw, cap));
    TRY(dalloc(h, &ps.lastw, cap));
    TRY(dalloc(h, &ps.pair, cap));
    TRY(dalloc(h, &ps.rpair, cap));
    TRY(dalloc(h, &ps.rows, 4 * cap));
    TRY(dalloc(h, &ps.hit, cap));
    TRY(dalloc(h, &ps.done, cap));
    TRY(dalloc(h, &ps.pres, cap));
    TRY(dalloc(h, &ps.la_key, ht));
    TRY(dalloc(h, &ps.la_idx, ht));
    TRY(dalloc(h, &ps.la_list, 2 * cap));
    TRY(dalloc(h, &ps.la_count, 1));
    TRY(dalloc(h, &ps.la_buf, 2 * cap * I.page_bytes));
  }
  TRY(dalloc(h, &b.pos_page, 2 * cap));
  TRY(dalloc(h, &b.pos_slot, 2 * cap));
  TRY(dalloc(h, &b.block_cnt, 2 * ((2 * cap + 255) / 256) + 2));
  TRY(dalloc(h, &b.trace_base, 2));
  for (int s = 0; s < 2; s++) {
    TRY(dalloc(h, &h->s_ht_key[s], ht));
    TRY(dalloc(h, &h->s_ht_min[s], ht));
    TRY(dalloc(h, &h->s_dbuf[s], (uint64_t)ht * I.page_bytes));
    TRY(dalloc(h, &h->s_dslot[s], 2 * cap));
    TRY(dalloc(h, &h->s_dpage[s], 2 * cap));
    TRY(dalloc(h, &h->s_dcount[s], 1));
  }
  TRY(dalloc(h, &b.removed, ht));
  TRY(dalloc(h, &b.init_val, cap * vb));
  TRY(dalloc(h, &b.init_present, cap));
  TRY(dalloc(h, &b.rval, cap * vb));
  TRY(dalloc(h, &b.fpres, cap));
  TRY(dalloc(h, &b.rdest, cap));
  TRY(dalloc(h, &b.rrow, cap));
  TRY(dalloc(h, &h->d_kdf, 16));
  TRY(dalloc(h, &h->d_flag, 1));
#undef TRY
  h->allocated = true;
  return BOLT_OK;
}

int grow_build_scratch(bolt* h, uint64_t n) {
  BuildScratch& s = h->bs;
  uint64_t tag_cap = 8192;
  while (tag_cap < n) tag_cap <<= 1;
  const uint64_t nblocks = (h->info.M + 1 + 8192 - 1) / 8192 + 1;
  if (s.cap >= n && s.tag_cap >= tag_cap && s.block_cap >= nblocks && s.page_off) return BOLT_OK;
  sync_all(h);
  cudaFree(s.tags); cudaFree(s.bins); cudaFree(s.dest); cudaFree(s.prow);
  cudaFree(s.page_off); cudaFree(s.block_sums); cudaFree(s.counters);
  cudaFree(s.rows4); cudaFree(s.keysort);
  s = BuildScratch{};
  const uint64_t cap = n > 0 ? n : 1;
  cudaError_t e = cudaSuccess;
  e = e ? e : cudaMalloc(&s.tags, tag_cap * sizeof(uint64_t));
  e = e ? e : cudaMalloc(&s.keysort, 2 * tag_cap * sizeof(uint64_t));
  e = e ? e : cudaMalloc(&s.rows4, cap * sizeof(uint4));
  e = e ? e : cudaMalloc(&s.bins, cap * sizeof(uint64_t));
  e = e ? e : cudaMalloc(&s.dest, cap * sizeof(uint32_t));
  e = e ? e : cudaMalloc(&s.prow, cap * sizeof(uint32_t));
  e = e ? e : cudaMalloc(&s.page_off, (h->info.M + 1) * sizeof(uint32_t));
  e = e ? e : cudaMalloc(&s.block_sums, nblocks * sizeof(uint32_t));
  e = e ? e : cudaMalloc(&s.counters, 2 * sizeof(unsigned long long));
  if (e != cudaSuccess) {
    cudaFree(s.tags); cudaFree(s.bins); cudaFree(s.dest); cudaFree(s.prow);
    cudaFree(s.page_off); cudaFree(s.block_sums); cudaFree(s.counters);
    cudaFree(s.rows4); cudaFree(s.keysort);
    s = BuildScratch{};
    return cuda_fail(e);
  }
  s.cap = cap;
  s.tag_cap = tag_cap;
  s.block_cap = nblocks;
  h->scratch_bytes = tag_cap * 24 + cap * (16 + 8 + 4 + 4) + (h->info.M + 1) * 4 + nblocks * 4 + 16;
  return BOLT_OK;
}

// KDF: ChaCha20 block under the 256-bit key seed || 0^192, nonce "BOLT" || 0;
// words 0-7 -> K_prf, words 8-15 -> K_enc.
__global__ void k_kdf(uint64_t seed, uint32_t* out) {
  const uint32_t key[8] = {(uint32_t)seed, (uint32_t)(seed >> 32), 0, 0, 0, 0, 0, 0};
  uint32_t w[16];
  chacha_block(key, 0, 0x544c4f42u, 0, 0, w);
  for (int i = 0; i < 16; i++) out[i] = w[i];
}

// keys must be distinct (Sec. 2.1): sort a copy, flag equal neighbours
__global__ void k_copy_keys(const uint64_t* keys, uint64_t n, uint64_t n_pow2, uint64_t* out) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pow2;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = i < n ? keys[i] : ~0ull;
}
// keys must be distinct (Sec. 2.1), hashed variant: every key goes into an
// open-addressing table of 2 * half slots (two buffers of `half`) by
// compare-and-swap; a key met twice raises the flag.  A slot holds key ^ SALT
// (0 = empty); the one key equal to SALT is counted apart in *salt_count.
constexpr uint64_t DUP_SALT = 0x9E3779B97F4A7C15ull;
__global__ void k_dup_insert(const uint64_t* keys, uint64_t n, uint64_t* t0, uint64_t* t1,
                             uint64_t half, uint32_t* flag, unsigned long long* salt_count) {
  const uint64_t mask = 2 * half - 1;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    const uint64_t e = k ^ DUP_SALT;
    if (e == 0) {
      if (atomicAdd(salt_count, 1ull) > 0) *flag = 1;
      continue;
    }
    uint64_t h = k;
    h ^= h >> 33; h *= 0xff51afd7ed558ccdull; h ^= h >> 33; h *= 0xc4ceb9fe1a85ec53ull;
    h ^= h >> 33;
    h &= mask;
    for (uint64_t probe = 0; probe <= mask; probe++) {
      unsigned long long* slot =
          reinterpret_cast<unsigned long long*>(h < half ? t0 + h : t1 + (h - half));
      const unsigned long long old = atomicCAS(slot, 0ull, (unsigned long long)e);
      if (old == 0) break;
      if (old == e) {
        *flag = 1;
        break;
      }
      h = (h + 1) & mask;
    }
  }
}

__global__ void k_adjacent_equal(const uint64_t* sorted, uint64_t n, uint32_t* flag) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    if (sorted[i] == sorted[i - 1]) *flag = 1;
}

int sm_count() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

int read_err(bolt* h, uint32_t* out) {
  if (sync_all(h) != cudaSuccess) return BOLT_E_CUDA;
  cudaError_t e = cudaMemcpyAsync(h->h_err, h->m.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return BOLT_E_CUDA;
  *out = *h->h_err;
  return BOLT_OK;
}

int err_to_rc(uint32_t err) {
  // a wait that gave up first: the steps after it may have flagged the
  // half-built state as well
  if (err & ERR_TIMEOUT) return BOLT_E_TIMEOUT;
  // an altered page: what the batch did after reading it is void
  if (err & ERR_INTEGRITY) return BOLT_E_INTEGRITY;
  if (err & ERR_OVERFLOW_MASK) return BOLT_E_OVERFLOW;
  if (err) return BOLT_E_INTERNAL;
  return BOLT_OK;
}

// The build on the device.  `bs` must hold at least n records, a tag buffer
// of a power of two >= max(n, 8192) entries and M + 1 page offsets.
// The view of slot s of the batch buffers for a batch of n ops: the slot's
// preparation outputs, page hash table and page buffers, table sizes for n,
// and the previous batch's written pages (the other slot).
BatchDev slot_view(bolt* h, BatchDev b, uint32_t n, int s) {
  const int ps = s ^ 1;
  uint32_t ht = 256, kt = 128;
  while (ht < 4 * n) ht <<= 1;
  while (kt < 2 * n) kt <<= 1;
  b.ht_mask = ht - 1;
  b.kt_mask = kt - 1;
  const bolt::PrepSet& p = h->s_prep[s];
  b.skeys = p.skeys;
  b.kt_own = p.kt_own;
  b.leader = p.leader;
  b.prevw = p.prevw;
  b.lastw = p.lastw;
  b.pair = p.pair;
  b.rpair = p.rpair;
  b.rows = p.rows;
  b.hit = p.hit;
  b.done = p.done;
  b.pres = p.pres;
  b.la_key = p.la_key;
  b.la_idx = p.la_idx;
  b.la_list = p.la_list;
  b.la_count = p.la_count;
  b.la_buf = p.la_buf;
  b.la_on = 0;
  b.la_limit = 0;
  b.ht_key = h->s_ht_key[s];
  b.ht_min = h->s_ht_min[s];
  b.dbuf = h->s_dbuf[s];
  b.dslot = h->s_dslot[s];
  b.dpage = h->s_dpage[s];
  b.dcount = h->s_dcount[s];
  b.prev_valid = h->prev_valid ? 1u : 0u;
  b.prev_ht_key = h->s_ht_key[ps];
  b.prev_dbuf = h->s_dbuf[ps];
  b.prev_ht_mask = h->slot_ht_mask[ps];
  b.clr_ht_key = h->prev_valid ? h->s_ht_key[ps] : nullptr;
  b.clr_ht_min = h->s_ht_min[ps];
  b.clr_mask = h->slot_ht_mask[ps];
  return b;
}

// The main part of a batch in the current slot, on stream st, once its
// preparation has been enqueued (on st, or on st_prep with st waiting for it):
// waits for the flush that last used the slot, launches, flips the slot.
cudaError_t main_batch(bolt* h, const BatchDev& b, uint32_t n, cudaStream_t st,
                       bool lookahead = false, bool defer_own = false) {
  const int s = h->slot;
  if (h->flush_pending[s]) {
    cudaError_t e = cudaStreamWaitEvent(st, h->ev_flushed[s], 0);
    if (e != cudaSuccess) return e;
  }
  FlushCtx fc{h->st_fl, h->ev_evicted[s], h->ev_flushed[s],
              lookahead ? h->ev_looked[s] : nullptr, lookahead ? 1 : 0};
  fc.defer_own = defer_own ? 1 : 0;
  if (h->deferred) {
    // the previous batch (the other slot) left its write-back to this one
    fc.prev = &h->deferred_b;
    fc.prev_n = h->deferred_n;
    fc.prev_fast = h->defer_flush >= 2 ? 1 : 0;
    fc.prev_flushed = h->ev_flushed[s ^ 1];
    fc.ev_reads_done = h->ev_reads_done;
  }
  cudaError_t e = launch_main(h->m, b, n, st, fc);
  if (e != cudaSuccess) return e;
  h->deferred = defer_own;
  if (defer_own) {
    h->deferred_b = b;
    h->deferred_n = n;
  }
  h->flush_pending[s] = true;
  h->slot_ht_mask[s] = b.ht_mask;
  h->prev_valid = true;
  h->slot = s ^ 1;
  return cudaSuccess;
}

// A batch of n <= FUSED_MAX_OPS ops as one launch in the current slot.  Its
// pages reach the host from the kernel itself, so it first orders st after
// every write-back still in flight (one could be of a page it rewrites) and
// leaves none pending.
// early_in: the batch's inputs are complete even if the kernel before it on
// st is not (see launch_fused)
cudaError_t fused_batch(bolt* h, const BatchDev& b, uint32_t n, uint64_t t0, cudaStream_t st,
                        bool early_in = false, const FusedInline* inl = nullptr) {
  const int s = h->slot;
  for (int k = 0; k < 2; k++)
    if (h->flush_pending[k]) {
      cudaError_t e = cudaStreamWaitEvent(st, h->ev_flushed[k], 0);
      if (e != cudaSuccess) return e;
      h->flush_pending[k] = false;
    }
  const BatchDev v = slot_view(h, b, n, s);
  cudaError_t e = launch_fused(h->m, v, n, t0, st, early_in, inl);
  if (e != cudaSuccess) return e;
  h->slot_ht_mask[s] = v.ht_mask;
  h->prev_valid = true;
  h->slot = s ^ 1;
  return cudaSuccess;
}

// One access batch, preparation and main part, on stream st.
cudaError_t access_batch(bolt* h, BatchDev b, uint32_t n, cudaStream_t st) {
  if (h->fused && n <= FUSED_MAX_OPS) return fused_batch(h, b, n, h->t, st);
  const BatchDev v = slot_view(h, b, n, h->slot);
  cudaError_t e = launch_prep(h->m, v, n, h->t, st);
  if (e != cudaSuccess) return e;
  return main_batch(h, v, n, st);
}

// ceil(n / w) batches of w ops (the last one ragged) over device arrays, in
// order, on stream st -- the same result as one access_batch per slice.  The
// preparation of batch j + 1 depends only on its own inputs, and its
// lookahead only on state that batch j does not change, so both run on
// st_prep while batch j's main part runs on st; slot s's buffers are reused
// two batches later, after ev_pfree[s] (recorded once the main part that
// read them is done).
cudaError_t access_batches(bolt* h, BatchDev b, uint64_t n, uint32_t w, cudaStream_t st) {
  const uint64_t nb = (n + w - 1) / w;
  auto slice = [&](uint64_t j, uint32_t& cnt) {
    BatchDev x = b;
    const uint64_t lo = j * w;
    cnt = (uint32_t)(n - lo < w ? n - lo : w);
    x.ops = b.ops + lo;
    x.keys = b.keys + lo;
    x.vin = b.vin + lo * h->vb;
    x.vout = b.vout + lo * h->vb;
    x.status = b.status + lo;
    return x;
  };
  if (nb == 1) {
    uint32_t cnt = 0;
    const BatchDev x = slice(0, cnt);
    cudaError_t e = access_batch(h, x, cnt, st);
    if (e == cudaSuccess) {
      h->t += cnt;
      h->batches++;
    }
    return e;
  }
  if (h->fused && w <= FUSED_MAX_OPS) {
    // small batches: one launch each, in order on st; from the second on,
    // the kernel before each is the previous batch of this call, whose own
    // start came after the caller's work, so the inputs are complete
    for (uint64_t j = 0; j < nb; j++) {
      uint32_t cnt = 0;
      const BatchDev x = slice(j, cnt);
      cudaError_t e = fused_batch(h, x, cnt, h->t, st, j > 0);
      if (e != cudaSuccess) return e;
      h->t += cnt;
      h->batches++;
    }
    return cudaSuccess;
  }
  // the inputs are ready once the caller's earlier work on st is done
  cudaError_t e = cudaEventRecord(h->ev_in, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->st_prep, h->ev_in, 0);
  if (e != cudaSuccess) return e;
  const uint64_t t_start = h->t;
  const bool la = h->la_frac > 0.0;
  auto la_limit = [&](uint32_t cnt) {
    return (uint32_t)(h->la_frac * 2.0 * cnt + 0.5);
  };
  auto prep = [&](uint64_t j, int s) -> cudaError_t {
    uint32_t cnt = 0;
    const BatchDev x = slice(j, cnt);
    BatchDev v = slot_view(h, x, cnt, s);
    if (j >= 2) {
      cudaError_t pe = cudaStreamWaitEvent(h->st_prep, h->ev_pfree[s], 0);
      if (pe != cudaSuccess) return pe;
    }
    cudaError_t pe = launch_prep(h->m, v, cnt, t_start + j * w, h->st_prep);
    if (pe == cudaSuccess && la && j >= 1) {
      // lookahead against batch j - 1 (its key table is in the other slot):
      // the position-map search runs at once; the page reads wait until
      // batch j - 1's own page reads are done (they then overlap its
      // find/exec/evict/remap) and the flush two batches back has landed
      uint32_t pc = 0;
      const BatchDev px = slice(j - 1, pc);
      uint32_t kt = 128;
      while (kt < 2 * pc) kt <<= 1;
      const bolt::PrepSet& pp = h->s_prep[s ^ 1];
      v.la_on = 1;
      v.la_limit = la_limit(cnt);
      v.prev_kt_own = pp.kt_own;
      v.prev_keys = px.keys;
      v.prev_ops = px.ops;
      v.prev_leader = pp.leader;
      v.prev_lastw = pp.lastw;
      v.prev_rpair = pp.rpair;
      v.prev_pres = pp.pres;
      v.prev_kt_mask = kt - 1;
      pe = launch_ahead_lookup(h->m, v, cnt, h->st_prep);
      if (pe == cudaSuccess) pe = cudaStreamWaitEvent(h->st_prep, h->ev_looked[s ^ 1], 0);
      if (pe == cudaSuccess && h->flush_pending[s])
        pe = cudaStreamWaitEvent(h->st_prep, h->ev_flushed[s], 0);
      if (pe == cudaSuccess) pe = launch_ahead_gather(h->m, v, v.la_limit, h->st_prep);
    }
    if (pe == cudaSuccess) pe = cudaEventRecord(h->ev_prep[s], h->st_prep);
    return pe;
  };
  // batch j's main part is enqueued before batch j + 1's preparation, so that
  // the lookahead's wait binds to batch j's page reads (the streams still run
  // the two side by side)
  e = prep(0, h->slot);
  for (uint64_t j = 0; j < nb && e == cudaSuccess; j++) {
    const int s = h->slot;
    e = cudaStreamWaitEvent(st, h->ev_prep[s], 0);
    if (e != cudaSuccess) break;
    uint32_t cnt = 0;
    const BatchDev x = slice(j, cnt);
    BatchDev v = slot_view(h, x, cnt, s);
    v.la_on = la && j >= 1 ? 1u : 0u;
    v.la_limit = la_limit(cnt);
    // with BOLT_PARAM_DEFER_FLUSH every batch but the last leaves its
    // write-back to the next one (not with the lookahead, whose page reads
    // wait for the write-backs)
    e = main_batch(h, v, cnt, st, la, h->defer_flush > 0 && !la && j + 1 < nb);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_pfree[s], st);
    if (e != cudaSuccess) break;
    h->t += cnt;
    h->batches++;
    if (j + 1 < nb) e = prep(j + 1, s ^ 1);
  }
  return e;
}

// Order stream st after every pending page flush and forget the previous
// batch (a build rewrites every page).
void drain_flushes(bolt* h, cudaStream_t st) {
  h->deferred = false;  // a write-back never enqueued: the build rewrites every page
  for (int s = 0; s < 2; s++) {
    if (h->flush_pending[s]) {
      cudaStreamWaitEvent(st, h->ev_flushed[s], 0);
      h->flush_pending[s] = false;
    }
    // both page tables start empty (a batch clears its predecessor's table)
    cudaMemsetAsync(h->s_ht_key[s], 0xff, ((uint64_t)h->b.ht_mask + 1) * 4, st);
    cudaMemsetAsync(h->s_ht_min[s], 0xff, ((uint64_t)h->b.ht_mask + 1) * 4, st);
  }
  h->prev_valid = false;
  h->slot = 0;
}

// The start of every build: the handle's earlier work done, the map state
// reset, the working keys derived from the seed.
int build_prologue(bolt* h, uint64_t seed, cudaStream_t st) {
  // work the handle left on another stream (a caller stream of the access
  // calls) finishes before the build resets the map
  if (h->last_st && h->last_st != st && sync_all(h) != cudaSuccess) return BOLT_E_CUDA;
  drain_flushes(h, st);
  MapDev& m = h->m;
  const bolt_info_t& I = h->info;
  h->initialized = false;
  h->poisoned = false;
  // reset the map state
  cudaMemsetAsync(m.load, 0, (I.B / 4 + 2) * 4, st);
  cudaMemsetAsync(m.rowcnt, 0, (I.rows / 4 + 2) * 4, st);
  cudaMemsetAsync(m.pm_meta, 0, I.rows * I.R * 4, st);
  cudaMemsetAsync(m.vs_live, 0, I.vs_cap, st);
  cudaMemsetAsync(m.revcnt, 0, (I.M / 4 + 2) * 4, st);
  cudaMemsetAsync(m.version, 0, I.M * 8, st);
  cudaMemsetAsync(m.err, 0, 4, st);
  cudaMemsetAsync(m.stat, 0, ST_WORDS * 8, st);
  cudaMemsetAsync(m.trace_len, 0, 8, st);
  // keys -> K_prf, K_enc
  k_kdf<<<1, 1, 0, st>>>(seed, h->d_kdf);
  count_launch();
  uint32_t kw[16];
  cudaError_t e = cudaMemcpyAsync(kw, h->d_kdf, sizeof kw, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return BOLT_E_CUDA;
  for (int i = 0; i < 8; i++) {
    m.kprf[i] = kw[i];
    m.kenc[i] = kw[8 + i];
  }
  return BOLT_OK;
}

// The end of every build: the error word (and the key check's flag) read
// back, the handle poisoned or made ready.
int build_epilogue(bolt* h, cudaStream_t st, bool check) {
  uint32_t err = 0;
  h->last_st = st;
  int rc = read_err(h, &err);
  if (rc) return rc;
  if (check) {
    uint32_t flag = 0;
    if (cudaMemcpy(&flag, h->d_flag, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return BOLT_E_CUDA;
    if (flag) return BOLT_E_DUPKEY;
  }
  rc = err_to_rc(err);
  if (rc) {
    h->poisoned = true;
    return rc;
  }
  h->t = 0;
  h->batches = 0;
  h->initialized = true;
  return BOLT_OK;
}

int init_impl(bolt* h, const uint64_t* d_keys, const uint8_t* d_vals, uint64_t n, uint64_t seed,
              cudaStream_t st, BuildScratch& bs, cudaEvent_t vals_ready = nullptr) {
  ProfSpan whole(P_BUILD, st);
  int rc = build_prologue(h, seed, st);
  if (rc) return rc;
  MapDev& m = h->m;
  const int sms = sm_count();
  bs.log_tile = h->sort_log_tile;
  // key uniqueness (Sec. 2.1).  With the key-sort buffer available it is a
  // hashed check on the side stream (below); otherwise a sorted copy of the
  // keys in line, flagging equal neighbours.
  const bool check = h->check_keys && n > 1;
  const bool side = check && bs.keysort && h->st2;
  if (check) cudaMemsetAsync(h->d_flag, 0, 4, st);
  auto key_check = [&](cudaStream_t ks, uint64_t* kbuf) -> cudaError_t {
    ProfSpan ps(P_KEYCHECK, ks);
    k_copy_keys<<<sms * 8, 256, 0, ks>>>(d_keys, n, bs.tag_cap, kbuf);
    count_launch();
    cudaError_t ke = sort_tags_u64(kbuf, bs.tag_cap, bs.log_tile, ks, P_KSORT_GLOBAL, P_KSORT_TILE);
    if (ke != cudaSuccess) return ke;
    k_adjacent_equal<<<sms * 8, 256, 0, ks>>>(kbuf, n, h->d_flag);
    count_launch();
    return cudaGetLastError();
  };
  cudaError_t e = cudaSuccess;
  if (check && !side) {
    e = key_check(st, bs.tags);  // in line, before the build reuses `tags`
    if (e != cudaSuccess) return BOLT_E_CUDA;
  }
  bs.prf_rounds = h->prf_rounds;
  e = launch_build(m, d_keys, d_vals, n, bs, st, vals_ready, h->st2, h->ev_pfork, h->ev_pjoin,
                   h->st_fl, h->ev_evicted, h->ev_flushed);
  if (e != cudaSuccess) return BOLT_E_CUDA;
  if (side) {
    // hashed check on the side stream after the placement, both beside the
    // page build (its kernel waits on the copy engine; its host traffic goes
    // through the copy engine, not through the SMs), in a table of its own
    ProfSpan ps(P_KEYCHECK, h->st2);
    unsigned long long* salt_count = reinterpret_cast<unsigned long long*>(h->d_kdf + 2);
    cudaMemsetAsync(bs.keysort, 0, 2 * bs.tag_cap * sizeof(uint64_t), h->st2);
    cudaMemsetAsync(salt_count, 0, sizeof(unsigned long long), h->st2);
    k_dup_insert<<<sms * 8, 256, 0, h->st2>>>(d_keys, n, bs.keysort, bs.keysort + bs.tag_cap,
                                               bs.tag_cap, h->d_flag, salt_count);
    count_launch();
    cudaEventRecord(h->ev_join, h->st2);
    cudaStreamWaitEvent(st, h->ev_join, 0);
  }
  return build_epilogue(h, st, check);
}

}  // namespace

extern "C" {

const char* bolt_strerror(int code) {
  switch (code) {
    case BOLT_OK: return "ok";
    case BOLT_E_ARG: return "invalid argument";
    case BOLT_E_NOMEM: return "out of device or pinned host memory (or HBM budget too small)";
    case BOLT_E_OVERFLOW: return "capacity bound exceeded (map poisoned until re-init)";
    case BOLT_E_STATE: return "map not initialised or poisoned";
    case BOLT_E_DUPKEY: return "duplicate keys in bolt_init";
    case BOLT_E_CUDA: return "CUDA runtime error";
    case BOLT_E_TIMEOUT: return "bounded device wait timed out";
    case BOLT_E_INTEGRITY: return "a host page failed its integrity tag (map poisoned until re-init)";
    case BOLT_E_INTERNAL: return "internal consistency check failed";
    default: return "unknown error";
  }
}

int bolt_plan(uint64_t N, uint32_t key_bytes, uint32_t val_bytes, uint64_t hbm_budget,
              double alpha, uint32_t c, bolt_info_t* out) {
  if (!out || (key_bytes != 8 && key_bytes != 4) || val_bytes < 8 || val_bytes % 8 ||
      val_bytes > 504 || N < 64 || N > (1ull << 31) || c < 1 || c > 32)
    return BOLT_E_ARG;
  bolt tmp;
  tmp.N = N;
  tmp.vb = val_bytes;
  tmp.hbm_budget = hbm_budget;
  tmp.alpha_override = alpha;
  tmp.c = c;
  int rc = choose_plan(&tmp, out);
  if (rc == BOLT_OK) out->key_bytes = key_bytes;
  return rc;
}

int bolt_create(uint64_t N, uint32_t key_bytes, uint32_t val_bytes, uint64_t hbm_budget,
                bolt_t** out) {
  if (!out || (key_bytes != 8 && key_bytes != 4) || val_bytes < 8 || val_bytes % 8 ||
      val_bytes > 504 || N < 64 || N > (1ull << 31))
    return BOLT_E_ARG;
  *out = nullptr;
  bolt* h = new (std::nothrow) bolt();
  if (!h) return BOLT_E_NOMEM;
  h->N = N;
  h->kb = key_bytes;
  h->vb = val_bytes;
  h->hbm_budget = hbm_budget;
  cudaError_t e = cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->st2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_pfork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_pjoin, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->st_fl, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->st_prep, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->st_out, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_reads_done, cudaEventDisableTiming);
  for (int s = 0; s < 2 && e == cudaSuccess; s++) {
    e = cudaEventCreateWithFlags(&h->ev_looked[s], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_ioready[s], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_h2d[s], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_d2h[s], cudaEventDisableTiming);
  }
  for (int s = 0; s < 2 && e == cudaSuccess; s++) {
    e = cudaEventCreateWithFlags(&h->ev_evicted[s], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_flushed[s], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_prep[s], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_pfree[s], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    destroy_streams(h);
    delete h;
    return BOLT_E_CUDA;
  }
  void* p = nullptr;
  const uint64_t set_bytes = MAXB * (1 + 8 + 2 * (uint64_t)val_bytes + 1);
  const uint64_t res_bytes = (FUSED_MAX_OPS * (val_bytes + 1) + 4 + 6) / 7 * 8;
  e = cudaHostAlloc(&p, 2 * set_bytes + 64 + res_bytes, cudaHostAllocMapped);
  void* pd = nullptr;
  if (e == cudaSuccess && cudaHostGetDevicePointer(&pd, p, 0) != cudaSuccess) {
    cudaFreeHost(p);
    e = cudaErrorMemoryAllocation;
  }
  if (e != cudaSuccess) {
    destroy_streams(h);
    delete h;
    return BOLT_E_NOMEM;
  }
  // the fused small-batch call reads and writes this staging from the device
  h->io_dev_delta = static_cast<uint8_t*>(pd) - static_cast<uint8_t*>(p);
  // the same two parts as a device I/O set (MAXB is a multiple of 8)
  uint8_t* q = static_cast<uint8_t*>(p);
  for (int s = 0; s < 2; s++) {
    bolt::IoSet& io = h->h_io[s];
    io.keys = reinterpret_cast<uint64_t*>(q); q += MAXB * 8;
    io.vin = q; q += (uint64_t)MAXB * val_bytes;
    io.ops = q; q += MAXB;
    io.vout = q; q += (uint64_t)MAXB * val_bytes;
    io.status = q; q += MAXB;
  }
  h->h_keys = h->h_io[0].keys;
  h->h_vin = h->h_io[0].vin;
  h->h_vout = h->h_io[0].vout;
  h->h_ops = h->h_io[0].ops;
  h->h_status = h->h_io[0].status;
  h->h_err = reinterpret_cast<uint32_t*>((reinterpret_cast<uintptr_t>(q) + 7) & ~uintptr_t(7));
  h->h_res = reinterpret_cast<uint64_t*>(h->h_err + 2);
  int rc = alloc_state(h);
  if (rc) {
    cudaFreeHost(h->h_keys);
    destroy_streams(h);
    delete h;
    return rc;
  }
  *out = h;
  return BOLT_OK;
}

int bolt_destroy(bolt_t* h) {
  if (!h) return BOLT_OK;
  free_state(h);
  if (h->h_keys) cudaFreeHost(h->h_keys);
  destroy_streams(h);
  delete h;
  return BOLT_OK;
}

int bolt_set_param(bolt_t* h, int which, double v) {
  if (!h) return BOLT_E_ARG;
  switch (which) {
    case BOLT_PARAM_ALPHA:
      if (!(v >= 0.0 && v < 1.0)) return BOLT_E_ARG;
      h->alpha_override = v;
      break;
    case BOLT_PARAM_C:
      if (!(v >= 1.0 && v <= 32.0)) return BOLT_E_ARG;  // lmax <= 32 is checked by the plan
      h->c = (uint32_t)v;
      break;
    case BOLT_PARAM_TRACE:
      h->trace_on = v != 0.0;
      h->m.trace_on = h->trace_on ? 1 : 0;
      return BOLT_OK;
    case BOLT_PARAM_BATCH:
      if (!(v >= 1.0 && v <= (double)h->cap_batch)) return BOLT_E_ARG;
      h->batch_width = (uint32_t)v;
      return BOLT_OK;
    case BOLT_PARAM_LOOKAHEAD:
      if (!(v >= 0.0 && v <= 1.0)) return BOLT_E_ARG;
      if (v > 0.0 && h->integrity) return BOLT_E_ARG;  // ahead reads are not verified
      h->la_frac = v;
      return BOLT_OK;
    case BOLT_PARAM_DEFER_FLUSH:
      if (!(v == 0.0 || v == 1.0 || v == 2.0)) return BOLT_E_ARG;
      h->defer_flush = (int)v;
      return BOLT_OK;
    case BOLT_PARAM_FUSED:
      if (!(v == 0.0 || v == 1.0)) return BOLT_E_ARG;
      h->fused = v != 0.0;
      return BOLT_OK;
    case BOLT_PARAM_INTEGRITY:
      if (!(v == 0.0 || v == 1.0)) return BOLT_E_ARG;
      if (v != 0.0 && h->la_frac > 0.0) return BOLT_E_ARG;
      h->integrity = v != 0.0;
      break;
    case BOLT_PARAM_ROUNDS_PRF:
      if (!(v == 0.0 || v == 1.0 || v == 2.0)) return BOLT_E_ARG;
      h->prf_rounds = (int)v;
      return BOLT_OK;
    case BOLT_PARAM_SPIN_LIMIT:
      if (!(v >= 0.0 && v <= (double)(1u << 22))) return BOLT_E_ARG;
      h->spin_limit = (uint32_t)v;
      h->m.spin_limit = h->spin_limit;
      return BOLT_OK;
    case BOLT_PARAM_BATCH_CAP:
      if (!(v >= 1.0 && v <= (double)MAXB)) return BOLT_E_ARG;
      h->cap_batch = (uint32_t)v;
      if (h->batch_width > h->cap_batch) h->batch_width = h->cap_batch;
      break;
    case BOLT_PARAM_TRACE_CAP:
      if (!(v >= 1.0 && v <= (double)(1ull << 32))) return BOLT_E_ARG;
      h->trace_cap = (uint64_t)v;
      break;
    case BOLT_PARAM_CHECK_KEYS:
      h->check_keys = v != 0.0;
      return BOLT_OK;
    case BOLT_PARAM_PROFILE:
      h->prof.on = v != 0.0;
      return BOLT_OK;
    default:
      return BOLT_E_ARG;
  }
  free_state(h);
  return alloc_state(h);
}

int bolt_get_info(const bolt_t* h, bolt_info_t* out) {
  if (!h || !out) return BOLT_E_ARG;
  *out = h->info;
  return BOLT_OK;
}

int bolt_init_device(bolt_t* h, const void* d_keys, const void* d_vals, uint64_t n, uint64_t seed,
                     void* stream) {
  if (!h || !h->allocated || n > h->N || (n && (!d_keys || !d_vals))) return BOLT_E_ARG;
  ProfScope prof_scope(h);
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : h->st;
  int rc = grow_build_scratch(h, n);
  if (rc) return rc;
  return init_impl(h, static_cast<const uint64_t*>(d_keys), static_cast<const uint8_t*>(d_vals), n,
                   seed, st, h->bs);
}

int bolt_init(bolt_t* h, const void* keys, const void* vals, uint64_t n, uint64_t seed) {
  if (!h || !h->allocated || n > h->N || (n && (!keys || !vals))) return BOLT_E_ARG;
  ProfScope prof_scope(h);
  const uint64_t cap = n > 0 ? n : 1;
  if (h->in_cap < cap) {
    cudaFree(h->in_keys);
    cudaFree(h->in_vals);
    h->in_keys = nullptr;
    h->in_vals = nullptr;
    h->in_cap = 0;
    cudaError_t e = cudaMalloc(&h->in_keys, cap * 8);
    if (e == cudaSuccess) e = cudaMalloc(&h->in_vals, cap * h->vb);
    if (e != cudaSuccess) return cuda_fail(e);
    h->in_cap = cap;
  }
  int rc = grow_build_scratch(h, n);
  if (rc) return rc;
  if (h->last_st && h->last_st != h->st && sync_all(h) != cudaSuccess) return BOLT_E_CUDA;
  // 4-byte keys are zero-extended: the map holds every key as a uint64
  std::vector<uint64_t> wide;
  if (n && h->kb == 4) {
    wide.resize(n);
    const uint32_t* k32 = static_cast<const uint32_t*>(keys);
    for (uint64_t i = 0; i < n; i++) wide[i] = k32[i];
    keys = wide.data();
  }
  if (n) {
    // keys first (the PRF phase reads them); the values, read only by the
    // placement and the page build, arrive on the side stream meanwhile
    cudaError_t e = cudaMemcpyAsync(h->in_keys, keys, n * 8, cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->in_vals, vals, n * h->vb, cudaMemcpyHostToDevice, h->st2);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_in, h->st2);
    if (e != cudaSuccess) return BOLT_E_CUDA;
  }
  return init_impl(h, h->in_keys, h->in_vals, n, seed, h->st, h->bs, n ? h->ev_in : nullptr);
}

int bolt_prepare_device(bolt_t* h, const void* d_keys, const void* d_vals, uint64_t n,
                        uint64_t seed, const bolt_image_t* out, void* stream) {
  if (!h || !h->allocated || !out || !out->counts || n > h->N ||
      (n && (!out->keys || !out->vals || !out->pairs || !out->rows)))
    return BOLT_E_ARG;
  int rc = bolt_init_device(h, d_keys, d_vals, n, seed, stream);
  if (rc) return rc;
  ProfScope prof_scope(h);
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : h->st;
  // the build's placement is still in its scratch: dest, rows, pairs
  cudaError_t e = launch_image_export(h->m, static_cast<const uint64_t*>(d_keys),
                                      static_cast<const uint8_t*>(d_vals), n, h->bs, st, out->keys,
                                      static_cast<uint8_t*>(out->vals), out->pairs, out->rows,
                                      out->counts);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? BOLT_OK : BOLT_E_CUDA;
}

int bolt_init_prepared(bolt_t* h, const bolt_image_t* img, uint64_t n, uint64_t seed,
                       void* stream) {
  if (!h || !h->allocated || !img || !img->counts || n > h->N ||
      (n && (!img->keys || !img->vals || !img->pairs || !img->rows)))
    return BOLT_E_ARG;
  ProfScope prof_scope(h);
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : h->st;
  int rc = grow_build_scratch(h, n);
  if (rc) return rc;
  ProfSpan whole(P_BUILD, st);
  rc = build_prologue(h, seed, st);
  if (rc) return rc;
  cudaError_t e = launch_image_load(h->m, img->keys, static_cast<const uint8_t*>(img->vals),
                                    img->pairs, img->rows, img->counts, n, h->bs, st, h->st2,
                                    h->ev_pfork, h->ev_pjoin, h->st_fl, h->ev_evicted,
                                    h->ev_flushed);
  if (e != cudaSuccess) return BOLT_E_CUDA;
  return build_epilogue(h, st, false);
}

int bolt_sync(bolt_t* h) {
  if (!h) return BOLT_E_ARG;
  uint32_t err = 0;
  int rc = read_err(h, &err);
  if (rc) return rc;
  rc = err_to_rc(err);
  if (rc) h->poisoned = true;
  return rc;
}

int bolt_access_device(bolt_t* h, const uint8_t* d_ops, const void* d_keys, const void* d_vals_in,
                       void* d_vals_out, uint8_t* d_status, uint64_t n, void* stream) {
  if (!h) return BOLT_E_ARG;
  if (!h->initialized || h->poisoned) return BOLT_E_STATE;
  if (n == 0) return BOLT_OK;
  if (n > h->cap_batch || !d_ops || !d_keys || !d_vals_in || !d_vals_out) return BOLT_E_ARG;
  ProfScope prof_scope(h);
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : h->st;
  BatchDev b = h->b;
  b.ops = const_cast<uint8_t*>(d_ops);
  b.keys = static_cast<uint64_t*>(const_cast<void*>(d_keys));
  b.vin = static_cast<uint8_t*>(const_cast<void*>(d_vals_in));
  b.vout = static_cast<uint8_t*>(d_vals_out);
  if (d_status) b.status = d_status;
  if (h->last_st != st) {
    // order this batch after work the handle left on another stream
    if (h->last_st && sync_all(h) != cudaSuccess) return BOLT_E_CUDA;
    h->last_st = st;
  }
  cudaError_t e = access_batch(h, b, (uint32_t)n, st);
  if (e != cudaSuccess) return BOLT_E_CUDA;
  h->t += n;
  h->batches++;
  return BOLT_OK;
}

int bolt_access_device_batches(bolt_t* h, const uint8_t* d_ops, const void* d_keys,
                               const void* d_vals_in, void* d_vals_out, uint8_t* d_status,
                               uint64_t n, uint32_t width, void* stream) {
  if (!h) return BOLT_E_ARG;
  if (!h->initialized || h->poisoned) return BOLT_E_STATE;
  if (n == 0) return BOLT_OK;
  if (width == 0) width = h->batch_width;
  if (width > h->cap_batch || !d_ops || !d_keys || !d_vals_in || !d_vals_out || !d_status)
    return BOLT_E_ARG;
  ProfScope prof_scope(h);
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : h->st;
  BatchDev b = h->b;
  b.ops = const_cast<uint8_t*>(d_ops);
  b.keys = static_cast<uint64_t*>(const_cast<void*>(d_keys));
  b.vin = static_cast<uint8_t*>(const_cast<void*>(d_vals_in));
  b.vout = static_cast<uint8_t*>(d_vals_out);
  b.status = d_status;
  if (h->last_st != st) {
    if (h->last_st && sync_all(h) != cudaSuccess) return BOLT_E_CUDA;
    h->last_st = st;
  }
  return access_batches(h, b, n, width, st) == cudaSuccess ? BOLT_OK : BOLT_E_CUDA;
}

static bool host_pinned(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

// Chunks of up to cap_batch ops (whole batches of batch_width), alternating
// between two device I/O sets; each chunk is one access_batches call.  A
// chunk whose arrays are pageable, or small, is packed through pinned
// staging so that its inputs and its results each cross the link in one copy
// (io_packed); large pinned caller arrays are copied directly.  With several
// chunks the next chunk's inputs are staged and the previous chunk's results
// copied out while a chunk runs; a single chunk keeps every copy on the
// batch stream.
constexpr uint64_t PACK_MAX_BYTES = 64 << 10;

int bolt_access(bolt_t* h, const uint8_t* ops, const void* keys, const void* vals_in,
                void* vals_out, uint8_t* status_out, uint64_t n) {
  if (!h) return BOLT_E_ARG;
  if (!h->initialized || h->poisoned) return BOLT_E_STATE;
  if (n == 0) return BOLT_OK;
  if (!ops || !keys || !vals_in || !vals_out) return BOLT_E_ARG;
  uint8_t bad = 0;
  for (uint64_t i = 0; i < n; i++) bad |= (uint8_t)(ops[i] > BOLT_DEL);
  if (bad) return BOLT_E_ARG;
  ProfScope prof_scope(h);
  const uint64_t vb = h->vb;
  const uint8_t* kin = static_cast<const uint8_t*>(keys);
  const uint8_t* vin = static_cast<const uint8_t*>(vals_in);
  uint8_t* vout = static_cast<uint8_t*>(vals_out);
  cudaStream_t st = h->st;
  if (h->last_st != st) {
    if (h->last_st && sync_all(h) != cudaSuccess) return BOLT_E_CUDA;
    h->last_st = st;
  }
  const uint32_t w = h->batch_width;
  if (h->fused && n <= FUSED_MAX_OPS && n <= w && n <= h->cap_batch) {
    // one small batch: a single fused launch that takes its inputs in its
    // parameters (or, when they do not fit, from the pinned staging) and
    // writes its results and the error word back to the staging, so the
    // call is one launch and one stream wait (no copies)
    const IoPacked hp = io_packed(h->h_io[0], n, vb);
    const IoPacked dp = io_packed(h->d_io[0], n, vb);
    FusedInline fi;
    const uint64_t in_bytes = n * (9 + vb);
    const bool inl = in_bytes <= FUSED_INLINE_MAX;
    uint8_t* at = inl ? reinterpret_cast<uint8_t*>(fi.d) : reinterpret_cast<uint8_t*>(hp.keys);
    if (inl) {
      fi.bytes = (uint32_t)in_bytes;
      fi.d[(in_bytes - 1) / 16] = make_uint4(0, 0, 0, 0);  // a defined tail
    }
    uint64_t* kdst = reinterpret_cast<uint64_t*>(at);
    if (h->kb == 4) {
      const uint32_t* k32 = reinterpret_cast<const uint32_t*>(kin);
      for (uint64_t i = 0; i < n; i++) kdst[i] = k32[i];
    } else {
      std::memcpy(kdst, kin, n * 8);
    }
    std::memcpy(at + n * 8, vin, n * vb);
    std::memcpy(at + n * (8 + vb), ops, n);
    BatchDev b = h->b;
    b.ops = dp.ops;
    b.keys = dp.keys;
    b.vin = dp.vin;
    b.vout = dp.vout;
    b.status = dp.status;
    b.h_in = inl ? nullptr : reinterpret_cast<const uint8_t*>(hp.keys) + h->io_dev_delta;
    // the result words start untagged; the kernel tags each one it writes
    const uint64_t res_words = (n * (vb + 1) + 4 + 6) / 7;
    volatile uint64_t* res = h->h_res;
    for (uint64_t w = 0; w < res_words; w++) res[w] = 0;
    b.h_res = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(h->h_res) + h->io_dev_delta);
    b.res_tag = ++h->done_seq % 255 + 1;
    // (the inputs are in the staging, written before the launch)
    cudaError_t e = fused_batch(h, b, (uint32_t)n, h->t, st, true, inl ? &fi : nullptr);
    if (e != cudaSuccess) return BOLT_E_CUDA;
    // the wait ends when every result word carries the call's tag (each is
    // one 8-byte store the host sees whole: no completion word, and no
    // system-scope fence in the kernel before one); if they have not all come
    // within seconds, wait for the stream and let its error (or the missing
    // words) speak
    const uint64_t tag = (uint64_t)b.res_tag << 56;
    uint64_t got = 0;
    const auto t_wait = std::chrono::steady_clock::now();
    for (uint32_t spin = 1; got < res_words; spin++) {
      while (got < res_words && (res[got] & (0xffull << 56)) == tag) got++;
      if (got < res_words && (spin & 4095) == 0 &&
          std::chrono::steady_clock::now() - t_wait > std::chrono::seconds(5)) {
        if (cudaStreamSynchronize(st) != cudaSuccess) return BOLT_E_CUDA;
        while (got < res_words && (res[got] & (0xffull << 56)) == tag) got++;
        if (got < res_words) return BOLT_E_INTERNAL;
      }
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    h->t += n;
    h->batches++;
    // the stream vout | status | error word, 7 bytes per word
    const uint64_t nv = n * vb;
    uint32_t err = 0;
    for (uint64_t w = 0; w < res_words; w++) {
      const uint64_t v = res[w];
      for (uint64_t k = 0, i = 7 * w; k < 7; k++, i++) {
        const uint8_t byte = (uint8_t)(v >> (8 * k));
        if (i < nv) vout[i] = byte;
        else if (i < nv + n) { if (status_out) status_out[i - nv] = byte; }
        else if (i < nv + n + 4) err |= (uint32_t)byte << (8 * (i - nv - n));
      }
    }
    const int rc = err_to_rc(err);
    if (rc) h->poisoned = true;
    return rc;
  }
  const uint64_t chunk = (uint64_t)(h->cap_batch / w) * w;
  const bool single = n <= chunk;
  // several chunks: host<->device copies run beside the batches on st --
  // inputs on st2 (idle outside bolt_init), outputs on st_out -- so chunk
  // k + 1's inputs arrive and chunk k - 1's outputs leave while chunk k runs
  cudaStream_t cs = single ? st : h->st2, co = single ? st : h->st_out;
  // whether the caller's arrays can feed the copy engine directly (only
  // asked where a chunk is too large to pack)
  const bool pin_in = h->kb == 8 && n * (9 + vb) > PACK_MAX_BYTES && host_pinned(ops) &&
                      host_pinned(keys) && host_pinned(vals_in);
  const bool pin_out = n * (vb + 1) > PACK_MAX_BYTES && host_pinned(vals_out) &&
                       (!status_out || host_pinned(status_out));
  bool pending[2] = {false, false};
  uint64_t plo[2] = {0, 0}, pcnt[2] = {0, 0};
  // a packed chunk's results, from staging to the caller's arrays
  auto copy_out = [&](int s) -> int {
    if (!pending[s]) return BOLT_OK;
    pending[s] = false;
    if (cudaEventSynchronize(h->ev_d2h[s]) != cudaSuccess) return BOLT_E_CUDA;
    const IoPacked hp = io_packed(h->h_io[s], pcnt[s], vb);
    std::memcpy(vout + plo[s] * vb, hp.vout, pcnt[s] * vb);
    if (status_out) std::memcpy(status_out + plo[s], hp.status, pcnt[s]);
    return BOLT_OK;
  };
  cudaError_t e = cudaSuccess;
  int k = 0;
  for (uint64_t lo = 0; lo < n && e == cudaSuccess; lo += chunk, k ^= 1) {
    const uint64_t cnt = n - lo < chunk ? n - lo : chunk;
    const bolt::IoSet& d = h->d_io[k];
    const IoPacked dp = io_packed(d, cnt, vb);
    const bool pack_in = !pin_in || cnt * (9 + vb) <= PACK_MAX_BYTES;
    const bool pack_out = !pin_out || cnt * (vb + 1) <= PACK_MAX_BYTES;
    BatchDev b = h->b;
    // the device set was last used by chunk k - 2: its batches and output copy
    e = lo >= 2 * chunk ? cudaStreamWaitEvent(cs, h->ev_d2h[k], 0) : cudaSuccess;
    if (e != cudaSuccess) break;
    if (pack_in) {
      // the staging set was last read by the copy two chunks back
      if (cudaEventSynchronize(h->ev_h2d[k]) != cudaSuccess) return BOLT_E_CUDA;
      const IoPacked hp = io_packed(h->h_io[k], cnt, vb);
      if (h->kb == 4) {
        // zero-extended into the uint64 keys the map holds
        const uint32_t* k32 = reinterpret_cast<const uint32_t*>(kin) + lo;
        for (uint64_t i = 0; i < cnt; i++) hp.keys[i] = k32[i];
      } else {
        std::memcpy(hp.keys, kin + lo * 8, cnt * 8);
      }
      std::memcpy(hp.vin, vin + lo * vb, cnt * vb);
      std::memcpy(hp.ops, ops + lo, cnt);
      e = cudaMemcpyAsync(dp.keys, hp.keys, dp.in_bytes, cudaMemcpyHostToDevice, cs);
      b.ops = dp.ops;
      b.keys = dp.keys;
      b.vin = dp.vin;
    } else {
      e = cudaMemcpyAsync(d.ops, ops + lo, cnt, cudaMemcpyHostToDevice, cs);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d.keys, kin + lo * 8, cnt * 8, cudaMemcpyHostToDevice, cs);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d.vin, vin + lo * vb, cnt * vb, cudaMemcpyHostToDevice, cs);
      b.ops = d.ops;
      b.keys = d.keys;
      b.vin = d.vin;
    }
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_h2d[k], cs);
    if (e == cudaSuccess && cs != st) e = cudaStreamWaitEvent(st, h->ev_h2d[k], 0);
    if (e != cudaSuccess) break;
    b.vout = pack_out ? dp.vout : d.vout;
    b.status = pack_out ? dp.status : d.status;
    e = access_batches(h, b, cnt, w, st);
    if (e == cudaSuccess && co != st) {
      e = cudaEventRecord(h->ev_ioready[k], st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(co, h->ev_ioready[k], 0);
    }
    if (e != cudaSuccess) break;
    if (pack_out) {
      const IoPacked hp = io_packed(h->h_io[k], cnt, vb);
      e = cudaMemcpyAsync(hp.vout, dp.vout, dp.out_bytes, cudaMemcpyDeviceToHost, co);
    } else {
      e = cudaMemcpyAsync(vout + lo * vb, d.vout, cnt * vb, cudaMemcpyDeviceToHost, co);
      if (e == cudaSuccess && status_out)
        e = cudaMemcpyAsync(status_out + lo, d.status, cnt, cudaMemcpyDeviceToHost, co);
    }
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_d2h[k], co);
    if (e != cudaSuccess) break;
    // the previous chunk's results, while this one runs
    int rc = copy_out(k ^ 1);
    if (rc) return rc;
    pending[k] = pack_out;
    plo[k] = lo;
    pcnt[k] = cnt;
  }
  if (e != cudaSuccess) return BOLT_E_CUDA;
  // the error word rides behind the last batch on st, so one wait covers it
  e = cudaMemcpyAsync(h->h_err, h->m.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  for (int s = 0; s < 2; s++) {
    int rc = copy_out(s ^ k);
    if (rc) return rc;
  }
  if (sync_all(h) != cudaSuccess || e != cudaSuccess) return BOLT_E_CUDA;
  const int rc = err_to_rc(*h->h_err);
  if (rc) h->poisoned = true;
  return rc;
}

int bolt_read_pages(bolt_t* h, uint64_t first, uint64_t count, void* dst) {
  if (!h || !h->allocated || !dst || first > h->info.M || count > h->info.M - first)
    return BOLT_E_ARG;
  if (sync_all(h) != cudaSuccess) return BOLT_E_CUDA;
  std::memcpy(dst, h->pages_host + first * h->info.page_bytes, count * h->info.page_bytes);
  return BOLT_OK;
}

int bolt_write_pages(bolt_t* h, uint64_t first, uint64_t count, const void* src) {
  if (!h || !h->allocated || !src || first > h->info.M || count > h->info.M - first)
    return BOLT_E_ARG;
  if (sync_all(h) != cudaSuccess) return BOLT_E_CUDA;
  std::memcpy(h->pages_host + first * h->info.page_bytes, src, count * h->info.page_bytes);
  return BOLT_OK;
}

int bolt_read_trace(bolt_t* h, uint32_t* dst, uint64_t cap, uint64_t* len) {
  if (!h || !h->allocated || !len || (cap && !dst)) return BOLT_E_ARG;
  unsigned long long tl = 0;
  if (sync_all(h) != cudaSuccess) return BOLT_E_CUDA;
  cudaError_t e = cudaMemcpyAsync(&tl, h->m.trace_len, 8, cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return BOLT_E_CUDA;
  uint64_t stored = tl < h->m.trace_cap ? tl : h->m.trace_cap;
  uint64_t ncopy = stored < cap ? stored : cap;
  if (ncopy) {
    e = cudaMemcpy(dst, h->m.trace, ncopy * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return BOLT_E_CUDA;
  }
  *len = tl;  // may exceed the capacity: entries beyond it were dropped
  cudaMemsetAsync(h->m.trace_len, 0, 8, h->st);
  if (cudaStreamSynchronize(h->st) != cudaSuccess) return BOLT_E_CUDA;
  return BOLT_OK;
}

int bolt_read_loads(bolt_t* h, uint8_t* dst) {
  if (!h || !h->allocated || !dst) return BOLT_E_ARG;
  if (sync_all(h) != cudaSuccess) return BOLT_E_CUDA;
  return cudaMemcpy(dst, h->m.load, h->info.B, cudaMemcpyDeviceToHost) == cudaSuccess
             ? BOLT_OK : BOLT_E_CUDA;
}

int bolt_read_rowcounts(bolt_t* h, uint8_t* dst) {
  if (!h || !h->allocated || !dst) return BOLT_E_ARG;
  if (sync_all(h) != cudaSuccess) return BOLT_E_CUDA;
  return cudaMemcpy(dst, h->m.rowcnt, h->info.rows, cudaMemcpyDeviceToHost) == cudaSuccess
             ? BOLT_OK : BOLT_E_CUDA;
}

int bolt_read_profile(bolt_t* h, bolt_profile_t* out, int reset) {
  if (!h || !out) return BOLT_E_ARG;
  if (sync_all(h) != cudaSuccess) return BOLT_E_CUDA;
  Prof& p = h->prof;
  for (const Prof::Span& s : p.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(s.b) == cudaSuccess && cudaEventElapsedTime(&ms, s.a, s.b) == cudaSuccess) {
      p.ms[s.cls] += ms;
      p.count[s.cls] += 1;
    }
    cudaEventDestroy(s.a);
    cudaEventDestroy(s.b);
  }
  p.pending.clear();
  std::memset(out, 0, sizeof *out);
  out->launches = p.launches;
  for (int c = 0; c < BOLT_PROF_CLASSES && c < P_NCLASS; c++) {
    out->spans[c] = p.count[c];
    out->ms[c] = p.ms[c];
  }
  if (reset) {
    p.launches = 0;
    for (int c = 0; c < P_NCLASS; c++) {
      p.ms[c] = 0.0;
      p.count[c] = 0;
    }
  }
  return BOLT_OK;
}

int bolt_get_stats(bolt_t* h, bolt_stats_t* out) {
  if (!h || !out) return BOLT_E_ARG;
  std::memset(out, 0, sizeof *out);
  out->ops = h->t;
  out->batches = h->batches;
  if (!h->allocated) return BOLT_OK;
  const bolt_info_t& I = h->info;
  std::vector<uint8_t> loads(I.B), rows(I.rows), rc(I.M);
  if (bolt_read_loads(h, loads.data()) || bolt_read_rowcounts(h, rows.data())) return BOLT_E_CUDA;
  if (cudaMemcpy(rc.data(), h->m.revcnt, I.M, cudaMemcpyDeviceToHost) != cudaSuccess)
    return BOLT_E_CUDA;
  for (uint64_t b = 0; b < I.B; b++) {
    if (b < I.K) out->n_hbm += loads[b];
    if (loads[b] > out->max_load) out->max_load = loads[b];
  }
  for (uint64_t r = 0; r < I.rows; r++)
    if (rows[r] > out->max_row) out->max_row = rows[r];
  for (uint64_t q = 0; q < I.M; q++) out->n_stash += rc[q];
  unsigned long long tl = 0, st[ST_WORDS] = {};
  if (cudaMemcpy(&tl, h->m.trace_len, 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(st, h->m.stat, sizeof st, cudaMemcpyDeviceToHost) != cudaSuccess)
    return BOLT_E_CUDA;
  out->trace_len = tl;
  // (the counts the last batch ended with: a fused batch leaves them to the
  // next batch to take into the peaks)
  out->peak_hbm = std::max(st[ST_PEAK_HBM], st[ST_HBM]);
  out->peak_stash = std::max(st[ST_PEAK_STASH], st[ST_STASH]);
  out->peak_load = (uint32_t)st[ST_PEAK_LOAD];
  if (h->initialized && !h->poisoned && (st[ST_HBM] != out->n_hbm || st[ST_STASH] != out->n_stash))
    return BOLT_E_INTERNAL;
  return BOLT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// bolt_init_device_noalloc: the device build with its scratch in a
// file-scope device array instead of memory the handle allocates.
//
// Layout of the array (offsets 256-byte aligned), for at most
// NOALLOC_MAX_RECORDS records and NOALLOC_MAX_PAGES host pages:
//   tags   u64[NOALLOC_MAX_RECORDS]   (tag buffer, a power of two >= 8192)
//   bins   u64[NOALLOC_MAX_RECORDS]
//   dest   u32[NOALLOC_MAX_RECORDS]
//   prow   u32[NOALLOC_MAX_RECORDS]
//   page_off u32[NOALLOC_MAX_PAGES + 1]
//   block_sums u32[64], counters u64[2]
namespace {

constexpr uint64_t NOALLOC_MAX_RECORDS = 1ull << 18;
constexpr uint64_t NOALLOC_MAX_PAGES = 1ull << 18;
constexpr uint64_t NA_OFF_TAGS = 0;
constexpr uint64_t NA_OFF_BINS = NA_OFF_TAGS + NOALLOC_MAX_RECORDS * 8;
constexpr uint64_t NA_OFF_DEST = NA_OFF_BINS + NOALLOC_MAX_RECORDS * 8;
constexpr uint64_t NA_OFF_PROW = NA_OFF_DEST + NOALLOC_MAX_RECORDS * 4;
constexpr uint64_t NA_OFF_PAGE = NA_OFF_PROW + NOALLOC_MAX_RECORDS * 4;
constexpr uint64_t NA_OFF_BSUM = NA_OFF_PAGE + ((NOALLOC_MAX_PAGES + 1) * 4 + 255) / 256 * 256;
constexpr uint64_t NA_BSUM_CAP = 64;
constexpr uint64_t NA_OFF_CTR = NA_OFF_BSUM + 256;
constexpr uint64_t NA_BYTES = NA_OFF_CTR + 256;
static_assert(NA_BYTES == BOLT_NOALLOC_SCRATCH_BYTES, "the header states the array's size");
static_assert(NOALLOC_MAX_RECORDS >= 8192, "tag buffer must hold one sort tile");
static_assert((NOALLOC_MAX_PAGES + 1 + 8191) / 8192 + 1 <= NA_BSUM_CAP, "block sums");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[NA_MAX_DEVICES] = {};

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (the name is only a host-side stand-in in host code).
int noalloc_scratch(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return BOLT_E_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return BOLT_E_CUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
  return BOLT_OK;
}

}  // namespace

extern "C" int bolt_init_device_noalloc(bolt_t* h, const void* d_keys, const void* d_vals,
                                        uint64_t n, uint64_t seed, void* stream) {
  if (!h || !h->allocated || n > h->N || (n && (!d_keys || !d_vals))) return BOLT_E_ARG;
  if (n > NOALLOC_MAX_RECORDS || h->info.M > NOALLOC_MAX_PAGES) return BOLT_E_ARG;
  unsigned char* base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc) return rc;
  BuildScratch s{};
  s.cap = NOALLOC_MAX_RECORDS;
  s.tag_cap = 8192;
  while (s.tag_cap < n) s.tag_cap <<= 1;
  s.tags = reinterpret_cast<uint64_t*>(base + NA_OFF_TAGS);
  s.bins = reinterpret_cast<uint64_t*>(base + NA_OFF_BINS);
  s.dest = reinterpret_cast<uint32_t*>(base + NA_OFF_DEST);
  s.prow = reinterpret_cast<uint32_t*>(base + NA_OFF_PROW);
  s.page_off = reinterpret_cast<uint32_t*>(base + NA_OFF_PAGE);
  s.block_sums = reinterpret_cast<uint32_t*>(base + NA_OFF_BSUM);
  s.block_cap = NA_BSUM_CAP;
  s.counters = reinterpret_cast<unsigned long long*>(base + NA_OFF_CTR);
  // no ProfScope: the kernel-class profiler creates events and grows a host
  // vector per span, which this call must not do (its spans are not recorded)
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : h->st;
  return init_impl(h, static_cast<const uint64_t*>(d_keys), static_cast<const uint8_t*>(d_vals), n,
                   seed, st, s);
}

// ---------------------------------------------------------------------------
// internal entry points for the serving layer (serve.cu)
namespace brt {

cudaError_t enqueue_batch(bolt* h, uint32_t n, cudaStream_t st) {
  if (h->last_st != st) {
    if (h->last_st) {
      cudaError_t e = sync_all(h);
      if (e != cudaSuccess) return e;
    }
    h->last_st = st;
  }
  cudaError_t e = access_batch(h, h->b, n, st);
  if (e != cudaSuccess) return e;
  h->t += n;
  h->batches++;
  return cudaSuccess;
}

cudaError_t enqueue_batch_packed(bolt* h, uint32_t n, cudaStream_t st) {
  const IoPacked dp = io_packed(h->d_io[0], n, h->vb);
  BatchDev saved = h->b;
  h->b.ops = dp.ops;
  h->b.keys = dp.keys;
  h->b.vin = dp.vin;
  h->b.vout = dp.vout;
  h->b.status = dp.status;
  cudaError_t e = enqueue_batch(h, n, st);
  h->b = saved;
  return e;
}

int err_rc(uint32_t err) { return err_to_rc(err); }

cudaError_t sync_handle(bolt* h) { return sync_all(h); }

uint64_t resident_estimate(const bolt_info_t& I, uint64_t cap, uint64_t trace_cap) {
  const uint64_t slots = I.rows * I.R, vb = I.val_bytes;
  uint64_t b = 4 * (I.B / 4 + 2) + 4 * (I.rows / 4 + 2) + slots * (8 + 8 + 4) +
               I.vs_cap * (8 + vb + 4 + 1 + 4) + 16 + I.M * I.lmax * 4 + 4 * (I.M / 4 + 2) +
               I.M * 8 + 4 + ST_WORDS * 8 + trace_cap * 4 + 8;
  uint64_t cap2 = 1;
  while (cap2 < cap) cap2 <<= 1;
  const uint64_t sort_cap = cap2 <= 512 ? 512 : (cap2 < 4096 ? 4096 : cap2);
  const uint64_t kt = 2 * cap2 < 128 ? 128 : 2 * cap2;
  const uint64_t ht = 4 * cap2 < 256 ? 256 : 4 * cap2;
  b += 2 * ((cap * (9 + vb) + 255) / 256 * 256 + cap * (vb + 1)) + 2 * cap * 8 +
       (2 * ((2 * cap + 255) / 256) + 2) * 4 + 16;
  b += 2 * (sort_cap * 8 + kt * 4 + cap * 12 + cap * 16 + cap * 16 + cap * 4 + 2 * cap + ht * 8 +
            2 * cap * 4 + 4 + 2 * cap * I.page_bytes);
  b += 2 * (ht * 8 + ht * I.page_bytes + 2 * cap * 8 + 4);
  b += ht * 8 + cap * vb + cap + cap * vb + cap + cap * 8 + 16 * 4 + 4;
  return b;
}

uint64_t build_estimate(const bolt_info_t& I, uint64_t n) {
  const uint64_t cap = n > 0 ? n : 1;
  uint64_t tag_cap = 8192;
  while (tag_cap < n) tag_cap <<= 1;
  const uint64_t nblocks = (I.M + 1 + 8192 - 1) / 8192 + 1;
  return tag_cap * 24 + cap * (16 + 8 + 4 + 4) + (I.M + 1) * 4 + nblocks * 4 + 16 +
         cap * (8 + (uint64_t)I.val_bytes);  // + the host-pointer staging copy
}

}  // namespace brt

extern "C" int bolt_trim(bolt_t* h) {
  if (!h) return BOLT_E_ARG;
  if (sync_all(h) != cudaSuccess) return BOLT_E_CUDA;
  free_build_scratch(h);
  return BOLT_OK;
}

extern "C" int bolt_footprint(const bolt_t* h, uint64_t* resident_bytes, uint64_t* scratch_bytes) {
  if (!h) return BOLT_E_ARG;
  if (resident_bytes) *resident_bytes = h->dev_bytes;
  if (scratch_bytes) *scratch_bytes = h->scratch_bytes + h->in_cap * (8 + (uint64_t)h->vb);
  return BOLT_OK;
}

namespace {
__device__ __forceinline__ uint64_t probe_page(uint32_t w, uint32_t salt, uint64_t M) {
  uint64_t x = ((uint64_t)salt << 32) ^ w;
  x ^= x >> 33; x *= 0xff51afd7ed558ccdull; x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ull; x ^= x >> 33;
  return x % M;
}
// warps [0, reads): read random page set `salt_r` into buf_r (warp per page);
// warps [reads, reads + writes): write buf_w back to the pages of set
// `salt_w`, which the previous launch read into it (so their bytes do not
// change) -- the access path's pattern of one batch's page reads beside the
// previous batch's write-back
__global__ void k_probe_link(const MapDev m, uint32_t reads, uint32_t writes, uint32_t salt_r,
                             uint32_t salt_w, uint8_t* buf_r, const uint8_t* buf_w) {
  const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t nu4 = m.page_bytes / 16;
  if (w < reads) {
    const uint4* pg = reinterpret_cast<const uint4*>(m.pages + probe_page(w, salt_r, m.M) * m.page_bytes);
    uint4* dst = reinterpret_cast<uint4*>(buf_r + (uint64_t)w * m.page_bytes);
    for (uint32_t c = lane; c < nu4; c += 32) dst[c] = pg[c];
  } else if (w < reads + writes) {
    const uint32_t k = w - reads;
    uint4* pg = reinterpret_cast<uint4*>(m.pages + probe_page(k, salt_w, m.M) * m.page_bytes);
    const uint4* src = reinterpret_cast<const uint4*>(buf_w + (uint64_t)k * m.page_bytes);
    for (uint32_t c = lane; c < nu4; c += 32) pg[c] = src[c];
  }
}
}  // namespace

extern "C" int bolt_probe_link(bolt_t* h, uint32_t pages, uint32_t launches,
                               double* read_pages_per_s, double* pipelined_pages_per_s) {
  if (!h || pages == 0 || launches == 0 || !read_pages_per_s || !pipelined_pages_per_s)
    return BOLT_E_ARG;
  if (!h->initialized) return BOLT_E_STATE;
  if (h->info.M == 0 || pages > (1u << 22)) return BOLT_E_ARG;
  // nothing of the handle may be in flight: a page write-back racing the
  // probe's writes could be overwritten with older bytes
  if (sync_all(h) != cudaSuccess) return BOLT_E_CUDA;
  const uint64_t pb = h->info.page_bytes;
  uint8_t* buf = nullptr;
  if (cudaMalloc(&buf, 2 * (uint64_t)pages * pb) != cudaSuccess) {
    cudaGetLastError();
    return BOLT_E_NOMEM;
  }
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  double rate[2] = {0, 0};
  const uint32_t salt0 = 0x51ED0000u + (uint32_t)(h->batches & 0xffff) * 131u;
  for (int pipelined = 0; pipelined < 2 && e == cudaSuccess; pipelined++) {
    uint32_t salt = salt0 + (uint32_t)pipelined * 0x10000u;
    const uint32_t wr = pipelined ? pages : 0;
    const uint32_t blocks = (uint32_t)(((uint64_t)(pages + wr) * 32 + 255) / 256);
    // launch 0 reads the first set (nothing to write back yet); launch i
    // reads set i into buffer i % 2 and writes set i - 1 back from the other
    k_probe_link<<<(pages * 32 + 255) / 256, 256, 0, h->st>>>(h->m, pages, 0, salt, 0, buf,
                                                              buf + pages * pb);
    e = cudaEventRecord(a, h->st);
    for (uint32_t i = 1; i <= launches && e == cudaSuccess; i++) {
      uint8_t* br = buf + (uint64_t)(i & 1) * pages * pb;
      const uint8_t* bw = buf + (uint64_t)((i - 1) & 1) * pages * pb;
      k_probe_link<<<blocks, 256, 0, h->st>>>(h->m, pages, wr, salt + i, salt + i - 1, br, bw);
    }
    if (e == cudaSuccess) e = cudaEventRecord(b, h->st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && ms > 0) rate[pipelined] = (double)pages * launches / (ms * 1e-3);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(buf);
  if (e != cudaSuccess) return BOLT_E_CUDA;
  *read_pages_per_s = rate[0];
  *pipelined_pages_per_s = rate[1];
  return BOLT_OK;
}

extern "C" int bolt_plan_bytes(uint64_t N, uint32_t val_bytes, uint64_t hbm_budget,
                               uint32_t batch_cap, uint64_t n_init, uint64_t* resident_bytes,
                               uint64_t* build_bytes) {
  bolt_info_t I;
  int rc = bolt_plan(N, 8, val_bytes, hbm_budget, -1.0, 8, &I);
  if (rc) return rc;
  if (batch_cap < 1 || batch_cap > MAXB || n_init > N) return BOLT_E_ARG;
  if (resident_bytes) *resident_bytes = brt::resident_estimate(I, batch_cap, 1ull << 22);
  if (build_bytes) *build_bytes = brt::build_estimate(I, n_init);
  return BOLT_OK;
}

// ---------------------------------------------------------------------------
// autotuner: performance knobs only (nothing it picks changes a result, a
// ciphertext or the trace of later calls, except through the accesses it
// runs itself)
namespace {

__global__ void k_fill_tags(uint64_t* t, uint64_t n, uint64_t salt) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t x = (i + salt) * 0x9E3779B97F4A7C15ull;
    x ^= x >> 29;
    t[i] = x * 0xBF58476D1CE4E5B9ull;
  }
}

}  // namespace

extern "C" int bolt_autotune(bolt_t* h, const void* sample_keys, uint64_t n_sample,
                             double max_batch_us, bolt_tune_t* out) {
  if (!h || !out || !h->allocated) return BOLT_E_ARG;
  if (!h->initialized || h->poisoned) return BOLT_E_STATE;
  std::memset(out, 0, sizeof *out);
  ProfScope prof_scope(h);
  cudaStream_t st = h->st;
  if (sync_all(h) != cudaSuccess) return BOLT_E_CUDA;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return BOLT_E_CUDA;
  // 1. bitonic tile: sort a scratch array the size of this map's tag buffer
  uint64_t n = 8192;
  while (n < h->N) n <<= 1;
  uint64_t* tags = nullptr;
  int rc = BOLT_OK;
  if (cudaMalloc(&tags, n * 8) != cudaSuccess) {
    rc = BOLT_E_NOMEM;
  } else {
    const int tiles[2] = {12, 13};
    double best = 1e30;
    for (int k = 0; k < 2; k++) {
      float ms = 0;
      for (int rep = 0; rep < 2; rep++) {  // the first run warms up
        k_fill_tags<<<256, 256, 0, st>>>(tags, n, (uint64_t)rep);
        cudaEventRecord(a, st);
        sort_tags_u64(tags, n, tiles[k], st);
        cudaEventRecord(b, st);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&ms, a, b);
      }
      out->sort_ms[k] = ms;
      if (ms < best) {
        best = ms;
        out->sort_log_tile = (uint32_t)tiles[k];
      }
    }
    cudaFree(tags);
    h->sort_log_tile = (int)out->sort_log_tile;
  }
  // 2. access batch width: Get batches over the caller's key sample
  if (rc == BOLT_OK && sample_keys && n_sample) {
    const uint32_t cand[BOLT_TUNE_WIDTHS] = {64, 256, 1024, 4096, 16384, 65536};
    double best_rate = 0;
    out->batch_width = 1;
    // sample keys are key_bytes wide (4-byte keys zero-extended)
    auto sample = [&](uint64_t j) -> uint64_t {
      return h->kb == 4 ? static_cast<const uint32_t*>(sample_keys)[j]
                        : static_cast<const uint64_t*>(sample_keys)[j];
    };
    for (int k = 0; k < BOLT_TUNE_WIDTHS && rc == BOLT_OK; k++) {
      const uint32_t w = cand[k];
      out->widths[k] = w;
      if (w > h->cap_batch) continue;
      const int reps = 3;
      float ms = 0;
      for (int rep = 0; rep <= reps && rc == BOLT_OK; rep++) {
        for (uint32_t i = 0; i < w; i++) {
          h->h_keys[i] = sample((rep * (uint64_t)w + i) % n_sample);
          h->h_ops[i] = BOLT_GET;
        }
        std::memset(h->h_vin, 0, (uint64_t)w * h->vb);
        cudaMemcpyAsync(h->b.ops, h->h_ops, w, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(h->b.keys, h->h_keys, (uint64_t)w * 8, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(h->b.vin, h->h_vin, (uint64_t)w * h->vb, cudaMemcpyHostToDevice, st);
        if (rep == 1) cudaEventRecord(a, st);  // rep 0 warms up
        if (access_batch(h, h->b, w, st) != cudaSuccess) rc = BOLT_E_CUDA;
        h->t += w;
        h->batches++;
      }
      cudaEventRecord(b, st);
      cudaEventSynchronize(b);
      cudaEventElapsedTime(&ms, a, b);
      const double us = ms * 1e3 / reps;
      out->width_us[k] = us;
      const double rate = w / (us * 1e-6);
      if ((max_batch_us <= 0 || us <= max_batch_us) && rate > best_rate) {
        best_rate = rate;
        out->batch_width = w;
      }
    }
    uint32_t err = 0;
    if (rc == BOLT_OK && (rc = read_err(h, &err)) == BOLT_OK) rc = err_to_rc(err);
    if (rc == BOLT_OK) h->batch_width = out->batch_width;
    else if (rc == BOLT_E_OVERFLOW) h->poisoned = true;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return rc;
}
