// handle.h -- the map handle behind the C ABI (shared by runtime.cu and
// serve.cu; not part of the public interface).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "batch.cuh"
#include "bolt_internal.cuh"

constexpr uint32_t MAXB = BOLT_MAX_BATCH;

struct bolt {
  uint64_t dev_bytes = 0;     // device bytes of the resident state + batch buffers
  uint64_t scratch_bytes = 0; // device bytes of the build scratch
  int sort_log_tile = 13;      // bitonic tile chosen by bolt_autotune
  uint64_t N = 0;
  uint32_t vb = 0;
  uint32_t kb = 8;            // key bytes at the host-pointer boundary (4 or 8)
  uint64_t hbm_budget = 0;
  double alpha_override = -1.0;
  uint32_t c = 8;
  uint32_t batch_width = MAXB;
  uint32_t cap_batch = MAXB;  // capacity of the batch buffers (ops per batch)
  uint64_t trace_cap = 1ull << 22;
  bool trace_on = false;
  bool check_keys = true;
  double la_frac = 0.0;       // BOLT_PARAM_LOOKAHEAD: share of a batch's pages read ahead
  int defer_flush = 0;        // BOLT_PARAM_DEFER_FLUSH: write-back after the next batch's reads
  uint32_t spin_limit = 1u << 22;  // BOLT_PARAM_SPIN_LIMIT: bounded device waits
  int prf_rounds = 0;              // BOLT_PARAM_ROUNDS_PRF
  bool fused = true;          // BOLT_PARAM_FUSED: batches of <= FUSED_MAX_OPS in one launch
  bool integrity = false;     // BOLT_PARAM_INTEGRITY: sealed pages (tag checked on read)
  bolt_info_t info{};

  bdev::MapDev m{};
  bdev::BatchDev b{};
  bdev::BuildScratch bs{};
  cudaStream_t st = nullptr;
  uint8_t* pages_host = nullptr;
  std::vector<void*> dev_allocs;  // state + batch buffers (freed by free_state)

  // host-pointer staging
  uint64_t* in_keys = nullptr;
  uint8_t* in_vals = nullptr;
  uint64_t in_cap = 0;
  uint8_t* h_ops = nullptr;
  uint64_t* h_keys = nullptr;
  uint8_t* h_vin = nullptr;
  uint8_t* h_vout = nullptr;
  uint8_t* h_status = nullptr;
  uint32_t* h_err = nullptr;
  // a one-batch host call's results as tagged words (pinned, mapped; room
  // for FUSED_MAX_OPS ops) and the count of such calls, whose low byte
  // (never 0) tags them
  uint64_t* h_res = nullptr;
  uint32_t done_seq = 0;
  ptrdiff_t io_dev_delta = 0;  // device address of the pinned staging minus its host address
  // bolt_access moves chunks of ops through two alternating sets of pinned
  // staging (set 0 is h_ops ... h_status) and device I/O buffers (set 0 is
  // b.ops ... b.status), so that one chunk's host copies overlap another's
  // batches.  Each set is one block: an input part keys | vin | ops of
  // cap * (9 + vb) bytes from `keys`, and an output part vout | status of
  // cap * (vb + 1) bytes from `vout` (see io_packed).
  struct IoSet {
    uint8_t* ops = nullptr;
    uint64_t* keys = nullptr;
    uint8_t* vin = nullptr;
    uint8_t* vout = nullptr;
    uint8_t* status = nullptr;
  } h_io[2], d_io[2];
  cudaEvent_t ev_h2d[2] = {nullptr, nullptr}, ev_d2h[2] = {nullptr, nullptr};
  cudaEvent_t ev_ioready[2] = {nullptr, nullptr};  // a chunk's batches are done
  uint32_t* d_kdf = nullptr;
  uint32_t* d_flag = nullptr;

  uint64_t t = 0, batches = 0;
  bool allocated = false, initialized = false, poisoned = false;
  bdev::Prof prof;
  cudaStream_t last_st = nullptr;  // stream of the last enqueued work
  cudaStream_t st2 = nullptr;      // side stream (key-uniqueness check)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_pfork = nullptr, ev_pjoin = nullptr;  // build: placement on the side stream
  // access batches alternate between two buffer slots; a slot's written pages
  // reach the host on st_fl while the next batch runs
  cudaStream_t st_fl = nullptr;
  cudaEvent_t ev_evicted[2] = {nullptr, nullptr}, ev_flushed[2] = {nullptr, nullptr};
  bool flush_pending[2] = {false, false};
  int slot = 0;
  bool prev_valid = false;
  uint32_t slot_ht_mask[2] = {0, 0};
  uint32_t* s_ht_key[2] = {nullptr, nullptr};
  uint32_t* s_ht_min[2] = {nullptr, nullptr};
  uint8_t* s_dbuf[2] = {nullptr, nullptr};
  uint32_t* s_dslot[2] = {nullptr, nullptr};
  uint32_t* s_dpage[2] = {nullptr, nullptr};
  uint32_t* s_dcount[2] = {nullptr, nullptr};
  // per-slot outputs of a batch's preparation (grouping, PRF pairs, rows)
  // and lookahead (position-map hits, pages read ahead), so that the next
  // batch's preparation and lookahead can run on st_prep while this batch's
  // main part runs
  struct PrepSet {
    uint64_t* skeys = nullptr;
    uint32_t* kt_own = nullptr;
    uint32_t* leader = nullptr;
    uint32_t* prevw = nullptr;
    uint32_t* lastw = nullptr;
    uint64_t* pair = nullptr;
    uint64_t* rpair = nullptr;
    uint32_t* rows = nullptr;
    uint32_t* hit = nullptr;
    uint8_t* done = nullptr;
    uint8_t* pres = nullptr;
    uint32_t* la_key = nullptr;
    uint32_t* la_idx = nullptr;
    uint32_t* la_list = nullptr;
    uint32_t* la_count = nullptr;
    uint8_t* la_buf = nullptr;
  } s_prep[2];
  cudaStream_t st_prep = nullptr;
  cudaStream_t st_out = nullptr;  // bolt_access: device-to-host result copies
  cudaEvent_t ev_in = nullptr, ev_prep[2] = {nullptr, nullptr}, ev_pfree[2] = {nullptr, nullptr};
  cudaEvent_t ev_looked[2] = {nullptr, nullptr};  // a slot's batch finished its page reads
  // a batch whose write-back waits for the next batch's page reads (only
  // between the batches of one call; every call ends with none deferred)
  bool deferred = false;
  bdev::BatchDev deferred_b{};
  uint32_t deferred_n = 0;
  cudaEvent_t ev_reads_done = nullptr;
};


// n ops packed back to back from the start of an I/O set's two parts --
// inputs keys[n] | vin[n * vb] | ops[n], outputs vout[n * vb] | status[n] --
// so that a batch's inputs and its results each cross the link in one copy
struct IoPacked {
  uint64_t* keys;
  uint8_t* vin;
  uint8_t* ops;
  uint8_t* vout;
  uint8_t* status;
  uint64_t in_bytes, out_bytes;
};
inline IoPacked io_packed(const bolt::IoSet& s, uint64_t n, uint64_t vb) {
  uint8_t* in = reinterpret_cast<uint8_t*>(s.keys);
  return {s.keys, in + n * 8, in + n * (8 + vb), s.vout, s.vout + n * vb, n * (9 + vb), n * (vb + 1)};
}

// points the kernel-side profiler at the handle for one ABI call
struct ProfScope {
  explicit ProfScope(bolt* h) { bdev::g_prof = &h->prof; }
  ~ProfScope() { bdev::g_prof = nullptr; }
};

namespace brt {
// one access batch of n <= cap_batch ops whose inputs are already in the
// handle's device batch buffers, enqueued on st (outputs in h->b.vout/status)
cudaError_t enqueue_batch(bolt* h, uint32_t n, cudaStream_t st);
// the same, with its inputs and outputs packed in I/O set 0 (io_packed)
cudaError_t enqueue_batch_packed(bolt* h, uint32_t n, cudaStream_t st);
// BOLT_OK / BOLT_E_* for a device error word
int err_rc(uint32_t err);
// wait for every stream of the handle
cudaError_t sync_handle(bolt* h);
// device bytes the planner expects a map to hold resident, and its build
// scratch for n records
uint64_t resident_estimate(const bolt_info_t& I, uint64_t cap_batch, uint64_t trace_cap);
uint64_t build_estimate(const bolt_info_t& I, uint64_t n);
}  // namespace brt
