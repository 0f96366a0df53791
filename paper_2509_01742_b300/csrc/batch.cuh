// batch.cuh -- device buffers of one access batch (capacity BOLT_MAX_BATCH).
#pragma once
#include "bolt_internal.cuh"

namespace bdev {

struct BatchDev {
  // staged inputs / outputs
  uint8_t* ops;        // [cap]
  uint64_t* keys;      // [cap]
  uint8_t* vin;        // [cap * vb]
  uint8_t* vout;       // [cap * vb]
  uint8_t* status;     // [cap]
  // grouping
  uint64_t* skeys;     // [cap] grouping keys: key slot << 16 | op index
  uint32_t* kt_own;    // [kt_mask + 1] key hash table: owner op + 1, or 0
  uint32_t kt_mask, pad1;
  uint32_t* leader;    // [cap] first op on the same key
  uint32_t* prevw;     // [cap] previous PUT/DEL on the same key, or NONE
  uint32_t* lastw;     // [cap] (leaders) last PUT/DEL of the key group, or NONE
  // key search
  uint64_t* pair;      // [cap] bins read by the op: stored pair or DUMMY pair
  uint64_t* rpair;     // [cap] REMAP pair
  uint32_t* rows;      // [4 * cap] position-map rows
  uint32_t* hit;       // [cap] position-map slot of a leader hit, or NONE
  uint32_t* hit_meta;  // [cap] that slot's metadata as the search read it (fused
                       // launch only; null: find_remove reads the map)
  // pages read by the batch
  uint32_t* pos_page;  // [2 cap] host page of read position 2i + j, or NONE
  uint32_t* pos_slot;  // [2 cap] hash-table slot of that page
  uint32_t* block_cnt; // [2 * blocks] per-block (valid, first) read counts, then offsets
  unsigned long long* trace_base;  // [2] trace offset of the batch, its read count
  uint32_t* ht_key;    // [ht_mask + 1] page hash table: host page, or NONE
  uint32_t* ht_min;    // [ht_mask + 1] first read position of the page
  uint32_t ht_mask, pad0;
  uint8_t* dbuf;       // [(ht_mask + 1) * page_bytes] per page-table slot: the
                       // decrypted page, then the ciphertext written back
                       // (flushed to the host later)
  uint64_t* removed;   // [ht_mask + 1] page slots taken out by find_remove
  uint32_t* dslot;     // [2 cap] page-table slots holding a page, claim order
  uint32_t* dpage;     // [2 cap] their pages (the write-back reads these: the
                       // table itself is cleared by the next batch)
  uint32_t* dcount;    // [1]
  // the previous batch's written pages, until its flush has landed: a page it
  // wrote is read from prev_dbuf (ciphertext, at its slot in prev_ht_key)
  // instead of the host
  const uint32_t* prev_ht_key;
  const uint8_t* prev_dbuf;
  uint32_t prev_ht_mask, prev_valid;
  // the previous batch's page table, cleared by this batch once read (the
  // entries up to clr_mask; none when clr_ht_key is null)
  uint32_t* clr_ht_key;
  uint32_t* clr_ht_min;
  uint32_t clr_mask, pad3;
  // values
  uint8_t* init_val;   // [cap * vb] value found for a leader hit
  uint8_t* init_present;  // [cap]
  uint8_t* rval;       // [cap * vb] value to re-place (leaders)
  uint8_t* fpres;      // [cap] key present after the batch (leaders)
  uint32_t* rdest;     // [cap] P2C destination
  uint32_t* rrow;      // [cap] position-map row for a new key
  // lookahead: while the previous batch runs, leaders whose key is not in it
  // search the position map, and the pages of every read position whose bin
  // is then known are read and decrypted ahead
  uint32_t la_on, la_limit;  // la_limit: queued pages read ahead (the first ones)
  uint8_t* done;       // [cap] leader searched ahead (its hit is in hit[])
  uint32_t* la_key;    // [ht_mask + 1] page read ahead, or NONE
  uint32_t* la_idx;    // [ht_mask + 1] its row in la_buf
  uint32_t* la_list;   // [2 cap] pages read ahead, in claim order
  uint32_t* la_count;  // [1]
  uint8_t* la_buf;     // [2 cap * page_bytes] their plaintexts
  uint8_t* pres;       // [cap] (leaders) key present before the batch as
                       // seen ahead: 0 no, 1 yes, 2 not known
  // the previous batch: key table, keys, ops, grouping, REMAP pairs and
  // presence seen ahead (a key it touches is re-mapped to its leader's REMAP
  // pair when present after it, so the bins this batch reads for the key are
  // known before the previous batch ends)
  const uint32_t* prev_kt_own;
  const uint64_t* prev_keys;
  const uint8_t* prev_ops;
  const uint32_t* prev_leader;
  const uint32_t* prev_lastw;
  const uint64_t* prev_rpair;
  const uint8_t* prev_pres;
  uint32_t prev_kt_mask, pad2;
  // a host-pointer call of one small batch (fused launch only): the packed
  // inputs keys | vin | ops in pinned host staging, copied by the kernel into
  // the device inputs above (laid out the same way from `keys`); the results
  // vout | status (packed) and the error word back to h_res as 8-byte words,
  // each 7 bytes of that stream and res_tag in its top byte
  const uint8_t* h_in;
  uint64_t* h_res;
  uint32_t res_tag, pad4;
};

cudaError_t sort_batch_keys(uint64_t* keys, uint32_t n_pow2, cudaStream_t st);
cudaError_t sort_batch_keys32(uint32_t* keys, uint32_t n_pow2, cudaStream_t st);
// Host page write-back runs on `flush_st` after `ev_evicted` (recorded on st
// once the batch's ciphertexts are in dbuf); `ev_flushed` is recorded on
// flush_st when the batch's pages are in host memory.  With `defer_own` the
// batch's write-back is not enqueued here: the next batch's launch_main
// enqueues it (as `prev`) once that batch's own page reads are done, so the
// writes fill the link while that batch finds, executes and remaps.
struct FlushCtx {
  cudaStream_t flush_st;
  cudaEvent_t ev_evicted;
  cudaEvent_t ev_flushed;
  cudaEvent_t ev_looked;   // recorded on st once the batch's page reads are done
  int fast_flush;          // 1: the write-back may use twice the warps
  int defer_own;           // 1: leave this batch's write-back to the next batch
  const BatchDev* prev;    // a deferred write-back to enqueue after the page reads
  uint32_t prev_n;         // its batch's op count (sizes its grid)
  int prev_fast;           // 1: that write-back uses twice the warps
  cudaEvent_t prev_flushed;  // recorded on flush_st when it has landed
  cudaEvent_t ev_reads_done; // scratch event: this batch's page reads are done
};

cudaError_t launch_prep(const MapDev& m, const BatchDev& b, uint32_t n, uint64_t t0,
                        cudaStream_t st);
// A whole batch of n <= FUSED_MAX_OPS ops (preparation, main part and the
// host write-back of its pages) in one single-CTA launch; op i has sequence
// number t0 + i.  Same tables, buffers, results, pages and trace as
// launch_prep + launch_main + the write-back.  No write-back of an earlier
// batch may still be in flight when it starts.  It is launched as a
// programmatic dependent of the previous kernel on st; early_in = the inputs
// (b.h_in, or b.keys / b.vin / b.ops) are complete even if that kernel is
// not (host staging written before the launch, or the previous kernel is an
// earlier fused batch of the same call), so they are read before the wait.
// inl (or null): the batch's inputs carried in the launch's own parameters,
// in the staging's layout (keys as 8-byte words | values | ops), so the
// kernel reads none of them from host memory; they then take the place of
// b.h_in / b.keys / b.vin / b.ops.
constexpr uint32_t FUSED_MAX_OPS = 32;
constexpr uint32_t FUSED_INLINE_MAX = 256;
struct FusedInline {
  uint32_t bytes;  // 0: no inputs here
  uint32_t pad[3];
  uint4 d[FUSED_INLINE_MAX / 16];
};
cudaError_t launch_fused(const MapDev& m, const BatchDev& b, uint32_t n, uint64_t t0,
                         cudaStream_t st, bool early_in = false,
                         const FusedInline* inl = nullptr);
cudaError_t launch_main(const MapDev& m, const BatchDev& b, uint32_t n, cudaStream_t st,
                        const FlushCtx& fc);
// The lookahead part of a batch (b.la_on = 1), after its preparation:
// launch_ahead_lookup searches the position map for the leaders whose key
// the previous batch does not touch and queues the pages it can predict; it
// may run while the previous batch's main part runs.  launch_ahead_gather
// reads and decrypts the first `limit` queued pages; it runs once the
// previous batch's own page reads are done and the flush two batches back
// has landed.
cudaError_t launch_ahead_lookup(const MapDev& m, const BatchDev& b, uint32_t n, cudaStream_t st);
cudaError_t launch_ahead_gather(const MapDev& m, const BatchDev& b, uint32_t limit,
                                cudaStream_t st);

}  // namespace bdev
