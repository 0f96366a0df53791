// serve.cu -- continuous-batching server for many oblivious maps.
//
// Every map is a full handle (its own streams, device state and pinned host
// pages).  The server admits maps while their planned device footprint fits
// the HBM budget (the rest wait, in order, until a removed map frees memory),
// keeps every admitted map resident, and runs a scheduler thread:
//   - requests (Get/Put/Delete batches of at most max_batch ops) queue per map
//     as they arrive;
//   - whenever a map has no batch on the GPU and requests are queued, the
//     scheduler packs the queued requests (in arrival order, up to max_batch
//     ops) into one access batch on that map's stream; so requests that arrive
//     while the map is busy ride the next batch, and batches of different maps
//     run concurrently on the device;
//   - a completed batch (CUDA event) returns each request's values and
//     status, timestamped, to the client;
//   - a small pool of dispatch threads enqueues the packed batches, so the
//     host cost of enqueueing does not serialise the maps.
// Each batch is exactly one bolt access batch (Alg. 1 over a batch), so a
// request's results do not depend on what it was batched with; the per-map
// log of batch sizes lets a replay reproduce ciphertexts and the trace.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "handle.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  uint32_t map = 0;
  uint32_t n = 0;
  std::vector<uint8_t> ops;
  std::vector<uint64_t> keys;
  std::vector<uint8_t> vin, vout, status;
  double t_submit = 0, t_start = 0, t_done = 0;  // microseconds since server start
  int rc = 0;
  bool done = false;
};

enum MapState : int { MAP_PENDING = 0, MAP_READY = 1, MAP_REMOVED = 2 };

struct Map {
  uint32_t id = 0;
  uint64_t N = 0;
  uint32_t vb = 0;
  uint64_t seed = 0;
  std::vector<uint64_t> init_keys;
  std::vector<uint8_t> init_vals;
  uint64_t resident = 0, build = 0;  // planned device bytes
  int state = MAP_PENDING;
  int error = 0;
  bolt* h = nullptr;
  std::deque<Request*> queue;
  std::vector<Request*> inflight;
  std::atomic<bool> dispatched{false};  // the in-flight batch's done_ev is recorded
  bool remove_requested = false;
  cudaEvent_t done_ev = nullptr;
  // pinned staging of one batch
  uint8_t* h_buf = nullptr;
  bolt::IoSet io;              // the input and output parts of h_buf
  IoPacked packed{};           // the in-flight batch's layout in them
  uint32_t* h_err = nullptr;
  std::vector<uint32_t> batch_log;
};

}  // namespace

struct bolt_server {
  uint64_t budget = 0, used = 0;
  uint32_t max_batch = 4096;
  std::vector<Map*> maps;
  std::unordered_map<uint64_t, Request*> requests;
  std::mutex mu;
  std::condition_variable work_cv, done_cv;
  std::thread worker;
  // dispatch workers: enqueueing a batch (staging copies and about twenty
  // stream operations) takes tens of microseconds of host time, so several
  // threads enqueue the batches of different maps at once
  std::vector<std::thread> dispatchers;
  std::deque<std::pair<Map*, std::vector<Request*>>> jobs;  // guarded by mu
  std::condition_variable job_cv;
  std::atomic<bool> stop{false};
  std::atomic<uint64_t> work_seq{0};  // bumped by every submit / add / remove
  uint64_t next_id = 1;
  Clock::time_point t0 = Clock::now();
  uint64_t batches = 0, ops = 0;
  int device = 0;

  double now_us() const {
    return std::chrono::duration<double, std::micro>(Clock::now() - t0).count();
  }
};

namespace {

constexpr uint64_t SERVER_TRACE_CAP = 1024;
constexpr int SERVER_DISPATCHERS = 4;

void free_map_device(Map* m) {
  if (m->h) {
    bolt_destroy(m->h);
    m->h = nullptr;
  }
  if (m->done_ev) cudaEventDestroy(m->done_ev);
  m->done_ev = nullptr;
  if (m->h_buf) cudaFreeHost(m->h_buf);
  m->h_buf = nullptr;
}

// create, build and trim one map (scheduler thread, outside the lock)
int build_map(bolt_server* s, Map* m) {
  bolt_t* h = nullptr;
  int rc = bolt_create(m->N, 8, m->vb, ~0ull, &h);
  if (rc) return rc;
  m->h = h;
  if ((rc = bolt_set_param(h, BOLT_PARAM_TRACE_CAP, (double)SERVER_TRACE_CAP)) ||
      (rc = bolt_set_param(h, BOLT_PARAM_BATCH_CAP, (double)s->max_batch)))
    return rc;
  rc = bolt_init(h, m->init_keys.data(), m->init_vals.data(), m->init_keys.size(), m->seed);
  if (rc) return rc;
  rc = bolt_trim(h);
  if (rc) return rc;
  // staging laid out like the handle's device I/O set 0: an input part and an
  // output part, each filled back to back for the batch's n ops (io_packed)
  const uint64_t cap = s->max_batch, vb = m->vb;
  const uint64_t in_bytes = (cap * (9 + vb) + 63) / 64 * 64;
  const uint64_t bytes = in_bytes + cap * (vb + 1) + 64;
  if (cudaHostAlloc(reinterpret_cast<void**>(&m->h_buf), bytes, cudaHostAllocDefault) != cudaSuccess)
    return BOLT_E_NOMEM;
  m->io.keys = reinterpret_cast<uint64_t*>(m->h_buf);
  m->io.vout = m->h_buf + in_bytes;
  uint8_t* q = m->io.vout + cap * (vb + 1);
  m->h_err = reinterpret_cast<uint32_t*>((reinterpret_cast<uintptr_t>(q) + 7) & ~uintptr_t(7));
  if (cudaEventCreateWithFlags(&m->done_ev, cudaEventDisableTiming) != cudaSuccess) return BOLT_E_CUDA;
  std::vector<uint64_t>().swap(m->init_keys);
  std::vector<uint8_t>().swap(m->init_vals);
  return BOLT_OK;
}

// copy a packed batch's requests into the map's staging and enqueue the batch
// (a dispatch worker, lock not held; touches only the map's staging and its
// handle, and a map has at most one batch in flight)
cudaError_t dispatch(bolt_server* s, Map* m, const std::vector<Request*>& reqs, uint32_t* n_out) {
  bolt* h = m->h;
  const uint64_t vb = m->vb;
  uint32_t n = 0;
  for (Request* r : reqs) n += r->n;
  const IoPacked hp = io_packed(m->io, n, vb);
  const double t_start = s->now_us();
  uint32_t off = 0;
  for (Request* r : reqs) {
    std::memcpy(hp.ops + off, r->ops.data(), r->n);
    std::memcpy(hp.keys + off, r->keys.data(), (uint64_t)r->n * 8);
    std::memcpy(hp.vin + (uint64_t)off * vb, r->vin.data(), (uint64_t)r->n * vb);
    r->t_start = t_start;
    off += r->n;
  }
  *n_out = n;
  m->packed = hp;
  cudaStream_t st = h->st;
  ProfScope prof_scope(h);
  const IoPacked dp = io_packed(h->d_io[0], n, vb);
  cudaError_t e = cudaMemcpyAsync(dp.keys, hp.keys, hp.in_bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = brt::enqueue_batch_packed(h, n, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hp.vout, dp.vout, hp.out_bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->h_err, h->m.err, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventRecord(m->done_ev, st);
  return e;
}

// results of a finished batch back to its requests (scheduler thread, lock held)
void complete(bolt_server* s, Map* m) {
  const uint64_t vb = m->vb;
  int rc = m->error ? m->error : brt::err_rc(*m->h_err);
  if (rc) {
    m->error = rc;
    m->h->poisoned = true;
  }
  const double t_done = s->now_us();
  uint32_t off = 0;
  for (Request* r : m->inflight) {
    r->vout.assign(m->packed.vout + (uint64_t)off * vb, m->packed.vout + (uint64_t)(off + r->n) * vb);
    r->status.assign(m->packed.status + off, m->packed.status + off + r->n);
    r->rc = rc;
    r->t_done = t_done;
    r->done = true;
    off += r->n;
  }
  s->batches++;
  s->ops += off;
  m->inflight.clear();
}

void fail_queue(Map* m, int rc, double t) {
  for (Request* r : m->queue) {
    r->rc = rc;
    r->done = true;
    r->t_done = t;
  }
  m->queue.clear();
}

void scheduler(bolt_server* s) {
  cudaSetDevice(s->device);
  std::vector<Map*> busy_maps;
  while (!s->stop.load()) {
    const uint64_t seq = s->work_seq.load();
    std::unique_lock<std::mutex> lock(s->mu);
    bool progress = false;
    // 1. completions (a batch whose event reports an error completes with
    //    BOLT_E_CUDA rather than never)
    for (size_t i = 0; i < s->maps.size(); i++) {
      Map* m = s->maps[i];
      if (m->inflight.empty() || !m->dispatched.load()) continue;
      const cudaError_t q = cudaEventQuery(m->done_ev);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) m->error = BOLT_E_CUDA;
      m->dispatched.store(false);
      complete(s, m);
      progress = true;
    }
    if (progress) s->done_cv.notify_all();
    // 2. removals of idle maps (the lock is dropped inside these loops: index
    //    them, the list only grows and Map pointers are stable)
    for (size_t i = 0; i < s->maps.size(); i++) {
      Map* m = s->maps[i];
      if (m->remove_requested && m->state == MAP_READY && m->inflight.empty() && m->queue.empty()) {
        lock.unlock();
        free_map_device(m);
        lock.lock();
        s->used -= m->resident;
        m->state = MAP_REMOVED;
        progress = true;
      } else if (m->remove_requested && m->state == MAP_PENDING) {
        fail_queue(m, BOLT_E_STATE, s->now_us());
        m->state = MAP_REMOVED;
        progress = true;
        s->done_cv.notify_all();
      }
    }
    // 3. admission, in order: build while the planned footprint fits
    for (size_t i = 0; i < s->maps.size(); i++) {
      Map* m = s->maps[i];
      if (m->state != MAP_PENDING || m->remove_requested) continue;
      if (s->used + m->resident + m->build > s->budget) break;
      s->used += m->resident + m->build;
      lock.unlock();
      const int rc = build_map(s, m);
      lock.lock();
      s->used -= m->build;
      if (rc) {
        lock.unlock();
        free_map_device(m);
        lock.lock();
        s->used -= m->resident;
        m->error = rc;
        m->state = MAP_REMOVED;
        fail_queue(m, rc, s->now_us());
        s->done_cv.notify_all();
      } else {
        m->state = MAP_READY;
      }
      progress = true;
    }
    // 4. dispatch: every idle ready map with queued requests gets a batch
    for (size_t i = 0; i < s->maps.size(); i++) {
      Map* m = s->maps[i];
      if (m->state != MAP_READY || !m->inflight.empty() || m->queue.empty()) continue;
      if (m->error) {
        fail_queue(m, BOLT_E_STATE, s->now_us());
        s->done_cv.notify_all();
        continue;
      }
      std::vector<Request*> reqs;
      uint32_t n = 0;
      while (!m->queue.empty() && n + m->queue.front()->n <= s->max_batch) {
        reqs.push_back(m->queue.front());
        n += m->queue.front()->n;
        m->queue.pop_front();
      }
      m->inflight = reqs;
      m->dispatched.store(false);
      s->jobs.emplace_back(m, std::move(reqs));
      s->job_cv.notify_one();
      progress = true;
    }
    if (progress) continue;
    busy_maps.clear();
    for (Map* m : s->maps)
      if (!m->inflight.empty()) busy_maps.push_back(m);
    if (busy_maps.empty()) {
      // idle: sleep until new work arrives
      s->work_cv.wait_for(lock, std::chrono::milliseconds(2),
                          [&] { return s->stop.load() || s->work_seq.load() != seq; });
      continue;
    }
    lock.unlock();
    // batches on the GPU: poll their events without the lock, until one is
    // done or new work arrives (clients never wait on the scheduler's lock)
    for (;;) {
      if (s->stop.load() || s->work_seq.load() != seq) break;
      bool any = false;
      for (Map* m : busy_maps)
        if (m->dispatched.load() && cudaEventQuery(m->done_ev) != cudaErrorNotReady) any = true;
      if (any) break;
      std::this_thread::yield();
    }
  }
}

// dispatch worker: enqueue the batches the scheduler packed
void dispatcher(bolt_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lock(s->mu);
  for (;;) {
    s->job_cv.wait(lock, [&] { return s->stop.load() || !s->jobs.empty(); });
    if (s->jobs.empty()) return;  // stopping
    auto job = std::move(s->jobs.front());
    s->jobs.pop_front();
    Map* m = job.first;
    lock.unlock();
    uint32_t packed = 0;
    const cudaError_t e = dispatch(s, m, job.second, &packed);
    lock.lock();
    m->batch_log.push_back(packed);
    if (e != cudaSuccess) {
      // the batch never ran: fail its requests now
      m->error = BOLT_E_CUDA;
      *m->h_err = 0;
      complete(s, m);
      s->done_cv.notify_all();
    } else {
      m->dispatched.store(true);
    }
    s->work_seq.fetch_add(1);
    s->work_cv.notify_all();
  }
}

Map* find_map(bolt_server* s, uint32_t id) {
  return id < s->maps.size() ? s->maps[id] : nullptr;
}

}  // namespace

extern "C" {

int bolt_server_create(uint64_t hbm_budget, uint32_t max_batch, bolt_server_t** out) {
  if (!out || max_batch < 1 || max_batch > MAXB) return BOLT_E_ARG;
  bolt_server* s = new (std::nothrow) bolt_server();
  if (!s) return BOLT_E_NOMEM;
  s->budget = hbm_budget;
  // the library's allocation-free build array is resident on every device
  // that loaded it: counted once, before any map
  s->used = BOLT_NOALLOC_SCRATCH_BYTES;
  s->max_batch = max_batch;
  cudaGetDevice(&s->device);
  s->worker = std::thread(scheduler, s);
  for (int i = 0; i < SERVER_DISPATCHERS; i++) s->dispatchers.emplace_back(dispatcher, s);
  *out = s;
  return BOLT_OK;
}

int bolt_server_add_map(bolt_server_t* s, uint64_t N, uint32_t val_bytes, const void* keys,
                        const void* vals, uint64_t n, uint64_t seed, uint32_t* map_id) {
  if (!s || !map_id || n > N || (n && (!keys || !vals))) return BOLT_E_ARG;
  bolt_info_t I;
  int rc = bolt_plan(N, 8, val_bytes, ~0ull, -1.0, 8, &I);
  if (rc) return rc;
  Map* m = new (std::nothrow) Map();
  if (!m) return BOLT_E_NOMEM;
  m->N = N;
  m->vb = val_bytes;
  m->seed = seed;
  m->init_keys.assign(static_cast<const uint64_t*>(keys), static_cast<const uint64_t*>(keys) + n);
  m->init_vals.assign(static_cast<const uint8_t*>(vals), static_cast<const uint8_t*>(vals) + n * val_bytes);
  m->resident = brt::resident_estimate(I, s->max_batch, SERVER_TRACE_CAP);
  m->build = brt::build_estimate(I, n);
  if (m->resident + m->build + BOLT_NOALLOC_SCRATCH_BYTES > s->budget) {
    delete m;
    return BOLT_E_NOMEM;  // could never be admitted
  }
  std::lock_guard<std::mutex> lock(s->mu);
  m->id = (uint32_t)s->maps.size();
  s->maps.push_back(m);
  *map_id = m->id;
  s->work_seq.fetch_add(1);
  s->work_cv.notify_one();
  return BOLT_OK;
}

int bolt_server_map_state(bolt_server_t* s, uint32_t map_id) {
  if (!s) return BOLT_E_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  Map* m = find_map(s, map_id);
  if (!m) return BOLT_E_ARG;
  if (m->error) return m->error;
  return m->state;
}

int bolt_server_remove_map(bolt_server_t* s, uint32_t map_id) {
  if (!s) return BOLT_E_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  Map* m = find_map(s, map_id);
  if (!m) return BOLT_E_ARG;
  m->remove_requested = true;
  s->work_seq.fetch_add(1);
  s->work_cv.notify_one();
  return BOLT_OK;
}

int bolt_server_submit(bolt_server_t* s, uint32_t map_id, const uint8_t* ops, const void* keys,
                       const void* vals_in, uint32_t n, uint64_t* req_id) {
  if (!s || !req_id || n == 0 || n > s->max_batch || !ops || !keys || !vals_in) return BOLT_E_ARG;
  for (uint32_t i = 0; i < n; i++)
    if (ops[i] > BOLT_DEL) return BOLT_E_ARG;
  Request* r = new (std::nothrow) Request();
  if (!r) return BOLT_E_NOMEM;
  std::unique_lock<std::mutex> lock(s->mu);
  Map* m = find_map(s, map_id);
  if (!m || m->state == MAP_REMOVED || m->remove_requested) {
    delete r;
    return m ? BOLT_E_STATE : BOLT_E_ARG;
  }
  const uint64_t vb = m->vb;
  lock.unlock();
  r->map = map_id;
  r->n = n;
  r->ops.assign(ops, ops + n);
  r->keys.assign(static_cast<const uint64_t*>(keys), static_cast<const uint64_t*>(keys) + n);
  r->vin.assign(static_cast<const uint8_t*>(vals_in), static_cast<const uint8_t*>(vals_in) + (uint64_t)n * vb);
  lock.lock();
  // the map may have been removed while the request was copied: a request
  // queued on it now would never be served
  if (m->state == MAP_REMOVED || m->remove_requested) {
    delete r;
    return BOLT_E_STATE;
  }
  r->id = s->next_id++;
  r->t_submit = s->now_us();
  s->requests[r->id] = r;
  m->queue.push_back(r);
  *req_id = r->id;
  s->work_seq.fetch_add(1);
  s->work_cv.notify_one();
  return BOLT_OK;
}

int bolt_server_submit_many(bolt_server_t* s, uint32_t count, const uint32_t* map_ids,
                            const uint8_t* const* ops, const void* const* keys,
                            const void* const* vals_in, const uint32_t* ns, uint64_t* req_ids) {
  if (!s || (count && (!map_ids || !ops || !keys || !vals_in || !ns || !req_ids))) return BOLT_E_ARG;
  const double t = s->now_us();  // every request arrives with the call
  std::vector<uint64_t> vbs(count);
  {
    std::lock_guard<std::mutex> lock(s->mu);
    for (uint32_t j = 0; j < count; j++) {
      Map* m = find_map(s, map_ids[j]);
      if (!m) return BOLT_E_ARG;
      if (m->state == MAP_REMOVED || m->remove_requested) return BOLT_E_STATE;
      vbs[j] = m->vb;
    }
  }
  for (uint32_t j = 0; j < count; j++) {
    if (ns[j] == 0 || ns[j] > s->max_batch || !ops[j] || !keys[j] || !vals_in[j]) return BOLT_E_ARG;
    for (uint32_t i = 0; i < ns[j]; i++)
      if (ops[j][i] > BOLT_DEL) return BOLT_E_ARG;
  }
  // copies outside the lock
  std::vector<Request*> rs(count, nullptr);
  for (uint32_t j = 0; j < count; j++) {
    Request* r = new (std::nothrow) Request();
    if (!r) {
      for (Request* q : rs) delete q;
      return BOLT_E_NOMEM;
    }
    const uint32_t n = ns[j];
    r->map = map_ids[j];
    r->n = n;
    r->ops.assign(ops[j], ops[j] + n);
    r->keys.assign(static_cast<const uint64_t*>(keys[j]), static_cast<const uint64_t*>(keys[j]) + n);
    r->vin.assign(static_cast<const uint8_t*>(vals_in[j]),
                  static_cast<const uint8_t*>(vals_in[j]) + (uint64_t)n * vbs[j]);
    rs[j] = r;
  }
  std::unique_lock<std::mutex> lock(s->mu);
  // a map removed while the requests were copied: queue none
  for (uint32_t j = 0; j < count; j++) {
    Map* m = find_map(s, map_ids[j]);
    if (m->state == MAP_REMOVED || m->remove_requested) {
      for (Request* q : rs) delete q;
      return BOLT_E_STATE;
    }
  }
  for (uint32_t j = 0; j < count; j++) {
    Request* r = rs[j];
    r->id = s->next_id++;
    r->t_submit = t;
    s->requests[r->id] = r;
    find_map(s, map_ids[j])->queue.push_back(r);
    req_ids[j] = r->id;
  }
  s->work_seq.fetch_add(1);
  s->work_cv.notify_one();
  return BOLT_OK;
}

int bolt_server_wait(bolt_server_t* s, uint64_t req_id, void* vals_out, uint8_t* status_out,
                     bolt_req_info_t* info, int timeout_ms) {
  if (!s) return BOLT_E_ARG;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->requests.find(req_id);
  if (it == s->requests.end()) return BOLT_E_ARG;
  Request* r = it->second;
  auto pred = [&] { return r->done; };
  if (timeout_ms < 0) {
    s->done_cv.wait(lock, pred);
  } else if (!s->done_cv.wait_for(lock, std::chrono::milliseconds(timeout_ms), pred)) {
    return BOLT_E_TIMEOUT;
  }
  if (vals_out && !r->vout.empty()) std::memcpy(vals_out, r->vout.data(), r->vout.size());
  if (status_out && !r->status.empty()) std::memcpy(status_out, r->status.data(), r->status.size());
  if (info) {
    info->id = r->id;
    info->map = r->map;
    info->n = r->n;
    info->rc = r->rc;
    info->submit_us = r->t_submit;
    info->start_us = r->t_start;
    info->done_us = r->t_done;
  }
  const int rc = r->rc;
  s->requests.erase(it);
  delete r;
  return rc;
}

int bolt_server_map_batches(bolt_server_t* s, uint32_t map_id, uint32_t* sizes, uint64_t cap,
                            uint64_t* count) {
  if (!s || !count || (cap && !sizes)) return BOLT_E_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  Map* m = find_map(s, map_id);
  if (!m) return BOLT_E_ARG;
  const uint64_t n = m->batch_log.size();
  for (uint64_t i = 0; i < n && i < cap; i++) sizes[i] = m->batch_log[i];
  *count = n;
  return BOLT_OK;
}

int bolt_server_map_handle(bolt_server_t* s, uint32_t map_id, bolt_t** out) {
  if (!s || !out) return BOLT_E_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  Map* m = find_map(s, map_id);
  if (!m || m->state != MAP_READY) return BOLT_E_STATE;
  *out = m->h;
  return BOLT_OK;
}

int bolt_server_stats(bolt_server_t* s, bolt_server_stats_t* out) {
  if (!s || !out) return BOLT_E_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  std::memset(out, 0, sizeof *out);
  out->budget = s->budget;
  out->used = s->used;
  out->batches = s->batches;
  out->ops = s->ops;
  for (Map* m : s->maps) {
    if (m->state == MAP_PENDING) out->maps_pending++;
    if (m->state == MAP_READY) out->maps_ready++;
    out->queued += m->queue.size();
  }
  return BOLT_OK;
}

int bolt_server_destroy(bolt_server_t* s) {
  if (!s) return BOLT_OK;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop.store(true);
  }
  s->work_cv.notify_all();
  s->job_cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (std::thread& t : s->dispatchers)
    if (t.joinable()) t.join();
  for (Map* m : s->maps) {
    if (m->h) brt::sync_handle(m->h);
    free_map_device(m);  // queued requests are freed with s->requests below
    delete m;
  }
  for (auto& kv : s->requests) delete kv.second;
  delete s;
  return BOLT_OK;
}

}  // extern "C"
