// em_server.cu -- the served form: a continuous-batching request loop.
//
// Host side only (no kernels of its own): the worker thread admits requests by
// slots and memory budget, forms batches of distinct idle maps, launches each
// batch with em_update_batch on a free stream, and polls the streams' events
// to complete tickets.  A map is never in two batches in flight at once, and a
// map takes one update per batch, so each request is fused against exactly
// the map state it would see if it were served alone.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "em.h"
#include "em_host.h"

using namespace em;

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

enum ReqState { kPending, kAdmitted, kRunning, kDone };

struct Request {
  int32_t map_id = 0;
  std::vector<em_cloud> clouds;
  int64_t points = 0;
  int64_t bytes = 0;
  cudaEvent_t ready = nullptr;  // the caller's "points written" event, or null
  uint32_t read_mask = 0;       // layers to write to read_dst after the update
  float* read_dst = nullptr;    // device-writable address (device or mapped host memory)
  float* read_host = nullptr;   // the caller's host address when read_dst is host memory
  int64_t read_floats = 0;
  bool on_host = false;         // the clouds' points are page-locked host memory, copied to the arena
  int64_t in_off = -1;          // first float of its copy in the input arena (set at admission)
  int64_t in_len = 0;           // floats it holds there
  bool in_copy = false;         // admitted, copy not issued yet
  cudaEvent_t in_ev = nullptr;  // recorded on the copy stream after its copies
  ReqState state = kPending;
  em_result res{};
};

struct Flight {
  bool busy = false;
  bool holds_maps = false;      // its maps are released once ev_maps has passed
  cudaEvent_t ev = nullptr;     // everything done (read-backs landed): tickets complete
  cudaEvent_t ev_maps = nullptr;  // updates and layer reads done: the maps may take new updates
  std::vector<uint64_t> tickets;
  std::vector<int32_t> maps;
  int64_t bytes = 0;
};

constexpr int64_t kRecordBytes = EM_SERVE_RECORD_BYTES;  // one grouped record per point
static_assert(kRecordBytes == sizeof(float4), "record size");

}  // namespace

struct em_server {
  em_server_cfg cfg{};
  std::vector<em_map*> maps;
  std::vector<int64_t> map_bytes;
  std::vector<char> map_busy;
  std::vector<char> blocked;  // batch-builder scratch, one flag per map
  std::vector<cudaStream_t> streams;
  std::vector<em_batch*> batches;
  std::vector<float*> stage;  // per batch stream: layer reads bound for host memory land here first
  int64_t stage_cap = 0;      // floats per stage buffer
  // host clouds: copied at admission, on a stream of their own, into a ring
  // arena of device memory (allocated on the first host request), so the copy
  // of a waiting request overlaps the batches already running
  float* in_arena = nullptr;
  int64_t in_cap = 0;                       // floats
  struct InAlloc { uint64_t ticket; int64_t off, end; bool done; };
  std::deque<InAlloc> in_allocs;            // allocation order
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<Flight> flights;            // batched: one per stream; plain: grows as needed
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> pending, admitted;
  std::unordered_map<uint64_t, Request> reqs;
  uint64_t next_ticket = 1;
  int64_t bytes_in_use = 0, fixed_bytes = 0;
  int32_t slots_in_use = 0;
  int32_t maps_added = 0;
  em_server_stats st{};
  bool stop = false;
  std::thread worker;
};

namespace {

// Floats a request's host clouds take in the arena (each cloud 16-byte aligned).
int64_t host_floats(const Request& r) {
  int64_t f = 0;
  for (const em_cloud& c : r.clouds) f += (c.n * c.stride + 3) & ~int64_t(3);
  return f;
}

// Ring allocation of `len` floats in the input arena (allocations are freed
// roughly in order; the oldest live one bounds the ring); -1 when full.
int64_t arena_alloc(em_server* s, uint64_t ticket, int64_t len) {
  int64_t off = -1;
  if (s->in_allocs.empty()) {
    off = len <= s->in_cap ? 0 : -1;
  } else {
    const int64_t tail = s->in_allocs.front().off, head = s->in_allocs.back().end;
    if (head >= tail) {  // used region [tail, head)
      if (head + len <= s->in_cap) off = head;
      else if (len <= tail) off = 0;
    } else if (head + len <= tail) {  // wrapped: used [tail, cap) and [0, head)
      off = head;
    }
  }
  if (off >= 0) s->in_allocs.push_back({ticket, off, off + len, false});
  return off;
}

void arena_free(em_server* s, uint64_t ticket) {
  for (auto& a : s->in_allocs)
    if (a.ticket == ticket) a.done = true;
  while (!s->in_allocs.empty() && s->in_allocs.front().done) s->in_allocs.pop_front();
}

// Release what an admitted or finished request holds besides its slot and bytes.
void release_host(em_server* s, uint64_t ticket, Request& r) {
  if (r.in_off >= 0) arena_free(s, ticket);
  r.in_off = -1;
  if (r.in_ev) s->ev_pool.push_back(r.in_ev);
  r.in_ev = nullptr;
}

// Move pending requests into the admitted set while slots and memory allow
// (strict arrival order); a request with host clouds also needs room in the
// input arena and an event for its copy.  Caller holds the lock.
void admit(em_server* s) {
  while (!s->pending.empty()) {
    Request& r = s->reqs[s->pending.front()];
    if (s->slots_in_use >= s->cfg.max_slots) break;
    if (s->bytes_in_use + r.bytes > s->cfg.budget_bytes) break;
    if (r.on_host) {
      if (s->ev_pool.empty()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) break;
        s->ev_pool.push_back(e);
      }
      r.in_len = host_floats(r);
      r.in_off = arena_alloc(s, s->pending.front(), r.in_len);
      if (r.in_off < 0) break;
      r.in_ev = s->ev_pool.back();
      s->ev_pool.pop_back();
      r.in_copy = true;
    }
    s->bytes_in_use += r.bytes;
    if (s->bytes_in_use > s->st.peak_bytes) s->st.peak_bytes = s->bytes_in_use;
    s->slots_in_use += 1;
    r.state = kAdmitted;
    s->admitted.push_back(s->pending.front());
    s->pending.pop_front();
  }
}

void complete(em_server* s, Flight& f, int status) {
  const int64_t t = now_ns();
  for (uint64_t tk : f.tickets) {
    Request& r = s->reqs[tk];
    release_host(s, tk, r);
    r.state = kDone;
    r.res.status = status;
    r.res.t_done_ns = t;
    s->bytes_in_use -= r.bytes;
    s->slots_in_use -= 1;
    s->st.completed += 1;
  }
  if (f.holds_maps)
    for (int32_t m : f.maps) s->map_busy[m] = 0;
  f.holds_maps = false;
  f.tickets.clear();
  f.maps.clear();
  f.busy = false;
}

// The device clouds of an admitted host request: its clouds' copies in the arena.
void arena_clouds(em_server* s, const Request& r, std::vector<em_cloud>& out) {
  int64_t off = r.in_off;
  for (const em_cloud& c : r.clouds) {
    em_cloud d = c;
    d.points = s->in_arena + off;
    off += (c.n * c.stride + 3) & ~int64_t(3);
    out.push_back(d);
  }
}

// Issue the arena copies of newly admitted host requests on the copy stream
// (each after the request's ready event) and record their events.  Called
// with the lock held; drops it while the copies are issued.
void issue_host_copies(em_server* s, std::unique_lock<std::mutex>& lk) {
  struct Job { const float* src; float* dst; size_t bytes; };
  struct Rq { std::vector<Job> jobs; cudaEvent_t ready, ev; };
  std::vector<Rq> todo;
  for (uint64_t tk : s->admitted) {
    Request& r = s->reqs[tk];
    if (!r.in_copy) continue;
    r.in_copy = false;
    Rq q{{}, r.ready, r.in_ev};
    int64_t off = r.in_off;
    for (const em_cloud& c : r.clouds) {
      const size_t floats = (size_t)(c.n * c.stride);
      if (floats) q.jobs.push_back({c.points, s->in_arena + off, floats * sizeof(float)});
      off += (int64_t)((floats + 3) & ~size_t(3));
    }
    todo.push_back(q);
  }
  if (todo.empty()) return;
  lk.unlock();
  for (const Rq& q : todo) {
    if (q.ready) cudaStreamWaitEvent(s->copy_stream, q.ready, 0);
    for (const Job& j : q.jobs) {
      cudaError_t e = cudaMemcpyAsync(j.dst, j.src, j.bytes, cudaMemcpyHostToDevice, s->copy_stream);
      if (e != cudaSuccess) map_record_error("host cloud copy", e);  // the batch's event reports it
    }
    cudaEventRecord(q.ev, s->copy_stream);
  }
  lk.lock();
}

// One worker pass: complete finished flights, admit, launch.  Returns true when
// anything is in flight or waiting (the worker keeps polling).
bool worker_pass(em_server* s, std::unique_lock<std::mutex>& lk) {
  // completions (cudaEventQuery does not block)
  for (Flight& f : s->flights) {
    if (!f.busy) continue;
    if (f.holds_maps && f.ev_maps && cudaEventQuery(f.ev_maps) == cudaSuccess) {
      // the maps are read: later updates may run while the read-backs travel
      for (int32_t m : f.maps) s->map_busy[m] = 0;
      f.holds_maps = false;
    }
    cudaError_t q = cudaEventQuery(f.ev);
    if (q == cudaErrorNotReady) continue;
    complete(s, f, q == cudaSuccess ? EM_OK : map_record_error("request", q));
    s->cv_done.notify_all();
  }
  admit(s);
  issue_host_copies(s, lk);
  if (s->cfg.mode == EM_SERVE_PLAIN) {
    // one update per request, arrival order, one stream
    while (!s->admitted.empty()) {
      const uint64_t tk = s->admitted.front();
      Request& r = s->reqs[tk];
      size_t fi = 0;
      while (fi < s->flights.size() && s->flights[fi].busy) ++fi;
      if (fi == s->flights.size()) {
        Flight nf;
        if (cudaEventCreateWithFlags(&nf.ev, cudaEventDisableTiming) != cudaSuccess) break;
        s->flights.push_back(nf);
      }
      Flight& f = s->flights[fi];
      s->admitted.pop_front();
      r.state = kRunning;
      r.res.t_start_ns = now_ns();
      r.res.batch_size = 1;
      f.busy = true;
      f.tickets.assign(1, tk);
      f.maps.clear();
      em_map* m = s->maps[r.map_id];
      std::vector<em_cloud> cl;
      if (r.on_host) arena_clouds(s, r, cl);
      else cl = r.clouds;
      cudaEvent_t ready = r.on_host ? r.in_ev : r.ready;  // host clouds: their copy (after ready)
      const uint32_t read_mask = r.read_mask;
      float* read_dst = r.read_dst;
      lk.unlock();
      if (ready) cudaStreamWaitEvent(s->streams[0], ready, 0);
      int rc = em_update_multi(m, cl.data(), (int32_t)cl.size(), (em_stream_t)s->streams[0]);
      if (rc == EM_OK && read_mask) rc = map_read_layers(m, read_mask, read_dst, s->streams[0]);
      if (rc == EM_OK) cudaEventRecord(f.ev, s->streams[0]);
      lk.lock();
      s->st.batches += 1;
      s->st.batched_requests += 1;
      if (s->st.max_batch_size < 1) s->st.max_batch_size = 1;
      if (rc != EM_OK) complete(s, f, rc);
    }
  } else {
    for (size_t si = 0; si < s->streams.size(); ++si) {
      Flight& f = s->flights[si];
      if (f.busy || s->admitted.empty()) continue;
      // distinct idle maps in arrival order, within the batch limits; a map whose
      // earlier request is not taken (the batch is full) takes no later one, so
      // each map's updates stay in arrival order
      std::vector<uint64_t> take;
      std::vector<int32_t> bmaps;
      int64_t pts = 0;
      s->blocked.assign(s->maps.size(), 0);
      for (auto it = s->admitted.begin(); it != s->admitted.end();) {
        Request& r = s->reqs[*it];
        const bool skip = s->map_busy[r.map_id] != 0 || s->blocked[r.map_id] != 0 ||
                          (int32_t)bmaps.size() >= s->cfg.max_batch_maps || pts + r.points > s->cfg.max_batch_points;
        s->blocked[r.map_id] = 1;  // at most one request per map, the earliest
        if (skip) {
          ++it;
          continue;
        }
        take.push_back(*it);
        bmaps.push_back(r.map_id);
        pts += r.points;
        it = s->admitted.erase(it);
      }
      if (take.empty()) break;
      std::vector<em_map*> pm;
      std::vector<em_cloud> pc;
      std::vector<cudaEvent_t> ready;
      // layer reads: host-bound ones through this stream's stage buffer while it
      // has room (then copied by DMA after the maps are released), others direct
      std::vector<em_map*> rmaps;
      std::vector<uint32_t> rmasks;
      std::vector<float*> rdst;
      struct Staged { float* host; int64_t off, floats; };
      std::vector<Staged> staged;
      int64_t stage_used = 0;
      const int64_t t0 = now_ns();
      for (uint64_t tk : take) {
        Request& r = s->reqs[tk];
        if (r.on_host) ready.push_back(r.in_ev);  // its copy, which waited for ready
        else if (r.ready) ready.push_back(r.ready);
        if (r.read_mask) {
          rmaps.push_back(s->maps[r.map_id]);
          rmasks.push_back(r.read_mask);
          if (r.read_host && stage_used + r.read_floats <= s->stage_cap) {
            rdst.push_back(s->stage[si] + stage_used);
            staged.push_back({r.read_host, stage_used, r.read_floats});
            stage_used += r.read_floats;
          } else {
            rdst.push_back(r.read_dst);
          }
        }
        r.state = kRunning;
        r.res.t_start_ns = t0;
        r.res.batch_size = (int32_t)take.size();
        const size_t c0 = pc.size();
        if (r.on_host) arena_clouds(s, r, pc);
        else pc.insert(pc.end(), r.clouds.begin(), r.clouds.end());
        for (size_t i = c0; i < pc.size(); ++i) pm.push_back(s->maps[r.map_id]);
        s->map_busy[r.map_id] = 1;
      }
      f.busy = true;
      f.holds_maps = true;
      f.tickets = take;
      f.maps = bmaps;
      s->st.batches += 1;
      s->st.batched_requests += (int64_t)take.size();
      if ((int64_t)take.size() > s->st.max_batch_size) s->st.max_batch_size = (int64_t)take.size();
      lk.unlock();
      for (cudaEvent_t e : ready) cudaStreamWaitEvent(s->streams[si], e, 0);
      int rc = em_update_batch(s->batches[si], pm.data(), pc.data(), (int32_t)pc.size(), (em_stream_t)s->streams[si]);
      if (rc == EM_OK && !rmaps.empty())
        rc = maps_read_layers(rmaps.data(), rmasks.data(), rdst.data(), (int)rmaps.size(), s->streams[si]);
      if (rc == EM_OK) cudaEventRecord(f.ev_maps, s->streams[si]);
      for (size_t i = 0; i < staged.size() && rc == EM_OK; ++i) {
        cudaError_t ce = cudaMemcpyAsync(staged[i].host, s->stage[si] + staged[i].off, staged[i].floats * sizeof(float),
                                         cudaMemcpyDeviceToHost, s->streams[si]);
        if (ce != cudaSuccess) rc = map_record_error("read-back copy", ce);
      }
      if (rc == EM_OK) cudaEventRecord(f.ev, s->streams[si]);
      lk.lock();
      if (rc != EM_OK) {
        complete(s, f, rc);
        s->cv_done.notify_all();
      }
    }
  }
  bool busy = !s->pending.empty() || !s->admitted.empty();
  for (const Flight& f : s->flights) busy |= f.busy;
  return busy;
}

void worker_main(em_server* s) {
  cudaSetDevice(s->cfg.device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    const bool busy = worker_pass(s, lk);
    if (s->stop && !busy) break;
    if (busy) {
      // poll the in-flight events; let submitters in between
      lk.unlock();
      std::this_thread::yield();
      lk.lock();
    } else {
      s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty(); });
    }
  }
}

int64_t map_device_bytes(const em_map* m) {
  em_info i;
  em_get_info(m, &i);
  return i.device_bytes;
}

}  // namespace

extern "C" {

int em_server_create(const em_server_cfg* cfg, em_server** out) {
  if (!cfg || !out) return EM_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->budget_bytes <= 0 || cfg->max_slots < 1 || cfg->n_streams < 1 || cfg->max_batch_maps < 1 ||
      cfg->max_batch_points < 1 || cfg->max_map_cells < 1 || (cfg->mode != EM_SERVE_BATCHED && cfg->mode != EM_SERVE_PLAIN))
    return EM_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) return EM_ERR_INVALID_ARG;
  if (cudaSetDevice(cfg->device) != cudaSuccess) return EM_ERR_CUDA;
  em_server* s = new (std::nothrow) em_server();
  if (!s) return EM_ERR_OOM;
  s->cfg = *cfg;
  const int ns = cfg->mode == EM_SERVE_PLAIN ? 1 : cfg->n_streams;
  int rc = EM_OK;
  for (int i = 0; i < ns && rc == EM_OK; ++i) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { rc = EM_ERR_CUDA; break; }
    s->streams.push_back(st);
    if (cfg->mode == EM_SERVE_BATCHED) {
      em_batch* b = nullptr;
      rc = em_batch_create(cfg->device, cfg->max_batch_maps, cfg->max_batch_maps * 8, cfg->max_batch_points,
                           cfg->max_map_cells, cfg->batch_flags, &b);
      if (rc == EM_OK) {
        s->batches.push_back(b);
        s->fixed_bytes += cfg->max_batch_points * kRecordBytes;
      }
      Flight f;
      if (rc == EM_OK && cudaEventCreateWithFlags(&f.ev, cudaEventDisableTiming) != cudaSuccess) rc = EM_ERR_CUDA;
      if (rc == EM_OK && cudaEventCreateWithFlags(&f.ev_maps, cudaEventDisableTiming) != cudaSuccess) rc = EM_ERR_CUDA;
      s->flights.push_back(f);
      // one layer of every map of a full batch, at most 64 MiB (reads that do not
      // fit are written to their destination directly)
      s->stage_cap = std::min<int64_t>((int64_t)cfg->max_batch_maps * cfg->max_map_cells, int64_t(1) << 24);
      float* st = nullptr;
      if (rc == EM_OK && cudaMalloc((void**)&st, (size_t)s->stage_cap * sizeof(float)) != cudaSuccess) rc = EM_ERR_OOM;
      s->stage.push_back(st);
      if (rc == EM_OK) s->fixed_bytes += s->stage_cap * (int64_t)sizeof(float);
    }
  }
  if (rc == EM_OK && s->fixed_bytes > cfg->budget_bytes) rc = EM_ERR_REJECTED;
  if (rc != EM_OK) {
    for (em_batch* b : s->batches) em_batch_destroy(b);
    for (Flight& f : s->flights) {
      if (f.ev) cudaEventDestroy(f.ev);
      if (f.ev_maps) cudaEventDestroy(f.ev_maps);
    }
    for (float* st : s->stage) cudaFree(st);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    delete s;
    return rc;
  }
  s->bytes_in_use = s->fixed_bytes;
  s->st.bytes_in_use = s->bytes_in_use;
  s->worker = std::thread(worker_main, s);
  *out = s;
  return EM_OK;
}

int em_server_add_map(em_server* s, const em_params* params, int32_t* map_id) {
  if (!s || !params || !map_id) return EM_ERR_INVALID_ARG;
  if ((int64_t)params->width * params->height > s->cfg.max_map_cells) return EM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  s->maps_added += 1;
  if (s->cfg.fail_alloc_at > 0 && s->maps_added == s->cfg.fail_alloc_at) return EM_ERR_OOM;
  em_params p = *params;
  p.flags &= ~(uint32_t)EM_F_TRACE;
  em_map* m = nullptr;
  int rc = em_create(&p, s->cfg.device, &m);
  if (rc) return rc;
  const int64_t bytes = map_device_bytes(m);
  if (s->bytes_in_use + bytes > s->cfg.budget_bytes) {
    em_destroy(m);
    return EM_ERR_REJECTED;
  }
  s->bytes_in_use += bytes;
  s->maps.push_back(m);
  s->map_bytes.push_back(bytes);
  s->map_busy.push_back(0);
  *map_id = (int32_t)s->maps.size() - 1;
  return EM_OK;
}

int em_server_map(em_server* s, int32_t map_id, em_map** out) {
  if (!s || !out) return EM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (map_id < 0 || map_id >= (int32_t)s->maps.size()) return EM_ERR_INVALID_ARG;
  *out = s->maps[map_id];
  return EM_OK;
}

int em_server_submit(em_server* s, int32_t map_id, const em_cloud* clouds, int32_t n_clouds, uint64_t* ticket) {
  return em_server_submit_after(s, map_id, clouds, n_clouds, nullptr, ticket);
}

int em_server_submit_after(em_server* s, int32_t map_id, const em_cloud* clouds, int32_t n_clouds, void* ready,
                           uint64_t* ticket) {
  if (!ticket) return EM_ERR_INVALID_ARG;
  em_request r{};
  r.map_id = map_id;
  r.n_clouds = n_clouds;
  r.clouds = clouds;
  return em_server_submit_many(s, &r, 1, ready, ticket);
}

int em_server_submit_many(em_server* s, const em_request* reqs, int32_t n, void* ready, uint64_t* tickets) {
  if (!s || !reqs || n < 1 || !tickets) return EM_ERR_INVALID_ARG;
  std::vector<int64_t> pts(n, 0);
  std::vector<float*> dst(n, nullptr);
  bool any_host = false;
  for (int32_t q = 0; q < n; ++q) {
    const em_request& r = reqs[q];
    if (!r.clouds || r.n_clouds < 1 || r.n_clouds > 8) return EM_ERR_INVALID_ARG;
    for (int i = 0; i < r.n_clouds; ++i) {
      const em_cloud& c = r.clouds[i];
      if (c.n < 0 || (c.stride != 3 && c.stride != 4) || (c.n > 0 && !c.points) || !word_aligned(c.points))
        return EM_ERR_INVALID_ARG;
      if (r.clouds_on_host && c.n > 0) {  // page-locked host memory: the copy is asynchronous DMA
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, c.points) != cudaSuccess) {
          cudaGetLastError();
          return EM_ERR_INVALID_ARG;
        }
        if (a.type != cudaMemoryTypeHost) return EM_ERR_INVALID_ARG;
      }
      pts[q] += c.n;
    }
    any_host |= r.clouds_on_host != 0;
    if (r.read_mask) {
      if ((r.read_mask >> 11) || !r.read_dst || !word_aligned(r.read_dst)) return EM_ERR_INVALID_ARG;
      // the GPU writes the read-back itself: device memory, or page-locked host
      // memory mapped into the device's address space
      cudaPointerAttributes a{};
      if (cudaPointerGetAttributes(&a, r.read_dst) != cudaSuccess) {
        cudaGetLastError();
        return EM_ERR_INVALID_ARG;
      }
      const bool host = a.type == cudaMemoryTypeHost;
      const bool devmem = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
      if ((r.read_to_host != 0) != host || !(host || devmem) || !a.devicePointer) return EM_ERR_INVALID_ARG;
      if (devmem && a.device != s->cfg.device) return EM_ERR_INVALID_ARG;
      dst[q] = static_cast<float*>(a.devicePointer);
    }
  }
  std::lock_guard<std::mutex> lk(s->mu);
  const int64_t maps_bytes = [&] {
    int64_t t = 0;
    for (int64_t b : s->map_bytes) t += b;
    return t;
  }();
  for (int32_t q = 0; q < n; ++q) {
    if (reqs[q].map_id < 0 || reqs[q].map_id >= (int32_t)s->maps.size()) return EM_ERR_INVALID_ARG;
  }
  if (any_host && !s->in_arena) {
    // the input arena: full batches of stride-4 points for every stream and two more
    // (the admitted requests waiting for a stream), each cloud padded to 16 bytes
    const int64_t per = s->cfg.max_batch_points * 4 + 4 * (int64_t)s->cfg.max_batch_maps * 8;
    const int64_t cap = per * ((int64_t)s->streams.size() + 2);
    const int64_t bytes = cap * (int64_t)sizeof(float);
    if (s->bytes_in_use + bytes > s->cfg.budget_bytes) return EM_ERR_REJECTED;
    cudaSetDevice(s->cfg.device);
    if (cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      s->copy_stream = nullptr;
      return EM_ERR_CUDA;
    }
    if (cudaMalloc((void**)&s->in_arena, (size_t)bytes) != cudaSuccess) {
      cudaGetLastError();
      s->in_arena = nullptr;
      return EM_ERR_OOM;
    }
    s->in_cap = cap;
    s->fixed_bytes += bytes;
    s->bytes_in_use += bytes;
    if (s->bytes_in_use > s->st.peak_bytes) s->st.peak_bytes = s->bytes_in_use;
  }
  for (int32_t q = 0; q < n; ++q) {
    if (pts[q] > s->cfg.max_batch_points || s->fixed_bytes + maps_bytes + pts[q] * kRecordBytes > s->cfg.budget_bytes) {
      s->st.submitted += 1;
      s->st.rejected += 1;
      return EM_ERR_REJECTED;
    }
  }
  const int64_t t_submit = now_ns();
  for (int32_t q = 0; q < n; ++q) {
    const em_request& in = reqs[q];
    s->st.submitted += 1;
    const uint64_t tk = s->next_ticket++;
    Request& r = s->reqs[tk];
    r.map_id = in.map_id;
    r.clouds.assign(in.clouds, in.clouds + in.n_clouds);
    r.points = pts[q];
    r.bytes = pts[q] * kRecordBytes;
    r.ready = (cudaEvent_t)ready;
    r.read_mask = in.read_mask;
    r.read_dst = dst[q];
    r.read_host = in.read_mask && in.read_to_host ? in.read_dst : nullptr;
    r.on_host = in.clouds_on_host != 0;
    if (in.read_mask)
      r.read_floats = (int64_t)__builtin_popcount(in.read_mask) * map_cells(s->maps[in.map_id]);
    r.res.map_id = in.map_id;
    r.res.points = pts[q];
    r.res.t_submit_ns = t_submit;
    s->pending.push_back(tk);
    tickets[q] = tk;
  }
  s->cv_work.notify_one();
  return EM_OK;
}

int em_server_wait(em_server* s, uint64_t ticket, int64_t timeout_us, em_result* out) {
  if (!s) return EM_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->reqs.find(ticket) == s->reqs.end()) return EM_ERR_INVALID_ARG;
  // find, never operator[]: another thread may have waited for (and forgotten)
  // the same ticket meanwhile, and a lookup must not bring it back
  auto done = [&] {
    auto it = s->reqs.find(ticket);
    return it == s->reqs.end() || it->second.state == kDone;
  };
  if (timeout_us < 0) {
    s->cv_done.wait(lk, done);
  } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done)) {
    return EM_ERR_TIMEOUT;
  }
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return EM_ERR_INVALID_ARG;
  if (out) *out = it->second.res;
  s->reqs.erase(it);
  return EM_OK;
}

int em_server_wait_many(em_server* s, const uint64_t* tickets, int32_t n, int64_t timeout_us, em_result* out) {
  if (!s || n < 0 || (n > 0 && !tickets)) return EM_ERR_INVALID_ARG;
  {  // each ticket once
    std::vector<uint64_t> t(tickets, tickets + n);
    std::sort(t.begin(), t.end());
    if (std::adjacent_find(t.begin(), t.end()) != t.end()) return EM_ERR_INVALID_ARG;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  for (int32_t i = 0; i < n; ++i)
    if (s->reqs.find(tickets[i]) == s->reqs.end()) return EM_ERR_INVALID_ARG;
  auto done = [&] {  // (find, never operator[]: see em_server_wait)
    for (int32_t i = 0; i < n; ++i) {
      auto it = s->reqs.find(tickets[i]);
      if (it != s->reqs.end() && it->second.state != kDone) return false;
    }
    return true;
  };
  if (timeout_us < 0) {
    s->cv_done.wait(lk, done);
  } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done)) {
    return EM_ERR_TIMEOUT;
  }
  int rc = EM_OK;
  for (int32_t i = 0; i < n; ++i) {
    auto it = s->reqs.find(tickets[i]);
    if (it == s->reqs.end()) {  // forgotten by a concurrent wait
      rc = EM_ERR_INVALID_ARG;
      continue;
    }
    if (out) out[i] = it->second.res;
    s->reqs.erase(it);
  }
  return rc;
}

int em_server_cancel(em_server* s, uint64_t ticket) {
  if (!s) return EM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return EM_ERR_INVALID_ARG;
  Request& r = it->second;
  if (r.state == kRunning || r.state == kDone) return EM_ERR_BUSY;
  auto drop = [&](std::deque<uint64_t>& q) {
    for (auto q_it = q.begin(); q_it != q.end(); ++q_it)
      if (*q_it == ticket) { q.erase(q_it); return true; }
    return false;
  };
  if (r.state == kAdmitted) {
    drop(s->admitted);
    s->bytes_in_use -= r.bytes;
    s->slots_in_use -= 1;
    release_host(s, ticket, r);  // a copy in flight lands before any later copy reuses the room
  } else {
    drop(s->pending);
  }
  r.state = kDone;
  r.res.status = EM_ERR_TIMEOUT;
  r.res.t_done_ns = now_ns();
  s->st.cancelled += 1;
  s->cv_done.notify_all();
  s->cv_work.notify_one();
  return EM_OK;
}

int em_server_drain(em_server* s, int64_t timeout_us) {
  if (!s) return EM_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto idle = [&] {
    if (!s->pending.empty() || !s->admitted.empty()) return false;
    for (const Flight& f : s->flights)
      if (f.busy) return false;
    return true;
  };
  if (timeout_us < 0) {
    s->cv_done.wait(lk, idle);
  } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), idle)) {
    return EM_ERR_TIMEOUT;
  }
  return EM_OK;
}

int em_server_get_stats(em_server* s, em_server_stats* out) {
  if (!s || !out) return EM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->bytes_in_use = s->bytes_in_use;
  out->slots_in_use = s->slots_in_use;
  return EM_OK;
}

int em_server_set_tuning(em_server* s, const em_tuning* t) {
  if (!s || !t) return EM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  for (em_batch* b : s->batches) {
    int rc = em_batch_set_tuning(b, t);
    if (rc) return rc;
  }
  return EM_OK;
}

int em_server_destroy(em_server* s) {
  if (!s) return EM_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->cfg.device);
  for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
  for (em_batch* b : s->batches) em_batch_destroy(b);
  for (Flight& f : s->flights) {
    if (f.ev) cudaEventDestroy(f.ev);
    if (f.ev_maps) cudaEventDestroy(f.ev_maps);
  }
  for (float* st : s->stage) cudaFree(st);
  if (s->copy_stream) cudaStreamSynchronize(s->copy_stream);
  cudaFree(s->in_arena);
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  for (auto& kv : s->reqs)
    if (kv.second.in_ev) cudaEventDestroy(kv.second.in_ev);
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  for (em_map* m : s->maps) em_destroy(m);
  delete s;
  return EM_OK;
}

}  // extern "C"
