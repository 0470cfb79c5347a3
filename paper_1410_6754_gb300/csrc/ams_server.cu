// Serving loop: continuous batching of sort requests on one GPU.
//
// Requests (device buffers, any size and key type) are submitted from host threads
// and complete asynchronously.  One host thread runs the loop:
//   * completions: a worker stream whose batch event has fired hands its requests
//     back (status from the worker's context, host completion time), and their
//     scratch leaves the budget;
//   * admission, first come first served: a request enters when the scratch of the
//     requests in flight plus its own stays within the budget and a worker stream is
//     free (a request larger than the whole budget runs alone);
//   * packing: consecutive keys-only requests of one key type, each of at most
//     `pack_max_keys` keys, are gathered into one staging buffer and sorted by one
//     segmented sort (one level loop over all of them), then copied back; other
//     requests run as one sort each.
// Every worker stream has its own context (scratch, tables) that stays allocated
// between requests, so requests overlap on the device.  Built on the public C ABI.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "ams.h"

namespace {

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

size_t key_bytes(ams_key_type kt) { return kt == AMS_U64 ? 8 : 4; }

struct Job {
  uint64_t ticket;
  ams_request rq;
  uint32_t buckets[8];
  uint64_t scratch;  // budget charge
  uint64_t t_submit;
};

struct TicketState {
  bool done = false;
  ams_status status = AMS_OK;
  uint64_t t_submit = 0, t_done = 0;
};

struct Worker {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  void* ctx = nullptr;
  bool busy = false;
  std::vector<Job> jobs;       // the batch in flight
  ams_status launch_status = AMS_OK;
  // packing buffers (grown on demand; freed only at the end)
  void* stage = nullptr;
  size_t stage_bytes = 0;
  uint64_t* d_off = nullptr;
  uint64_t* h_off = nullptr;  // pinned
  size_t off_cap = 0;
};

}  // namespace

struct ams_server {
  uint64_t budget = 0;
  uint64_t pack_max = 0;
  uint64_t pack_total = 0;  // largest packed batch (keys)
  int device = 0;
  std::vector<Worker> workers;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job> queue;
  std::unordered_map<uint64_t, TicketState> tickets;
  uint64_t next_ticket = 1;
  uint64_t in_flight_bytes = 0;
  bool stop = false;
  std::thread loop;
  std::atomic<uint64_t> batches{0}, packed_requests{0};
};

namespace {

// Scratch a request holds while in flight: its context workspace (the library's own
// figure for the request's plan) plus, for a packable request, its share of the
// packing stage.
uint64_t scratch_of(const ams_request& rq) {
  const uint64_t ws = ams_request_scratch_bytes(&rq);
  return ws + rq.n * key_bytes(rq.kt) + (1u << 16);
}

constexpr uint64_t kFreeSpare = 256ull << 20;  // device memory kept free at admission

// Bytes the worker's context would have to add to run `j` (0 if it fits already).
uint64_t growth_of(const Worker& wk, const Job& j) {
  const uint64_t need = ams_request_scratch_bytes(&j.rq);
  const uint64_t have = ams_context_scratch_bytes(wk.ctx);
  return need > have ? need - have : 0;
}

ams_status grow_stage(Worker& wk, size_t bytes, size_t segs) {
  if (bytes > wk.stage_bytes) {
    if (wk.stage && cudaFree(wk.stage) != cudaSuccess) return AMS_ERR_CUDA;
    wk.stage = nullptr;
    if (cudaMalloc(&wk.stage, bytes) != cudaSuccess) return AMS_ERR_OOM;
    wk.stage_bytes = bytes;
  }
  if (segs + 1 > wk.off_cap) {
    if (wk.d_off) cudaFree(wk.d_off);
    if (wk.h_off) cudaFreeHost(wk.h_off);
    wk.d_off = nullptr;
    wk.h_off = nullptr;
    const size_t cap = (segs + 1) * 2;
    if (cudaMalloc(&wk.d_off, cap * 8) != cudaSuccess) return AMS_ERR_OOM;
    if (cudaMallocHost(&wk.h_off, cap * 8) != cudaSuccess) return AMS_ERR_OOM;
    wk.off_cap = cap;
  }
  return AMS_OK;
}

// Enqueue the worker's batch on its stream (called with the server lock released).
ams_status launch(ams_server* s, Worker& wk) {
  if (cudaSetDevice(s->device) != cudaSuccess) return AMS_ERR_CUDA;
  for (Job& j : wk.jobs) j.rq.buckets_per_level = j.buckets;  // (jobs were copied)
  ams_status st = AMS_OK;
  if (wk.jobs.size() == 1) {
    st = ams_sort_request(wk.ctx, &wk.jobs[0].rq, wk.stream);
  } else {
    // packed keys-only requests of one key type: gather, one segmented sort, scatter
    const ams_key_type kt = wk.jobs[0].rq.kt;
    const size_t w = key_bytes(kt);
    uint64_t total = 0;
    for (const Job& j : wk.jobs) total += j.rq.n;
    if ((st = grow_stage(wk, total * w, wk.jobs.size())) != AMS_OK) return st;
    char* stage = (char*)wk.stage;
    uint64_t off = 0;
    for (size_t i = 0; i < wk.jobs.size(); ++i) {
      const ams_request& r = wk.jobs[i].rq;
      wk.h_off[i] = off;
      if (r.n && cudaMemcpyAsync(stage + off * w, r.keys_in, r.n * w, cudaMemcpyDeviceToDevice, wk.stream) !=
                     cudaSuccess)
        return AMS_ERR_CUDA;
      off += r.n;
    }
    wk.h_off[wk.jobs.size()] = off;
    if (cudaMemcpyAsync(wk.d_off, wk.h_off, (wk.jobs.size() + 1) * 8, cudaMemcpyHostToDevice, wk.stream) !=
        cudaSuccess)
      return AMS_ERR_CUDA;
    ams_request seg = wk.jobs[0].rq;
    seg.keys_in = stage;
    seg.keys_out = stage;
    seg.vals_in = nullptr;
    seg.vals_out = nullptr;
    seg.d_offsets = wk.d_off;
    seg.nseg = wk.jobs.size();
    seg.n = total;
    if ((st = ams_sort_request(wk.ctx, &seg, wk.stream)) != AMS_OK) return st;
    for (size_t i = 0; i < wk.jobs.size(); ++i) {
      const ams_request& r = wk.jobs[i].rq;
      if (r.n && cudaMemcpyAsync(r.keys_out, stage + wk.h_off[i] * w, r.n * w, cudaMemcpyDeviceToDevice,
                                 wk.stream) != cudaSuccess)
        return AMS_ERR_CUDA;
    }
  }
  if (st == AMS_OK && cudaEventRecord(wk.done, wk.stream) != cudaSuccess) st = AMS_ERR_CUDA;
  return st;
}

bool packable(const ams_server* s, const Job& j) {
  return j.rq.vals_in == nullptr && j.rq.d_offsets == nullptr && j.rq.n <= s->pack_max;
}

void run_loop(ams_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    // completions
    bool any_busy = false;
    for (Worker& wk : s->workers) {
      if (!wk.busy) continue;
      cudaError_t q = wk.launch_status == AMS_OK ? cudaEventQuery(wk.done) : cudaSuccess;
      if (q == cudaErrorNotReady) {
        any_busy = true;
        continue;
      }
      ams_status st = wk.launch_status;
      if (st == AMS_OK) st = q == cudaSuccess ? ams_context_sync(wk.ctx) : AMS_ERR_CUDA;
      const uint64_t t = now_ns();
      for (const Job& j : wk.jobs) {
        TicketState& ts = s->tickets[j.ticket];
        ts.done = true;
        ts.status = st;
        ts.t_done = t;
        s->in_flight_bytes -= j.scratch;
      }
      wk.jobs.clear();
      wk.busy = false;
      s->cv_done.notify_all();
    }
    // admission and dispatch
    for (Worker& wk : s->workers) {
      if (wk.busy || s->queue.empty()) continue;
      const Job& head = s->queue.front();
      {
        // admission by budget and by free device memory: a context that must grow
        // allocates, so the growth has to fit in what the device has free now
        const uint64_t grow = s->in_flight_bytes > 0 ? growth_of(wk, head) : 0;
        size_t free_b = 0, total_b = 0;
        if (grow > 0 && cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) break;
        if (!ams_server_admits(s->in_flight_bytes, head.scratch, s->budget, grow, free_b)) break;
      }
      wk.jobs.clear();
      wk.jobs.push_back(head);
      s->in_flight_bytes += head.scratch;
      s->queue.pop_front();
      if (packable(s, wk.jobs[0])) {
        uint64_t total = wk.jobs[0].rq.n;
        while (!s->queue.empty()) {
          const Job& nx = s->queue.front();
          if (!packable(s, nx) || nx.rq.kt != wk.jobs[0].rq.kt || total + nx.rq.n > s->pack_total ||
              (s->budget && s->in_flight_bytes + nx.scratch > s->budget))
            break;
          total += nx.rq.n;
          s->in_flight_bytes += nx.scratch;
          wk.jobs.push_back(nx);
          s->queue.pop_front();
        }
      }
      wk.busy = true;
      any_busy = true;
      s->batches++;
      if (wk.jobs.size() > 1) s->packed_requests += wk.jobs.size();
      lk.unlock();
      wk.launch_status = launch(s, wk);
      // a launch can fail after part of the batch is already queued (a gather copy,
      // the sort itself): let that work drain before the completion pass hands the
      // requests back, so no queued copy or kernel touches buffers the caller may
      // free once its wait returns, and the next batch cannot overwrite the stage
      if (wk.launch_status != AMS_OK) cudaStreamSynchronize(wk.stream);
      lk.lock();
    }
    if (s->stop && s->queue.empty() && !any_busy) break;
    if (any_busy) {
      // poll the device again soon; new submissions wake the loop at once
      s->cv_work.wait_for(lk, std::chrono::microseconds(20));
    } else {
      s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
    }
  }
}

}  // namespace

extern "C" {

AMS_API ams_status ams_server_create(uint64_t hbm_budget_bytes, int streams, uint64_t pack_max_keys,
                                     ams_server** out) {
  if (!out || streams < 1 || streams > 64) return AMS_ERR_INVALID;
  *out = nullptr;
  ams_server* s = new ams_server();
  s->budget = hbm_budget_bytes;
  s->pack_max = pack_max_keys;
  s->pack_total = pack_max_keys ? pack_max_keys * 64 : 0;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return AMS_ERR_CUDA;
  }
  s->workers.resize(streams);
  ams_status st = AMS_OK;
  for (Worker& wk : s->workers) {
    if (cudaStreamCreateWithFlags(&wk.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&wk.done, cudaEventDisableTiming) != cudaSuccess) {
      st = AMS_ERR_CUDA;
      break;
    }
    if ((st = ams_context_create(0, &wk.ctx)) != AMS_OK) break;
  }
  if (st != AMS_OK) {
    ams_server_destroy(s);
    return st;
  }
  s->loop = std::thread(run_loop, s);
  *out = s;
  return AMS_OK;
}

AMS_API int ams_server_admits(uint64_t in_flight, uint64_t scratch, uint64_t budget, uint64_t growth,
                              uint64_t free_bytes) {
  if (in_flight == 0) return 1;  // a request larger than everything runs alone
  if (budget && in_flight + scratch > budget) return 0;
  if (growth && free_bytes < growth + kFreeSpare) return 0;
  return 1;
}

AMS_API ams_status ams_server_reserve(ams_server* s, const ams_request* largest) {
  if (!s || !largest) return AMS_ERR_INVALID;
  const uint64_t need = ams_request_scratch_bytes(largest);
  if (need == 0) return AMS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);  // (the loop launches only with the lock released)
  if (cudaSetDevice(s->device) != cudaSuccess) return AMS_ERR_CUDA;
  for (Worker& wk : s->workers) {
    if (wk.busy) return AMS_ERR_INVALID;  // reserve before submitting
    ams_status st = ams_context_reserve(wk.ctx, need);
    if (st != AMS_OK) return st;
    // the packing stage holds up to pack_total keys of any type, from at most
    // pack_total / 1024 requests of 2^10 keys or more (more grow it in the loop)
    if (s->pack_total && (st = grow_stage(wk, (size_t)s->pack_total * 8, 4096)) != AMS_OK) return st;
  }
  return AMS_OK;
}

AMS_API ams_status ams_server_submit(ams_server* s, const ams_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return AMS_ERR_INVALID;
  if (req->levels < 1 || req->levels > 8 || !req->buckets_per_level) return AMS_ERR_INVALID;
  if (req->n && (!req->keys_in || !req->keys_out)) return AMS_ERR_INVALID;
  Job j{};
  j.rq = *req;
  for (int l = 0; l < req->levels; ++l) j.buckets[l] = req->buckets_per_level[l];
  j.rq.buckets_per_level = j.buckets;
  j.scratch = scratch_of(*req);
  j.t_submit = now_ns();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return AMS_ERR_INVALID;
    j.ticket = s->next_ticket++;
    TicketState& ts = s->tickets[j.ticket];
    ts.t_submit = j.t_submit;
    s->queue.push_back(j);  // (buckets_per_level is re-pointed at launch)
    *ticket = j.ticket;
  }
  s->cv_work.notify_one();
  return AMS_OK;
}

AMS_API ams_status ams_server_wait(ams_server* s, uint64_t ticket, uint64_t* t_submit_ns, uint64_t* t_done_ns) {
  if (!s) return AMS_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return AMS_ERR_INVALID;
  s->cv_done.wait(lk, [&] { return s->tickets[ticket].done; });
  const TicketState ts = s->tickets[ticket];
  s->tickets.erase(ticket);
  if (t_submit_ns) *t_submit_ns = ts.t_submit;
  if (t_done_ns) *t_done_ns = ts.t_done;
  return ts.status;
}

AMS_API int ams_server_done(ams_server* s, uint64_t ticket) {
  if (!s) return -1;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return -1;
  return it->second.done ? 1 : 0;
}

AMS_API ams_status ams_server_counters(ams_server* s, uint64_t* batches, uint64_t* packed_requests) {
  if (!s) return AMS_ERR_INVALID;
  if (batches) *batches = s->batches.load();
  if (packed_requests) *packed_requests = s->packed_requests.load();
  return AMS_OK;
}

AMS_API ams_status ams_server_destroy(ams_server* s) {
  if (!s) return AMS_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->loop.joinable()) s->loop.join();
  ams_status st = AMS_OK;
  for (Worker& wk : s->workers) {
    if (wk.stream && cudaStreamSynchronize(wk.stream) != cudaSuccess) st = AMS_ERR_CUDA;
    if (wk.ctx) ams_context_destroy(wk.ctx);
    if (wk.stage) cudaFree(wk.stage);
    if (wk.d_off) cudaFree(wk.d_off);
    if (wk.h_off) cudaFreeHost(wk.h_off);
    if (wk.done) cudaEventDestroy(wk.done);
    if (wk.stream) cudaStreamDestroy(wk.stream);
  }
  delete s;
  return st;
}

}  // extern "C"
