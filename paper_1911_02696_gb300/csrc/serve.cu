// Serving runtime: continuous batching of pospopcnt jobs on one GPU.
//
// Jobs (width, device pointer, word count) arrive from clients at any time.
// A worker thread owns the GPU side:
//   1. completion: polls the event of every batch in flight; when one has
//      finished, copies each job's counts (already on the host, pinned) to
//      its sink, stamps the completion time and releases the job's bytes
//      from the HBM budget;
//   2. admission: moves arrived jobs, oldest first, from the waiting queue
//      to the pending queue of their width while the payload bytes admitted
//      and not yet completed stay within the budget (AdmissionPolicy);
//   3. launch: while a slot (stream + pinned descriptor and result buffers +
//      device buffers) is free, takes up to max_batch_jobs pending jobs of
//      the width whose oldest job arrived first and launches them as one
//      segmented count (descriptor form of the batched kernel), followed by
//      the copy of their counts to the host and an event.
// Several batches run on the GPU at once, and jobs that arrive while others
// are on the GPU join the next batch as soon as a slot and budget free up:
// batching is continuous, not a queue drained one batch at a time.
// In per-request mode every job is its own plain count launch (the
// comparison the batched form is measured against).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"
#include "pospopcnt.h"

namespace ppc {

double now_seconds() {
  using clock = std::chrono::steady_clock;
  return std::chrono::duration<double>(clock::now().time_since_epoch()).count();
}

// Bytes of payload admitted and not yet completed, against a budget.  A job
// is admitted when it fits; jobs larger than the whole budget are rejected
// at submission.
struct AdmissionPolicy {
  uint64_t budget = 0;
  uint64_t in_flight = 0;
  bool fits(uint64_t bytes) const { return in_flight + bytes <= budget; }
  void admit(uint64_t bytes) { in_flight += bytes; }
  void release(uint64_t bytes) { in_flight -= bytes; }
};

namespace {

struct Job {
  uint64_t tag = 0;
  int width = 16;
  uint64_t addr = 0;
  uint64_t n = 0;
  uint64_t bytes = 0;
  double t_arrival = 0, t_admit = 0, t_launch = 0, t_done = 0;
  bool deferred = false;  // counted once in the deferral statistic
};

int widx(int w) { return w == 8 ? 0 : w == 16 ? 1 : 2; }

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  uint64_t* h_desc = nullptr;               // pinned: bounds[m+1] then addr[m]
  unsigned long long* h_results = nullptr;  // pinned: m x width
  uint64_t* d_desc = nullptr;
  unsigned long long* d_results = nullptr;
  void* d_queue = nullptr;
  std::vector<Job> jobs;
  int width = 16;
  bool busy = false;
};

}  // namespace

struct Server {
  int device = 0;
  pospopcnt_server_config cfg{};
  DeviceState* st = nullptr;
  std::vector<Slot> slots;
  void* d_pool = nullptr;  // one allocation for every slot's device buffers

  std::mutex in_mu;
  std::deque<Job> incoming;
  std::deque<Job> waiting;
  std::deque<Job> pending[3];
  AdmissionPolicy adm;
  uint64_t admitted_jobs = 0;

  std::thread worker;
  std::atomic<bool> stop{false};
  std::atomic<int> worker_error{0};

  // sinks: the poll queue, or the arrays of a trace being replayed
  std::mutex done_mu;
  std::deque<pospopcnt_result> done;
  std::atomic<double*> trace_latency{nullptr};
  std::atomic<uint64_t*> trace_counts{nullptr};
  std::atomic<int*> trace_status{nullptr};
  std::atomic<uint64_t> total_submitted{0};
  std::atomic<uint64_t> total_completed{0};

  // stats (worker thread writes; readers take stats_mu)
  std::mutex stats_mu;
  pospopcnt_server_stats stats{};

  ~Server() = default;

  void emit(const Job& j, const unsigned long long* counts, int status) {
    double* lat = trace_latency.load(std::memory_order_acquire);
    if (lat) {
      lat[j.tag] = j.t_done - j.t_arrival;
      int* st_out = trace_status.load(std::memory_order_relaxed);
      uint64_t* cnt = trace_counts.load(std::memory_order_relaxed);
      if (st_out) st_out[j.tag] = status;
      if (cnt) {
        uint64_t* dst = cnt + j.tag * 32;
        std::memset(dst, 0, 32 * sizeof(uint64_t));
        if (status == POSPOPCNT_OK) std::memcpy(dst, counts, sizeof(uint64_t) * size_t(j.width));
      }
    } else {
      pospopcnt_result r{};
      r.tag = j.tag, r.status = status, r.width = j.width, r.n = j.n;
      r.t_arrival = j.t_arrival, r.t_admit = j.t_admit, r.t_launch = j.t_launch, r.t_done = j.t_done;
      if (status == POSPOPCNT_OK) std::memcpy(r.counts, counts, sizeof(uint64_t) * size_t(j.width));
      std::lock_guard<std::mutex> lk(done_mu);
      done.push_back(r);
    }
    total_completed.fetch_add(1, std::memory_order_release);
  }

  bool poll_completions() {
    bool any = false;
    for (Slot& s : slots) {
      if (!s.busy) continue;
      const cudaError_t q = cudaEventQuery(s.done);
      if (q == cudaErrorNotReady) continue;
      const double t = now_seconds();
      const int status = q == cudaSuccess ? POSPOPCNT_OK : cuda_fail(q);
      uint64_t bytes = 0;
      for (size_t i = 0; i < s.jobs.size(); ++i) {
        Job& j = s.jobs[i];
        j.t_done = t;
        adm.release(j.bytes);
        bytes += j.bytes;
        emit(j, s.h_results + i * size_t(s.width), status);
      }
      admitted_jobs -= s.jobs.size();
      {
        std::lock_guard<std::mutex> lk(stats_mu);
        stats.completed += s.jobs.size();
        stats.bytes_completed += bytes;
      }
      s.jobs.clear();
      s.busy = false;
      any = true;
    }
    return any;
  }

  bool admit() {
    {
      std::lock_guard<std::mutex> lk(in_mu);
      while (!incoming.empty()) {
        waiting.push_back(incoming.front());
        incoming.pop_front();
      }
    }
    bool any = false;
    const uint64_t max_admitted = uint64_t(slots.size()) * uint64_t(cfg.max_batch_jobs) * 2;
    while (!waiting.empty()) {
      Job& j = waiting.front();
      if (!adm.fits(j.bytes) || admitted_jobs >= max_admitted) {
        if (!j.deferred) {
          j.deferred = true;
          std::lock_guard<std::mutex> lk(stats_mu);
          ++stats.deferrals;
        }
        break;
      }
      adm.admit(j.bytes);
      ++admitted_jobs;
      j.t_admit = now_seconds();
      pending[widx(j.width)].push_back(j);
      waiting.pop_front();
      any = true;
    }
    if (any) {
      std::lock_guard<std::mutex> lk(stats_mu);
      stats.max_bytes_in_flight = std::max(stats.max_bytes_in_flight, adm.in_flight);
    }
    return any;
  }

  // width index whose oldest pending job arrived first, or -1
  int oldest_width() const {
    int best = -1;
    for (int w = 0; w < 3; ++w)
      if (!pending[w].empty() && (best < 0 || pending[w].front().t_arrival < pending[best].front().t_arrival))
        best = w;
    return best;
  }

  int launch(Slot& s, int wi) {
    static const int widths[3] = {8, 16, 32};
    const int width = widths[wi];
    const size_t take = std::min<size_t>(pending[wi].size(), size_t(cfg.max_batch_jobs));
    s.width = width;
    s.jobs.assign(pending[wi].begin(), pending[wi].begin() + long(take));
    pending[wi].erase(pending[wi].begin(), pending[wi].begin() + long(take));
    const double t = now_seconds();
    for (Job& j : s.jobs) j.t_launch = t;
    const size_t m = s.jobs.size();
    cudaError_t e;
    int rc = POSPOPCNT_OK;
    if (cfg.per_request) {
      const Job& j = s.jobs[0];
      rc = pospopcnt_count(width, POSPOPCNT_KERNEL_AUTO, reinterpret_cast<const void*>(j.addr), size_t(j.n),
                           reinterpret_cast<uint64_t*>(s.d_results), s.stream);
    } else {
      int64_t* hb = reinterpret_cast<int64_t*>(s.h_desc);
      uint64_t* ha = s.h_desc + (m + 1);
      hb[0] = 0;
      for (size_t i = 0; i < m; ++i) {
        hb[i + 1] = hb[i] + int64_t(s.jobs[i].n);
        ha[i] = s.jobs[i].addr;
      }
      const size_t desc_bytes = (2 * m + 1) * sizeof(uint64_t);
      if ((e = cudaMemcpyAsync(s.d_desc, s.h_desc, desc_bytes, cudaMemcpyHostToDevice, s.stream)) != cudaSuccess)
        rc = cuda_fail(e);
      else if ((e = cudaMemsetAsync(s.d_results, 0, m * size_t(width) * 8, s.stream)) != cudaSuccess)
        rc = cuda_fail(e);
      else
        rc = launch_batched(*st, nullptr, reinterpret_cast<const int64_t*>(s.d_desc), m, width, s.d_results,
                            s.d_queue, (128 * 1024) / (width / 8), s.stream, s.d_desc + (m + 1));
    }
    if (rc == POSPOPCNT_OK &&
        (e = cudaMemcpyAsync(s.h_results, s.d_results, m * size_t(width) * 8, cudaMemcpyDeviceToHost,
                             s.stream)) != cudaSuccess)
      rc = cuda_fail(e);
    if (rc == POSPOPCNT_OK && (e = cudaEventRecord(s.done, s.stream)) != cudaSuccess) rc = cuda_fail(e);
    if (rc != POSPOPCNT_OK) {  // fail the jobs on the host; nothing is in flight for them
      const double td = now_seconds();
      for (Job& j : s.jobs) {
        j.t_done = td;
        adm.release(j.bytes);
        emit(j, nullptr, rc);
      }
      admitted_jobs -= m;
      s.jobs.clear();
      return rc;
    }
    s.busy = true;
    std::lock_guard<std::mutex> lk(stats_mu);
    ++stats.batches;
    stats.jobs_in_batches += m;
    stats.max_batch = std::max<uint64_t>(stats.max_batch, m);
    return POSPOPCNT_OK;
  }

  bool launch_ready() {
    bool any = false;
    for (Slot& s : slots) {
      if (s.busy) continue;
      const int wi = oldest_width();
      if (wi < 0) break;
      launch(s, wi);
      any = true;
    }
    return any;
  }

  bool idle() {
    for (const Slot& s : slots)
      if (s.busy) return false;
    if (!waiting.empty() || !pending[0].empty() || !pending[1].empty() || !pending[2].empty()) return false;
    std::lock_guard<std::mutex> lk(in_mu);
    return incoming.empty();
  }

  void loop() {
    cudaSetDevice(device);
    for (;;) {
      bool progressed = poll_completions();
      progressed |= admit();
      progressed |= launch_ready();
      if (stop.load(std::memory_order_acquire) && idle()) break;
      if (!progressed) std::this_thread::yield();
    }
  }
};

}  // namespace ppc

using ppc::Server;

struct pospopcnt_server {
  Server impl;
};

extern "C" {

int pospopcnt_server_create(int device, const pospopcnt_server_config* cfg_in, pospopcnt_server** out) {
  if (!out) return POSPOPCNT_ERR_INVALID;
  *out = nullptr;
  pospopcnt_server_config cfg{};
  if (cfg_in) cfg = *cfg_in;
  if (cfg.hbm_budget_bytes == 0) cfg.hbm_budget_bytes = uint64_t(64) << 30;
  if (cfg.max_inflight == 0) cfg.max_inflight = cfg.per_request ? 64 : 4;
  if (cfg.max_batch_jobs == 0) cfg.max_batch_jobs = 4096;
  if (cfg.per_request) cfg.max_batch_jobs = 1;
  if (cfg.max_inflight < 1 || cfg.max_inflight > 256 || cfg.max_batch_jobs < 1 || cfg.max_batch_jobs > 65536)
    return POSPOPCNT_ERR_INVALID;
  int rc = pospopcnt_init(device);
  if (rc != POSPOPCNT_OK) return rc;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return ppc::cuda_fail(e);
  ppc::DeviceState* st = ppc::current_state(&rc);
  if (!st) {
    cudaSetDevice(prev);
    return rc;
  }
  auto* srv = new pospopcnt_server();
  Server& s = srv->impl;
  s.device = device;
  s.cfg = cfg;
  s.st = st;
  s.adm.budget = cfg.hbm_budget_bytes;
  const size_t B = size_t(cfg.max_batch_jobs);
  const size_t desc_bytes = (2 * B + 1) * sizeof(uint64_t);
  const size_t res_bytes = B * 32 * sizeof(uint64_t);
  const size_t per_slot = ((desc_bytes + 255) / 256 + (res_bytes + 255) / 256 + 1) * 256;
  s.slots.resize(size_t(cfg.max_inflight));
  if ((e = cudaMalloc(&s.d_pool, per_slot * s.slots.size())) != cudaSuccess) rc = ppc::cuda_fail(e);
  if (rc == POSPOPCNT_OK && (e = cudaMemset(s.d_pool, 0, per_slot * s.slots.size())) != cudaSuccess)
    rc = ppc::cuda_fail(e);
  for (size_t i = 0; rc == POSPOPCNT_OK && i < s.slots.size(); ++i) {
    ppc::Slot& sl = s.slots[i];
    char* base = static_cast<char*>(s.d_pool) + i * per_slot;
    sl.d_desc = reinterpret_cast<uint64_t*>(base);
    sl.d_results = reinterpret_cast<unsigned long long*>(base + (desc_bytes + 255) / 256 * 256);
    sl.d_queue = base + per_slot - 256;
    if ((e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaHostAlloc(reinterpret_cast<void**>(&sl.h_desc), desc_bytes, cudaHostAllocDefault)) != cudaSuccess ||
        (e = cudaHostAlloc(reinterpret_cast<void**>(&sl.h_results), res_bytes, cudaHostAllocDefault)) != cudaSuccess)
      rc = ppc::cuda_fail(e);
  }
  cudaSetDevice(prev);
  if (rc != POSPOPCNT_OK) {
    pospopcnt_server_destroy(srv);
    return rc;
  }
  s.worker = std::thread([&s] { s.loop(); });
  *out = srv;
  return POSPOPCNT_OK;
}

int pospopcnt_server_destroy(pospopcnt_server* srv) {
  if (!srv) return POSPOPCNT_ERR_INVALID;
  Server& s = srv->impl;
  s.stop.store(true, std::memory_order_release);
  if (s.worker.joinable()) s.worker.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s.device);
  for (ppc::Slot& sl : s.slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream), cudaStreamDestroy(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.h_desc) cudaFreeHost(sl.h_desc);
    if (sl.h_results) cudaFreeHost(sl.h_results);
  }
  if (s.d_pool) cudaFree(s.d_pool);
  cudaSetDevice(prev);
  delete srv;
  return POSPOPCNT_OK;
}

static int submit_job(Server& s, int width, const void* d_in, size_t n, uint64_t tag, double t_arrival) {
  if (width != 8 && width != 16 && width != 32) return POSPOPCNT_ERR_INVALID;
  if (n > 0 && !d_in) return POSPOPCNT_ERR_INVALID;
  if (reinterpret_cast<uintptr_t>(d_in) % uintptr_t(width / 8) != 0) return POSPOPCNT_ERR_MISALIGNED;
  const uint64_t bytes = uint64_t(n) * uint64_t(width / 8);
  if (bytes > s.cfg.hbm_budget_bytes) {
    std::lock_guard<std::mutex> lk(s.stats_mu);
    ++s.stats.rejected;
    return POSPOPCNT_ERR_TOO_LARGE;
  }
  ppc::Job j;
  j.tag = tag, j.width = width, j.addr = reinterpret_cast<uint64_t>(d_in), j.n = n, j.bytes = bytes;
  j.t_arrival = t_arrival;
  s.total_submitted.fetch_add(1, std::memory_order_acq_rel);
  {
    std::lock_guard<std::mutex> lk(s.in_mu);
    s.incoming.push_back(j);
  }
  std::lock_guard<std::mutex> lk(s.stats_mu);
  ++s.stats.submitted;
  return POSPOPCNT_OK;
}

int pospopcnt_server_submit(pospopcnt_server* srv, int width, const void* d_in, size_t n, uint64_t tag) {
  if (!srv) return POSPOPCNT_ERR_INVALID;
  if (srv->impl.trace_latency.load()) return POSPOPCNT_ERR_INVALID;  // a trace is being replayed
  return submit_job(srv->impl, width, d_in, n, tag, ppc::now_seconds());
}

int pospopcnt_server_poll(pospopcnt_server* srv, pospopcnt_result* out, int max, int* n_out) {
  if (!srv || !n_out || (max > 0 && !out)) return POSPOPCNT_ERR_INVALID;
  Server& s = srv->impl;
  std::lock_guard<std::mutex> lk(s.done_mu);
  int k = 0;
  while (k < max && !s.done.empty()) {
    out[k++] = s.done.front();
    s.done.pop_front();
  }
  *n_out = k;
  if (s.worker_error.load()) return s.worker_error.load();
  return POSPOPCNT_OK;
}

int pospopcnt_server_run_trace(pospopcnt_server* srv, size_t n, const double* t_arrival, const int* width,
                               const uint64_t* d_addr, const uint64_t* nwords, double* latency_out,
                               uint64_t* counts_out, int* status_out) {
  if (!srv || (n > 0 && (!t_arrival || !width || !d_addr || !nwords || !latency_out)))
    return POSPOPCNT_ERR_INVALID;
  Server& s = srv->impl;
  if (s.trace_latency.load()) return POSPOPCNT_ERR_INVALID;
  // jobs submitted earlier must finish first: their results go to the poll queue
  const double drain_deadline = ppc::now_seconds() + 600.0;
  while (s.total_completed.load(std::memory_order_acquire) < s.total_submitted.load(std::memory_order_acquire)) {
    if (ppc::now_seconds() > drain_deadline) return POSPOPCNT_ERR_TIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
  for (size_t i = 0; i < n; ++i) {
    latency_out[i] = std::nan("");
    if (status_out) status_out[i] = POSPOPCNT_ERR_INVALID;
  }
  s.trace_counts.store(counts_out);
  s.trace_status.store(status_out);
  s.trace_latency.store(latency_out, std::memory_order_release);
  const uint64_t base = s.total_completed.load(std::memory_order_acquire);
  uint64_t expected = 0;
  const double t0 = ppc::now_seconds() + 0.005;
  size_t i = 0;
  while (i < n) {
    const double now = ppc::now_seconds();
    const double due = t0 + t_arrival[i];
    if (now < due) {
      if (due - now > 200e-6) std::this_thread::sleep_for(std::chrono::microseconds(50));
      continue;
    }
    // submit every request that is due, stamped with its scheduled arrival
    for (; i < n && t0 + t_arrival[i] <= now; ++i) {
      const int rc = submit_job(s, width[i], reinterpret_cast<const void*>(d_addr[i]), size_t(nwords[i]),
                                uint64_t(i), t0 + t_arrival[i]);
      if (rc == POSPOPCNT_OK)
        ++expected;
      else if (status_out)
        status_out[i] = rc;
    }
  }
  const double deadline = ppc::now_seconds() + 600.0;
  int rc = POSPOPCNT_OK;
  while (s.total_completed.load(std::memory_order_acquire) - base < expected) {
    if (ppc::now_seconds() > deadline) {
      rc = POSPOPCNT_ERR_TIMEOUT;
      break;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
  if (rc != POSPOPCNT_OK) {  // keep the sinks: late completions still land in the caller's arrays
    return rc;
  }
  s.trace_latency.store(nullptr, std::memory_order_release);
  s.trace_counts.store(nullptr);
  s.trace_status.store(nullptr);
  return POSPOPCNT_OK;
}

int pospopcnt_server_get_stats(pospopcnt_server* srv, pospopcnt_server_stats* out) {
  if (!srv || !out) return POSPOPCNT_ERR_INVALID;
  std::lock_guard<std::mutex> lk(srv->impl.stats_mu);
  *out = srv->impl.stats;
  return POSPOPCNT_OK;
}

int pospopcnt_admission_simulate(uint64_t budget, size_t n, const double* t_arrival, const uint64_t* bytes,
                                 const double* service_s, double* t_admit_out, int* status_out) {
  if (n > 0 && (!t_arrival || !bytes || !service_s || !t_admit_out || !status_out)) return POSPOPCNT_ERR_INVALID;
  ppc::AdmissionPolicy adm;
  adm.budget = budget;
  struct Running {
    double t_end;
    uint64_t bytes;
  };
  std::vector<Running> running;
  std::deque<size_t> queue;
  size_t next = 0;
  double clock = 0.0;
  for (size_t i = 0; i < n; ++i) {
    t_admit_out[i] = std::nan("");
    status_out[i] = POSPOPCNT_OK;
    if (i && t_arrival[i] < t_arrival[i - 1]) return POSPOPCNT_ERR_INVALID;
  }
  // discrete-event loop over arrivals and completions (mock clock)
  while (next < n || !queue.empty()) {
    double t_next_arrival = next < n ? t_arrival[next] : INFINITY;
    double t_next_done = INFINITY;
    for (const Running& r : running) t_next_done = std::min(t_next_done, r.t_end);
    if (t_next_done <= t_next_arrival) {
      clock = t_next_done;
      for (size_t k = 0; k < running.size();)
        if (running[k].t_end <= clock) {
          adm.release(running[k].bytes);
          running[k] = running.back();
          running.pop_back();
        } else {
          ++k;
        }
    } else {
      clock = t_next_arrival;
      if (bytes[next] > budget)
        status_out[next] = POSPOPCNT_ERR_TOO_LARGE;
      else
        queue.push_back(next);
      ++next;
    }
    while (!queue.empty() && adm.fits(bytes[queue.front()])) {  // FIFO admission
      const size_t j = queue.front();
      queue.pop_front();
      adm.admit(bytes[j]);
      t_admit_out[j] = clock;
      running.push_back({clock + service_s[j], bytes[j]});
    }
    if (queue.empty() && next >= n) break;
  }
  return POSPOPCNT_OK;
}

}  // extern "C"
