// Serving runtime: continuous batching of pospopcnt jobs on one GPU.
//
// Jobs (width, device pointer, word count) arrive from clients at any time.
// A worker thread owns the GPU side:
//   1. completion: reads, for every job in flight, a flag in pinned host
//      memory that the GPU sets when that job's counts are final (a job
//      finishes on its own, not with its batch); a finished job's counts are
//      already on the host; its bytes are released from the HBM budget;
//   2. admission: moves arrived jobs, oldest first, from the waiting queue
//      to the pending queue of their width while the payload bytes admitted
//      and not yet completed stay within the budget (AdmissionPolicy);
//   3. launch: while a slot (stream + device rows + pinned result area) is
//      free, takes up to max_batch_jobs (<= 240) pending jobs of the width
//      whose oldest job arrived first and launches them as one segmented
//      count.  The job table travels in the kernel's parameters; the grid
//      has one CTA per tile of the batch.
// Several batches run on the GPU at once, and jobs that arrive while others
// are on the GPU join the next batch as soon as a slot and budget free up:
// batching is continuous, not a queue drained one batch at a time.
//
// Device side (serve_kernel): one CTA per 32 KiB tile of the batch's
// virtual word space (short-lived CTAs, so batches on other streams share
// the SMs at fine grain); each warp counts the pieces of its 4 KiB sub-range
// in one trip (segment helpers shared with the batched kernel) and adds them
// into the job's row in device memory.  Every warp then bumps the job's
// piece counter; the warp that completes it (the number of sub-ranges a job
// overlaps is known from its bounds) reads and re-zeroes the row, writes the
// counts to the job's pinned host slot, fences at system scope and stores
// the batch ticket into the job's flag.  Rows and counters are left zero for
// the slot's next batch, so no memset or device-to-host copy is issued.
//
// Jobs of at least large_job_bytes (default 4 MiB) gain nothing from
// batching -- their transfer time dwarfs a launch -- and would make every
// warp of a batch add into one row; each is launched on its own slot with
// the tuned plain count (block-level reduction; the bulk-copy ring from 64
// MiB) adding into a row kept at zero, followed by a one-warp kernel that
// publishes the counts and the flag the same way.  In per-request mode every job takes that route (the
// comparison the batched form is measured against).  Launches carry the job
// table sized to their batch (8 or 240 entries); no event is recorded --
// the watchdog asks the slot's stream whether it ran dry.
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
#include "segment_common.cuh"

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

constexpr int SERVE_MAX_JOBS = 240;  // job table in the kernel parameters (< 4 KiB)
// One CTA: 8 warps x 4 KiB, and a warp's 4 KiB is one trip of its piece
// counter (32 lanes x 8 vectors): every load of the piece is issued at once,
// so a cold payload costs one DRAM round trip per warp, not one per trip.
constexpr int SERVE_VPL = 8;
constexpr uint64_t SERVE_TILE_BYTES = uint64_t(BT_WARPS) * 32 * SERVE_VPL * 16;  // 32 KiB

// Job table in the kernel parameters, CAP jobs at most: a launch carries
// only the table size its batch needs (parameters are copied at every launch).
constexpr int SERVE_SMALL_CAP = 8;

template <int CAP>
struct ServeArgs {
  int64_t bounds[CAP + 1];  // virtual word offsets: job s is [bounds[s], bounds[s+1])
  uint64_t addr[CAP];       // byte address of each job's first word
  uint32_t nseg;
  uint32_t ticket;                     // stored into a job's flag when its counts are final
  uint64_t tile_words;                 // multiple of 8 warps x 16 bytes
  unsigned long long* rows;            // device, SERVE_MAX_JOBS x 32, zero on entry and exit
  unsigned* pieces;                    // device, SERVE_MAX_JOBS, zero on entry and exit
  unsigned long long* h_counts;        // device view of pinned host memory, SERVE_MAX_JOBS x 32
  unsigned* h_flags;                   // device view of pinned host memory, SERVE_MAX_JOBS
};

// Short-lived CTAs: three per SM is enough residency, and leaves each
// thread the registers of a whole one-trip piece (32 data registers).
template <int K, int CAP>
__global__ void __launch_bounds__(BT_THREADS, 3) serve_kernel(const __grid_constant__ ServeArgs<CAP> a) {
  constexpr int WB = K / 8;
  constexpr int SH = 5 - ilog2<K>::value;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t oN = a.bounds[a.nseg];  // bounds[0] == 0
  const uint64_t T = a.tile_words, Tw = a.tile_words / BT_WARPS;
  // one CTA per tile (no persistent loop): CTAs live a few microseconds, so
  // the kernels of other batches get SM slots without waiting for this one
  {
    const uint64_t tile = blockIdx.x;
    int64_t w0 = int64_t(tile * T + warp * Tw);
    int64_t w1 = w0 + int64_t(Tw);
    if (w1 > oN) w1 = oN;
    if (w0 >= w1) return;
    uint64_t s = find_segment(a.bounds, a.nseg, w0);
    int64_t seg_lo = a.bounds[s];
    for (;;) {
      const int64_t seg_hi = a.bounds[s + 1];
      const int64_t pa = seg_lo > w0 ? seg_lo : w0;
      const int64_t pb = seg_hi < w1 ? seg_hi : w1;
      if (pa < pb) {
        const uint8_t* pbase = reinterpret_cast<const uint8_t*>(a.addr[s] - uint64_t(seg_lo) * WB);
        const uint32_t v = warp_piece_counts<K, SERVE_VPL>(pbase, uint64_t(pa), uint64_t(pb));
        unsigned long long* row = a.rows + s * 32;
        if ((lane & ((1 << SH) - 1)) == 0 && v) atomicAdd(row + (lane >> SH), (unsigned long long)v);
        // the warp that adds the job's last piece publishes its counts
        const unsigned expected = unsigned((uint64_t(seg_hi) - 1) / Tw - uint64_t(seg_lo) / Tw + 1);
        __syncwarp();
        unsigned last = 0;
        if (lane == 0) {
          __threadfence();
          last = atomicAdd(a.pieces + s, 1u) + 1u == expected ? 1u : 0u;
        }
        last = __shfl_sync(FULL_MASK, last, 0);
        if (last) {
          __threadfence();
          // lane p moves count p to the host in one coalesced store; every
          // storing lane fences its own store before the warp syncs and
          // lane 0 raises the flag
          if (lane < K) a.h_counts[s * 32 + lane] = atomicExch(row + lane, 0ull);
          if (lane == 0) a.pieces[s] = 0;
          __threadfence_system();
          __syncwarp();
          if (lane == 0) *reinterpret_cast<volatile unsigned*>(a.h_flags + s) = a.ticket;
        }
      }
      if (seg_hi >= w1 || s + 1 >= a.nseg) break;
      ++s;
      seg_lo = seg_hi;
    }
  }
}

// A job counted by a plain launch: its counts were accumulated into d_row
// (kept zero between jobs); one warp moves them to the host, re-zeroes the
// row and raises the job's flag, as the serving kernel does for its jobs.
template <int K>
__global__ void serve_publish_kernel(unsigned long long* d_row, unsigned long long* h_counts, unsigned* h_flag,
                                     unsigned ticket) {
  const int lane = threadIdx.x & 31;
  if (lane < K) {
    h_counts[lane] = d_row[lane];
    d_row[lane] = 0;
  }
  __threadfence_system();
  __syncwarp();
  if (lane == 0) *reinterpret_cast<volatile unsigned*>(h_flag) = ticket;
}

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
  unsigned long long* d_rows = nullptr;     // device SERVE_MAX_JOBS x 32, zero between batches
  unsigned* d_pieces = nullptr;             // device SERVE_MAX_JOBS
  unsigned long long* d_single = nullptr;   // device, 32: a single job's counts, zero between jobs
  unsigned long long* h_counts = nullptr;   // pinned, mapped: SERVE_MAX_JOBS x 32
  unsigned* h_flags = nullptr;              // pinned, mapped: SERVE_MAX_JOBS
  unsigned long long* dv_counts = nullptr;  // device views of h_counts / h_flags
  unsigned* dv_flags = nullptr;
  uint32_t ticket = 0;
  std::vector<Job> jobs;
  std::vector<char> finished;
  size_t remaining = 0;
  double t_launch = 0;
  int width = 16;
  bool busy = false;
  bool single = false;  // one job counted by a plain launch, published by serve_publish_kernel
};

}  // namespace

struct Server {
  int device = 0;
  pospopcnt_server_config cfg{};
  DeviceState* st = nullptr;
  std::vector<Slot> slots;
  void* d_pool = nullptr;  // one allocation for every slot's device buffers
  size_t d_pool_bytes = 0;
  void* h_pool = nullptr;  // one pinned, mapped allocation for every slot's host results

  std::mutex in_mu;
  std::deque<Job> incoming;
  std::deque<Job> waiting;
  std::deque<Job> pending[3];   // small jobs, per width: batched
  std::deque<Job> pending_large;  // jobs of >= large_job_bytes: one plain launch each
  uint64_t large_job_bytes = 0;
  int large_limit = 0;           // large jobs on the GPU at once (0: no limit)
  int large_in_flight = 0;
  AdmissionPolicy adm;
  uint64_t admitted_jobs = 0;

  std::thread worker;
  std::atomic<bool> stop{false};
  std::atomic<int> worker_error{0};

  // sinks: the poll queue, or the arrays of a trace being replayed
  std::mutex done_mu;
  std::deque<pospopcnt_result> done;
  std::atomic<double*> trace_latency{nullptr};
  std::atomic<double*> trace_stages{nullptr};  // n x 3: admit, launch, done - arrival
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
      if (double* stg = trace_stages.load(std::memory_order_relaxed)) {
        stg[3 * j.tag + 0] = j.t_admit - j.t_arrival;
        stg[3 * j.tag + 1] = j.t_launch - j.t_arrival;
        stg[3 * j.tag + 2] = j.t_done - j.t_arrival;
      }
      int* st_out = trace_status.load(std::memory_order_relaxed);
      uint64_t* cnt = trace_counts.load(std::memory_order_relaxed);
      if (st_out) st_out[j.tag] = status;
      if (cnt) {
        uint64_t* dst = cnt + j.tag * 32;
        std::memset(dst, 0, 32 * sizeof(uint64_t));
        if (status == POSPOPCNT_OK && counts) std::memcpy(dst, counts, sizeof(uint64_t) * size_t(j.width));
      }
    } else {
      pospopcnt_result r{};
      r.tag = j.tag, r.status = status, r.width = j.width, r.n = j.n;
      r.t_arrival = j.t_arrival, r.t_admit = j.t_admit, r.t_launch = j.t_launch, r.t_done = j.t_done;
      if (status == POSPOPCNT_OK && counts) std::memcpy(r.counts, counts, sizeof(uint64_t) * size_t(j.width));
      std::lock_guard<std::mutex> lk(done_mu);
      done.push_back(r);
    }
    total_completed.fetch_add(1, std::memory_order_release);
  }

  void finish(Slot& s, size_t i, const unsigned long long* counts, int status, double t) {
    Job& j = s.jobs[i];
    j.t_done = t;
    adm.release(j.bytes);
    emit(j, counts, status);
    s.finished[i] = 1;
    --s.remaining;
    --admitted_jobs;
    std::lock_guard<std::mutex> lk(stats_mu);
    ++stats.completed;
    stats.bytes_completed += j.bytes;
  }

  bool poll_completions() {
    bool any = false;
    for (Slot& s : slots) {
      if (!s.busy) continue;
      // every job -- batched or counted alone -- is published through its flag
      for (size_t i = 0; i < s.jobs.size(); ++i) {
        if (s.finished[i]) continue;
        if (__atomic_load_n(s.h_flags + i, __ATOMIC_ACQUIRE) != s.ticket) continue;
        finish(s, i, s.h_counts + i * 32, POSPOPCNT_OK, now_seconds());
        any = true;
      }
      // watchdog: the slot's stream ran dry (or failed) without publishing every job
      if (s.remaining && now_seconds() - s.t_launch > 0.5) {
        const cudaError_t q = cudaStreamQuery(s.stream);
        if (q != cudaErrorNotReady) {
          const double t = now_seconds();
          for (size_t i = 0; i < s.jobs.size(); ++i) {
            if (s.finished[i]) continue;
            if (__atomic_load_n(s.h_flags + i, __ATOMIC_ACQUIRE) == s.ticket)
              finish(s, i, s.h_counts + i * 32, POSPOPCNT_OK, t);
            else
              finish(s, i, nullptr, q == cudaSuccess ? POSPOPCNT_ERR_CUDA : cuda_fail(q), t);
          }
          if (s.single) cudaMemsetAsync(s.d_single, 0, 32 * sizeof(unsigned long long), s.stream);
        }
      }
      if (s.remaining == 0) {
        if (s.single && !cfg.per_request) --large_in_flight;
        s.jobs.clear();
        s.busy = false;
        any = true;
      }
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
    const uint64_t max_admitted = uint64_t(slots.size()) * uint64_t(cfg.max_batch_jobs) * 4;
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
      if (cfg.per_request || j.bytes >= large_job_bytes)
        pending_large.push_back(j);
      else
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

  // the queue whose oldest job arrived first: 0..2 = small jobs of width
  // 8/16/32, 3 = large jobs; -1 if nothing is pending
  int oldest_queue() const {
    int best = -1;
    double t = 0;
    for (int w = 0; w < 3; ++w)
      if (!pending[w].empty() && (best < 0 || pending[w].front().t_arrival < t)) best = w, t = pending[w].front().t_arrival;
    const bool large_ok = large_limit <= 0 || large_in_flight < large_limit;
    if (large_ok && !pending_large.empty() && (best < 0 || pending_large.front().t_arrival < t)) best = 3;
    return best;
  }

  // One batch of m jobs: the job table sized to the batch, then the kernel.
  template <int K, int CAP>
  cudaError_t launch_serve(Slot& s, size_t m) {
    ServeArgs<CAP> args;
    args.bounds[0] = 0;
    for (size_t i = 0; i < m; ++i) {
      args.bounds[i + 1] = args.bounds[i] + int64_t(s.jobs[i].n);
      args.addr[i] = s.jobs[i].addr;
    }
    args.nseg = uint32_t(m);
    args.ticket = s.ticket;
    args.tile_words = uint64_t(SERVE_TILE_BYTES / (K / 8));
    args.rows = s.d_rows;
    args.pieces = s.d_pieces;
    args.h_counts = s.dv_counts;
    args.h_flags = s.dv_flags;
    const uint64_t total = uint64_t(args.bounds[m]);
    const uint64_t tiles = (total + args.tile_words - 1) / args.tile_words;
    serve_kernel<K, CAP><<<unsigned(std::max<uint64_t>(1, tiles)), BT_THREADS, 0, s.stream>>>(args);
    note_launch();
    return cudaGetLastError();
  }

  template <int K>
  cudaError_t launch_serve_k(Slot& s, size_t m) {
    return m <= size_t(SERVE_SMALL_CAP) ? launch_serve<K, SERVE_SMALL_CAP>(s, m) : launch_serve<K, SERVE_MAX_JOBS>(s, m);
  }

  int launch(Slot& s, int qi) {
    static const int widths[3] = {8, 16, 32};
    std::deque<Job>& src = qi == 3 ? pending_large : pending[qi];
    const size_t take = qi == 3 ? 1 : std::min<size_t>(src.size(), size_t(cfg.max_batch_jobs));
    s.single = qi == 3;
    if (s.single && !cfg.per_request) ++large_in_flight;
    const int width = s.single ? src.front().width : widths[qi];
    s.width = width;
    s.jobs.assign(src.begin(), src.begin() + long(take));
    src.erase(src.begin(), src.begin() + long(take));
    const size_t m = s.jobs.size();
    s.finished.assign(m, 0);
    s.remaining = m;
    s.t_launch = now_seconds();
    for (Job& j : s.jobs) j.t_launch = s.t_launch;
    s.busy = true;
    cudaError_t e = cudaSuccess;
    int rc = POSPOPCNT_OK;
    ++s.ticket;
    if (s.single) {
      // the tuned plain count adds into d_single (zero between jobs); one
      // warp then publishes it like a batched job: no memset, copy or event.
      // From 64 MiB the count takes the bulk-copy ring (the launch the
      // table gives inputs of 256 MiB and up): a served payload is a
      // read-only slice, so the L2 holds no dirty lines that would favour
      // register loads there, and on GB300 the ring cut p99 at 50k req/s
      // from 67.4 to 61.7 us (per-request launches: 70.7 to 65.3 us).
      const Job& j = s.jobs[0];
      const uint64_t bytes = j.n * uint64_t(width / 8);
      const uint64_t ring_from = uint64_t(64) << 20, ring_class = uint64_t(256) << 20;
      const size_t n_cfg = bytes >= ring_from && bytes < ring_class ? size_t(ring_class / uint64_t(width / 8))
                                                                    : size_t(j.n);
      pospopcnt_config pc{};
      rc = pospopcnt_get_config(width, n_cfg, &pc);
      if (rc == POSPOPCNT_OK) rc = ppc::normalize_config(*st, width, &pc);
      if (rc == POSPOPCNT_OK)
        rc = ppc::launch_plain(*st, width, pc, reinterpret_cast<const void*>(j.addr), size_t(j.n), s.d_single,
                               false, s.stream);
      if (rc == POSPOPCNT_OK) {
        auto pub = width == 8 ? serve_publish_kernel<8> : width == 16 ? serve_publish_kernel<16>
                                                                      : serve_publish_kernel<32>;
        pub<<<1, 32, 0, s.stream>>>(s.d_single, s.dv_counts, s.dv_flags, s.ticket);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) rc = cuda_fail(e);
      }
      if (rc != POSPOPCNT_OK) cudaMemsetAsync(s.d_single, 0, 32 * sizeof(unsigned long long), s.stream);
    } else {
      // empty jobs have no piece on the device: they complete here
      size_t live = 0;
      for (size_t i = 0; i < m; ++i) {
        live += s.jobs[i].n > 0;
        if (s.jobs[i].n == 0) {
          static const unsigned long long zeros[32] = {};
          finish(s, i, zeros, POSPOPCNT_OK, now_seconds());
        }
      }
      if (live) {
        e = width == 8 ? launch_serve_k<8>(s, m) : width == 16 ? launch_serve_k<16>(s, m) : launch_serve_k<32>(s, m);
        if (e != cudaSuccess) rc = cuda_fail(e);
      }
    }
    if (rc != POSPOPCNT_OK) {  // fail the unfinished jobs on the host
      const double td = now_seconds();
      for (size_t i = 0; i < m; ++i)
        if (!s.finished[i]) finish(s, i, nullptr, rc, td);
    }
    if (s.remaining == 0) {
      if (s.single && !cfg.per_request) --large_in_flight;
      s.jobs.clear();
      s.busy = false;
    }
    std::lock_guard<std::mutex> lk(stats_mu);
    ++stats.batches;
    stats.jobs_in_batches += m;
    stats.max_batch = std::max<uint64_t>(stats.max_batch, m);
    return rc;
  }

  bool launch_ready() {
    bool any = false;
    for (Slot& s : slots) {
      if (s.busy) continue;
      const int qi = oldest_queue();
      if (qi < 0) break;
      launch(s, qi);
      any = true;
    }
    return any;
  }

  bool idle() {
    for (const Slot& s : slots)
      if (s.busy) return false;
    if (!waiting.empty() || !pending[0].empty() || !pending[1].empty() || !pending[2].empty() ||
        !pending_large.empty())
      return false;
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
  if (cfg.max_inflight == 0) cfg.max_inflight = cfg.per_request ? 64 : 16;
  if (cfg.max_batch_jobs == 0) cfg.max_batch_jobs = ppc::SERVE_MAX_JOBS;
  if (cfg.per_request) cfg.max_batch_jobs = 1;
  if (cfg.max_inflight < 1 || cfg.max_inflight > 256 || cfg.max_batch_jobs < 1 ||
      cfg.max_batch_jobs > ppc::SERVE_MAX_JOBS)
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
  s.large_job_bytes = cfg.large_job_bytes ? cfg.large_job_bytes : (uint64_t(4) << 20);
  s.large_limit = cfg.max_large_inflight;
  const size_t rows_bytes = size_t(ppc::SERVE_MAX_JOBS) * 32 * sizeof(uint64_t);
  const size_t pieces_bytes = size_t(ppc::SERVE_MAX_JOBS) * sizeof(unsigned);
  const size_t pieces_pad = ((pieces_bytes + 255) / 256) * 256;
  const size_t per_slot = rows_bytes + pieces_pad + 256;  // + the single-job row
  const size_t host_per_slot = rows_bytes + pieces_pad;
  s.slots.resize(size_t(cfg.max_inflight));
  s.d_pool_bytes = per_slot * s.slots.size();
  if ((e = ppc::device_alloc(&s.d_pool, s.d_pool_bytes)) != cudaSuccess) rc = ppc::cuda_fail(e);
  if (rc == POSPOPCNT_OK && (e = cudaMemset(s.d_pool, 0, per_slot * s.slots.size())) != cudaSuccess)
    rc = ppc::cuda_fail(e);
  if (rc == POSPOPCNT_OK &&
      (e = cudaHostAlloc(&s.h_pool, host_per_slot * s.slots.size(), cudaHostAllocMapped)) != cudaSuccess)
    rc = ppc::cuda_fail(e);
  if (rc == POSPOPCNT_OK) std::memset(s.h_pool, 0, host_per_slot * s.slots.size());
  void* dv_pool = nullptr;
  if (rc == POSPOPCNT_OK && (e = cudaHostGetDevicePointer(&dv_pool, s.h_pool, 0)) != cudaSuccess)
    rc = ppc::cuda_fail(e);
  for (size_t i = 0; rc == POSPOPCNT_OK && i < s.slots.size(); ++i) {
    ppc::Slot& sl = s.slots[i];
    char* base = static_cast<char*>(s.d_pool) + i * per_slot;
    sl.d_rows = reinterpret_cast<unsigned long long*>(base);
    sl.d_pieces = reinterpret_cast<unsigned*>(base + rows_bytes);
    sl.d_single = reinterpret_cast<unsigned long long*>(base + rows_bytes + pieces_pad);
    char* hb = static_cast<char*>(s.h_pool) + i * host_per_slot;
    char* dvb = static_cast<char*>(dv_pool) + i * host_per_slot;
    sl.h_counts = reinterpret_cast<unsigned long long*>(hb);
    sl.h_flags = reinterpret_cast<unsigned*>(hb + rows_bytes);
    sl.dv_counts = reinterpret_cast<unsigned long long*>(dvb);
    sl.dv_flags = reinterpret_cast<unsigned*>(dvb + rows_bytes);
    if ((e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking)) != cudaSuccess) rc = ppc::cuda_fail(e);
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
  }
  ppc::device_free(s.d_pool, s.d_pool_bytes);
  if (s.h_pool) cudaFreeHost(s.h_pool);
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
  return pospopcnt_server_run_trace_timed(srv, n, t_arrival, width, d_addr, nwords, latency_out, counts_out,
                                          status_out, nullptr);
}

int pospopcnt_server_run_trace_timed(pospopcnt_server* srv, size_t n, const double* t_arrival, const int* width,
                                     const uint64_t* d_addr, const uint64_t* nwords, double* latency_out,
                                     uint64_t* counts_out, int* status_out, double* stages_out) {
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
  if (stages_out)
    for (size_t i = 0; i < 3 * n; ++i) stages_out[i] = std::nan("");
  s.trace_counts.store(counts_out);
  s.trace_status.store(status_out);
  s.trace_stages.store(stages_out);
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
  s.trace_stages.store(nullptr);
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
