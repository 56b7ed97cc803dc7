// Internal interfaces between the translation units of the library.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <mutex>

#include <cuda_runtime_api.h>

#include "pospopcnt.h"

namespace ppc {

// Per-device state owned by the library (created by pospopcnt_init).
struct DeviceState {
  bool ready = false;
  int device = -1;
  int sms = 0;
  int smem_optin = 0;
  unsigned* d_err = nullptr;      // device error word
  void* d_queue = nullptr;        // batched work-queue slots (QUEUE_SLOTS x 128 B)
  void* d_plain = nullptr;        // plain-count accumulators (PLAIN_SLOTS x PLAIN_SLOT_BYTES)
  // host-buffer path
  void* d_stage[2] = {nullptr, nullptr};
  unsigned long long* d_acc = nullptr;
  cudaStream_t hstream[2] = {nullptr, nullptr};
  cudaEvent_t hevent[2] = {nullptr, nullptr};
};

constexpr int QUEUE_SLOTS = 256;
constexpr int QUEUE_SLOT_BYTES = 128;
constexpr int PLAIN_SLOTS = 1024;
constexpr int PLAIN_SLOT_BYTES = 1024;  // 64 x uint64 accumulator at 0, arrival counter at 512
constexpr size_t HOST_STAGE_BYTES = size_t(64) << 20;

// Returns the state of the current device, initialising it if needed, or
// nullptr (with *status set) on failure.
DeviceState* current_state(int* status);

// Records a CUDA failure for pospopcnt_last_cuda_error and returns
// POSPOPCNT_ERR_CUDA.
int cuda_fail(cudaError_t e);

// Counts one kernel launch.
void note_launch();

// Resident blocks per SM of kernel `func` with `threads` threads and `smem`
// bytes of dynamic shared memory on `device` (the current device), at least
// 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor, asked once per kernel,
// device, block size and shared-memory size and then remembered, since the
// answer cannot change within a process.
int resident_blocks(const void* func, int device, int threads, size_t smem);

// cudaMalloc / cudaFree of device memory the library owns; the bytes held
// are counted for pospopcnt_device_bytes_allocated.
cudaError_t device_alloc(void** p, size_t bytes);
void device_free(void* p, size_t bytes);

// Device address of the allocation-free batched form's error word on
// `device`, or nullptr if that form has not run there (batched.cu).
unsigned* noalloc_error_word(int device);

// Head / body / tail split of n words of `width` bits at addr.
struct Split {
  size_t head_words, body_vectors, tail_words;
};
Split plan_split(int width, uint64_t addr, size_t n);

// A stream's accumulator for overwriting counts without a memset: 64
// uint64 values and an arrival counter, zero between launches on that
// stream (the last block of each launch leaves them so).
struct PlainAcc {
  unsigned long long* acc = nullptr;
  unsigned* arrived = nullptr;
};

// Launch of one single-stream count.  zero_first: the counts are
// overwritten (a direct store by a one-CTA grid; else, with `acc`, blocks
// add into the stream's accumulator and the last block writes the counts;
// else a memset + atomics); otherwise the kernel adds into d_counts.
int launch_plain(const DeviceState& st, int width, const pospopcnt_config& cfg, const void* d_in,
                 size_t n, unsigned long long* d_counts, bool zero_first, cudaStream_t stream,
                 const PlainAcc& acc = PlainAcc{});

// The accumulator bound to `stream` on the state's device (binding one of
// the device's stream slots on first use), or an empty one when the memset
// path must be taken: the stream is being captured into a CUDA graph (a
// graph may be replayed on any stream), it is the per-thread default stream
// (one handle, many streams), or no slot is free.
PlainAcc plain_acc_for(DeviceState& st, cudaStream_t stream);

// Count of n words in pinned host memory mapped into the device address
// space (d_in: its device address), adding into d_counts.
int launch_plain_sysmem(const DeviceState& st, int width, const void* d_in, size_t n,
                        unsigned long long* d_counts, cudaStream_t stream);

// Validates a configuration for a width; fills defaults for zero fields.
int normalize_config(const DeviceState& st, int width, pospopcnt_config* cfg);

// Launch of the batched kernel (counts zeroed by the caller).  tile_words:
// words per scheduling unit (a multiple of 128 bytes); blocks_per_sm: CTAs
// per SM of the persistent grid (0, or more than fit: as many as fit);
// ring_stages: per-warp ring depth 2, 3 or 4 (0: 2); vpl: vectors per lane
// per trip 4, 8 or 16 (0: 8; 16 takes at most 3 stages).
int launch_batched(const DeviceState& st, const void* d_in, const int64_t* d_offsets, size_t nseg,
                   int width, unsigned long long* d_counts, void* queue_slot, int tile_words,
                   int blocks_per_sm, int ring_stages, int vpl, cudaStream_t stream);

// Checks offsets on the device before a batched launch on the same slot:
// a violation makes that launch count nothing and sets the error word.
int launch_offsets_check(const DeviceState& st, const int64_t* d_offsets, size_t nseg, uint64_t n_words,
                         void* queue_slot, cudaStream_t stream);

// Raises kernel Kern's dynamic shared-memory limit to `bytes` on the
// current device once (one cache per kernel -- the template argument is the
// kernel itself, not its type, which instances of one template share -- and
// per device), so later launches, including launches captured into a CUDA
// graph, make no attribute call.
// Threads that race on the first launch take the mutex; the limit only
// grows.
template <auto Kern>
cudaError_t ensure_dynamic_smem(int device, int bytes) {
  static std::atomic<int> done[64];  // largest limit already set, per device (zero-initialised)
  static std::mutex mu;
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  if (done[device].load(std::memory_order_acquire) >= bytes) return cudaSuccess;
  std::lock_guard<std::mutex> lk(mu);
  if (done[device].load(std::memory_order_relaxed) >= bytes) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done[device].store(bytes, std::memory_order_release);
  return e;
}

// Monotonic host clock in seconds.
double now_seconds();

}  // namespace ppc
