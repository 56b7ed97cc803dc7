// The C ABI of include/pospopcnt.h: argument checks, per-device state,
// launch configuration tables, the host-buffer path and the autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "device_common.cuh"
#include "internal.h"
#include "pospopcnt.h"

namespace ppc {

namespace {

constexpr int MAX_DEVICES = 64;
constexpr int NCLASSES = 21;  // floor(log4(bytes)) for bytes < 2^42

std::mutex g_mutex;
DeviceState g_state[MAX_DEVICES];
// Work-queue slots of the batched form, per device: bound to a stream on its
// first batched call, returned by pospopcnt_release_stream (or when a graph
// that owns one is destroyed) and handed out again.
std::unordered_map<cudaStream_t, int> g_slots[MAX_DEVICES];
std::vector<int> g_free_slots[MAX_DEVICES];
int g_next_slot[MAX_DEVICES] = {};
// Plain-count accumulators, per device: bound to a stream on its first
// overwriting count, returned with the stream's work-queue slot.  A count
// on a stream that finds none free takes the memset path.
std::unordered_map<cudaStream_t, int> g_plain_slots[MAX_DEVICES];
std::vector<int> g_free_plain[MAX_DEVICES];
int g_next_plain[MAX_DEVICES] = {};
pospopcnt_config g_cfg[MAX_DEVICES][4][NCLASSES];
bool g_cfg_ready[MAX_DEVICES] = {};
// Batched form, per device and width (8, 16, 32): 32 KiB units, 2 CTAs per
// SM (what the autotuner picks on GB300 for the 20,000-segment log-uniform
// layout), until pospopcnt_batched_set_config/autotune.
pospopcnt_batched_config g_bcfg[MAX_DEVICES][3] = {};
bool g_bcfg_set[MAX_DEVICES][3] = {};
constexpr pospopcnt_batched_config BATCHED_DEFAULT = {32768, 2, 2, 8};
std::mutex g_host_mutex[MAX_DEVICES];
std::atomic<uint64_t> g_launches{0};
std::atomic<uint64_t> g_device_bytes{0};
thread_local int t_last_cuda = 0;

int width_index(int width) {
  return width == 8 ? 0 : width == 16 ? 1 : width == 32 ? 2 : width == 64 ? 3 : -1;
}

int size_class(uint64_t bytes) {
  int c = 0;
  while (c + 1 < NCLASSES && (uint64_t(1) << (2 * (c + 1))) <= bytes) ++c;
  return c;
}

pospopcnt_config default_config() {
  pospopcnt_config c;
  c.kernel = POSPOPCNT_KERNEL_CSA;
  c.threads = 256;
  c.unroll = 4;
  c.blocks_per_sm = 0;
  c.stages = 4;
  c.chunk_bytes = 32768;
  c.flags = 0;
  return c;
}

// Defaults per width and size class (floor(log4 bytes)), from the library's
// autotuner run on a GB300 (152 SMs, 2070 MHz): below 256 KiB one wide CTA
// (512 threads x 8 vectors covers 64 KiB in one trip, and a one-CTA grid
// stores its counts without a memset); up to 64 MiB the register-load CSA
// kernel; from 64 MiB (u16, u32) and 256 MiB (u8) the bulk-copy ring with
// ~192 KiB per SM in flight (u16 4 x 48 KiB, u32 3 x 64 KiB, u8 4 x 32 KiB).
// Every ring shape with that much in flight measured within 1.5 % of the
// others at 2 GiB: the kernel is at the DRAM limit there.
pospopcnt_config tuned_default(int width, int cls) {
  pospopcnt_config c = default_config();
  if (width == 64) {  // two circuits per thread; the bulk-copy ring from 64 MiB
    if (cls >= 13) {
      // 2 x 96 KiB: the autotuner's pick on GB300 at 256 MiB, 1 GiB and 2 GiB
      // (with the evict-first hint from 256 MiB up)
      c.kernel = POSPOPCNT_KERNEL_TMA, c.stages = 2, c.chunk_bytes = 98304;
      if (cls >= 14) c.flags = POSPOPCNT_FLAG_EVICT_FIRST;
      return c;
    }
    c.threads = 256, c.unroll = cls <= 11 ? 4 : 8;
    return c;
  }
  if (cls <= 8) {
    c.threads = 512, c.unroll = 8;
    return c;
  }
  if (cls <= 11) {
    c.threads = 128, c.unroll = 4;
    return c;
  }
  if (width == 8) {
    if (cls >= 14) {  // 256 MiB and up: the ring, 4 x 32 KiB (5 x 32 KiB from 1 GiB)
      c.kernel = POSPOPCNT_KERNEL_TMA, c.stages = cls >= 15 ? 5 : 4, c.chunk_bytes = 32768;
      return c;
    }
    c.threads = cls >= 13 ? 512 : 256;
    c.unroll = 4;
    return c;
  }
  if (cls == 12) {
    c.threads = 128, c.unroll = 8;
    return c;
  }
  if (cls == 13) {
    // 64..256 MiB: register loads.  Timed with L2 holding the input (warm),
    // unrelated clean lines, or unrelated dirty lines that must be written
    // back during the read, this kernel is as fast as the bulk-copy ring in
    // the first two states and 10-20 % faster in the third.
    c.threads = 512, c.unroll = 8;
    return c;
  }
  c.kernel = POSPOPCNT_KERNEL_TMA;
  if (width == 16) {
    c.stages = 4, c.chunk_bytes = 49152;  // 192 KiB in flight per SM
  } else {
    c.stages = 3, c.chunk_bytes = 65536;
  }
  // 256 MiB..1 GiB: the ring with an evict-first hint, which keeps its speed
  // with a clean L2 and halves most of its loss when the L2 is full of dirty
  // lines; from 1 GiB the hint measured no better.
  if (cls == 14) c.flags = POSPOPCNT_FLAG_EVICT_FIRST;
  return c;
}

void init_configs(int dev) {
  if (g_cfg_ready[dev]) return;
  const int widths[4] = {8, 16, 32, 64};
  for (int w = 0; w < 4; ++w)
    for (int c = 0; c < NCLASSES; ++c) g_cfg[dev][w][c] = tuned_default(widths[w], c);
  g_cfg_ready[dev] = true;
}

int init_locked(int device) {
  if (device < 0 || device >= MAX_DEVICES) return POSPOPCNT_ERR_INVALID;
  DeviceState& st = g_state[device];
  if (st.ready) return POSPOPCNT_OK;
  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e != cudaSuccess) return cuda_fail(e);
  if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e);
  int rc = POSPOPCNT_OK;
  do {
    if ((e = cudaDeviceGetAttribute(&st.sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) break;
    if ((e = cudaDeviceGetAttribute(&st.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device)) !=
        cudaSuccess)
      break;
    if ((e = device_alloc(reinterpret_cast<void**>(&st.d_err), 256)) != cudaSuccess) break;
    if ((e = cudaMemset(st.d_err, 0, 256)) != cudaSuccess) break;
    if ((e = device_alloc(&st.d_queue, size_t(QUEUE_SLOTS) * QUEUE_SLOT_BYTES)) != cudaSuccess) break;
    if ((e = cudaMemset(st.d_queue, 0, size_t(QUEUE_SLOTS) * QUEUE_SLOT_BYTES)) != cudaSuccess) break;
    if ((e = device_alloc(&st.d_plain, size_t(PLAIN_SLOTS) * PLAIN_SLOT_BYTES)) != cudaSuccess) break;
    if ((e = cudaMemset(st.d_plain, 0, size_t(PLAIN_SLOTS) * PLAIN_SLOT_BYTES)) != cudaSuccess) break;
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) break;
  } while (false);
  if (e != cudaSuccess) rc = cuda_fail(e);
  cudaSetDevice(prev);
  if (rc == POSPOPCNT_OK) {
    st.device = device;
    init_configs(device);
    st.ready = true;
  }
  return rc;
}

}  // namespace

int cuda_fail(cudaError_t e) {
  t_last_cuda = int(e);
  return POSPOPCNT_ERR_CUDA;
}

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {
struct OccupancyEntry {
  const void* func;
  int device, threads;
  size_t smem;
  int blocks;
};
constexpr int OCCUPANCY_ENTRIES = 512;  // kernels x devices x launch shapes the library can use
std::mutex g_occ_mu;
OccupancyEntry g_occ[OCCUPANCY_ENTRIES];
int g_occ_used = 0;
}  // namespace

int resident_blocks(const void* func, int device, int threads, size_t smem) {
  {
    std::lock_guard<std::mutex> lk(g_occ_mu);
    for (int i = 0; i < g_occ_used; ++i) {
      const OccupancyEntry& e = g_occ[i];
      if (e.func == func && e.device == device && e.threads == threads && e.smem == smem) return e.blocks;
    }
  }
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, func, threads, smem) != cudaSuccess || blocks < 1)
    return 1;  // not remembered: a failed query is asked again next time
  std::lock_guard<std::mutex> lk(g_occ_mu);
  if (g_occ_used < OCCUPANCY_ENTRIES) g_occ[g_occ_used++] = OccupancyEntry{func, device, threads, smem, blocks};
  return blocks;
}

cudaError_t device_alloc(void** p, size_t bytes) {
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) g_device_bytes.fetch_add(bytes, std::memory_order_relaxed);
  return e;
}

void device_free(void* p, size_t bytes) {
  if (!p) return;
  if (cudaFree(p) == cudaSuccess) g_device_bytes.fetch_sub(bytes, std::memory_order_relaxed);
}

DeviceState* current_state(int* status) {
  int dev = -1;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    t_last_cuda = int(e);
    *status = POSPOPCNT_ERR_NOT_INITIALIZED;
    return nullptr;
  }
  if (dev < 0 || dev >= MAX_DEVICES) {
    *status = POSPOPCNT_ERR_NOT_INITIALIZED;
    return nullptr;
  }
  if (!g_state[dev].ready) {
    std::lock_guard<std::mutex> lk(g_mutex);
    const int rc = init_locked(dev);
    if (rc != POSPOPCNT_OK) {
      *status = rc;
      return nullptr;
    }
  }
  *status = POSPOPCNT_OK;
  return &g_state[dev];
}

namespace {
// The slot of `map` bound to `stream`, binding a free one on first use; -1
// if all `capacity` slots are bound.  Caller holds g_mutex.
int bind_slot(std::unordered_map<cudaStream_t, int>& m, std::vector<int>& fl, int& next, int capacity,
              cudaStream_t stream) {
  auto it = m.find(stream);
  if (it != m.end()) return it->second;
  int slot;
  if (!fl.empty()) {
    slot = fl.back();
    fl.pop_back();
  } else {
    if (next >= capacity) return -1;
    slot = next++;
  }
  m.emplace(stream, slot);
  return slot;
}

// The batched work-queue slot bound to `stream` on `device`.
int stream_slot(int device, cudaStream_t stream) {
  std::lock_guard<std::mutex> lk(g_mutex);
  return bind_slot(g_slots[device], g_free_slots[device], g_next_slot[device], QUEUE_SLOTS, stream);
}
}  // namespace

PlainAcc plain_acc_for(DeviceState& st, cudaStream_t stream) {
  if (stream == cudaStreamPerThread) return PlainAcc{};
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) {
    cudaGetLastError();
    return PlainAcc{};
  }
  if (cs != cudaStreamCaptureStatusNone) return PlainAcc{};
  int slot;
  {
    std::lock_guard<std::mutex> lk(g_mutex);
    slot = bind_slot(g_plain_slots[st.device], g_free_plain[st.device], g_next_plain[st.device], PLAIN_SLOTS,
                     stream);
  }
  if (slot < 0) return PlainAcc{};
  char* base = static_cast<char*>(st.d_plain) + size_t(slot) * PLAIN_SLOT_BYTES;
  return PlainAcc{reinterpret_cast<unsigned long long*>(base), reinterpret_cast<unsigned*>(base + 512)};
}

Split plan_split(int width, uint64_t addr, size_t n) {
  const uint64_t wb = uint64_t(width / 8);
  const uint64_t nbytes = uint64_t(n) * wb;
  uint64_t head = (16 - (addr & 15)) & 15;
  if (head > nbytes) head = nbytes;
  head -= head % wb;  // addr is word aligned, so this is already whole words
  const uint64_t body = (nbytes - head) / 16;
  const uint64_t tail = nbytes - head - body * 16;
  return Split{size_t(head / wb), size_t(body), size_t(tail / wb)};
}

int normalize_config(const DeviceState& st, int width, pospopcnt_config* c) {
  if (width_index(width) < 0) return POSPOPCNT_ERR_INVALID;
  const pospopcnt_config d = default_config();
  if (c->kernel == POSPOPCNT_KERNEL_AUTO) c->kernel = d.kernel;
  if (c->threads == 0) c->threads = 256;
  if (c->blocks_per_sm < 0 || c->blocks_per_sm > 32) return POSPOPCNT_ERR_INVALID;
  if (c->flags & ~POSPOPCNT_FLAG_EVICT_FIRST) return POSPOPCNT_ERR_INVALID;
  if (width == 64 && c->kernel != POSPOPCNT_KERNEL_TMA) {  // 64-bit words: CSA 128/256 threads, unroll 4/8
    if (c->unroll == 0) c->unroll = 8;
    if (c->kernel != POSPOPCNT_KERNEL_CSA || (c->threads != 128 && c->threads != 256) ||
        (c->unroll != 4 && c->unroll != 8))
      return POSPOPCNT_ERR_INVALID;
    return POSPOPCNT_OK;
  }
  switch (c->kernel) {
    case POSPOPCNT_KERNEL_CSA:
      if (c->unroll == 0) c->unroll = 4;
      if (c->threads != 128 && c->threads != 256 && c->threads != 512) return POSPOPCNT_ERR_INVALID;
      if (c->unroll != 2 && c->unroll != 4 && c->unroll != 8) return POSPOPCNT_ERR_INVALID;
      return POSPOPCNT_OK;
    case POSPOPCNT_KERNEL_BALLOT:
      if (c->unroll == 0) c->unroll = 2;
      if (c->threads != 256) return POSPOPCNT_ERR_INVALID;
      if (c->unroll != 1 && c->unroll != 2 && c->unroll != 4) return POSPOPCNT_ERR_INVALID;
      return POSPOPCNT_OK;
    case POSPOPCNT_KERNEL_TMA: {
      if (c->stages == 0) c->stages = d.stages;
      if (c->chunk_bytes == 0) c->chunk_bytes = d.chunk_bytes;
      if (c->stages < 2 || c->stages > 16) return POSPOPCNT_ERR_INVALID;
      if (c->chunk_bytes < 16384 || c->chunk_bytes % 16384 != 0 || c->chunk_bytes > 196608)
        return POSPOPCNT_ERR_INVALID;
      const long smem = long(c->stages) * long(c->chunk_bytes);
      const long limit = st.smem_optin > 0 ? std::min<long>(st.smem_optin - 1024, 196608) : 196608;
      if (smem > limit) return POSPOPCNT_ERR_INVALID;
      return POSPOPCNT_OK;
    }
  }
  return POSPOPCNT_ERR_INVALID;
}

template <int K>
int launch_plain_k(const DeviceState&, const pospopcnt_config&, const void*, size_t, unsigned long long*, bool,
                   cudaStream_t, const PlainAcc&);

int launch_plain(const DeviceState& st, int width, const pospopcnt_config& cfg, const void* d_in, size_t n,
                 unsigned long long* d_counts, bool zero_first, cudaStream_t stream, const PlainAcc& acc) {
  switch (width) {
    case 1: return launch_plain_k<1>(st, cfg, d_in, n, d_counts, zero_first, stream, acc);
    case 8: return launch_plain_k<8>(st, cfg, d_in, n, d_counts, zero_first, stream, acc);
    case 16: return launch_plain_k<16>(st, cfg, d_in, n, d_counts, zero_first, stream, acc);
    case 32: return launch_plain_k<32>(st, cfg, d_in, n, d_counts, zero_first, stream, acc);
    case 64: return launch_plain_k<64>(st, cfg, d_in, n, d_counts, zero_first, stream, acc);
  }
  return POSPOPCNT_ERR_INVALID;
}

template <int K>
int launch_plain_sysmem_k(const DeviceState&, const void*, size_t, unsigned long long*, cudaStream_t);

int launch_plain_sysmem(const DeviceState& st, int width, const void* d_in, size_t n, unsigned long long* d_counts,
                        cudaStream_t stream) {
  switch (width) {
    case 8: return launch_plain_sysmem_k<8>(st, d_in, n, d_counts, stream);
    case 16: return launch_plain_sysmem_k<16>(st, d_in, n, d_counts, stream);
    case 32: return launch_plain_sysmem_k<32>(st, d_in, n, d_counts, stream);
  }
  return POSPOPCNT_ERR_INVALID;
}

namespace {

// Device address of [h, h + bytes) if the whole range is pinned host memory
// mapped into the current device's address space, else nullptr.
const void* mapped_device_view(const void* h, size_t bytes) {
  if (bytes == 0) return nullptr;
  cudaPointerAttributes a0, a1;
  const char* last = static_cast<const char*>(h) + bytes - 1;
  if (cudaPointerGetAttributes(&a0, h) != cudaSuccess || cudaPointerGetAttributes(&a1, last) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error of an unregistered pointer
    return nullptr;
  }
  if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer || !a1.devicePointer)
    return nullptr;
  if (static_cast<const char*>(a1.devicePointer) - static_cast<const char*>(a0.devicePointer) !=
      static_cast<ptrdiff_t>(bytes - 1))
    return nullptr;
  return a0.devicePointer;
}

int check_args(int width, const void* d_in, size_t n, const void* d_counts) {
  if (width_index(width) < 0) return POSPOPCNT_ERR_INVALID;
  if (!d_counts || (n > 0 && !d_in)) return POSPOPCNT_ERR_INVALID;
  if (reinterpret_cast<uintptr_t>(d_counts) % 8 != 0) return POSPOPCNT_ERR_MISALIGNED;
  if (reinterpret_cast<uintptr_t>(d_in) % uintptr_t(width / 8) != 0) return POSPOPCNT_ERR_MISALIGNED;
  if (n > (size_t(1) << 42) / size_t(width / 8)) return POSPOPCNT_ERR_TOO_LARGE;
  return POSPOPCNT_OK;
}

pospopcnt_config config_for(const DeviceState& st, int width, size_t n) {
  std::lock_guard<std::mutex> lk(g_mutex);  // set_config / autotune may write the table concurrently
  return g_cfg[st.device][width_index(width)][size_class(uint64_t(n) * uint64_t(width / 8))];
}

int count_impl(int width, const pospopcnt_config* cfg_in, bool zero, const void* d_in, size_t n,
               uint64_t* d_counts, cudaStream_t stream) {
  int rc = check_args(width, d_in, n, d_counts);
  if (rc != POSPOPCNT_OK) return rc;
  DeviceState* st = current_state(&rc);
  if (!st) return rc;
  pospopcnt_config cfg = cfg_in ? *cfg_in : config_for(*st, width, n);
  if ((rc = normalize_config(*st, width, &cfg)) != POSPOPCNT_OK) return rc;
  const PlainAcc acc = zero ? plain_acc_for(*st, stream) : PlainAcc{};
  return launch_plain(*st, width, cfg, d_in, n, reinterpret_cast<unsigned long long*>(d_counts), zero, stream, acc);
}

}  // namespace

}  // namespace ppc

using namespace ppc;

extern "C" {

int pospopcnt_init(int device) {
  std::lock_guard<std::mutex> lk(g_mutex);
  return init_locked(device);
}

int pospopcnt_u8(const void* d_in, size_t n, uint64_t* d_counts, cudaStream_t stream) {
  return count_impl(8, nullptr, true, d_in, n, d_counts, stream);
}
int pospopcnt_u16(const void* d_in, size_t n, uint64_t* d_counts, cudaStream_t stream) {
  return count_impl(16, nullptr, true, d_in, n, d_counts, stream);
}
int pospopcnt_u32(const void* d_in, size_t n, uint64_t* d_counts, cudaStream_t stream) {
  return count_impl(32, nullptr, true, d_in, n, d_counts, stream);
}
int pospopcnt_u64(const void* d_in, size_t n, uint64_t* d_counts, cudaStream_t stream) {
  return count_impl(64, nullptr, true, d_in, n, d_counts, stream);
}

int pospopcnt_count(int width, int kernel, const void* d_in, size_t n, uint64_t* d_counts,
                    cudaStream_t stream) {
  if (kernel == POSPOPCNT_KERNEL_AUTO) return count_impl(width, nullptr, true, d_in, n, d_counts, stream);
  if (kernel < 0 || kernel > POSPOPCNT_KERNEL_BALLOT) return POSPOPCNT_ERR_INVALID;
  pospopcnt_config cfg = default_config();
  cfg.kernel = kernel;
  cfg.unroll = kernel == POSPOPCNT_KERNEL_BALLOT ? 2 : width == 64 ? 8 : 4;
  return count_impl(width, &cfg, true, d_in, n, d_counts, stream);
}

int pospopcnt_count_config(int width, const pospopcnt_config* cfg, const void* d_in, size_t n,
                           uint64_t* d_counts, cudaStream_t stream) {
  if (!cfg) return POSPOPCNT_ERR_INVALID;
  return count_impl(width, cfg, true, d_in, n, d_counts, stream);
}

int pospopcnt_count_accumulate(int width, const void* d_in, size_t n, uint64_t* d_counts,
                               cudaStream_t stream) {
  return count_impl(width, nullptr, false, d_in, n, d_counts, stream);
}

int pospopcnt_popcount(const void* d_in, size_t nbytes, uint64_t* d_count, cudaStream_t stream) {
  if (!d_count || (nbytes > 0 && !d_in)) return POSPOPCNT_ERR_INVALID;
  if (reinterpret_cast<uintptr_t>(d_count) % 8 != 0) return POSPOPCNT_ERR_MISALIGNED;
  if (nbytes > (size_t(1) << 42)) return POSPOPCNT_ERR_TOO_LARGE;
  int rc = POSPOPCNT_OK;
  DeviceState* st = current_state(&rc);
  if (!st) return rc;
  // the launch shapes of the 16-bit count serve the single counter too,
  // except that its bulk-copy ring keeps three 48 KiB stages instead of four:
  // at 2 GiB on GB300, 7307 against 6956 GB/s (sustained, same box; 4 x 32,
  // 2 x 96 and 3 x 64 KiB measured 7244, 7221 and 7077)
  pospopcnt_config cfg = tuned_default(16, size_class(uint64_t(nbytes)));
  if (cfg.kernel == POSPOPCNT_KERNEL_TMA) cfg.stages = 3, cfg.chunk_bytes = 49152;
  if ((rc = normalize_config(*st, 16, &cfg)) != POSPOPCNT_OK) return rc;
  return launch_plain(*st, 1, cfg, d_in, nbytes, reinterpret_cast<unsigned long long*>(d_count), true, stream,
                      plain_acc_for(*st, stream));
}

int pospopcnt_count_host(int width, const void* h_in, size_t n, uint64_t* h_counts) {
  int rc = POSPOPCNT_OK;
  if (width_index(width) < 0 || !h_counts || (n > 0 && !h_in)) return POSPOPCNT_ERR_INVALID;
  if (reinterpret_cast<uintptr_t>(h_in) % uintptr_t(width / 8) != 0) return POSPOPCNT_ERR_MISALIGNED;
  DeviceState* st = current_state(&rc);
  if (!st) return rc;
  std::lock_guard<std::mutex> lk(g_host_mutex[st->device]);
  cudaError_t e = cudaSuccess;
  if (!st->d_acc) {
    for (int i = 0; i < 2; ++i) {
      if ((e = device_alloc(&st->d_stage[i], HOST_STAGE_BYTES)) != cudaSuccess) return cuda_fail(e);
      if ((e = cudaStreamCreateWithFlags(&st->hstream[i], cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e);
      if ((e = cudaEventCreateWithFlags(&st->hevent[i], cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e);
    }
    if ((e = device_alloc(reinterpret_cast<void**>(&st->d_acc), 64 * sizeof(uint64_t))) != cudaSuccess)
      return cuda_fail(e);
  }
  cudaStream_t s0 = st->hstream[0], s1 = st->hstream[1];
  const size_t wb = size_t(width / 8);
  // pinned, mapped host memory: the kernel reads it in place across C2C
  if (const void* dview = width != 64 ? mapped_device_view(h_in, n * wb) : nullptr) {
    if ((e = cudaMemsetAsync(st->d_acc, 0, sizeof(uint64_t) * size_t(width), s0)) != cudaSuccess)
      return cuda_fail(e);
    if ((rc = launch_plain_sysmem(*st, width, dview, n, st->d_acc, s0)) != POSPOPCNT_OK) return rc;
    if ((e = cudaMemcpyAsync(h_counts, st->d_acc, sizeof(uint64_t) * size_t(width), cudaMemcpyDeviceToHost,
                             s0)) != cudaSuccess)
      return cuda_fail(e);
    if ((e = cudaStreamSynchronize(s0)) != cudaSuccess) return cuda_fail(e);
    return POSPOPCNT_OK;
  }
  const size_t chunk_words = HOST_STAGE_BYTES / wb;
  const pospopcnt_config cfg = config_for(*st, width, chunk_words);
  if ((e = cudaMemsetAsync(st->d_acc, 0, sizeof(uint64_t) * size_t(width), s0)) != cudaSuccess)
    return cuda_fail(e);
  if ((e = cudaEventRecord(st->hevent[0], s0)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaStreamWaitEvent(s1, st->hevent[0], 0)) != cudaSuccess) return cuda_fail(e);
  const uint8_t* src = static_cast<const uint8_t*>(h_in);
  size_t done = 0;
  for (int j = 0; done < n; ++j) {
    const size_t words = std::min(chunk_words, n - done);
    cudaStream_t s = st->hstream[j & 1];
    void* buf = st->d_stage[j & 1];
    if ((e = cudaMemcpyAsync(buf, src + done * wb, words * wb, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return cuda_fail(e);
    if ((rc = launch_plain(*st, width, cfg, buf, words, st->d_acc, false, s)) != POSPOPCNT_OK) return rc;
    done += words;
  }
  if ((e = cudaEventRecord(st->hevent[1], s1)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaStreamWaitEvent(s0, st->hevent[1], 0)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMemcpyAsync(h_counts, st->d_acc, sizeof(uint64_t) * size_t(width), cudaMemcpyDeviceToHost,
                           s0)) != cudaSuccess)
    return cuda_fail(e);
  if ((e = cudaStreamSynchronize(s0)) != cudaSuccess) return cuda_fail(e);
  return POSPOPCNT_OK;
}

int pospopcnt_host_is_mapped(const void* h_in, size_t nbytes) {
  int rc = POSPOPCNT_OK;
  if (!current_state(&rc)) return 0;
  return mapped_device_view(h_in, nbytes) ? 1 : 0;
}

namespace ppc {
namespace {
int batched_impl(const void* d_in, const int64_t* d_offsets, size_t nseg, int width, uint64_t* d_counts,
                 cudaStream_t stream, bool checked, uint64_t n_words, const pospopcnt_batched_config* cfg);
bool batched_config_valid(const pospopcnt_batched_config& c);
pospopcnt_batched_config batched_config(int device, int width);
}  // namespace
}  // namespace ppc

int pospopcnt_batched(const void* d_in, const int64_t* d_offsets, size_t nseg, int width, uint64_t* d_counts,
                      cudaStream_t stream) {
  return ppc::batched_impl(d_in, d_offsets, nseg, width, d_counts, stream, false, 0, nullptr);
}

int pospopcnt_batched_checked(const void* d_in, size_t n_words, const int64_t* d_offsets, size_t nseg, int width,
                              uint64_t* d_counts, cudaStream_t stream) {
  return ppc::batched_impl(d_in, d_offsets, nseg, width, d_counts, stream, true, n_words, nullptr);
}

}  // extern "C"

namespace ppc {
namespace {
pospopcnt_batched_config batched_config(int device, int width) {
  std::lock_guard<std::mutex> lk(g_mutex);
  const int w = width_index(width);
  return g_bcfg_set[device][w] ? g_bcfg[device][w] : BATCHED_DEFAULT;
}

bool batched_config_valid(const pospopcnt_batched_config& c) {
  return c.unit_bytes >= 4096 && c.unit_bytes <= (1 << 20) && c.unit_bytes % 128 == 0 && c.blocks_per_sm >= 0 &&
         c.blocks_per_sm <= 32 && (c.ring_stages == 0 || (c.ring_stages >= 2 && c.ring_stages <= 4)) &&
         (c.vectors_per_lane == 0 || c.vectors_per_lane == 4 || c.vectors_per_lane == 8 ||
          c.vectors_per_lane == 16) &&
         !(c.vectors_per_lane == 16 && c.ring_stages == 4);  // 8 warps x 4 x 8 KiB: more than a ring may take
}

int batched_impl(const void* d_in, const int64_t* d_offsets, size_t nseg, int width, uint64_t* d_counts,
                 cudaStream_t stream, bool checked, uint64_t n_words, const pospopcnt_batched_config* cfg) {
  if (width != 8 && width != 16 && width != 32) return POSPOPCNT_ERR_INVALID;
  if (nseg == 0) return POSPOPCNT_OK;
  if (!d_in || !d_offsets || !d_counts) return POSPOPCNT_ERR_INVALID;
  if (reinterpret_cast<uintptr_t>(d_in) % uintptr_t(width / 8) != 0) return POSPOPCNT_ERR_MISALIGNED;
  if (reinterpret_cast<uintptr_t>(d_offsets) % 8 != 0 || reinterpret_cast<uintptr_t>(d_counts) % 8 != 0)
    return POSPOPCNT_ERR_MISALIGNED;
  if (nseg > (size_t(1) << 40)) return POSPOPCNT_ERR_TOO_LARGE;
  int rc = POSPOPCNT_OK;
  DeviceState* st = current_state(&rc);
  if (!st) return rc;
  const int slot = stream_slot(st->device, stream);
  if (slot < 0) return POSPOPCNT_ERR_TOO_LARGE;
  cudaError_t e = cudaMemsetAsync(d_counts, 0, sizeof(uint64_t) * size_t(width) * nseg, stream);
  if (e != cudaSuccess) return cuda_fail(e);
  void* q = static_cast<char*>(st->d_queue) + size_t(slot) * QUEUE_SLOT_BYTES;
  if (checked && (rc = launch_offsets_check(*st, d_offsets, nseg, n_words, q, stream)) != POSPOPCNT_OK) return rc;
  const pospopcnt_batched_config c = cfg ? *cfg : batched_config(st->device, width);
  return launch_batched(*st, d_in, d_offsets, nseg, width, reinterpret_cast<unsigned long long*>(d_counts), q,
                        c.unit_bytes / (width / 8), c.blocks_per_sm, c.ring_stages, c.vectors_per_lane, stream);
}
}  // namespace
}  // namespace ppc

extern "C" {

int pospopcnt_plain_segments(const void* d_in, const int64_t* h_offsets, size_t nseg, int width,
                             uint64_t* d_counts, cudaStream_t stream) {
  if (width_index(width) < 0) return POSPOPCNT_ERR_INVALID;
  if (nseg == 0) return POSPOPCNT_OK;
  if (!d_in || !h_offsets || !d_counts) return POSPOPCNT_ERR_INVALID;
  for (size_t s = 0; s < nseg; ++s)
    if (h_offsets[s] < 0 || h_offsets[s + 1] < h_offsets[s]) return POSPOPCNT_ERR_INVALID;
  const size_t wb = size_t(width / 8);
  const uint8_t* base = static_cast<const uint8_t*>(d_in);
  for (size_t s = 0; s < nseg; ++s) {
    const int rc = count_impl(width, nullptr, true, base + size_t(h_offsets[s]) * wb,
                              size_t(h_offsets[s + 1] - h_offsets[s]), d_counts + s * size_t(width), stream);
    if (rc != POSPOPCNT_OK) return rc;
  }
  return POSPOPCNT_OK;
}

}  // extern "C"

namespace ppc {
namespace {
// Returns the work-queue slot bound to `stream` on `device` to the free list.
void release_slot(int device, cudaStream_t stream) {
  std::lock_guard<std::mutex> lk(g_mutex);
  auto& m = g_slots[device];
  auto it = m.find(stream);
  if (it != m.end()) {
    g_free_slots[device].push_back(it->second);
    m.erase(it);
  }
  auto& mp = g_plain_slots[device];
  auto ip = mp.find(stream);
  if (ip != mp.end()) {
    g_free_plain[device].push_back(ip->second);
    mp.erase(ip);
  }
}
}  // namespace
}  // namespace ppc

struct pospopcnt_graph {
  cudaStream_t stream = nullptr;  // the capture stream: its queue slot belongs to the graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int device = -1;
};

extern "C" {

int pospopcnt_batched_graph_create(const void* d_in, const int64_t* d_offsets, size_t nseg, int width,
                                   uint64_t* d_counts, pospopcnt_graph** out) {
  if (!out) return POSPOPCNT_ERR_INVALID;
  *out = nullptr;
  int rc = POSPOPCNT_OK;
  DeviceState* st = current_state(&rc);  // workspace first: nothing is allocated during capture
  if (!st) return rc;
  auto* g = new pospopcnt_graph();
  g->device = st->device;
  cudaError_t e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    rc = cuda_fail(e);
  } else {
    rc = pospopcnt_batched(d_in, d_offsets, nseg, width, d_counts, g->stream);
    const cudaError_t e2 = cudaStreamEndCapture(g->stream, &g->graph);
    if (rc == POSPOPCNT_OK && e2 != cudaSuccess) rc = cuda_fail(e2);
    if (rc == POSPOPCNT_OK && (e = cudaGraphInstantiate(&g->exec, g->graph, 0)) != cudaSuccess) rc = cuda_fail(e);
  }
  if (rc != POSPOPCNT_OK) {
    pospopcnt_graph_destroy(g);
    return rc;
  }
  *out = g;
  return POSPOPCNT_OK;
}

int pospopcnt_graph_launch(pospopcnt_graph* g, cudaStream_t stream) {
  if (!g || !g->exec) return POSPOPCNT_ERR_INVALID;
  const cudaError_t e = cudaGraphLaunch(g->exec, stream);
  return e == cudaSuccess ? POSPOPCNT_OK : cuda_fail(e);
}

int pospopcnt_graph_destroy(pospopcnt_graph* g) {
  if (!g) return POSPOPCNT_ERR_INVALID;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->stream) {
    if (g->device >= 0) ppc::release_slot(g->device, g->stream);
    cudaStreamDestroy(g->stream);
  }
  delete g;
  return POSPOPCNT_OK;
}

int pospopcnt_release_stream(cudaStream_t stream) {
  int rc = POSPOPCNT_OK;
  DeviceState* st = current_state(&rc);
  if (!st) return rc;
  ppc::release_slot(st->device, stream);
  return POSPOPCNT_OK;
}

int pospopcnt_check_device_error(cudaStream_t stream) {
  // Creates nothing: a word that does not exist on this device cannot hold
  // an error.
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  if (dev < 0 || dev >= MAX_DEVICES) return POSPOPCNT_ERR_NOT_INITIALIZED;
  if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e);
  unsigned* words[2] = {nullptr, ppc::noalloc_error_word(dev)};
  {
    std::lock_guard<std::mutex> lk(g_mutex);
    if (g_state[dev].ready) words[0] = g_state[dev].d_err;
  }
  unsigned all = 0;
  for (unsigned* w : words) {
    if (!w) continue;
    unsigned h = 0;
    if ((e = cudaMemcpy(&h, w, sizeof h, cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(e);
    if (h && (e = cudaMemset(w, 0, sizeof h)) != cudaSuccess) return cuda_fail(e);
    all |= h;
  }
  if (all)
    return (all & ERR_BIT_BAD_OFFSETS) && !(all & ~unsigned(ERR_BIT_BAD_OFFSETS)) ? POSPOPCNT_ERR_INVALID
                                                                                    : POSPOPCNT_ERR_TIMEOUT;
  return POSPOPCNT_OK;
}

int pospopcnt_plan_split(int width, uint64_t addr, size_t n, size_t* head_words, size_t* body_vectors,
                         size_t* tail_words) {
  if (width_index(width) < 0 || !head_words || !body_vectors || !tail_words) return POSPOPCNT_ERR_INVALID;
  if (addr % uint64_t(width / 8) != 0) return POSPOPCNT_ERR_MISALIGNED;
  const Split s = plan_split(width, addr, n);
  *head_words = s.head_words;
  *body_vectors = s.body_vectors;
  *tail_words = s.tail_words;
  return POSPOPCNT_OK;
}

int pospopcnt_get_config(int width, size_t n, pospopcnt_config* cfg) {
  if (width_index(width) < 0 || !cfg) return POSPOPCNT_ERR_INVALID;
  int rc = POSPOPCNT_OK;
  DeviceState* st = current_state(&rc);
  if (!st) return rc;
  *cfg = config_for(*st, width, n);
  return normalize_config(*st, width, cfg);
}

int pospopcnt_set_config(int width, int size_class_, const pospopcnt_config* cfg) {
  if (width_index(width) < 0 || !cfg || size_class_ < -1 || size_class_ >= NCLASSES) return POSPOPCNT_ERR_INVALID;
  int rc = POSPOPCNT_OK;
  DeviceState* st = current_state(&rc);
  if (!st) return rc;
  pospopcnt_config c = *cfg;
  if ((rc = normalize_config(*st, width, &c)) != POSPOPCNT_OK) return rc;
  std::lock_guard<std::mutex> lk(g_mutex);
  for (int k = 0; k < NCLASSES; ++k)
    if (size_class_ == -1 || k == size_class_) g_cfg[st->device][width_index(width)][k] = c;
  return POSPOPCNT_OK;
}

int pospopcnt_autotune(int width, const void* d_in, size_t n, uint64_t* d_scratch_counts, pospopcnt_config* best,
                       float* best_ms) {
  int rc = check_args(width, d_in, n, d_scratch_counts);
  if (rc != POSPOPCNT_OK) return rc;
  if (!best || n == 0) return POSPOPCNT_ERR_INVALID;
  DeviceState* st = current_state(&rc);
  if (!st) return rc;
  std::vector<pospopcnt_config> cands;
  for (int t : {128, 256, 512})
    for (int u : {2, 4, 8}) {
      pospopcnt_config c = default_config();
      c.kernel = POSPOPCNT_KERNEL_CSA, c.threads = t, c.unroll = u;
      if (normalize_config(*st, width, &c) == POSPOPCNT_OK) cands.push_back(c);
    }
  for (int s : {2, 3, 4, 6, 8})
    for (int ch : {16384, 32768, 49152, 65536, 98304})
      for (int fl : {0, POSPOPCNT_FLAG_EVICT_FIRST}) {
        pospopcnt_config c = default_config();
        c.kernel = POSPOPCNT_KERNEL_TMA, c.stages = s, c.chunk_bytes = ch, c.flags = fl;
        if (normalize_config(*st, width, &c) == POSPOPCNT_OK) cands.push_back(c);
      }
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e);
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // Times `reps` back-to-back calls of candidate i; mean ms per call.
  auto time_calls = [&](size_t i, int reps, float* ms) -> int {
    cudaEventRecord(e0, s);
    int r = POSPOPCNT_OK;
    for (int k = 0; k < reps && r == POSPOPCNT_OK; ++k) r = count_impl(width, &cands[i], true, d_in, n, d_scratch_counts, s);
    cudaEventRecord(e1, s);
    if (r != POSPOPCNT_OK) return r;
    const cudaError_t se = cudaEventSynchronize(e1);
    if (se != cudaSuccess) return cuda_fail(se);
    cudaEventElapsedTime(ms, e0, e1);
    *ms /= float(reps);
    return POSPOPCNT_OK;
  };
  // Pass 1: warm-up, a first timing (sets each candidate's repetitions to
  // about 2 ms of calls, 5..200) and the check that every candidate agrees.
  std::vector<uint64_t> ref(static_cast<size_t>(width), 0), got(static_cast<size_t>(width), 0);
  std::vector<int> reps(cands.size(), 5);
  rc = POSPOPCNT_OK;
  for (size_t i = 0; i < cands.size() && rc == POSPOPCNT_OK; ++i) {
    for (int w = 0; w < 2 && rc == POSPOPCNT_OK; ++w)
      rc = count_impl(width, &cands[i], true, d_in, n, d_scratch_counts, s);
    float ms = 0.f;
    if (rc == POSPOPCNT_OK) rc = time_calls(i, 5, &ms);
    if (rc != POSPOPCNT_OK) break;
    reps[i] = std::max(5, std::min(200, int(2.0f / std::max(ms, 1e-4f))));
    if ((e = cudaMemcpy(got.data(), d_scratch_counts, sizeof(uint64_t) * size_t(width), cudaMemcpyDeviceToHost)) !=
        cudaSuccess) {
      rc = cuda_fail(e);
      break;
    }
    if (i == 0) {
      ref = got;
    } else if (got != ref) {
      rc = POSPOPCNT_ERR_INVALID;  // candidates disagree: refuse to tune
      break;
    }
  }
  // Passes 2..4: three rounds, each timing every candidate once, so that a
  // slow stretch of the GPU (clocks, a neighbour) hits all of them alike;
  // a candidate's time is its median round.
  constexpr int ROUNDS = 3;
  std::vector<std::vector<float>> t(cands.size());
  for (int round = 0; round < ROUNDS && rc == POSPOPCNT_OK; ++round)
    for (size_t i = 0; i < cands.size() && rc == POSPOPCNT_OK; ++i) {
      float ms = 0.f;
      rc = time_calls(i, reps[i], &ms);
      t[i].push_back(ms);
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  ppc::release_slot(st->device, s);  // the accumulator the timed calls bound to the private stream
  cudaStreamDestroy(s);
  if (rc != POSPOPCNT_OK) return rc;
  float best_t = 1e30f;
  int best_i = -1;
  for (size_t i = 0; i < cands.size(); ++i) {
    std::vector<float> v = t[i];
    std::sort(v.begin(), v.end());
    const float med = v[v.size() / 2];
    if (med < best_t) best_t = med, best_i = int(i);
  }
  *best = cands[size_t(best_i)];
  if (best_ms) *best_ms = best_t;
  std::lock_guard<std::mutex> lk(g_mutex);
  g_cfg[st->device][width_index(width)][size_class(uint64_t(n) * uint64_t(width / 8))] = *best;
  return POSPOPCNT_OK;
}

int pospopcnt_batched_get_config(int width, pospopcnt_batched_config* cfg) {
  if ((width != 8 && width != 16 && width != 32) || !cfg) return POSPOPCNT_ERR_INVALID;
  int rc = POSPOPCNT_OK;
  DeviceState* st = current_state(&rc);
  if (!st) return rc;
  *cfg = batched_config(st->device, width);
  return POSPOPCNT_OK;
}

int pospopcnt_batched_set_config(int width, const pospopcnt_batched_config* cfg) {
  if ((width != 8 && width != 16 && width != 32) || (cfg && !batched_config_valid(*cfg))) return POSPOPCNT_ERR_INVALID;
  int rc = POSPOPCNT_OK;
  DeviceState* st = current_state(&rc);
  if (!st) return rc;
  std::lock_guard<std::mutex> lk(g_mutex);
  const int w = width_index(width);
  g_bcfg_set[st->device][w] = cfg != nullptr;
  if (cfg) g_bcfg[st->device][w] = *cfg;
  return POSPOPCNT_OK;
}

int pospopcnt_batched_autotune(const void* d_in, const int64_t* d_offsets, size_t nseg, int width,
                               uint64_t* d_counts, pospopcnt_batched_config* best, float* best_ms,
                               cudaStream_t stream) {
  if (!best || nseg == 0) return POSPOPCNT_ERR_INVALID;
  int rc = POSPOPCNT_OK;
  DeviceState* st = current_state(&rc);
  if (!st) return rc;
  std::vector<pospopcnt_batched_config> cands;
  for (int unit : {4096, 8192, 16384, 32768, 65536})
    for (int bps : {1, 2, 0})
      for (int stages : {2, 3, 4})
        for (int vpl : {4, 8, 16}) {
          const pospopcnt_batched_config c{unit, bps, stages, vpl};
          if (batched_config_valid(c)) cands.push_back(c);
        }
  const size_t row_words = size_t(width) * nseg;
  std::vector<uint64_t> ref(row_words), got(row_words);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(e);
  }
  // Times `reps` back-to-back calls of candidate i; mean ms per call.
  auto time_calls = [&](size_t i, int reps, float* ms) -> int {
    cudaEventRecord(e0, stream);
    int r = POSPOPCNT_OK;
    for (int k = 0; k < reps && r == POSPOPCNT_OK; ++k)
      r = batched_impl(d_in, d_offsets, nseg, width, d_counts, stream, false, 0, &cands[i]);
    cudaEventRecord(e1, stream);
    if (r != POSPOPCNT_OK) return r;
    const cudaError_t se = cudaEventSynchronize(e1);
    if (se != cudaSuccess) return cuda_fail(se);
    cudaEventElapsedTime(ms, e0, e1);
    *ms /= float(reps);
    return POSPOPCNT_OK;
  };
  // Pass 1: warm-up, a first timing (about 2 ms of calls per round
  // afterwards, 3..200) and the check that every candidate agrees.
  std::vector<int> reps(cands.size(), 3);
  for (size_t i = 0; i < cands.size() && rc == POSPOPCNT_OK; ++i) {
    rc = batched_impl(d_in, d_offsets, nseg, width, d_counts, stream, false, 0, &cands[i]);  // warm-up
    float ms = 0.f;
    if (rc == POSPOPCNT_OK) rc = time_calls(i, 3, &ms);
    if (rc != POSPOPCNT_OK) break;
    reps[i] = std::max(3, std::min(200, int(2.0f / std::max(ms, 1e-4f))));
    if ((e = cudaMemcpy(got.data(), d_counts, sizeof(uint64_t) * row_words, cudaMemcpyDeviceToHost)) != cudaSuccess) {
      rc = cuda_fail(e);
      break;
    }
    if (i == 0) {
      ref = got;
    } else if (got != ref) {
      rc = POSPOPCNT_ERR_INVALID;  // candidates disagree: refuse to tune
      break;
    }
  }
  // Three rounds, each timing every candidate once; median round.
  constexpr int ROUNDS = 3;
  std::vector<std::vector<float>> t(cands.size());
  for (int round = 0; round < ROUNDS && rc == POSPOPCNT_OK; ++round)
    for (size_t i = 0; i < cands.size() && rc == POSPOPCNT_OK; ++i) {
      float ms = 0.f;
      rc = time_calls(i, reps[i], &ms);
      t[i].push_back(ms);
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != POSPOPCNT_OK) return rc;
  float best_t = 1e30f;
  int best_i = -1;
  for (size_t i = 0; i < cands.size(); ++i) {
    std::vector<float> v = t[i];
    std::sort(v.begin(), v.end());
    const float med = v[v.size() / 2];
    if (med < best_t) best_t = med, best_i = int(i);
  }
  *best = cands[size_t(best_i)];
  if (best_ms) *best_ms = best_t;
  std::lock_guard<std::mutex> lk(g_mutex);
  g_bcfg[st->device][width_index(width)] = *best;
  g_bcfg_set[st->device][width_index(width)] = true;
  return POSPOPCNT_OK;
}

const char* pospopcnt_strerror(int status) {
  switch (status) {
    case POSPOPCNT_OK: return "ok";
    case POSPOPCNT_ERR_INVALID: return "invalid argument";
    case POSPOPCNT_ERR_MISALIGNED: return "pointer not aligned to the word size";
    case POSPOPCNT_ERR_CUDA: return "CUDA runtime error (see pospopcnt_last_cuda_error)";
    case POSPOPCNT_ERR_NOT_INITIALIZED: return "no usable CUDA device";
    case POSPOPCNT_ERR_TIMEOUT: return "a bounded device-side wait gave up";
    case POSPOPCNT_ERR_TOO_LARGE: return "size beyond a documented limit";
  }
  return "unknown status";
}

int pospopcnt_last_cuda_error(void) { return t_last_cuda; }

uint64_t pospopcnt_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

uint64_t pospopcnt_device_bytes_allocated(void) { return g_device_bytes.load(std::memory_order_relaxed); }

}  // extern "C"
