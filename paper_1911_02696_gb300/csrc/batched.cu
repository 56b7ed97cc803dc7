// Segmented pospopcnt in one persistent launch.
//
// Segment s covers words [offsets[s], offsets[s+1]).  The word range
// [offsets[0], offsets[nseg]) is cut into units of `tile_words` words whose
// inner boundaries fall on 16-byte addresses.  Every warp of a persistent
// grid claims runs of consecutive units from an atomic work queue (guided
// self-scheduling: about 1/(2 x warps) of what is left, at least one unit),
// so no warp waits for another.  A warp finds the segment holding the first
// word of its run with a 32-way search over the offsets, then walks the
// pieces (segment ∩ run): each piece is counted like a plain call --
// unaligned head and ragged tail word by word, the body in 16-byte vectors
// through the carry-save circuit F_5 (§2, §4.1) with popc flushes -- and its
// counts are reduced across the warp and added with one 64-bit atomic per
// position into the segment's row.  Rows are zeroed beforehand by a memset.
//
// The queue counter lives in a 128-byte slot of the library's workspace; the
// last CTA to finish resets it, so consecutive launches on one stream (and
// replays of a captured graph) reuse the slot without a memset.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "device_common.cuh"
#include "internal.h"
#include "segment_common.cuh"

namespace ppc {

// Segment s is words [offsets[s], offsets[s+1]) of `base`.
struct BatchedArgs {
  const uint8_t* base;
  const int64_t* offsets;
  uint64_t nseg;
  unsigned long long* counts;
  QueueSlot* q;
  uint64_t tile_words;  // multiple of 8 warps x 16 bytes
  unsigned* err;        // device error word (bounded waits)
};

// Per-warp bulk-copy ring: lane 0 streams the 16-byte-aligned body of a long
// piece into STAGES shared-memory stages of one trip (32 lanes x VPL
// vectors) each, one mbarrier per stage; the warp counts from shared memory
// while the next trips are in flight.  VPL -- the words each lane takes per
// trip -- sets the copy size (2, 4 or 8 KiB per stage) and the circuit: F_4
// over 4 vectors per lane, F_5 over 8, and for 16 two runs of F_5 per trip.
// Two stages of 4 KiB (64 KiB per CTA) measured faster than three (96 KiB)
// on the 20,000-segment layout, and faster than three stages of 2 KiB at
// any CTA count per SM.
constexpr int RING_STAGES = 2;  // default ring depth (a launch may pick 3 or 4)
constexpr int RING_VPL = 8;     // default vectors per lane per trip (a launch may pick 4 or 16)

template <int VPL>
struct ring_shape {
  static constexpr int TRIP_VECS = 32 * VPL;
  static constexpr int TRIP_BYTES = TRIP_VECS * 16;
  static constexpr int MIN_VECS = 2 * TRIP_VECS;  // shorter bodies are loaded directly
  static constexpr int SUB = VPL < 8 ? VPL : 8;   // vectors per lane per circuit run
  static constexpr int R = 4 * SUB;
  static constexpr int L = ilog2<R>::value;
};
template <int STAGES, int VPL>
constexpr size_t bt_ring_smem() { return size_t(BT_WARPS) * STAGES * ring_shape<VPL>::TRIP_BYTES; }
// Largest ring a launch may ask for (8 warps x stages x trip bytes).
constexpr size_t BT_RING_MAX_SMEM = 196608;

struct WarpRing {
  uint8_t* buf;    // STAGES x TRIP_BYTES
  uint64_t* full;  // STAGES barriers
  uint32_t seq;    // trips issued (and consumed) by this warp so far
};

// warp_piece_counts with the body streamed through the warp's ring when it
// is long enough.  Returns false (after recording the error) if a bounded
// wait gave up; the warp then stops counting.
template <int K, int STAGES, int VPL>
__device__ __forceinline__ bool warp_piece_counts_ring(const uint8_t* base, uint64_t pa, uint64_t pb,
                                                       WarpRing& r, unsigned* err, uint32_t& out) {
  using RS = ring_shape<VPL>;
  constexpr int WB = K / 8;
  constexpr int TRIP_VECS = RS::TRIP_VECS, TRIP_BYTES = RS::TRIP_BYTES, SUB = RS::SUB, R = RS::R, L = RS::L;
  const int lane = threadIdx.x & 31;
  const uint64_t A = reinterpret_cast<uint64_t>(base) + pa * WB;
  const uint64_t E = reinterpret_cast<uint64_t>(base) + pb * WB;
  uint64_t bodyA = (A + 15) & ~uint64_t(15);
  if (bodyA > E) bodyA = E;
  uint64_t bodyE = E & ~uint64_t(15);
  if (bodyE < bodyA) bodyE = bodyA;
  const uint64_t nvec = (bodyE - bodyA) / 16;
  if (nvec < RS::MIN_VECS) {
    out = warp_piece_counts<K, BT_VPL>(base, pa, pb);
    return true;
  }
  const uint32_t head_words = uint32_t((bodyA - A) / WB);
  const uint32_t tail_words = uint32_t((E - bodyE) / WB);
  uint32_t edge = 0;
  if (uint32_t(lane) < head_words)
    edge = load_word<K>(reinterpret_cast<const uint8_t*>(A) + lane * WB);
  else if (lane >= 16 && uint32_t(lane - 16) < tail_words)
    edge = load_word<K>(reinterpret_cast<const uint8_t*>(bodyE) + (lane - 16) * WB);

  const uint4* src = reinterpret_cast<const uint4*>(bodyA);
  const uint32_t ntrips = uint32_t((nvec + TRIP_VECS - 1) / TRIP_VECS);
  auto issue = [&](uint32_t t) {  // lane 0 only
    const uint32_t s = (r.seq + t) % STAGES;
    const uint64_t left = nvec - uint64_t(t) * TRIP_VECS;
    const uint32_t bytes = uint32_t(left < TRIP_VECS ? left : TRIP_VECS) * 16u;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier reads of the stage first
    mbar_arrive_expect_tx(&r.full[s], bytes);
    bulk_g2s(r.buf + size_t(s) * TRIP_BYTES, src + uint64_t(t) * TRIP_VECS, bytes, &r.full[s]);
  };
  if (lane == 0)
    for (uint32_t t = 0; t < ntrips && t < uint32_t(STAGES); ++t) issue(t);

  uint32_t B[L];
#pragma unroll
  for (int l = 0; l < L; ++l) B[l] = 0;
  uint32_t top[K];
#pragma unroll
  for (int p = 0; p < K; ++p) top[p] = 0;
  for (uint32_t t = 0; t < ntrips; ++t) {
    const uint32_t seq = r.seq + t;
    const uint32_t s = seq % STAGES;
    const bool ok = __all_sync(FULL_MASK, mbar_wait_bounded(&r.full[s], (seq / STAGES) & 1u, WAIT_LIMIT_NS));
    if (!ok) {
      if (lane == 0) {
        atomicOr(err, ERR_BIT_TIMEOUT_FULL);
        // wait (bounded) for the copies still in flight into this warp's ring
        for (uint32_t u = t; u < ntrips && u < t + STAGES; ++u)
          if (!mbar_wait_bounded(&r.full[(r.seq + u) % STAGES], ((r.seq + u) / STAGES) & 1u,
                                 WAIT_LIMIT_NS)) {
            atomicOr(err, ERR_BIT_TIMEOUT_DRAIN);
            break;
          }
      }
      __syncwarp();
      return false;
    }
    const uint64_t left = nvec - uint64_t(t) * TRIP_VECS;
    const uint32_t nv = uint32_t(left < TRIP_VECS ? left : TRIP_VECS);
    const uint4* sv = reinterpret_cast<const uint4*>(r.buf + size_t(s) * TRIP_BYTES);
#pragma unroll
    for (int h = 0; h < VPL / SUB; ++h) {
      uint32_t d[R];
#pragma unroll
      for (int j = 0; j < SUB; ++j) {
        const uint32_t idx = uint32_t(h * SUB + j) * 32 + uint32_t(lane);
        const uint4 x = idx < nv ? sv[idx] : make_uint4(0, 0, 0, 0);
        d[4 * j + 0] = x.x, d[4 * j + 1] = x.y, d[4 * j + 2] = x.z, d[4 * j + 3] = x.w;
      }
      flush<K>(top, Circuit<L>::run(d, B));
    }
    __syncwarp();  // every lane has read the stage
    if (lane == 0 && t + STAGES < ntrips) issue(t + STAGES);
  }
  r.seq += ntrips;
  uint32_t c[K];
  finalize<K, L>(c, top, B);
  count_word<K>(c, edge);
  out = warp_reduce_positions<K>(c);
  return true;
}


// Counts words [pa, pb) of `base` with the whole warp and adds the result to
// row[0..K-1]; false if a bounded wait gave up.
template <int K, int STAGES, int VPL>
__device__ __forceinline__ bool warp_count_piece(const uint8_t* base, uint64_t pa, uint64_t pb,
                                                 unsigned long long* row, WarpRing& ring, unsigned* err) {
  constexpr int SH = 5 - ilog2<K>::value;
  const int lane = threadIdx.x & 31;
  uint32_t v = 0;
  if (!warp_piece_counts_ring<K, STAGES, VPL>(base, pa, pb, ring, err, v)) return false;
  if ((lane & ((1 << SH) - 1)) == 0 && v) atomicAdd(row + (lane >> SH), (unsigned long long)v);
  return true;
}

template <int K, int STAGES, int VPL>
__global__ void __launch_bounds__(BT_THREADS, bt_batched_min_blocks<K>::value) batched_kernel(BatchedArgs a) {
  constexpr int WB = K / 8;
  extern __shared__ __align__(128) uint8_t bt_ring[];
  __shared__ __align__(8) uint64_t bt_full[BT_WARPS][STAGES];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  if (*reinterpret_cast<volatile unsigned*>(&a.q->bad)) {  // the offsets check failed: touch no input
    retire_cta(a.q);
    return;
  }
  WarpRing ring{bt_ring + size_t(warp) * STAGES * ring_shape<VPL>::TRIP_BYTES, bt_full[warp], 0};
  if (lane == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&ring.full[s], 1);
    mbar_fence_init();
  }
  __syncwarp();
  bool failed = false;
  const int64_t o0 = a.offsets[0];
  const int64_t oN = a.offsets[a.nseg];
  // units start at the 16-byte boundary at or before word o0, so inner unit
  // boundaries are aligned
  const uint64_t mis = (reinterpret_cast<uint64_t>(a.base) + uint64_t(o0) * WB) & 15;
  const int64_t start = o0 - int64_t(mis / WB);
  const uint64_t U = a.tile_words;  // words per scheduling unit
  const uint64_t units = oN > start ? (uint64_t(oN - start) + U - 1) / U : 0;
  const uint64_t nwarps = uint64_t(gridDim.x) * BT_WARPS;

  // Guided self-scheduling per warp: take about 1/(2 nwarps) of the units
  // still unclaimed (at least one), so early grabs are large, late ones
  // small, and no warp waits for another.  Every warp's first grab is the
  // one it would get at the start, k0 units at k0 x (its index), taken
  // without the queue; the queue hands out the units after them, so the
  // launch does not begin with every warp contending for one counter.
  const uint64_t k0 = units / (2 * nwarps) > 1 ? units / (2 * nwarps) : 1;
  const uint64_t dyn_base = nwarps * k0;  // first unit the queue hands out
  bool first = true;
  while (!failed) {
    uint64_t u0 = 0, u1 = 0;
    if (first) {
      first = false;
      u0 = (uint64_t(blockIdx.x) * BT_WARPS + uint64_t(warp)) * k0;
      u1 = u0 + k0 < units ? u0 + k0 : units;
      if (u0 >= units) continue;  // nothing static for this warp: on to the queue
    } else {
      if (lane == 0) {
        const uint64_t seen = dyn_base + *reinterpret_cast<volatile unsigned long long*>(&a.q->next);
        const uint64_t left = seen < units ? units - seen : 0;
        const uint64_t k = left / (2 * nwarps) > 1 ? left / (2 * nwarps) : 1;
        u0 = dyn_base + atomicAdd(&a.q->next, (unsigned long long)k);
        u1 = u0 + k < units ? u0 + k : units;
      }
      u0 = __shfl_sync(FULL_MASK, u0, 0);
      u1 = __shfl_sync(FULL_MASK, u1, 0);
      if (u0 >= units) break;
    }
    int64_t w0 = start + int64_t(u0 * U);
    int64_t w1 = start + int64_t(u1 * U);
    if (w0 < o0) w0 = o0;
    if (w1 > oN) w1 = oN;
    if (w0 >= w1) continue;
    uint64_t s = find_segment(a.offsets, a.nseg, w0);
    int64_t seg_lo = a.offsets[s];
    for (;;) {
      const int64_t seg_hi = a.offsets[s + 1];
      const int64_t pa = seg_lo > w0 ? seg_lo : w0;
      const int64_t pb = seg_hi < w1 ? seg_hi : w1;
      if (pa < pb) {
        if (!warp_count_piece<K, STAGES, VPL>(a.base, uint64_t(pa), uint64_t(pb), a.counts + s * K, ring, a.err)) {
          failed = true;
          break;
        }
      }
      if (seg_hi >= w1 || s + 1 >= a.nseg) break;
      ++s;
      seg_lo = seg_hi;
    }
  }
  retire_cta(a.q);
}

template <int K, int STAGES, int VPL>
static int launch_batched_ks(const DeviceState& st, const BatchedArgs& a, cudaStream_t stream,
                            int blocks_per_sm = 0) {
  auto kern = batched_kernel<K, STAGES, VPL>;
  constexpr size_t smem = bt_ring_smem<STAGES, VPL>();
  static_assert(smem <= BT_RING_MAX_SMEM, "ring larger than a launch may ask for");
  if (const cudaError_t e = ensure_dynamic_smem<batched_kernel<K, STAGES, VPL>>(st.device, int(smem)))
    return cuda_fail(e);
  const int occ = resident_blocks(reinterpret_cast<const void*>(kern), st.device, BT_THREADS, smem);
  const int bps = blocks_per_sm > 0 && blocks_per_sm < occ ? blocks_per_sm : occ;
  const unsigned grid = unsigned(st.sms) * unsigned(bps);
  kern<<<grid, BT_THREADS, smem, stream>>>(a);
  note_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? POSPOPCNT_OK : cuda_fail(e);
}

template <int K, int VPL>
static int launch_batched_kv(const DeviceState& st, const BatchedArgs& a, cudaStream_t stream, int blocks_per_sm,
                             int ring_stages) {
  switch (ring_stages) {
    case 3: return launch_batched_ks<K, 3, VPL>(st, a, stream, blocks_per_sm);
    case 4:
      if constexpr (bt_ring_smem<4, VPL>() <= BT_RING_MAX_SMEM) return launch_batched_ks<K, 4, VPL>(st, a, stream, blocks_per_sm);
      return POSPOPCNT_ERR_INVALID;
    default: return launch_batched_ks<K, RING_STAGES, VPL>(st, a, stream, blocks_per_sm);
  }
}

// ring_stages: the per-warp ring depth, 2 (default, also for 0), 3 or 4;
// vpl: vectors per lane per trip, 4, 8 (default, also for 0) or 16 (16 with
// at most 3 stages).
template <int K>
static int launch_batched_k(const DeviceState& st, const BatchedArgs& a, cudaStream_t stream, int blocks_per_sm = 0,
                            int ring_stages = 0, int vpl = 0) {
  switch (vpl) {
    case 4: return launch_batched_kv<K, 4>(st, a, stream, blocks_per_sm, ring_stages);
    case 16: return launch_batched_kv<K, 16>(st, a, stream, blocks_per_sm, ring_stages);
    default: return launch_batched_kv<K, RING_VPL>(st, a, stream, blocks_per_sm, ring_stages);
  }
}

// Offsets check (checked batched form): offsets[0] >= 0, nondecreasing,
// offsets[nseg] <= n_words.  Any violation sets q->bad and the error word.
__global__ void offsets_check_kernel(const int64_t* offsets, uint64_t nseg, uint64_t n_words, QueueSlot* q,
                                     unsigned* err) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  bool bad = false;
  for (uint64_t s = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < nseg; s += stride)
    bad |= offsets[s] > offsets[s + 1];
  if (blockIdx.x == 0 && threadIdx.x == 0)
    bad |= offsets[0] < 0 || uint64_t(offsets[nseg]) > n_words || offsets[nseg] < 0;
  if (__any_sync(FULL_MASK, bad) && (threadIdx.x & 31) == 0) {
    atomicExch(&q->bad, 1u);
    atomicOr(err, ERR_BIT_BAD_OFFSETS);
  }
}

int launch_offsets_check(const DeviceState& st, const int64_t* d_offsets, size_t nseg, uint64_t n_words,
                         void* queue_slot, cudaStream_t stream) {
  QueueSlot* q = static_cast<QueueSlot*>(queue_slot);
  cudaError_t e = cudaMemsetAsync(&q->bad, 0, sizeof(unsigned), stream);
  if (e != cudaSuccess) return cuda_fail(e);
  const uint64_t blocks = std::min<uint64_t>((nseg + 255) / 256, uint64_t(st.sms) * 8);
  offsets_check_kernel<<<unsigned(std::max<uint64_t>(blocks, 1)), 256, 0, stream>>>(d_offsets, nseg, n_words, q,
                                                                                     st.d_err);
  note_launch();
  e = cudaGetLastError();
  return e == cudaSuccess ? POSPOPCNT_OK : cuda_fail(e);
}

int launch_batched(const DeviceState& st, const void* d_in, const int64_t* d_offsets, size_t nseg,
                   int width, unsigned long long* d_counts, void* queue_slot, int tile_words,
                   int blocks_per_sm, int ring_stages, int vpl, cudaStream_t stream) {
  BatchedArgs a;
  a.base = static_cast<const uint8_t*>(d_in);
  a.offsets = d_offsets;
  a.nseg = nseg;
  a.counts = d_counts;
  a.q = static_cast<QueueSlot*>(queue_slot);
  a.tile_words = uint64_t(tile_words);
  a.err = st.d_err;
  switch (width) {
    case 8: return launch_batched_k<8>(st, a, stream, blocks_per_sm, ring_stages, vpl);
    case 16: return launch_batched_k<16>(st, a, stream, blocks_per_sm, ring_stages, vpl);
    case 32: return launch_batched_k<32>(st, a, stream, blocks_per_sm, ring_stages, vpl);
  }
  return POSPOPCNT_ERR_INVALID;
}

}  // namespace ppc

// ---------------------------------------------------------------------------
// Allocation-free form of the batched count.
//
// Some callers cannot call cudaMalloc: a host process whose device memory
// is owned by another runtime's pool allocator (which must see every
// allocation), code that must not allocate once it has started (a
// latency-critical or memory-capped service), or an embedding that forbids
// third-party libraries from allocating at all.  pospopcnt_batched and the
// other entry points allocate the library workspace on their first call;
// pospopcnt_batched_noalloc never does.  The only scratch the batched
// kernel needs -- the work-queue state of one launch and the word where a
// bounded wait records that it gave up -- lives in the static array below,
// which every GPU that loads this library holds until the process exits.
//
// In host code g_noalloc_scratch names a host-side stand-in, not a device
// address: the device address is looked up with cudaGetSymbolAddress once
// per device (on that device's first call, with the device current) and
// passed to the kernel.

namespace ppc {

// What one launch of the allocation-free form keeps in the static array;
// every call clears all of it on its stream before launching.
struct NoallocScratch {
  QueueSlot q;   // work-queue state
  unsigned err;  // error bits of bounded waits (read by pospopcnt_check_device_error)
};

constexpr size_t NOALLOC_SCRATCH_BYTES = 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
int g_noalloc_sms[NOALLOC_MAX_DEVICES] = {};
}  // namespace

unsigned* noalloc_error_word(int device) {
  if (device < 0 || device >= NOALLOC_MAX_DEVICES) return nullptr;
  std::lock_guard<std::mutex> lk(g_noalloc_mutex);
  if (!g_noalloc_ptr[device]) return nullptr;
  return &static_cast<NoallocScratch*>(g_noalloc_ptr[device])->err;
}

}  // namespace ppc

extern "C" int pospopcnt_batched_noalloc(const void* d_in, const int64_t* d_offsets, size_t nseg, int width,
                                         uint64_t* d_counts, cudaStream_t stream) {
  using namespace ppc;
  if (width != 8 && width != 16 && width != 32) return POSPOPCNT_ERR_INVALID;
  if (nseg == 0) return POSPOPCNT_OK;
  if (!d_in || !d_offsets || !d_counts) return POSPOPCNT_ERR_INVALID;
  if (reinterpret_cast<uintptr_t>(d_in) % uintptr_t(width / 8) != 0) return POSPOPCNT_ERR_MISALIGNED;
  if (reinterpret_cast<uintptr_t>(d_offsets) % 8 != 0 || reinterpret_cast<uintptr_t>(d_counts) % 8 != 0)
    return POSPOPCNT_ERR_MISALIGNED;
  if (nseg > (size_t(1) << 40)) return POSPOPCNT_ERR_TOO_LARGE;
  // scratch one launch needs: fixed, independent of the input
  const size_t need = sizeof(NoallocScratch);
  if (need > NOALLOC_SCRATCH_BYTES) return POSPOPCNT_ERR_TOO_LARGE;

  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return POSPOPCNT_ERR_NOT_INITIALIZED;
  void* scratch = nullptr;
  int sms = 0;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {  // set-up, once per device, with that device current
      void* p = nullptr;
      if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess) return cuda_fail(e);
      int n = 0;
      if ((e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_fail(e);
      if (!p || n <= 0) return POSPOPCNT_ERR_NOT_INITIALIZED;
      g_noalloc_sms[dev] = n;
      g_noalloc_ptr[dev] = p;
    }
    scratch = g_noalloc_ptr[dev];
    sms = g_noalloc_sms[dev];
  }
  // The array keeps the previous call's contents: the queue state and the
  // error word must start at zero, and the rows are overwritten.
  if ((e = cudaMemsetAsync(scratch, 0, need, stream)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMemsetAsync(d_counts, 0, sizeof(uint64_t) * size_t(width) * nseg, stream)) != cudaSuccess)
    return cuda_fail(e);
  DeviceState st;
  st.sms = sms;
  st.device = dev;
  NoallocScratch* ns = static_cast<NoallocScratch*>(scratch);
  BatchedArgs a;
  a.base = static_cast<const uint8_t*>(d_in);
  a.offsets = d_offsets;
  a.nseg = nseg;
  a.counts = reinterpret_cast<unsigned long long*>(d_counts);
  a.q = &ns->q;
  a.tile_words = uint64_t((16 * 1024) / (width / 8));
  a.err = &ns->err;
  switch (width) {
    case 8: return launch_batched_k<8>(st, a, stream);
    case 16: return launch_batched_k<16>(st, a, stream);
    default: return launch_batched_k<32>(st, a, stream);
  }
}
