// Single-stream pospopcnt kernels and their host launcher, templated on the
// word width K (8, 16, 32).  Each width is instantiated in its own
// translation unit (plain_w8.cu, plain_w16.cu, plain_w32.cu).
//
//   csa_kernel    128-bit coalesced loads straight into registers, grid-stride,
//                 `U` vectors per thread per trip = one circuit F_L over
//                 4U registers (L = log2 4U), popc flush per trip.
//   tma_kernel    persistent CTAs; one producer lane streams fixed-size chunks
//                 with cp.async.bulk into an S-stage shared-memory ring guarded
//                 by full/empty mbarriers; 8 consumer warps run F_4 over the
//                 chunk from shared memory.  Every wait is bounded.
//   ballot_kernel bit transpose by __ballot_sync: for each of the 32 bits of a
//                 lane register, the warp's vote mask is popc'ed into the
//                 counter of that bit's position (comparison kernel).
//
// All three count the unaligned head and the ragged tail word by word in
// block 0 and finish with one 64-bit atomic add per position per block.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace ppc {

struct PlainArgs {
  const uint4* body;      // 16-byte aligned vectors
  uint64_t nvec;          // number of vectors
  const uint8_t* head;    // first head word
  uint32_t head_words;
  const uint8_t* tail;    // first tail word
  uint32_t tail_words;
  unsigned long long* counts;
  unsigned* err;
  uint32_t store;  // 1: single-CTA grid writes the counts (no memset, no atomics)
  uint32_t publish;          // 1: blocks add into acc; the last one writes the counts
  unsigned long long* acc;   // the stream's accumulator (publish), zero between launches
  unsigned* arrived;         // blocks that have added into acc (publish)
};

// The block's counts c[0..KC) of positions [base, base + KC): added into
// the counts (or the stream's accumulator), or stored by a one-CTA grid.
template <int KC, int NWARPS>
__device__ __forceinline__ void plain_reduce(uint32_t (&c)[KC], const PlainArgs& a, int base = 0) {
  block_reduce_add<KC, NWARPS>(c, (a.publish ? a.acc : a.counts) + base, a.store != 0);
}

template <int K, int NTHREADS>
__device__ __forceinline__ void count_head_tail(uint32_t (&c)[K], const PlainArgs& a) {
  static_assert(NTHREADS >= 64, "head/tail lanes need two warps");
  if (blockIdx.x != 0) return;
  const unsigned t = threadIdx.x;
  constexpr int WB = word_bytes<K>::value;
  if (t < a.head_words) count_word<K>(c, load_word<K>(a.head + t * WB));
  if (t >= 32 && t - 32 < a.tail_words) count_word<K>(c, load_word<K>(a.tail + (t - 32) * WB));
}

// ---------------------------------------------------------------------------
// SYSMEM: the input is pinned host memory mapped into the device's address
// space; it is read with plain coherent loads instead of the read-only path.
template <int K, int U, int NTHREADS, bool SYSMEM = false>
__global__ void __launch_bounds__(NTHREADS) csa_kernel(PlainArgs a) {
  constexpr int R = 4 * U;
  constexpr int L = ilog2<R>::value;
  uint32_t B[L];
#pragma unroll
  for (int l = 0; l < L; ++l) B[l] = 0;
  uint32_t top[K];
#pragma unroll
  for (int p = 0; p < K; ++p) top[p] = 0;

  const uint64_t stride = uint64_t(gridDim.x) * NTHREADS;
  uint64_t v = uint64_t(blockIdx.x) * NTHREADS + threadIdx.x;
  const uint64_t reach = uint64_t(U - 1) * stride;
  const uint64_t full_end = a.nvec > reach ? a.nvec - reach : 0;
  for (; v < full_end; v += U * stride) {
    uint32_t d[R];
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const uint4 x = SYSMEM ? ld_coherent(a.body + v + i * stride) : ld_stream(a.body + v + i * stride);
      d[4 * i + 0] = x.x, d[4 * i + 1] = x.y, d[4 * i + 2] = x.z, d[4 * i + 3] = x.w;
    }
    flush<K>(top, Circuit<L>::run(d, B));
  }
  if (v < a.nvec) {  // last, partial trip: missing vectors read as zero
    uint32_t d[R];
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const uint64_t idx = v + i * stride;
      const uint4 x = idx < a.nvec ? (SYSMEM ? ld_coherent(a.body + idx) : ld_stream(a.body + idx))
                                   : make_uint4(0, 0, 0, 0);
      d[4 * i + 0] = x.x, d[4 * i + 1] = x.y, d[4 * i + 2] = x.z, d[4 * i + 3] = x.w;
    }
    flush<K>(top, Circuit<L>::run(d, B));
  }
  uint32_t c[K];
  finalize<K, L>(c, top, B);
  count_head_tail<K, NTHREADS>(c, a);
  plain_reduce<K, NTHREADS / 32>(c, a);
  if (a.publish) block_publish(a.acc, a.arrived, a.counts, K);
}

// ---------------------------------------------------------------------------
constexpr int TMA_CWARPS = 8;                       // consumer warps
constexpr int TMA_THREADS = (TMA_CWARPS + 1) * 32;  // + one producer warp
constexpr int TMA_MAX_STAGES = 16;
constexpr int TMA_CHUNK_QUANTUM = 4 * TMA_CWARPS * 32 * 16;  // one F_4 per consumer thread

struct TmaArgs {
  PlainArgs p;
  const uint8_t* body_bytes_ptr;
  uint64_t body_bytes;  // multiple of 16
  uint32_t chunk_bytes;  // multiple of TMA_CHUNK_QUANTUM
  uint32_t stages;
  uint32_t evict_first;  // L2 evict-first hint on the bulk copies
};

// Register classes of the TMA consumers: for K <= 32 every 32-bit register
// of a vector holds all K positions; for 64-bit words registers alternate
// between positions 0..31 (x, z) and 32..63 (y, w), one circuit per class.
template <int K>
struct tma_shape {
  static constexpr int NC = K == 64 ? 2 : 1;        // register classes
  static constexpr int KC = K == 64 ? 32 : K;       // positions per class
  static constexpr int VPT = K == 64 ? 8 : 4;       // 16-byte vectors per thread per trip
  static constexpr int RC = 4 * VPT / NC;           // registers per class per trip
  static constexpr int L = ilog2<RC>::value;        // circuit depth per class
};

template <int K>
__global__ void __launch_bounds__(TMA_THREADS) tma_kernel(TmaArgs a) {
  using S = tma_shape<K>;
  constexpr int NC = S::NC, KC = S::KC, VPT = S::VPT, RC = S::RC, L = S::L;
  extern __shared__ __align__(128) uint8_t ring[];
  __shared__ __align__(8) uint64_t full[TMA_MAX_STAGES];
  __shared__ __align__(8) uint64_t empty[TMA_MAX_STAGES];
  __shared__ uint32_t s_issued;              // chunks the producer issued
  __shared__ uint32_t s_consumed[TMA_CWARPS];  // chunks each consumer warp finished
  __shared__ uint32_t s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t S_ = a.stages;
  const uint64_t nchunks = (a.body_bytes + a.chunk_bytes - 1) / a.chunk_bytes;
  const uint32_t my_chunks =
      blockIdx.x < nchunks ? uint32_t((nchunks - 1 - blockIdx.x) / gridDim.x + 1) : 0u;

  if (threadIdx.x == 0) {
    for (uint32_t s = 0; s < S_; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], TMA_CWARPS);
    }
    s_issued = 0;
    s_abort = 0;
    mbar_fence_init();
  }
  __syncthreads();

  uint32_t c[NC][KC];
#pragma unroll
  for (int q = 0; q < NC; ++q)
#pragma unroll
    for (int p = 0; p < KC; ++p) c[q][p] = 0;

  if (warp == TMA_CWARPS) {
    // producer: one lane issues every copy
    if (lane == 0) {
      const uint64_t policy = a.evict_first ? l2_policy_evict_first() : 0;
      uint32_t i = 0;
      for (; i < my_chunks; ++i) {
        const uint32_t s = i % S_, use = i / S_;
        if (use > 0 && !mbar_wait_bounded(&empty[s], (use - 1) & 1u, WAIT_LIMIT_NS)) {
          atomicOr(a.p.err, ERR_BIT_TIMEOUT_EMPTY);
          atomicExch(&s_abort, 1u);
          break;
        }
        if (*((volatile uint32_t*)&s_abort)) break;
        const uint64_t chunk = blockIdx.x + uint64_t(i) * gridDim.x;
        const uint64_t off = chunk * a.chunk_bytes;
        const uint64_t rem = a.body_bytes - off;
        const uint32_t bytes = rem < a.chunk_bytes ? uint32_t(rem) : a.chunk_bytes;
        mbar_arrive_expect_tx(&full[s], bytes);
        if (a.evict_first)
          bulk_g2s_hint(ring + size_t(s) * a.chunk_bytes, a.body_bytes_ptr + off, bytes, &full[s], policy);
        else
          bulk_g2s(ring + size_t(s) * a.chunk_bytes, a.body_bytes_ptr + off, bytes, &full[s]);
      }
      s_issued = i;
    }
  } else {
    // consumers
    constexpr int CT = TMA_CWARPS * 32;
    uint32_t B[NC][L];
    uint32_t top[NC][KC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
#pragma unroll
      for (int l = 0; l < L; ++l) B[q][l] = 0;
#pragma unroll
      for (int p = 0; p < KC; ++p) top[q][p] = 0;
    }
    uint32_t i = 0;
    for (; i < my_chunks; ++i) {
      const uint32_t s = i % S_, use = i / S_;
      // every lane waits (each acquires the copied bytes); the verdict is
      // made warp-uniform so the warp leaves the loop together
      const bool ok = __all_sync(FULL_MASK, mbar_wait_bounded(&full[s], use & 1u, WAIT_LIMIT_NS));
      if (!ok) {
        if (lane == 0) {
          atomicOr(a.p.err, ERR_BIT_TIMEOUT_FULL);
          atomicExch(&s_abort, 1u);
        }
        break;
      }
      const uint64_t chunk = blockIdx.x + uint64_t(i) * gridDim.x;
      const uint64_t off = chunk * a.chunk_bytes;
      const uint64_t rem = a.body_bytes - off;
      const uint32_t nv = (rem < a.chunk_bytes ? uint32_t(rem) : a.chunk_bytes) / 16u;
      const uint4* sv = reinterpret_cast<const uint4*>(ring + size_t(s) * a.chunk_bytes);
      for (uint32_t base = 0; base < nv; base += VPT * CT) {
        uint32_t d[NC][RC];
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
          const uint32_t idx = base + j * CT + threadIdx.x;
          const uint4 x = idx < nv ? sv[idx] : make_uint4(0, 0, 0, 0);
          const uint32_t r[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) d[q % NC][(4 * j + q) / NC] = r[q];
        }
#pragma unroll
        for (int q = 0; q < NC; ++q) flush<KC>(top[q], Circuit<L>::run(d[q], B[q]));
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
      if (__any_sync(FULL_MASK, *((volatile uint32_t*)&s_abort) != 0u)) {
        ++i;
        break;
      }
    }
    if (lane == 0) s_consumed[warp] = i;
#pragma unroll
    for (int q = 0; q < NC; ++q) finalize<KC, L>(c[q], top[q], B[q]);
  }
  __syncthreads();
  // After an abort, wait (bounded) for copies still in flight before the
  // shared memory they target goes away.
  if (s_abort && threadIdx.x == 0) {
    uint32_t lo = s_issued;
    for (int w = 0; w < TMA_CWARPS; ++w) lo = s_consumed[w] < lo ? s_consumed[w] : lo;
    for (uint32_t i = lo; i < s_issued; ++i) {
      if (!mbar_wait_bounded(&full[i % S_], (i / S_) & 1u, WAIT_LIMIT_NS)) {
        atomicOr(a.p.err, ERR_BIT_TIMEOUT_DRAIN);
        break;
      }
    }
  }
  if constexpr (K == 64) {
    if (blockIdx.x == 0) {
      if (threadIdx.x < a.p.head_words) count_word64(c[0], c[1], a.p.head + threadIdx.x * 8);
      if (threadIdx.x >= 32 && threadIdx.x - 32 < a.p.tail_words)
        count_word64(c[0], c[1], a.p.tail + (threadIdx.x - 32) * 8);
    }
  } else {
    count_head_tail<K, TMA_THREADS>(c[0], a.p);
  }
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    if (q) __syncthreads();  // the reduction's shared buffer is reused
    plain_reduce<KC, TMA_CWARPS + 1>(c[q], a.p, 32 * q);
  }
  if (a.p.publish) block_publish(a.p.acc, a.p.arrived, a.p.counts, K);
}

// ---------------------------------------------------------------------------
template <int K, int U, int NTHREADS>
__global__ void __launch_bounds__(NTHREADS) ballot_kernel(PlainArgs a) {
  uint32_t acc[K];
#pragma unroll
  for (int p = 0; p < K; ++p) acc[p] = 0;
  const int lane = threadIdx.x & 31;
  const uint64_t gw = (uint64_t(blockIdx.x) * NTHREADS + threadIdx.x) >> 5;
  const uint64_t nw = uint64_t(gridDim.x) * (NTHREADS / 32);
  for (uint64_t base = gw * 32 * U; base < a.nvec; base += nw * 32 * U) {  // warp-uniform
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const uint64_t idx = base + uint64_t(i) * 32 + lane;
      const uint4 x = idx < a.nvec ? ld_stream(a.body + idx) : make_uint4(0, 0, 0, 0);
      const uint32_t r[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int b = 0; b < 32; ++b) acc[b & (K - 1)] += __popc(__ballot_sync(FULL_MASK, (r[q] >> b) & 1u));
      }
    }
  }
  uint32_t c[K];
#pragma unroll
  for (int p = 0; p < K; ++p) c[p] = lane == 0 ? acc[p] : 0u;  // every lane holds the warp total
  count_head_tail<K, NTHREADS>(c, a);
  plain_reduce<K, NTHREADS / 32>(c, a);
  if (a.publish) block_publish(a.acc, a.arrived, a.counts, K);
}

// ---------------------------------------------------------------------------
// 64-bit words (wider words as two 32-bit streams, §4): in a 16-byte vector
// of two words the registers x, z hold positions 0..31 and y, w hold
// positions 32..63, so each thread runs one carry-save circuit per class
// (F_L over 2U registers each) and flushes each like a 32-bit stream.
template <int U, int NTHREADS>
__global__ void __launch_bounds__(NTHREADS) csa64_kernel(PlainArgs a) {
  constexpr int H = 2 * U;  // registers per class per trip
  constexpr int L = ilog2<H>::value;
  uint32_t Blo[L], Bhi[L];
#pragma unroll
  for (int l = 0; l < L; ++l) Blo[l] = 0, Bhi[l] = 0;
  uint32_t tlo[32], thi[32];
#pragma unroll
  for (int p = 0; p < 32; ++p) tlo[p] = 0, thi[p] = 0;
  const uint64_t stride = uint64_t(gridDim.x) * NTHREADS;
  uint64_t v = uint64_t(blockIdx.x) * NTHREADS + threadIdx.x;
  for (; v < a.nvec; v += U * stride) {  // every trip predicated: U loads, missing ones zero
    uint32_t dlo[H], dhi[H];
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const uint64_t idx = v + i * stride;
      const uint4 x = idx < a.nvec ? ld_stream(a.body + idx) : make_uint4(0, 0, 0, 0);
      dlo[2 * i] = x.x, dhi[2 * i] = x.y, dlo[2 * i + 1] = x.z, dhi[2 * i + 1] = x.w;
    }
    flush<32>(tlo, Circuit<L>::run(dlo, Blo));
    flush<32>(thi, Circuit<L>::run(dhi, Bhi));
  }
  uint32_t clo[32], chi[32];
  finalize<32, L>(clo, tlo, Blo);
  finalize<32, L>(chi, thi, Bhi);
  if (blockIdx.x == 0) {  // head and tail words (at most one each: 8-byte words, 16-byte vectors)
    if (threadIdx.x < a.head_words) count_word64(clo, chi, a.head + threadIdx.x * 8);
    if (threadIdx.x >= 32 && threadIdx.x - 32 < a.tail_words) count_word64(clo, chi, a.tail + (threadIdx.x - 32) * 8);
  }
  plain_reduce<32, NTHREADS / 32>(clo, a);
  __syncthreads();  // the reduction's shared buffer is reused
  plain_reduce<32, NTHREADS / 32>(chi, a, 32);
  if (a.publish) block_publish(a.acc, a.arrived, a.counts, 64);
}

// ---------------------------------------------------------------------------
// Host launcher for width K.

template <typename Kern>
static int occupancy(const DeviceState& st, Kern kern, int threads, size_t smem) {
  return resident_blocks(reinterpret_cast<const void*>(kern), st.device, threads, smem);
}

// Smallest grid whose per-thread, per-warp and per-block u32 partial counts
// stay exact.  A byte adds at most 8 to the one counter of the array
// popcount (K = 1) and at most 1 to any position's count otherwise, so a
// block whose share of the input holds at most 2^31 counts per position
// cannot wrap a u32 partial.  Every family gives a block at most
// nbytes / grid bytes plus one unit of work (a trip of vectors, a chunk of
// at most 192 KiB), so with grid >= this value a block's count stays below
// 2^31 + 8 x 192 Ki < 2^32.
template <int K>
static inline uint64_t min_blocks_for(uint64_t nbytes) {
  constexpr uint64_t per_byte = K == 1 ? 8 : 1;
  return ((nbytes * per_byte) >> 31) + 1;
}

// Overwrite semantics: a one-CTA grid stores its counts; a larger grid adds
// into the stream's accumulator and its last block publishes them (when the
// caller passed one), else adds atomically into counts zeroed first by a
// stream-ordered memset.
template <int K>
static int prepare_counts(PlainArgs& a, uint64_t grid, bool zero_first, cudaStream_t stream) {
  a.store = (zero_first && grid == 1) ? 1u : 0u;
  a.publish = (zero_first && grid > 1 && a.acc && a.arrived) ? 1u : 0u;
  if (zero_first && grid > 1 && !a.publish) {
    const cudaError_t e = cudaMemsetAsync(a.counts, 0, sizeof(unsigned long long) * K, stream);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return POSPOPCNT_OK;
}

template <int K, int U, int T, bool SYSMEM = false>
static int launch_csa(const DeviceState& st, PlainArgs a, int bps, bool zero_first, cudaStream_t stream) {
  auto kern = csa_kernel<K, U, T, SYSMEM>;
  const int occ = occupancy(st, kern, T, 0);
  const uint64_t cap = uint64_t(st.sms) * uint64_t(std::min(bps > 0 ? bps : occ, occ));
  const uint64_t need = (a.nvec + uint64_t(U) * T - 1) / (uint64_t(U) * T);
  uint64_t grid = std::max<uint64_t>(1, std::min(cap, need));
  grid = std::max(grid, min_blocks_for<K>(a.nvec * 16));
  if (const int rc = prepare_counts<K>(a, grid, zero_first, stream)) return rc;
  kern<<<unsigned(grid), T, 0, stream>>>(a);
  note_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? POSPOPCNT_OK : cuda_fail(e);
}

template <int K, int U, int T>
static int launch_ballot(const DeviceState& st, PlainArgs a, int bps, bool zero_first, cudaStream_t stream) {
  auto kern = ballot_kernel<K, U, T>;
  const int occ = occupancy(st, kern, T, 0);
  const uint64_t cap = uint64_t(st.sms) * uint64_t(std::min(bps > 0 ? bps : occ, occ));
  const uint64_t per = uint64_t(32) * U * (T / 32);
  const uint64_t need = (a.nvec + per - 1) / per;
  uint64_t grid = std::max<uint64_t>(1, std::min(cap, need));
  grid = std::max(grid, min_blocks_for<K>(a.nvec * 16));
  if (const int rc = prepare_counts<K>(a, grid, zero_first, stream)) return rc;
  kern<<<unsigned(grid), T, 0, stream>>>(a);
  note_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? POSPOPCNT_OK : cuda_fail(e);
}

template <int K>
static int launch_tma(const DeviceState& st, const PlainArgs& p, int bps, int stages, int chunk, bool zero_first,
                      cudaStream_t stream, int flags = 0) {
  auto kern = tma_kernel<K>;
  const size_t smem = size_t(stages) * size_t(chunk);
  if (const cudaError_t e = ensure_dynamic_smem<tma_kernel<K>>(st.device, int(smem))) return cuda_fail(e);
  TmaArgs a;
  a.p = p;
  a.body_bytes_ptr = reinterpret_cast<const uint8_t*>(p.body);
  a.body_bytes = p.nvec * 16;
  a.chunk_bytes = uint32_t(chunk);
  a.stages = uint32_t(stages);
  a.evict_first = (flags & POSPOPCNT_FLAG_EVICT_FIRST) ? 1u : 0u;
  const int occ = occupancy(st, kern, TMA_THREADS, smem);
  const uint64_t cap = uint64_t(st.sms) * uint64_t(std::min(bps > 0 ? bps : occ, occ));
  const uint64_t nchunks = (a.body_bytes + chunk - 1) / chunk;
  uint64_t grid = std::max<uint64_t>(1, std::min(cap, nchunks));
  grid = std::max(grid, std::min<uint64_t>(nchunks, min_blocks_for<K>(a.body_bytes)));
  if (const int rc = prepare_counts<K>(a.p, grid, zero_first, stream)) return rc;
  kern<<<unsigned(grid), TMA_THREADS, smem, stream>>>(a);
  note_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? POSPOPCNT_OK : cuda_fail(e);
}

template <int K, int T>
static int launch_csa_u(const DeviceState& st, const PlainArgs& a, const pospopcnt_config& cfg, bool zero_first,
                        cudaStream_t stream) {
  switch (cfg.unroll) {
    case 2: return launch_csa<K, 2, T>(st, a, cfg.blocks_per_sm, zero_first, stream);
    case 4: return launch_csa<K, 4, T>(st, a, cfg.blocks_per_sm, zero_first, stream);
    case 8: return launch_csa<K, 8, T>(st, a, cfg.blocks_per_sm, zero_first, stream);
  }
  return POSPOPCNT_ERR_INVALID;
}

template <int K>
static PlainArgs make_args(const DeviceState& st, const void* d_in, size_t n, unsigned long long* d_counts,
                           const PlainAcc& acc = PlainAcc{}) {
  constexpr int WB = word_bytes<K>::value;
  const Split sp = plan_split(8 * WB, reinterpret_cast<uint64_t>(d_in), n);
  const uint8_t* base = static_cast<const uint8_t*>(d_in);
  PlainArgs a;
  a.head = base;
  a.head_words = uint32_t(sp.head_words);
  a.body = reinterpret_cast<const uint4*>(base + sp.head_words * WB);
  a.nvec = sp.body_vectors;
  a.tail = base + sp.head_words * WB + sp.body_vectors * 16;
  a.tail_words = uint32_t(sp.tail_words);
  a.counts = d_counts;
  a.err = st.d_err;
  a.store = 0;
  a.publish = 0;
  a.acc = acc.acc;
  a.arrived = acc.arrived;
  return a;
}

// Count of words in pinned host memory mapped into the device address space
// (d_in is its device address); adds into d_counts.
template <int K>
int launch_plain_sysmem_k(const DeviceState& st, const void* d_in, size_t n, unsigned long long* d_counts,
                          cudaStream_t stream) {
  PlainArgs a = make_args<K>(st, d_in, n, d_counts);
  if (a.nvec == 0 && a.head_words == 0 && a.tail_words == 0) return POSPOPCNT_OK;
  return launch_csa<K, 4, 256, true>(st, a, 0, false, stream);
}

template <int U, int T>
static int launch_csa64(const DeviceState& st, PlainArgs a, int bps, bool zero_first, cudaStream_t stream) {
  auto kern = csa64_kernel<U, T>;
  const int occ = occupancy(st, kern, T, 0);
  const uint64_t cap = uint64_t(st.sms) * uint64_t(std::min(bps > 0 ? bps : occ, occ));
  const uint64_t need = (a.nvec + uint64_t(U) * T - 1) / (uint64_t(U) * T);
  uint64_t grid = std::max<uint64_t>(1, std::min(cap, need));
  grid = std::max(grid, min_blocks_for<64>(a.nvec * 16));
  if (const int rc = prepare_counts<64>(a, grid, zero_first, stream)) return rc;
  kern<<<unsigned(grid), T, 0, stream>>>(a);
  note_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? POSPOPCNT_OK : cuda_fail(e);
}

template <int K>
int launch_plain_k(const DeviceState& st, const pospopcnt_config& cfg, const void* d_in, size_t n,
                   unsigned long long* d_counts, bool zero_first, cudaStream_t stream, const PlainAcc& acc) {
  PlainArgs a = make_args<K>(st, d_in, n, d_counts, acc);
  if (a.nvec == 0 && a.head_words == 0 && a.tail_words == 0) {
    if (!zero_first) return POSPOPCNT_OK;
    const cudaError_t e = cudaMemsetAsync(d_counts, 0, sizeof(unsigned long long) * K, stream);
    return e == cudaSuccess ? POSPOPCNT_OK : cuda_fail(e);
  }
  if constexpr (K == 64) {  // 64-bit words: the CSA and TMA families
    if (cfg.kernel == POSPOPCNT_KERNEL_TMA) {
      if (a.nvec == 0) return launch_csa64<4, 256>(st, a, 1, zero_first, stream);  // head/tail only
      return launch_tma<K>(st, a, cfg.blocks_per_sm, cfg.stages, cfg.chunk_bytes, zero_first, stream, cfg.flags);
    }
    switch (cfg.threads) {
      case 128: return cfg.unroll == 8 ? launch_csa64<8, 128>(st, a, cfg.blocks_per_sm, zero_first, stream)
                                       : launch_csa64<4, 128>(st, a, cfg.blocks_per_sm, zero_first, stream);
      case 256: return cfg.unroll == 8 ? launch_csa64<8, 256>(st, a, cfg.blocks_per_sm, zero_first, stream)
                                       : launch_csa64<4, 256>(st, a, cfg.blocks_per_sm, zero_first, stream);
    }
    return POSPOPCNT_ERR_INVALID;
  } else {
  switch (cfg.kernel) {
    case POSPOPCNT_KERNEL_CSA:
      switch (cfg.threads) {
        case 128: return launch_csa_u<K, 128>(st, a, cfg, zero_first, stream);
        case 256: return launch_csa_u<K, 256>(st, a, cfg, zero_first, stream);
        case 512: return launch_csa_u<K, 512>(st, a, cfg, zero_first, stream);
      }
      return POSPOPCNT_ERR_INVALID;
    case POSPOPCNT_KERNEL_TMA:
      if (a.nvec == 0) return launch_csa<K, 4, 256>(st, a, 1, zero_first, stream);  // head/tail only
      return launch_tma<K>(st, a, cfg.blocks_per_sm, cfg.stages, cfg.chunk_bytes, zero_first, stream, cfg.flags);
    case POSPOPCNT_KERNEL_BALLOT:
      switch (cfg.unroll) {
        case 1: return launch_ballot<K, 1, 256>(st, a, cfg.blocks_per_sm, zero_first, stream);
        case 2: return launch_ballot<K, 2, 256>(st, a, cfg.blocks_per_sm, zero_first, stream);
        case 4: return launch_ballot<K, 4, 256>(st, a, cfg.blocks_per_sm, zero_first, stream);
      }
      return POSPOPCNT_ERR_INVALID;
  }
  return POSPOPCNT_ERR_INVALID;
  }
}

}  // namespace ppc
