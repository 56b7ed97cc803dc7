// Segment helpers shared by the batched and serving kernels: the 32-way
// search for the segment holding a word, and the warp-wide count of one
// piece (a segment's words inside a warp's sub-range).
#pragma once

#include <cstdint>

#include "device_common.cuh"

namespace ppc {

// Work-queue state of one persistent launch (128-byte slot).
struct QueueSlot {
  unsigned long long next;  // next tile index to hand out
  unsigned int done;        // CTAs that have finished
  unsigned int bad;         // set by the offsets check: the launch counts nothing
};

constexpr int BT_THREADS = 256;
constexpr int BT_WARPS = BT_THREADS / 32;
// resident CTAs per SM the segment kernels are compiled for (register cap
// 65536 / (256 x this))
template <int K>
struct bt_min_blocks {
  static constexpr int value = K == 32 ? 3 : 5;
};
// the batched kernel's trips carry 8 vectors per lane: fewer, fuller warps
constexpr int BT_VPL = 8;
template <int K>
struct bt_batched_min_blocks {
  static constexpr int value = K == 32 ? 2 : 3;
};

// Pops the next tile index for the CTA (every thread gets it).
__device__ __forceinline__ uint64_t pop_tile(QueueSlot* q) {
  __shared__ unsigned long long s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(&q->next, 1ull);
  __syncthreads();
  const uint64_t tile = s_tile;
  __syncthreads();
  return tile;
}

// Called by every thread after its last pop: the last CTA out resets the
// queue slot for the next launch.
__device__ __forceinline__ void retire_cta(QueueSlot* q) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&q->done, 1u);
    if (prev == gridDim.x - 1) {
      atomicExch(&q->next, 0ull);
      atomicExch(&q->done, 0u);
      atomicExch(&q->bad, 0u);
      __threadfence();
    }
  }
}

// Largest s in [0, nseg) with bounds[s] <= w (requires bounds[0] <= w <
// bounds[nseg]).  Each round the 32 lanes probe 32 evenly spaced candidates.
__device__ __forceinline__ uint64_t find_segment(const int64_t* bounds, uint64_t nseg, int64_t w) {
  const int lane = threadIdx.x & 31;
  uint64_t lo = 0, hi = nseg - 1;  // answer in [lo, hi]
  while (hi > lo) {
    const uint64_t span = hi - lo + 1;
    const uint64_t step = (span + 31) / 32;
    const uint64_t idx = lo + uint64_t(lane) * step;
    const bool le = idx <= hi && bounds[idx] <= w;
    const unsigned m = __ballot_sync(FULL_MASK, le);  // lane 0 always true
    const int j = 31 - __clz(m);
    lo = lo + uint64_t(j) * step;
    const uint64_t nhi = lo + step - 1;
    hi = nhi < hi ? nhi : hi;
    if (step == 1) break;
  }
  return lo;
}

// Counts words [pa, pb) of `base` with the whole warp: the unaligned head
// and ragged tail word by word, the 16-byte body in trips of VPL vectors per
// lane through F_{log2 4 VPL} with popc flushes.  Returns, in lanes with
// (lane & (2^(5 - log2 K) - 1)) == 0, the warp total of position
// lane >> (5 - log2 K); other lanes return partials.
template <int K, int VPL = 4>
__device__ __forceinline__ uint32_t warp_piece_counts(const uint8_t* base, uint64_t pa, uint64_t pb) {
  constexpr int R = 4 * VPL;
  constexpr int L = ilog2<R>::value;
  constexpr int WB = K / 8;
  const int lane = threadIdx.x & 31;
  const uint64_t A = reinterpret_cast<uint64_t>(base) + pa * WB;
  const uint64_t E = reinterpret_cast<uint64_t>(base) + pb * WB;
  uint64_t bodyA = (A + 15) & ~uint64_t(15);
  if (bodyA > E) bodyA = E;
  uint64_t bodyE = E & ~uint64_t(15);
  if (bodyE < bodyA) bodyE = bodyA;
  const uint64_t nvec = (bodyE - bodyA) / 16;
  // lanes 0..14 take the head words, lanes 16..30 the tail words (<= 15 each);
  // loaded before the body loop so only this word stays live across it
  const uint32_t head_words = uint32_t((bodyA - A) / WB);
  const uint32_t tail_words = uint32_t((E - bodyE) / WB);
  uint32_t edge = 0;
  if (uint32_t(lane) < head_words)
    edge = load_word<K>(reinterpret_cast<const uint8_t*>(A) + lane * WB);
  else if (lane >= 16 && uint32_t(lane - 16) < tail_words)
    edge = load_word<K>(reinterpret_cast<const uint8_t*>(bodyE) + (lane - 16) * WB);

  uint32_t B[L];
#pragma unroll
  for (int l = 0; l < L; ++l) B[l] = 0;
  uint32_t top[K];
#pragma unroll
  for (int p = 0; p < K; ++p) top[p] = 0;
  const uint4* vp = reinterpret_cast<const uint4*>(bodyA);
  for (uint64_t bv = 0; bv < nvec; bv += 32 * VPL) {  // 32 lanes x VPL vectors per trip
    uint32_t d[R];
#pragma unroll
    for (int j = 0; j < VPL; ++j) {
      const uint64_t idx = bv + uint64_t(j) * 32 + lane;
      const uint4 x = idx < nvec ? ld_stream(vp + idx) : make_uint4(0, 0, 0, 0);
      d[4 * j + 0] = x.x, d[4 * j + 1] = x.y, d[4 * j + 2] = x.z, d[4 * j + 3] = x.w;
    }
    flush<K>(top, Circuit<L>::run(d, B));
  }
  uint32_t c[K];
  finalize<K, L>(c, top, B);
  count_word<K>(c, edge);
  return warp_reduce_positions<K>(c);
}

}  // namespace ppc
