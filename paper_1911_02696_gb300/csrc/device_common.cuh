// Device building blocks shared by the pospopcnt kernels (sm_103a).
//
// The arithmetic follows the paper's method (arXiv 1911.02696) mapped onto
// a GPU thread: a 32-bit register holds 32/k words of k bits side by side,
// so bit j of the register belongs to word position j mod k.  A thread feeds
// 2^L such registers through the Harley-Seal carry-save circuit F_L (§2,
// built recursively from two F_{L-1} and one more CSA), keeping the running
// bit-sliced sums B_0..B_{L-1} in registers, and flushes the top register
// B_L (weight 2^L, §4.1) into k positional counters with popc.  The weight
// 2^L is applied once at the end (the deferred multiplication of §4.1), and
// B_0..B_{L-1} are flushed there with weights 2^l.
#pragma once

#include <cstdint>

namespace ppc {

constexpr unsigned FULL_MASK = 0xFFFFFFFFu;

template <int X>
struct ilog2 {
  static constexpr int value = 1 + ilog2<X / 2>::value;
};
template <>
struct ilog2<1> {
  static constexpr int value = 0;
};

// Bit 0 of every k-bit lane of a 32-bit register; shifted left by p it
// selects word position p in every lane.
template <int K>
struct lane_mask;
template <>
struct lane_mask<1> {  // K = 1: the array popcount, every bit is position 0
  static constexpr uint32_t value = 0xFFFFFFFFu;
};
template <>
struct lane_mask<8> {
  static constexpr uint32_t value = 0x01010101u;
};
template <>
struct lane_mask<16> {
  static constexpr uint32_t value = 0x00010001u;
};
template <>
struct lane_mask<32> {
  static constexpr uint32_t value = 0x00000001u;
};

// ---- carry-save adder: two three-input logic ops -------------------------
// h = majority(a, b, c) and l = a ^ b ^ c (§2, Fig. 3).  The lop3 immediates
// are those of §3 / Table 2: 0xE8 for the carry, 0x96 for the sum.
__device__ __forceinline__ void csa(uint32_t& h, uint32_t& l, uint32_t a, uint32_t b,
                                    uint32_t c) {
  uint32_t hh, ll;
  asm("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(hh) : "r"(a), "r"(b), "r"(c));
  asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(ll) : "r"(a), "r"(b), "r"(c));
  h = hh;
  l = ll;
}

// F_N over d[0 .. 2^N): updates B[0..N-1] in place and returns the new top
// register (weight 2^N).  Fully unrolled at compile time; all in registers.
template <int N>
struct Circuit {
  __device__ __forceinline__ static uint32_t run(const uint32_t* d, uint32_t* B) {
    const uint32_t x = Circuit<N - 1>::run(d, B);
    const uint32_t y = Circuit<N - 1>::run(d + (1 << (N - 1)), B);
    uint32_t h;
    csa(h, B[N - 1], B[N - 1], x, y);
    return h;
  }
};
template <>
struct Circuit<1> {
  __device__ __forceinline__ static uint32_t run(const uint32_t* d, uint32_t* B) {
    uint32_t h;
    csa(h, B[0], B[0], d[0], d[1]);
    return h;
  }
};

// top[p] += number of bits at word position p in register t.
template <int K>
__device__ __forceinline__ void flush(uint32_t (&top)[K], uint32_t t) {
#pragma unroll
  for (int p = 0; p < K; ++p) top[p] += __popc(t & (lane_mask<K>::value << p));
}

// Final per-thread counts: c[p] = top[p] * 2^L + sum_l popc(B_l & M_p) * 2^l.
template <int K, int L>
__device__ __forceinline__ void finalize(uint32_t (&c)[K], const uint32_t (&top)[K],
                                         const uint32_t* B) {
#pragma unroll
  for (int p = 0; p < K; ++p) c[p] = top[p] << L;
#pragma unroll
  for (int l = 0; l < L; ++l) {
#pragma unroll
    for (int p = 0; p < K; ++p) c[p] += static_cast<uint32_t>(__popc(B[l] & (lane_mask<K>::value << p))) << l;
  }
}

// Bytes per word (K = 1, the array popcount, walks its head and tail byte
// by byte).
template <int K>
struct word_bytes {
  static constexpr int value = K == 1 ? 1 : K / 8;
};

// One word counted bit by bit (head and tail words, §4.1's residual).
template <int K>
__device__ __forceinline__ void count_word(uint32_t (&c)[K], uint32_t w) {
  if constexpr (K == 1) {
    c[0] += __popc(w);
  } else {
#pragma unroll
    for (int p = 0; p < K; ++p) c[p] += (w >> p) & 1u;
  }
}

template <int K>
__device__ __forceinline__ uint32_t load_word(const uint8_t* p) {
  if constexpr (K == 8 || K == 1) return *p;
  if constexpr (K == 16) return *reinterpret_cast<const uint16_t*>(p);
  return *reinterpret_cast<const uint32_t*>(p);
}

// One 64-bit word counted bit by bit into two 32-position halves.
__device__ __forceinline__ void count_word64(uint32_t (&lo)[32], uint32_t (&hi)[32], const uint8_t* p) {
  const uint64_t w = *reinterpret_cast<const uint64_t*>(p);
  count_word<32>(lo, uint32_t(w));
  count_word<32>(hi, uint32_t(w >> 32));
}

// ---- streaming 16-byte load ------------------------------------------------
// Read-only, no L1 allocation, 256-byte L2 prefetch: every input byte is
// read exactly once.
__device__ __forceinline__ uint4 ld_stream(const uint4* p) {
  uint4 r;
  asm("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0, %1, %2, %3}, [%4];"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
      : "l"(p));
  return r;
}

// Plain coherent 16-byte load, for inputs that live in pinned host memory
// mapped into the device address space (read across NVLink-C2C).
__device__ __forceinline__ uint4 ld_coherent(const uint4* p) {
  uint4 r;
  asm volatile("ld.global.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p));
  return r;
}

// ---- warp reduction of K position counters --------------------------------
// Transpose-reduce: at each step with lane offset `off` a lane keeps one
// half of its m values, sends the other half to its partner and adds what it
// receives, so m halves while the lanes specialise.  After log2(K) steps each
// lane holds one position, p = lane >> (5 - log2 K), summed over the lanes
// that differ in the bits used; plain xor-adds finish the sum over all 32
// lanes.  Costs K - 1 + (5 - log2 K) shuffles instead of 5 K.
template <int K>
__device__ __forceinline__ uint32_t warp_reduce_positions(uint32_t (&v)[K]) {
  const int lane = threadIdx.x & 31;
  constexpr int LK = ilog2<K>::value;
#pragma unroll
  for (int s = 0; s < LK; ++s) {
    const int m = K >> s;
    const int off = 16 >> s;
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < m / 2; ++i) {
      const uint32_t send = upper ? v[i] : v[i + m / 2];
      const uint32_t keep = upper ? v[i + m / 2] : v[i];
      v[i] = keep + __shfl_xor_sync(FULL_MASK, send, off);
    }
  }
#pragma unroll
  for (int s = LK; s < 5; ++s) v[0] += __shfl_xor_sync(FULL_MASK, v[0], 16 >> s);
  return v[0];
}

// Block reduction followed by one 64-bit atomic add per position per block,
// or, when the block is the whole grid and the caller asked for it (store),
// a plain store of every position (no prior memset needed).  Only positions
// below `limit` are written.  Every thread of the block must call it.
template <int K, int NWARPS>
__device__ __forceinline__ void block_reduce_add(uint32_t (&c)[K], unsigned long long* counts,
                                                 bool store = false, int limit = K) {
  __shared__ uint32_t red[NWARPS][K];
  constexpr int SH = 5 - ilog2<K>::value;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t v = warp_reduce_positions<K>(c);
  if ((lane & ((1 << SH) - 1)) == 0) red[warp][lane >> SH] = v;
  __syncthreads();
  if (int(threadIdx.x) < limit) {  // positions >= limit are not part of the output
    unsigned long long s = 0;
#pragma unroll
    for (int w = 0; w < NWARPS; ++w) s += red[w][threadIdx.x];
    if (store)
      counts[threadIdx.x] = s;
    else if (s)
      atomicAdd(counts + threadIdx.x, s);
  }
}

// Overwrite without a memset before the kernel (the last block publishes).
// Every block has added its counts into acc -- an accumulator owned by the
// caller's stream, zero between launches -- with block_reduce_add; each
// block then arrives once on `arrived`, and the block that arrives last
// moves acc[0..k) into counts and leaves acc and the counter at zero for the
// next launch on the stream.  Every thread of the block must call it, after
// its own additions.
// `last` is a word of shared memory the block may use for the verdict.
__device__ __forceinline__ void block_publish_via(unsigned long long* acc, unsigned* arrived,
                                                  unsigned long long* counts, int k, volatile unsigned* last) {
  __threadfence();  // this thread's additions into acc come before the arrival
  __syncthreads();
  if (threadIdx.x == 0) *last = atomicAdd(arrived, 1u) == gridDim.x - 1 ? 1u : 0u;
  __syncthreads();
  if (*last) {
    __threadfence();
    if (int(threadIdx.x) < k) counts[threadIdx.x] = atomicExch(acc + threadIdx.x, 0ull);
    if (threadIdx.x == 0) atomicExch(arrived, 0u);
  }
}

__device__ __forceinline__ void block_publish(unsigned long long* acc, unsigned* arrived,
                                              unsigned long long* counts, int k) {
  __shared__ unsigned s_last;
  block_publish_via(acc, arrived, counts, k, &s_last);
}

// ---- mbarrier / bulk-copy helpers (inline PTX) ----------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the phase of parity `parity` of `bar` to complete, for at most
// limit_ns nanoseconds of wall time.  Returns false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
  return true;
}

// One-dimensional bulk copy global -> shared, completing `bytes` of
// transaction count on `bar`.  src, dst 16-byte aligned; bytes a multiple
// of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// An L2 policy that marks lines evict-first (for data read exactly once).
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// bulk_g2s with an L2 cache-policy hint.
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

// Error bits written to the library's device error word.
enum : unsigned {
  ERR_BIT_TIMEOUT_FULL = 1u,
  ERR_BIT_TIMEOUT_EMPTY = 2u,
  ERR_BIT_TIMEOUT_DRAIN = 4u,
  ERR_BIT_BAD_OFFSETS = 8u
};

constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s per wait

}  // namespace ppc
