// Fused one-hot encode + positional count: categorical ids -> frequency
// histogram without materialising the one-hot words.
//
// The paper's motivation (§1, Table 1) is exactly this pipeline: values are
// one-hot encoded and the positional population count of the encoded words
// is the histogram.  Here each thread loads 16-byte vectors of ids, builds
// the one-hot words directly in registers -- with lanes of LW = 8, 16 or 32
// bits (the smallest that holds k positions), 32/LW ids share one 32-bit
// register -- and feeds those registers through the same carry-save circuit
// and popc flush as the plain count.  Ids >= k encode to the empty word.
// 32-bit ids are encoded by a clamped shift and a mask (onehot_kernel for
// small inputs: circuit F_4, F_5 for one id per register).  8- and 16-bit
// ids are encoded by lookups in a table in shared memory (onehot_lut_kernel
// for small inputs).  From 4 MiB of 8-bit ids and 8 MiB of wider ids
// (ring_min_bytes) every id width goes through onehot_ring_kernel, fed by
// bulk copies, with the same two encodings; for 8-bit ids and k <= 16 it
// looks up pairs of ids below 16, one lookup for two ids.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace ppc {

struct OnehotArgs {
  const uint4* body;
  uint64_t nvec;
  const uint8_t* head;
  uint32_t head_ids;
  const uint8_t* tail;
  uint32_t tail_ids;
  unsigned long long* counts;
  uint32_t k;
  uint32_t store;
  uint32_t one;  // 1: multiplier of the FMA-pipe additions in the lookup kernels
  unsigned* err;  // device error word (bounded waits of the ring kernel)
  uint32_t publish;         // 1: blocks add into acc; the last one writes the counts
  unsigned long long* acc;  // the stream's accumulator (publish), zero between launches
  unsigned* arrived;        // blocks that have added into acc (publish)
};

// The j-th id of a 16-byte vector of IDB-byte ids (j known at compile time),
// zero-extended with one byte permute.
template <int IDB>
__device__ __forceinline__ uint32_t id_at(const uint4& x, int j) {
  const uint32_t r[4] = {x.x, x.y, x.z, x.w};
  if constexpr (IDB == 4) return r[j];
  if constexpr (IDB == 2) return __byte_perm(r[j / 2], 0u, (j % 2) ? 0x4432u : 0x4410u);
  return __byte_perm(r[j / 4], 0u, 0x4440u | unsigned(j % 4));
}

// base << amount with the PTX rule that amounts above 32 give 0, so an id
// of 32 or more shifts the one-hot bit out of the register.
__device__ __forceinline__ uint32_t shl_clamped(uint32_t base, uint32_t amount) {
  uint32_t d;
  asm("shl.b32 %0, %1, %2;" : "=r"(d) : "r"(base), "r"(amount));
  return d;
}

template <int IDB>
__device__ __forceinline__ uint32_t load_id(const uint8_t* p) {
  if constexpr (IDB == 1) return *p;
  if constexpr (IDB == 2) return *reinterpret_cast<const uint16_t*>(p);
  return *reinterpret_cast<const uint32_t*>(p);
}

// Trip of the shift-and-mask kernel: R registers through the circuit F_L,
// U vectors per thread.  One id per register (LW = 32) takes 32 registers
// (8 vectors of 32-bit ids in flight per thread) instead of 16: with 4
// vectors per trip the loads in flight were too few to cover DRAM latency.
template <int IDB, int LW>
struct IdTrip {
  static constexpr int IDS_PER_VEC = 16 / IDB;
  static constexpr int IDS_PER_REG = 32 / LW;
  static constexpr int REGS_PER_VEC = IDS_PER_VEC / IDS_PER_REG;
  static constexpr int R = LW == 32 ? 32 : 16;
  static constexpr int L = ilog2<R>::value;
  static constexpr int U = R / REGS_PER_VEC;  // vectors per trip
};

template <int IDB, int LW, int NTHREADS>
__global__ void __launch_bounds__(NTHREADS) onehot_kernel(OnehotArgs a) {
  using TS = IdTrip<IDB, LW>;
  constexpr int IDS_PER_REG = TS::IDS_PER_REG, REGS_PER_VEC = TS::REGS_PER_VEC, R = TS::R, L = TS::L, U = TS::U;
  const uint32_t k = a.k;
  // lane q of a register holds the one-hot bit of its id at bit q*LW + id;
  // the mask keeps bits q*LW .. q*LW + k - 1 (ids >= k, which could spill
  // into the next lane, are dropped)
  const uint32_t km = k >= 32 ? 0xFFFFFFFFu : (1u << k) - 1u;
  uint32_t lane_mask_q[IDS_PER_REG];
#pragma unroll
  for (int q = 0; q < IDS_PER_REG; ++q) lane_mask_q[q] = km << (q * LW);
  uint32_t B[L];
#pragma unroll
  for (int l = 0; l < L; ++l) B[l] = 0;
  uint32_t top[LW];
#pragma unroll
  for (int p = 0; p < LW; ++p) top[p] = 0;
  const uint64_t stride = uint64_t(gridDim.x) * NTHREADS;
  for (uint64_t v = uint64_t(blockIdx.x) * NTHREADS + threadIdx.x; v < a.nvec; v += U * stride) {
    uint32_t d[R];
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const uint64_t idx = v + i * stride;
      const bool live = idx < a.nvec;  // a missing vector is no data (not ids of zero)
      const uint4 x = live ? ld_stream(a.body + idx) : make_uint4(0, 0, 0, 0);
#pragma unroll
      for (int r = 0; r < REGS_PER_VEC; ++r) {
        uint32_t reg = 0;
#pragma unroll
        for (int q = 0; q < IDS_PER_REG; ++q) {
          const uint32_t id = id_at<IDB>(x, r * IDS_PER_REG + q);
          reg |= shl_clamped(1u << (q * LW), id) & lane_mask_q[q];  // one shift, one masked or
        }
        d[i * REGS_PER_VEC + r] = live ? reg : 0u;
      }
    }
    flush<LW>(top, Circuit<L>::run(d, B));
  }
  uint32_t c[LW];
  finalize<LW, L>(c, top, B);
  if (blockIdx.x == 0) {  // head and tail ids (fewer than 16 each), one by one
    const unsigned t = threadIdx.x;
    if (t < a.head_ids) {
      const uint32_t id = load_id<IDB>(a.head + t * IDB);
      count_word<LW>(c, id < k ? 1u << id : 0u);
    }
    if (t >= 32 && t - 32 < a.tail_ids) {
      const uint32_t id = load_id<IDB>(a.tail + (t - 32) * IDB);
      count_word<LW>(c, id < k ? 1u << id : 0u);
    }
  }
  block_reduce_add<LW, NTHREADS / 32>(c, a.publish ? a.acc : a.counts, a.store != 0, int(k));
  if (a.publish) block_publish(a.acc, a.arrived, a.counts, int(k));
}

// 8- and 16-bit ids: the one-hot lane comes from a lookup table in shared
// memory instead of a shift and a mask.  Row e of the table (256 bytes) holds, for
// each of the 32 lanes of a warp, its own copy of two encodings of id e: at
// byte 4*l the low-lane word lo(e), at byte 128 + 4*l the high-lane word
// hi(e) (both zero for e >= k).  The 32 lookups of a warp thus fall in 32
// different banks whatever the ids, and the byte offset of a lookup,
// (id << 8) | (4 * lane), is one byte permute of the loaded word.
//   LW = 32: lo(e) = 1 << e (one id per register);
//   LW = 16: lo(e) = 1 << e, hi(e) = 1 << (e + 16): a register of two ids is
//            lo(a) + hi(b);
//   LW = 8:  lo(e) = 0x00010001 << e, hi(e) = 0x01000100 << e: lo(a) + hi(b)
//            holds ids a, b in bytes 0, 1 (and again in 2, 3), and one byte
//            permute of two such pairs gives the register of four ids.
// The sums have disjoint bits, so they are integer multiply-adds by a runtime
// 1 (OnehotArgs::one): they run on the FMA pipe, which is otherwise idle,
// instead of the ALU pipe that the byte permutes and the circuit fill.
constexpr int LUT_ROW = 256;
constexpr int LUT_BYTES = 256 * LUT_ROW;  // 64 KiB

template <int LW>
__device__ __forceinline__ uint32_t lut_lo(uint32_t e, uint32_t k) {
  if (e >= k) return 0u;
  return LW == 8 ? 0x00010001u << e : 1u << e;
}

template <int LW>
__device__ __forceinline__ uint32_t lut_hi(uint32_t e, uint32_t k) {
  if (e >= k || LW == 32) return 0u;
  return LW == 8 ? 0x01000100u << e : 1u << (e + 16);
}

// x * one + y on the FMA pipe (one == 1 at run time, unknown to the compiler).
__device__ __forceinline__ uint32_t mad_one(uint32_t x, uint32_t one, uint32_t y) {
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(x), "r"(one), "r"(y));
  return d;
}

// Table reads.  With IMM != 0 the table's shared-window address is the
// compile-time constant IMM and rides in the load instruction as its
// immediate (no add per lookup); with IMM == 0 it is added at run time.
template <uint32_t IMM>
struct LutRef {
  uint32_t base;  // shared-window address of the table
  template <uint32_t D>
  __device__ __forceinline__ uint32_t at(uint32_t off) const {
    uint32_t v;
    if constexpr (IMM != 0)
      asm("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(off), "n"(IMM + D));
    else
      asm("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(off + base), "n"(D));
    return v;
  }
};

// Encoded registers of the 4 ids in word w (byte j = id j): LW = 32 gives 4
// registers, 16 gives 2, 8 gives 1.
template <int LW, uint32_t IMM>
__device__ __forceinline__ void encode_word(uint32_t* r, uint32_t w, LutRef<IMM> t, uint32_t lanebase,
                                            uint32_t one) {
  uint32_t off[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) off[j] = __byte_perm(w, lanebase, 0x7604u | (unsigned(j) << 4));  // {4*lane, id j, 0, 0}
  if constexpr (LW == 32) {
#pragma unroll
    for (int j = 0; j < 4; ++j) r[j] = t.template at<0>(off[j]);
  } else if constexpr (LW == 16) {
    r[0] = mad_one(t.template at<128>(off[1]), one, t.template at<0>(off[0]));
    r[1] = mad_one(t.template at<128>(off[3]), one, t.template at<0>(off[2]));
  } else {
    const uint32_t p01 = mad_one(t.template at<128>(off[1]), one, t.template at<0>(off[0]));
    const uint32_t p23 = mad_one(t.template at<128>(off[3]), one, t.template at<0>(off[2]));
    r[0] = __byte_perm(p01, p23, 0x7610u);
  }
}

// 16-bit ids: each 16-bit half of w clamped to at most 255 (one instruction
// for both), so that any id >= 256 reads table row 255, which is empty
// (k <= 32); an id below 256 keeps its low byte.
__device__ __forceinline__ uint32_t clamp_ids16(uint32_t w) {
  uint32_t d;
  asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(w), "r"(0x00FF00FFu));
  return d;
}

// Encoded registers of the 16 bytes of ids in x (IDB bytes per id): 16/IDB
// ids, 32/LW per register.
template <int LW, int IDB, uint32_t IMM>
__device__ __forceinline__ void encode_vec(uint32_t* d, const uint4& x, LutRef<IMM> t, uint32_t lanebase,
                                           uint32_t one) {
  const uint32_t w[4] = {x.x, x.y, x.z, x.w};
  if constexpr (IDB == 1) {
    constexpr int RPW = 4 / (32 / LW);  // registers per word of 4 ids
#pragma unroll
    for (int q = 0; q < 4; ++q) encode_word<LW, IMM>(d + q * RPW, w[q], t, lanebase, one);
  } else {
    // two ids per word: bytes 0 and 2 of the clamped word are their rows
    uint32_t p[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t c = clamp_ids16(w[q]);
      const uint32_t off0 = __byte_perm(c, lanebase, 0x7604u), off1 = __byte_perm(c, lanebase, 0x7624u);
      if constexpr (LW == 32) {
        d[2 * q] = t.template at<0>(off0);
        d[2 * q + 1] = t.template at<0>(off1);
      } else {
        p[q] = mad_one(t.template at<128>(off1), one, t.template at<0>(off0));
      }
    }
    if constexpr (LW == 16) {
#pragma unroll
      for (int q = 0; q < 4; ++q) d[q] = p[q];
    } else if constexpr (LW == 8) {  // p holds its two ids in bytes 0, 1 (and 2, 3)
      d[0] = __byte_perm(p[0], p[1], 0x7610u);
      d[1] = __byte_perm(p[2], p[3], 0x7610u);
    }
  }
}

// Pairs of 8-bit ids below 16 (the bulk-copy kernel, k <= 16).  For a word
// w of four such ids a, b, c, d (bytes 0..3), w + (w >> 4) -- one integer
// multiply-add, mad.hi(w, 2^28, w), on the FMA pipe -- holds a | b << 4 in
// byte 0 and c | d << 4 in byte 2 (no carries: every nibble sum is below
// 256).  Row a | b << 4 of the pair table holds the encoded register of the
// pair: one lookup for two ids, no combine.
__device__ __forceinline__ uint32_t pack_id_pairs(uint32_t w) {
  uint32_t d;
  asm("mad.hi.u32 %0, %1, %2, %1;" : "=r"(d) : "r"(w), "r"(0x10000000u));
  return d;
}

template <int LW>
__device__ __forceinline__ uint32_t pair_lo(uint32_t row, uint32_t k) {
  const uint32_t a = row & 15u, b = row >> 4;
  const uint32_t ea = a < k ? 1u << a : 0u, eb = b < k ? 1u << b : 0u;
  return LW == 16 ? ea | (eb << 16) : ea | (eb << 8);
}

template <int LW>
__device__ __forceinline__ uint32_t pair_hi(uint32_t row, uint32_t k) {
  return LW == 8 ? pair_lo<8>(row, k) << 16 : 0u;
}

template <int LW, uint32_t IMM>
__device__ __forceinline__ void encode_vec_pairs(uint32_t* d, const uint4& x, LutRef<IMM> t, uint32_t lanebase,
                                                 uint32_t one) {
  const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t pr = pack_id_pairs(w[q]);
    const uint32_t off0 = __byte_perm(pr, lanebase, 0x7604u), off1 = __byte_perm(pr, lanebase, 0x7624u);
    if constexpr (LW == 16) {
      d[2 * q] = t.template at<0>(off0);
      d[2 * q + 1] = t.template at<0>(off1);
    } else {
      d[q] = mad_one(t.template at<128>(off1), one, t.template at<0>(off0));
    }
  }
}

// Any 8-bit ids: clamped shift and mask per id (the trips that hold an id of
// 16 or more, where the pair table does not apply).  km = (1 << k) - 1.
template <int LW>
__device__ __forceinline__ void encode_vec_shift(uint32_t* d, const uint4& x, uint32_t km) {
  constexpr int IPR = 32 / LW;  // ids per register
  const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
  for (int r = 0; r < 16 / IPR; ++r) {
    uint32_t reg = 0;
#pragma unroll
    for (int q = 0; q < IPR; ++q) {
      const int j = r * IPR + q;
      const uint32_t id = __byte_perm(w[j / 4], 0u, 0x4440u | unsigned(j % 4));
      reg |= shl_clamped(1u << (q * LW), id) & (km << (q * LW));
    }
    d[r] = reg;
  }
}

// 32-bit ids (the bulk-copy kernel): each id by a clamped shift and a mask,
// 32/LW ids per register.  km = (1 << k) - 1; an id of 32 or more shifts
// its bit out of the register, one in [k, 32) is masked off.
template <int LW>
__device__ __forceinline__ void encode_vec_ids32(uint32_t* d, const uint4& x, uint32_t km) {
  constexpr int IPR = 32 / LW;  // ids per register
  const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
  for (int r = 0; r < 4 / IPR; ++r) {
    uint32_t reg = 0;
#pragma unroll
    for (int q = 0; q < IPR; ++q) reg |= shl_clamped(1u << (q * LW), w[r * IPR + q]) & (km << (q * LW));
    d[r] = reg;
  }
}

// flush() with the additions on the FMA pipe.
template <int K>
__device__ __forceinline__ void flush_mad(uint32_t (&top)[K], uint32_t t, uint32_t one) {
#pragma unroll
  for (int p = 0; p < K; ++p) top[p] = mad_one(__popc(t & (lane_mask<K>::value << p)), one, top[p]);
}

// Counts of the lookup kernels.  A trip's circuit F_N returns its top
// register (weight 2^N).  Top registers of consecutive trips are combined
// as a binary counter of carry-save adders, D levels deep: level j holds at
// most one pending register of weight 2^(N+j); a second one meets it in a
// CSA whose sum bit goes to B[N+j] and whose carry (weight 2^(N+j+1)) moves
// up a level, and the carry out of the last level is flushed.  The flush
// thus runs once per 2^D trips -- the circuit F_(N+D) without holding
// 2^(N+D) registers at once.  PairedCounts (the register-load kernels) takes
// two levels and flushes with popc into LW counters per thread;
// ColumnCounts (the bulk-copy kernel) flushes through the warp and takes
// ring_depth levels: four for one id per register (LW = 32), whose ALU pipe
// is filled by the circuit (flush every 16 trips), two otherwise.
template <int LW>
struct ring_depth {
  static constexpr int value = LW == 32 ? 4 : 2;
};

template <int LW, int N, int D = 2>
struct PairedCounts {
  uint32_t B[N + D];   // B[l] at weight 2^l
  uint32_t pend[D];    // pend[j]: unpaired register of weight 2^(N+j)
  uint32_t trips = 0;
  uint32_t top[LW];    // units of 2^(N+D)
  __device__ __forceinline__ PairedCounts() {
#pragma unroll
    for (int l = 0; l < N + D; ++l) B[l] = 0;
#pragma unroll
    for (int j = 0; j < D; ++j) pend[j] = 0;
#pragma unroll
    for (int p = 0; p < LW; ++p) top[p] = 0;
  }
  // t (weight 2^(N+J)) meets the pending registers of levels J.. up to
  // level `lvl`, the first one that is free.
  template <int J>
  __device__ __forceinline__ void carry_into(uint32_t t, int lvl, uint32_t one) {
    if constexpr (J == D) {
      flush_mad<LW>(top, t, one);
    } else {
      if (lvl == J) {
        pend[J] = t;
      } else {
        uint32_t h;
        csa(h, B[N + J], B[N + J], pend[J], t);
        pend[J] = 0;
        carry_into<J + 1>(h, lvl, one);
      }
    }
  }
  __device__ __forceinline__ void add_trip(const uint32_t* d, uint32_t one) {
    const uint32_t t = Circuit<N>::run(d, B);
    if constexpr (D == 2) {
      if ((trips & 1u) == 0) {
        pend[0] = t;
      } else {
        uint32_t h;
        csa(h, B[N], B[N], pend[0], t);
        pend[0] = 0;
        if ((trips & 2u) == 0) {
          pend[1] = h;
        } else {
          uint32_t h2;
          csa(h2, B[N + 1], B[N + 1], pend[1], h);
          pend[1] = 0;
          flush_mad<LW>(top, h2, one);
        }
      }
    } else {
      // levels 0 .. lvl-1 hold a pending register (the trailing ones of
      // `trips`), level lvl is free (lvl == D: the carry is flushed)
      carry_into<0>(t, __ffs(~trips) - 1, one);
    }
    ++trips;
  }
  __device__ __forceinline__ void finish(uint32_t (&c)[LW]) const {
    finalize<LW, N + D>(c, top, B);  // top at 2^(N+D), B[l] at 2^l
#pragma unroll
    for (int j = 0; j < D; ++j) {
#pragma unroll
      for (int p = 0; p < LW; ++p)
        c[p] += static_cast<uint32_t>(__popc(pend[j] & (lane_mask<LW>::value << p))) << (N + j);
    }
  }
};

// Column sums of a warp's 32 x 32 bit matrix (row = lane, column = bit):
// lane p receives the number of lanes whose x has bit p set.  Five exchange
// stages transpose the matrix -- at stage s, lanes l and l ^ s swap the
// blocks of s columns that the other one needs (byte permutes for s = 16
// and 8; a rotate and a bit select for 4, 2, 1) -- after which lane p holds
// column p as a word, and its popc is the sum.  Every lane of the warp must
// call it.
__device__ __forceinline__ uint32_t warp_column_counts(uint32_t x) {
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t y = __shfl_xor_sync(FULL_MASK, x, 16);
  x = __byte_perm(x, y, (lane & 16u) ? 0x3276u : 0x5410u);  // upper: {y2 y3 x2 x3}, lower: {x0 x1 y0 y1}
  y = __shfl_xor_sync(FULL_MASK, x, 8);
  x = __byte_perm(x, y, (lane & 8u) ? 0x3715u : 0x6240u);  // upper: {y1 x1 y3 x3}, lower: {x0 y0 x2 y2}
#pragma unroll
  for (int s = 4; s >= 1; s >>= 1) {
    const uint32_t m = s == 4 ? 0x0F0F0F0Fu : s == 2 ? 0x33333333u : 0x55555555u;
    const bool up = (lane & uint32_t(s)) != 0;
    y = __shfl_xor_sync(FULL_MASK, x, s);
    // lower lane: its own m-blocks and the partner's, moved up by s; upper
    // lane: its own ~m-blocks and the partner's, moved down by s (the
    // rotate's wrapped bits fall outside the blocks kept)
    const uint32_t r = __funnelshift_l(y, y, up ? 32u - uint32_t(s) : uint32_t(s));
    const uint32_t mk = up ? ~m : m;
    x = (x & mk) | (r & ~mk);
  }
  return static_cast<uint32_t>(__popc(x));
}

// The counter of PairedCounts with the flush done by the warp: the carry
// out of the last level (weight 2^(N+D)) goes through warp_column_counts,
// so lane q keeps the warp's count of register bit q in one register
// instead of every lane keeping LW counters; bits q, q + LW, ... are the
// same category and are summed once, at the end (on 2 GiB of 8-bit ids:
// 4809 -> 5137 GB/s for 17-32 categories, 6855 -> 7039 for 9-16, 7097 ->
// 7133 for up to 8, against the per-thread flush).  finish() returns the
// warp's counts in the layout of warp_reduce_positions (lane i: position
// i >> (5 - log2 LW)).  Every lane of a warp must add the same number of
// trips (the bulk-copy kernel's trips are the same for the whole CTA), as
// the flush is a warp-wide exchange.
template <int LW, int N, int D>
struct ColumnCounts {
  uint32_t B[N + D];  // B[l] at weight 2^l
  uint32_t pend[D];   // pend[j]: unpaired register of weight 2^(N+j)
  uint32_t trips = 0;
  uint32_t top = 0;   // lane q: the warp's carries at bit q, units of 2^(N+D)
  uint32_t ones = 0;  // lane q: single words added at bit q (add_word)
  __device__ __forceinline__ ColumnCounts() {
#pragma unroll
    for (int l = 0; l < N + D; ++l) B[l] = 0;
#pragma unroll
    for (int j = 0; j < D; ++j) pend[j] = 0;
  }
  template <int J>
  __device__ __forceinline__ void carry_into(uint32_t t, int lvl) {
    if constexpr (J == D) {
      top += warp_column_counts(t);
    } else {
      if (lvl == J) {
        pend[J] = t;
      } else {
        uint32_t h;
        csa(h, B[N + J], B[N + J], pend[J], t);
        pend[J] = 0;
        carry_into<J + 1>(h, lvl);
      }
    }
  }
  __device__ __forceinline__ void add_trip(const uint32_t* d, uint32_t /*one*/) {
    const uint32_t t = Circuit<N>::run(d, B);
    carry_into<0>(t, __ffs(~trips) - 1);
    ++trips;
  }
  // One encoded word of weight 1 (every lane of the warp calls it).
  __device__ __forceinline__ void add_word(uint32_t w) { ones += warp_column_counts(w); }
  __device__ __forceinline__ uint32_t finish() const {
    uint32_t v = (top << (N + D)) + ones;
#pragma unroll
    for (int l = 0; l < N + D; ++l) v += warp_column_counts(B[l]) << l;
#pragma unroll
    for (int j = 0; j < D; ++j) v += warp_column_counts(pend[j]) << (N + j);
    if constexpr (LW < 32) {
      constexpr int SH = 5 - ilog2<LW>::value;
#pragma unroll
      for (int s = 16; s >= LW; s >>= 1) v += __shfl_down_sync(FULL_MASK, v, s);  // lane p < LW: category p
      v = __shfl_sync(FULL_MASK, v, (threadIdx.x & 31u) >> SH);
    }
    return v;
  }
};

// The block's counts: each warp reduces its lanes' counters, warps
// [0, CWARPS) leave their sums in `red` (CWARPS x LW words of shared memory
// that no thread reads or writes any more), and threads 0..k-1 add them
// into counts[p] (or the stream's accumulator, whose last block then writes
// the counts; `last` is a free word of shared memory for that verdict) with
// one atomic each, or store them when the grid is one CTA.  Every thread of
// the block calls it.
// reduce_warp_sums_in takes the warps' sums already made (lane i of a
// warp: the warp's count of position i >> (5 - log2 LW)).
template <int LW, int CWARPS>
__device__ __forceinline__ void reduce_warp_sums_in(uint32_t* red, uint32_t vsum, const OnehotArgs& a,
                                                    volatile unsigned* last) {
  constexpr int SH = 5 - ilog2<LW>::value;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  __syncthreads();
  if (warp < uint32_t(CWARPS) && (lane & ((1u << SH) - 1u)) == 0) red[warp * LW + (lane >> SH)] = vsum;
  __syncthreads();
  if (threadIdx.x < a.k) {
    unsigned long long sum = 0;
#pragma unroll
    for (int w = 0; w < CWARPS; ++w) sum += red[w * LW + threadIdx.x];
    if (a.store)
      a.counts[threadIdx.x] = sum;
    else if (sum)
      atomicAdd((a.publish ? a.acc : a.counts) + threadIdx.x, sum);
  }
  if (a.publish) block_publish_via(a.acc, a.arrived, a.counts, int(a.k), last);
}

template <int LW, int CWARPS>
__device__ __forceinline__ void reduce_counts_in(uint32_t* red, uint32_t (&c)[LW], const OnehotArgs& a,
                                                 volatile unsigned* last) {
  reduce_warp_sums_in<LW, CWARPS>(red, warp_reduce_positions<LW>(c), a, last);
}

// A trip is U = 4 vectors per thread (2 for one 8-bit id per register),
// through the circuit F_N over their R = 2^N registers (N <= 5).
template <int LW, int IDB>
struct LutTrip {
  static constexpr int REGS_PER_VEC = (16 / IDB) / (32 / LW);
  static constexpr int N = ilog2<4 * REGS_PER_VEC>::value < 5 ? ilog2<4 * REGS_PER_VEC>::value : 5;
  static constexpr int R = 1 << N;
  static constexpr int U = R / REGS_PER_VEC;  // vectors per trip
};

// The thread's share of the body: whole trips, then at most one partial trip.
template <int LW, int IDB, int NTHREADS, uint32_t IMM>
__device__ __forceinline__ void lut_count_body(const OnehotArgs& a, LutRef<IMM> t, uint32_t lanebase,
                                               PairedCounts<LW, LutTrip<LW, IDB>::N>& acc) {
  constexpr int REGS_PER_VEC = LutTrip<LW, IDB>::REGS_PER_VEC, R = LutTrip<LW, IDB>::R, U = LutTrip<LW, IDB>::U;
  const uint32_t one = a.one;
  const uint64_t stride = uint64_t(gridDim.x) * NTHREADS;
  const uint64_t span = uint64_t(U - 1) * stride;
  uint64_t v = uint64_t(blockIdx.x) * NTHREADS + threadIdx.x;
  // Whole trips (every vector present).  Each vector of the next trip is
  // loaded into x[i] as soon as x[i] has been encoded, so the loads are in
  // flight while the rest of the trip is encoded and counted.
  uint4 x[U];
  bool full = v + span < a.nvec;
  if (full) {
#pragma unroll
    for (int i = 0; i < U; ++i) x[i] = ld_stream(a.body + v + i * stride);
  }
  while (full) {
    const uint64_t vn = v + U * stride;
    const bool full_n = vn + span < a.nvec;
    uint32_t d[R];
#pragma unroll
    for (int i = 0; i < U; ++i) {
      encode_vec<LW, IDB, IMM>(d + i * REGS_PER_VEC, x[i], t, lanebase, one);
      if (full_n) x[i] = ld_stream(a.body + vn + i * stride);
    }
    acc.add_trip(d, one);
    v = vn;
    full = full_n;
  }
  if (v < a.nvec) {  // last, partial trip: a missing vector reads as all-ones ids, which encode to nothing
    uint32_t d[R];
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const uint64_t idx = v + i * stride;
      const uint4 y = idx < a.nvec ? ld_stream(a.body + idx) : make_uint4(~0u, ~0u, ~0u, ~0u);
      encode_vec<LW, IDB, IMM>(d + i * REGS_PER_VEC, y, t, lanebase, one);
    }
    acc.add_trip(d, one);
  }
}

// Shared-window address of dynamic shared memory in a kernel with no static
// shared memory: the GPU reserves the first 1 KiB of every block's window.
// The kernel checks it at run time and adds the address itself otherwise.
constexpr uint32_t LUT_USUAL_BASE = 1024;

template <int LW, int IDB, int NTHREADS>
__global__ void __launch_bounds__(NTHREADS, 3) onehot_lut_kernel(OnehotArgs a) {
  extern __shared__ __align__(1024) uint8_t lut[];  // the only shared memory of this kernel
  constexpr int N = LutTrip<LW, IDB>::N;
  const uint32_t lane = threadIdx.x & 31u;
  for (uint32_t e = threadIdx.x >> 5; e < 256u; e += NTHREADS / 32) {
    *reinterpret_cast<uint32_t*>(lut + e * LUT_ROW + lane * 4u) = lut_lo<LW>(e, a.k);
    *reinterpret_cast<uint32_t*>(lut + e * LUT_ROW + 128u + lane * 4u) = lut_hi<LW>(e, a.k);
  }
  __syncthreads();
  // Every lookup depends on lanebase, made here, after the barrier, so no
  // lookup can be scheduled before the table is complete.
  uint32_t lanebase;
  asm volatile("mov.u32 %0, %1;" : "=r"(lanebase) : "r"(lane * 4u));
  const uint32_t base = static_cast<uint32_t>(__cvta_generic_to_shared(lut));
  PairedCounts<LW, N> acc;
  if (base == LUT_USUAL_BASE)
    lut_count_body<LW, IDB, NTHREADS, LUT_USUAL_BASE>(a, LutRef<LUT_USUAL_BASE>{base}, lanebase, acc);
  else
    lut_count_body<LW, IDB, NTHREADS, 0>(a, LutRef<0>{base}, lanebase, acc);
  uint32_t c[LW];
  acc.finish(c);
  if (blockIdx.x == 0) {  // head and tail ids (fewer than 16 each), one by one
    const unsigned t = threadIdx.x;
    if (t < a.head_ids) {
      const uint32_t id = load_id<IDB>(a.head + t * IDB);
      count_word<LW>(c, id < a.k ? 1u << id : 0u);
    }
    if (t >= 32 && t - 32 < a.tail_ids) {
      const uint32_t id = load_id<IDB>(a.tail + (t - 32) * IDB);
      count_word<LW>(c, id < a.k ? 1u << id : 0u);
    }
  }
  // block reduction in the table's memory, free once every warp is past its
  // last lookup
  reduce_counts_in<LW, NTHREADS / 32>(reinterpret_cast<uint32_t*>(lut), c, a,
                                      reinterpret_cast<unsigned*>(lut + LUT_BYTES - 4));
}

template <int LW, int IDB>
static int launch_onehot_lut(const DeviceState& st, OnehotArgs a, cudaStream_t stream) {
  constexpr int T = 256;
  constexpr int U = LutTrip<LW, IDB>::U;
  auto kern = onehot_lut_kernel<LW, IDB, T>;
  if (const cudaError_t e = ensure_dynamic_smem<onehot_lut_kernel<LW, IDB, T>>(st.device, LUT_BYTES))
    return cuda_fail(e);
  const int occ = resident_blocks(reinterpret_cast<const void*>(kern), st.device, T, LUT_BYTES);
  const uint64_t cap = uint64_t(st.sms) * uint64_t(occ);
  const uint64_t need = (a.nvec + uint64_t(U) * T - 1) / (uint64_t(U) * T);
  uint64_t grid = std::max<uint64_t>(1, std::min(cap, need));
  grid = std::max<uint64_t>(grid, ((a.nvec * 16) >> 31) + 1);  // per-CTA u32 partials stay exact
  a.store = grid == 1 ? 1u : 0u;
  a.publish = grid > 1 && a.acc && a.arrived ? 1u : 0u;
  if (grid > 1 && !a.publish) {
    const cudaError_t e = cudaMemsetAsync(a.counts, 0, sizeof(unsigned long long) * a.k, stream);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  kern<<<unsigned(grid), T, LUT_BYTES, stream>>>(a);
  note_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? POSPOPCNT_OK : cuda_fail(e);
}

// ---------------------------------------------------------------------------
// Large inputs of 8-bit ids: the same encoding and circuit, with the ids
// brought in by bulk copies.  One CTA per SM: one producer lane streams
// 48 KiB chunks into a 3-stage ring (full/empty mbarriers, bounded waits),
// 24 consumer warps read them back with 16-byte shared loads.  Up to 144 KiB
// per SM is in flight without holding a register, and the 64 KiB table is
// shared by 24 warps instead of 8.  Everything lives in dynamic shared
// memory -- table, ring, barriers -- so the table keeps the usual address.
constexpr int RING_CWARPS = 24;
constexpr int RING_THREADS = (RING_CWARPS + 1) * 32;
constexpr uint32_t RING_CHUNK = 49152;  // one trip of 4 vectors for each of the 768 consumer threads
constexpr uint32_t RING_STAGES = 3;

struct RingCtl {
  uint64_t full[RING_STAGES];
  uint64_t empty[RING_STAGES];
  uint32_t issued;                 // chunks the producer issued
  uint32_t abort;
  uint32_t consumed[RING_CWARPS];  // chunks each consumer warp finished
  uint32_t last;                   // this block arrived last on the stream's accumulator
};

constexpr size_t RING_SMEM = size_t(LUT_BYTES) + size_t(RING_STAGES) * RING_CHUNK + sizeof(RingCtl);

// The bulk-copy kernel's table is the pair table for 8-bit ids and k <= 16.
template <int LW, int IDB>
struct RingPairs {
  static constexpr bool value = IDB == 1 && LW <= 16;
};
static_assert(RING_CHUNK % (16 * 4 * RING_CWARPS * 32) == 0 && RING_CHUNK % (16 * 2 * RING_CWARPS * 32) == 0,
              "a chunk is a whole number of consumer trips");
// Smallest body (bytes) that takes the bulk-copy kernel: where it overtook
// the register-load kernels in same-box A/B runs (8-bit ids: behind at 1-2
// MiB, ahead from 4 MiB for 16 and 32 categories; 16- and 32-bit ids: level
// or behind at 4 MiB, ahead at 16 MiB).
template <int IDB>
constexpr uint64_t ring_min_bytes() {
  return (IDB == 1 ? uint64_t(4) : uint64_t(8)) << 20;
}

// The bulk-copy kernel's trip: that of the lookup kernels, except for one
// 8-bit id per register, where a trip is 4 vectors per thread, 64 ids
// through F_6 (one trip per thread per ring chunk): 2 % faster than 32-id
// trips once the flush no longer holds 32 counters per thread.
template <int LW, int IDB>
struct RingTrip : LutTrip<LW, IDB> {};
template <>
struct RingTrip<32, 1> {
  static constexpr int REGS_PER_VEC = 16;
  static constexpr int N = 6;
  static constexpr int R = 64;
  static constexpr int U = 4;
};

// The ring kernel's counter: the flush done by the warp, at every width.
template <int LW, int IDB>
struct RingAccT {
  using type = ColumnCounts<LW, RingTrip<LW, IDB>::N, ring_depth<LW>::value>;
};
template <int LW, int IDB>
using RingAcc = typename RingAccT<LW, IDB>::type;

// One trip over vectors [base, base + U*CT) of a ring stage; GUARD: some may
// lie past nv (the partial last chunk of the input) and read as ids 255.
template <int LW, int IDB, uint32_t IMM, bool GUARD>
__device__ __forceinline__ void ring_trip(const uint4* sv, uint32_t base, uint32_t nv, LutRef<IMM> t,
                                          uint32_t lanebase, uint32_t one, uint32_t km,
                                          RingAcc<LW, IDB>& acc) {
  constexpr int REGS_PER_VEC = RingTrip<LW, IDB>::REGS_PER_VEC, R = RingTrip<LW, IDB>::R, U = RingTrip<LW, IDB>::U;
  constexpr uint32_t CT = RING_CWARPS * 32;
  uint4 y[U];
#pragma unroll
  for (int j = 0; j < U; ++j) {
    const uint32_t idx = base + j * CT + threadIdx.x;
    y[j] = (!GUARD || idx < nv) ? sv[idx] : make_uint4(~0u, ~0u, ~0u, ~0u);  // all-ones ids: nothing
  }
  uint32_t d[R];
  if constexpr (RingPairs<LW, IDB>::value) {
    uint32_t high = 0;  // any id of 16 or more in this thread's vectors
#pragma unroll
    for (int j = 0; j < U; ++j) high |= (y[j].x | y[j].y | y[j].z | y[j].w) & 0xF0F0F0F0u;
    if (__all_sync(FULL_MASK, high == 0)) {
#pragma unroll
      for (int j = 0; j < U; ++j) encode_vec_pairs<LW, IMM>(d + j * REGS_PER_VEC, y[j], t, lanebase, one);
    } else {
#pragma unroll
      for (int j = 0; j < U; ++j) encode_vec_shift<LW>(d + j * REGS_PER_VEC, y[j], km);
    }
  } else if constexpr (IDB == 4) {
#pragma unroll
    for (int j = 0; j < U; ++j) encode_vec_ids32<LW>(d + j * REGS_PER_VEC, y[j], km);
  } else {
#pragma unroll
    for (int j = 0; j < U; ++j) encode_vec<LW, IDB, IMM>(d + j * REGS_PER_VEC, y[j], t, lanebase, one);
  }
  acc.add_trip(d, one);
}

// Block 0's consumer threads 0..15 and 32..47 count the head and tail ids
// (fewer than 16 each, outside the 16-byte vectors): the encoded word of
// the thread's id, or 0.
template <int LW, int IDB>
__device__ __forceinline__ uint32_t head_tail_word(const OnehotArgs& a) {
  const unsigned t = threadIdx.x;
  uint32_t id = 0xFFFFFFFFu;
  if (t < a.head_ids) id = load_id<IDB>(a.head + t * IDB);
  if (t >= 32 && t - 32 < a.tail_ids) id = load_id<IDB>(a.tail + (t - 32) * IDB);
  return id < a.k ? 1u << id : 0u;
}

// The consumer warps' loop over this CTA's chunks; returns the chunks it
// finished.  A wait that runs out sets the error word and ends the loop (the
// producer's own bounded waits end it there).
template <int LW, int IDB, uint32_t IMM>
__device__ __forceinline__ uint32_t ring_consume(const OnehotArgs& a, const uint8_t* ring, RingCtl* ctl,
                                                 uint32_t my_chunks, LutRef<IMM> t, uint32_t lanebase,
                                                 RingAcc<LW, IDB>& acc) {
  constexpr uint32_t TRIP = RingTrip<LW, IDB>::U * RING_CWARPS * 32;  // vectors per trip; divides a chunk
  constexpr uint32_t CV = RING_CHUNK / 16;                       // vectors per chunk
  const uint32_t one = a.one, lane = threadIdx.x & 31u;
  const uint32_t km = a.k >= 32 ? ~0u : (1u << a.k) - 1u;
  // Only the input's last chunk can be partial; it is this CTA's last chunk
  // if this CTA holds it.
  const uint64_t body_bytes = a.nvec * 16;
  const uint64_t nchunks = (body_bytes + RING_CHUNK - 1) / RING_CHUNK;
  const bool last_partial = body_bytes % RING_CHUNK != 0 && (nchunks - 1) % gridDim.x == blockIdx.x;
  const uint32_t full_chunks = last_partial ? my_chunks - 1 : my_chunks;
  uint32_t i = 0, s = 0, parity = 0;
  for (; i < my_chunks; ++i) {
    // every lane waits (each acquires the copied bytes); the verdict is made
    // warp-uniform so the warp leaves the loop together
    if (!__all_sync(FULL_MASK, mbar_wait_bounded(&ctl->full[s], parity, WAIT_LIMIT_NS))) {
      if (lane == 0) {
        atomicOr(a.err, ERR_BIT_TIMEOUT_FULL);
        atomicExch(&ctl->abort, 1u);
      }
      break;
    }
    const uint4* sv = reinterpret_cast<const uint4*>(ring + size_t(s) * RING_CHUNK);
    if (i < full_chunks) {
#pragma unroll
      for (uint32_t base = 0; base < CV; base += TRIP)
        ring_trip<LW, IDB, IMM, false>(sv, base, CV, t, lanebase, one, km, acc);
    } else {
      const uint32_t nv = uint32_t(body_bytes % RING_CHUNK) / 16u;
      for (uint32_t base = 0; base < nv; base += TRIP) ring_trip<LW, IDB, IMM, true>(sv, base, nv, t, lanebase, one, km, acc);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&ctl->empty[s]);
    if (++s == RING_STAGES) {
      s = 0;
      parity ^= 1u;
    }
  }
  return i;
}

template <int LW, int IDB>
__global__ void __launch_bounds__(RING_THREADS, 1) onehot_ring_kernel(OnehotArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];  // the only shared memory of this kernel
  uint8_t* lut = smem;
  const uint8_t* ring = smem + LUT_BYTES;
  RingCtl* ctl = reinterpret_cast<RingCtl*>(smem + LUT_BYTES + size_t(RING_STAGES) * RING_CHUNK);
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint64_t body_bytes = a.nvec * 16;
  const uint64_t nchunks = (body_bytes + RING_CHUNK - 1) / RING_CHUNK;
  const uint32_t my_chunks =
      blockIdx.x < nchunks ? uint32_t((nchunks - 1 - blockIdx.x) / gridDim.x + 1) : 0u;

  if (threadIdx.x == 0) {
    for (uint32_t s = 0; s < RING_STAGES; ++s) {
      mbar_init(&ctl->full[s], 1);
      mbar_init(&ctl->empty[s], RING_CWARPS);
    }
    ctl->issued = 0;
    ctl->abort = 0;
    mbar_fence_init();
  }
  if constexpr (IDB < 4) {  // 32-bit ids need no table
    for (uint32_t e = warp; e < 256u; e += RING_CWARPS + 1) {
      const bool pairs = RingPairs<LW, IDB>::value;
      *reinterpret_cast<uint32_t*>(lut + e * LUT_ROW + lane * 4u) = pairs ? pair_lo<LW>(e, a.k) : lut_lo<LW>(e, a.k);
      *reinterpret_cast<uint32_t*>(lut + e * LUT_ROW + 128u + lane * 4u) =
          pairs ? pair_hi<LW>(e, a.k) : lut_hi<LW>(e, a.k);
    }
  }
  __syncthreads();

  uint32_t vsum = 0;  // the warp's counts, lane i: position i >> (5 - log2 LW)
  if (warp == RING_CWARPS) {
    if (lane == 0) {  // producer: one lane issues every copy
      uint32_t i = 0;
      for (; i < my_chunks; ++i) {
        const uint32_t s = i % RING_STAGES, use = i / RING_STAGES;
        if (use > 0 && !mbar_wait_bounded(&ctl->empty[s], (use - 1) & 1u, WAIT_LIMIT_NS)) {
          atomicOr(a.err, ERR_BIT_TIMEOUT_EMPTY);
          atomicExch(&ctl->abort, 1u);
          break;
        }
        if (*((volatile uint32_t*)&ctl->abort)) break;
        const uint64_t off = (blockIdx.x + uint64_t(i) * gridDim.x) * RING_CHUNK;
        const uint64_t rem = body_bytes - off;
        const uint32_t bytes = rem < RING_CHUNK ? uint32_t(rem) : RING_CHUNK;
        mbar_arrive_expect_tx(&ctl->full[s], bytes);
        bulk_g2s(smem + LUT_BYTES + size_t(s) * RING_CHUNK, reinterpret_cast<const uint8_t*>(a.body) + off, bytes,
                 &ctl->full[s]);
      }
      ctl->issued = i;
    }
  } else {
    // Every lookup depends on lanebase, made after the barrier above.
    uint32_t lanebase;
    asm volatile("mov.u32 %0, %1;" : "=r"(lanebase) : "r"(lane * 4u));
    const uint32_t base = static_cast<uint32_t>(__cvta_generic_to_shared(lut));
    RingAcc<LW, IDB> acc;
    const uint32_t done =
        base == LUT_USUAL_BASE
            ? ring_consume<LW, IDB, LUT_USUAL_BASE>(a, ring, ctl, my_chunks, LutRef<LUT_USUAL_BASE>{base},
                                                    lanebase, acc)
            : ring_consume<LW, IDB, 0>(a, ring, ctl, my_chunks, LutRef<0>{base}, lanebase, acc);
    if (lane == 0) ctl->consumed[warp] = done;
    if (blockIdx.x == 0) acc.add_word(head_tail_word<LW, IDB>(a));  // every lane of the warp
    vsum = acc.finish();
  }
  __syncthreads();
  // After an abort, wait (bounded) for copies still in flight before the
  // shared memory they target goes away.
  if (ctl->abort && threadIdx.x == 0) {
    uint32_t lo = ctl->issued;
    for (int w = 0; w < RING_CWARPS; ++w) lo = ctl->consumed[w] < lo ? ctl->consumed[w] : lo;
    for (uint32_t i = lo; i < ctl->issued; ++i) {
      if (!mbar_wait_bounded(&ctl->full[i % RING_STAGES], (i / RING_STAGES) & 1u, WAIT_LIMIT_NS)) {
        atomicOr(a.err, ERR_BIT_TIMEOUT_DRAIN);
        break;
      }
    }
  }
  // block reduction in the table's memory; the producer warp holds no counts
  reduce_warp_sums_in<LW, RING_CWARPS>(reinterpret_cast<uint32_t*>(lut), vsum, a, &ctl->last);
}

template <int LW, int IDB>
static int launch_onehot_ring(const DeviceState& st, OnehotArgs a, cudaStream_t stream) {
  auto kern = onehot_ring_kernel<LW, IDB>;
  if (const cudaError_t e = ensure_dynamic_smem<onehot_ring_kernel<LW, IDB>>(st.device, int(RING_SMEM)))
    return cuda_fail(e);
  const uint64_t nchunks = (a.nvec * 16 + RING_CHUNK - 1) / RING_CHUNK;
  uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(uint64_t(st.sms), nchunks));
  // a consumer warp's u32 partials stay exact: at most 2^31 ids per warp
  grid = std::max(grid, std::min<uint64_t>(nchunks, ((a.nvec * 16) >> 35) + 1));
  a.store = grid == 1 ? 1u : 0u;
  a.publish = grid > 1 && a.acc && a.arrived ? 1u : 0u;
  if (grid > 1 && !a.publish) {
    const cudaError_t e = cudaMemsetAsync(a.counts, 0, sizeof(unsigned long long) * a.k, stream);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  kern<<<unsigned(grid), RING_THREADS, RING_SMEM, stream>>>(a);
  note_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? POSPOPCNT_OK : cuda_fail(e);
}

template <int IDB, int LW>
static int launch_onehot(const DeviceState& st, OnehotArgs a, cudaStream_t stream) {
  constexpr int T = 256;
  constexpr int U = IdTrip<IDB, LW>::U;
  auto kern = onehot_kernel<IDB, LW, T>;
  const int occ = resident_blocks(reinterpret_cast<const void*>(kern), st.device, T, 0);
  const uint64_t cap = uint64_t(st.sms) * uint64_t(occ);
  const uint64_t need = (a.nvec + uint64_t(U) * T - 1) / (uint64_t(U) * T);
  uint64_t grid = std::max<uint64_t>(1, std::min(cap, need));
  grid = std::max<uint64_t>(grid, ((a.nvec * 16) >> 31) + 1);  // per-CTA u32 partials stay exact
  a.store = grid == 1 ? 1u : 0u;
  a.publish = grid > 1 && a.acc && a.arrived ? 1u : 0u;
  if (grid > 1 && !a.publish) {
    const cudaError_t e = cudaMemsetAsync(a.counts, 0, sizeof(unsigned long long) * a.k, stream);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  kern<<<unsigned(grid), T, 0, stream>>>(a);
  note_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? POSPOPCNT_OK : cuda_fail(e);
}

template <int IDB>
static int launch_onehot_idb(const DeviceState& st, const OnehotArgs& a, cudaStream_t stream) {
  if (a.nvec * 16 >= ring_min_bytes<IDB>()) {
    if (a.k <= 8) return launch_onehot_ring<8, IDB>(st, a, stream);
    if (a.k <= 16) return launch_onehot_ring<16, IDB>(st, a, stream);
    return launch_onehot_ring<32, IDB>(st, a, stream);
  }
  if constexpr (IDB <= 2) {
    if (a.k <= 8) return launch_onehot_lut<8, IDB>(st, a, stream);
    if (a.k <= 16) return launch_onehot_lut<16, IDB>(st, a, stream);
    return launch_onehot_lut<32, IDB>(st, a, stream);
  } else {
    if (a.k <= 8) return launch_onehot<IDB, 8>(st, a, stream);
    if (a.k <= 16) return launch_onehot<IDB, 16>(st, a, stream);
    return launch_onehot<IDB, 32>(st, a, stream);
  }
}

}  // namespace ppc

extern "C" int pospopcnt_onehot_counts(const void* d_ids, size_t n, int id_bytes, int k, uint64_t* d_counts,
                                       cudaStream_t stream) {
  using namespace ppc;
  if (id_bytes != 1 && id_bytes != 2 && id_bytes != 4) return POSPOPCNT_ERR_INVALID;
  if (k < 1 || k > 32 || !d_counts || (n > 0 && !d_ids)) return POSPOPCNT_ERR_INVALID;
  if (reinterpret_cast<uintptr_t>(d_ids) % uintptr_t(id_bytes) != 0 || reinterpret_cast<uintptr_t>(d_counts) % 8)
    return POSPOPCNT_ERR_MISALIGNED;
  if (n > (size_t(1) << 42) / size_t(id_bytes)) return POSPOPCNT_ERR_TOO_LARGE;
  int rc = POSPOPCNT_OK;
  DeviceState* st = current_state(&rc);
  if (!st) return rc;
  const Split sp = plan_split(8 * id_bytes, reinterpret_cast<uint64_t>(d_ids), n);
  const uint8_t* base = static_cast<const uint8_t*>(d_ids);
  OnehotArgs a;
  a.head = base;
  a.head_ids = uint32_t(sp.head_words);
  a.body = reinterpret_cast<const uint4*>(base + sp.head_words * size_t(id_bytes));
  a.nvec = sp.body_vectors;
  a.tail = base + sp.head_words * size_t(id_bytes) + sp.body_vectors * 16;
  a.tail_ids = uint32_t(sp.tail_words);
  a.counts = reinterpret_cast<unsigned long long*>(d_counts);
  a.k = uint32_t(k);
  a.store = 0;
  a.one = 1;
  a.err = st->d_err;
  const PlainAcc acc = plain_acc_for(*st, stream);
  a.publish = 0;
  a.acc = acc.acc;
  a.arrived = acc.arrived;
  if (n == 0) {
    const cudaError_t e = cudaMemsetAsync(d_counts, 0, sizeof(uint64_t) * size_t(k), stream);
    return e == cudaSuccess ? POSPOPCNT_OK : cuda_fail(e);
  }
  switch (id_bytes) {
    case 1: return launch_onehot_idb<1>(*st, a, stream);
    case 2: return launch_onehot_idb<2>(*st, a, stream);
    default: return launch_onehot_idb<4>(*st, a, stream);
  }
}
