// Fused one-hot encode + positional count: categorical ids -> frequency
// histogram without materialising the one-hot words.
//
// The paper's motivation (§1, Table 1) is exactly this pipeline: values are
// one-hot encoded and the positional population count of the encoded words
// is the histogram.  Here each thread loads 16-byte vectors of ids, builds
// the one-hot words directly in registers -- with lanes of LW = 8, 16 or 32
// bits (the smallest that holds k positions), 32/LW ids share one 32-bit
// register -- and feeds those registers through the same carry-save circuit
// F_4 and popc flush as the plain count.  Ids >= k encode to the empty word.
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

template <int IDB, int LW, int NTHREADS>
__global__ void __launch_bounds__(NTHREADS) onehot_kernel(OnehotArgs a) {
  constexpr int IDS_PER_VEC = 16 / IDB;
  constexpr int IDS_PER_REG = 32 / LW;
  constexpr int REGS_PER_VEC = IDS_PER_VEC / IDS_PER_REG;
  constexpr int U = 16 / REGS_PER_VEC;  // vectors per trip: 16 registers, circuit F_4
  const uint32_t k = a.k;
  // lane q of a register holds the one-hot bit of its id at bit q*LW + id;
  // the mask keeps bits q*LW .. q*LW + k - 1 (ids >= k, which could spill
  // into the next lane, are dropped)
  const uint32_t km = k >= 32 ? 0xFFFFFFFFu : (1u << k) - 1u;
  uint32_t lane_mask_q[IDS_PER_REG];
#pragma unroll
  for (int q = 0; q < IDS_PER_REG; ++q) lane_mask_q[q] = km << (q * LW);
  uint32_t B[4] = {0, 0, 0, 0};
  uint32_t top[LW];
#pragma unroll
  for (int p = 0; p < LW; ++p) top[p] = 0;
  const uint64_t stride = uint64_t(gridDim.x) * NTHREADS;
  for (uint64_t v = uint64_t(blockIdx.x) * NTHREADS + threadIdx.x; v < a.nvec; v += U * stride) {
    uint32_t d[16];
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
    flush<LW>(top, Circuit<4>::run(d, B));
  }
  uint32_t c[LW];
  finalize<LW, 4>(c, top, B);
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
  block_reduce_add<LW, NTHREADS / 32>(c, a.counts, a.store != 0, int(k));
}

template <int IDB, int LW>
static int launch_onehot(const DeviceState& st, OnehotArgs a, cudaStream_t stream) {
  constexpr int T = 256;
  constexpr int U = 16 / ((16 / IDB) / (32 / LW));
  auto kern = onehot_kernel<IDB, LW, T>;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, T, 0) != cudaSuccess || occ < 1) occ = 1;
  const uint64_t cap = uint64_t(st.sms) * uint64_t(occ);
  const uint64_t need = (a.nvec + uint64_t(U) * T - 1) / (uint64_t(U) * T);
  uint64_t grid = std::max<uint64_t>(1, std::min(cap, need));
  grid = std::max<uint64_t>(grid, ((a.nvec * 16) >> 31) + 1);  // per-CTA u32 partials stay exact
  a.store = grid == 1 ? 1u : 0u;
  if (grid > 1) {
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
  if (a.k <= 8) return launch_onehot<IDB, 8>(st, a, stream);
  if (a.k <= 16) return launch_onehot<IDB, 16>(st, a, stream);
  return launch_onehot<IDB, 32>(st, a, stream);
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
