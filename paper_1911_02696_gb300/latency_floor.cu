// Launch-to-host latency floors of this GPU, the reference points for the
// serving runtime's completion path.  A stand-alone program (not part of the
// library): bench.py's `latency_floor` workload builds and runs it.
//
// Each line times, from just before the launch call to the moment the host
// sees the result, 2000 repetitions after as many warm-up ones:
//   empty kernel + stream synchronize;
//   a one-block kernel that fences at system scope and sets a flag in
//   mapped host memory, the host spinning on the flag (16-byte and 4 KiB
//   kernel parameters);
//   the same with 8 blocks, the last one to finish setting the flag;
//   memset + kernel + 128-byte device-to-host copy + event poll;
//   the launch call alone (host time);
//   the flag kernel launched on 16 streams in turn (the serving slots);
//   a one-block kernel that first reads a cold 64 KiB slice of a 4 GiB
//   buffer with 8 warps (a median small serving job), then sets the flag.
// Host spins give up after 1 s.  Output: one line per path, then the CUDA
// status.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cstdio>
#include <vector>

struct SmallArgs {
  unsigned* flag;
  unsigned v;
};
struct BigArgs {  // about 4 KiB of kernel parameters
  unsigned* flag;
  unsigned v;
  uint64_t pad[500];
};

__global__ void k_empty() {}

__global__ void k_flag_small(SmallArgs a) {
  if (threadIdx.x == 0) {
    __threadfence_system();
    *reinterpret_cast<volatile unsigned*>(a.flag) = a.v;
  }
}

__global__ void k_flag_big(BigArgs a) {
  if (threadIdx.x == 0) {
    __threadfence_system();
    *reinterpret_cast<volatile unsigned*>(a.flag) = a.v + unsigned(a.pad[7] & 0u);
  }
}

__global__ void k_flag_grid(SmallArgs a, unsigned long long* ctr) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(ctr, 1ull) == gridDim.x - 1) {
      *ctr = 0;
      __threadfence_system();
      *reinterpret_cast<volatile unsigned*>(a.flag) = a.v;
    }
  }
}

// 8 warps read a 64 KiB slice (16-byte loads), fold it into one word,
// then thread 0 publishes: the shape of a median small serving job.
__global__ void k_read_flag(const uint4* src, SmallArgs a, unsigned* sink) {
  __shared__ unsigned red[256];
  unsigned acc = 0;
  for (int i = threadIdx.x; i < 4096; i += 256) {
    const uint4 x = src[i];
    acc ^= x.x ^ x.y ^ x.z ^ x.w;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = 0;
    for (int i = 0; i < 256; ++i) t ^= red[i];
    *sink = t;
    __threadfence_system();
    *reinterpret_cast<volatile unsigned*>(a.flag) = a.v;
  }
}

static double now() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static bool spin(volatile unsigned* f, unsigned v) {
  const double t0 = now();
  while (*f != v)
    if (now() - t0 > 1.0) return false;
  return true;
}

static void report(const char* name, std::vector<double>& us) {
  std::sort(us.begin(), us.end());
  std::printf("%s|%.2f|%.2f|%.2f|%.2f\n", name, us[us.size() / 2], us[us.size() * 9 / 10], us[us.size() * 99 / 100],
              us[0]);
}

int main() {
  if (cudaSetDevice(0) != cudaSuccess) return 1;
  cudaStream_t s;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  unsigned* h_flag = nullptr;
  if (cudaHostAlloc(reinterpret_cast<void**>(&h_flag), 64, cudaHostAllocMapped) != cudaSuccess) return 1;
  unsigned* d_flag = nullptr;
  cudaHostGetDevicePointer(reinterpret_cast<void**>(&d_flag), h_flag, 0);
  unsigned long long* ctr = nullptr;
  cudaMalloc(&ctr, 8);
  cudaMemset(ctr, 0, 8);
  unsigned long long* d_small = nullptr;
  cudaMalloc(&d_small, 256);
  unsigned long long* h_small = nullptr;
  cudaHostAlloc(reinterpret_cast<void**>(&h_small), 256, 0);
  cudaEvent_t ev;
  cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  cudaStream_t rr[16];
  for (auto& q : rr) cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking);
  const size_t pool_bytes = size_t(4) << 30;  // 4 GiB: 64 KiB slices at spread offsets stay cold
  uint8_t* pool = nullptr;
  if (cudaMalloc(&pool, pool_bytes) != cudaSuccess) return 1;
  cudaMemset(pool, 0x5A, pool_bytes);
  unsigned* sink = nullptr;
  cudaMalloc(&sink, 4);
  *h_flag = 0;
  const int N = 2000;
  unsigned v = 0;
  bool ok = true;
  for (int rep = 0; rep < 2 && ok; ++rep) {  // the first pass warms up
    std::vector<double> a, b, c, d, e, f, g, h;
    for (int i = 0; i < N && ok; ++i) {
      double t0 = now();
      k_empty<<<1, 32, 0, s>>>();
      cudaStreamSynchronize(s);
      a.push_back((now() - t0) * 1e6);
      SmallArgs sm{d_flag, ++v};
      t0 = now();
      k_flag_small<<<1, 32, 0, s>>>(sm);
      ok = ok && spin(h_flag, v);
      b.push_back((now() - t0) * 1e6);
      BigArgs bg{};
      bg.flag = d_flag;
      bg.v = ++v;
      t0 = now();
      k_flag_big<<<1, 32, 0, s>>>(bg);
      ok = ok && spin(h_flag, v);
      c.push_back((now() - t0) * 1e6);
      SmallArgs sg{d_flag, ++v};
      t0 = now();
      k_flag_grid<<<8, 256, 0, s>>>(sg, ctr);
      ok = ok && spin(h_flag, v);
      d.push_back((now() - t0) * 1e6);
      t0 = now();
      cudaMemsetAsync(d_small, 0, 128, s);
      k_empty<<<1, 32, 0, s>>>();
      cudaMemcpyAsync(h_small, d_small, 128, cudaMemcpyDeviceToHost, s);
      cudaEventRecord(ev, s);
      while (cudaEventQuery(ev) == cudaErrorNotReady) {
      }
      e.push_back((now() - t0) * 1e6);
      t0 = now();
      k_empty<<<1, 32, 0, s>>>();
      f.push_back((now() - t0) * 1e6);
      cudaStreamSynchronize(s);
      SmallArgs sr{d_flag, ++v};
      t0 = now();
      k_flag_small<<<1, 32, 0, rr[i % 16]>>>(sr);
      ok = ok && spin(h_flag, v);
      g.push_back((now() - t0) * 1e6);
      // slice i: offsets 2 MiB + 64 KiB apart wrap around the 4 GiB pool
      const size_t off = (size_t(i) * ((size_t(2) << 20) + 65536)) % (pool_bytes - 65536);
      SmallArgs sd{d_flag, ++v};
      t0 = now();
      k_read_flag<<<1, 256, 0, s>>>(reinterpret_cast<const uint4*>(pool + off), sd, sink);
      ok = ok && spin(h_flag, v);
      h.push_back((now() - t0) * 1e6);
    }
    if (ok && rep == 1) {
      report("empty kernel + stream synchronize", a);
      report("flag kernel, 16 B parameters, host spin", b);
      report("flag kernel, 4 KiB parameters, host spin", c);
      report("8-block kernel, last block sets the flag", d);
      report("memset + kernel + 128 B copy to host + event poll", e);
      report("launch call alone (host time)", f);
      report("flag kernel on 16 streams in turn, host spin", g);
      report("64 KiB cold read by 8 warps, then the flag", h);
    }
  }
  const cudaError_t err = cudaDeviceSynchronize();
  std::printf("status|%d|%s\n", int(err), ok ? "ok" : "flag spin gave up");
  return err == cudaSuccess && ok ? 0 : 1;
}
