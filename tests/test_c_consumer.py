"""A plain C11 program includes the public header and links the library:
the header is valid C (not only C++), every declared function resolves at
link time, and the argument checks answer with the documented status codes
(no device is touched: every call below fails validation first)."""
import os
import shutil
import subprocess
import tempfile

import pytest

from paper_1911_02696_gb300 import _build

C_PROGRAM = r"""
#include <stdio.h>
#include "pospopcnt.h"

int main(void) {
  uint64_t* good = (uint64_t*)(uintptr_t)(1u << 20);  /* never dereferenced */
  int fails = 0;
  fails += pospopcnt_u16(NULL, 5, good, 0) != POSPOPCNT_ERR_INVALID;
  fails += pospopcnt_u16((const void*)((uintptr_t)good + 1), 5, good, 0) != POSPOPCNT_ERR_MISALIGNED;
  fails += pospopcnt_u64((const void*)((uintptr_t)good + 4), 5, good, 0) != POSPOPCNT_ERR_MISALIGNED;
  fails += pospopcnt_count(12, POSPOPCNT_KERNEL_AUTO, good, 5, good, 0) != POSPOPCNT_ERR_INVALID;
  fails += pospopcnt_batched(good, (const int64_t*)good, 0, 16, good, 0) != POSPOPCNT_OK;
  fails += pospopcnt_onehot_counts(good, 5, 3, 8, good, 0) != POSPOPCNT_ERR_INVALID;
  size_t h = 0, b = 0, t = 0;
  fails += pospopcnt_plan_split(16, 2, 100, &h, &b, &t) != POSPOPCNT_OK || h != 7 || b != 11 || t != 5;
  pospopcnt_config cfg = {POSPOPCNT_KERNEL_TMA, 0, 0, 0, 3, 65536, POSPOPCNT_FLAG_EVICT_FIRST};
  (void)cfg;
  printf("%s %d\n", pospopcnt_strerror(POSPOPCNT_ERR_TIMEOUT), fails);
  return fails;
}
"""


def test_header_is_c_and_links():
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc unavailable")
    lib = _build.build()
    cuda_inc = "/usr/local/cuda/include"
    if not os.path.exists(os.path.join(cuda_inc, "cuda_runtime_api.h")):
        pytest.skip("CUDA headers unavailable")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "consumer.c")
        exe = os.path.join(d, "consumer")
        open(src, "w").write(C_PROGRAM)
        subprocess.check_call([gcc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(_build.ROOT, "include"),
                               "-I", cuda_inc, src, "-o", exe, lib, f"-Wl,-rpath,{os.path.dirname(lib)}"])
        r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
        assert r.returncode == 0, r.stdout + r.stderr
        assert r.stdout.split()[-1] == "0"


C_GPU_PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <cuda_runtime_api.h>
#include "pospopcnt.h"

/* Reads a whole binary file into malloc'd memory. */
static void* slurp(const char* path, size_t* n) {
  FILE* f = fopen(path, "rb");
  if (!f) return NULL;
  fseek(f, 0, SEEK_END);
  *n = (size_t)ftell(f);
  fseek(f, 0, SEEK_SET);
  void* p = malloc(*n ? *n : 1);
  if (fread(p, 1, *n, f) != *n) { fclose(f); free(p); return NULL; }
  fclose(f);
  return p;
}

static void print_row(const char* tag, const uint64_t* v, size_t k) {
  printf("%s", tag);
  for (size_t i = 0; i < k; ++i) printf(" %llu", (unsigned long long)v[i]);
  printf("\n");
}

#define CHECK(x) do { int rc_ = (x); if (rc_ != POSPOPCNT_OK) { \
  printf("FAIL %s: %s\n", #x, pospopcnt_strerror(rc_)); return 1; } } while (0)
#define CUDA(x) do { if ((x) != cudaSuccess) { printf("FAIL %s\n", #x); return 1; } } while (0)

int main(int argc, char** argv) {
  if (argc != 4) return 2;
  size_t nw = 0, no = 0, ni = 0;
  unsigned char* words = (unsigned char*)slurp(argv[1], &nw);   /* u16 words */
  int64_t* offsets = (int64_t*)slurp(argv[2], &no);             /* nseg + 1 */
  unsigned char* ids = (unsigned char*)slurp(argv[3], &ni);     /* u8 ids */
  if (!words || !offsets || !ids) return 3;
  const size_t nseg = no / 8 - 1;
  unsigned char *d_words, *d_ids;
  int64_t* d_off;
  uint64_t *d_counts, *d_rows;
  cudaStream_t s;
  CUDA(cudaStreamCreate(&s));
  CUDA(cudaMalloc((void**)&d_words, nw + 16));
  CUDA(cudaMalloc((void**)&d_ids, ni));
  CUDA(cudaMalloc((void**)&d_off, no));
  CUDA(cudaMalloc((void**)&d_counts, 64 * sizeof(uint64_t)));
  CUDA(cudaMalloc((void**)&d_rows, nseg * 16 * sizeof(uint64_t)));
  /* the words start 2 bytes past an allocation boundary: a ragged head */
  CUDA(cudaMemcpy(d_words + 2, words, nw, cudaMemcpyHostToDevice));
  CUDA(cudaMemcpy(d_ids, ids, ni, cudaMemcpyHostToDevice));
  CUDA(cudaMemcpy(d_off, offsets, no, cudaMemcpyHostToDevice));
  uint64_t h[64];

  CHECK(pospopcnt_u16(d_words + 2, nw / 2, d_counts, s));
  CUDA(cudaMemcpyAsync(h, d_counts, 16 * 8, cudaMemcpyDeviceToHost, s));
  CUDA(cudaStreamSynchronize(s));
  print_row("u16", h, 16);

  CHECK(pospopcnt_popcount(d_words + 2, nw, d_counts, s));
  CUDA(cudaMemcpyAsync(h, d_counts, 8, cudaMemcpyDeviceToHost, s));
  CUDA(cudaStreamSynchronize(s));
  print_row("popcount", h, 1);

  CHECK(pospopcnt_onehot_counts(d_ids, ni, 1, 20, d_counts, s));
  CUDA(cudaMemcpyAsync(h, d_counts, 20 * 8, cudaMemcpyDeviceToHost, s));
  CUDA(cudaStreamSynchronize(s));
  print_row("onehot20", h, 20);

  uint64_t* rows = (uint64_t*)malloc(nseg * 16 * sizeof(uint64_t));
  CHECK(pospopcnt_batched(d_words + 2, d_off, nseg, 16, d_rows, s));
  CUDA(cudaMemcpyAsync(rows, d_rows, nseg * 16 * 8, cudaMemcpyDeviceToHost, s));
  CUDA(cudaStreamSynchronize(s));
  for (size_t r = 0; r < nseg; ++r) print_row("row", rows + 16 * r, 16);

  CHECK(pospopcnt_batched_noalloc(d_words + 2, d_off, nseg, 16, d_rows, s));
  CUDA(cudaMemcpyAsync(rows, d_rows, nseg * 16 * 8, cudaMemcpyDeviceToHost, s));
  CUDA(cudaStreamSynchronize(s));
  for (size_t r = 0; r < nseg; ++r) print_row("nrow", rows + 16 * r, 16);
  CHECK(pospopcnt_check_device_error(s));

  CHECK(pospopcnt_count_host(16, words, nw / 2, h));  /* pageable host memory */
  print_row("host", h, 16);

  CHECK(pospopcnt_release_stream(s));
  CUDA(cudaStreamDestroy(s));
  printf("done\n");
  return 0;
}
"""


@pytest.mark.gpu
def test_c_program_on_the_gpu():
    """A C11 program with its own CUDA runtime allocates device memory and
    calls the library (plain u16 count at a 2-byte offset, popcount, one-hot
    histogram, batched and allocation-free batched rows, host-buffer count);
    every result it prints equals the oracle on the same data."""
    import numpy as np

    import oracle
    import synth
    gcc = shutil.which("gcc")
    cuda = "/usr/local/cuda"
    if not gcc or not os.path.exists(os.path.join(cuda, "include", "cuda_runtime_api.h")):
        pytest.skip("gcc or CUDA headers unavailable")
    lib = _build.build()
    words = synth.uniform_bits(51, (3 << 20) + 5, 16)
    lens = synth.log_uniform_lengths(52, 300, max_len=1 << 14)
    off = synth.offsets_from_lengths(lens, start=3)
    assert off[-1] <= words.size
    ids = synth.categorical_ids(53, (5 << 20) + 3, synth.zipf_cdf(24), np.uint8)
    with tempfile.TemporaryDirectory() as d:
        paths = [os.path.join(d, n) for n in ("words.bin", "off.bin", "ids.bin")]
        words.tofile(paths[0])
        off.astype(np.int64).tofile(paths[1])
        ids.tofile(paths[2])
        src, exe = os.path.join(d, "gpu_consumer.c"), os.path.join(d, "gpu_consumer")
        open(src, "w").write(C_GPU_PROGRAM)
        libdir = os.path.join(cuda, "lib64")
        subprocess.check_call([gcc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(_build.ROOT, "include"),
                               "-I", os.path.join(cuda, "include"), src, "-o", exe, lib, "-L", libdir, "-lcudart",
                               f"-Wl,-rpath,{os.path.dirname(lib)}", f"-Wl,-rpath,{libdir}"])
        r = subprocess.run([exe, *paths], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.rstrip().endswith("done"), r.stdout[-2000:] + r.stderr[-2000:]
    out = {}
    for line in r.stdout.splitlines():
        tag, *vals = line.split()
        out.setdefault(tag, []).append(np.array([int(v) for v in vals], dtype=np.uint64))
    ref16 = oracle.pospopcnt(words, 16)
    assert np.array_equal(out["u16"][0], ref16)
    assert np.array_equal(out["host"][0], ref16)
    assert int(out["popcount"][0][0]) == int(ref16.sum())
    assert np.array_equal(out["onehot20"][0], oracle.onehot_counts(ids, 20))
    rows = oracle.pospopcnt_segments(words, off, 16)
    assert np.array_equal(np.stack(out["row"]), rows)
    assert np.array_equal(np.stack(out["nrow"]), rows)
