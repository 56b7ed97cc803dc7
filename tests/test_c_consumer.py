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
