"""The allocation-free batched entry point (pospopcnt_batched_noalloc).

Some callers cannot call cudaMalloc -- a process whose device memory is
owned by another runtime's pool allocator, or a service that must not
allocate once it runs -- so this entry point keeps its only scratch (the
work-queue state and the error word of one launch) in a static device array.

Two checks, both through the C ABI, both bit-exact against the oracle
(tolerance 0, the tolerance of every parity test here), each on two calls in
a row on the same inputs:

- in a child process whose first call into the library is this entry point:
  the library's count of device bytes it allocated stays 0 across both calls
  and the error check after them (and becomes non-zero once pospopcnt_init
  creates the workspace, so the count is live);
- in this process, after every other test has run (this file is collected
  last, so a run stopping at the first failure has run everything else),
  where it must also agree with pospopcnt_batched.
"""
import ctypes
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_1911_02696_gb300 as ppc  # noqa: E402

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _layout():
    """700 segments of up to 150,000 u16 words (empty and one-word segments
    among them), one-hot with a per-segment rotation, starting at word 5."""
    rng = np.random.default_rng(2024)
    lens = rng.integers(0, 150000, size=700).astype(np.int64)
    lens[::9] = 0
    lens[1::11] = 1
    off = synth.offsets_from_lengths(lens, start=5)
    words = synth.segmented_one_hot(3, off, 16)
    return lens, off, words


def _noalloc_twice(lib, x, d_off, nseg, dev):
    stream = torch.cuda.current_stream(dev)
    results = []
    for _ in range(2):
        out = torch.full((nseg, 16), -1, dtype=torch.int64, device=dev)
        rc = lib.pospopcnt_batched_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(d_off.data_ptr()),
                                           nseg, 16, ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, ppc.pospopcnt_strerror(rc)
        torch.cuda.synchronize()
        results.append(out.cpu().numpy().view(np.uint64).copy())
    return results


def _device_input(words, dev):
    buf = torch.zeros(words.nbytes + 512, dtype=torch.uint8, device=dev)
    x = buf[6: 6 + words.nbytes]  # 6 bytes past a 256-byte boundary
    x.copy_(torch.from_numpy(words.view(np.uint8)))
    return buf, x


_CHILD = textwrap.dedent("""
    import ctypes, sys
    import numpy as np
    import torch
    sys.path.insert(0, {root!r})
    sys.path.insert(0, {tests!r})
    import oracle
    import paper_1911_02696_gb300 as ppc
    import test_zz_no_alloc as t
    lib = ppc.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    lens, off, words = t._layout()
    buf, x = t._device_input(words, dev)
    d_off = torch.from_numpy(off).to(dev)
    nseg = off.size - 1
    ref = oracle.pospopcnt_segments(words, off, 16)
    torch.cuda.synchronize()
    assert lib.pospopcnt_device_bytes_allocated() == 0, "allocated before the first call"
    for got in t._noalloc_twice(lib, x, d_off, nseg, dev):
        assert np.array_equal(got, ref), "rows differ from the oracle"
    assert lib.pospopcnt_check_device_error(ctypes.c_void_p(0)) == 0
    held = lib.pospopcnt_device_bytes_allocated()
    assert held == 0, f"the allocation-free calls allocated {{held}} bytes"
    assert lib.pospopcnt_init(0) == 0
    assert lib.pospopcnt_device_bytes_allocated() > 0, "the allocation count does not see the workspace"
    print("child ok")
""")


def test_noalloc_first_call_in_fresh_process_allocates_nothing():
    tests = os.path.join(ROOT, "tests")
    code = _CHILD.format(root=ROOT, tests=tests)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0 and "child ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]


def test_noalloc_matches_oracle_and_batched_after_other_tests():
    lib = ppc.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    lens, off, words = _layout()
    buf, x = _device_input(words, dev)
    d_off = torch.from_numpy(off).to(dev)
    nseg = off.size - 1
    ref = oracle.pospopcnt_segments(words, off, 16)
    held = ppc.pospopcnt_device_bytes_allocated()
    results = _noalloc_twice(lib, x, d_off, nseg, dev)
    assert ppc.pospopcnt_device_bytes_allocated() == held
    assert ppc.pospopcnt_check_device_error() == 0
    batched = ppc.pospopcnt_batched(x, d_off, 16).cpu().numpy().view(np.uint64)
    for got in results:
        assert np.array_equal(got, ref)
        assert np.array_equal(got, batched)
    assert np.array_equal(ref.sum(axis=1), lens.astype(np.uint64))


def test_noalloc_rejects_bad_arguments():
    lib = ppc.load()
    P = ctypes.c_void_p
    assert lib.pospopcnt_batched_noalloc(P(1 << 20), P(1 << 20), 0, 16, P(1 << 20), None) == 0
    assert lib.pospopcnt_batched_noalloc(P(1 << 20), P(1 << 20), 4, 12, P(1 << 20), None) == 1
    assert lib.pospopcnt_batched_noalloc(None, P(1 << 20), 4, 16, P(1 << 20), None) == 1
    assert lib.pospopcnt_batched_noalloc(P((1 << 20) + 1), P(1 << 20), 4, 16, P(1 << 20), None) == 2
