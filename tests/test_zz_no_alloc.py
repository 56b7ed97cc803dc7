"""The allocation-free batched entry point (pospopcnt_batched_noalloc).

It exists for callers that cannot call cudaMalloc -- for example a process
whose device memory is owned by another runtime's pool allocator -- and keeps
its only scratch, the work-queue state, in a static device array.  This file
is collected last so that a run stopping at the first failure has already
run every other test.  The test calls the entry point through the C ABI
first (in a fresh process, before anything else in the library has
allocated its workspace), twice in a row on the same inputs, and compares
each result with the regular pospopcnt_batched entry point bit-exactly
(tolerance 0, the tolerance of every parity test here)."""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
import paper_1911_02696_gb300 as ppc  # noqa: E402

pytestmark = pytest.mark.gpu


def test_noalloc_batched_matches_batched_on_two_calls():
    lib = ppc.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rng = np.random.default_rng(2024)
    lens = rng.integers(0, 150000, size=700).astype(np.int64)
    lens[::9] = 0
    lens[1::11] = 1
    off = synth.offsets_from_lengths(lens, start=5)
    words = synth.segmented_one_hot(3, off, 16)
    buf = torch.zeros(len(words) * 2 + 512, dtype=torch.uint8, device=dev)
    x = buf[6: 6 + words.nbytes]  # 6 bytes past a 256-byte boundary
    x.copy_(torch.from_numpy(words.view(np.uint8)))
    d_off = torch.from_numpy(off).to(dev)
    nseg = off.size - 1
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
    ref = ppc.pospopcnt_batched(x, d_off, 16).cpu().numpy().view(np.uint64)
    for got in results:
        assert np.array_equal(got, ref)
    assert np.array_equal(ref.sum(axis=1), lens.astype(np.uint64))


def test_noalloc_rejects_bad_arguments():
    lib = ppc.load()
    P = ctypes.c_void_p
    assert lib.pospopcnt_batched_noalloc(P(1 << 20), P(1 << 20), 0, 16, P(1 << 20), None) == 0
    assert lib.pospopcnt_batched_noalloc(P(1 << 20), P(1 << 20), 4, 12, P(1 << 20), None) == 1
    assert lib.pospopcnt_batched_noalloc(None, P(1 << 20), 4, 16, P(1 << 20), None) == 1
    assert lib.pospopcnt_batched_noalloc(P((1 << 20) + 1), P(1 << 20), 4, 16, P(1 << 20), None) == 2
