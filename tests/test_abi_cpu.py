"""The C-ABI library on a machine without a GPU: it builds, loads, exports
every entry point the public header declares, and its host-side logic
(argument checks, head/body/tail planning, status strings) behaves.
Nothing here launches a kernel."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1911_02696_gb300 as ppc
from paper_1911_02696_gb300 import _build

HEADER_DIR = os.path.join(_build.ROOT, "include")


def declared_functions():
    names = []
    for h in sorted(os.listdir(HEADER_DIR)):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(pospopcnt_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_builds_and_loads():
    lib = ppc.load()
    assert os.path.exists(_build.LIB)
    assert isinstance(lib, ctypes.CDLL)


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert "pospopcnt_u16" in names and "pospopcnt_batched" in names and len(names) >= 15
    lib = ppc.load()
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True)
    if out.returncode == 0:
        exported = set(re.findall(r"\bT (pospopcnt_\w+)", out.stdout))
        assert set(names) <= exported


def test_no_undeclared_exports():
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("nm unavailable")
    exported = set(re.findall(r"\bT (pospopcnt_\w+)", out.stdout))
    assert exported <= set(declared_functions())


def _split_model(width, addr, n):
    wb = width // 8
    nbytes = n * wb
    head = min((16 - addr % 16) % 16, nbytes)
    body = (nbytes - head) // 16
    tail = nbytes - head - 16 * body
    return head // wb, body, tail // wb


@pytest.mark.parametrize("width", [8, 16, 32])
def test_plan_split(width):
    wb = width // 8
    rng = np.random.default_rng(width)
    cases = [(a, n) for a in range(0, 64, wb) for n in range(0, 70)]
    cases += [(int(rng.integers(0, 1 << 40)) // wb * wb, int(rng.integers(0, 1 << 34))) for _ in range(200)]
    for addr, n in cases:
        h, b, t = ppc.pospopcnt_plan_split(width, addr, n)
        assert (h, b, t) == _split_model(width, addr, n)
        assert h * wb + 16 * b + t * wb == n * wb
        assert h * wb < 16 and t * wb < 16
        if b:
            assert (addr + h * wb) % 16 == 0


def test_plan_split_rejects():
    with pytest.raises(ppc.PospopcntError) as e:
        ppc.pospopcnt_plan_split(16, 1, 10)
    assert e.value.status == 2
    with pytest.raises(ppc.PospopcntError) as e:
        ppc.pospopcnt_plan_split(12, 0, 10)
    assert e.value.status == 1


def test_argument_checks_need_no_device():
    """Every check below returns before any CUDA call."""
    lib = ppc.load()
    P = ctypes.c_void_p
    good = P(1 << 20)  # never dereferenced: the calls fail validation first
    # null input with n > 0, null counts
    assert lib.pospopcnt_u16(None, 5, good, None) == 1
    assert lib.pospopcnt_u8(good, 5, None, None) == 1
    # misaligned input / counts
    assert lib.pospopcnt_u16(P((1 << 20) + 1), 5, good, None) == 2
    assert lib.pospopcnt_u32(P((1 << 20) + 2), 5, good, None) == 2
    assert lib.pospopcnt_u16(good, 5, P((1 << 20) + 4), None) == 2
    # bad width / kernel / config
    assert lib.pospopcnt_count(12, 0, good, 5, good, None) == 1
    assert lib.pospopcnt_count(16, 9, good, 5, good, None) == 1
    assert lib.pospopcnt_count(16, -1, good, 5, good, None) == 1
    assert lib.pospopcnt_count_config(16, None, good, 5, good, None) == 1
    assert lib.pospopcnt_count_accumulate(7, good, 5, good, None) == 1
    # too large
    assert lib.pospopcnt_u8(good, 1 << 43, good, None) == 6
    # array popcount: null pointers, misaligned count
    assert lib.pospopcnt_popcount(None, 5, good, None) == 1
    assert lib.pospopcnt_popcount(good, 5, P((1 << 20) + 4), None) == 2
    # 64-bit words: 8-byte alignment
    assert lib.pospopcnt_u64(P((1 << 20) + 4), 5, good, None) == 2
    # batched: nseg == 0 is a no-op; null pointers; bad width; misalignment
    assert lib.pospopcnt_batched(None, None, 0, 16, None, None) == 0
    assert lib.pospopcnt_batched(good, None, 3, 16, good, None) == 1
    assert lib.pospopcnt_batched(good, good, 3, 24, good, None) == 1
    assert lib.pospopcnt_batched(good, good, 3, 64, good, None) == 1
    assert lib.pospopcnt_batched(P((1 << 20) + 1), good, 3, 16, good, None) == 2
    assert lib.pospopcnt_batched(good, P((1 << 20) + 4), 3, 16, good, None) == 2
    # batched launch configuration: bad width, out-of-range fields, null outputs
    cfg = ppc.BatchedConfig(16384, 0, 0)
    assert lib.pospopcnt_batched_get_config(12, ctypes.byref(cfg)) == 1
    assert lib.pospopcnt_batched_get_config(16, None) == 1
    for unit, bps, stages, vpl in ((2048, 0, 0, 0), (4096 + 64, 0, 0, 0), (2 << 20, 0, 0, 0), (4096, -1, 0, 0),
                                   (4096, 33, 0, 0), (4096, 0, 1, 0), (4096, 0, 5, 0), (4096, 0, 0, 2),
                                   (4096, 0, 0, 12), (4096, 0, 0, 32), (4096, 0, 4, 16)):
        bad = ppc.BatchedConfig(unit, bps, stages, vpl)
        assert lib.pospopcnt_batched_set_config(16, ctypes.byref(bad)) == 1, (unit, bps, stages, vpl)
    assert lib.pospopcnt_batched_set_config(64, None) == 1
    assert lib.pospopcnt_batched_autotune(good, good, 3, 16, good, None, None, None) == 1
    assert lib.pospopcnt_batched_autotune(good, good, 0, 16, good, ctypes.byref(cfg), None, None) == 1
    # one-hot counts: id width, k range, alignment
    assert lib.pospopcnt_onehot_counts(good, 5, 3, 16, good, None) == 1
    assert lib.pospopcnt_onehot_counts(good, 5, 1, 0, good, None) == 1
    assert lib.pospopcnt_onehot_counts(good, 5, 1, 33, good, None) == 1
    assert lib.pospopcnt_onehot_counts(P((1 << 20) + 1), 5, 2, 16, good, None) == 2
    # serving: null server / outputs
    assert lib.pospopcnt_server_run_trace_timed(None, 0, None, None, None, None, None, None, None, None) == 1
    # host path
    assert lib.pospopcnt_count_host(16, None, 4, good) == 1
    assert lib.pospopcnt_count_host(32, P((1 << 20) + 2), 4, good) == 2
    assert lib.pospopcnt_count_host(16, good, 4, None) == 1


def test_binding_rejects_host_tensors():
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        ppc.pospopcnt_u16(torch.zeros(8, dtype=torch.int16))


def test_status_strings():
    msgs = [ppc.pospopcnt_strerror(s) for s in range(7)]
    assert msgs[0] == "ok" and len(set(msgs)) == 7
    assert ppc.pospopcnt_strerror(99) == "unknown status"


def test_selftest_rejects_long_wait():
    lib = ppc.load()
    assert lib.pospopcnt_selftest_timeout(2_000_000_000, None) == 1
