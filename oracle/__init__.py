"""pospopcnt ORACLE -- test infrastructure only.

Plain scalar CPU implementation of the positional population count
(Klarqvist, Mula, Lemire, arXiv 1911.02696), written in C
(``pospopcnt_oracle.c``) and loaded with ctypes.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package; the product library never does, and shares no code
with it.

Functions (each cites the passage it follows in the C source):

* ``pospopcnt(words, width)`` -- the definition (Abstract, §1, §4 Fig. 6).
* ``pospopcnt_mt(words, width, nthreads)`` -- the same over threads.
* ``pospopcnt_segments(words, offsets, width)`` -- one definition per segment.
* ``csa_pospopcnt(words, width, N)`` -- the paper's Harley-Seal method
  (§2 Fig. 3-4, §3, §4.1), which reaches the definition exactly.
* ``csa_truth(which)`` / ``csa_circuit_size(N)`` -- Table 2 immediates and
  the 2^N - 1 circuit size of §2.
* ``popcount(data)`` -- the number of set bits (Abstract, §2): the single sum
  pospopcnt generalises.
* ``onehot_counts(ids, k)`` -- one-hot encode then count: the frequency
  histogram of §1 / Table 1.

Parity pins: tests/test_oracle_pins.py.  No function here is "parity
unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pospopcnt_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with plain gcc -O2 (no intrinsics, no -march)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               _SRC, "-o", tmp])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32, u64, vp, i64 = ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_long
            lib.oracle_pospopcnt.restype = i32
            lib.oracle_pospopcnt.argtypes = [i32, vp, u64, vp]
            lib.oracle_pospopcnt_add.restype = i32
            lib.oracle_pospopcnt_add.argtypes = [i32, vp, u64, vp]
            lib.oracle_pospopcnt_mt.restype = i32
            lib.oracle_pospopcnt_mt.argtypes = [i32, vp, u64, vp, i32]
            lib.oracle_pospopcnt_segments.restype = i32
            lib.oracle_pospopcnt_segments.argtypes = [i32, vp, vp, u64, vp]
            lib.oracle_csa_pospopcnt.restype = i64
            lib.oracle_csa_pospopcnt.argtypes = [i32, vp, u64, i32, vp]
            lib.oracle_csa_truth.restype = i32
            lib.oracle_csa_truth.argtypes = [i32]
            lib.oracle_csa_circuit_size.restype = i64
            lib.oracle_csa_circuit_size.argtypes = [i32]
            lib.oracle_popcount.restype = i32
            lib.oracle_popcount.argtypes = [vp, u64, vp]
            lib.oracle_onehot_counts.restype = i32
            lib.oracle_onehot_counts.argtypes = [vp, u64, i32, i32, vp]
            _lib = lib
    return _lib


def _as_bytes(words) -> np.ndarray:
    a = np.ascontiguousarray(words)
    return a


def _nwords(a: np.ndarray, width: int) -> int:
    nbytes = a.size * a.itemsize
    assert nbytes % (width // 8) == 0, "byte length is not a whole number of words"
    return nbytes // (width // 8)


def pospopcnt(words, width: int | None = None) -> np.ndarray:
    """counts[p] = number of words with bit p set (uint64[width])."""
    a = _as_bytes(words)
    width = width or a.itemsize * 8
    out = np.zeros(width, dtype=np.uint64)
    rc = _load().oracle_pospopcnt(width, a.ctypes.data, _nwords(a, width), out.ctypes.data)
    assert rc == 0, "oracle rejected the arguments"
    return out


def pospopcnt_add(words, counts: np.ndarray, width: int | None = None) -> np.ndarray:
    """The paper's accumulate form: counts += pospopcnt(words)."""
    a = _as_bytes(words)
    width = width or a.itemsize * 8
    assert counts.dtype == np.uint64 and counts.size == width and counts.flags.c_contiguous
    rc = _load().oracle_pospopcnt_add(width, a.ctypes.data, _nwords(a, width), counts.ctypes.data)
    assert rc == 0
    return counts


def pospopcnt_mt(words, width: int | None = None, nthreads: int | None = None):
    """Threaded form; returns (counts, threads_used)."""
    a = _as_bytes(words)
    width = width or a.itemsize * 8
    out = np.zeros(width, dtype=np.uint64)
    used = _load().oracle_pospopcnt_mt(width, a.ctypes.data, _nwords(a, width), out.ctypes.data,
                                       int(nthreads or os.cpu_count() or 1))
    assert used >= 1
    return out, used


def pospopcnt_segments(words, offsets, width: int | None = None) -> np.ndarray:
    """Row s = pospopcnt(words[offsets[s]:offsets[s+1]]); shape (nseg, width)."""
    a = _as_bytes(words)
    width = width or a.itemsize * 8
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nseg = off.size - 1
    out = np.zeros((max(nseg, 0), width), dtype=np.uint64)
    if nseg > 0:
        assert int(off[-1]) * (width // 8) <= a.size * a.itemsize
        rc = _load().oracle_pospopcnt_segments(width, a.ctypes.data, off.ctypes.data, nseg,
                                               out.ctypes.data)
        assert rc == 0, "bad offsets"
    return out


def csa_pospopcnt(words, width: int | None = None, N: int = 4):
    """The paper's CSA method with a 2^N-register circuit; returns
    (counts, csa_calls)."""
    a = _as_bytes(words)
    width = width or a.itemsize * 8
    out = np.zeros(width, dtype=np.uint64)
    calls = _load().oracle_csa_pospopcnt(width, a.ctypes.data, _nwords(a, width), N,
                                         out.ctypes.data)
    assert calls >= 0
    return out, int(calls)


def popcount(data) -> int:
    """Number of set bits in the bytes of `data` (bit by bit)."""
    a = np.ascontiguousarray(data)
    out = np.zeros(1, dtype=np.uint64)
    assert _load().oracle_popcount(a.ctypes.data, a.size * a.itemsize, out.ctypes.data) == 0
    return int(out[0])


def onehot_counts(ids, k: int) -> np.ndarray:
    """Frequency histogram of categorical ids by one-hot encoding then
    positional counting (§1); ids >= k are not counted.  uint64[k]."""
    a = np.ascontiguousarray(ids)
    assert a.dtype in (np.uint8, np.uint16, np.uint32)
    out = np.zeros(k, dtype=np.uint64)
    assert _load().oracle_onehot_counts(a.ctypes.data, a.size, a.itemsize, k, out.ctypes.data) == 0
    return out


def csa_truth(which: int) -> int:
    """8-bit truth-table immediate of the CSA sum bit (0) or carry bit (1)."""
    return int(_load().oracle_csa_truth(which))


def csa_circuit_size(N: int) -> int:
    """Number of CSA calls in one run of the circuit F_N."""
    return int(_load().oracle_csa_circuit_size(N))
