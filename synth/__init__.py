"""Seeded synthetic inputs for pospopcnt tests and benchmarks.

This module holds none of the pospopcnt arithmetic: it only produces the
input words (and, for one-hot data, the positions it drew).  The bytes are
made on the host by ``synth.c`` (counter-based SplitMix64, multithreaded by
index range) and reach the GPU through a host->device copy, so the CPU oracle
and the CUDA path always see the same input.

Recipes (the workload shapes of the paper's experiments, §5, which draw
random words; and the segment and skew shapes of the batched workload):

* ``uniform_bits``: every bit i.i.d. Bernoulli(1/2).
* ``one_hot``: one bit per word; its position is categorical: uniform, or
  Zipf(s) over the ``width`` positions (P(j) proportional to (j+1)^-s).
* ``sparse``: every bit i.i.d. Bernoulli(thr/2^24), thr = 167772 ~ 0.01.
* ``log_uniform_lengths``: segment lengths floor(exp(U ln max_len)) clamped
  to [1, max_len].
* ``segmented_one_hot``: one-hot words per segment with a per-segment
  rotation of a Zipf rank order.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_OUT = os.path.join(_HERE, "_build", "libsynth.so")
_lock = threading.Lock()
_lib = None

SPARSE_THR_001 = 167772  # round(0.01 * 2^24)


def build(force: bool = False) -> str:
    """Compile synth.c into a shared library (plain gcc, no intrinsics)."""
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
            u64, vp, i32 = ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int
            lib.synth_draw.restype = u64
            lib.synth_draw.argtypes = [u64, u64]
            lib.synth_uniform_bits.restype = None
            lib.synth_uniform_bits.argtypes = [u64, vp, u64, i32]
            lib.synth_one_hot.restype = i32
            lib.synth_one_hot.argtypes = [u64, i32, vp, vp, u64, vp, i32]
            lib.synth_sparse.restype = i32
            lib.synth_sparse.argtypes = [u64, i32, ctypes.c_uint32, vp, u64, i32]
            lib.synth_categorical_ids.restype = i32
            lib.synth_categorical_ids.argtypes = [u64, i32, vp, i32, vp, u64, i32]
            lib.synth_segmented_one_hot.restype = i32
            lib.synth_segmented_one_hot.argtypes = [u64, i32, vp, vp, vp, u64, vp, i32]
            _lib = lib
    return _lib


def _threads(nthreads):
    return int(nthreads) if nthreads else min(os.cpu_count() or 1, 32)


_DT = {8: np.uint8, 16: np.uint16, 32: np.uint32, 64: np.uint64}


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def draw(seed: int, i: int) -> int:
    """The i-th 64-bit draw of stream ``seed``."""
    return int(_load().synth_draw(seed, i))


def uniform_bits(seed: int, n: int, width: int = 16, out: np.ndarray | None = None,
                 nthreads: int | None = None) -> np.ndarray:
    """n words of ``width`` bits whose bits are i.i.d. Bernoulli(1/2)."""
    dt = _DT[width]
    if out is None:
        out = np.empty(n, dtype=dt)
    assert out.dtype == dt and out.size == n and out.flags.c_contiguous
    if n:
        _load().synth_uniform_bits(seed, _ptr(out), n * (width // 8), _threads(nthreads))
    return out


def uniform_bytes(seed: int, nbytes: int, nthreads: int | None = None) -> np.ndarray:
    return uniform_bits(seed, nbytes, 8, nthreads=nthreads)


def zipf_cdf(m: int, s: float = 1.1) -> np.ndarray:
    """Cumulative Zipf(s) probabilities over m positions, scaled to 2^32."""
    w = [(j + 1) ** (-s) for j in range(m)]
    tot = math.fsum(w)
    acc = 0.0
    cdf = []
    for j in range(m - 1):
        acc += w[j]
        cdf.append(min(int(math.floor(acc / tot * 2.0 ** 32)), 2 ** 32))
    cdf.append(2 ** 32)
    return np.array(cdf, dtype=np.uint64)


def uniform_cdf(m: int) -> np.ndarray:
    """Cumulative uniform probabilities over m positions, scaled to 2^32."""
    return np.array([((j + 1) << 32) // m for j in range(m)], dtype=np.uint64)


def one_hot(seed: int, n: int, width: int = 16, cdf: np.ndarray | None = None,
            return_positions: bool = False, nthreads: int | None = None):
    """n one-hot words; the set position is drawn from ``cdf`` (default
    Zipf(1.1)).  With ``return_positions`` also returns the drawn positions."""
    if cdf is None:
        cdf = zipf_cdf(width)
    cdf = np.ascontiguousarray(cdf, dtype=np.uint64)
    assert cdf.size == width and int(cdf[-1]) == 2 ** 32
    out = np.empty(n, dtype=_DT[width])
    pos = np.empty(n, dtype=np.uint8) if return_positions else None
    if n:
        rc = _load().synth_one_hot(seed, width, _ptr(cdf), _ptr(out), n,
                                   _ptr(pos) if pos is not None else None, _threads(nthreads))
        assert rc == 0
    return (out, pos) if return_positions else out


def sparse(seed: int, n: int, width: int = 16, thr24: int = SPARSE_THR_001,
           nthreads: int | None = None) -> np.ndarray:
    """n words whose bits are i.i.d. Bernoulli(thr24 / 2^24)."""
    out = np.empty(n, dtype=_DT[width])
    if n:
        assert _load().synth_sparse(seed, width, thr24, _ptr(out), n, _threads(nthreads)) == 0
    return out


def log_uniform_lengths(seed: int, nseg: int, max_len: int = 1 << 20) -> np.ndarray:
    """Segment lengths floor(exp(U * ln max_len)) clamped to [1, max_len],
    U = draw(s) >> 11 scaled to [0, 1)."""
    u = np.array([draw(seed, s) >> 11 for s in range(nseg)], dtype=np.float64) * 2.0 ** -53
    lens = np.floor(np.exp(u * math.log(max_len))).astype(np.int64)
    return np.clip(lens, 1, max_len)


def offsets_from_lengths(lens: np.ndarray, start: int = 0) -> np.ndarray:
    off = np.empty(lens.size + 1, dtype=np.int64)
    off[0] = start
    np.cumsum(lens, out=off[1:])
    off[1:] += start
    return off


def segmented_one_hot(seed: int, offsets: np.ndarray, width: int = 16, s: float = 1.1,
                      nthreads: int | None = None) -> np.ndarray:
    """Words [0, offsets[-1]); segment k's words are one-hot with a Zipf(s)
    rank order rotated by rot[k] = draw(seed ^ 0x5EC, k) mod width.  Words
    before offsets[0] are zero."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    nseg = offsets.size - 1
    total = int(offsets[-1])
    out = np.zeros(total, dtype=_DT[width])
    rot = np.array([draw(seed ^ 0x5EC, k) % width for k in range(nseg)], dtype=np.uint32)
    cdf = zipf_cdf(width, s)
    if nseg:
        assert _load().synth_segmented_one_hot(seed, width, _ptr(cdf), _ptr(offsets), _ptr(rot),
                                               nseg, _ptr(out), _threads(nthreads)) == 0
    return out


def serving_trace(seed: int, rate: float, duration: float, pool_bytes: int, min_bytes: int = 1024,
                  max_bytes: int = 256 << 20, widths=(8, 16, 32), weights=(0.2, 0.6, 0.2)):
    """Open-loop request trace: Poisson arrivals at `rate` per second over
    `duration` seconds; width drawn from `widths` with `weights`; payload size
    log-uniform in [min_bytes, max_bytes] bytes, rounded down to whole words;
    each payload a slice of a device pool of pool_bytes bytes starting at a
    uniform word-aligned offset.  Returns a dict of arrays (t_arrival,
    width, offset_bytes, nwords)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_est = int(rate * duration * 1.2) + 100
    gaps = rng.exponential(1.0 / rate, size=n_est)
    t = np.cumsum(gaps)
    while t[-1] < duration:  # extend if the estimate fell short
        more = np.cumsum(rng.exponential(1.0 / rate, size=n_est)) + t[-1]
        t = np.concatenate([t, more])
    t = t[t < duration]
    n = t.size
    w = rng.choice(np.array(widths, dtype=np.int32), size=n, p=np.array(weights) / np.sum(weights))
    logb = rng.uniform(np.log(min_bytes), np.log(max_bytes), size=n)
    nbytes = np.floor(np.exp(logb)).astype(np.int64)
    wb = (w // 8).astype(np.int64)
    nwords = np.maximum(nbytes // wb, 1)
    nbytes = nwords * wb
    assert int(nbytes.max()) <= pool_bytes
    span = pool_bytes - nbytes
    off = (rng.uniform(0, 1, size=n) * (span // wb + 1)).astype(np.int64) * wb
    return {"t_arrival": t.astype(np.float64), "width": w, "offset_bytes": off, "nwords": nwords.astype(np.uint64)}


def categorical_ids(seed: int, n: int, cdf: np.ndarray, dtype=np.uint8, nthreads: int | None = None) -> np.ndarray:
    """n category ids drawn from the categorical distribution `cdf` (scaled
    to 2^32; len(cdf) categories), as unsigned integers of `dtype`."""
    cdf = np.ascontiguousarray(cdf, dtype=np.uint64)
    assert int(cdf[-1]) == 2 ** 32
    out = np.empty(n, dtype=dtype)
    if n:
        assert _load().synth_categorical_ids(seed, cdf.size, _ptr(cdf), out.itemsize, _ptr(out), n,
                                             _threads(nthreads)) == 0
    return out
