"""pospopcnt on GB300: Python binding of the C ABI in include/pospopcnt.h.

The positional population count (Klarqvist, Mula, Lemire, arXiv 1911.02696):
for k-bit words w_i, counts[p] = sum_i ((w_i >> p) & 1), p = 0..k-1.

Every function here has the name of a C entry point and only marshals
arguments: tensors become device pointers and word counts, the stream
becomes a cudaStream_t, and a non-zero status becomes a PospopcntError.
All counting runs in the library's CUDA kernels; there is no CPU path.
PyTorch supplies device memory and streams.  Counts are returned in int64
tensors (the values are uint64 and never exceed 2^63 here).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = [
    "PospopcntError", "load", "pospopcnt_init", "pospopcnt_u8", "pospopcnt_u16", "pospopcnt_u32", "pospopcnt_u64", "pospopcnt_popcount", "pospopcnt_onehot_counts",
    "pospopcnt_count", "pospopcnt_count_config", "pospopcnt_count_accumulate", "pospopcnt_count_host",
    "pospopcnt_host_is_mapped",
    "pospopcnt_batched", "pospopcnt_batched_checked", "pospopcnt_batched_noalloc",
    "pospopcnt_batched_graph_create", "pospopcnt_graph_launch", "pospopcnt_graph_destroy", "pospopcnt_plain_segments", "pospopcnt_check_device_error", "pospopcnt_plan_split",
    "pospopcnt_get_config", "pospopcnt_set_config", "pospopcnt_autotune", "pospopcnt_strerror",
    "pospopcnt_last_cuda_error", "pospopcnt_launch_count", "pospopcnt_device_bytes_allocated", "pospopcnt_selftest_timeout", "KERNELS",
    "Config", "pospopcnt_server_create", "pospopcnt_server_destroy", "pospopcnt_server_submit",
    "pospopcnt_server_poll", "pospopcnt_server_run_trace", "pospopcnt_server_run_trace_timed",
    "pospopcnt_server_get_stats",
    "pospopcnt_admission_simulate",
]

KERNELS = {"auto": 0, "csa": 1, "tma": 2, "ballot": 3}
STATUS = {0: "OK", 1: "ERR_INVALID", 2: "ERR_MISALIGNED", 3: "ERR_CUDA", 4: "ERR_NOT_INITIALIZED",
          5: "ERR_TIMEOUT", 6: "ERR_TOO_LARGE"}


class PospopcntError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib().pospopcnt_strerror(status).decode()
        extra = ""
        if status == 3:
            extra = f" (cudaError {_lib().pospopcnt_last_cuda_error()})"
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}{extra}")


class Config(ctypes.Structure):
    """pospopcnt_config: kernel, threads, unroll, blocks_per_sm, stages, chunk_bytes, flags."""
    _fields_ = [("kernel", ctypes.c_int), ("threads", ctypes.c_int), ("unroll", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int), ("stages", ctypes.c_int), ("chunk_bytes", ctypes.c_int),
                ("flags", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class BatchedConfig(ctypes.Structure):
    """pospopcnt_batched_config: unit_bytes, blocks_per_sm, ring_stages, vectors_per_lane."""
    _fields_ = [("unit_bytes", ctypes.c_int), ("blocks_per_sm", ctypes.c_int), ("ring_stages", ctypes.c_int),
                ("vectors_per_lane", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServerConfig(ctypes.Structure):
    """pospopcnt_server_config."""
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_int),
                ("max_batch_jobs", ctypes.c_int), ("per_request", ctypes.c_int),
                ("large_job_bytes", ctypes.c_uint64), ("max_large_inflight", ctypes.c_int)]


class Result(ctypes.Structure):
    """pospopcnt_result."""
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int), ("width", ctypes.c_int),
                ("n", ctypes.c_uint64), ("t_arrival", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_launch", ctypes.c_double), ("t_done", ctypes.c_double), ("counts", ctypes.c_uint64 * 32)]


class ServerStats(ctypes.Structure):
    """pospopcnt_server_stats."""
    _fields_ = [(f, ctypes.c_uint64) for f in ("submitted", "completed", "rejected", "batches", "jobs_in_batches",
                                                "max_batch", "deferrals", "bytes_completed",
                                                "max_bytes_in_flight")]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


_lock = threading.Lock()
_handle = None


def load(build_if_needed: bool = True) -> ctypes.CDLL:
    """Loads libpospopcnt_gb300.so (building it first if it is missing or
    stale).  Raises if it cannot be built or loaded: there is no fallback."""
    global _handle
    with _lock:
        if _handle is None:
            path = _build.build() if build_if_needed else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not built: {path}")
            lib = ctypes.CDLL(path)
            _declare(lib)
            _handle = lib
    return _handle


_lib = load


def _declare(lib):
    i32, u64, vp, sz = ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_size_t
    P = ctypes.POINTER
    sig = {
        "pospopcnt_init": (i32, [i32]),
        "pospopcnt_u8": (i32, [vp, sz, vp, vp]),
        "pospopcnt_u16": (i32, [vp, sz, vp, vp]),
        "pospopcnt_u32": (i32, [vp, sz, vp, vp]),
        "pospopcnt_u64": (i32, [vp, sz, vp, vp]),
        "pospopcnt_popcount": (i32, [vp, sz, vp, vp]),
        "pospopcnt_onehot_counts": (i32, [vp, sz, i32, i32, vp, vp]),
        "pospopcnt_count": (i32, [i32, i32, vp, sz, vp, vp]),
        "pospopcnt_count_config": (i32, [i32, P(Config), vp, sz, vp, vp]),
        "pospopcnt_count_accumulate": (i32, [i32, vp, sz, vp, vp]),
        "pospopcnt_count_host": (i32, [i32, vp, sz, vp]),
        "pospopcnt_host_is_mapped": (i32, [vp, sz]),
        "pospopcnt_batched": (i32, [vp, vp, sz, i32, vp, vp]),
        "pospopcnt_plain_segments": (i32, [vp, vp, sz, i32, vp, vp]),
        "pospopcnt_batched_noalloc": (i32, [vp, vp, sz, i32, vp, vp]),
        "pospopcnt_batched_checked": (i32, [vp, sz, vp, sz, i32, vp, vp]),
        "pospopcnt_batched_graph_create": (i32, [vp, vp, sz, i32, vp, P(vp)]),
        "pospopcnt_batched_get_config": (i32, [i32, P(BatchedConfig)]),
        "pospopcnt_batched_set_config": (i32, [i32, P(BatchedConfig)]),
        "pospopcnt_batched_autotune": (i32, [vp, vp, sz, i32, vp, P(BatchedConfig), P(ctypes.c_float), vp]),
        "pospopcnt_graph_launch": (i32, [vp, vp]),
        "pospopcnt_graph_destroy": (i32, [vp]),
        "pospopcnt_release_stream": (i32, [vp]),
        "pospopcnt_check_device_error": (i32, [vp]),
        "pospopcnt_plan_split": (i32, [i32, u64, sz, P(sz), P(sz), P(sz)]),
        "pospopcnt_get_config": (i32, [i32, sz, P(Config)]),
        "pospopcnt_set_config": (i32, [i32, i32, P(Config)]),
        "pospopcnt_autotune": (i32, [i32, vp, sz, vp, P(Config), P(ctypes.c_float)]),
        "pospopcnt_strerror": (ctypes.c_char_p, [i32]),
        "pospopcnt_last_cuda_error": (i32, []),
        "pospopcnt_launch_count": (u64, []),
        "pospopcnt_device_bytes_allocated": (u64, []),
        "pospopcnt_selftest_timeout": (i32, [u64, vp]),
        "pospopcnt_server_create": (i32, [i32, P(ServerConfig), P(vp)]),
        "pospopcnt_server_destroy": (i32, [vp]),
        "pospopcnt_server_submit": (i32, [vp, i32, vp, sz, u64]),
        "pospopcnt_server_poll": (i32, [vp, P(Result), i32, P(i32)]),
        "pospopcnt_server_run_trace": (i32, [vp, sz, vp, vp, vp, vp, vp, vp, vp]),
        "pospopcnt_server_run_trace_timed": (i32, [vp, sz, vp, vp, vp, vp, vp, vp, vp, vp]),
        "pospopcnt_server_get_stats": (i32, [vp, P(ServerStats)]),
        "pospopcnt_admission_simulate": (i32, [u64, sz, vp, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args


def _check(status: int, where: str):
    if status != 0:
        raise PospopcntError(status, where)


# ---------------------------------------------------------------------------
# tensor marshalling

def _torch():
    import torch
    return torch


def _stream_handle(stream, device):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _words(x, width: int):
    """(device pointer, word count) of a contiguous CUDA tensor viewed as
    `width`-bit words."""
    if not x.is_cuda:
        raise ValueError("input must be a CUDA tensor (use pospopcnt_count_host for host memory)")
    if not x.is_contiguous():
        raise ValueError("input must be contiguous")
    nbytes = x.numel() * x.element_size()
    if nbytes % (width // 8):
        raise ValueError(f"{nbytes} bytes is not a whole number of {width}-bit words")
    return x.data_ptr(), nbytes // (width // 8)


def _counts_out(counts, width: int, rows: int | None, device):
    torch = _torch()
    shape = (width,) if rows is None else (rows, width)
    if counts is None:
        return torch.empty(shape, dtype=torch.int64, device=device)
    if counts.dtype not in (torch.int64, getattr(torch, "uint64", torch.int64)) or not counts.is_contiguous():
        raise ValueError("counts must be a contiguous 64-bit integer tensor")
    if counts.numel() != int(np.prod(shape)) or counts.device != device:
        raise ValueError(f"counts must hold {shape} values on {device}")
    return counts


def pospopcnt_init(device: int = 0) -> None:
    _check(_lib().pospopcnt_init(device), "pospopcnt_init")


def _plain(name: str, width: int, x, counts, stream):
    torch = _torch()
    ptr, n = _words(x, width)
    out = _counts_out(counts, width, None, x.device)
    with torch.cuda.device(x.device):
        _check(getattr(_lib(), name)(ptr, n, out.data_ptr(), _stream_handle(stream, x.device)), name)
    return out


def pospopcnt_u8(x, counts=None, stream=None):
    """Counts of the 8-bit words of CUDA tensor x (int64[8])."""
    return _plain("pospopcnt_u8", 8, x, counts, stream)


def pospopcnt_u16(x, counts=None, stream=None):
    """Counts of the 16-bit words of CUDA tensor x (int64[16])."""
    return _plain("pospopcnt_u16", 16, x, counts, stream)


def pospopcnt_u32(x, counts=None, stream=None):
    """Counts of the 32-bit words of CUDA tensor x (int64[32])."""
    return _plain("pospopcnt_u32", 32, x, counts, stream)


def pospopcnt_u64(x, counts=None, stream=None):
    """Counts of the 64-bit words of CUDA tensor x (int64[64])."""
    return _plain("pospopcnt_u64", 64, x, counts, stream)


def pospopcnt_popcount(x, count=None, stream=None):
    """Number of set bits in the bytes of CUDA tensor x (int64[1])."""
    torch = _torch()
    ptr, nbytes = _words(x, 8)
    out = _counts_out(count, 1, None, x.device)
    with torch.cuda.device(x.device):
        _check(_lib().pospopcnt_popcount(ptr, nbytes, out.data_ptr(), _stream_handle(stream, x.device)),
               "pospopcnt_popcount")
    return out


def pospopcnt_onehot_counts(ids, k: int, counts=None, stream=None):
    """Histogram of categorical ids (CUDA tensor of uint8/int16/int32 viewed
    as unsigned ids) over k <= 32 categories; ids >= k are not counted."""
    torch = _torch()
    idb = ids.element_size()
    if idb not in (1, 2, 4):
        raise ValueError("ids must be 1-, 2- or 4-byte integers")
    ptr, n = _words(ids, 8 * idb)
    out = _counts_out(counts, k, None, ids.device)
    with torch.cuda.device(ids.device):
        _check(_lib().pospopcnt_onehot_counts(ptr, n, idb, k, out.data_ptr(), _stream_handle(stream, ids.device)),
               "pospopcnt_onehot_counts")
    return out


def pospopcnt_count(width: int, x, kernel="auto", counts=None, stream=None):
    torch = _torch()
    ptr, n = _words(x, width)
    out = _counts_out(counts, width, None, x.device)
    k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    with torch.cuda.device(x.device):
        _check(_lib().pospopcnt_count(width, k, ptr, n, out.data_ptr(), _stream_handle(stream, x.device)),
               "pospopcnt_count")
    return out


def _make_config(cfg) -> Config:
    if isinstance(cfg, Config):
        return cfg
    c = Config()
    for k, v in dict(cfg).items():
        setattr(c, k, KERNELS[v] if k == "kernel" and isinstance(v, str) else int(v))
    return c


def pospopcnt_count_config(width: int, cfg, x, counts=None, stream=None):
    torch = _torch()
    ptr, n = _words(x, width)
    out = _counts_out(counts, width, None, x.device)
    c = _make_config(cfg)
    with torch.cuda.device(x.device):
        _check(_lib().pospopcnt_count_config(width, ctypes.byref(c), ptr, n, out.data_ptr(),
                                             _stream_handle(stream, x.device)), "pospopcnt_count_config")
    return out


def pospopcnt_count_accumulate(width: int, x, counts, stream=None):
    """counts += pospopcnt(x) (the paper's accumulate convention)."""
    torch = _torch()
    ptr, n = _words(x, width)
    out = _counts_out(counts, width, None, x.device)
    with torch.cuda.device(x.device):
        _check(_lib().pospopcnt_count_accumulate(width, ptr, n, out.data_ptr(),
                                                 _stream_handle(stream, x.device)), "pospopcnt_count_accumulate")
    return out


def pospopcnt_count_host(width: int, h, out: np.ndarray | None = None) -> np.ndarray:
    """Counts of host memory h (numpy array or CPU tensor; pinned memory is
    fastest).  Synchronous; returns uint64[width]."""
    if hasattr(h, "data_ptr"):
        if h.is_cuda or not h.is_contiguous():
            raise ValueError("h must be a contiguous host tensor")
        ptr, nbytes = h.data_ptr(), h.numel() * h.element_size()
    else:
        a = np.ascontiguousarray(h)
        ptr, nbytes = a.ctypes.data, a.nbytes
    if nbytes % (width // 8):
        raise ValueError("not a whole number of words")
    if out is None:
        out = np.zeros(width, dtype=np.uint64)
    assert out.dtype == np.uint64 and out.size == width and out.flags.c_contiguous
    _check(_lib().pospopcnt_count_host(width, ptr, nbytes // (width // 8), out.ctypes.data),
           "pospopcnt_count_host")
    return out


def pospopcnt_host_is_mapped(h) -> bool:
    """Whether pospopcnt_count_host reads host buffer h in place."""
    if hasattr(h, "data_ptr"):
        ptr, nbytes = h.data_ptr(), h.numel() * h.element_size()
    else:
        a = np.ascontiguousarray(h)
        ptr, nbytes = a.ctypes.data, a.nbytes
    return bool(_lib().pospopcnt_host_is_mapped(ctypes.c_void_p(ptr), nbytes))


def pospopcnt_batched(x, offsets, width: int, counts=None, stream=None):
    """Row s = counts of words [offsets[s], offsets[s+1]) of x; offsets is a
    CUDA int64 tensor of nseg+1 word offsets.  Returns int64[nseg, width]."""
    torch = _torch()
    ptr, _ = _words(x, width)
    if offsets.dtype != torch.int64 or not offsets.is_cuda or not offsets.is_contiguous():
        raise ValueError("offsets must be a contiguous CUDA int64 tensor")
    nseg = max(offsets.numel() - 1, 0)
    out = _counts_out(counts, width, nseg, x.device)
    with torch.cuda.device(x.device):
        _check(_lib().pospopcnt_batched(ptr, offsets.data_ptr(), nseg, width, out.data_ptr(),
                                        _stream_handle(stream, x.device)), "pospopcnt_batched")
    return out


def pospopcnt_batched_get_config(width: int, device=None) -> dict:
    """The batched form's launch configuration for `width` (dict)."""
    torch = _torch()
    c = BatchedConfig()
    with torch.cuda.device(device if device is not None else torch.cuda.current_device()):
        _check(_lib().pospopcnt_batched_get_config(width, ctypes.byref(c)), "pospopcnt_batched_get_config")
    return c.as_dict()


def pospopcnt_batched_set_config(width: int, cfg, device=None) -> None:
    """Installs cfg (dict with unit_bytes and optionally blocks_per_sm,
    ring_stages, vectors_per_lane; None: the default)."""
    torch = _torch()
    ref = None
    if cfg is not None:
        c = BatchedConfig(int(cfg["unit_bytes"]), int(cfg.get("blocks_per_sm", 0)), int(cfg.get("ring_stages", 0)),
                          int(cfg.get("vectors_per_lane", 0)))
        ref = ctypes.byref(c)
    with torch.cuda.device(device if device is not None else torch.cuda.current_device()):
        _check(_lib().pospopcnt_batched_set_config(width, ref), "pospopcnt_batched_set_config")


def pospopcnt_batched_autotune(x, offsets, width: int, counts=None, stream=None):
    """Times the batched form's launch configurations on this layout; installs
    and returns the fastest (dict) and its time per call in ms."""
    torch = _torch()
    ptr, _ = _words(x, width)
    if offsets.dtype != torch.int64 or not offsets.is_cuda or not offsets.is_contiguous():
        raise ValueError("offsets must be a contiguous CUDA int64 tensor")
    nseg = max(offsets.numel() - 1, 0)
    out = _counts_out(counts, width, nseg, x.device)
    c, ms = BatchedConfig(), ctypes.c_float()
    with torch.cuda.device(x.device):
        _check(_lib().pospopcnt_batched_autotune(ptr, offsets.data_ptr(), nseg, width, out.data_ptr(),
                                                 ctypes.byref(c), ctypes.byref(ms), _stream_handle(stream, x.device)),
               "pospopcnt_batched_autotune")
    return c.as_dict(), ms.value


def pospopcnt_release_stream(stream=None, device=None) -> None:
    """Returns the work-queue slot the stream's batched calls hold."""
    torch = _torch()
    dev = device if device is not None else torch.cuda.current_device()
    with torch.cuda.device(dev):
        _check(_lib().pospopcnt_release_stream(_stream_handle(stream, torch.device("cuda", dev))),
               "pospopcnt_release_stream")


def pospopcnt_batched_graph_create(x, offsets, width: int, counts) -> int:
    """Captures pospopcnt_batched on these buffers into a CUDA graph; returns
    its handle (launch with pospopcnt_graph_launch)."""
    torch = _torch()
    ptr, _ = _words(x, width)
    nseg = max(offsets.numel() - 1, 0)
    out = _counts_out(counts, width, nseg, x.device)
    h = ctypes.c_void_p()
    with torch.cuda.device(x.device):
        _check(_lib().pospopcnt_batched_graph_create(ptr, offsets.data_ptr(), nseg, width, out.data_ptr(),
                                                     ctypes.byref(h)), "pospopcnt_batched_graph_create")
    return h.value


def pospopcnt_graph_launch(graph: int, stream=None, device=None) -> None:
    torch = _torch()
    device = device if device is not None else torch.cuda.current_device()
    with torch.cuda.device(device):
        _check(_lib().pospopcnt_graph_launch(ctypes.c_void_p(graph), _stream_handle(stream, device)),
               "pospopcnt_graph_launch")


def pospopcnt_graph_destroy(graph: int) -> None:
    _check(_lib().pospopcnt_graph_destroy(ctypes.c_void_p(graph)), "pospopcnt_graph_destroy")


def pospopcnt_batched_checked(x, offsets, width: int, counts=None, stream=None):
    """pospopcnt_batched with the offsets validated on the device against
    the words of x; bad offsets count nothing and are reported by
    pospopcnt_check_device_error (status 1)."""
    torch = _torch()
    ptr, n_words = _words(x, width)
    if offsets.dtype != torch.int64 or not offsets.is_cuda or not offsets.is_contiguous():
        raise ValueError("offsets must be a contiguous CUDA int64 tensor")
    nseg = max(offsets.numel() - 1, 0)
    out = _counts_out(counts, width, nseg, x.device)
    with torch.cuda.device(x.device):
        _check(_lib().pospopcnt_batched_checked(ptr, n_words, offsets.data_ptr(), nseg, width, out.data_ptr(),
                                                _stream_handle(stream, x.device)), "pospopcnt_batched_checked")
    return out


def pospopcnt_batched_noalloc(x, offsets, width: int, counts, stream=None):
    """pospopcnt_batched that allocates nothing (see the C header): the
    caller passes the output rows; the library uses only a static device
    array as scratch, shared by every call on the device."""
    torch = _torch()
    ptr, _ = _words(x, width)
    if offsets.dtype != torch.int64 or not offsets.is_cuda or not offsets.is_contiguous():
        raise ValueError("offsets must be a contiguous CUDA int64 tensor")
    nseg = max(offsets.numel() - 1, 0)
    out = _counts_out(counts, width, nseg, x.device)
    with torch.cuda.device(x.device):
        _check(_lib().pospopcnt_batched_noalloc(ptr, offsets.data_ptr(), nseg, width, out.data_ptr(),
                                                _stream_handle(stream, x.device)), "pospopcnt_batched_noalloc")
    return out


def pospopcnt_plain_segments(x, offsets: np.ndarray, width: int, counts=None, stream=None):
    """One plain count per segment, issued from a host loop; offsets is a
    host int64 array of nseg+1 word offsets.  Returns int64[nseg, width]."""
    torch = _torch()
    ptr, _ = _words(x, width)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nseg = max(off.size - 1, 0)
    out = _counts_out(counts, width, nseg, x.device)
    with torch.cuda.device(x.device):
        _check(_lib().pospopcnt_plain_segments(ptr, off.ctypes.data, nseg, width, out.data_ptr(),
                                               _stream_handle(stream, x.device)), "pospopcnt_plain_segments")
    return out


def pospopcnt_check_device_error(stream=None, device=None) -> int:
    """Synchronises the stream and returns the device error status (0 = OK)."""
    torch = _torch()
    device = device if device is not None else torch.cuda.current_device()
    with torch.cuda.device(device):
        return int(_lib().pospopcnt_check_device_error(_stream_handle(stream, device)))


def pospopcnt_plan_split(width: int, addr: int, n: int):
    """(head_words, body_vectors, tail_words) for n words at address addr."""
    h, b, t = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(_lib().pospopcnt_plan_split(width, addr, n, ctypes.byref(h), ctypes.byref(b), ctypes.byref(t)),
           "pospopcnt_plan_split")
    return h.value, b.value, t.value


def pospopcnt_get_config(width: int, n: int) -> dict:
    c = Config()
    _check(_lib().pospopcnt_get_config(width, n, ctypes.byref(c)), "pospopcnt_get_config")
    return c.as_dict()


def pospopcnt_set_config(width: int, size_class: int, cfg) -> None:
    c = _make_config(cfg)
    _check(_lib().pospopcnt_set_config(width, size_class, ctypes.byref(c)), "pospopcnt_set_config")


def pospopcnt_autotune(width: int, x, scratch_counts=None):
    """Times the candidate configurations on x; installs and returns the best
    (dict) and its time in ms."""
    torch = _torch()
    ptr, n = _words(x, width)
    out = _counts_out(scratch_counts, width, None, x.device)
    c, ms = Config(), ctypes.c_float()
    with torch.cuda.device(x.device):
        _check(_lib().pospopcnt_autotune(width, ptr, n, out.data_ptr(), ctypes.byref(c), ctypes.byref(ms)),
               "pospopcnt_autotune")
    return c.as_dict(), ms.value


def pospopcnt_strerror(status: int) -> str:
    return _lib().pospopcnt_strerror(status).decode()


def pospopcnt_last_cuda_error() -> int:
    return int(_lib().pospopcnt_last_cuda_error())


def pospopcnt_launch_count() -> int:
    return int(_lib().pospopcnt_launch_count())


def pospopcnt_device_bytes_allocated() -> int:
    """Bytes of device memory the library holds from its own allocations."""
    return int(_lib().pospopcnt_device_bytes_allocated())


def pospopcnt_selftest_timeout(limit_ns: int = 1_000_000, stream=None, device=None) -> None:
    """Runs the bounded-wait self-test kernel (see the C header)."""
    torch = _torch()
    device = device if device is not None else torch.cuda.current_device()
    with torch.cuda.device(device):
        _check(_lib().pospopcnt_selftest_timeout(limit_ns, _stream_handle(stream, device)),
               "pospopcnt_selftest_timeout")


# ---------------------------------------------------------------------------
# serving

def pospopcnt_server_create(device: int = 0, hbm_budget_bytes: int = 0, max_inflight: int = 0,
                            max_batch_jobs: int = 0, per_request: bool = False, large_job_bytes: int = 0,
                            max_large_inflight: int = 0) -> int:
    """Creates a serving runtime (see the C header); returns its handle."""
    cfg = ServerConfig(hbm_budget_bytes, max_inflight, max_batch_jobs, int(per_request), large_job_bytes,
                       max_large_inflight)
    h = ctypes.c_void_p()
    _check(_lib().pospopcnt_server_create(device, ctypes.byref(cfg), ctypes.byref(h)), "pospopcnt_server_create")
    return h.value


def pospopcnt_server_destroy(server: int) -> None:
    _check(_lib().pospopcnt_server_destroy(ctypes.c_void_p(server)), "pospopcnt_server_destroy")


def pospopcnt_server_submit(server: int, width: int, x, tag: int) -> None:
    """Submits the words of CUDA tensor x (kept alive by the caller until the
    job completes)."""
    ptr, n = _words(x, width)
    _check(_lib().pospopcnt_server_submit(ctypes.c_void_p(server), width, ctypes.c_void_p(ptr), n, tag),
           "pospopcnt_server_submit")


def pospopcnt_server_poll(server: int, max_results: int = 1024):
    """Completed jobs as dicts (tag, status, width, n, times, counts)."""
    buf = (Result * max_results)()
    k = ctypes.c_int()
    _check(_lib().pospopcnt_server_poll(ctypes.c_void_p(server), buf, max_results, ctypes.byref(k)),
           "pospopcnt_server_poll")
    out = []
    for r in buf[:k.value]:
        out.append({"tag": r.tag, "status": r.status, "width": r.width, "n": r.n, "t_arrival": r.t_arrival,
                    "t_admit": r.t_admit, "t_launch": r.t_launch, "t_done": r.t_done,
                    "counts": np.frombuffer(bytes(r.counts), dtype=np.uint64)[: r.width].copy()})
    return out


def pospopcnt_server_run_trace(server: int, t_arrival, width, d_addr, nwords, want_counts: bool = False,
                               want_stages: bool = False):
    """Replays an open-loop trace; returns (latency_s, counts or None, status),
    plus, with want_stages, an n x 3 array of seconds from each request's
    arrival to its admission, its launch and its completion."""
    t = np.ascontiguousarray(t_arrival, dtype=np.float64)
    w = np.ascontiguousarray(width, dtype=np.int32)
    a = np.ascontiguousarray(d_addr, dtype=np.uint64)
    nw = np.ascontiguousarray(nwords, dtype=np.uint64)
    n = t.size
    assert w.size == n and a.size == n and nw.size == n
    lat = np.empty(n, dtype=np.float64)
    status = np.empty(n, dtype=np.int32)
    counts = np.zeros((n, 32), dtype=np.uint64) if want_counts else None
    stages = np.empty((n, 3), dtype=np.float64) if want_stages else None
    _check(_lib().pospopcnt_server_run_trace_timed(
        ctypes.c_void_p(server), n, t.ctypes.data, w.ctypes.data, a.ctypes.data, nw.ctypes.data, lat.ctypes.data,
        counts.ctypes.data if counts is not None else None, status.ctypes.data,
        stages.ctypes.data if stages is not None else None), "pospopcnt_server_run_trace")
    return (lat, counts, status, stages) if want_stages else (lat, counts, status)


def pospopcnt_server_get_stats(server: int) -> dict:
    st = ServerStats()
    _check(_lib().pospopcnt_server_get_stats(ctypes.c_void_p(server), ctypes.byref(st)),
           "pospopcnt_server_get_stats")
    return st.as_dict()


def pospopcnt_admission_simulate(budget: int, t_arrival, nbytes, service_s):
    """The server's admission policy on a mock clock (no device): returns
    (t_admit, status) per job."""
    t = np.ascontiguousarray(t_arrival, dtype=np.float64)
    b = np.ascontiguousarray(nbytes, dtype=np.uint64)
    sv = np.ascontiguousarray(service_s, dtype=np.float64)
    n = t.size
    t_admit = np.empty(n, dtype=np.float64)
    status = np.empty(n, dtype=np.int32)
    _check(_lib().pospopcnt_admission_simulate(budget, n, t.ctypes.data, b.ctypes.data, sv.ctypes.data,
                                               t_admit.ctypes.data, status.ctypes.data),
           "pospopcnt_admission_simulate")
    return t_admit, status
