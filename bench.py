#!/usr/bin/env python3
"""Benchmark of the pospopcnt CUDA path on GB300.

Default workload (one JSON line on stdout): single-stream pospopcnt_u16 over
n = 2^30 16-bit words (2 GiB) of uniform random bits, input resident in HBM;
a step is one pospopcnt_u16 call (memset + one kernel).  The metric is GB/s
of input counted (and its fraction of the measured HBM copy bandwidth).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload u16|u16_onehot|u16_sparse|u16_misaligned|u8|u32|sweep|batched]

Timing: CUDA events on the launching stream, a barrier and a device
synchronisation on both sides of the K timed steps, the maximum over ranks.
The input (2 GiB) is larger than L2, so no flush is needed between steps.
Under torchrun each rank counts its own 2 GiB input (weak scaling, no
collective on the data path).  `e2e` times the host-buffer entry point
(pinned host memory -> device copies inside the timed region).  The CPU
baseline and the `--impl reference` arm time the scalar CPU oracle on the
host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pospopcnt_u16 GB/s"
UNIT = "GB/s"
FALLBACK_HBM_GBS = 6800.0
ALU_OPS_PER_ID_ONEHOT32 = 3.28  # one-hot count of 8-bit ids over 17..32 categories


# ---------------------------------------------------------------------------
# helpers

def peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


KERNEL_SOURCES = ("device_common.cuh", "plain_kernels.cuh")


def csrc_hash(files=KERNEL_SOURCES):
    """Hash of the sources that define the single-stream kernels."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1911_02696_gb300", "csrc")
    for name in files:
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_key: str, nbytes: int):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    e = rec.get(kernel_key)
    if not e or e.get("csrc_hash") != csrc_hash(tuple(e.get("sources", KERNEL_SOURCES))):
        return None
    # scale by input bytes (traffic grows in proportion for a streaming scan)
    return int(e["dram_bytes_per_launch"] * nbytes / e["input_bytes"])


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.marks = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self):
        self.marks.append(time.time())

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.lines:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        t0, t1 = (self.marks[0], self.marks[-1]) if len(self.marks) >= 2 else (0, 1e30)
        rows = [line for t, line in self.lines if t0 <= t <= t1 + 0.25]
        in_region = len(rows)
        if not rows:
            rows = [line for _, line in self.lines]
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            f = [x.strip() for x in r.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "samples_in_timed_region": in_region,
                "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------
# distributed plumbing (timing harness only; the data path has no collective)

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def dist_max(value: float, world: int, device=None) -> float:
    """Maximum of a per-rank float over all ranks."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_all(flag: bool, world: int, device=None) -> bool:
    """True on every rank iff `flag` is true on every rank."""
    if world <= 1:
        return flag
    import torch
    import torch.distributed as dist
    t = torch.tensor([1 if flag else 0], dtype=torch.int32, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MIN)
    return bool(t.item())


def dist_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def whole_job_throughput(bytes_per_rank_step: int, steps: int, world: int, max_ms: float) -> float:
    """GB/s of the whole job: every rank's bytes over the slowest rank's time."""
    return bytes_per_rank_step * steps * world / (max_ms * 1e-3) / 1e9


# ---------------------------------------------------------------------------
# workloads

def make_input(kind: str, seed: int, log2_words: int | None = None, limit: int | None = None, onehot_k: int = 16):
    """(host words, width, start offset in bytes, description).  With `limit`
    only the first `limit` words are made -- the same words as the first ones
    of the full input, every generator being a function of (seed, index) --
    while the description still names the full workload."""
    import synth
    K = int(onehot_k)
    zipf16 = synth.zipf_cdf(K)  # the one-hot workloads' category distribution (k = 16 by default)
    if log2_words is not None:  # a smaller case of the same workload (profiling)
        n = 1 << log2_words
        table = {
            "popcount": (1, f"array popcount of 2^{log2_words} uniform random bytes",
                         lambda m: synth.uniform_bytes(seed, m)),
            "onehot": (-K, f"fused one-hot encode + count: 2^{log2_words} u8 ids, Zipf(1.1) over {K} categories",
                       lambda m: synth.categorical_ids(seed, m, zipf16, np.uint8)),
            "onehot_u16ids": (-K, f"fused one-hot encode + count: 2^{log2_words} u16 ids, Zipf(1.1) over {K} "
                                  "categories", lambda m: synth.categorical_ids(seed, m, zipf16, np.uint16)),
            "onehot_u32ids": (-K, f"fused one-hot encode + count: 2^{log2_words} u32 ids, Zipf(1.1) over {K} "
                                  "categories", lambda m: synth.categorical_ids(seed, m, zipf16, np.uint32)),
        }
        width = {"u8": 8, "u8_onehot": 8, "u32": 32, "u32_onehot": 32, "u64": 64}.get(kind, 16)
        width, desc, gen = table.get(kind, (width, f"pospopcnt_u{width} n=2^{log2_words} uniform random bits",
                                            lambda m: synth.uniform_bits(seed, m, width)))
        return gen(min(n, limit or n)), width, 0, desc
    table = {  # kind: (words, width, start offset in bytes, description, generator)
        "u16": (1 << 30, 16, 0, "pospopcnt_u16 n=2^30 uniform random bits (2 GiB)",
                lambda m: synth.uniform_bits(seed, m, 16)),
        "u16_onehot": (1 << 30, 16, 0, "pospopcnt_u16 n=2^30 one-hot Zipf(1.1) (2 GiB)",
                       lambda m: synth.one_hot(seed, m, 16)),
        "u16_sparse": (1 << 30, 16, 0, "pospopcnt_u16 n=2^30 sparse Bernoulli(0.01) (2 GiB)",
                       lambda m: synth.sparse(seed, m, 16)),
        "u16_misaligned": ((1 << 30) + 7, 16, 2,
                           "pospopcnt_u16 n=2^30+7 uniform bits, start 2 bytes past a 256-byte boundary",
                           lambda m: synth.uniform_bits(seed, m, 16)),
        "u8": (1 << 31, 8, 0, "pospopcnt_u8 n=2^31 uniform random bits (2 GiB)",
               lambda m: synth.uniform_bits(seed, m, 8)),
        "u8_onehot": (1 << 31, 8, 0, "pospopcnt_u8 n=2^31 one-hot, position uniform over 8 (2 GiB)",
                      lambda m: synth.one_hot(seed, m, 8, cdf=synth.uniform_cdf(8))),
        "u32_onehot": (1 << 29, 32, 0, "pospopcnt_u32 n=2^29 one-hot, position uniform over 32 (2 GiB)",
                       lambda m: synth.one_hot(seed, m, 32, cdf=synth.uniform_cdf(32))),
        "onehot": (1 << 31, -K, 0, f"fused one-hot encode + count: 2^31 u8 ids, Zipf(1.1) over {K} categories (2 GiB)",
                   lambda m: synth.categorical_ids(seed, m, zipf16, np.uint8)),
        "onehot_u16ids": (1 << 30, -K, 0,
                          f"fused one-hot encode + count: 2^30 u16 ids, Zipf(1.1) over {K} categories (2 GiB)",
                          lambda m: synth.categorical_ids(seed, m, zipf16, np.uint16)),
        "onehot_u32ids": (1 << 29, -K, 0,
                          f"fused one-hot encode + count: 2^29 u32 ids, Zipf(1.1) over {K} categories (2 GiB)",
                          lambda m: synth.categorical_ids(seed, m, zipf16, np.uint32)),
        "popcount": (1 << 31, 1, 0, "array popcount of 2 GiB of uniform random bits",
                     lambda m: synth.uniform_bytes(seed, m)),
        "u64": (1 << 28, 64, 0, "pospopcnt_u64 n=2^28 uniform random bits (2 GiB)",
                lambda m: synth.uniform_bits(seed, m, 64)),
        "u32": (1 << 29, 32, 0, "pospopcnt_u32 n=2^29 uniform random bits (2 GiB)",
                lambda m: synth.uniform_bits(seed, m, 32)),
    }
    if kind not in table:
        raise ValueError(kind)
    n, width, offset, desc, gen = table[kind]
    return gen(min(n, limit or n)), width, offset, desc


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the ISA)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


def cpu_baseline(words, width, onehot_k=0, budget_s=8.0):
    """The oracle as it stands on a bounded sample of the same input: 2^26-word
    chunks until budget_s of wall time has passed.  pospopcnt runs on all host
    cores (plus a one-core figure on the first 2^25 words); the popcount and
    one-hot oracles are single-threaded."""
    import oracle
    cores = os.cpu_count() or 1
    chunk = 1 << 26
    done, t0, used = 0, time.perf_counter(), 1
    while done < words.size:
        part = words[done: done + chunk]
        if onehot_k:
            oracle.onehot_counts(part, onehot_k)
        elif width == 1:
            oracle.popcount(part)
        else:
            _, used = oracle.pospopcnt_mt(part, width, cores)
        done += part.size
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    nbytes = done * words.itemsize
    what = "one-hot encode + count" if onehot_k else "popcount" if width == 1 else "pospopcnt"
    out = {"value": round(nbytes / dt / 1e9, 4), "unit": UNIT, "cores": used, "kind": "oracle",
           "sample": f"{what} oracle on the first {done} of {words.size} words ({nbytes / 2**20:.0f} MiB) "
                     f"of the same input, {dt:.1f} s wall on {used} threads",
           "cpu_model": cpu_model(), "host_cores": cores}
    if not onehot_k and width != 1 and used > 1:
        part = words[: 1 << 25]
        t1 = time.perf_counter()
        oracle.pospopcnt_mt(part, width, 1)
        out["single_core_value"] = round(part.size * words.itemsize / (time.perf_counter() - t1) / 1e9, 4)
    return out


def oracle_reference(words, width, onehot_k=0):
    """The oracle's result for the whole input: its pospopcnt on all host
    cores, or its one-hot and popcount routines over contiguous chunks on
    host threads, the chunk results added (the definition is additive)."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    cores = os.cpu_count() or 1
    if not onehot_k and width != 1:
        return oracle.pospopcnt_mt(words, width, cores)[0]
    chunk = max(1, -(-words.size // cores))
    parts = [words[i: i + chunk] for i in range(0, words.size, chunk)]
    with ThreadPoolExecutor(max_workers=cores) as ex:
        if onehot_k:
            res = list(ex.map(lambda part: oracle.onehot_counts(part, onehot_k), parts))
            return np.sum(np.stack(res), axis=0, dtype=np.uint64) if res else np.zeros(onehot_k, np.uint64)
        return np.array([sum(ex.map(oracle.popcount, parts))], dtype=np.uint64)


class CheckFailed(RuntimeError):
    """A timed result differs from the oracle's: the bench prints no value."""


def run_plain(args, world, rank, local):
    import torch
    import paper_1911_02696_gb300 as ppc
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    words, width, offset, desc = make_input(args.workload, seed=rank, log2_words=args.log2_words,
                                            onehot_k=args.onehot_k)
    nbytes = words.nbytes  # width 1 is the array popcount over bytes
    host = torch.from_numpy(words.view(np.uint8))
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    x = buf[offset: offset + nbytes]
    x.copy_(host)
    onehot_k = -width if width < 0 else 0  # negative width marks the one-hot workload (k categories)
    if onehot_k:
        width = 1
    counts = torch.empty(onehot_k or width, dtype=torch.int64, device=dev)
    ppc.pospopcnt_init(local)
    if onehot_k:
        id_dtype = {1: torch.uint8, 2: torch.int16, 4: torch.int32}[words.itemsize]

        def fn(t, counts):
            return ppc.pospopcnt_onehot_counts(t.view(id_dtype), onehot_k, counts=counts)
    elif args.kernel:  # a named kernel family in its default configuration (comparison / profiling)
        fixed = {"kernel": args.kernel}

        def fn(t, counts):
            return ppc.pospopcnt_count_config(width, fixed, t, counts=counts)
    else:
        fn = {8: ppc.pospopcnt_u8, 16: ppc.pospopcnt_u16, 32: ppc.pospopcnt_u32, 64: ppc.pospopcnt_u64,
          1: lambda t, counts: ppc.pospopcnt_popcount(t, count=counts)}[width]
    stream = torch.cuda.current_stream(dev)

    fn(x, counts=counts)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.6)
    for _ in range(args.warmup):
        fn(x, counts=counts)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    launches0 = ppc.pospopcnt_launch_count()
    dist_barrier(world)
    torch.cuda.synchronize()
    clocks.mark()
    # a short spin ahead of the first event keeps the GPU busy while the host
    # enqueues the first steps, so the region starts with work queued and
    # times device work only (the spin itself is outside the events)
    torch.cuda._sleep(3_000_000)
    ev[0].record(stream)
    for i in range(args.steps):
        fn(x, counts=counts)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    clocks.mark()
    dist_barrier(world)
    launches = ppc.pospopcnt_launch_count() - launches0
    time.sleep(0.3)
    clocks.stop()
    # the counts of the last timed step against the oracle on the whole input;
    # every rank learns every rank's verdict, so all stop together on a mismatch
    got = counts.cpu().numpy().view(np.uint64).copy()
    ref = oracle_reference(words, width, onehot_k)
    ok = bool(np.array_equal(got, ref))
    if not dist_all(ok, world, device=dev if world > 1 else None):
        raise CheckFailed(f"rank {rank}: timed counts {got.tolist()} vs the oracle's {ref.tolist()}"
                          if not ok else f"rank {rank}: another rank's timed counts differ from the oracle's")
    total_ms = ev[0].elapsed_time(ev[-1])
    per_step = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    max_ms = dist_max(total_ms, world, device=dev if world > 1 else None)
    value = whole_job_throughput(nbytes, args.steps, world, max_ms)

    # end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e and not onehot_k and width != 1:
        pinned = host.pin_memory()
        ppc.pospopcnt_count_host(width, pinned)  # allocates staging once
        k_e2e = max(1, min(args.steps, args.e2e_steps))
        dist_barrier(world)
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            got_e2e = ppc.pospopcnt_count_host(width, pinned)
        e2e_s = dist_max(time.perf_counter() - t0, world, device=dev if world > 1 else None)
        if not np.array_equal(got_e2e, ref):
            raise CheckFailed(f"rank {rank}: host-buffer counts differ from the oracle's")
        e2e = {"value": round(nbytes * k_e2e * world / e2e_s / 1e9, 3), "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": width * 8, "steps": k_e2e}

    # the metric's other two numbers, on the default workload at one GPU:
    # batched segments/s (20,000 segments, one graph-replayed launch vs 20,000
    # plain launches) and served p50 / p99 (a short trace, both modes)
    extras = None
    if (world == 1 and not args.no_extras and args.workload == "u16" and args.log2_words is None
            and not args.kernel):
        del x, buf
        torch.cuda.empty_cache()
        b = measure_batched(local, rank, 20000, warmup=3, steps=min(args.steps, 20))
        sv = measure_serve(local, rank, 50000.0, args.extras_serve_seconds, 16, 16)
        bm, pm = sv["modes"]["batched"], sv["modes"]["per_request"]
        extras = {
            "batched_segments_per_s": round(b["segments_per_s"], 1),
            "batched_GBps": round(b["GBps"], 1),
            "batched_vs_plain": round(b["plain_ms"] / b["ms"], 2),
            "serve_p50_us": round(bm["p50_ms"] * 1e3, 2), "serve_p99_us": round(bm["p99_ms"] * 1e3, 2),
            "serve_per_request_p50_us": round(pm["p50_ms"] * 1e3, 2),
            "serve_per_request_p99_us": round(pm["p99_ms"] * 1e3, 2),
            "serve_p99_vs_per_request": round(pm["p99_ms"] / bm["p99_ms"], 3),
            "extras_config": {
                "batched": f"20,000 u16 segments log-uniform [1, 2^20] words ({b['total_bytes']} bytes), one-hot "
                           f"rotated Zipf(1.1); one graph-replayed batched launch ({b['ms']:.4f} ms, mean of "
                           f"{b['steps']}) vs 20,000 plain launches from the host loop ({b['plain_ms']:.3f} ms); "
                           + b["checked"],
                "serve": f"Poisson 50,000 req/s for {args.extras_serve_seconds:g} s ({sv['requests']} requests), "
                         "widths 8/16/32, sizes log-uniform 1 KiB..256 MiB, budget 64 GiB, 16 slots in both "
                         f"modes; mean jobs per batched launch {bm['mean_jobs_per_batch']}; " + sv["checked"]},
        }
    peak, peak_src = peak_hbm()
    launch_ms = statistics.mean(per_step)
    counts_bytes = (onehot_k or width) * 8
    achieved = (nbytes + counts_bytes) / (launch_ms * 1e-3) / 1e9
    cfg = ppc.pospopcnt_get_config(16 if width == 1 else width, words.size // (2 if width == 1 else 1))
    if width == 1 and cfg["kernel"] == 2:  # the popcount keeps a 3-stage ring of the 16-bit shape
        cfg.update(stages=3, chunk_bytes=49152)
    if args.kernel:
        cfg = {"kernel": ppc.KERNELS[args.kernel], "note": "library default launch for this family"}
    kname = {1: "csa", 2: "tma", 3: "ballot"}[cfg["kernel"]]
    kernel_label = f"{kname}_kernel<{width}>"
    if onehot_k:
        cfg, kname = {"kernel": "onehot", "k": onehot_k}, "onehot"
        lw = 8 if onehot_k <= 8 else 16 if onehot_k <= 16 else 32
        idb = words.itemsize
        ring_from = (4 if idb == 1 else 8) << 20  # the library's ring_min_bytes
        kernel_label = (f"onehot_ring_kernel<{lw}, {idb}>" if nbytes >= ring_from else
                        f"onehot_lut_kernel<{lw}, {idb}, 256>" if idb <= 2 else
                        f"onehot_kernel<{idb}, {lw}, 256>") + f" ({8 * idb}-bit ids, k = {onehot_k})"
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_source": f"{peak_src} (copy bandwidth)",
                "traffic": profiled_traffic((f"onehot_k{onehot_k}" if words.itemsize == 1 else
                                             f"onehot{8 * words.itemsize}_k{onehot_k}") if onehot_k
                                            else f"{kname}_u{width}", nbytes),
                "kernel": kernel_label + " (counts written by the last block, no memset)"}
    clk = clocks.summary()
    if onehot_k > 16 and words.itemsize == 1:
        # One 8-bit id per 32-bit register: the kernel is bound by its ALU
        # pipe, not by HBM.  Its ALU operations per id, counted by ncu
        # (smsp__inst_executed_pipe_alu of a 2^27-id and a 2^30-id launch):
        # 3.26 per id between the two sizes, plus the per-CTA work (table
        # set-up, ring ramp, reduction) spread over a 2^31-id launch, 0.02:
        # 3.28.  The ALU pipe retires 16 thread-operations per cycle per SM
        # sub-partition, 64 per SM.
        sm_ghz = (clk.get("sm_mhz") or 2070.0) / 1e3
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        ids_per_s = words.size / (launch_ms * 1e-3) / 1e9
        alu_peak = 64 * sms * sm_ghz / ALU_OPS_PER_ID_ONEHOT32
        roofline = {"bound": "alu", "achieved": round(ids_per_s, 1), "peak": round(alu_peak, 1),
                    "unit": "G ids/s", "frac": round(ids_per_s / alu_peak, 4),
                    "peak_source": f"derived: 64 ALU operations per cycle per SM x {sms} SMs x {sm_ghz:.3f} GHz / "
                                   f"{ALU_OPS_PER_ID_ONEHOT32} ALU operations per id",
                    "traffic": roofline["traffic"], "kernel": roofline["kernel"],
                    "hbm": {"achieved": roofline["achieved"], "peak": peak, "unit": "GB/s",
                            "frac": roofline["frac"]}}
    out = None
    if rank == 0:
        out = {
            "metric": METRIC if width == 16 else ("onehot_counts GB/s" if onehot_k else
                                                  "popcount GB/s" if width == 1 else f"pospopcnt_u{width} GB/s"),
            "value": round(value, 2),
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(max_ms / args.steps, 5),
            "ms_per_step_median": round(statistics.median(per_step), 5), "ms_per_step_min": round(min(per_step), 5),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": f"u{8 * words.itemsize}" if onehot_k else "u8" if width == 1 else f"u{width}",
            "data": "synthetic (seeded SplitMix64 on the host)",
            "config": {"workload": desc, "n_words": int(words.size), "width": width, "start_offset_bytes": offset,
                       "bytes_per_rank_step": nbytes, "launch_config": cfg, "parallelism": f"replicas x{world}",
                       "l2": f"input {nbytes / 2**20:.0f} MiB vs L2 126 MB: "
                             + ("more than twice L2, no flush needed" if nbytes > 2 * 126_000_000 else
                                "larger than L2, partly re-read from L2" if nbytes > 126_000_000 else
                                "L2-resident (small case)")},
            "words_per_s": round(value * 1e9 / max(1, width // 8), 1),
            "pct_hbm_peak": round(100 * value / world / peak, 2),
            "roofline": roofline,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk,
            "checked": True,
            "checked_against": "oracle on the whole input (host threads), counts of the last timed step, "
                               "bit-exact",
        }
        if extras:
            out.update(extras)
        if not args.no_cpu_baseline and world == 1:
            out["cpu_baseline"] = cpu_baseline(words, width, onehot_k)
    return out


def run_sweep(args, world, rank, local):
    """u16 input-size sweep 1 KiB .. 4 GiB in powers of 4; inputs at or
    below the L2 size are reported warm (repeated) and cold (L2 flushed by
    a 256 MiB write between steps)."""
    import torch
    import paper_1911_02696_gb300 as ppc
    import synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ppc.pospopcnt_init(local)
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    counts = torch.empty(16, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)
    points = []
    big = torch.from_numpy(synth.uniform_bytes(rank, 4 << 30)).to(dev)

    def device_us(fn, reps=50):
        ts = []
        for _ in range(reps):
            torch.cuda._sleep(200000)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b) * 1e3)
        return round(statistics.median(ts), 2)

    # floors measured the same way: nothing between the events, and one
    # near-empty kernel (torch's spin kernel asked for 0 cycles)
    floors = {"events_only_us": device_us(lambda: None), "empty_kernel_us": device_us(lambda: torch.cuda._sleep(0)),
              "memset_128B_us": device_us(lambda: counts.zero_())}
    for e in range(5, 17):
        nbytes = 1 << (2 * e)
        x = big[:nbytes]
        reps = max(3, min(args.steps, int(2e9 // nbytes) + 3))
        for _ in range(args.warmup):
            ppc.pospopcnt_u16(x, counts=counts)
        res = {"bytes": nbytes}
        modes = ["warm", "cold"] if nbytes <= l2 else ["cold"]
        for mode in modes:
            ts = []
            for _ in range(reps):
                if mode == "cold" and nbytes <= l2:
                    flush.fill_(1)
                torch.cuda._sleep(200000)  # GPU busy while the host enqueues: events see device time only
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ppc.pospopcnt_u16(x, counts=counts)
                b.record(stream)
                b.synchronize()
                ts.append(a.elapsed_time(b))
            med = statistics.median(ts)
            res[mode] = {"median_us": round(med * 1e3, 2), "min_us": round(min(ts) * 1e3, 2),
                         "GBps": round(nbytes / (med * 1e-3) / 1e9, 2)}
        points.append(res)
    if rank != 0:
        return None
    return {"metric": "pospopcnt_u16 GB/s vs input size", "value": points[-1]["cold"]["GBps"], "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u16", "data": "synthetic",
            "config": {"workload": "u16 size sweep 1 KiB..4 GiB, powers of 4", "l2_bytes": l2},
            "floors": floors, "points": points}


def oracle_segments(words, off, width):
    """The oracle's rows for every segment, computed over groups of
    consecutive segments on host threads."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    nseg = off.size - 1
    cores = os.cpu_count() or 1
    bounds = np.linspace(0, nseg, min(nseg, 4 * cores) + 1).astype(np.int64)
    groups = [(int(a), int(b)) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
    with ThreadPoolExecutor(max_workers=cores) as ex:
        rows = list(ex.map(lambda g: oracle.pospopcnt_segments(words, off[g[0]: g[1] + 1], width), groups))
    return np.concatenate(rows, axis=0)


def measure_batched(local, rank, nseg, warmup, steps, autotune=False):
    """nseg segments, lengths log-uniform in [1, 2^20] words, one-hot rotated
    Zipf(1.1) per segment: one batched launch replayed from a CUDA graph vs
    nseg plain pospopcnt_u16 launches on one stream, both checked
    bit-exactly against the oracle's rows."""
    import torch
    import paper_1911_02696_gb300 as ppc
    import synth
    dev = torch.device("cuda", local)
    lens = synth.log_uniform_lengths(rank, nseg)
    off = synth.offsets_from_lengths(lens)
    words = synth.segmented_one_hot(rank, off, 16)
    x = torch.from_numpy(words.view(np.uint8)).to(dev)
    d_off = torch.from_numpy(off).to(dev)
    out = torch.empty((nseg, 16), dtype=torch.int64, device=dev)
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    tuned = None
    if autotune:  # tune the launch on this layout first (installed for width 16)
        best, best_ms = ppc.pospopcnt_batched_autotune(x, d_off, 16, counts=out, stream=s)
        tuned = {"config": best, "autotune_ms_per_call": round(best_ms, 4)}
    with torch.cuda.stream(s):
        for _ in range(max(warmup, 1)):
            ppc.pospopcnt_batched(x, d_off, 16, counts=out, stream=s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ppc.pospopcnt_batched(x, d_off, 16, counts=out, stream=s)
    for _ in range(warmup):
        g.replay()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(1, min(steps, 50))
    cur = torch.cuda.current_stream(dev)
    torch.cuda.synchronize()
    launches0 = ppc.pospopcnt_launch_count()
    a.record(cur)
    for _ in range(steps):
        g.replay()
    b.record(cur)
    torch.cuda.synchronize()
    batched_ms = a.elapsed_time(b) / steps
    got = out.cpu().numpy().view(np.uint64).copy()
    ref = oracle_segments(words, off, 16)
    if not np.array_equal(got, ref):
        raise CheckFailed(f"rank {rank}: batched rows differ from the oracle's")
    # nseg plain launches on one stream, same data: from the native host
    # loop, and replayed from a CUDA graph that captured that loop
    plain_out = torch.empty((nseg, 16), dtype=torch.int64, device=dev)
    with torch.cuda.stream(s):
        ppc.pospopcnt_plain_segments(x, off, 16, counts=plain_out, stream=s)
    s.synchronize()
    a.record(s)
    with torch.cuda.stream(s):
        ppc.pospopcnt_plain_segments(x, off, 16, counts=plain_out, stream=s)
    b.record(s)
    torch.cuda.synchronize()
    plain_ms = a.elapsed_time(b)
    if not np.array_equal(plain_out.cpu().numpy().view(np.uint64), ref):
        raise CheckFailed(f"rank {rank}: plain per-segment rows differ from the oracle's")
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2, stream=s):
        ppc.pospopcnt_plain_segments(x, off, 16, counts=plain_out, stream=s)
    g2.replay()
    torch.cuda.synchronize()
    a.record(cur)
    g2.replay()
    b.record(cur)
    torch.cuda.synchronize()
    plain_graph_ms = a.elapsed_time(b)
    total = int(off[-1]) * 2
    del g, g2, x, d_off, out, plain_out
    torch.cuda.empty_cache()
    return {"segments": nseg, "total_bytes": total, "ms": batched_ms, "steps": steps,
            "segments_per_s": nseg / (batched_ms * 1e-3), "GBps": total / (batched_ms * 1e-3) / 1e9,
            "plain_ms": plain_ms, "plain_graph_ms": plain_graph_ms, "tuned": tuned,
            "launch_config": ppc.pospopcnt_batched_get_config(16),
            "checked": "batched and plain rows equal the oracle's, bit-exact"}


def run_batched(args, world, rank, local):
    """20,000 segments, lengths log-uniform in [1, 2^20] words, one-hot
    rotated Zipf(1.1) per segment: one batched launch (replayed from a CUDA
    graph) vs 20,000 plain pospopcnt_u16 launches on one stream."""
    import torch
    import paper_1911_02696_gb300 as ppc
    torch.cuda.set_device(local)
    ppc.pospopcnt_init(local)
    m = measure_batched(local, rank, args.batched_nseg, args.warmup, args.steps, args.batched_autotune)
    nseg = m["segments"]
    if rank != 0:
        return None
    return {"metric": "batched segments/s", "value": round(m["segments_per_s"], 1), "unit": "segments/s",
            "n_gpus": world, "steps": m["steps"], "warmup": args.warmup, "ms_per_step": round(m["ms"], 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16",
            "data": "synthetic", "config": {"workload": f"{nseg:,} segments log-uniform [1, 2^20] words, one-hot "
                                                        "rotated Zipf(1.1), one graph-replayed batched launch",
                                            "total_bytes": m["total_bytes"],
                                            "launch_config": m["launch_config"],
                                            "autotuned": m["tuned"]},
            "batched_GBps": round(m["GBps"], 1),
            "plain_launches": {"ms": round(m["plain_ms"], 3),
                               "segments_per_s": round(nseg / (m["plain_ms"] * 1e-3), 1),
                               "graph_ms": round(m["plain_graph_ms"], 3),
                               "graph_segments_per_s": round(nseg / (m["plain_graph_ms"] * 1e-3), 1)},
            "speedup_vs_plain": round(m["plain_ms"] / m["ms"], 2), "checked": m["checked"]}


def run_peaks(args, world, rank, local):
    """Measured rooflines beside the driver's copy figure: a read-only scan
    (torch's fp32 sum over 2 GiB: every byte read once, nothing written),
    a device-to-device copy (read + write bytes), and the u16 pospopcnt
    kernel on the same buffer; CUDA events, best and median of the reps,
    inputs larger than L2."""
    import torch
    import paper_1911_02696_gb300 as ppc
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ppc.pospopcnt_init(local)
    nbytes = 2 << 30
    a = torch.randint(0, 1 << 30, (nbytes // 4,), dtype=torch.int32, device=dev)
    b = torch.empty_like(a)
    counts = torch.empty(16, dtype=torch.int64, device=dev)
    x16 = a.view(torch.uint8)
    reps = max(10, min(args.steps, 50))

    def timed(fn):  # back to back on the current stream, one event between reps
        for _ in range(max(args.warmup, 3)):
            fn()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
        torch.cuda.synchronize()
        ev[0].record()
        for i in range(reps):
            fn()
            ev[i + 1].record()
        torch.cuda.synchronize()
        ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(reps)]
        return min(ms), statistics.median(ms)

    af = a.view(torch.float32)
    res = {}
    for name, fn, moved in (("read_sum_fp32", lambda: torch.sum(af), nbytes),
                            ("copy_d2d", lambda: b.copy_(a), 2 * nbytes),
                            ("pospopcnt_u16", lambda: ppc.pospopcnt_u16(x16, counts=counts), nbytes)):
        best, med = timed(fn)
        res[name] = {"bytes_moved": moved, "best_ms": round(best, 4), "median_ms": round(med, 4),
                     "best_GBps": round(moved / (best * 1e-3) / 1e9, 1),
                     "median_GBps": round(moved / (med * 1e-3) / 1e9, 1)}
    peak, src = peak_hbm()
    if rank != 0:
        return None
    return {"metric": "measured rooflines GB/s", "value": res["read_sum_fp32"]["best_GBps"], "unit": UNIT,
            "n_gpus": world, "steps": reps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic (torch.randint on the device)",
            "config": {"workload": "2 GiB: read-only fp32 sum, device-to-device copy, pospopcnt_u16"},
            "results": res, "copy_peak_file": {"hbm_gbs": peak, "source": src},
            "nominal_hbm_GBps": 7900.0}


def run_l2_states(args, world, rank, local):
    """u16 at 64 MiB .. 1 GiB, each candidate configuration timed with the
    L2 in three states before each call: holding the input (warm: the same
    call repeated), full of clean lines of another buffer (a 256 MiB read),
    or full of dirty lines of another buffer (a 256 MiB write, which must be
    written back during the read).  Device time between CUDA events,
    median of 30."""
    import torch
    import paper_1911_02696_gb300 as ppc
    import synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ppc.pospopcnt_init(local)
    stream = torch.cuda.current_stream(dev)
    other = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    counts = torch.empty(16, dtype=torch.int64, device=dev)
    big = torch.from_numpy(synth.uniform_bytes(rank, 1 << 30)).to(dev)
    cands = [dict(kernel="csa", threads=128, unroll=4), dict(kernel="csa", threads=512, unroll=8),
             dict(kernel="tma", stages=4, chunk_bytes=49152), dict(kernel="tma", stages=3, chunk_bytes=65536),
             dict(kernel="tma", stages=4, chunk_bytes=49152, flags=1)]
    prep = {"warm": lambda: None, "clean": lambda: other.sum(), "dirty": lambda: other.fill_(1)}
    rows = []
    for mib in (64, 128, 256, 512, 1024):
        x = big[: mib << 20]
        default = ppc.pospopcnt_get_config(16, x.numel() // 2)
        for cfg in cands + [{"default": default}]:
            run_cfg = default if "default" in cfg else cfg
            row = {"MiB": mib, "config": cfg}
            for state, fn in prep.items():
                ts = []
                for _ in range(30):
                    fn()
                    torch.cuda._sleep(200000)
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    ppc.pospopcnt_count_config(16, run_cfg, x, counts=counts)
                    b.record(stream)
                    b.synchronize()
                    ts.append(a.elapsed_time(b) * 1e3)
                row[f"{state}_us"] = round(statistics.median(ts), 1)
            rows.append(row)
    if rank != 0:
        return None
    return {"metric": "pospopcnt_u16 device time by L2 state", "value": None, "unit": "us", "n_gpus": world,
            "steps": 30, "warmup": 0, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "u16", "data": "synthetic", "config": {"workload": "u16 64 MiB..1 GiB, three L2 states"},
            "rows": rows}


def run_ring_ab(args, world, rank, local):
    """Ring configurations of the bulk-copy kernel at 2 GiB, sustained: each
    of ten shapes counts the same buffer 300 times back to back (CUDA events
    around the calls, after 10 untimed ones) at each width, three rounds
    interleaved across the shapes, every result checked against the oracle;
    GB/s per round and the median."""
    import torch
    import paper_1911_02696_gb300 as ppc
    import synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ppc.pospopcnt_init(local)
    stream = torch.cuda.current_stream(dev)
    host = synth.uniform_bytes(rank, 2 << 30)
    x = torch.from_numpy(host).to(dev)
    shapes = [(3, 49152, 0), (3, 49152, 1), (4, 49152, 0), (3, 65536, 0), (2, 98304, 0), (2, 98304, 1),
              (4, 32768, 0), (5, 32768, 0), (2, 65536, 0), (3, 32768, 0)]
    cands = {w: [dict(kernel="tma", stages=st, chunk_bytes=ch, flags=fl) for st, ch, fl in shapes]
             for w in (8, 16, 32, 64)}
    rows = []
    calls = 300
    for width, cl in cands.items():
        counts = torch.empty(width, dtype=torch.int64, device=dev)
        ref = oracle_reference(host.view({8: np.uint8, 16: np.uint16, 32: np.uint32, 64: np.uint64}[width]), width)
        res = [[] for _ in cl]
        for _ in range(3):
            for i, cfg in enumerate(cl):
                for _ in range(10):
                    ppc.pospopcnt_count_config(width, cfg, x, counts=counts)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record(stream)
                for _ in range(calls):
                    ppc.pospopcnt_count_config(width, cfg, x, counts=counts)
                b.record(stream)
                torch.cuda.synchronize()
                if not np.array_equal(counts.cpu().numpy().view(np.uint64), ref):
                    raise CheckFailed(f"rank {rank}: ring {cfg} u{width} differs from the oracle")
                res[i].append(round(x.numel() * calls / (a.elapsed_time(b) * 1e-3) / 1e9, 1))
        default = ppc.pospopcnt_get_config(width, x.numel() // (width // 8))
        for i, cfg in enumerate(cl):
            rows.append({"width": width, "config": cfg, "GBps_rounds": res[i],
                         "median_GBps": statistics.median(res[i])})
        rows.append({"width": width, "library_default": default})
    if rank != 0:
        return None
    return {"metric": "pospopcnt GB/s by ring configuration (2 GiB, sustained)", "value": None, "unit": UNIT,
            "n_gpus": world, "steps": calls, "warmup": 10, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8/u16/u32/u64", "data": "synthetic",
            "config": {"workload": "2 GiB uniform bits, three interleaved rounds of 300 calls per shape"},
            "rows": rows, "checked": True}


def candidate_configs():
    cfgs = [dict(kernel="csa", threads=t, unroll=u) for t in (128, 256, 512) for u in (2, 4, 8)]
    cfgs += [dict(kernel="tma", stages=st, chunk_bytes=c, flags=fl) for st in (2, 3, 4, 6, 8)
             for c in (16384, 32768, 49152, 65536, 98304) for fl in (0, 1) if st * c <= 196608]
    cfgs += [dict(kernel="tma", stages=3, chunk_bytes=32768, blocks_per_sm=2, flags=fl) for fl in (0, 1)]
    cfgs += [dict(kernel="tma", stages=2, chunk_bytes=49152, blocks_per_sm=2, flags=fl) for fl in (0, 1)]
    cfgs += [dict(kernel="ballot", unroll=u) for u in (1, 2, 4)]
    return cfgs


def run_kernels(args, world, rank, local):
    """Every launch configuration of every kernel family on the 2 GiB
    uniform-bits input of each width (u8 2^31, u16 2^30, u32 2^29 words),
    plus the autotuner's pick."""
    import torch
    import paper_1911_02696_gb300 as ppc
    import synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ppc.pospopcnt_init(local)
    stream = torch.cuda.current_stream(dev)
    x = torch.from_numpy(synth.uniform_bytes(rank, 1 << 31)).to(dev)
    peak, _ = peak_hbm()
    table = {}
    steps = max(5, min(args.steps, 50))
    for width in (8, 16, 32):
        counts = torch.empty(width, dtype=torch.int64, device=dev)
        ref = None
        rows = []
        for cfg in candidate_configs():
            for _ in range(args.warmup):
                ppc.pospopcnt_count_config(width, cfg, x, counts=counts)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(steps):
                ppc.pospopcnt_count_config(width, cfg, x, counts=counts)
            b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b) / steps
            got = counts.cpu().numpy().copy()
            ref = got if ref is None else ref
            assert np.array_equal(got, ref), ("configs disagree", width, cfg)
            gbs = (1 << 31) / (ms * 1e-3) / 1e9
            rows.append({**cfg, "ms": round(ms, 4), "GBps": round(gbs, 1), "frac": round(gbs / peak, 4)})
        best, best_ms = ppc.pospopcnt_autotune(width, x, counts)
        table[f"u{width}"] = {"configs": rows, "autotune": {**best, "ms": round(best_ms, 4),
                                                            "GBps": round((1 << 31) / (best_ms * 1e-3) / 1e9, 1)}}
    if rank != 0:
        return None
    top = max(r["GBps"] for r in table["u16"]["configs"])
    return {"metric": "pospopcnt GB/s per kernel configuration", "value": top, "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8/u16/u32", "data": "synthetic",
            "config": {"workload": "2 GiB uniform random bits per width", "peak_GBps": peak}, "table": table}


def run_autotune(args, world, rank, local):
    """The library's autotuner at every size class from 64 KiB to 4 GiB for
    each width (prefixes of one 4 GiB uniform-bits buffer)."""
    import torch
    import paper_1911_02696_gb300 as ppc
    import synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ppc.pospopcnt_init(local)
    x = torch.from_numpy(synth.uniform_bytes(rank, 4 << 30)).to(dev)
    table = {}
    for width in (8, 16, 32):
        counts = torch.empty(width, dtype=torch.int64, device=dev)
        rows = []
        for e in range(8, 17):
            nbytes = 1 << (2 * e)
            best, ms = ppc.pospopcnt_autotune(width, x[:nbytes], counts)
            rows.append({"size_class": e, "bytes": nbytes, **best, "ms": round(ms, 5),
                         "GBps": round(nbytes / (ms * 1e-3) / 1e9, 1)})
        table[f"u{width}"] = rows
    if rank != 0:
        return None
    return {"metric": "autotuned configuration per size class", "value": None, "unit": UNIT, "n_gpus": world,
            "steps": 5, "warmup": 2, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u8/u16/u32", "data": "synthetic", "config": {"workload": "prefixes of 4 GiB uniform bits"},
            "table": table}


def measure_serve(local, rank, rate, seconds, slots, slots_plain, large_mib=4.0, large_inflight=0,
                  max_kib=256 * 1024, modes=("batched", "per_request"), oracle_sample=200, pool=None):
    """Serving: open-loop Poisson arrivals at `rate` per second for `seconds`
    of requests with width 8/16/32 (weights 0.2/0.6/0.2) and payloads
    log-uniform in 1 KiB..max_kib KiB, each a slice of a 4 GiB device pool of
    uniform random bits, HBM admission budget 64 GiB.  The same trace runs
    through the continuous-batching runtime and through per-request plain
    launches; latency = completion seen on the host - scheduled arrival.
    Every request's counts must be equal in both modes (each job in
    per-request mode is counted alone), and a sample of the small requests
    equal to the oracle on a host copy of their payload."""
    import torch
    import oracle
    import paper_1911_02696_gb300 as ppc
    import synth
    dev = torch.device("cuda", local)
    pool_bytes = 4 << 30
    if pool is None:
        pool = torch.from_numpy(synth.uniform_bytes(100 + rank, pool_bytes)).to(dev)
    tr = synth.serving_trace(rank, rate=rate, duration=seconds, pool_bytes=pool_bytes,
                             max_bytes=int(max_kib) * 1024)
    n = tr["t_arrival"].size
    wb = (tr["width"] // 8).astype(np.uint64)
    nbytes = tr["nwords"] * wb
    addr = np.uint64(pool.data_ptr()) + tr["offset_bytes"].astype(np.uint64)
    total = int(nbytes.sum())
    large = nbytes >= int(large_mib * (1 << 20))

    def serve(per_request):
        srv = ppc.pospopcnt_server_create(local, hbm_budget_bytes=64 << 30, per_request=per_request,
                                          max_inflight=slots_plain if per_request else slots,
                                          max_batch_jobs=1 if per_request else 240,
                                          large_job_bytes=int(large_mib * (1 << 20)),
                                          max_large_inflight=0 if per_request else large_inflight)
        try:
            # warm-up: a short slice of the trace
            k = min(n, 2000)
            ppc.pospopcnt_server_run_trace(srv, tr["t_arrival"][:k] - tr["t_arrival"][0], tr["width"][:k],
                                           addr[:k], tr["nwords"][:k])
            t0 = time.perf_counter()
            lat, counts, status, stages = ppc.pospopcnt_server_run_trace(srv, tr["t_arrival"], tr["width"], addr,
                                                                         tr["nwords"], want_counts=True,
                                                                         want_stages=True)
            wall = time.perf_counter() - t0
            st = ppc.pospopcnt_server_get_stats(srv)
        finally:
            ppc.pospopcnt_server_destroy(srv)
        if not np.all(status == 0):
            raise CheckFailed(f"rank {rank}: {int(np.sum(status != 0))} requests failed")
        q = np.percentile(lat, [50, 99, 99.9]) * 1e3

        def breakdown(mask):  # microseconds from arrival: p50 / p99 of each stage boundary
            if not mask.any():
                return None
            st_us = stages[mask] * 1e6
            out = {"requests": int(mask.sum())}
            for k, nm in enumerate(("admit", "launch", "done")):
                out[f"{nm}_p50_us"] = round(float(np.percentile(st_us[:, k], 50)), 2)
                out[f"{nm}_p99_us"] = round(float(np.percentile(st_us[:, k], 99)), 2)
            gpu = st_us[:, 2] - st_us[:, 1]
            out["launch_to_done_p50_us"] = round(float(np.percentile(gpu, 50)), 2)
            out["launch_to_done_p99_us"] = round(float(np.percentile(gpu, 99)), 2)
            return out
        return {"p50_ms": round(float(q[0]), 4), "p99_ms": round(float(q[1]), 4), "p999_ms": round(float(q[2]), 4),
                "max_ms": round(float(lat.max()) * 1e3, 4), "mean_ms": round(float(lat.mean()) * 1e3, 4),
                "aggregate_GBps": round(total / wall / 1e9, 2), "wall_s": round(wall, 3),
                "slots": slots_plain if per_request else slots,
                "batches": st["batches"], "mean_jobs_per_batch": round(st["jobs_in_batches"] / max(st["batches"], 1), 2),
                "max_batch": st["max_batch"], "deferrals": st["deferrals"],
                "max_GiB_in_flight": round(st["max_bytes_in_flight"] / 2**30, 3),
                "stages_small": breakdown(~large), "stages_large": breakdown(large)}, counts

    res, counts = {}, {}
    for mode in modes:
        res[mode], counts[mode] = serve(mode == "per_request")
    if len(counts) == 2 and not np.array_equal(counts["batched"], counts["per_request"]):
        raise CheckFailed(f"rank {rank}: served counts differ between the batched mix and requests counted alone")
    # a sample of the requests below 1 MiB against the oracle on their bytes
    small = np.flatnonzero(nbytes < (1 << 20))
    rng = np.random.default_rng(rank)
    sample = rng.choice(small, size=min(small.size, oracle_sample), replace=False) if small.size else small
    for i in sample:
        w, o = int(tr["width"][i]), int(tr["offset_bytes"][i])
        host = pool[o: o + int(nbytes[i])].cpu().numpy()
        ref = oracle.pospopcnt(host, w)
        for mode in counts:
            if not np.array_equal(counts[mode][i, :w], ref):
                raise CheckFailed(f"rank {rank}: request {i} ({mode}) differs from the oracle")
    return {"requests": int(n), "total_bytes": total, "offered_GBps": total / seconds / 1e9, "modes": res,
            "checked": (f"every request equal in both modes (per-request = each job counted alone); "
                        f"{sample.size} requests below 1 MiB equal to the oracle") if len(counts) == 2 else
                       f"{sample.size} requests below 1 MiB equal to the oracle"}


def run_serve(args, world, rank, local):
    """Serving at one load: the continuous-batching runtime and per-request
    plain launches on the same trace (see measure_serve), `--serve-runs`
    times each, median and spread of p50 / p99."""
    import torch
    import paper_1911_02696_gb300 as ppc
    import synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ppc.pospopcnt_init(local)
    pool = torch.from_numpy(synth.uniform_bytes(100 + rank, 4 << 30)).to(dev)
    runs = []
    for r in range(max(1, args.serve_runs)):
        runs.append(measure_serve(local, rank, args.serve_rate, args.serve_seconds, args.serve_slots,
                                  args.serve_slots_plain, args.serve_large_mib, args.serve_large_inflight,
                                  args.serve_max_kib, pool=pool))
    if rank != 0:
        return None

    def spread(mode, key):
        v = [r["modes"][mode][key] for r in runs]
        return {"median": statistics.median(v), "min": min(v), "max": max(v), "runs": v}
    summary = {mode: {k: spread(mode, k) for k in ("p50_ms", "p99_ms", "p999_ms", "mean_jobs_per_batch")}
               for mode in ("batched", "per_request")}
    last = runs[-1]
    return {"metric": "served p99 latency", "value": summary["batched"]["p99_ms"]["median"], "unit": "ms",
            "n_gpus": world, "steps": len(runs), "warmup": 1, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8/u16/u32", "data": "synthetic",
            "config": {"workload": f"Poisson {args.serve_rate:g} req/s for {args.serve_seconds:g} s, widths 8/16/32 "
                                   f"(0.2/0.6/0.2), sizes log-uniform 1 KiB..{args.serve_max_kib:g} KiB, 4 GiB "
                                   "device pool, budget 64 GiB",
                       "requests": last["requests"], "total_GB": round(last["total_bytes"] / 1e9, 2),
                       "offered_GBps": round(last["offered_GBps"], 1),
                       "batched_slots": args.serve_slots, "per_request_slots": args.serve_slots_plain,
                       "large_job_MiB": args.serve_large_mib, "max_large_inflight": args.serve_large_inflight},
            "summary": summary,
            "p99_speedup_vs_per_request": round(summary["per_request"]["p99_ms"]["median"] /
                                                summary["batched"]["p99_ms"]["median"], 2),
            "runs": [r["modes"] for r in runs], "checked": last["checked"]}


def run_e2e(args, world, rank, local):
    """Host-buffer counting of 2^30 u16 words: pinned memory read in place,
    pageable memory through the staging copies, and a plain pinned copy to
    the device (the link reference), all through public calls."""
    import torch
    import oracle
    import paper_1911_02696_gb300 as ppc
    import synth
    torch.cuda.set_device(local)
    ppc.pospopcnt_init(local)
    words = synth.uniform_bits(rank, 1 << 30, 16)
    nbytes = words.nbytes
    pinned = torch.from_numpy(words.view(np.uint8)).pin_memory()
    dev = torch.empty(nbytes, dtype=torch.uint8, device=torch.device("cuda", local))

    def rate(f, reps):
        f()
        t0 = time.perf_counter()
        for _ in range(reps):
            f()
        return nbytes * reps / (time.perf_counter() - t0) / 1e9

    def copy():
        dev.copy_(pinned, non_blocking=True)
        torch.cuda.synchronize()
    k = max(2, min(args.steps, 10))
    res = {"pinned_in_place_GBps": round(rate(lambda: ppc.pospopcnt_count_host(16, pinned), k), 2),
           "pinned_is_mapped": ppc.pospopcnt_host_is_mapped(pinned),
           "pageable_staged_GBps": round(rate(lambda: ppc.pospopcnt_count_host(16, words), max(2, k // 2)), 2),
           "memcpy_pinned_GBps": round(rate(copy, k), 2)}
    ref, _ = oracle.pospopcnt_mt(words, 16)
    res["bit_exact"] = bool(np.array_equal(ppc.pospopcnt_count_host(16, pinned), ref) and
                            np.array_equal(ppc.pospopcnt_count_host(16, words), ref))
    if rank != 0:
        return None
    return {"metric": "pospopcnt_u16 GB/s from host memory", "value": res["pinned_in_place_GBps"], "unit": UNIT,
            "n_gpus": world, "steps": k, "warmup": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u16", "data": "synthetic",
            "config": {"workload": "pospopcnt_count_host, n=2^30 u16 words (2 GiB) in host memory"}, **res,
            "frac_of_link": round(res["pinned_in_place_GBps"] / res["memcpy_pinned_GBps"], 4)}


REFERENCE_WORKLOADS = ("u16", "u16_onehot", "u16_sparse", "u16_misaligned", "u8", "u8_onehot", "u32", "u32_onehot",
                       "u64", "popcount", "onehot",
                       "onehot_u16ids", "onehot_u32ids")


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle on the host cores, on the same
    workload and config as our arm, each step a bounded sample of it (its
    first 2^26 words, which the generators make identically)."""
    if rank != 0:
        return None
    import oracle
    kind = args.workload if args.workload in REFERENCE_WORKLOADS else "u16"
    words, width, offset, desc = make_input(kind, seed=0, log2_words=args.log2_words, limit=1 << 26,
                                            onehot_k=args.onehot_k)
    onehot_k = -width if width < 0 else 0
    cores = os.cpu_count() or 1

    def step():
        if onehot_k:
            oracle.onehot_counts(words, onehot_k)
            return 1
        if width == 1:
            oracle.popcount(words)
            return 1
        return oracle.pospopcnt_mt(words, width, cores)[1]

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    used = 1
    for _ in range(args.steps):
        used = step()
    dt = time.perf_counter() - t0
    nbytes = words.size * words.itemsize
    value = nbytes * args.steps / dt / 1e9
    metric = METRIC if width == 16 else ("onehot_counts GB/s" if onehot_k else
                                         "popcount GB/s" if width == 1 else f"pospopcnt_u{width} GB/s")
    sample = f"the first {words.size} words ({nbytes >> 20} MiB) of the workload per step, {used} threads"
    return {"impl": "reference", "metric": metric,
            "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt * 1e3 / args.steps, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": f"u{8 * words.itemsize}" if width < 0 else "u8" if width == 1 else f"u{width}",
            "data": "synthetic (seeded SplitMix64 on the host)",
            "config": {"workload": desc, "width": 1 if onehot_k else width, "start_offset_bytes": offset,
                       "parallelism": "replicas x1", "sample_per_step": sample},
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": used, "kind": "oracle",
                             "sample": sample, "cpu_model": cpu_model(), "host_cores": cores},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="u16",
                   choices=["u16", "u16_onehot", "u16_sparse", "u16_misaligned", "u8", "u8_onehot", "u32", "u32_onehot",
                            "u64", "popcount", "onehot",
                            "onehot_u16ids", "onehot_u32ids", "sweep", "batched",
                            "kernels", "autotune", "serve", "e2e", "peaks", "l2_states",
                            "ring_ab"])
    p.add_argument("--batched-nseg", type=int, default=20000)
    p.add_argument("--onehot-k", type=int, default=16, choices=range(1, 33), metavar="K",
                   help="one-hot workloads: number of categories (1..32)")
    p.add_argument("--batched-autotune", action="store_true",
                   help="batched workload: autotune the launch on the layout before timing")
    p.add_argument("--serve-rate", type=float, default=50000.0)
    p.add_argument("--serve-seconds", type=float, default=60.0)
    p.add_argument("--serve-slots", type=int, default=16, help="batches in flight (continuous batching)")
    p.add_argument("--serve-slots-plain", type=int, default=16, help="requests in flight (per-request mode)")
    p.add_argument("--serve-runs", type=int, default=1, help="serving: runs of each mode (median and spread)")
    p.add_argument("--serve-max-kib", type=float, default=256 * 1024,
                   help="serving: largest payload in KiB (sizes log-uniform from 1 KiB)")
    p.add_argument("--serve-large-mib", type=float, default=4.0,
                   help="jobs at least this large are launched on their own")
    p.add_argument("--serve-large-inflight", type=int, default=0,
                   help="large jobs on the GPU at once in continuous batching (0: no limit)")
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--kernel", choices=["csa", "tma", "ballot"], default=None,
                   help="time one kernel family instead of the tuned default")
    p.add_argument("--log2-words", type=int, default=None,
                   help="run a smaller uniform-bits case of 2^k words (profiling only)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="default workload: skip the batched and serving numbers")
    p.add_argument("--extras-serve-seconds", type=float, default=5.0,
                   help="default workload: length of the serving trace per mode")
    args = p.parse_args(argv)
    if args.warmup < 3:
        p.error("--warmup must be >= 3")
    world, rank, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, world, rank)
    else:
        import torch
        if world > 1:
            torch.cuda.set_device(local)
            dist_init(world, "nccl")
        if args.workload == "sweep":
            out = run_sweep(args, world, rank, local)
        elif args.workload == "batched":
            out = run_batched(args, world, rank, local)
        elif args.workload == "kernels":
            out = run_kernels(args, world, rank, local)
        elif args.workload == "autotune":
            out = run_autotune(args, world, rank, local)
        elif args.workload == "serve":
            out = run_serve(args, world, rank, local)
        elif args.workload == "e2e":
            out = run_e2e(args, world, rank, local)
        elif args.workload == "peaks":
            out = run_peaks(args, world, rank, local)
        elif args.workload == "l2_states":
            out = run_l2_states(args, world, rank, local)
        elif args.workload == "ring_ab":
            out = run_ring_ab(args, world, rank, local)
        else:
            out = run_plain(args, world, rank, local)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)
    return 0


def cli(argv=None) -> int:
    """main() with the result check's verdict as the exit status: a timed
    result that differs from the oracle's prints no value and returns 3."""
    try:
        return main(argv)
    except CheckFailed as exc:
        print(f"bench: result check failed, no value printed: {exc}", file=sys.stderr, flush=True)
        return 3


if __name__ == "__main__":
    sys.exit(cli())
