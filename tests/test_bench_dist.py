"""bench.py's multi-rank harness on CPU with the gloo backend (world size
2): the slowest rank's time is what every rank reports, the whole-job value
counts every rank's bytes, a result check failing on one rank fails on every
rank, and under torchrun only rank 0 prints its JSON line.  The data path itself has no collective (each rank counts its own
input), so nothing else crosses ranks."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    bench.dist_init(world, "gloo")
    slowest = bench.dist_max(10.0 + rank, world)
    bench.dist_barrier(world)
    value = bench.whole_job_throughput(1 << 31, 100, world, slowest * 1000)
    # a result check that fails on one rank fails on every rank
    all_ok = bench.dist_all(True, world)
    one_bad = bench.dist_all(rank != 1, world)
    q.put((rank, slowest, value, all_ok, one_bad))
    dist.destroy_process_group()


def test_gloo_max_and_whole_job_value():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slowest, value, all_ok, one_bad in got:
        assert slowest == 11.0  # the max over ranks, on every rank
        assert value == pytest.approx(2 * 100 * (1 << 31) / 11.0 / 1e9)
        assert all_ok is True and one_bad is False


def test_torchrun_reference_arm_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
    # same workload and metric as the GPU arm's default line
    sys.path.insert(0, ROOT)
    import bench
    _, width, _, desc = bench.make_input("u16", seed=0, limit=16)
    assert d["config"]["workload"] == desc and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True
