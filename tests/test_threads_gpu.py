"""Calls from several host threads at once, each on its own stream: plain
counts of every width, batched counts and one-hot counts, all checked
against the oracle.  The library's shared state (device workspace, launch
configurations, work-queue slots, shared-memory limits) is taken under its
locks, so concurrent first calls and steady traffic give exact results."""
import threading

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_1911_02696_gb300 as ppc  # noqa: E402

pytestmark = pytest.mark.gpu


def _worker(tid, errors):
    try:
        torch.cuda.set_device(0)
        s = torch.cuda.Stream()
        rng = np.random.default_rng(tid)
        for it in range(6):
            width = (8, 16, 32, 64)[(tid + it) % 4]
            n = int(rng.integers(1, 1 << 20))
            words = synth.uniform_bits(tid * 100 + it, n, width)
            with torch.cuda.stream(s):
                x = torch.from_numpy(words.view(np.uint8)).to("cuda", non_blocking=False)
                got = ppc.pospopcnt_count(width, x, stream=s)
                lens = rng.integers(0, 5000, size=40).astype(np.int64)
                off = synth.offsets_from_lengths(lens)
                seg = synth.uniform_bits(tid * 100 + it + 50, int(off[-1]), 16)
                xs = torch.from_numpy(seg.view(np.uint8)).to("cuda")
                rows = ppc.pospopcnt_batched(xs, torch.from_numpy(off).to("cuda"), 16, stream=s)
                ids = synth.categorical_ids(tid + it, 1 << 16, synth.zipf_cdf(20), np.uint8)
                hist = ppc.pospopcnt_onehot_counts(torch.from_numpy(ids).to("cuda"), 16, stream=s)
            s.synchronize()
            assert np.array_equal(got.cpu().numpy().view(np.uint64), oracle.pospopcnt(words, width)), (tid, it)
            assert np.array_equal(rows.cpu().numpy().view(np.uint64), oracle.pospopcnt_segments(seg, off, 16))
            assert np.array_equal(hist.cpu().numpy().view(np.uint64), oracle.onehot_counts(ids, 16))
        ppc.pospopcnt_release_stream(s)
    except Exception as e:  # reported by the main thread
        errors.append((tid, repr(e)))


def test_concurrent_host_threads():
    errors = []
    threads = [threading.Thread(target=_worker, args=(t, errors)) for t in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not any(t.is_alive() for t in threads), "a worker thread did not finish"
    assert not errors, errors
    assert ppc.pospopcnt_check_device_error() == 0
