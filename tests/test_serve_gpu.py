"""The serving runtime on the GPU: every request's counts are the same
served alone (its own plain count) and served in the mix of a
continuously batched open-loop trace, and both equal the CPU oracle
(tolerance 0).  Also the submit/poll interface, per-request mode, the HBM
budget (deferral, never exceeded) and rejection of oversized jobs."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_1911_02696_gb300 as ppc  # noqa: E402

pytestmark = pytest.mark.gpu

POOL = 64 << 20


@pytest.fixture(scope="module")
def pool():
    host = synth.uniform_bytes(77, POOL)
    dev = torch.from_numpy(host).cuda()
    return host, dev


def _trace(seed, rate, duration, max_bytes):
    return synth.serving_trace(seed, rate=rate, duration=duration, pool_bytes=POOL, max_bytes=max_bytes)


def _oracle_rows(host, tr):
    rows = np.zeros((tr["t_arrival"].size, 32), dtype=np.uint64)
    for i in range(rows.shape[0]):
        w = int(tr["width"][i])
        a = int(tr["offset_bytes"][i])
        nb = int(tr["nwords"][i]) * (w // 8)
        rows[i, :w] = oracle.pospopcnt(host[a:a + nb], w)
    return rows


def _solo_rows(dev, tr):
    """Each request alone: one plain pospopcnt call on its slice."""
    n = tr["t_arrival"].size
    out = torch.zeros((n, 32), dtype=torch.int64, device="cuda")
    for i in range(n):
        w = int(tr["width"][i])
        a = int(tr["offset_bytes"][i])
        nb = int(tr["nwords"][i]) * (w // 8)
        ppc.pospopcnt_count(w, dev[a:a + nb], counts=out[i, :w])
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint64)


def _run(server, dev, tr):
    addr = dev.data_ptr() + tr["offset_bytes"].astype(np.uint64)
    lat, counts, status = ppc.pospopcnt_server_run_trace(server, tr["t_arrival"], tr["width"], addr, tr["nwords"],
                                                         want_counts=True)
    return lat, counts, status


def test_same_alone_and_in_the_mix(pool):
    host, dev = pool
    tr = _trace(1, rate=20000, duration=0.15, max_bytes=4 << 20)
    # one slot: every job that arrives while a batch runs joins the next one
    # (about a fifth of the arrivals at this rate), so batching does not
    # depend on how fast the GPU drains the others
    srv = ppc.pospopcnt_server_create(0, max_inflight=1, max_batch_jobs=240)
    try:
        lat, mixed, status = _run(srv, dev, tr)
        st = ppc.pospopcnt_server_get_stats(srv)
    finally:
        ppc.pospopcnt_server_destroy(srv)
    assert np.all(status == 0)
    assert np.all(np.isfinite(lat)) and np.all(lat > 0)
    alone = _solo_rows(dev, tr)
    ref = _oracle_rows(host, tr)
    assert np.array_equal(alone, ref)
    assert np.array_equal(mixed, ref)
    # it really batched: fewer launches than requests, several jobs per batch
    assert st["completed"] == tr["t_arrival"].size
    assert st["batches"] < st["completed"] and st["max_batch"] > 1


def test_per_request_mode_same_results(pool):
    host, dev = pool
    tr = _trace(2, rate=5000, duration=0.1, max_bytes=1 << 20)
    srv = ppc.pospopcnt_server_create(0, per_request=True, max_inflight=16)
    try:
        lat, counts, status = _run(srv, dev, tr)
        st = ppc.pospopcnt_server_get_stats(srv)
    finally:
        ppc.pospopcnt_server_destroy(srv)
    assert np.all(status == 0)
    assert st["batches"] == st["completed"] == tr["t_arrival"].size
    assert np.array_equal(counts, _oracle_rows(host, tr))


def test_budget_defers_and_holds(pool):
    host, dev = pool
    budget = 3 << 20
    # a burst: ~400 requests (~60 MB) arriving within 4 microseconds
    tr = _trace(3, rate=1e8, duration=4e-6, max_bytes=1 << 20)
    assert tr["t_arrival"].size > 100
    srv = ppc.pospopcnt_server_create(0, hbm_budget_bytes=budget, max_inflight=4, max_batch_jobs=64)
    try:
        lat, counts, status = _run(srv, dev, tr)
        st = ppc.pospopcnt_server_get_stats(srv)
    finally:
        ppc.pospopcnt_server_destroy(srv)
    assert np.all(status == 0)
    assert st["max_bytes_in_flight"] <= budget
    assert st["deferrals"] > 0
    assert np.array_equal(counts, _oracle_rows(host, tr))


def test_submit_poll_and_rejection(pool):
    host, dev = pool
    srv = ppc.pospopcnt_server_create(0, hbm_budget_bytes=1 << 20, max_inflight=2, max_batch_jobs=8)
    try:
        with pytest.raises(ppc.PospopcntError) as e:
            ppc.pospopcnt_server_submit(srv, 16, dev[: 2 << 20], 99)
        assert e.value.status == 6
        rng = np.random.default_rng(4)
        jobs = {}
        for tag in range(100):
            w = int(rng.choice([8, 16, 32]))
            nb = int(rng.integers(0, 4096)) * (w // 8)
            a = int(rng.integers(0, 1000)) * (w // 8)
            ppc.pospopcnt_server_submit(srv, w, dev[a:a + nb], tag)
            jobs[tag] = (w, a, nb)
        got = {}
        import time
        t_end = time.time() + 30
        while len(got) < 100 and time.time() < t_end:
            for r in ppc.pospopcnt_server_poll(srv):
                got[r["tag"]] = r
        st = ppc.pospopcnt_server_get_stats(srv)
    finally:
        ppc.pospopcnt_server_destroy(srv)
    assert len(got) == 100 and st["rejected"] == 1
    for tag, (w, a, nb) in jobs.items():
        r = got[tag]
        assert r["status"] == 0 and r["width"] == w
        assert r["t_arrival"] <= r["t_admit"] <= r["t_launch"] <= r["t_done"]
        assert np.array_equal(r["counts"], oracle.pospopcnt(host[a:a + nb], w))


def test_mixed_routes_same_results(pool):
    """Small jobs batched and large jobs on their own launches, in one mix."""
    host, dev = pool
    tr = _trace(5, rate=20000, duration=0.1, max_bytes=8 << 20)
    srv = ppc.pospopcnt_server_create(0, max_inflight=8, large_job_bytes=256 << 10)
    try:
        lat, mixed, status = _run(srv, dev, tr)
        st = ppc.pospopcnt_server_get_stats(srv)
    finally:
        ppc.pospopcnt_server_destroy(srv)
    assert np.all(status == 0)
    nbytes = tr["nwords"].astype(np.int64) * (tr["width"] // 8)
    assert np.any(nbytes >= 256 << 10) and np.any(nbytes < 256 << 10)
    assert np.array_equal(mixed, _oracle_rows(host, tr))
    assert np.array_equal(mixed, _solo_rows(dev, tr))
    assert st["completed"] == tr["t_arrival"].size


def test_high_rate_batches_form_and_results_match(pool):
    """Arrivals faster than one launch per request (400k req/s of payloads up
    to 64 KiB for 0.25 s) with 16 slots in both modes: continuous batching
    puts several jobs in a launch, and every request's counts are the same in
    the batched mix, in per-request mode (each job counted alone) and in the
    oracle."""
    host, dev = pool
    tr = _trace(9, rate=400000, duration=0.25, max_bytes=64 << 10)
    res = {}
    for per_request in (False, True):
        srv = ppc.pospopcnt_server_create(0, max_inflight=16, per_request=per_request,
                                          max_batch_jobs=1 if per_request else 240)
        try:
            lat, counts, status = _run(srv, dev, tr)
            st = ppc.pospopcnt_server_get_stats(srv)
        finally:
            ppc.pospopcnt_server_destroy(srv)
        assert np.all(status == 0)
        assert st["completed"] == tr["t_arrival"].size
        res[per_request] = (counts, st)
    batched, st_b = res[False]
    assert st_b["max_batch"] > 1 and st_b["batches"] < st_b["completed"]
    assert np.array_equal(batched, res[True][0])
    assert np.array_equal(batched, _oracle_rows(host, tr))
