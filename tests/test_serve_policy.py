"""The serving runtime's admission policy on a mock clock (no device):
oldest-first admission while the admitted, not yet completed payload bytes
fit the HBM budget; jobs larger than the budget are rejected.  Checked
against a plain event-by-event Python model of the same rule and against
the invariants it must keep."""
import heapq
import math

import numpy as np
import pytest

import paper_1911_02696_gb300 as ppc


def model(budget, t_arr, nbytes, service):
    """Reference: process arrivals and completions in time order; after every
    event admit from the head of the queue while the head fits."""
    n = len(t_arr)
    t_admit = [math.nan] * n
    status = [0] * n
    queue, running, in_flight, nxt = [], [], 0, 0
    while nxt < n or queue:
        t_a = t_arr[nxt] if nxt < n else math.inf
        t_d = running[0][0] if running else math.inf
        if t_d <= t_a:
            clock = t_d
            while running and running[0][0] <= clock:
                _, b = heapq.heappop(running)
                in_flight -= b
        else:
            clock = t_a
            if nbytes[nxt] > budget:
                status[nxt] = 6
            else:
                queue.append(nxt)
            nxt += 1
        while queue and in_flight + nbytes[queue[0]] <= budget:
            j = queue.pop(0)
            in_flight += nbytes[j]
            t_admit[j] = clock
            heapq.heappush(running, (clock + service[j], nbytes[j]))
    return np.array(t_admit), np.array(status)


def test_small_example():
    t, s = ppc.pospopcnt_admission_simulate(10, [0, 0, 0, 1, 1], [6, 4, 5, 20, 1], [2, 2, 2, 2, 2])
    assert list(s) == [0, 0, 0, 6, 0]
    assert list(t[[0, 1, 2, 4]]) == [0, 0, 2, 2] and math.isnan(t[3])


@pytest.mark.parametrize("seed", range(6))
def test_matches_model_and_keeps_budget(seed):
    rng = np.random.default_rng(seed)
    n = 400
    budget = int(rng.integers(50, 500))
    t_arr = np.cumsum(rng.exponential(0.01, size=n))
    nbytes = rng.integers(1, budget + budget // 4, size=n).astype(np.uint64)  # some too large
    service = rng.uniform(0.001, 0.2, size=n)
    t_admit, status = ppc.pospopcnt_admission_simulate(budget, t_arr, nbytes, service)
    ref_t, ref_s = model(budget, list(t_arr), [int(b) for b in nbytes], list(service))
    assert np.array_equal(status, ref_s)
    assert np.allclose(np.nan_to_num(t_admit, nan=-1), np.nan_to_num(ref_t, nan=-1), rtol=0, atol=0)
    ok = status == 0
    assert np.all((status == 6) == (nbytes > budget))
    # FIFO and no admission before arrival
    ta = t_admit[ok]
    assert np.all(np.diff(ta) >= 0) and np.all(ta >= t_arr[ok])
    # the budget holds at every admission instant
    ends = t_admit + service
    for j in np.nonzero(ok)[0]:
        live = ok & (t_admit <= t_admit[j]) & (ends > t_admit[j])
        assert int(nbytes[live].sum()) <= budget


def test_no_wait_when_idle():
    t, s = ppc.pospopcnt_admission_simulate(1 << 30, [0.0, 0.5, 1.0], [10, 10, 10], [0.1, 0.1, 0.1])
    assert list(t) == [0.0, 0.5, 1.0] and list(s) == [0, 0, 0]


def test_rejects_bad_arguments():
    lib = ppc.load()
    assert lib.pospopcnt_admission_simulate(10, 3, None, None, None, None, None) == 1
    with pytest.raises(ppc.PospopcntError):
        ppc.pospopcnt_admission_simulate(10, [1.0, 0.5], [1, 1], [1, 1])  # arrivals out of order


def test_serving_trace_shape():
    import synth
    tr = synth.serving_trace(0, rate=50000, duration=0.2, pool_bytes=1 << 30)
    n = tr["t_arrival"].size
    assert 9000 < n < 11000
    assert np.all(np.diff(tr["t_arrival"]) >= 0) and tr["t_arrival"][-1] < 0.2
    wb = tr["width"] // 8
    nbytes = tr["nwords"].astype(np.int64) * wb
    assert nbytes.min() >= 1000 and nbytes.max() <= 256 << 20
    assert np.all(tr["offset_bytes"] % wb == 0) and np.all(tr["offset_bytes"] + nbytes <= 1 << 30)
    frac16 = np.mean(tr["width"] == 16)
    assert 0.55 < frac16 < 0.65
