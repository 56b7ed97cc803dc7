"""Fused one-hot encode + count on the GPU against the oracle (which one-hot
encodes each id and then counts positions, §1): every id width, k on both
sides of the 8/16/32-bit lane boundaries, ids >= k present, every small
length at every aligned start, ragged large sizes, skewed ids, both 8-bit-id
kernels (register loads below 4 MiB of 8-bit ids or 8 MiB of wider ids,
bulk-copy ring above; 32-bit ids too), 2 GiB."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_1911_02696_gb300 as ppc  # noqa: E402

pytestmark = pytest.mark.gpu
DT = {1: np.uint8, 2: np.uint16, 4: np.uint32}
TORCH_DT = {1: torch.uint8, 2: torch.int16, 4: torch.int32}


def _dev(ids, offset):
    """Device copy of the ids, `offset` bytes past a 256-byte boundary, with
    guard bytes around it."""
    b = ids.view(np.uint8)
    buf = torch.full((256 + offset + b.size + 256,), 0x07, dtype=torch.uint8, device="cuda")
    if b.size:
        buf[256 + offset: 256 + offset + b.size].copy_(torch.from_numpy(b))
    x = buf[256 + offset: 256 + offset + b.size]
    return x if ids.itemsize == 1 else x.view(TORCH_DT[ids.itemsize])


def _run(ids, k, offset=0):
    x = _dev(ids, offset)
    full = torch.full((k + 4,), -9, dtype=torch.int64, device="cuda")
    ppc.pospopcnt_onehot_counts(x, k, counts=full[:k])
    torch.cuda.synchronize()
    got = full.cpu().numpy()
    assert np.all(got[k:] == -9)
    return got[:k].view(np.uint64)


@pytest.mark.parametrize("idb", [1, 2, 4])
@pytest.mark.parametrize("k", [1, 3, 8, 9, 16, 17, 32])
def test_small_lengths_every_offset(idb, k):
    rng = np.random.default_rng(idb * 100 + k)
    ids = rng.integers(0, 2 * k + 2, size=200).astype(DT[idb])
    for offset in range(0, 16, idb):
        for n in list(range(0, 40)) + [63, 64, 65, 127, 128, 129, 199, 200]:
            assert np.array_equal(_run(ids[:n], k, offset), oracle.onehot_counts(ids[:n], k)), (offset, n)


@pytest.mark.parametrize("idb", [1, 2, 4])
def test_ragged_large_and_skewed(idb):
    rng = np.random.default_rng(idb)
    for k in (5, 16, 32):
        for _ in range(3):
            n = int(rng.integers(1, (24 << 20) // idb))
            ids = synth.categorical_ids(int(rng.integers(1 << 30)), n, synth.zipf_cdf(min(2 * k, 64)), DT[idb])
            off = int(rng.integers(0, 16 // idb)) * idb
            assert np.array_equal(_run(ids, k, off), oracle.onehot_counts(ids, k))


@pytest.mark.parametrize("k", [1, 7, 8, 12, 16, 20, 32])
def test_u8_every_id_value(k):
    """8-bit ids over all 256 values (most of them >= k, each of which must
    encode to nothing), at lengths that end a thread's run of vectors
    anywhere inside its last trip."""
    rng = np.random.default_rng(k)
    for n in (16 * 256 * 8 - 16, 16 * 256 * 8 + 16, 3 * (1 << 20) + 5, (1 << 22) + 16 * 4 * 256 * 3 + 1):
        ids = rng.integers(0, 256, size=n).astype(np.uint8)
        assert np.array_equal(_run(ids, k, int(rng.integers(0, 16))), oracle.onehot_counts(ids, k)), n


@pytest.mark.parametrize("idb", [1, 2, 4])
@pytest.mark.parametrize("k", [3, 8, 16, 17, 32])
def test_bulk_copy_sizes(idb, k):
    """Ids from 4 MiB (8-bit) or 8 MiB (16- and 32-bit) up go through bulk
    copies into a shared-memory ring (8- and 16-bit ids encoded by table
    lookups, 32-bit ids by shift and mask): the exact threshold and just
    below it, a ragged chunk count, a partial last chunk at an odd start,
    ids over the whole id range (for 32-bit ids, also ids below 64, most of
    them counted) and skewed ids."""
    rng = np.random.default_rng(100 + k + 1000 * idb)
    top = {1: 256, 2: 65536, 4: 1 << 32}[idb]
    ring_from = (4 if idb == 1 else 8) << 20
    sizes = [(ring_from, 0), (ring_from - 16, 0), (152 * 32768 * 7 + 16 * 100 + 3, 5), ((40 << 20) + 17, 3)]
    for nbytes, off in sizes:
        n = nbytes // idb
        ids = rng.integers(0, top, size=n).astype(DT[idb])
        if idb == 4 and nbytes % 2:
            ids = rng.integers(0, 64, size=n).astype(DT[idb])
        assert np.array_equal(_run(ids, k, off - off % idb), oracle.onehot_counts(ids, k)), (n, off)
    ids = synth.categorical_ids(k, ((48 << 20) + 9) // idb, synth.zipf_cdf(min(2 * k, 64)), DT[idb])
    assert np.array_equal(_run(ids, k, idb), oracle.onehot_counts(ids, k))


@pytest.mark.parametrize("k", [1, 3, 8, 9, 16])
def test_u8_pairs_and_mixed_trips(k):
    """8-bit ids all below 16 take the pair-table path of the bulk-copy
    kernel (k <= 16), trips holding any id of 16 or more take the
    shift-and-mask path: ids below k only, ids in [k, 16) (counted nowhere,
    still the pair path), and the same input with a few ids >= 16 planted
    at random places so that some trips switch path."""
    rng = np.random.default_rng(300 + k)
    n = (40 << 20) + 11
    below_k = rng.integers(0, k, size=n).astype(np.uint8)
    assert np.array_equal(_run(below_k, k, 3), oracle.onehot_counts(below_k, k))
    below_16 = rng.integers(0, 16, size=n).astype(np.uint8)
    assert np.array_equal(_run(below_16, k, 0), oracle.onehot_counts(below_16, k))
    mixed = below_16.copy()
    spots = rng.choice(n, size=200, replace=False)
    mixed[spots] = rng.integers(16, 256, size=spots.size).astype(np.uint8)
    mixed[spots[:50]] = 16  # the smallest id outside the pair table
    got = _run(mixed, k, 5)
    assert np.array_equal(got, oracle.onehot_counts(mixed, k))
    assert int(got.sum()) == int(np.sum(mixed < k))


@pytest.mark.parametrize("k", [20, 32])
def test_ring_warp_flush_one_id_per_register(k):
    """17..32 categories on the bulk-copy path: each warp transposes its
    lanes' carry registers so that lane p collects position p.  Ids that are
    a function of the 16-byte vector's index (so of the lane that counts
    them; ids 20..31 count nothing at k = 20), and one constant id per input
    at the edges of the transpose's 16-, 8-, 4-, 2- and 1-column blocks,
    each with a partial last ring chunk."""
    n = (40 << 20) + 4099
    v = np.arange(n, dtype=np.int64) // 16
    ids = ((v * 7 + (v >> 5)) % 32).astype(np.uint8)
    assert np.array_equal(_run(ids, k, 1), oracle.onehot_counts(ids, k))
    for c in (0, 1, 2, 3, 4, 7, 8, 15, 16, 23, 24, 31):
        ids = np.full(n, c, dtype=np.uint8)
        got = _run(ids, k)
        assert np.array_equal(got, oracle.onehot_counts(ids, k)), c
        assert int(got.sum()) == (n if c < k else 0), c


@pytest.mark.parametrize("k", [1, 8, 16, 32])
def test_u16_ids_with_high_bytes(k):
    """16-bit ids whose low byte is a valid category but whose high byte is
    not zero (257, 0x1F01, 0xFF00 + j, 0xFFFF) must count nowhere; mixed
    with valid ids, at sizes for both 16-bit-id kernels."""
    rng = np.random.default_rng(7 + k)
    decoys = np.array([256 + j for j in range(32)] + [0x1F00 + j for j in range(32)] +
                      [0xFF00 + j for j in range(32)] + [0xFFFF, 0x8000, 0x0100], dtype=np.uint16)
    for n in (1000, 3 * (1 << 20) + 5, (20 << 20) + 3):
        valid = rng.integers(0, k, size=n).astype(np.uint16)
        ids = np.where(rng.random(n) < 0.5, valid, decoys[rng.integers(0, decoys.size, size=n)]).astype(np.uint16)
        got = _run(ids, k, 2 * int(rng.integers(0, 8)))
        assert np.array_equal(got, oracle.onehot_counts(ids, k)), n
        assert int(got.sum()) == int(np.sum(ids < k))


@pytest.mark.parametrize("k", [1, 8, 9, 16, 17, 32])
def test_u32_ids_decoys(k):
    """32-bit ids are encoded by a clamped shift: ids of 32 and more (low
    bits a valid category, high bits set, 2^31, 0xFFFFFFFF) must count
    nowhere, mixed with valid ids, on both kernels (register loads for the
    small input, the bulk-copy ring for the two large ones)."""
    rng = np.random.default_rng(11 + k)
    decoys = np.array([32 + j for j in range(32)] + [0x100 + j for j in range(32)] + [0x10000 + j for j in range(32)] +
                      [0xFFFFFFE0 + j for j in range(32)] + [1 << 31, 0xFFFFFFFF], dtype=np.uint32)
    for n in (1000, (3 << 20) + 5, (10 << 20) + 3):
        valid = rng.integers(0, k, size=n).astype(np.uint32)
        ids = np.where(rng.random(n) < 0.5, valid, decoys[rng.integers(0, decoys.size, size=n)]).astype(np.uint32)
        got = _run(ids, k, 4 * int(rng.integers(0, 4)))
        assert np.array_equal(got, oracle.onehot_counts(ids, k)), n
        assert int(got.sum()) == int(np.sum(ids < k))


def test_rejects():
    x = torch.zeros(16, dtype=torch.uint8, device="cuda")
    for k in (0, 33):
        with pytest.raises(ppc.PospopcntError):
            ppc.pospopcnt_onehot_counts(x, k)


@pytest.mark.slow
def test_full_u8_ids_zipf16():
    ids = synth.categorical_ids(0, 1 << 31, synth.zipf_cdf(16), np.uint8)
    got = _run(ids, 16)
    assert int(got.sum()) == 1 << 31
    assert np.array_equal(got, oracle.onehot_counts(ids, 16))


def test_overwrite_on_streams_mixed_with_plain_counts():
    """One-hot counts overwrite their outputs through the stream's
    accumulator, which plain counts on the same stream share: six streams
    each alternate one-hot counts (every id width, both 8-bit-id kernels) and
    plain u16 counts of other inputs, 3 rounds, outputs pre-filled with
    garbage; every result equals the oracle."""
    rng = np.random.default_rng(55)
    streams = [torch.cuda.Stream() for _ in range(6)]
    jobs = []
    for i, s in enumerate(streams):
        idb = (1, 2, 4, 1, 1, 2)[i]
        k = (32, 17, 16, 9, 32, 5)[i]
        # ids per stream: both kernels of 8- and 16-bit ids, the ring of 32-bit ids
        n = ((2 << 20) + 5, (3 << 20) + 7, (5 << 20) + 1, (3 << 20) + 11, (24 << 20) + 3, (12 << 20) + 9)[i]
        ids = synth.categorical_ids(200 + i, n, synth.zipf_cdf(min(2 * k, 64)), DT[idb])
        words = synth.uniform_bits(300 + i, int(rng.integers(1 << 20, 6 << 20)), 16)
        wx = torch.from_numpy(words.view(np.uint8)).cuda()
        jobs.append((s, k, _dev(ids, 0), oracle.onehot_counts(ids, k), wx, oracle.pospopcnt(words, 16)))
    torch.cuda.synchronize()
    for _ in range(3):
        outs = []
        for s, k, x, ref, wx, wref in jobs:
            a = torch.randint(-2 ** 62, 2 ** 62, (k,), dtype=torch.int64, device="cuda")
            b = torch.randint(-2 ** 62, 2 ** 62, (16,), dtype=torch.int64, device="cuda")
            s.wait_stream(torch.cuda.current_stream())
            ppc.pospopcnt_onehot_counts(x, k, counts=a, stream=s)
            ppc.pospopcnt_u16(wx, counts=b, stream=s)
            ppc.pospopcnt_onehot_counts(x, k, counts=a, stream=s)
            outs.append((a, b))
        torch.cuda.synchronize()
        for (s, k, x, ref, wx, wref), (a, b) in zip(jobs, outs):
            assert np.array_equal(a.cpu().numpy().view(np.uint64), ref), k
            assert np.array_equal(b.cpu().numpy().view(np.uint64), wref)


def _oracle_threads(ids, k, parts=16):
    """The oracle over contiguous parts on host threads, results added (the
    histogram of a concatenation is the sum of the parts' histograms)."""
    from concurrent.futures import ThreadPoolExecutor
    chunks = np.array_split(ids, parts)
    with ThreadPoolExecutor(parts) as ex:
        return np.sum(np.stack(list(ex.map(lambda c: oracle.onehot_counts(c, k), chunks))), axis=0,
                      dtype=np.uint64)


@pytest.mark.slow
def test_four_gib_u8_ids():
    """2^32 8-bit ids (4 GiB): all zero, so category 0 counts exactly 2^32
    (past any 32-bit partial), and Zipf(1.1) over 32 categories against the
    oracle; one-hot words of 17..32 categories go through the ALU-bound
    bulk-copy kernel."""
    zeros = np.zeros(1 << 32, dtype=np.uint8)
    got = _run(zeros, 32)
    assert got[0] == 1 << 32 and not got[1:].any()
    del zeros
    torch.cuda.empty_cache()
    ids = synth.categorical_ids(7, 1 << 32, synth.zipf_cdf(32), np.uint8)
    got = _run(ids, 32)
    assert int(got.sum()) == 1 << 32
    assert np.array_equal(got, _oracle_threads(ids, 32))


@pytest.mark.slow
def test_full_u16_and_u32_ids():
    """The bench's 16- and 32-bit-id workloads at full size (2 GiB: 2^30 u16
    ids, 2^29 u32 ids), Zipf(1.1) over 16 and over 32 categories, against
    the oracle."""
    for idb, n in ((2, 1 << 30), (4, 1 << 29)):
        for k in (16, 32):
            ids = synth.categorical_ids(60 + k, n, synth.zipf_cdf(k), DT[idb])
            got = _run(ids, k)
            assert int(got.sum()) == n
            assert np.array_equal(got, _oracle_threads(ids, k)), (idb, k)
            del ids
            torch.cuda.empty_cache()


def test_graph_capture_of_onehot_and_popcount():
    """One-hot and popcount calls captured into CUDA graphs (they zero their
    outputs with a memset while the stream is captured, so a graph may be
    replayed on any stream): replays on two other streams, outputs reset to
    garbage in between, equal the oracle."""
    ids = synth.categorical_ids(70, (9 << 20) + 1, synth.zipf_cdf(32), np.uint8)
    x = _dev(ids, 1)
    b = synth.uniform_bytes(71, (40 << 20) + 3)
    xb = torch.from_numpy(b).cuda()
    h = torch.empty(32, dtype=torch.int64, device="cuda")
    pc = torch.empty(1, dtype=torch.int64, device="cuda")
    ppc.pospopcnt_onehot_counts(x, 32, counts=h)
    ppc.pospopcnt_popcount(xb, count=pc)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ppc.pospopcnt_onehot_counts(x, 32, counts=h)
        ppc.pospopcnt_popcount(xb, count=pc)
    ref_h = oracle.onehot_counts(ids, 32)
    ref_pc = int(oracle.pospopcnt(b, 8).sum())
    for s in (torch.cuda.Stream(), torch.cuda.Stream()):
        h.fill_(-3)
        pc.fill_(-3)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            g.replay()
        s.synchronize()
        assert np.array_equal(h.cpu().numpy().view(np.uint64), ref_h)
        assert int(pc.cpu()[0]) == ref_pc
