"""Parity of the segmented (batched) CUDA path with the oracle, bit-exact:
empty and length-1 segments, segments straddling tiles, a non-zero first
offset, unaligned bases, every width; row sums against a plain call over
the span; repeated launches, concurrent streams and CUDA-graph replays (the
work queue resets itself); and the full 20,000-segment workload."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_1911_02696_gb300 as ppc  # noqa: E402

pytestmark = pytest.mark.gpu

WIDTHS = (8, 16, 32)


def _dev(words: np.ndarray, offset: int = 0):
    b = np.ascontiguousarray(words).view(np.uint8)
    buf = torch.full((256 + offset + b.size + 256,), 0xFF, dtype=torch.uint8, device="cuda")
    if b.size:
        buf[256 + offset: 256 + offset + b.size].copy_(torch.from_numpy(b))
    return buf, buf[256 + offset: 256 + offset + b.size]


def _layout(rng, nseg, max_len, start=0, p_empty=0.1):
    lens = rng.integers(1, max_len + 1, size=nseg)
    lens[rng.random(nseg) < p_empty] = 0
    return synth.offsets_from_lengths(lens.astype(np.int64), start)


def _check(width, words, off, offset=0, stream=None):
    _, x = _dev(words, offset)
    d_off = torch.from_numpy(off).cuda()
    out = ppc.pospopcnt_batched(x, d_off, width, stream=stream)
    torch.cuda.synchronize()
    ref = oracle.pospopcnt_segments(words, off, width)
    got = out.cpu().numpy().view(np.uint64)
    assert got.shape == ref.shape
    bad = np.nonzero(np.any(got != ref, axis=1))[0]
    assert bad.size == 0, (width, offset, bad[:10])
    return got


@pytest.mark.parametrize("width", WIDTHS)
def test_small_layouts(width):
    rng = np.random.default_rng(width)
    wb = width // 8
    for trial in range(12):
        nseg = int(rng.integers(1, 300))
        off = _layout(rng, nseg, int(rng.choice([1, 7, 100, 5000, 200000])), start=int(rng.integers(0, 50)))
        words = synth.uniform_bits(trial, int(off[-1]) + int(rng.integers(0, 9)), width)
        _check(width, words, off, offset=int(rng.integers(0, 16 // wb)) * wb)


@pytest.mark.parametrize("width", WIDTHS)
def test_edge_layouts(width):
    w = synth.uniform_bits(3, 400000, width)
    cases = [
        [0, 0],                       # one empty segment
        [0, 1],                       # one word
        [5, 5, 5, 5],                 # all empty, non-zero start
        [0, 400000],                  # one long segment over many tiles
        [399999, 400000],             # last word only
        list(range(0, 300)),          # 299 segments of one word
        [0, 70000, 70000, 140001, 400000],
        [3, 65539, 131075, 196611],   # segments crossing tile boundaries
    ]
    for c in cases:
        _check(width, w, np.array(c, dtype=np.int64))


def test_row_sum_equals_plain_call():
    rng = np.random.default_rng(4)
    off = _layout(rng, 1000, 3000, start=17)
    words = synth.uniform_bits(4, int(off[-1]), 16)
    got = _check(16, words, off, offset=6)
    _, x = _dev(words, 6)
    plain = ppc.pospopcnt_u16(x[2 * 17: 2 * int(off[-1])])
    torch.cuda.synchronize()
    assert np.array_equal(got.sum(axis=0, dtype=np.uint64), plain.cpu().numpy().view(np.uint64))


def test_repeated_launches_and_two_streams():
    rng = np.random.default_rng(5)
    off = _layout(rng, 500, 100000)
    words = synth.uniform_bits(5, int(off[-1]), 16)
    _, x = _dev(words)
    d_off = torch.from_numpy(off).cuda()
    ref = oracle.pospopcnt_segments(words, off, 16)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    for i in range(4):
        s = (s1, s2)[i % 2]
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            outs.append(ppc.pospopcnt_batched(x, d_off, 16, stream=s))
    torch.cuda.synchronize()
    for o in outs:
        assert np.array_equal(o.cpu().numpy().view(np.uint64), ref)


def test_graph_replays():
    rng = np.random.default_rng(6)
    off = _layout(rng, 2000, 20000, start=3)
    words = synth.one_hot(6, int(off[-1]) + 1, 16)
    _, x = _dev(words, 2)
    d_off = torch.from_numpy(off).cuda()
    out = torch.empty((2000, 16), dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        ppc.pospopcnt_batched(x, d_off, 16, counts=out, stream=s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ppc.pospopcnt_batched(x, d_off, 16, counts=out, stream=s)
    ref = oracle.pospopcnt_segments(words, off, 16)
    for _ in range(3):
        out.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint64), ref)


@pytest.mark.slow
def test_full_20k_segments_one_hot():
    """20,000 segments, lengths log-uniform in [1, 2^20] words, one-hot with
    a per-segment rotated Zipf(1.1) position, int64 offsets."""
    lens = synth.log_uniform_lengths(0, 20000)
    off = synth.offsets_from_lengths(lens)
    words = synth.segmented_one_hot(0, off, 16)
    got = _check(16, words, off)
    assert np.array_equal(got.sum(axis=1), lens.astype(np.uint64))


@pytest.mark.slow
def test_four_gib_segment_among_small_ones():
    """One segment of 2^31 all-ones u16 words (4 GiB: every count 2^31, a
    closed form) between small segments of uniform bits (the oracle), through
    the batched form and its allocation-free variant."""
    big = 1 << 31
    small = synth.uniform_bits(12, 3000, 16)
    words = np.empty(big + small.size, dtype=np.uint16)
    words[:1000] = small[:1000]
    words[1000: 1000 + big] = 0xFFFF
    words[1000 + big:] = small[1000:]
    off = np.array([0, 1, 1000, 1000 + big, 1000 + big + 7, words.size], dtype=np.int64)
    _, x = _dev(words, 2)
    d_off = torch.from_numpy(off).cuda()
    ref = np.zeros((off.size - 1, 16), dtype=np.uint64)
    for sgm in (0, 1, 3, 4):
        ref[sgm] = oracle.pospopcnt(words[off[sgm]: off[sgm + 1]], 16)
    ref[2] = big
    got = ppc.pospopcnt_batched(x, d_off, 16).cpu().numpy().view(np.uint64)
    assert np.array_equal(got, ref)
    rows = torch.full((off.size - 1, 16), -1, dtype=torch.int64, device="cuda")
    ppc.pospopcnt_batched_noalloc(x, d_off, 16, rows)
    torch.cuda.synchronize()
    assert np.array_equal(rows.cpu().numpy().view(np.uint64), ref)
    del x
    torch.cuda.empty_cache()


def test_checked_form_valid_and_invalid_offsets():
    """pospopcnt_batched_checked counts valid offsets like pospopcnt_batched
    and turns offsets beyond the buffer or decreasing into an error status
    (nothing counted, no access outside the input); the next call on the
    same stream works again."""
    rng = np.random.default_rng(8)
    off = _layout(rng, 300, 5000, start=2)
    words = synth.uniform_bits(8, int(off[-1]), 16)
    _, x = _dev(words, 4)
    d_off = torch.from_numpy(off).cuda()
    assert ppc.pospopcnt_check_device_error() == 0
    got = ppc.pospopcnt_batched_checked(x, d_off, 16)
    assert ppc.pospopcnt_check_device_error() == 0
    assert np.array_equal(got.cpu().numpy().view(np.uint64), oracle.pospopcnt_segments(words, off, 16))
    beyond = off.copy()
    beyond[-1] += 1000  # past the end of x
    dec = off.copy()
    dec[5], dec[6] = dec[6] + 1, dec[5]  # not monotone
    neg = off.copy()
    neg[0] = -1
    for bad in (beyond, dec, neg):
        out = torch.full((300, 16), 7, dtype=torch.int64, device="cuda")
        ppc.pospopcnt_batched_checked(x, torch.from_numpy(bad).cuda(), 16, counts=out)
        assert ppc.pospopcnt_check_device_error() == 1
        assert torch.all(out == 0)
    # the slot is clean again: unchecked and checked calls both count
    got = ppc.pospopcnt_batched(x, d_off, 16)
    got2 = ppc.pospopcnt_batched_checked(x, d_off, 16)
    assert ppc.pospopcnt_check_device_error() == 0
    ref = oracle.pospopcnt_segments(words, off, 16)
    assert np.array_equal(got.cpu().numpy().view(np.uint64), ref)
    assert np.array_equal(got2.cpu().numpy().view(np.uint64), ref)


def test_native_graph_api():
    """pospopcnt_batched_graph_create captures once; every launch recounts
    the current contents of the same buffers."""
    rng = np.random.default_rng(9)
    off = _layout(rng, 400, 30000, start=1)
    _, x = _dev(synth.uniform_bits(0, int(off[-1]), 16), 2)
    d_off = torch.from_numpy(off).cuda()
    out = torch.empty((400, 16), dtype=torch.int64, device="cuda")
    g = ppc.pospopcnt_batched_graph_create(x, d_off, 16, out)
    try:
        for seed in (1, 2, 3):
            words = synth.uniform_bits(seed, int(off[-1]), 16)
            x.copy_(torch.from_numpy(words.view(np.uint8)))
            out.fill_(-1)
            torch.cuda.synchronize()
            ppc.pospopcnt_graph_launch(g)
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy().view(np.uint64), oracle.pospopcnt_segments(words, off, 16))
    finally:
        ppc.pospopcnt_graph_destroy(g)


def test_batched_autotune_and_config():
    """The autotuner times every unit size x CTAs-per-SM x ring depth on the caller's
    layout, refuses to install unless all agree, and installs the fastest;
    counts stay bit-exact under every configuration, and out-of-range
    configurations are rejected."""
    rng = np.random.default_rng(10)
    off = _layout(rng, 1500, 40000, start=5)
    words = synth.uniform_bits(10, int(off[-1]) + 3, 16)
    _, x = _dev(words, 2)
    d_off = torch.from_numpy(off).cuda()
    ref = oracle.pospopcnt_segments(words, off, 16)
    try:
        best, ms = ppc.pospopcnt_batched_autotune(x, d_off, 16)
        assert ms > 0 and best["unit_bytes"] in (4096, 8192, 16384, 32768, 65536)
        assert ppc.pospopcnt_batched_get_config(16) == best
        got = ppc.pospopcnt_batched(x, d_off, 16)
        assert np.array_equal(got.cpu().numpy().view(np.uint64), ref)
        for cfg in ({"unit_bytes": 4096, "blocks_per_sm": 1}, {"unit_bytes": 1 << 20, "blocks_per_sm": 32},
                    {"unit_bytes": 8192 + 128, "blocks_per_sm": 0}, {"unit_bytes": 16384, "ring_stages": 3},
                    {"unit_bytes": 65536, "blocks_per_sm": 1, "ring_stages": 4},
                    {"unit_bytes": 16384, "vectors_per_lane": 4, "ring_stages": 4},
                    {"unit_bytes": 131072, "vectors_per_lane": 16, "ring_stages": 3}):
            ppc.pospopcnt_batched_set_config(16, cfg)
            got = ppc.pospopcnt_batched(x, d_off, 16)
            assert np.array_equal(got.cpu().numpy().view(np.uint64), ref), cfg
        for bad in ({"unit_bytes": 2048}, {"unit_bytes": 4096 + 64}, {"unit_bytes": 2 << 20},
                    {"unit_bytes": 4096, "blocks_per_sm": -1}, {"unit_bytes": 4096, "blocks_per_sm": 33},
                    {"unit_bytes": 4096, "ring_stages": 1}, {"unit_bytes": 4096, "ring_stages": 5},
                    {"unit_bytes": 4096, "vectors_per_lane": 2}, {"unit_bytes": 4096, "vectors_per_lane": 32},
                    {"unit_bytes": 4096, "vectors_per_lane": 16, "ring_stages": 4}):
            with pytest.raises(ppc.PospopcntError):
                ppc.pospopcnt_batched_set_config(16, bad)
    finally:
        ppc.pospopcnt_batched_set_config(16, None)
    assert ppc.pospopcnt_batched_get_config(16) == {"unit_bytes": 32768, "blocks_per_sm": 2, "ring_stages": 2,
                                                    "vectors_per_lane": 8}


@pytest.mark.parametrize("width", (8, 16, 32))
def test_every_autotune_candidate_matches_oracle(width):
    """Every configuration the autotuner may pick -- unit size x CTAs per SM
    x ring depth x vectors per lane, 120 in all -- gives the oracle's rows
    on a layout with empty, one-word, misaligned and ring-length segments."""
    rng = np.random.default_rng(20 + width)
    lens = rng.integers(0, 60000, size=240).astype(np.int64)
    lens[::7] = 0
    lens[3::11] = 1
    lens[5::13] = 300000  # long enough for every ring shape, several trips
    off = synth.offsets_from_lengths(lens, start=3)
    words = synth.uniform_bits(30 + width, int(off[-1]) + 5, width)
    _, x = _dev(words, width // 8)
    d_off = torch.from_numpy(off).cuda()
    ref = oracle.pospopcnt_segments(words, off, width)
    n = 0
    try:
        for unit in (4096, 8192, 16384, 32768, 65536):
            for bps in (1, 2, 0):
                for stages in (2, 3, 4):
                    for vpl in (4, 8, 16):
                        if vpl == 16 and stages == 4:
                            continue
                        cfg = {"unit_bytes": unit, "blocks_per_sm": bps, "ring_stages": stages,
                               "vectors_per_lane": vpl}
                        ppc.pospopcnt_batched_set_config(width, cfg)
                        got = torch.full((off.size - 1, width), -1, dtype=torch.int64, device="cuda")
                        ppc.pospopcnt_batched(x, d_off, width, counts=got)
                        assert np.array_equal(got.cpu().numpy().view(np.uint64), ref), cfg
                        n += 1
    finally:
        ppc.pospopcnt_batched_set_config(width, None)
    assert n == 120


def test_stream_slots_are_released_and_reused():
    """Each stream that makes batched calls holds one of 256 work-queue
    slots; pospopcnt_release_stream returns it, so 300 short-lived streams
    in turn never run out, and every count stays exact."""
    rng = np.random.default_rng(11)
    off = _layout(rng, 50, 3000, start=1)
    words = synth.uniform_bits(11, int(off[-1]), 16)
    _, x = _dev(words)
    d_off = torch.from_numpy(off).cuda()
    ref = oracle.pospopcnt_segments(words, off, 16)
    for i in range(300):
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            out = ppc.pospopcnt_batched(x, d_off, 16, stream=s)
        s.synchronize()
        ppc.pospopcnt_release_stream(s)
        if i % 50 == 0:
            assert np.array_equal(out.cpu().numpy().view(np.uint64), ref), i
        del s
    ppc.pospopcnt_release_stream(torch.cuda.Stream())  # a stream without a slot: nothing to do
