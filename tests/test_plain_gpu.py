"""Parity of the single-stream CUDA path with the CPU oracle: bit-exact
(tolerance 0) for every kernel family and width, for every start alignment,
for every small length, across tiles and ragged tails, at the full 2 GiB
workloads, and on the edge cases (empty, all-ones, all-zeros, one-hot,
sparse).  Guard bytes of 0xFF surround every input slice, so a kernel that
read and counted a byte outside its input would fail parity; guard words
after the counts catch stray writes."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_1911_02696_gb300 as ppc  # noqa: E402

pytestmark = pytest.mark.gpu

WIDTHS = (8, 16, 32)
KERNELS = ("csa", "tma", "ballot")
DT = {8: np.uint8, 16: np.uint16, 32: np.uint32}
GUARD = 256
SENTINEL = -7


def _device_slice(words: np.ndarray, offset: int):
    """A device copy of `words` starting `offset` bytes past a 256-byte
    boundary, with 0xFF guard bytes on both sides."""
    b = np.ascontiguousarray(words).view(np.uint8)
    buf = torch.full((GUARD + offset + b.size + GUARD,), 0xFF, dtype=torch.uint8, device="cuda")
    if b.size:
        buf[GUARD + offset: GUARD + offset + b.size].copy_(torch.from_numpy(b))
    return buf, buf[GUARD + offset: GUARD + offset + b.size]


def _counts_with_guard(width):
    c = torch.full((width + 8,), SENTINEL, dtype=torch.int64, device="cuda")
    return c, c[:width]


def _as_u64(t):
    return t.cpu().numpy().view(np.uint64)


def run_kernel(width, kernel, x, out, cfg=None):
    if cfg is not None:
        return ppc.pospopcnt_count_config(width, cfg, x, counts=out)
    if kernel is None:
        return {8: ppc.pospopcnt_u8, 16: ppc.pospopcnt_u16, 32: ppc.pospopcnt_u32, 64: ppc.pospopcnt_u64}[width](x, counts=out)
    return ppc.pospopcnt_count(width, x, kernel, counts=out)


def check(width, kernel, words, offset=0, cfg=None):
    _, x = _device_slice(words, offset)
    full, out = _counts_with_guard(width)
    run_kernel(width, kernel, x, out, cfg)
    torch.cuda.synchronize()
    got = _as_u64(out)
    ref = oracle.pospopcnt(words, width)
    assert np.array_equal(got, ref), (width, kernel, words.size, offset, got, ref)
    assert torch.all(full[width:] == SENTINEL)


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("kernel", KERNELS)
def test_every_small_length_and_alignment(width, kernel):
    """n = 0..299 words at every word-aligned start offset 0..15 bytes."""
    wb = width // 8
    words = synth.uniform_bits(1000 + width, 300, width)
    for offset in range(0, 16, wb):
        _, x_all = _device_slice(words, offset)
        full = torch.full((300, width + 8), SENTINEL, dtype=torch.int64, device="cuda")
        for n in range(300):
            run_kernel(width, kernel, x_all[: n * wb], full[n, :width])
        torch.cuda.synchronize()
        got = full.cpu().numpy()
        for n in range(300):
            ref = oracle.pospopcnt(words[:n], width)
            assert np.array_equal(got[n, :width].view(np.uint64), ref), (offset, n)
            assert np.all(got[n, width:] == SENTINEL)


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("kernel", KERNELS)
def test_ragged_multi_tile(width, kernel):
    """Sizes that span many CTAs and leave partial trips, ragged tails and
    partial TMA chunks."""
    rng = np.random.default_rng(width * 7 + len(kernel))
    for i in range(6):
        nbytes = int(rng.integers(1 << 16, 48 << 20))
        n = nbytes // (width // 8)
        offset = int(rng.integers(0, 16 // (width // 8))) * (width // 8)
        check(width, kernel, synth.uniform_bits(2000 + i, n, width), offset)


@pytest.mark.parametrize("width", WIDTHS)
def test_special_inputs(width):
    n = (1 << 22) + 5
    dt = DT[width]
    for kernel in KERNELS:
        check(width, kernel, np.full(n, (1 << width) - 1, dtype=dt), 0)
        check(width, kernel, np.zeros(n, dtype=dt), width // 8)
        check(width, kernel, synth.one_hot(3, n, width), 0)
        check(width, kernel, synth.sparse(4, n, width), 0)
        check(width, kernel, np.zeros(0, dtype=dt), 0)


@pytest.mark.parametrize("width", WIDTHS)
def test_every_config(width):
    """Every configuration the autotuner may pick gives the same counts."""
    words = synth.uniform_bits(77, (9 << 20) // (width // 8) + 3, width)
    cfgs = [dict(kernel="csa", threads=t, unroll=u) for t in (128, 256, 512) for u in (2, 4, 8)]
    cfgs += [dict(kernel="tma", stages=s, chunk_bytes=c, flags=f) for s in (2, 3, 4, 6, 8)
             for c in (16384, 32768, 49152, 65536, 98304) for f in (0, 1) if s * c <= 196608]
    cfgs += [dict(kernel="ballot", unroll=u) for u in (1, 2, 4)]
    cfgs += [dict(kernel="csa", blocks_per_sm=1), dict(kernel="tma", blocks_per_sm=1, stages=2)]
    for cfg in cfgs:
        check(width, None, words, 2 * (width // 8) % 16, cfg)


def test_accumulate_form():
    words = synth.uniform_bits(5, 1 << 20, 16)
    _, x = _device_slice(words, 0)
    c = torch.zeros(16, dtype=torch.int64, device="cuda")
    ppc.pospopcnt_count_accumulate(16, x, c)
    ppc.pospopcnt_count_accumulate(16, x[: (1 << 19) * 2], c)
    torch.cuda.synchronize()
    ref = oracle.pospopcnt(words) + oracle.pospopcnt(words[: 1 << 19])
    assert np.array_equal(_as_u64(c), ref)


@pytest.mark.parametrize("width", WIDTHS)
def test_host_buffer_path(width):
    """pospopcnt_count_host: chunked copies through the staging buffers."""
    for nbytes in (0, 2, 4096 + 4, (64 << 20) - 4, (64 << 20) + 12, (200 << 20) + 4):
        n = nbytes // (width // 8)
        words = synth.uniform_bits(600 + nbytes % 97, n, width)
        got = ppc.pospopcnt_count_host(width, words)
        assert np.array_equal(got, oracle.pospopcnt(words, width)), nbytes
    pinned = torch.from_numpy(synth.uniform_bits(9, 3 << 20, width).view(np.uint8)).pin_memory()
    got = ppc.pospopcnt_count_host(width, pinned)
    assert np.array_equal(got, oracle.pospopcnt(pinned.numpy(), width))


def test_autotune_installs_a_valid_config():
    words = synth.uniform_bits(8, 32 << 20, 16)
    _, x = _device_slice(words, 0)
    best, ms = ppc.pospopcnt_autotune(16, x)
    assert ms > 0 and best["kernel"] in (1, 2)
    assert ppc.pospopcnt_get_config(16, words.size)["kernel"] == best["kernel"]
    check(16, None, words)


def test_bounded_wait_reports_timeout():
    """A wait that can never be satisfied gives up and the host reads
    ERR_TIMEOUT; the context stays usable afterwards."""
    assert ppc.pospopcnt_check_device_error() == 0
    ppc.pospopcnt_selftest_timeout(2_000_000)  # 2 ms
    assert ppc.pospopcnt_check_device_error() == 5
    assert ppc.pospopcnt_check_device_error() == 0
    check(16, "tma", synth.uniform_bits(1, 1 << 16, 16))


def test_launch_counter_counts_kernels():
    x = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    before = ppc.pospopcnt_launch_count()
    for _ in range(5):
        ppc.pospopcnt_u16(x)
    assert ppc.pospopcnt_launch_count() - before == 5


def test_stream_ordering_on_side_stream():
    words = synth.uniform_bits(10, 1 << 22, 32)
    _, x = _device_slice(words, 0)
    s = torch.cuda.Stream()
    out = torch.empty(32, dtype=torch.int64, device="cuda")
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        ppc.pospopcnt_u32(x, counts=out, stream=s)
    s.synchronize()
    assert np.array_equal(_as_u64(out), oracle.pospopcnt(words, 32))


def test_graph_capture_of_plain_call():
    words = synth.uniform_bits(11, 1 << 21, 16)
    _, x = _device_slice(words, 2)
    out = torch.empty(16, dtype=torch.int64, device="cuda")
    ppc.pospopcnt_init(torch.cuda.current_device())
    ppc.pospopcnt_u16(x, counts=out)  # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ppc.pospopcnt_u16(x, counts=out)
    out.fill_(0)
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(_as_u64(out), oracle.pospopcnt(words, 16))


# ---------------------------------------------------------------------------
# full-size workloads (2 GiB each), in the launch configuration the
# benchmark times

def _full(width, words, offset=0, kernels=("auto", "csa", "tma")):
    _, x = _device_slice(words, offset)
    ref, _ = oracle.pospopcnt_mt(words, width)
    for k in kernels:
        out = torch.empty(width, dtype=torch.int64, device="cuda")
        if k == "auto":
            run_kernel(width, None, x, out)
        else:
            run_kernel(width, k, x, out)
        torch.cuda.synchronize()
        assert np.array_equal(_as_u64(out), ref), k
    del x
    torch.cuda.empty_cache()
    return ref


@pytest.mark.slow
def test_full_u16_uniform():
    _full(16, synth.uniform_bits(0, 1 << 30, 16))


@pytest.mark.slow
def test_full_u16_one_hot_zipf():
    w, pos = synth.one_hot(0, 1 << 30, 16, return_positions=True)
    ref = _full(16, w)
    assert int(ref.sum()) == 1 << 30
    assert np.array_equal(ref, np.bincount(pos, minlength=16).astype(np.uint64))


@pytest.mark.slow
def test_full_u16_sparse():
    _full(16, synth.sparse(0, 1 << 30, 16))


@pytest.mark.slow
def test_full_u16_misaligned_ragged():
    """n = 2^30 + 7 words starting 2 bytes past a 256-byte boundary."""
    _full(16, synth.uniform_bits(1, (1 << 30) + 7, 16), offset=2)


@pytest.mark.slow
def test_full_u8_u32():
    for width, n in ((8, 1 << 31), (32, 1 << 29)):
        ref = _full(width, synth.one_hot(0, n, width, cdf=synth.uniform_cdf(width)), kernels=("auto",))
        assert int(ref.sum()) == n
        _full(width, synth.uniform_bits(0, n, width), kernels=("auto",))


@pytest.mark.parametrize("width", WIDTHS)
def test_overwrite_across_grid_sizes(width):
    """Counts are overwritten whether the grid is one CTA (direct store, no
    memset) or many (memset + atomics): sizes around the one-CTA limits of
    every default configuration, counts pre-filled with garbage."""
    wb = width // 8
    for nbytes in (wb, 1008, 4096, 16384, 65536 - 16, 65536, 65536 + 16, 131072 + 2 * wb, 262144 + 4 * wb,
                   (4 << 20) + 8, (16 << 20) + 4 * wb, (64 << 20) + 16):
        n = nbytes // wb
        words = synth.uniform_bits(nbytes, n, width)
        _, x = _device_slice(words, 0)
        out = torch.randint(-2 ** 62, 2 ** 62, (width,), dtype=torch.int64, device="cuda")
        run_kernel(width, None, x, out)
        torch.cuda.synchronize()
        assert np.array_equal(_as_u64(out), oracle.pospopcnt(words, width)), nbytes


def test_u64_every_small_length_and_alignment():
    """64-bit words: n = 0..299 at both 8-byte alignments within 16 bytes."""
    words = synth.uniform_bits(64, 300, 64)
    for offset in (0, 8):
        _, x_all = _device_slice(words, offset)
        full = torch.full((300, 72), SENTINEL, dtype=torch.int64, device="cuda")
        for n in range(300):
            ppc.pospopcnt_u64(x_all[: n * 8], counts=full[n, :64])
        torch.cuda.synchronize()
        got = full.cpu().numpy()
        for n in range(300):
            assert np.array_equal(got[n, :64].view(np.uint64), oracle.pospopcnt(words[:n], 64)), (offset, n)
            assert np.all(got[n, 64:] == SENTINEL)


def test_u64_configs_and_sizes():
    rng = np.random.default_rng(640)
    for cfg in (None, dict(kernel="csa", threads=128, unroll=4), dict(kernel="csa", threads=256, unroll=8),
                dict(kernel="tma", stages=3, chunk_bytes=65536), dict(kernel="tma", stages=4, chunk_bytes=16384)):
        for _ in range(3):
            n = int(rng.integers(1, 6 << 20))
            words = synth.uniform_bits(int(rng.integers(1 << 30)), n, 64)
            _, x = _device_slice(words, 8 * int(rng.integers(0, 2)))
            out = torch.full((64,), -3, dtype=torch.int64, device="cuda")
            if cfg is None:
                ppc.pospopcnt_u64(x, counts=out)
            else:
                ppc.pospopcnt_count_config(64, cfg, x, counts=out)
            torch.cuda.synchronize()
            assert np.array_equal(_as_u64(out), oracle.pospopcnt(words, 64))
    with pytest.raises(ppc.PospopcntError):
        ppc.pospopcnt_count(64, torch.zeros(64, dtype=torch.uint8, device="cuda"), "ballot")


@pytest.mark.slow
def test_full_u64():
    """2^28 64-bit words (2 GiB): uniform bits and one-hot over 64 positions."""
    _full(64, synth.uniform_bits(2, 1 << 28, 64), kernels=("auto", "csa", "tma"))
    ref = _full(64, synth.one_hot(2, 1 << 28, 64, cdf=synth.uniform_cdf(64)), kernels=("auto",))
    assert int(ref.sum()) == 1 << 28


def test_popcount_small_lengths_every_offset():
    """Array popcount (K = 1): n = 0..299 bytes at every start offset 0..15."""
    b = synth.uniform_bytes(1, 300)
    for offset in range(16):
        _, x_all = _device_slice(b, offset)
        out = torch.full((300, 2), SENTINEL, dtype=torch.int64, device="cuda")
        for n in range(300):
            ppc.pospopcnt_popcount(x_all[:n], count=out[n, :1])
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for n in range(300):
            assert int(got[n, 0]) == oracle.popcount(b[:n]), (offset, n)
            assert got[n, 1] == SENTINEL


def test_popcount_sizes_and_patterns():
    rng = np.random.default_rng(11)
    for _ in range(6):
        n = int(rng.integers(1, 80 << 20))
        b = synth.uniform_bytes(int(rng.integers(1 << 30)), n)
        _, x = _device_slice(b, int(rng.integers(0, 16)))
        got = int(ppc.pospopcnt_popcount(x).cpu()[0])
        assert got == oracle.popcount(b)
    ones = np.full((5 << 20) + 3, 0xFF, dtype=np.uint8)
    _, x = _device_slice(ones, 5)
    assert int(ppc.pospopcnt_popcount(x).cpu()[0]) == 8 * ones.size


@pytest.mark.slow
def test_popcount_full():
    b = synth.uniform_bytes(5, 1 << 31)
    _, x = _device_slice(b, 0)
    got = int(ppc.pospopcnt_popcount(x).cpu()[0])
    ref, _ = oracle.pospopcnt_mt(b, 8)
    assert got == int(ref.sum())


# ---------------------------------------------------------------------------
# 4 GiB, the top of the input-size sweep: counts reach 2^31 per position
# (u16) and 2^35 in total (popcount), past any 32-bit partial sum

FOUR_GIB_CONFIGS = (None, dict(kernel="csa"), dict(kernel="tma"), dict(kernel="csa", blocks_per_sm=1),
                    dict(kernel="tma", blocks_per_sm=1, stages=4, chunk_bytes=49152))


def _four_gib_u16(words, ref):
    _, x = _device_slice(words, 0)
    for cfg in FOUR_GIB_CONFIGS:
        out = torch.full((16,), SENTINEL, dtype=torch.int64, device="cuda")
        run_kernel(16, None, x, out, cfg)
        torch.cuda.synchronize()
        assert np.array_equal(_as_u64(out), ref), cfg
    del x
    torch.cuda.empty_cache()


@pytest.mark.slow
def test_four_gib_u16_uniform():
    """2^31 u16 words of uniform bits against the oracle."""
    words = synth.uniform_bits(4, 1 << 31, 16)
    ref, _ = oracle.pospopcnt_mt(words, 16)
    assert int(ref.sum()) > 1 << 33
    _four_gib_u16(words, ref)


@pytest.mark.slow
def test_four_gib_u16_all_ones():
    """2^31 all-ones u16 words: every position counts 2^31 (closed form, and
    the oracle on the same words)."""
    words = np.full(1 << 31, 0xFFFF, dtype=np.uint16)
    ref, _ = oracle.pospopcnt_mt(words, 16)
    assert np.array_equal(ref, np.full(16, 1 << 31, dtype=np.uint64))
    _four_gib_u16(words, ref)


@pytest.mark.slow
def test_four_gib_popcount():
    """Array popcount of 4 GiB of 0xFF (2^35 set bits) and of 4 GiB of
    uniform random bytes (the oracle's u8 positional counts summed)."""
    ones = np.full(1 << 32, 0xFF, dtype=np.uint8)
    _, x = _device_slice(ones, 0)
    assert int(ppc.pospopcnt_popcount(x).cpu()[0]) == 1 << 35
    del x, ones
    torch.cuda.empty_cache()
    b = synth.uniform_bytes(6, 1 << 32)
    _, x = _device_slice(b, 3)
    got = int(ppc.pospopcnt_popcount(x).cpu()[0])
    ref, _ = oracle.pospopcnt_mt(b, 8)
    assert got == int(ref.sum())
    del x
    torch.cuda.empty_cache()


# ---------------------------------------------------------------------------
# overwrite without a memset: multi-CTA counts add into an accumulator bound
# to the caller's stream and the last block writes the counts

def test_overwrite_on_many_streams_back_to_back():
    """Eight streams, each counting its own inputs of every width (u8 / u16 /
    u32 / u64 and the popcount) back to back, 3 rounds, counts pre-filled with
    garbage: every result equals the oracle, so no stream's accumulator leaks
    into another call."""
    rng = np.random.default_rng(77)
    streams = [torch.cuda.Stream() for _ in range(8)]
    jobs = []
    for i, s in enumerate(streams):
        for width in (8, 16, 32, 64, 1):
            nbytes = int(rng.integers(1 << 20, 24 << 20)) // 8 * 8
            wb = 1 if width == 1 else width // 8
            words = synth.uniform_bits(i * 10 + width, nbytes // wb, 8 if width == 1 else width)
            _, x = _device_slice(words, 0)
            ref = (np.array([oracle.pospopcnt(words, 8).sum()], dtype=np.uint64) if width == 1
                   else oracle.pospopcnt(words, width))
            jobs.append((s, width, ref, x))
    torch.cuda.synchronize()
    for _ in range(3):
        outs = []
        for s, width, ref, x in jobs:
            out = torch.randint(-2 ** 62, 2 ** 62, (max(width, 1),), dtype=torch.int64, device="cuda")
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                if width == 1:
                    ppc.pospopcnt_popcount(x, count=out, stream=s)
                else:
                    run_kernel(width, None, x, out)
            outs.append(out)
        torch.cuda.synchronize()
        for (s, width, ref, x), out in zip(jobs, outs):
            assert np.array_equal(_as_u64(out), ref), width


def test_overwrite_after_stream_release():
    """A stream's accumulator returns to the free list with the stream and
    serves the next stream correctly."""
    words = synth.uniform_bits(31, 5 << 20, 16)
    _, x = _device_slice(words, 2)
    ref = oracle.pospopcnt(words, 16)
    for _ in range(20):
        s = torch.cuda.Stream()
        out = torch.full((16,), -1, dtype=torch.int64, device="cuda")
        with torch.cuda.stream(s):
            ppc.pospopcnt_u16(x, counts=out, stream=s)
            ppc.pospopcnt_u16(x, counts=out, stream=s)
        s.synchronize()
        assert np.array_equal(_as_u64(out), ref)
        ppc.pospopcnt_release_stream(s)


def test_graph_replays_on_two_streams():
    """A captured plain count uses the memset path, so two replays of two
    graphs capturing the same call may overlap on different streams."""
    a = synth.uniform_bits(41, 7 << 20, 32)
    b = synth.uniform_bits(42, 9 << 20, 32)
    _, xa = _device_slice(a, 4)
    _, xb = _device_slice(b, 8)
    oa = torch.empty(32, dtype=torch.int64, device="cuda")
    ob = torch.empty(32, dtype=torch.int64, device="cuda")
    ppc.pospopcnt_u32(xa, counts=oa)
    torch.cuda.synchronize()
    ga, gb = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(ga):
        ppc.pospopcnt_u32(xa, counts=oa)
    with torch.cuda.graph(gb):
        ppc.pospopcnt_u32(xb, counts=ob)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    for _ in range(10):
        oa.fill_(-5)
        ob.fill_(-5)
        s1.wait_stream(torch.cuda.current_stream())
        s2.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s1):
            ga.replay()
        with torch.cuda.stream(s2):
            gb.replay()
        torch.cuda.synchronize()
        assert np.array_equal(_as_u64(oa), oracle.pospopcnt(a, 32))
        assert np.array_equal(_as_u64(ob), oracle.pospopcnt(b, 32))


def test_per_thread_default_stream_from_several_threads():
    """cudaStreamPerThread is one handle for a different stream in every
    host thread, so counts on it must not share a stream accumulator: four
    threads count different inputs on it at once, each repeatedly, and every
    result equals the oracle."""
    import ctypes
    import threading
    lib = ppc.load()
    per_thread = ctypes.c_void_p(2)  # cudaStreamPerThread
    inputs = []
    for i in range(4):
        words = synth.uniform_bits(90 + i, (6 << 20) + 131 * i, 16)
        _, x = _device_slice(words, 2 * i)
        inputs.append((x, oracle.pospopcnt(words, 16)))
    outs = [torch.full((16,), -1, dtype=torch.int64, device="cuda") for _ in inputs]
    torch.cuda.synchronize()
    errors = []

    def work(i):
        try:
            torch.cuda.set_device(0)
            x, ref = inputs[i]
            for _ in range(25):
                rc = lib.pospopcnt_u16(ctypes.c_void_p(x.data_ptr()), x.numel() // 2,
                                       ctypes.c_void_p(outs[i].data_ptr()), per_thread)
                assert rc == 0, ppc.pospopcnt_strerror(rc)
        except Exception as exc:  # reported on the main thread
            errors.append(exc)

    threads = [threading.Thread(target=work, args=(i,)) for i in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    torch.cuda.synchronize()
    assert not errors, errors
    for (x, ref), out in zip(inputs, outs):
        assert np.array_equal(_as_u64(out), ref)
