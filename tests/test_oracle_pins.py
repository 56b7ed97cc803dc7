"""Pins for the CPU oracle: what the paper and the mathematics fix,
independently of the oracle's own code.

Each pin takes a counting function ``count(words: np.ndarray, width) ->
uint64[width]`` so that the same pins also run against deliberately broken
copies of the oracle (bottom of this file) and must fail there.
"""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import synth

WIDTHS = (8, 16, 32)
DT = {8: np.uint8, 16: np.uint16, 32: np.uint32, 64: np.uint64}


# --------------------------------------------------------------------------
# fixtures transcribed from the paper
# --------------------------------------------------------------------------

def _read_sections(path):
    sec, out = None, {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                head = line[1:].split("]")[0]
                rest = line.split("]", 1)[1].strip()
                sec = head
                out[sec] = {"arg": rest, "rows": []}
                continue
            out[sec]["rows"].append(line.split())
    return out


def load_table1(golden_dir):
    t = _read_sections(os.path.join(golden_dir, "table1_one_hot.txt"))
    mapping = {r[0]: int(r[1], 2) for r in t["mapping"]["rows"]}
    stream = [(int(r[0], 2), r[1]) for r in t["stream"]["rows"]]
    freq = {r[0]: int(r[1]) for r in t["frequencies"]["rows"]}
    return mapping, stream, freq


# --------------------------------------------------------------------------
# pins (each a function of a counting routine)
# --------------------------------------------------------------------------

def pin_table1(count, golden_dir):
    """§1, Table 1: the stream's histogram is France 3, Portugal 2, USA 4,
    China 1 and nothing else; ten words in total."""
    mapping, stream, freq = load_table1(golden_dir)
    # each stream entry is the mapping's code for the value it names
    for code, name in stream:
        assert mapping[name] == code
    positions = {name: code.bit_length() - 1 for name, code in mapping.items()}
    assert sorted(positions.values()) == list(range(8))  # one-hot, distinct
    words = np.array([c for c, _ in stream], dtype=np.uint8)
    c = count(words, 8)
    for name, p in positions.items():
        assert int(c[p]) == freq.get(name, 0), name
    assert int(c.sum()) == len(stream) == 10


def pin_exhaustive(count):
    """Every k-bit value once: each position is set in exactly half of them;
    r copies give r * 2^(k-1)."""
    for k in (8, 16):
        allw = np.arange(1 << k, dtype=DT[k])
        assert np.all(count(allw, k) == 1 << (k - 1))
        assert np.all(count(np.tile(allw, 3), k) == 3 << (k - 1))
    # u32: the values 0..2^m-1 (low m bits vary), then shifted into the top
    m = 12
    low = np.arange(1 << m, dtype=np.uint32)
    c = count(low, 32)
    assert np.all(c[:m] == 1 << (m - 1)) and np.all(c[m:] == 0)
    c = count(low << np.uint32(32 - m), 32)
    assert np.all(c[:32 - m] == 0) and np.all(c[32 - m:] == 1 << (m - 1))


def pin_special(count):
    """All-ones gives n everywhere, all-zeros gives zeros, one word gives its
    own bits, the empty stream gives zeros."""
    rng = np.random.default_rng(7)
    for k in WIDTHS:
        n = 1000
        ones = np.full(n, (1 << k) - 1, dtype=DT[k])
        assert np.all(count(ones, k) == n)
        assert np.all(count(np.zeros(n, dtype=DT[k]), k) == 0)
        assert np.all(count(np.zeros(0, dtype=DT[k]), k) == 0)
        for _ in range(20):
            w = int(rng.integers(0, 1 << k, dtype=np.uint64))
            c = count(np.array([w], dtype=DT[k]), k)
            assert [int(x) for x in c] == [(w >> p) & 1 for p in range(k)]


def _popcount_total(words):
    bc = getattr(np, "bitwise_count", None)
    if bc is not None:
        return int(bc(words).astype(np.uint64).sum())
    return sum(int(x).bit_count() for x in words.tolist())


def pin_popcount_total(count):
    """sum_p counts[p] equals the total popcount (pospopcnt generalises
    popcount, Abstract), via an independent popcount."""
    for k in WIDTHS:
        for seed, n in ((1, 1), (2, 777), (3, 4096)):
            w = synth.uniform_bits(seed, n, k)
            assert int(count(w, k).sum()) == _popcount_total(w)


def pin_unpackbits(count):
    """Brute force: the 'vertical' column sums of the bit matrix (§1, Fig. 1)
    taken with numpy.unpackbits on the little-endian bytes."""
    for k in WIDTHS + (64,):
        for seed, n in ((10, 1), (11, 31), (12, 1000), (13, 4096)):
            w = synth.uniform_bits(seed, n, k)
            bits = np.unpackbits(w.view(np.uint8), bitorder="little").reshape(n, k)
            ref = bits.sum(axis=0, dtype=np.uint64)
            assert np.array_equal(count(w, k), ref)


def pin_cross_width(count):
    """Wider words are narrower streams side by side (§4): over the same
    little-endian bytes c8[p] = c16[p] + c16[p+8], c16[p] = c32[p] + c32[p+16]
    and c32[p] = c64[p] + c64[p+32]."""
    b = synth.uniform_bytes(21, 4096 * 8)
    c8, c16, c32 = count(b, 8), count(b.view(np.uint16), 16), count(b.view(np.uint32), 32)
    c64 = count(b.view(np.uint64), 64)
    assert np.array_equal(c8, c16[:8] + c16[8:])
    assert np.array_equal(c16, c32[:16] + c32[16:])
    assert np.array_equal(c32, c64[:32] + c64[32:])


def pin_complement(count):
    """counts(~w)[p] = n - counts(w)[p]."""
    for k in WIDTHS:
        w = synth.uniform_bits(31, 999, k)
        assert np.array_equal(count(~w, k), np.uint64(999) - count(w, k))


def pin_additivity(count):
    """counts(A || B) = counts(A) + counts(B) at every split point (the
    streaming loop of §4.1 relies on it)."""
    for k in WIDTHS:
        w = synth.uniform_bits(41, 300, k)
        full = count(w, k)
        for cut in (0, 1, 7, 150, 299, 300):
            assert np.array_equal(full, count(w[:cut], k) + count(w[cut:], k))


def pin_one_hot(count):
    """One-hot words (§1): the counts are the histogram of the drawn
    positions and sum to n."""
    for k in WIDTHS:
        w, pos = synth.one_hot(51, 5000, k, return_positions=True)
        c = count(w, k)
        assert int(c.sum()) == 5000
        assert np.array_equal(c, np.bincount(pos, minlength=k).astype(np.uint64))


ALL_PINS = [pin_exhaustive, pin_special, pin_popcount_total, pin_unpackbits,
            pin_cross_width, pin_complement, pin_additivity, pin_one_hot]


# --------------------------------------------------------------------------
# the oracle against its pins
# --------------------------------------------------------------------------

@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pins(pin):
    pin(oracle.pospopcnt)


def test_oracle_table1(golden_dir):
    pin_table1(oracle.pospopcnt, golden_dir)


def test_oracle_rejects_bad_width():
    lib = oracle._load()
    out = np.zeros(64, dtype=np.uint64)
    for k in (0, 1, 7, 12, 24, 128):
        assert lib.oracle_pospopcnt(k, None, 0, out.ctypes.data) == -1


def test_oracle_accumulate_form():
    """The paper's routine adds into the caller's counters (§4, Fig. 6)."""
    w = synth.uniform_bits(3, 100, 16)
    c = np.full(16, 5, dtype=np.uint64)
    oracle.pospopcnt_add(w, c)
    assert np.array_equal(c, oracle.pospopcnt(w) + np.uint64(5))


@pytest.mark.parametrize("k", WIDTHS)
def test_oracle_mt_equals_single(k):
    w = synth.uniform_bits(61, 100003, k)
    ref = oracle.pospopcnt(w, k)
    for t in (1, 2, 3, 8, 64):
        c, used = oracle.pospopcnt_mt(w, k, t)
        assert np.array_equal(c, ref) and 1 <= used <= t


def test_oracle_segments():
    """Each segment row is the definition on its slice; rows sum to the span."""
    k = 16
    w = synth.uniform_bits(71, 5000, k)
    off = np.array([3, 3, 4, 100, 1000, 1000, 4999, 5000], dtype=np.int64)
    rows = oracle.pospopcnt_segments(w, off, k)
    for s in range(off.size - 1):
        assert np.array_equal(rows[s], oracle.pospopcnt(w[off[s]:off[s + 1]], k))
    assert np.array_equal(rows.sum(axis=0, dtype=np.uint64), oracle.pospopcnt(w[3:5000], k))
    lib = oracle._load()
    bad = np.array([5, 4], dtype=np.int64)
    out = np.zeros((1, k), dtype=np.uint64)
    assert lib.oracle_pospopcnt_segments(k, w.ctypes.data, bad.ctypes.data, 1, out.ctypes.data) == -1


# --------------------------------------------------------------------------
# the paper's CSA method (§2-§4.1) reaches the definition exactly
# --------------------------------------------------------------------------

def test_csa_truth_tables_table2(golden_dir):
    """§3, Table 2: row by row, and the immediates 150 / 232 of the text."""
    t = _read_sections(os.path.join(golden_dir, "table2_csa_truth.txt"))
    for which, sec in ((0, "lsb"), (1, "msb")):
        imm = 0
        for in1, in2, in3, out, idx in (map(int, r) for r in t[sec]["rows"]):
            assert idx == in1 + 2 * in2 + 4 * in3
            s = in1 + in2 + in3
            assert out == ((s & 1) if which == 0 else (s >> 1))  # sum of three bits
            imm |= out << idx
        assert imm == int(t[sec]["arg"])
        assert oracle.csa_truth(which) == imm
    assert oracle.csa_truth(0) == 0b10010110 == 150
    assert oracle.csa_truth(1) == 0b11101000 == 232


def test_csa_circuit_size():
    """§2: 2^N - 1 CSAs suffice for 2^N inputs."""
    for N in range(1, 11):
        assert oracle.csa_circuit_size(N) == (1 << N) - 1


def test_section41_instruction_arithmetic(golden_dir):
    """§4.1: two logic instructions per CSA, plus 48 for the counter
    increment, divided by the 16-bit words of one block."""
    rows = [line.split() for line in open(os.path.join(golden_dir,
            "section41_instruction_counts.txt")) if line.strip() and not line.startswith("#")]
    assert len(rows) == 3
    for nbytes, regs, ins, total, per_word in rows:
        nbytes, regs, ins, total = int(nbytes), int(regs), int(ins), int(total)
        N = regs.bit_length() - 1
        assert nbytes == 64 * regs
        assert ins == 2 * oracle.csa_circuit_size(N)
        assert total == ins + 3 * 16
        assert f"{total / (nbytes // 2):.2f}" == per_word


@pytest.mark.parametrize("k", WIDTHS)
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_csa_method_equals_definition(k, N):
    block_words = (64 << N) // (k // 8)
    for seed, n in ((1, 0), (2, 1), (3, block_words - 1), (4, block_words),
                    (5, 3 * block_words + 5), (6, 40000)):
        w = synth.uniform_bits(100 * N + seed, n, k)
        c, calls = oracle.csa_pospopcnt(w, k, N)
        assert np.array_equal(c, oracle.pospopcnt(w, k))
        nblocks = (n * (k // 8)) // (64 << N)
        assert calls == nblocks * ((1 << N) - 1)


def test_csa_method_saturated_and_one_hot():
    k = 16
    ones = np.full(1 << 16, 0xFFFF, dtype=np.uint16)
    c, _ = oracle.csa_pospopcnt(ones, k, 4)
    assert np.all(c == 1 << 16)
    w = synth.one_hot(9, 70001, 16)
    c, _ = oracle.csa_pospopcnt(w, k, 3)
    assert np.array_equal(c, oracle.pospopcnt(w))


# --------------------------------------------------------------------------
# the pins catch plausible mistakes: broken copies of the oracle must fail
# --------------------------------------------------------------------------

MUTANTS = {
    "shift_off_by_one": ("counts[p] += (w >> p) & 1u;", "counts[p] += (w >> (p + 1)) & 1u;"),
    "big_endian_load": ("w |= (uint64_t)p[b] << (8 * b);", "w |= (uint64_t)p[b] << (8 * (k / 8 - 1 - b));"),
    "drops_last_word": ("for (uint64_t i = 0; i < n; ++i) {\n    uint64_t w = load_word",
                        "for (uint64_t i = 0; i + 1 < n; ++i) {\n    uint64_t w = load_word"),
    "reversed_position": ("counts[p] += (w >> p) & 1u;", "counts[k - 1 - p] += (w >> p) & 1u;"),
    "word_stride_one_byte": ("load_word(bytes + i * (uint64_t)(k / 8), k)", "load_word(bytes + i, k)"),
}


def _mutant_count(name, tmpdir):
    src = open(oracle._SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, name
    src = src.replace(old, new)
    cpath = os.path.join(tmpdir, f"m_{name}.c")
    so = os.path.join(tmpdir, f"m_{name}.so")
    open(cpath, "w").write(src)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread", cpath, "-o", so])
    lib = ctypes.CDLL(so)
    lib.oracle_pospopcnt.restype = ctypes.c_int
    lib.oracle_pospopcnt.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]

    def count(words, width):
        a = np.ascontiguousarray(words)
        out = np.zeros(width, dtype=np.uint64)
        n = a.size * a.itemsize // (width // 8)
        lib.oracle_pospopcnt(width, a.ctypes.data, n, out.ctypes.data)
        return out
    return count


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, golden_dir):
    with tempfile.TemporaryDirectory() as d:
        count = _mutant_count(name, d)
        failed = []
        for pin in ALL_PINS + [lambda c: pin_table1(c, golden_dir)]:
            try:
                pin(count)
            except AssertionError:
                failed.append(pin)
        assert failed, f"no pin caught mutant {name}"


# --------------------------------------------------------------------------
# array popcount (the single sum pospopcnt generalises)
# --------------------------------------------------------------------------

def test_popcount_pins():
    assert oracle.popcount(np.zeros(0, dtype=np.uint8)) == 0
    assert oracle.popcount(np.full(1000, 0xFF, dtype=np.uint8)) == 8000
    assert oracle.popcount(np.arange(256, dtype=np.uint8)) == 1024  # each bit set in half of 256 bytes
    for seed, n in ((1, 1), (2, 333), (3, 1 << 16)):
        b = synth.uniform_bytes(seed, n)
        ref = _popcount_total(b)  # independent library popcount
        assert oracle.popcount(b) == ref
        assert oracle.popcount(b) == int(oracle.pospopcnt(b, 8).sum())  # the sum of the positional counts


# --------------------------------------------------------------------------
# one-hot encode + count (the motivating pipeline of §1)
# --------------------------------------------------------------------------

def test_onehot_counts_table1(golden_dir):
    """§1, Table 1: the stream as category ids (the one-hot positions) gives
    France 3, Portugal 2, USA 4, China 1."""
    mapping, stream, freq = load_table1(golden_dir)
    pos = {name: code.bit_length() - 1 for name, code in mapping.items()}
    ids = np.array([pos[name] for _, name in stream], dtype=np.uint8)
    c = oracle.onehot_counts(ids, 8)
    for name, p in pos.items():
        assert int(c[p]) == freq.get(name, 0)


def pin_onehot_high_bits(onehot):
    """Ids whose low bits name a category but whose high bits are set
    (256 + j, 0xFF00 + j, 0xFFFF; for 32-bit ids also 0x10000 + j,
    0xFFFFFFE0 + j, 2^31, 2^32 - 1) are no category below k: only the valid
    ids are counted, as numpy.bincount counts them."""
    rng = np.random.default_rng(21)
    low = [256 + j for j in range(32)] + [0xFF00 + j for j in range(32)] + [0xFFFF]
    for dt, decoys in ((np.uint16, low),
                       (np.uint32, low + [0x10000 + j for j in range(32)] + [0xFFFFFFE0 + j for j in range(32)] +
                        [1 << 31, 0xFFFFFFFF])):
        for k in (1, 8, 16, 32):
            valid = rng.integers(0, k, size=3000)
            ids = np.concatenate([valid, np.repeat(np.array(decoys, dtype=np.int64), 5)]).astype(dt)
            rng.shuffle(ids)
            ref = np.bincount(valid, minlength=k)[:k].astype(np.uint64)
            assert np.array_equal(onehot(ids, k), ref), (dt, k)


def test_onehot_counts_ignore_ids_with_high_bits():
    pin_onehot_high_bits(oracle.onehot_counts)


ONEHOT_MUTANTS = {
    "id_low_byte_only": ("for (int j = 0; j < id_bytes; ++j) v |=", "for (int j = 0; j < 1; ++j) v |="),
    "id_low_five_bits": ("const uint64_t word = v < (uint64_t)k ?", "v &= 31u;\n    const uint64_t word = v < (uint64_t)k ?"),
}


@pytest.mark.parametrize("name", sorted(ONEHOT_MUTANTS))
def test_onehot_pin_catches_mutant(name):
    """A copy of the oracle that reads an id only in part counts decoys; the
    pin above must fail on it."""
    src = open(oracle._SRC).read()
    old, new = ONEHOT_MUTANTS[name]
    assert src.count(old) == 1, name
    with tempfile.TemporaryDirectory() as d:
        cpath, so = os.path.join(d, f"m_{name}.c"), os.path.join(d, f"m_{name}.so")
        open(cpath, "w").write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread", cpath, "-o", so])
        lib = ctypes.CDLL(so)
        lib.oracle_onehot_counts.restype = ctypes.c_int
        lib.oracle_onehot_counts.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_void_p]

        def onehot(ids, k):
            a = np.ascontiguousarray(ids)
            out = np.zeros(k, dtype=np.uint64)
            assert lib.oracle_onehot_counts(a.ctypes.data, a.size, a.itemsize, k, out.ctypes.data) == 0
            return out
        with pytest.raises(AssertionError):
            pin_onehot_high_bits(onehot)


@pytest.mark.parametrize("dt", [np.uint8, np.uint16, np.uint32])
def test_onehot_counts_equal_bincount(dt):
    rng = np.random.default_rng(3)
    for k in (1, 5, 8, 13, 16, 32, 64):
        ids = rng.integers(0, min(np.iinfo(dt).max, 3 * k) + 1, size=5000).astype(dt)
        ref = np.bincount(ids[ids < k].astype(np.int64), minlength=k)[:k].astype(np.uint64)
        assert np.array_equal(oracle.onehot_counts(ids, k), ref)
        # and equals the positional count of the explicitly encoded words (k <= 32)
        if k <= 32:
            words = np.where(ids < k, np.uint64(1) << np.minimum(ids, 63).astype(np.uint64), 0).astype(np.uint32)
            assert np.array_equal(oracle.onehot_counts(ids, k), oracle.pospopcnt(words, 32)[:k])
