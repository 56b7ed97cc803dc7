"""The seeded generators: deterministic, thread-count independent, and
shaped as their recipes say."""
import numpy as np

import synth


def test_thread_count_independent():
    for t in (1, 3, 16):
        assert np.array_equal(synth.uniform_bits(5, 300001, 16, nthreads=t),
                              synth.uniform_bits(5, 300001, 16, nthreads=1))
        assert np.array_equal(synth.one_hot(5, 100003, 32, nthreads=t),
                              synth.one_hot(5, 100003, 32, nthreads=1))
        assert np.array_equal(synth.sparse(5, 70001, 8, nthreads=t),
                              synth.sparse(5, 70001, 8, nthreads=1))


def test_uniform_bytes_follow_draws():
    b = synth.uniform_bytes(9, 20)
    for j in range(20):
        assert int(b[j]) == (synth.draw(9, j // 8) >> (8 * (j % 8))) & 0xFF
    # a prefix of a longer stream is the shorter stream
    assert np.array_equal(synth.uniform_bytes(9, 13), b[:13])


def test_uniform_density():
    w = synth.uniform_bits(0, 1 << 20, 16)
    bits = np.unpackbits(w.view(np.uint8))
    assert abs(bits.mean() - 0.5) < 2e-3


def test_sparse_density():
    w = synth.sparse(0, 1 << 18, 16)
    bits = np.unpackbits(w.view(np.uint8))
    assert abs(bits.mean() - 0.01) < 1e-3


def test_zipf_cdf_shape():
    c = synth.zipf_cdf(16, 1.1).astype(np.float64) / 2.0 ** 32
    p = np.diff(np.concatenate([[0.0], c]))
    assert np.all(np.diff(c) > 0) and c[-1] == 1.0
    ref = np.array([(j + 1) ** -1.1 for j in range(16)])
    ref /= ref.sum()
    assert np.allclose(p, ref, atol=1e-9)
    assert abs(p[0] - 0.330) < 2e-3 and abs(p[15] - 0.0156) < 5e-4


def test_one_hot_frequencies_follow_cdf():
    w, pos = synth.one_hot(3, 1 << 20, 16, return_positions=True)
    assert np.all(w == (np.uint16(1) << pos.astype(np.uint16)))
    freq = np.bincount(pos, minlength=16) / float(1 << 20)
    p = np.diff(np.concatenate([[0.0], synth.zipf_cdf(16).astype(np.float64) / 2.0 ** 32]))
    assert np.allclose(freq, p, atol=3e-3)


def test_lengths_and_offsets():
    lens = synth.log_uniform_lengths(0, 2000)
    assert lens.min() >= 1 and lens.max() <= 1 << 20
    # log-uniform: the median length is near 2^10
    assert 300 < np.median(lens) < 3000
    off = synth.offsets_from_lengths(lens, start=5)
    assert off[0] == 5 and np.all(np.diff(off) == lens)


def test_segmented_one_hot():
    lens = synth.log_uniform_lengths(1, 50, max_len=4096)
    off = synth.offsets_from_lengths(lens, start=3)
    w = synth.segmented_one_hot(1, off, 16)
    assert np.all(w[:3] == 0)
    body = w[3:]
    assert np.all((body != 0) & ((body & (body - np.uint16(1))) == 0))
