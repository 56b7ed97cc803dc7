"""The benchmark's result check, on CPU: the references it compares timed
results with are the oracle's own results (computed over chunks on host
threads, which additivity makes equal to one call over the whole input), and
a result that differs makes the benchmark print no value and exit 3."""
import json
import os
import sys

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("width", (8, 16, 32, 64))
def test_reference_of_words_is_the_oracle(width):
    words = synth.uniform_bits(3 + width, 300_001, width)
    assert np.array_equal(bench.oracle_reference(words, width), oracle.pospopcnt(words, width))


def test_reference_of_popcount_is_the_oracle():
    b = synth.uniform_bytes(9, 1_000_003)
    assert bench.oracle_reference(b, 1).tolist() == [oracle.popcount(b)]


@pytest.mark.parametrize("dtype", (np.uint8, np.uint16, np.uint32))
def test_reference_of_onehot_ids_is_the_oracle(dtype):
    k = 23
    ids = synth.categorical_ids(5, 400_009, synth.zipf_cdf(k), dtype)
    ids[::97] = 200  # ids >= k count nothing
    assert np.array_equal(bench.oracle_reference(ids, 1, onehot_k=k), oracle.onehot_counts(ids, k))


def test_segment_rows_are_the_oracle():
    lens = synth.log_uniform_lengths(4, 300, max_len=1 << 12)
    off = synth.offsets_from_lengths(lens, start=3)
    words = synth.segmented_one_hot(4, off, 16)
    assert np.array_equal(bench.oracle_segments(words, off, 16), oracle.pospopcnt_segments(words, off, 16))


def test_failed_check_prints_no_value(monkeypatch, capsys):
    def timed_run_with_a_wrong_result(args, world, rank, local):
        raise bench.CheckFailed("timed counts differ from the oracle's")

    pytest.importorskip("torch")
    monkeypatch.setattr(bench, "run_plain", timed_run_with_a_wrong_result)
    rc = bench.cli(["--steps", "1", "--warmup", "3"])
    out = capsys.readouterr()
    assert rc == 3
    assert not [ln for ln in out.out.splitlines() if ln.startswith("{")]
    assert "check failed" in out.err


def test_passing_run_prints_one_line(monkeypatch, capsys):
    monkeypatch.setattr(bench, "run_plain", lambda args, world, rank, local: {"metric": "m", "value": 1.0})
    pytest.importorskip("torch")
    assert bench.cli(["--steps", "1", "--warmup", "3"]) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1 and json.loads(lines[0])["value"] == 1.0
