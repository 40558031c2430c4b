"""The resumable sweep (Sec. 4 "Results") on the host: chunking, journal,
resume after an interruption, several ranks.

The chunk results come from the CPU oracle through a stand-in runner, so
this file needs no GPU; tests/test_gpu_sweep.py runs the same driver on the
device.  The totals are pinned to Table 4 (the exact histogram of odd
n < 2^20, recomputed here as a prefix) and to Table 3 (the records).
"""
import json
import os

import pytest

import tables
from paper_2411_01964_gb300 import sweep as sw


class OracleRunner:
    """launch/fetch through the CPU oracle (one pending chunk at a time)."""

    def __init__(self, orc, fail_after=None):
        self.orc = orc
        self.pending = None
        self.fetched = 0
        self.fail_after = fail_after

    def launch(self, a, b):
        assert self.pending is None
        self.pending = (a, b)

    def fetch(self):
        if self.fail_after is not None and self.fetched >= self.fail_after:
            raise RuntimeError("interrupted")
        a, b = self.pending
        self.pending = None
        self.fetched += 1
        return self.orc.verify_range(a, b)


def test_chunk_bounds_partition():
    for lo, hi, c in [(3, 1000, 5), (3, 1 << 12, 12), (1 << 20, (1 << 20) + 12345, 7), (5, 6, 3)]:
        ch = sw.chunk_bounds(lo, hi, c)
        assert ch[0][0] == lo and ch[-1][1] == hi
        assert all(b == a2 for (_, b), (a2, _) in zip(ch, ch[1:]))
        assert all(b % 2 == 0 for _, b in ch[:-1])  # inner cuts are even: no odd n is split
        assert sum(sw.odd_count(a, b) for a, b in ch) == sw.odd_count(lo, hi)


def test_parse_int():
    assert sw.parse_int("2**50") == 1 << 50
    assert sw.parse_int("2**40+17") == (1 << 40) + 17
    assert sw.parse_int("2**50-5") == (1 << 50) - 5
    assert sw.parse_int("0x10") == 16


def test_sweep_matches_the_unsplit_range_and_table3(orc, tmp_path):
    hi = 1 << 20
    tot = sw.sweep(OracleRunner(orc), 3, hi, str(tmp_path / "j.jsonl"), chunk_log2=16)
    whole = orc.verify_range(3, hi)
    assert tot.hist == list(whole.hist) and tot.first_n == list(whole.first_n)
    assert tot.n_odd == whole.n_odd and tot.chunks == 16 and tot.fail_count == 0
    rec = tables.table3_records()
    for m in range(1, 6):  # R(5) = 434977 < 2^20
        assert tot.record(m) == rec[m]
    assert tot.record(6) is None or tot.record(6) > hi


def test_interrupted_sweep_resumes_to_the_same_totals(orc, tmp_path):
    hi = 1 << 19
    j = str(tmp_path / "j.jsonl")
    with pytest.raises(RuntimeError):
        sw.sweep(OracleRunner(orc, fail_after=3), 3, hi, j, chunk_log2=14)
    with open(j) as f:
        assert len(f.readlines()) == 1 + 3  # header + three finished chunks
    part = sw.sweep(OracleRunner(orc), 3, hi, j, chunk_log2=14, stop_after=4)
    assert part.chunks == 7
    # a torn last line (the process died while writing it) is dropped
    with open(j, "a") as f:
        f.write('{"lo": 1, "hist": [')
    tot = sw.sweep(OracleRunner(orc), 3, hi, j, chunk_log2=14)
    ref = sw.sweep(OracleRunner(orc), 3, hi, str(tmp_path / "ref.jsonl"), chunk_log2=14)
    assert tot.chunks == ref.chunks == 32
    assert tot.hist == ref.hist and tot.first_n == ref.first_n and tot.n_odd == ref.n_odd
    with open(j) as f:
        lines = f.readlines()
    assert len(lines) == 33 and all(json.loads(x) for x in lines)


def test_journal_of_another_sweep_is_refused(orc, tmp_path):
    j = str(tmp_path / "j.jsonl")
    sw.sweep(OracleRunner(orc), 3, 1 << 14, j, chunk_log2=12)
    with pytest.raises(ValueError):
        sw.sweep(OracleRunner(orc), 3, 1 << 15, j, chunk_log2=12)


def test_ranks_merge_to_the_single_sweep(orc, tmp_path):
    hi = 1 << 18
    base = str(tmp_path / "j.jsonl")
    for r in range(3):
        sw.sweep(OracleRunner(orc), 3, hi, base, chunk_log2=13, rank=r, world=3)
    merged = sw.merge_journals([sw.journal_path(base, r, 3) for r in range(3)])
    one = sw.sweep(OracleRunner(orc), 3, hi, str(tmp_path / "one.jsonl"), chunk_log2=13)
    assert merged.hist == one.hist and merged.first_n == one.first_n
    assert merged.n_odd == one.n_odd and merged.chunks == one.chunks == 32
    assert os.path.exists(base + ".0") and not os.path.exists(base)
