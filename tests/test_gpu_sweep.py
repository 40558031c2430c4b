"""The resumable sweep on the device (Sec. 4 "Results").

The sweep over odd n < 2^30 must give Table 4's exact histogram and Table 3's
records m <= 8.  The same totals must come back after an interruption and a
resume from the journal.
"""
import pytest

import tables
from paper_2411_01964_gb300 import Verifier, sweep as sw

pytestmark = pytest.mark.gpu


def test_sweep_below_2p30_reproduces_tables_3_and_4(tmp_path):
    hi = 1 << 30
    j = str(tmp_path / "j.jsonl")
    with Verifier(max_hi=hi) as v:
        part = sw.sweep(sw.GpuRunner(v), 3, hi, j, chunk_log2=26, stop_after=5)
        assert part.chunks == 5
        tot = sw.sweep(sw.GpuRunner(v), 3, hi, j, chunk_log2=26)
    assert tot.chunks == 16 and tot.fail_count == 0
    t4 = tables.table4_histogram()
    assert all(tot.hist[k] == t4.get(k, 0) for k in range(64))
    assert sum(tot.hist) == tot.n_odd == (1 << 29) - 1 and tot.ksum == sum(k * c for k, c in t4.items())
    t3 = tables.table3_records()
    for m in range(1, 9):
        assert tot.record(m) == t3[m]


def test_full_sweep_below_2p50_reproduces_sec4(tmp_path):
    # Sec. 4: every odd 1 < n < 2^50 has mink(n) <= 13 (the Theorem), the sum
    # of all mink is 684465092067182, and the records are those of Table 3
    # (m = 1..12).  About a minute on one GB300.
    hi = 1 << 50
    with Verifier(max_hi=hi) as v:
        tot = sw.sweep(sw.GpuRunner(v), 3, hi, str(tmp_path / "j.jsonl"), chunk_log2=37)
    assert tot.n_odd == (1 << 49) - 1 == sum(tot.hist)
    assert tot.fail_count == 0 and tot.kmax == 13
    assert tot.ksum == 684465092067182
    t3 = tables.table3_records()
    assert {m: tot.record(m) for m in range(1, 13)} == t3


def test_two_ranks_on_one_gpu_merge_to_the_single_sweep(tmp_path):
    # the multi-process partition (rank r takes chunks i = r mod world), run
    # here as two ranks one after the other on the same GPU: the merged
    # journals must equal the single-rank sweep and Tables 3 and 4 below 2^30
    hi = 1 << 30
    base = str(tmp_path / "j.jsonl")
    with Verifier(max_hi=hi) as v:
        parts = [sw.sweep(sw.GpuRunner(v), 3, hi, base, chunk_log2=26, rank=r, world=2) for r in (0, 1)]
        single = sw.sweep(sw.GpuRunner(v), 3, hi, str(tmp_path / "single.jsonl"), chunk_log2=26)
    assert parts[0].chunks == parts[1].chunks == 8 and single.chunks == 16
    merged = sw.merge_journals([sw.journal_path(base, r, 2) for r in (0, 1)])
    assert merged.hist == single.hist and merged.first_n == single.first_n
    assert merged.n_odd == single.n_odd == (1 << 29) - 1 and merged.fail_count == 0
    t4 = tables.table4_histogram()
    assert all(merged.hist[k] == t4.get(k, 0) for k in range(64))
    assert merged.ksum == sum(k * c for k, c in t4.items())
    t3 = tables.table3_records()
    for m in range(1, 9):
        assert merged.record(m) == t3[m]
