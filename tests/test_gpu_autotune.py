"""The autotuner: it must return SV_OK, leave a valid configuration in the
context, and never change a result (the tuned configuration gives exactly what
the default gives, and what the oracle gives)."""
import numpy as np
import pytest

from paper_2411_01964_gb300 import Verifier, inputs

pytestmark = pytest.mark.gpu


def same(a, b):
    assert a.hist == b.hist and a.first_n == b.first_n and a.ksum == b.ksum and a.kmax == b.kmax
    assert np.array_equal(a.list_n, b.list_n) and np.array_equal(a.list_k, b.list_k)


def test_autotune_single_range(orc):
    lo, hi = (1 << 40) + 1, (1 << 40) + (1 << 26)
    with Verifier(max_hi=1 << 41) as v:
        before = v.verify_range(lo, hi)
        chosen = v.autotune(lo, hi)
        cfg = v.config
        for f in ("tile_log2", "threads", "ctas_per_sm", "margin_log2", "stamp_primes", "large_prime_min",
                  "mult_prime_log2", "bucket_capacity"):
            assert getattr(chosen, f) == getattr(cfg, f), f
        after = v.verify_range(lo, hi)
    same(after, before)
    same(after, orc.verify_range(lo, hi))


def test_autotune_batch_keeps_results(orc):
    reqs = inputs.batch_requests(7, 64)
    reqs = [(lo, lo + min(hi - lo, 1 << 22)) for lo, hi in reqs]
    los, his = [a for a, _ in reqs], [b for _, b in reqs]
    with Verifier(max_hi=inputs.TABLE_MAX_HI) as v:
        before = v.verify_batch(los, his, list_cap=4096)
        chosen = v.autotune_batch(los, his)
        assert 10 <= chosen.mult_prime_log2 <= 31 and chosen.large_prime_min > 0
        after = v.verify_batch(los, his, list_cap=4096)
    want = orc.verify_ranges(reqs)
    for a, b, o in zip(after, before, want):
        same(a, b)
        same(a, o)
