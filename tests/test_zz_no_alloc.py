"""sv_verify_range_noalloc: the verification entry point for callers that cannot
allocate memory when they verify.  Examples are a process whose GPU memory is
already held by another framework's caching allocator, where a cudaMalloc would
fail, and latency-critical loops, where cudaMalloc and cudaFree could stall the
device.  It must return exactly what sv_verify_range returns, on two calls in a
row: every call reuses the library's one fixed scratch array, so the second
call also checks that the first call's leftovers are cleared.

This file is collected last, so a run that stops at the first failure has
already run every other test."""
import numpy as np
import pytest

from paper_2411_01964_gb300 import B, Verifier
from paper_2411_01964_gb300 import _ResultBuffers

pytestmark = pytest.mark.gpu


def noalloc(v, lo, hi, list_cap=1 << 16, fail_cap=1024):
    buf = _ResultBuffers(list_cap, fail_cap, None)
    st = B.sv_verify_range_noalloc(v.ctx, lo, hi, buf.res)
    return st, buf.result()


def same(a, b):
    assert a.n_odd == b.n_odd
    assert a.hist == b.hist and a.first_n == b.first_n
    assert a.ksum == b.ksum and a.kmax == b.kmax
    assert a.list_len == b.list_len and a.fail_len == b.fail_len
    assert np.array_equal(a.list_n, b.list_n) and np.array_equal(a.list_k, b.list_k)
    assert np.array_equal(a.failures, b.failures)


RANGES = [
    (3, 1 << 24),                                             # from the start: records of Table 3
    ((1 << 40) + 12345, (1 << 40) + 12345 + (1 << 27) + 77),  # many tiles, ragged tail, buckets
    ((1 << 50) - (1 << 26) - 3, (1 << 50) + 5),               # the 2^25 prime table
]


@pytest.mark.parametrize("lo,hi", RANGES)
def test_matches_sv_verify_range_twice(lo, hi):
    with Verifier(max_hi=(1 << 50) + (1 << 20)) as v:
        want = v.verify_range(lo, hi, list_cap=1 << 16)
        for _ in range(2):
            st, got = noalloc(v, lo, hi)
            assert st == B.SV_OK, B.sv_strerror(st)
            same(got, want)


def test_small_list_capacity_keeps_the_smallest():
    lo, hi = (1 << 40), (1 << 40) + (1 << 26)
    with Verifier(max_hi=1 << 41) as v:
        want = v.verify_range(lo, hi, list_cap=7)
        st, got = noalloc(v, lo, hi, list_cap=7)
        assert st == B.SV_OK
        assert got.list_len == want.list_len > 7 and got.list_overflow
        assert np.array_equal(got.list_n, want.list_n) and np.array_equal(got.list_k, want.list_k)


def test_limits_are_reported():
    with Verifier(max_hi=1 << 45) as v:
        st, _ = noalloc(v, 1 << 40, (1 << 40) + (1 << 33))   # longer than the array allows
        assert st == B.SV_ERANGE
        st, got = noalloc(v, 10, 10)                           # empty range
        assert st == B.SV_OK and got.n_odd == 0 and sum(got.hist) == 0
        buf = _ResultBuffers(16, 16, 100)                      # per-n output is not offered
        assert B.sv_verify_range_noalloc(v.ctx, 3, 203, buf.res) == B.SV_EINVAL
