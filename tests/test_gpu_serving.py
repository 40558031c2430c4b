"""Serving (continuous batching): every request's result is the same alone
and in the mix, and equals the oracle; cancellation and stats behave."""
import numpy as np
import pytest

from paper_2411_01964_gb300 import B, Verifier, inputs

pytestmark = pytest.mark.gpu


def small_mix(n, seed=11):
    reqs = inputs.serving_requests(1e4, n, seed=seed, long_max_exp=25)
    return reqs


def test_mix_equals_alone_and_oracle(orc):
    reqs = small_mix(160)
    with Verifier(max_hi=inputs.TABLE_MAX_HI) as v:
        tickets = []
        for r in reqs:
            if r.kind == "points":
                tickets.append(v.submit_points(r.points))
            else:
                tickets.append(v.submit_range(r.lo, r.hi, list_cap=4096))
        for t in tickets:
            assert v.poll(t, -1) == B.SV_OK
        st = v.server_stats()
        assert st.completed == len(reqs) and st.p99_us >= st.p50_us > 0
        for i, (r, t) in enumerate(zip(reqs, tickets)):
            got = t.result()
            if r.kind == "points":
                assert np.array_equal(got, v.min_k(r.points))
                if i % 4 == 0:
                    assert np.array_equal(got, orc.min_k(r.points))
            else:
                alone = v.verify_range(r.lo, r.hi, list_cap=4096)
                assert got.hist == alone.hist and got.first_n == alone.first_n
                assert np.array_equal(got.list_n, alone.list_n)
                if r.kind == "short" or i % 8 == 0:
                    o = orc.verify_range(r.lo, r.hi)
                    assert got.hist == o.hist and got.first_n == o.first_n
                    assert np.array_equal(got.list_n, o.list_n)


def test_long_range_split_into_chunks(orc):
    lo = (1 << 45) + 1
    hi = lo + (1 << 31) + 12346  # several chunks plus a ragged one
    with Verifier(max_hi=1 << 46) as v:
        t = v.submit_range(lo, hi, list_cap=1 << 16)
        assert v.poll(t, -1) == B.SV_OK
        got = t.result()
        alone = v.verify_range(lo, hi, list_cap=1 << 16)
        assert got.hist == alone.hist and got.first_n == alone.first_n
        assert np.array_equal(got.list_n, alone.list_n)
        assert sum(got.hist) == got.n_odd


def test_cancel_and_unknown_ticket():
    with Verifier(max_hi=1 << 51) as v:
        ts = [v.submit_range((1 << 50) - (1 << 28) + 2 * i + 1, (1 << 50) - (1 << 28) + 2 * i + 1 + (1 << 28))
              for i in range(12)]
        outcomes = [v.cancel(t) for t in reversed(ts)]
        assert all(o in (B.SV_OK, B.SV_EAGAIN) for o in outcomes)
        for t, o in zip(reversed(ts), outcomes):
            st = v.poll(t, -1)
            assert st == (B.SV_ECANCELLED if o == B.SV_OK else B.SV_OK)
        assert B.sv_poll(v.ctx, 10 ** 9, 0) == B.SV_ENOTFOUND


def test_empty_and_invalid_requests():
    with Verifier(max_hi=1 << 41) as v:
        t = v.submit_range(10, 10)
        assert v.poll(t, -1) == B.SV_OK and t.result().n_odd == 0
        t = v.submit_points([])
        assert v.poll(t, -1) == B.SV_OK
        with pytest.raises(B.SvError):
            v.submit_range(1 << 42, (1 << 42) + 100)  # beyond the prime table
