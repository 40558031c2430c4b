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


# ---- admission by device memory and failure paths (all made on the host) ----

def test_budget_refuses_what_can_never_fit():
    with Verifier(max_hi=1 << 46, device_mem_budget=1 << 20) as v:
        with pytest.raises(B.SvError) as e:
            v.submit_range((1 << 45) + 1, (1 << 45) + (1 << 20))
        assert e.value.status == B.SV_ENOMEM
        with pytest.raises(B.SvError) as e:
            v.submit_points([3, 5, 7])
        assert e.value.status == B.SV_ENOMEM
        assert v.server_stats().refused == 2


def test_budget_queues_and_holds(orc):
    budget = 14 << 20  # about two 2^30-integer chunks in flight at once
    lo0 = (1 << 44) + 1
    ranges = [(lo0 + i * (1 << 31), lo0 + i * (1 << 31) + (1 << 30) + 2 * i) for i in range(8)]
    with Verifier(max_hi=1 << 46, device_mem_budget=budget) as v:
        ts = [v.submit_range(a, b, list_cap=1 << 14) for a, b in ranges]
        for t in ts:
            assert v.poll(t, -1) == B.SV_OK
        st = v.server_stats()
        assert st.completed == len(ranges) and st.refused == 0
        assert 0 < st.peak_mem_in_flight <= budget
        for (a, b), t in zip(ranges, ts):
            alone = v.verify_range(a, b, list_cap=1 << 14)
            got = t.result()
            assert got.hist == alone.hist and got.first_n == alone.first_n
            assert np.array_equal(got.list_n, alone.list_n)


def test_poll_with_finite_timeout():
    lo, hi = (1 << 50) - (1 << 36), 1 << 50  # 2^35 odd n: milliseconds of work
    with Verifier(max_hi=(1 << 50) + 1) as v:
        t = v.submit_range(lo, hi)
        assert v.poll(t, 0) == B.SV_EAGAIN
        assert v.poll(t, 100) == B.SV_EAGAIN
        assert v.poll(t, -1) == B.SV_OK
        assert sum(t.result().hist) == (hi - lo) // 2


def test_injected_allocation_failure_is_a_status(orc):
    lo, hi = (1 << 44) + 1, (1 << 44) + (1 << 30)
    try:
        with Verifier(max_hi=1 << 46) as v:
            t = v.submit_range((1 << 44) + 1, (1 << 44) + (1 << 16))  # warms one slot, small buffers
            assert v.poll(t, -1) == B.SV_OK
            B.sv_inject_alloc_failures(v.ctx, 1)  # the larger request's buffers must grow: that fails
            t = v.submit_range(lo, hi)
            assert v.poll(t, -1) == B.SV_ENOMEM
            B.sv_inject_alloc_failures(v.ctx, 0)
            t = v.submit_range(lo, hi)                                   # the server serves on
            assert v.poll(t, -1) == B.SV_OK
            o = orc.verify_range(lo, hi)
            assert t.result().hist == o.hist and np.array_equal(t.result().list_n, o.list_n)
        with Verifier(max_hi=1 << 46) as v:                              # the blocking path
            B.sv_inject_alloc_failures(v.ctx, 1)
            with pytest.raises(B.SvError) as e:
                v.verify_range(lo, hi)
            assert e.value.status == B.SV_ENOMEM
            B.sv_inject_alloc_failures(v.ctx, 0)
            assert v.verify_range(lo, hi).hist == orc.verify_range(lo, hi).hist
    finally:
        from paper_2411_01964_gb300 import binding
        binding.load().sv_inject_alloc_failures(binding._CTX(1), 0)


def test_burst_submission_equals_single(orc):
    reqs = small_mix(96, seed=13)
    with Verifier(max_hi=inputs.TABLE_MAX_HI) as v:
        burst = [v.prepare_points(r.points) if r.kind == "points" else v.prepare_range(r.lo, r.hi, list_cap=4096)
                 for r in reqs]
        v.submit_many(burst[:50])
        v.submit_many(burst[50:])
        for t in burst:
            assert v.poll(t, -1) == B.SV_OK
        for r, t in zip(reqs, burst):
            if r.kind == "points":
                assert np.array_equal(t.result(), orc.min_k(r.points))
            else:
                alone = v.verify_range(r.lo, r.hi, list_cap=4096)
                assert t.result().hist == alone.hist and np.array_equal(t.result().list_n, alone.list_n)
        # a bad request in a burst fails alone; the others are queued
        good = v.prepare_range((1 << 40) + 1, (1 << 40) + 1001)
        bad = v.prepare_range(1 << 52, (1 << 52) + 10)  # beyond the prime table
        with pytest.raises(B.SvError) as e:
            v.submit_many([good, bad])
        assert e.value.status == B.SV_ERANGE
        assert good.id is not None and v.poll(good, -1) == B.SV_OK
