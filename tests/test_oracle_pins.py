"""Pins of the CPU oracle to values fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: the expected values are the
paper's Tables 3 and 4, the squarefree counting function Q(x) (Moebius
formula and the textbook value Q(10^6) = 607926), sympy's factorisation and
prime counts, brute-force trial division written out in Python, and the
Chinese-remainder construction of the Remark in Sec. 2.
"""
import random

import numpy as np
import pytest
import sympy

import tables
from paper_2411_01964_gb300 import inputs


def mobius_upto(n):
    mu = np.ones(n + 1, dtype=np.int64)
    is_comp = np.zeros(n + 1, dtype=bool)
    for p in range(2, n + 1):
        if not is_comp[p]:
            is_comp[2 * p::p] = True
            mu[p::p] *= -1
            mu[p * p::p * p] = 0
    mu[0] = 0
    return mu


def Q(x, mu):
    """#squarefree in [1, x] = sum_{d <= sqrt x} mu(d) floor(x / d^2)."""
    return sum(int(mu[d]) * (x // (d * d)) for d in range(1, int(x ** 0.5) + 1) if mu[d])


def Q_odd(x, mu):
    """#odd squarefree in [1, x] = sum_{d odd} mu(d) * #odd multiples of d^2 <= x."""
    if x < 1:
        return 0
    return sum(int(mu[d]) * ((x // (d * d) + 1) // 2) for d in range(1, int(x ** 0.5) + 1, 2) if mu[d])


def sqf_sympy(s):
    return s >= 1 and all(e == 1 for e in sympy.factorint(s).values())


def mink_python(n):
    """The definition written out in Python (independent of the C oracle)."""
    k = 1
    while (1 << k) < n:
        if sqf_sympy(n - (1 << k)):
            return k
        k += 1
    return 255


# --- Table 4 and Table 3 ------------------------------------------------------

@pytest.fixture(scope="module")
def below_2p30(orc):
    return orc.verify_range(3, 1 << 30, list_k_threshold=6)


def test_table4_exact_histogram(below_2p30):
    want = tables.table4_histogram()
    got = below_2p30.hist
    for k, cnt in want.items():
        assert got[k] == cnt, (k, got[k], cnt)
    assert sum(got) == (1 << 29) - 1 == below_2p30.n_odd
    assert all(got[k] == 0 for k in range(10, 64))
    # Sec. 3 "Collecting the results": sum and maximum of the exponents
    assert below_2p30.ksum == sum(k * c for k, c in want.items())
    assert below_2p30.kmax == 9
    assert len(below_2p30.failures) == 0


def test_table3_records_from_range(below_2p30):
    rec = below_2p30.records()
    want = tables.table3_records()
    for m in range(1, 9):  # n_m < 2^30 for m <= 8
        assert rec[m] == want[m], m
    assert 9 not in rec  # n_9 = 6915752957 > 2^30


def test_table3_points_have_exact_mink(orc):
    want = tables.table3_records()
    pts = [want[m] for m in sorted(want)]
    got = orc.min_k(pts)
    assert list(got) == [m + 1 for m in sorted(want)]


def test_list_matches_histogram_tail(below_2p30):
    # every n with mink >= 6 is listed, ascending, with its k
    assert len(below_2p30.list_n) == sum(below_2p30.hist[6:])
    assert np.all(np.diff(below_2p30.list_n.astype(np.int64)) > 0)
    ks, cnt = np.unique(below_2p30.list_k, return_counts=True)
    assert {int(k): int(c) for k, c in zip(ks, cnt)} == {6: 3473, 7: 122, 8: 24, 9: 3}


# --- the sieve (Algorithm 1) ----------------------------------------------------

def test_Q_1e6_textbook(orc):
    x = 10 ** 6
    odd = int(orc.sieve_odd(1, x + 1).sum())
    half = int(orc.sieve_odd(1, x // 2 + 1).sum())
    assert odd + half == 607926  # Q(10^6)
    assert Q(x, mobius_upto(1000)) == 607926


@pytest.mark.parametrize("a,b", [(1, 2), (1, 100), (2, 3), (8, 9), (9, 10), (10, 10), (1, 65), (63, 130),
                                 (1 << 20, (1 << 20) + 4096), (10 ** 9 + 7, 10 ** 9 + 20011),
                                 ((1 << 40) - 999, (1 << 40) + 77777)])
def test_sieve_window_counts_match_moebius(orc, a, b):
    mu = mobius_upto(int(b ** 0.5) + 2)
    got = int(orc.sieve_odd(a, b).sum())
    assert got == Q_odd(b - 1, mu) - Q_odd(a - 1, mu)


def test_sieve_matches_sympy_small(orc):
    lo, hi = 1, 20000
    flags = orc.sieve_odd(lo, hi)
    want = [1 if sqf_sympy(m) else 0 for m in range(1, hi, 2)]
    assert list(flags) == want


def test_sieve_matches_sympy_high_window(orc):
    lo = (1 << 50) - 3001
    hi = lo + 2000
    flags = orc.sieve_odd(lo, hi)
    want = [1 if sqf_sympy(m) else 0 for m in range(lo | 1, hi, 2)]
    assert list(flags) == want


def test_primes_against_sympy(orc):
    for lim in (3, 4, 9, 100, 4096, 1056736, 1 << 20):
        assert len(orc.odd_primes(lim)) == sympy.primepi(lim) - 1
    assert list(orc.odd_primes(2000)) == list(sympy.primerange(3, 2001))


def test_isqrt_exact(orc):
    rnd = random.Random(5)
    for x in [0, 1, 2, 3, 4, 15, 16, 17, (1 << 62), (1 << 62) - 1, (1 << 64) - 1] + \
             [rnd.getrandbits(64) for _ in range(200)]:
        r = orc.isqrt(x)
        assert r * r <= x < (r + 1) * (r + 1)


def test_squarefree_against_sympy(orc):
    rnd = random.Random(11)
    vals = [1, 2, 3, 4, 8, 9, 12, 25, 49, 121, 3 * 5 * 7, 9 * 11, 2 ** 31 - 1, 1018081,  # 1009^2
            (1 << 50) - 1, 4093 ** 2 * 3, 1000003 ** 2]
    vals += [rnd.randrange(1, 1 << 40) for _ in range(300)]
    for s in vals:
        want = sqf_sympy(s)
        assert orc.is_squarefree(s) == want, s
        if s < 10 ** 9:
            assert orc.is_squarefree_brute(s) == want, s


# --- the scan (Algorithm 2) and the point path ------------------------------

def test_range_against_python_definition(orc):
    lo, hi = 3, 3001
    r = orc.verify_range(lo, hi, per_n=True, list_k_threshold=3)
    want = [mink_python(n) for n in range(3, hi, 2)]
    assert list(r.per_n_k) == want


def test_sieve_method_equals_definition(orc):
    for lo, hi in [(3, 100001), (1 << 33, (1 << 33) + 20000), (6915752957 - 4000, 6915752957 + 4000)]:
        a = orc.verify_range(lo, hi, per_n=True, list_k_threshold=4)
        b = orc.verify_range_brute(lo, hi, per_n=True, list_k_threshold=4)
        assert a.hist == b.hist and a.first_n == b.first_n
        assert np.array_equal(a.per_n_k, b.per_n_k)
        assert np.array_equal(a.list_n, b.list_n) and np.array_equal(a.list_k, b.list_k)


def test_margin_and_chunk_do_not_change_results(orc):
    lo, hi = (1 << 40) + 1000, (1 << 40) + 1000 + 300000
    ref = orc.verify_range(lo, hi, per_n=True)
    for margin, chunk in [(2, 1 << 10), (64, 1 << 12), (1 << 20, 1 << 16)]:
        r = orc.verify_range(lo, hi, per_n=True, margin=margin, chunk=chunk)
        assert np.array_equal(r.per_n_k, ref.per_n_k)


def test_points_against_python_definition(orc):
    rnd = random.Random(2)
    pts = [3, 5, 7, 9, 11, 13, 2, 4, 1, 0] + [rnd.randrange(3, 1 << 36) | 1 for _ in range(200)]
    got = orc.min_k(pts)
    for n, k in zip(pts, got):
        want = 0 if (n < 3 or n % 2 == 0) else mink_python(n)
        assert k == want, n


def test_crt_forced_lower_bound(orc):
    # Remark (Sec. 2): n = 2^k (mod p_{k+1}^2) for k <= ell forces mink >= ell + 1
    for ell in (2, 3, 4, 5, 6):
        pts = inputs.crt_forced(ell, 8, seed=ell, max_bits=46)
        for n, k in zip(pts, orc.min_k(pts)):
            assert k >= ell + 1, (ell, n, k)
            assert k == mink_python(n)


def test_certificates_of_listed_n(orc):
    r = orc.verify_range(1 << 36, (1 << 36) + (1 << 22), list_k_threshold=5)
    assert len(r.list_n) > 10
    for n, k in list(zip(r.list_n.tolist(), r.list_k.tolist()))[:40]:
        assert sqf_sympy(n - (1 << k))
        for j in range(1, k):
            assert not sqf_sympy(n - (1 << j))


def test_heuristic_fractions_plausible(orc):
    """Table 2 (Sec. 2): P(mink = k) = c_k - c_{k-1}; counts within 6 sigma."""
    probs = {1: 8.1056e-1, 2: 1.6530e-1, 3: 2.1980e-2, 4: 2.0092e-3, 5: 1.3216e-4}
    r = orc.verify_range((1 << 40), (1 << 40) + (1 << 25))
    N = r.n_odd
    for k, p in probs.items():
        mean, sd = N * p, (N * p * (1 - p)) ** 0.5
        assert abs(r.hist[k] - mean) < 6 * sd + 0.002 * mean, (k, r.hist[k], mean)


def test_batch_driver_equals_single_ranges(orc):
    # the batch driver (one prime list for all ranges, whole ranges per
    # worker) only reorganises the work: each range's result is the one the
    # pinned single-range route gives
    reqs = [(3, 1 << 20), (1 << 40, (1 << 40) + (1 << 20) + 2), ((1 << 50) - (1 << 18) - 3, (1 << 50) + 7),
            (12345, 12345), (9, 10), (3, 4)] + inputs.batch_requests(7, 6)
    reqs = [(lo, min(hi, lo + (1 << 20))) for lo, hi in reqs]
    got = orc.verify_ranges(reqs)
    for (lo, hi), g in zip(reqs, got):
        o = orc.verify_range(lo, hi)
        assert (g.lo, g.hi, g.n_odd, g.ksum, g.kmax) == (lo, hi, o.n_odd, o.ksum, o.kmax)
        assert g.hist == o.hist and g.first_n == o.first_n
        assert np.array_equal(g.list_n, o.list_n) and np.array_equal(g.list_k, o.list_k)
        assert np.array_equal(g.failures, o.failures)
