"""The seeded workload generators: deterministic, integer-only, shaped as stated."""
import math

from paper_2411_01964_gb300 import inputs


def test_splitmix64_reference_values():
    # first outputs of splitmix64 seeded with 0 (Vigna's reference implementation)
    g = inputs.SplitMix64(0)
    assert [g.next() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_batch_requests_shape():
    reqs = inputs.batch_requests(7, 4096)
    assert len(reqs) == 4096
    assert reqs == inputs.batch_requests(7, 4096)
    for lo, hi in reqs:
        assert lo % 2 == 1 and (1 << 30) <= lo < (1 << 50)
        L = hi - lo
        assert L % 2 == 0 and (1 << 10) <= L < (1 << 28)
    # octave resolution: every octave 10..27 is used
    octs = {int(math.log2(hi - lo)) for lo, hi in reqs}
    assert octs == set(range(10, 28))


def test_serving_mix():
    reqs = inputs.serving_requests(1e4, 2000)
    kinds = [r.kind for r in reqs]
    assert 0.6 < kinds.count("short") / 2000 < 0.8
    assert 0.13 < kinds.count("long") / 2000 < 0.27
    assert 0.05 < kinds.count("points") / 2000 < 0.15
    ts = [r.t_arrival for r in reqs]
    assert all(b >= a for a, b in zip(ts, ts[1:]))
    assert 0.15 < ts[-1] < 0.25  # 2000 arrivals at 1e4/s
    for r in reqs:
        if r.kind == "points":
            assert 1 <= len(r.points) <= 1024
            assert all(p % 2 == 1 and 3 <= p < (1 << 50) for p in r.points)
        else:
            assert r.lo % 2 == 1 and (r.hi - r.lo) % 2 == 0


def test_crt_forced_congruences():
    for ell in (3, 5):
        for n in inputs.crt_forced(ell, 5, max_bits=50):
            assert n % 2 == 1 and n < (1 << 50)
            primes = [3, 5, 7, 11, 13, 17][:ell]
            for k, p in enumerate(primes, start=1):
                assert (n - (1 << k)) % (p * p) == 0
