"""Seeded, synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds none of the method's arithmetic (no sieve, no squarefree
test): only the workload definitions and the random draws that shape them.
Everything is integer-only and platform independent (splitmix64; no libm), so
x86 and Arm hosts generate identical inputs.

Workloads (ranges are half-open; the odd n with max(lo, 3) <= n < hi):
  C1  [3, 2^24)                          primes <= 2^12
  C2  [2^40, 2^40 + 2^34)                primes <= isqrt(hi - 1) = 1056736
  C3  [2^50 - 2^36, 2^50)                primes <= 2^25
  C4  4096 requests, seed 7: start odd in [2^30, 2^50), length log-uniform in
      [2^10, 2^28] (at octave resolution, rounded to even)
  C5  serving mix, seed 11: Poisson arrivals; 70% short ranges (2^12..2^16),
      20% long ranges (2^24..2^30), 10% point batches (1..1024 odd points
      uniform in [3, 2^50))
"""
from __future__ import annotations

from dataclasses import dataclass

MASK64 = (1 << 64) - 1

C1 = (3, 1 << 24)
C2 = (1 << 40, (1 << 40) + (1 << 34))
C3 = ((1 << 50) - (1 << 36), 1 << 50)
CONFIGS = {"C1": C1, "C2": C2, "C3": C3}
TABLE_MAX_HI = (1 << 50) + (1 << 28)  # largest hi any C1..C5 request reaches


class SplitMix64:
    """Steele, Lea and Flood (2014) splitmix64 generator (its published constants)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def below(self, m: int) -> int:
        """Integer in [0, m) (modulo reduction; its bias below 2^-14 is accepted)."""
        return self.next() % m

    def unit(self) -> float:
        """53-bit uniform in [0, 1) (only for arrival times, never for ranges)."""
        return (self.next() >> 11) * (1.0 / (1 << 53))


def _log_uniform_even(rng: SplitMix64, lo_exp: int, hi_exp: int) -> int:
    """Length log-uniform over [2^lo_exp, 2^hi_exp] at octave resolution:
    octave e uniform in [lo_exp, hi_exp), then uniform inside [2^e, 2^(e+1)),
    rounded down to even (integer only)."""
    e = lo_exp + rng.below(hi_exp - lo_exp)
    length = (1 << e) + rng.below(1 << e)
    return length & ~1


def _odd_start(rng: SplitMix64, lo: int, hi: int) -> int:
    """Odd integer uniform in [lo, hi) (lo even)."""
    return lo + 1 + 2 * rng.below((hi - lo) // 2)


def batch_requests(seed: int = 7, count: int = 4096) -> list[tuple[int, int]]:
    """C4: `count` ranges (lo, hi); two draws per request, start then length."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        start = _odd_start(rng, 1 << 30, 1 << 50)
        length = _log_uniform_even(rng, 10, 28)
        out.append((start, start + length))
    return out


@dataclass
class ServeRequest:
    t_arrival: float  # seconds from the start of the run
    kind: str         # "short" | "long" | "points"
    lo: int = 0
    hi: int = 0
    points: tuple = ()


def serving_requests(rate_per_s: float, count: int, seed: int = 11,
                     long_max_exp: int = 30) -> list[ServeRequest]:
    """C5: open-loop Poisson arrivals at `rate_per_s`, mixed requests.

    Arrival gaps are exponential, drawn by inversion of a 53-bit uniform (the
    only floating point here: it only schedules requests, results never
    depend on it)."""
    import math
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    for _ in range(count):
        u = rng.unit()
        t += -math.log(1.0 - u) / rate_per_s
        c = rng.below(100)
        if c < 70:
            lo = _odd_start(rng, 1 << 30, 1 << 50)
            out.append(ServeRequest(t, "short", lo, lo + _log_uniform_even(rng, 12, 16)))
        elif c < 90:
            lo = _odd_start(rng, 1 << 30, 1 << 50)
            out.append(ServeRequest(t, "long", lo, lo + _log_uniform_even(rng, 24, long_max_exp)))
        else:
            npts = 1 + rng.below(1024)
            pts = tuple(_odd_start(rng, 2, 1 << 50) for _ in range(npts))
            out.append(ServeRequest(t, "points", points=pts))
    return out


def random_points(seed: int, count: int, lo: int, hi: int) -> list[int]:
    """Odd points uniform in [lo, hi) (lo even)."""
    rng = SplitMix64(seed)
    return [_odd_start(rng, lo, hi) for _ in range(count)]


def crt_forced(ell: int, count: int, seed: int = 3, max_bits: int = 62) -> list[int]:
    """Odd n with n = 2^k (mod p_{k+1}^2) for k = 1..ell (p_2 = 3, p_3 = 5, ...),
    which forces mink(n) >= ell + 1 (Remark in Sec. 2).  Built by the Chinese
    remainder theorem; n is the CRT solution plus a random multiple of the
    modulus, kept below 2^max_bits."""
    primes = []
    c = 3
    while len(primes) < ell:
        if all(c % p for p in range(3, int(c ** 0.5) + 1, 2)):
            primes.append(c)
        c += 2
    n, m = 1, 2  # n odd: n = 1 (mod 2)
    for k, p in enumerate(primes, start=1):
        q = p * p
        r = pow(2, k, q)
        # solve x = n (mod m), x = r (mod q)
        t = ((r - n) * pow(m, -1, q)) % q
        n, m = n + m * t, m * q
    rng = SplitMix64(seed)
    out = []
    limit = (1 << max_bits) // m
    for _ in range(count):
        j = rng.below(max(limit, 1))
        out.append(n + m * j)
    return out
