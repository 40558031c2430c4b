"""The heuristic a priori probabilities of Sec. 2, in high precision on the
host, and the statistics Sec. 4 compares the counts with.

For a random odd n, c_l is the probability that at least one of
n - 2^1, ..., n - 2^l is squarefree.  The heuristic treats congruences
modulo different prime squares as independent (Sec. 2).  Inclusion-exclusion
over the sets I of exponents then gives

    c_l = sum over nonempty I in {1..l} of (-1)^(|I|-1) (1 - |I mod 6| / 9) d'_|I|,

with d'_k = prod over primes p >= 5 of (1 - k / p^2) (Sec. 2, "Computing c_l
for 7 <= l <= 20").  For l <= 20, p = 3 is the only prime where two
exponents of I can have equal 2^k mod p^2 (2^6 = 1 mod 9).  For l <= 6 the
formula reduces to the binomial sum over d_m = (1 - m/9) d'_m (Table 1).

This module evaluates d'_k well past the digits that Tables 1 and 2 print.
Sec. 2's Lemma truncates log(1 - kx) after its x^2 term (the zeta(2) and
zeta(4) tails).  Here the whole expansion is kept:

    log(1 - k x) = sum over j >= 1 of b_j log(1 - x^j),
    b_j = (1/j) sum over d | j of mu(j/d) k^d

(comparing the coefficients of x^n gives k^n = sum over j | n of j b_j, then
Moebius inversion).  With x = 1/p^2, the primes above a cut m contribute
prod over j of (prod over p > m of (1 - p^(-2j)))^(b_j).  Each inner product
equals 1 / (zeta(2j) prod over p <= m of (1 - p^(-2j))), and zeta(2j) is
exact from the Bernoulli numbers.  Stopping at j = J leaves a relative error
of about (k / m^2)^(J+1): below 1e-80 for m = 10^4, J = 12.

Sec. 4 uses the results as follows.  The smallest exponent of a random odd n
is k with probability c_k - c_(k-1) (c_0 = 0).  Its mean and standard
deviation give the expected sum E_S and its deviation sigma_S for the odd n
below S, and the expected count and binomial deviation of each k over N odd
n (Table 4).
"""
from __future__ import annotations

from decimal import Decimal, localcontext
from fractions import Fraction
from functools import lru_cache
from math import comb

PREC = 70  # decimal digits of the evaluation


def _primes_upto(m: int) -> list[int]:
    sieve = bytearray([1]) * (m + 1)
    sieve[0:2] = b"\x00\x00"
    for i in range(2, int(m ** 0.5) + 1):
        if sieve[i]:
            sieve[i * i::i] = bytearray(len(range(i * i, m + 1, i)))
    return [i for i in range(m + 1) if sieve[i]]


def _pi() -> Decimal:
    """pi by Machin's formula, 16 arctan(1/5) - 4 arctan(1/239)."""
    def arctan_inv(x: int) -> Decimal:
        x2 = x * x
        term = Decimal(1) / x
        total, n, sign = term, 1, 1
        eps = Decimal(10) ** (-(PREC + 5))
        while abs(term) > eps:
            term /= x2
            n += 2
            sign = -sign
            total += sign * term / n
        return total
    return 16 * arctan_inv(5) - 4 * arctan_inv(239)


@lru_cache(maxsize=None)
def _bernoulli(n: int) -> Fraction:
    """B_n with B_1 = -1/2, from sum over k <= n of C(n+1, k) B_k = 0."""
    if n == 0:
        return Fraction(1)
    return -sum(comb(n + 1, k) * _bernoulli(k) for k in range(n)) / (n + 1)


def _zeta_even(j: int, pi: Decimal) -> Decimal:
    """zeta(2j) = (-1)^(j+1) B_2j (2 pi)^(2j) / (2 (2j)!)."""
    b = _bernoulli(2 * j)
    f = (-1) ** (j + 1) * b / (2 * _factorial(2 * j))
    return Decimal(f.numerator) / Decimal(f.denominator) * (2 * pi) ** (2 * j)


def _factorial(n: int) -> int:
    out = 1
    for i in range(2, n + 1):
        out *= i
    return out


def _mobius(n: int) -> int:
    out, d = 1, 2
    while d * d <= n:
        if n % d == 0:
            n //= d
            if n % d == 0:
                return 0
            out = -out
        d += 1
    return -out if n > 1 else out


def _b(j: int, k: int) -> int:
    """Coefficient of log(1 - x^j) in log(1 - k x)."""
    s = sum(_mobius(j // d) * k ** d for d in range(1, j + 1) if j % d == 0)
    assert s % j == 0
    return s // j


@lru_cache(maxsize=None)
def d_prime(kmax: int = 20, m: int = 10 ** 4, J: int = 12) -> tuple:
    """(d'_1, ..., d'_kmax) with d'_k = prod over primes p >= 5 of (1 - k/p^2)."""
    with localcontext() as ctx:
        ctx.prec = PREC
        pi = _pi()
        ps = _primes_upto(m)
        # prod over p > m of (1 - p^(-2j)) = 1 / (zeta(2j) prod over p <= m of (1 - p^(-2j)))
        tail = []
        for j in range(1, J + 1):
            head = Decimal(1)
            for p in ps:
                head *= 1 - Decimal(1) / Decimal(p) ** (2 * j)
            tail.append(1 / (_zeta_even(j, pi) * head))
        out = []
        for k in range(1, kmax + 1):
            v = Decimal(1)
            for p in ps:
                if p >= 5:
                    v *= 1 - Decimal(k) / (p * p)
            for j in range(1, J + 1):
                v *= tail[j - 1] ** _b(j, k)
            out.append(+v)
        return tuple(out)


def d(m: int) -> Decimal:
    """d_m = prod over odd primes of (1 - m/p^2) = (1 - m/9) d'_m (Table 1)."""
    with localcontext() as ctx:
        ctx.prec = PREC
        return (1 - Decimal(m) / 9) * d_prime()[m - 1]


def _subset_counts(l: int) -> dict:
    """{(|I|, |I mod 6|): number of subsets I of {1..l}} (including I = {})."""
    sizes = [sum(1 for k in range(1, l + 1) if k % 6 == r) for r in range(6)]
    poly = {(0, 0): 1}
    for n in sizes:
        nxt = {}
        for (s, r), cnt in poly.items():
            nxt[(s, r)] = nxt.get((s, r), 0) + cnt
            for t in range(1, n + 1):
                key = (s + t, r + 1)
                nxt[key] = nxt.get(key, 0) + cnt * comb(n, t)
        poly = nxt
    return poly


def c(l: int) -> Decimal:
    """c_l: the probability that one of n - 2^1 .. n - 2^l is squarefree (1 <= l <= 20)."""
    if l == 0:
        return Decimal(0)
    if not 1 <= l <= 20:
        raise ValueError("c_l is defined here for 0 <= l <= 20")
    dp = d_prime()
    with localcontext() as ctx:
        ctx.prec = PREC
        total = Decimal(0)
        for (s, r), cnt in _subset_counts(l).items():
            if s == 0:
                continue
            total += (-1) ** (s - 1) * cnt * (1 - Decimal(r) / 9) * dp[s - 1]
        return +total


def p_exponent(k: int) -> Decimal:
    """The probability that the smallest exponent is k: c_k - c_(k-1).
    The exponents above 20 (probability < 5e-28) count as 21."""
    with localcontext() as ctx:
        ctx.prec = PREC
        if k == 21:
            return 1 - c(20)
        return c(k) - c(k - 1)


def exponent_moments() -> tuple:
    """Mean and standard deviation of the smallest exponent of a random odd n."""
    with localcontext() as ctx:
        ctx.prec = PREC
        ps = [p_exponent(k) for k in range(1, 22)]
        mean = sum(k * p for k, p in zip(range(1, 22), ps))
        second = sum(k * k * p for k, p in zip(range(1, 22), ps))
        return mean, (second - mean * mean).sqrt()


def expected_sum(S: int) -> tuple:
    """(E_S, sigma_S): expected sum of the smallest exponents of the odd
    1 < n < S and its standard deviation, taking S/2 odd n as Sec. 4 does."""
    mean, sd = exponent_moments()
    with localcontext() as ctx:
        ctx.prec = PREC
        half = Decimal(S) / 2
        return mean * half, sd * half.sqrt()


def expected_counts(N: int, kmax: int = 20) -> list:
    """[(k, expected count, binomial deviation)] over N odd n (Table 4)."""
    out = []
    with localcontext() as ctx:
        ctx.prec = PREC
        for k in range(1, kmax + 1):
            p = p_exponent(k)
            out.append((k, N * p, (N * p * (1 - p)).sqrt()))
    return out


def deviations(hist, N: int) -> list:
    """[(k, count, expected, sigma, |delta| / sigma)] of a histogram of the
    smallest exponents over N odd n, against the heuristic (Sec. 4)."""
    out = []
    for k, e, s in expected_counts(N):
        cnt = hist[k] if k < len(hist) else 0
        out.append((k, cnt, float(e), float(s), float(abs(cnt - e) / s) if s else 0.0))
    return out
