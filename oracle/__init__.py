"""CPU oracle for the squarefree + power-of-two verification (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
and reference legs may import this package. The GPU library never does, and
this package never loads the GPU library.

The arithmetic lives in ``oracle.c`` (plain C, exact uint64); this module only
compiles it with gcc and marshals arguments through ctypes.

Conventions (C. Hercher, arXiv 2411.01964):
  * squarefree(s): s >= 1 and no p^2 | s; 1 is squarefree (Sec. 4 Theorem
    asks for a positive squarefree s).
  * mink(n) for odd n >= 3: smallest k >= 1 with 2^k < n and n - 2^k
    squarefree (Algorithm 2 without the k_max cap); 255 marks failure and 0 an
    invalid n (even or < 3) in the point interface.
  * A range [lo, hi) covers the odd n with max(lo, 3) <= n < hi
    (Algorithm 1's half-open "[start; end[").
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NO_N = (1 << 64) - 1
FAIL_K = 255


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, -O2, pthreads)."""
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-Wall", "-pthread", "-shared", "-fPIC",
             "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _Result(ctypes.Structure):
    _fields_ = [
        ("lo", ctypes.c_uint64), ("hi", ctypes.c_uint64),
        ("list_k_threshold", ctypes.c_uint32), ("pad", ctypes.c_uint32),
        ("n_odd", ctypes.c_uint64),
        ("hist", ctypes.c_uint64 * 64), ("first_n", ctypes.c_uint64 * 64),
        ("ksum", ctypes.c_uint64), ("kmax", ctypes.c_uint64),
        ("list", ctypes.POINTER(ctypes.c_uint64)), ("list_k", ctypes.POINTER(ctypes.c_uint8)),
        ("list_cap", ctypes.c_uint64), ("list_len", ctypes.c_uint64),
        ("list_overflow", ctypes.c_uint64),
        ("failures", ctypes.POINTER(ctypes.c_uint64)),
        ("fail_cap", ctypes.c_uint64), ("fail_len", ctypes.c_uint64),
        ("per_n_k", ctypes.POINTER(ctypes.c_uint8)),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u64, u8p, u64p = ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(ctypes.c_uint64)
            lib.or_isqrt.argtypes = [u64]
            lib.or_isqrt.restype = u64
            lib.or_odd_primes.argtypes = [u64, ctypes.POINTER(ctypes.c_uint32), ctypes.c_int64]
            lib.or_odd_primes.restype = ctypes.c_int64
            lib.or_is_squarefree_brute.argtypes = [u64]
            lib.or_is_squarefree_brute.restype = ctypes.c_int
            lib.or_is_squarefree.argtypes = [u64]
            lib.or_is_squarefree.restype = ctypes.c_int
            lib.or_sieve_odd.argtypes = [u64, u64, u8p]
            lib.or_sieve_odd.restype = ctypes.c_int
            lib.or_verify_range.argtypes = [ctypes.POINTER(_Result), ctypes.c_int, u64, u64]
            lib.or_verify_range.restype = ctypes.c_int
            lib.or_verify_ranges.argtypes = [ctypes.POINTER(_Result), ctypes.c_int64, ctypes.c_int, u64, u64]
            lib.or_verify_ranges.restype = ctypes.c_int
            lib.or_verify_range_brute.argtypes = [ctypes.POINTER(_Result), ctypes.c_int]
            lib.or_verify_range_brute.restype = ctypes.c_int
            lib.or_min_k.argtypes = [u64p, u64, u8p]
            lib.or_min_k.restype = ctypes.c_int
            _lib = lib
    return _lib


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def isqrt(x: int) -> int:
    return int(_load().or_isqrt(x))


def odd_primes(limit: int) -> np.ndarray:
    """Odd primes 3 <= p <= limit (Eratosthenes), uint32, ascending."""
    lib = _load()
    n = lib.or_odd_primes(limit, None, 0)
    _check(0 if n >= 0 else int(n), "odd_primes")
    out = np.zeros(max(n, 1), dtype=np.uint32)
    lib.or_odd_primes(limit, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), n)
    return out[:n]


def is_squarefree(s: int) -> bool:
    r = _load().or_is_squarefree(s)
    _check(0 if r >= 0 else r, "is_squarefree")
    return bool(r)


def is_squarefree_brute(s: int) -> bool:
    return bool(_load().or_is_squarefree_brute(s))


def sieve_odd(lo: int, hi: int) -> np.ndarray:
    """Algorithm 1 over [lo, hi): uint8 flag per odd integer from lo|1 upward."""
    first = lo | 1
    count = (hi - first + 1) // 2 if hi > first else 0
    out = np.zeros(max(count, 1), dtype=np.uint8)
    _check(_load().or_sieve_odd(lo, hi, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))), "sieve_odd")
    return out[:count]


def min_k(points) -> np.ndarray:
    """mink of each point by trial division (0 = invalid n, 255 = failure)."""
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.uint64))
    out = np.zeros(max(len(pts), 1), dtype=np.uint8)
    _check(_load().or_min_k(pts.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), len(pts),
                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))), "min_k")
    return out[:len(pts)]


@dataclass
class RangeResult:
    lo: int
    hi: int
    n_odd: int
    hist: list
    first_n: list
    ksum: int
    kmax: int
    list_n: np.ndarray
    list_k: np.ndarray
    list_overflow: bool
    failures: np.ndarray
    per_n_k: np.ndarray | None = field(default=None)

    def records(self) -> dict:
        """Table 3 style records of a range that starts at 3: for each m, the
        smallest n whose mink is >= m + 1 (min over first_n[k], k > m)."""
        out = {}
        for m in range(1, 63):
            cands = [self.first_n[k] for k in range(m + 1, 64) if self.first_n[k] != NO_N]
            if cands:
                out[m] = min(cands)
        return out


def _run_range(lo, hi, list_k_threshold, list_cap, per_n, brute, threads, margin, chunk):
    lib = _load()
    r = _Result()
    r.lo, r.hi, r.list_k_threshold = lo, hi, list_k_threshold
    nlo = max(lo, 3) | 1
    n_odd = (hi - nlo + 1) // 2 if hi > nlo else 0
    lst = np.zeros(max(list_cap, 1), dtype=np.uint64)
    lstk = np.zeros(max(list_cap, 1), dtype=np.uint8)
    fails = np.zeros(1024, dtype=np.uint64)
    r.list = lst.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    r.list_k = lstk.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    r.list_cap = list_cap
    r.failures = fails.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    r.fail_cap = len(fails)
    pn = None
    if per_n:
        pn = np.zeros(max(n_odd, 1), dtype=np.uint8)
        r.per_n_k = pn.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    if threads <= 0:
        threads = os.cpu_count() or 1
    if brute:
        rc = lib.or_verify_range_brute(ctypes.byref(r), threads)
    else:
        rc = lib.or_verify_range(ctypes.byref(r), threads, margin, chunk)
    _check(rc, "verify_range")
    ll = min(r.list_len, list_cap)
    return RangeResult(
        lo=lo, hi=hi, n_odd=int(r.n_odd), hist=[int(x) for x in r.hist],
        first_n=[int(x) for x in r.first_n], ksum=int(r.ksum), kmax=int(r.kmax),
        list_n=lst[:ll].copy(), list_k=lstk[:ll].copy(), list_overflow=bool(r.list_overflow),
        failures=fails[:min(r.fail_len, len(fails))].copy(),
        per_n_k=(pn[:n_odd] if pn is not None else None))


def verify_range(lo: int, hi: int, list_k_threshold: int = 6, list_cap: int = 1 << 20,
                 per_n: bool = False, threads: int = 0, margin: int = 1 << 16,
                 chunk: int = 1 << 24) -> RangeResult:
    """Algorithm 1 + Algorithm 2 over [lo, hi) (threads <= 0: all host cores)."""
    return _run_range(lo, hi, list_k_threshold, list_cap, per_n, False, threads, margin, chunk)


def verify_range_brute(lo: int, hi: int, list_k_threshold: int = 6, list_cap: int = 1 << 20,
                       per_n: bool = False, threads: int = 0) -> RangeResult:
    """The definition: every n - 2^k decided by trial division (small ranges)."""
    return _run_range(lo, hi, list_k_threshold, list_cap, per_n, True, threads, 0, 0)


# P(mink >= T) from Table 2 (Sec. 2), only to size list buffers: a range whose
# list does not fit is run again with exact room.
_TAIL = {1: 1.0, 2: 1.8943e-1, 3: 2.4129e-2, 4: 2.1482e-3, 5: 1.3902e-4, 6: 6.8527e-6, 7: 2.6694e-7}


def verify_ranges(ranges, list_k_threshold: int = 6, threads: int = 0, margin: int = 1 << 16,
                  chunk: int = 1 << 24) -> list:
    """verify_range for each (lo, hi) of `ranges`, with one prime list shared by
    all and whole ranges spread over the host cores (longest first)."""
    lib = _load()
    ranges = [(int(a), int(b)) for a, b in ranges]
    count = len(ranges)
    if count == 0:
        return []
    if threads <= 0:
        threads = os.cpu_count() or 1
    order = sorted(range(count), key=lambda i: -(ranges[i][1] - ranges[i][0]))
    arr = (_Result * count)()
    keep = []
    tail = _TAIL.get(list_k_threshold, 1.0 if list_k_threshold < 1 else 1e-7)
    for slot, i in enumerate(order):
        lo, hi = ranges[i]
        nlo = max(lo, 3) | 1
        n_odd = (hi - nlo + 1) // 2 if hi > nlo else 0
        cap = int(4 * tail * n_odd) + 1024
        lst = np.zeros(cap, dtype=np.uint64)
        lstk = np.zeros(cap, dtype=np.uint8)
        fails = np.zeros(64, dtype=np.uint64)
        r = arr[slot]
        r.lo, r.hi, r.list_k_threshold = lo, hi, list_k_threshold
        r.list = lst.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
        r.list_k = lstk.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        r.list_cap = cap
        r.failures = fails.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
        r.fail_cap = len(fails)
        keep.append((lst, lstk, fails))
    _check(lib.or_verify_ranges(arr, count, threads, margin, chunk), "verify_ranges")
    out = [None] * count
    for slot, i in enumerate(order):
        r = arr[slot]
        lo, hi = ranges[i]
        if r.list_overflow or r.fail_len > r.fail_cap:
            out[i] = verify_range(lo, hi, list_k_threshold, list_cap=int(r.list_len) + 1, threads=threads,
                                  margin=margin, chunk=chunk)
            continue
        lst, lstk, fails = keep[slot]
        ll = int(r.list_len)
        out[i] = RangeResult(
            lo=lo, hi=hi, n_odd=int(r.n_odd), hist=[int(x) for x in r.hist],
            first_n=[int(x) for x in r.first_n], ksum=int(r.ksum), kmax=int(r.kmax),
            list_n=lst[:ll].copy(), list_k=lstk[:ll].copy(), list_overflow=False,
            failures=fails[:int(r.fail_len)].copy())
    return out
