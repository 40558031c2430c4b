"""The sweep over every odd 1 < n < hi (Sec. 4 "Results"), chunk by chunk,
with a resumable journal.

Sec. 4 runs the method over all odd n below 2^50 and reports three things.
This module collects each of them:
  * the largest smallest exponent (the Theorem: mink(n) <= 13 below 2^50);
  * the sum of all smallest exponents (Sec. 3 "Collecting the results");
  * the records of Table 3: R(m), the smallest odd n whose n - 2^1 .. n - 2^m
    are all not squarefree, i.e. the smallest n with mink(n) >= m + 1.

The sweep cuts [lo, hi) into chunks at multiples of 2^chunk_log2, so every
odd n falls in exactly one chunk.  One chunk is one device-resident launch,
and the next chunk is launched before the previous one's results are
written, so the GPU never waits for the host.

Every finished chunk is appended to a journal (one JSON line: its bounds,
histogram, first occurrences and failures) and the file is synced at least
once a second.  A later run with the same journal skips the chunks it holds.
It drops a torn last line, so an interrupted sweep resumes where its journal
ends and ends with the same totals as an uninterrupted one.

With several processes, rank r takes the chunks i = r (mod world) into its
own journal, and `merge_journals` combines them.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time
from dataclasses import dataclass, field

NO_N = (1 << 64) - 1
KMAX = 64
JOURNAL_VERSION = 1


@dataclass
class SweepTotals:
    """Merged results of the chunks done so far."""
    lo: int
    hi: int
    chunks: int = 0
    n_odd: int = 0
    hist: list = field(default_factory=lambda: [0] * KMAX)
    first_n: list = field(default_factory=lambda: [NO_N] * KMAX)
    fail_count: int = 0
    failures: list = field(default_factory=list)  # the smallest ones, at most 1024

    def add(self, rec: dict) -> None:
        self.chunks += 1
        self.n_odd += rec["n_odd"]
        for k, c in enumerate(rec["hist"]):
            self.hist[k] += c
        for k, n in rec["first"].items():
            k = int(k)
            if n < self.first_n[k]:
                self.first_n[k] = n
        self.fail_count += rec["fail"]
        self.failures = sorted(self.failures + rec["fails"])[:1024]

    @property
    def ksum(self) -> int:
        return sum(k * c for k, c in enumerate(self.hist))

    @property
    def kmax(self) -> int:
        return max((k for k, c in enumerate(self.hist) if c), default=0)

    def record(self, m: int) -> int | None:
        """R(m) over the swept prefix: min over k > m of first_n[k].  Exact
        as a record of [3, covered) only when the sweep started at 3."""
        v = min(self.first_n[m + 1:], default=NO_N)
        return None if v == NO_N else v

    def summary(self) -> dict:
        out = {"lo": self.lo, "hi": self.hi, "chunks": self.chunks, "n_odd": self.n_odd,
               "hist": {k: c for k, c in enumerate(self.hist) if c}, "ksum": self.ksum, "kmax": self.kmax,
               "failures": self.fail_count,
               "records": {m: self.record(m) for m in range(1, self.kmax) if self.record(m) is not None}}
        if self.n_odd:
            out["heuristic"] = heuristic_check(self)
        return out


def heuristic_check(tot: SweepTotals, z_flag: float = 6.0) -> dict:
    """The swept counts against the heuristic of Sec. 2: per k the expected
    count and binomial deviation over the swept odd n, the sum of the
    exponents against its expectation (Sec. 4), and every k whose count
    lies more than z_flag deviations away."""
    from . import heuristics
    dev = heuristics.deviations(tot.hist, tot.n_odd)
    E, sig = heuristics.expected_sum(2 * tot.n_odd)  # S/2 odd n below S
    return {"expected": {k: round(e, 1) for k, _, e, _, _ in dev if e >= 0.05},
            "z": {k: round(z, 3) for k, _, e, _, z in dev if e >= 0.05},
            "ksum_expected": round(float(E)), "ksum_z": float((tot.ksum - E) / sig),
            "flagged": [k for k, _, e, _, z in dev if z > z_flag]}


def chunk_bounds(lo: int, hi: int, chunk_log2: int) -> list[tuple[int, int]]:
    """[lo, hi) cut at the multiples of 2^chunk_log2 (even boundaries)."""
    c = 1 << chunk_log2
    out, a = [], lo
    while a < hi:
        b = min(hi, (a // c + 1) * c)
        out.append((a, b))
        a = b
    return out


def odd_count(lo: int, hi: int) -> int:
    nlo = max(lo, 3) | 1
    return (hi - nlo + 1) // 2 if hi > nlo else 0


def chunk_record(a: int, b: int, res) -> dict:
    """The journal line of one finished chunk (res: a RangeResult-like
    object with hist, first_n and failures, and fail_len when the failures
    may be truncated)."""
    hist = [int(x) for x in res.hist]
    fails = sorted(int(x) for x in res.failures)
    return {"lo": a, "hi": b, "n_odd": odd_count(a, b), "hist": hist,
            "first": {str(k): int(n) for k, n in enumerate(res.first_n) if int(n) != NO_N},
            "fail": int(getattr(res, "fail_len", len(fails))), "fails": fails}


class Journal:
    """Append-only JSON-lines journal of one sweep (one rank)."""

    def __init__(self, path: str, header: dict, sync_seconds: float = 1.0):
        self.path = path
        self.header = dict(header, kind="sweep", version=JOURNAL_VERSION)
        self.sync_seconds = sync_seconds
        self.records: list[dict] = []
        good = 0  # bytes of complete, valid lines
        if os.path.exists(path):
            with open(path, "rb") as f:
                data = f.read()
            pos = 0
            lines = []
            while True:
                nl = data.find(b"\n", pos)
                if nl < 0:
                    break  # a torn last line (no newline) is dropped
                try:
                    lines.append(json.loads(data[pos:nl]))
                except json.JSONDecodeError:
                    break  # a torn line, and anything after it, is dropped
                pos = nl + 1
                good = pos
            if lines:
                if {k: lines[0].get(k) for k in self.header} != self.header:
                    raise ValueError(f"journal {path} belongs to another sweep: {lines[0]}")
                self.records = lines[1:]
        self.f = open(path, "ab" if good else "wb")
        if good:
            self.f.truncate(good)
        else:
            self.f.write((json.dumps(self.header) + "\n").encode())
            self.f.flush()
            os.fsync(self.f.fileno())
        self.last_sync = time.monotonic()

    def append(self, rec: dict) -> None:
        self.f.write((json.dumps(rec) + "\n").encode())
        self.records.append(rec)
        now = time.monotonic()
        if now - self.last_sync >= self.sync_seconds:
            self.sync()
            self.last_sync = now

    def sync(self) -> None:
        self.f.flush()
        os.fsync(self.f.fileno())

    def close(self) -> None:
        self.sync()
        self.f.close()


def journal_path(base: str, rank: int, world: int) -> str:
    return base if world == 1 else f"{base}.{rank}"


def sweep(runner, lo: int, hi: int, journal: str, *, chunk_log2: int = 37, rank: int = 0, world: int = 1,
          stop_after: int | None = None, sync_seconds: float = 1.0) -> SweepTotals:
    """Sweep this rank's chunks of [lo, hi), resuming from `journal`.

    runner.launch(a, b) starts a chunk on the device, and runner.fetch()
    waits for it and returns its result.  The next chunk is launched before
    the previous one is journaled.  stop_after ends the run after that many
    new chunks (it is used to interrupt a sweep)."""
    header = {"lo": lo, "hi": hi, "chunk_log2": chunk_log2, "rank": rank, "world": world}
    jr = Journal(journal_path(journal, rank, world), header, sync_seconds)
    mine = [c for i, c in enumerate(chunk_bounds(lo, hi, chunk_log2)) if i % world == rank]
    tot = SweepTotals(lo, hi)
    done = 0
    for rec, (a, b) in zip(jr.records, mine):
        if (rec["lo"], rec["hi"]) != (a, b):
            raise ValueError(f"journal {jr.path}: chunk {rec['lo']}..{rec['hi']} where {a}..{b} was expected")
        tot.add(rec)
        done += 1
    todo = mine[done:]
    if stop_after is not None:
        todo = todo[:stop_after]
    try:
        if todo:
            runner.launch(*todo[0])
        for i, (a, b) in enumerate(todo):
            res = runner.fetch()
            if i + 1 < len(todo):
                runner.launch(*todo[i + 1])
            rec = chunk_record(a, b, res)
            jr.append(rec)
            tot.add(rec)
    finally:
        jr.close()
    return tot


def merge_journals(paths: list[str]) -> SweepTotals:
    """Totals over the chunks of several ranks' journals."""
    tot = None
    for p in paths:
        with open(p) as f:
            lines = [json.loads(x) for x in f if x.endswith("\n")]
        h = lines[0]
        if tot is None:
            tot = SweepTotals(h["lo"], h["hi"])
        for rec in lines[1:]:
            tot.add(rec)
    return tot


class GpuRunner:
    """Chunks through a Verifier's device-resident launch (no lists: the
    records come from the first occurrences)."""

    def __init__(self, verifier):
        self.v = verifier

    def launch(self, a: int, b: int) -> None:
        self.v.launch_range(a, b)

    def fetch(self):
        return self.v.fetch_range(list_cap=0, fail_cap=64)


def parse_int(s: str) -> int:
    """An integer, or a power written 2**e (optionally plus/minus an integer)."""
    s = s.replace(" ", "")
    for sign in ("+", "-"):
        head, sep, tail = s.rpartition(sign)
        if sep and "**" in head and head:
            v = parse_int(head)
            return v + int(tail, 0) if sign == "+" else v - int(tail, 0)
    if "**" in s:
        b, e = s.split("**", 1)
        return int(b, 0) ** int(e, 0)
    return int(s, 0)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--lo", type=parse_int, default=3)
    ap.add_argument("--hi", type=parse_int, default=1 << 50, help="exclusive upper end: an integer or 2**e")
    ap.add_argument("--journal", required=True)
    ap.add_argument("--chunk-log2", type=int, default=37)
    ap.add_argument("--rank", type=int, default=int(os.environ.get("RANK", 0)))
    ap.add_argument("--world", type=int, default=int(os.environ.get("WORLD_SIZE", 1)))
    ap.add_argument("--stop-after", type=int, default=None)
    args = ap.parse_args(argv)
    import torch
    from . import Verifier
    if torch.cuda.is_available():
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    t0 = time.perf_counter()
    with Verifier(max_hi=args.hi) as v:
        tot = sweep(GpuRunner(v), args.lo, args.hi, args.journal, chunk_log2=args.chunk_log2, rank=args.rank,
                    world=args.world, stop_after=args.stop_after)
    s = tot.summary()
    s["seconds"] = time.perf_counter() - t0
    print(json.dumps(s))
    return 0


if __name__ == "__main__":
    sys.exit(main())
