"""GB300 (sm_103a) verifier for C. Hercher, "On the Sum of Squarefree Integers
and a Power of Two" (arXiv 2411.01964).

For every odd n in a range: mink(n) = the smallest k >= 1 with n - 2^k a
positive squarefree integer (Algorithms 1 and 2, Sec. 3), aggregated into
histograms, records and lists.  The work runs in the CUDA library behind the C
ABI of include/sv.h; ``binding`` holds the same-named ctypes wrappers and
``Verifier`` below is a convenience layer over them (argument marshalling
only; there is no CPU path).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np

from . import binding as B
from .binding import NO_N, FAIL_K, SvError  # noqa: F401

__all__ = ["Verifier", "RangeResult", "B", "NO_N", "FAIL_K", "SvError"]


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
    list_len: int
    list_overflow: bool
    failures: np.ndarray
    fail_len: int
    per_n_k: np.ndarray | None = field(default=None)

    def records(self) -> dict:
        """Smallest n with mink >= m + 1 for each m (Table 3), for ranges from 3."""
        out = {}
        for m in range(1, 63):
            c = [self.first_n[k] for k in range(m + 1, 64) if self.first_n[k] != NO_N]
            if c:
                out[m] = min(c)
        return out


class _ResultBuffers:
    """Host buffers wired into an sv_range_result (fresh per call: the result
    keeps views of them)."""

    def __init__(self, list_cap: int, fail_cap: int, n_per_n: int | None, pinned: bool = False):
        self.res = B.sv_range_result()
        if pinned:
            # page-locked host memory: the library copies a single range's list
            # straight into it (no staging, no host copy)
            import torch
            self._pinned = (torch.zeros(max(list_cap, 1), dtype=torch.int64, pin_memory=True),
                            torch.zeros(max(list_cap, 1), dtype=torch.uint8, pin_memory=True))
            self.list_n = self._pinned[0].numpy().view(np.uint64)
            self.list_k = self._pinned[1].numpy()
        else:
            self.list_n = np.zeros(max(list_cap, 1), dtype=np.uint64)
            self.list_k = np.zeros(max(list_cap, 1), dtype=np.uint8)
        self.fails = np.zeros(max(fail_cap, 1), dtype=np.uint64)
        self.per_n = np.zeros(max(n_per_n, 1), dtype=np.uint8) if n_per_n is not None else None
        r = self.res
        r.list = self.list_n.ctypes.data_as(B.P(B.u64))
        r.list_k = self.list_k.ctypes.data_as(B.P(B.u8))
        r.list_cap = list_cap
        r.failures = self.fails.ctypes.data_as(B.P(B.u64))
        r.fail_cap = fail_cap
        if self.per_n is not None:
            r.per_n_k = self.per_n.ctypes.data_as(B.P(B.u8))

    def result(self) -> RangeResult:
        r = self.res
        nl = min(r.list_len, r.list_cap)
        nf = min(r.fail_len, r.fail_cap)
        pn = None
        if self.per_n is not None:
            pn = self.per_n[: r.n_odd]
        return RangeResult(lo=r.lo, hi=r.hi, n_odd=r.n_odd, hist=[int(x) for x in r.hist],
                           first_n=[int(x) for x in r.first_n], ksum=r.ksum, kmax=r.kmax,
                           list_n=self.list_n[:nl], list_k=self.list_k[:nl],
                           list_len=r.list_len, list_overflow=bool(r.list_overflow),
                           failures=self.fails[:nf], fail_len=r.fail_len, per_n_k=pn)


def odd_count(lo: int, hi: int) -> int:
    nlo = max(lo, 3) | 1
    return (hi - nlo + 1) // 2 if hi > nlo else 0


class Verifier:
    """One library context on the current CUDA device."""

    def __init__(self, max_hi: int, *, stream=None, **knobs):
        cfg = B.sv_config()
        for k, v in knobs.items():
            setattr(cfg, k, v)
        if stream is not None:
            cfg.cuda_stream = ctypes.c_void_p(int(stream))
        self.ctx = B.sv_create(cfg)
        B.sv_init_primes(self.ctx, max_hi)
        self.max_hi = max_hi

    def close(self) -> None:
        if self.ctx:
            B.sv_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- configuration ------------------------------------------------------
    @property
    def config(self) -> B.sv_config:
        return B.sv_get_config(self.ctx)

    def set_config(self, **knobs) -> None:
        cfg = B.sv_get_config(self.ctx)
        for k, v in knobs.items():
            setattr(cfg, k, v)
        B.sv_set_config(self.ctx, cfg)

    def autotune(self, lo: int, hi: int) -> B.sv_config:
        return B.sv_autotune(self.ctx, lo, hi)

    def autotune_batch(self, los, his) -> B.sv_config:
        return B.sv_autotune_batch(self.ctx, np.asarray(los, dtype=np.uint64), np.asarray(his, dtype=np.uint64))

    def prime_count(self) -> tuple[int, int]:
        return B.sv_prime_count(self.ctx)

    # ---- blocking calls -----------------------------------------------------
    def verify_range(self, lo: int, hi: int, *, list_cap: int = 1 << 16, fail_cap: int = 1024,
                     per_n: bool = False) -> RangeResult:
        buf = _ResultBuffers(list_cap, fail_cap, odd_count(lo, hi) if per_n else None)
        B.check(B.sv_verify_range(self.ctx, lo, hi, buf.res), "sv_verify_range")
        return buf.result()

    def verify_range_plain(self, lo: int, hi: int, *, list_cap: int = 1 << 16, fail_cap: int = 1024,
                           per_n: bool = False) -> RangeResult:
        """The plain (unfused) path: the bitmap through device memory."""
        buf = _ResultBuffers(list_cap, fail_cap, odd_count(lo, hi) if per_n else None)
        B.check(B.sv_verify_range_plain(self.ctx, lo, hi, buf.res), "sv_verify_range_plain")
        return buf.result()

    def verify_batch(self, los, his, *, list_cap: int = 1 << 12, fail_cap: int = 64) -> list:
        n = len(los)
        bufs = [_ResultBuffers(list_cap, fail_cap, None) for _ in range(n)]
        arr = (B.sv_range_result * max(n, 1))()
        for i, b in enumerate(bufs):
            arr[i] = b.res
        B.check(B.sv_verify_batch(self.ctx, np.asarray(los, dtype=np.uint64), np.asarray(his, dtype=np.uint64),
                                  arr), "sv_verify_batch")
        out = []
        for i, b in enumerate(bufs):
            b.res = arr[i]
            out.append(b.result())
        return out

    def min_k(self, points) -> np.ndarray:
        pts = np.ascontiguousarray(np.asarray(points, dtype=np.uint64))
        out = np.zeros(max(len(pts), 1), dtype=np.uint8)
        B.check(B.sv_min_k(self.ctx, pts, out), "sv_min_k")
        return out[: len(pts)]

    def sieve_bitmap(self, lo: int, hi: int):
        """Algorithm 1 over [lo, hi) as a torch uint32 tensor on the device."""
        import torch
        nw = B.sv_bitmap_words(lo, hi)
        bm = torch.empty(max(nw, 1), dtype=torch.int32, device="cuda")
        B.check(B.sv_sieve_bitmap(self.ctx, lo, hi, bm.data_ptr()), "sv_sieve_bitmap")
        return bm[:nw]

    # ---- device-resident calls ------------------------------------------------
    def launch_range(self, lo: int, hi: int, d_per_n=None) -> None:
        ptr = d_per_n.data_ptr() if d_per_n is not None else None
        B.check(B.sv_launch_range(self.ctx, lo, hi, ptr), "sv_launch_range")

    def launch_range_plain(self, lo: int, hi: int, d_per_n=None) -> None:
        ptr = d_per_n.data_ptr() if d_per_n is not None else None
        B.check(B.sv_launch_range_plain(self.ctx, lo, hi, ptr), "sv_launch_range_plain")

    def fetch_range(self, *, list_cap: int = 1 << 16, fail_cap: int = 1024) -> RangeResult:
        buf = _ResultBuffers(list_cap, fail_cap, None)
        B.check(B.sv_fetch_range(self.ctx, buf.res), "sv_fetch_range")
        return buf.result()

    def launch_batch(self, los, his) -> None:
        self._pending_batch = len(los)
        B.check(B.sv_launch_batch(self.ctx, np.asarray(los, dtype=np.uint64), np.asarray(his, dtype=np.uint64)),
                "sv_launch_batch")

    def fetch_batch(self, *, list_cap: int = 1 << 12, fail_cap: int = 16) -> list:
        n = self._pending_batch
        bufs = [_ResultBuffers(list_cap, fail_cap, None) for _ in range(n)]
        arr = (B.sv_range_result * max(n, 1))()
        for i, b in enumerate(bufs):
            arr[i] = b.res
        B.check(B.sv_fetch_batch(self.ctx, arr, n), "sv_fetch_batch")
        out = []
        for i, b in enumerate(bufs):
            b.res = arr[i]
            out.append(b.result())
        return out

    def min_k_device(self, d_points, d_out) -> None:
        B.check(B.sv_min_k_device(self.ctx, d_points.data_ptr(), d_points.numel(), d_out.data_ptr()),
                "sv_min_k_device")

    def synchronize(self) -> None:
        B.check(B.sv_synchronize(self.ctx), "sv_synchronize")

    def last_transfer(self) -> tuple[int, int]:
        return B.sv_last_transfer(self.ctx)

    def kernel_launches(self) -> int:
        return B.sv_kernel_launches(self.ctx)


class Ticket:
    """A serving request and its buffers (kept alive until it is polled).
    Submitted on construction unless submit=False; then submit() sends it."""

    def __init__(self, v: "Verifier", kind: int, lo=0, hi=0, points=None, list_cap=4096, fail_cap=64,
                 submit: bool = True):
        self.kind = kind
        self.req = B.sv_request()
        self.req.kind = kind
        self.buf = None
        self.points = None
        self.out_k = None
        if kind == B.SV_REQ_RANGE:
            self.buf = _ResultBuffers(list_cap, fail_cap, None)
            self.req.lo, self.req.hi = lo, hi
            self.req.result = ctypes.pointer(self.buf.res)
        else:
            self.points = np.ascontiguousarray(np.asarray(points, dtype=np.uint64))
            self.out_k = np.zeros(max(len(self.points), 1), dtype=np.uint8)
            self.req.points = self.points.ctypes.data_as(B.P(B.u64))
            self.req.n_points = len(self.points)
            self.req.out_k = self.out_k.ctypes.data_as(B.P(B.u8))
        self.ctx = v.ctx
        self.id = None
        self.status = None
        if submit:
            self.submit()

    def submit(self) -> None:
        st, self.id = B.sv_submit(self.ctx, self.req)
        B.check(st, "sv_submit")

    def result(self):
        if self.kind == B.SV_REQ_RANGE:
            return self.buf.result()
        return self.out_k[: len(self.points)]


def _serving_methods():
    def submit_range(self, lo: int, hi: int, *, list_cap: int = 4096, fail_cap: int = 64) -> Ticket:
        return Ticket(self, B.SV_REQ_RANGE, lo=lo, hi=hi, list_cap=list_cap, fail_cap=fail_cap)

    def submit_points(self, points) -> Ticket:
        return Ticket(self, B.SV_REQ_POINTS, points=points)

    def poll(self, t: Ticket, timeout_us: int = -1) -> int:
        """SV_OK when finished (result ready), SV_EAGAIN while pending."""
        st = B.sv_poll(self.ctx, t.id, timeout_us)
        if st != B.SV_EAGAIN:
            t.status = st
        return st

    def cancel(self, t: Ticket) -> int:
        return B.sv_cancel(self.ctx, t.id)

    def server_stats(self) -> B.sv_server_stats:
        return B.sv_server_stats_get(self.ctx)

    def reset_server_stats(self) -> None:
        B.sv_server_stats_reset(self.ctx)

    def prepare_range(self, lo: int, hi: int, *, list_cap: int = 4096, fail_cap: int = 64) -> Ticket:
        """A range request with its buffers, not yet submitted (Ticket.submit)."""
        return Ticket(self, B.SV_REQ_RANGE, lo=lo, hi=hi, list_cap=list_cap, fail_cap=fail_cap, submit=False)

    def prepare_points(self, points) -> Ticket:
        return Ticket(self, B.SV_REQ_POINTS, points=points, submit=False)

    def submit_many(self, tickets) -> None:
        """Submits prepared tickets as one burst (sv_submit_many)."""
        n = len(tickets)
        if n == 0:
            return
        arr = (B.sv_request * n)()
        for i, t in enumerate(tickets):
            arr[i] = t.req
        ids = np.zeros(n, dtype=np.uint64)
        st = np.zeros(n, dtype=np.int32)
        B.sv_submit_many(self.ctx, arr, ids, st)
        for i, t in enumerate(tickets):
            B.check(int(st[i]), "sv_submit_many")
            t.id = int(ids[i])

    Verifier.submit_range = submit_range
    Verifier.submit_points = submit_points
    Verifier.poll = poll
    Verifier.cancel = cancel
    Verifier.server_stats = server_stats
    Verifier.reset_server_stats = reset_server_stats
    Verifier.prepare_range = prepare_range
    Verifier.prepare_points = prepare_points
    Verifier.submit_many = submit_many


_serving_methods()
