"""Thin ctypes binding of include/sv.h (argument marshalling only).

Every function named ``sv_*`` here calls the C entry point of the same name in
``_lib/libsqfree2k.so``; all computation happens in the CUDA kernels behind
it.  There is no CPU fallback: if the library is missing or cannot be loaded,
``load()`` raises.  PyTorch is used only for device buffers and the stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

u8, u32, u64 = ctypes.c_uint8, ctypes.c_uint32, ctypes.c_uint64
P = ctypes.POINTER

SV_OK, SV_EINVAL, SV_ERANGE, SV_ENOMEM, SV_EAGAIN, SV_ETIMEDOUT, SV_ECANCELLED = 0, 1, 2, 3, 4, 5, 6
SV_ECUDA, SV_ENOPRIMES, SV_ENOTFOUND, SV_EOVERFLOW = 7, 8, 9, 10
SV_REQ_RANGE, SV_REQ_POINTS = 0, 1
NO_N = (1 << 64) - 1
FAIL_K = 255


class sv_config(ctypes.Structure):
    _fields_ = [("tile_log2", u32), ("margin_log2", u32), ("threads", u32), ("large_prime_min", u32),
                ("bucket_capacity", u32), ("record_k_threshold", u32), ("ctas_per_sm", u32),
                ("stamp_primes", u32), ("list_capacity", u64), ("device_mem_budget", u64),
                ("cuda_stream", ctypes.c_void_p), ("list_stage_capacity", u32), ("mult_prime_log2", u32),
                ("serve_slots", u32), ("reserved1", u32)]


class sv_range_result(ctypes.Structure):
    _fields_ = [("lo", u64), ("hi", u64), ("n_odd", u64), ("hist", u64 * 64), ("first_n", u64 * 64),
                ("ksum", u64), ("kmax", u64), ("list", P(u64)), ("list_k", P(u8)), ("list_cap", u64),
                ("list_len", u64), ("failures", P(u64)), ("fail_cap", u64), ("fail_len", u64),
                ("per_n_k", P(u8)), ("list_overflow", u64)]


class sv_request(ctypes.Structure):
    _fields_ = [("kind", u32), ("reserved", u32), ("lo", u64), ("hi", u64), ("result", P(sv_range_result)),
                ("points", P(u64)), ("n_points", u64), ("out_k", P(u8))]


class sv_server_stats(ctypes.Structure):
    _fields_ = [("submitted", u64), ("completed", u64), ("cancelled", u64), ("refused", u64),
                ("odd_n_done", u64), ("launches", u64), ("in_flight", u64), ("queued", u64),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("peak_mem_in_flight", u64),
                ("wall_us", ctypes.c_double), ("loop_busy_us", ctypes.c_double)]


class sv_peaks(ctypes.Structure):
    _fields_ = [("smem_atomic_per_s", ctypes.c_double), ("smem_atomic_strike_per_s", ctypes.c_double),
                ("scan_mix_ops_per_s", ctypes.c_double), ("int_alu_ops_per_s", ctypes.c_double),
                ("popc_per_s", ctypes.c_double), ("sm_clock_max_mhz", ctypes.c_double), ("sms", u32),
                ("reserved", u32)]


_CTX = ctypes.c_void_p
_SIGS = {
    "sv_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "sv_create": (ctypes.c_int, [P(_CTX), P(sv_config)]),
    "sv_destroy": (None, [_CTX]),
    "sv_get_config": (ctypes.c_int, [_CTX, P(sv_config)]),
    "sv_set_config": (ctypes.c_int, [_CTX, P(sv_config)]),
    "sv_init_primes": (ctypes.c_int, [_CTX, u64]),
    "sv_prime_count": (ctypes.c_int, [_CTX, P(u64), P(u64)]),
    "sv_prime_table_copy": (ctypes.c_int, [_CTX, P(u32), P(u64), P(u64), P(u64), u64, P(u64)]),
    "sv_verify_range": (ctypes.c_int, [_CTX, u64, u64, P(sv_range_result)]),
    "sv_verify_range_noalloc": (ctypes.c_int, [_CTX, u64, u64, P(sv_range_result)]),
    "sv_verify_batch": (ctypes.c_int, [_CTX, P(u64), P(u64), ctypes.c_size_t, P(sv_range_result)]),
    "sv_launch_batch": (ctypes.c_int, [_CTX, P(u64), P(u64), ctypes.c_size_t]),
    "sv_fetch_batch": (ctypes.c_int, [_CTX, P(sv_range_result), ctypes.c_size_t]),
    "sv_min_k": (ctypes.c_int, [_CTX, P(u64), ctypes.c_size_t, P(u8)]),
    "sv_min_k_device": (ctypes.c_int, [_CTX, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "sv_sieve_bitmap": (ctypes.c_int, [_CTX, u64, u64, ctypes.c_void_p]),
    "sv_bitmap_words": (u64, [u64, u64]),
    "sv_launch_range": (ctypes.c_int, [_CTX, u64, u64, ctypes.c_void_p]),
    "sv_verify_range_plain": (ctypes.c_int, [_CTX, u64, u64, P(sv_range_result)]),
    "sv_launch_range_plain": (ctypes.c_int, [_CTX, u64, u64, ctypes.c_void_p]),
    "sv_fetch_range": (ctypes.c_int, [_CTX, P(sv_range_result)]),
    "sv_synchronize": (ctypes.c_int, [_CTX]),
    "sv_autotune": (ctypes.c_int, [_CTX, u64, u64, P(sv_config)]),
    "sv_autotune_batch": (ctypes.c_int, [_CTX, P(u64), P(u64), ctypes.c_size_t, P(sv_config)]),
    "sv_submit": (ctypes.c_int, [_CTX, P(sv_request), P(u64)]),
    "sv_submit_many": (ctypes.c_int, [_CTX, P(sv_request), ctypes.c_size_t, P(u64), P(ctypes.c_int)]),
    "sv_poll": (ctypes.c_int, [_CTX, u64, ctypes.c_int64]),
    "sv_cancel": (ctypes.c_int, [_CTX, u64]),
    "sv_server_stats_get": (ctypes.c_int, [_CTX, P(sv_server_stats)]),
    "sv_server_stats_reset": (ctypes.c_int, [_CTX]),
    "sv_last_transfer": (ctypes.c_int, [_CTX, P(u64), P(u64)]),
    "sv_kernel_launches": (u64, [_CTX]),
    "sv_measure_peaks": (ctypes.c_int, [_CTX, P(sv_peaks)]),
    "sv_inject_alloc_failures": (ctypes.c_int, [_CTX, u32]),
    "sv_inject_bulk_timeout": (ctypes.c_int, [_CTX, u32]),
    "sv_kernel_timing": (ctypes.c_int, [_CTX, ctypes.c_int]),
    "sv_kernel_time": (ctypes.c_int, [_CTX, ctypes.c_int, P(ctypes.c_double), P(u64)]),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load the GPU library (building it first if allowed); raises if impossible."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"GPU library missing: {_build.LIB} (run paper_2411_01964_gb300.build.build())")
            lib = ctypes.CDLL(_build.LIB)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class SvError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = load(False).sv_strerror(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")


def check(status: int, where: str) -> int:
    if status != SV_OK:
        raise SvError(status, where)
    return status


# --- same-named wrappers --------------------------------------------------

def sv_strerror(status: int) -> str:
    return load().sv_strerror(status).decode()


def sv_create(cfg: sv_config | None = None) -> ctypes.c_void_p:
    ctx = _CTX()
    check(load().sv_create(ctypes.byref(ctx), ctypes.byref(cfg) if cfg is not None else None), "sv_create")
    return ctx


def sv_destroy(ctx) -> None:
    load().sv_destroy(ctx)


def sv_get_config(ctx) -> sv_config:
    c = sv_config()
    check(load().sv_get_config(ctx, ctypes.byref(c)), "sv_get_config")
    return c


def sv_set_config(ctx, cfg: sv_config) -> None:
    check(load().sv_set_config(ctx, ctypes.byref(cfg)), "sv_set_config")


def sv_init_primes(ctx, max_hi: int) -> None:
    check(load().sv_init_primes(ctx, max_hi), "sv_init_primes")


def sv_prime_count(ctx) -> tuple[int, int]:
    n, m = u64(), u64()
    check(load().sv_prime_count(ctx, ctypes.byref(n), ctypes.byref(m)), "sv_prime_count")
    return n.value, m.value


def sv_prime_table_copy(ctx) -> tuple:
    """The resident prime table as numpy arrays (p, mu, inv, lim)."""
    n, _ = sv_prime_count(ctx)
    nd = u64()
    check(load().sv_prime_table_copy(ctx, None, None, None, None, 0, ctypes.byref(nd)), "sv_prime_table_copy")
    p = np.zeros(max(n, 1), dtype=np.uint32)
    mu = np.zeros(max(n, 1), dtype=np.uint64)
    inv = np.zeros(max(nd.value, 1), dtype=np.uint64)
    lim = np.zeros(max(nd.value, 1), dtype=np.uint64)
    check(load().sv_prime_table_copy(ctx, p.ctypes.data_as(P(u32)), mu.ctypes.data_as(P(u64)),
                                     inv.ctypes.data_as(P(u64)), lim.ctypes.data_as(P(u64)), n, ctypes.byref(nd)),
          "sv_prime_table_copy")
    return p[:n], mu[:n], inv[:nd.value], lim[:nd.value]


def sv_verify_range(ctx, lo: int, hi: int, out: sv_range_result) -> int:
    return load().sv_verify_range(ctx, lo, hi, ctypes.byref(out))


def sv_verify_range_noalloc(ctx, lo: int, hi: int, out: sv_range_result) -> int:
    return load().sv_verify_range_noalloc(ctx, lo, hi, ctypes.byref(out))


def sv_verify_batch(ctx, lo: np.ndarray, hi: np.ndarray, out) -> int:
    lo = np.ascontiguousarray(lo, dtype=np.uint64)
    hi = np.ascontiguousarray(hi, dtype=np.uint64)
    return load().sv_verify_batch(ctx, lo.ctypes.data_as(P(u64)), hi.ctypes.data_as(P(u64)), len(lo), out)


def sv_launch_batch(ctx, lo: np.ndarray, hi: np.ndarray) -> int:
    lo = np.ascontiguousarray(lo, dtype=np.uint64)
    hi = np.ascontiguousarray(hi, dtype=np.uint64)
    return load().sv_launch_batch(ctx, lo.ctypes.data_as(P(u64)), hi.ctypes.data_as(P(u64)), len(lo))


def sv_fetch_batch(ctx, out, count: int) -> int:
    return load().sv_fetch_batch(ctx, out, count)


def sv_min_k(ctx, points: np.ndarray, out_k: np.ndarray) -> int:
    return load().sv_min_k(ctx, points.ctypes.data_as(P(u64)), len(points), out_k.ctypes.data_as(P(u8)))


def sv_min_k_device(ctx, d_points_ptr: int, count: int, d_out_ptr: int) -> int:
    return load().sv_min_k_device(ctx, d_points_ptr, count, d_out_ptr)


def sv_sieve_bitmap(ctx, lo: int, hi: int, d_bitmap_ptr: int) -> int:
    return load().sv_sieve_bitmap(ctx, lo, hi, d_bitmap_ptr)


def sv_bitmap_words(lo: int, hi: int) -> int:
    return int(load().sv_bitmap_words(lo, hi))


def sv_launch_range(ctx, lo: int, hi: int, d_per_n_ptr: int | None = None) -> int:
    return load().sv_launch_range(ctx, lo, hi, d_per_n_ptr)


def sv_verify_range_plain(ctx, lo: int, hi: int, out: sv_range_result) -> int:
    return load().sv_verify_range_plain(ctx, lo, hi, ctypes.byref(out))


def sv_launch_range_plain(ctx, lo: int, hi: int, d_per_n_ptr: int | None = None) -> int:
    return load().sv_launch_range_plain(ctx, lo, hi, d_per_n_ptr)


def sv_fetch_range(ctx, out: sv_range_result) -> int:
    return load().sv_fetch_range(ctx, ctypes.byref(out))


def sv_synchronize(ctx) -> int:
    return load().sv_synchronize(ctx)


def sv_autotune(ctx, lo: int, hi: int) -> sv_config:
    c = sv_config()
    check(load().sv_autotune(ctx, lo, hi, ctypes.byref(c)), "sv_autotune")
    return c


def sv_autotune_batch(ctx, lo: np.ndarray, hi: np.ndarray) -> sv_config:
    lo = np.ascontiguousarray(lo, dtype=np.uint64)
    hi = np.ascontiguousarray(hi, dtype=np.uint64)
    c = sv_config()
    check(load().sv_autotune_batch(ctx, lo.ctypes.data_as(P(u64)), hi.ctypes.data_as(P(u64)), len(lo),
                                   ctypes.byref(c)), "sv_autotune_batch")
    return c


def sv_submit(ctx, req: sv_request) -> tuple[int, int]:
    t = u64()
    st = load().sv_submit(ctx, ctypes.byref(req), ctypes.byref(t))
    return st, t.value


def sv_submit_many(ctx, reqs, tickets, status) -> int:
    """reqs: a ctypes array of sv_request; tickets (uint64) and status (int32)
    numpy arrays of the same length."""
    return load().sv_submit_many(ctx, reqs, len(tickets), tickets.ctypes.data_as(P(u64)),
                                 status.ctypes.data_as(P(ctypes.c_int)))


def sv_poll(ctx, ticket: int, timeout_us: int) -> int:
    return load().sv_poll(ctx, ticket, timeout_us)


def sv_cancel(ctx, ticket: int) -> int:
    return load().sv_cancel(ctx, ticket)


def sv_server_stats_get(ctx) -> sv_server_stats:
    s = sv_server_stats()
    check(load().sv_server_stats_get(ctx, ctypes.byref(s)), "sv_server_stats_get")
    return s


def sv_server_stats_reset(ctx) -> None:
    check(load().sv_server_stats_reset(ctx), "sv_server_stats_reset")


def sv_last_transfer(ctx) -> tuple[int, int]:
    a, b = u64(), u64()
    check(load().sv_last_transfer(ctx, ctypes.byref(a), ctypes.byref(b)), "sv_last_transfer")
    return a.value, b.value


def sv_kernel_launches(ctx) -> int:
    return int(load().sv_kernel_launches(ctx))


KERNEL_IDS = {"init": 0, "bucket_fill": 1, "tile": 2, "stragglers": 3, "points": 4, "list_compact": 5,
              "sieve_pass": 6, "scan_pass": 7}


def sv_kernel_timing(ctx, enable) -> None:
    """enable: False (off), True (every kernel), or an iterable of KERNEL_IDS names."""
    if enable is True:
        arg = -1
    elif not enable:
        arg = 0
    else:
        arg = 0
        for name in enable:
            arg |= 1 << KERNEL_IDS[name]
    check(load().sv_kernel_timing(ctx, arg), "sv_kernel_timing")


def sv_kernel_time(ctx, kernel: int) -> tuple[float, int]:
    ms, n = ctypes.c_double(), u64()
    check(load().sv_kernel_time(ctx, kernel, ctypes.byref(ms), ctypes.byref(n)), "sv_kernel_time")
    return ms.value, n.value


def sv_measure_peaks(ctx) -> dict:
    """Measured shared-memory atomic and integer peaks of the context's GPU."""
    pk = sv_peaks()
    check(load().sv_measure_peaks(ctx, ctypes.byref(pk)), "sv_measure_peaks")
    return {name: getattr(pk, name) for name, _ in sv_peaks._fields_ if name != "reserved"}


def sv_inject_alloc_failures(ctx, count: int) -> None:
    """Test hook: the next `count` buffer allocations of the library fail."""
    check(load().sv_inject_alloc_failures(ctx, count), "sv_inject_alloc_failures")


def sv_inject_bulk_timeout(ctx, count: int) -> None:
    """Test hook: the next `count` plain-path launches let their bounded bulk-load waits run out."""
    check(load().sv_inject_bulk_timeout(ctx, count), "sv_inject_bulk_timeout")
