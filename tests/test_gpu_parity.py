"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Everything here is integer work, so the bar is bit-exact equality: the
prime table, the sieve bitmap, every per-n mink, histograms, first
occurrences, lists and failures.  Sizes span several tiles and a ragged tail;
the knob sweeps (tile size, margin, threads, bucket threshold, CTAs per SM)
must never change a result.
"""
import numpy as np
import pytest

import tables
from paper_2411_01964_gb300 import Verifier, inputs

pytestmark = pytest.mark.gpu


def unpack_bitmap(words, lo, hi):
    """Flags of the odd integers of [lo, hi) from the sv_sieve_bitmap layout."""
    bits = np.unpackbits(words.view(np.uint8), bitorder="little")
    first = lo | 1
    f0 = (first - 1) // 2 - 32 * (lo // 64)
    cnt = (hi - first + 1) // 2 if hi > first else 0
    return bits, f0, cnt


def assert_same_range(g, o, per_n=True):
    assert g.n_odd == o.n_odd
    assert g.hist == o.hist
    assert g.first_n == o.first_n
    assert g.ksum == o.ksum and g.kmax == o.kmax
    assert np.array_equal(g.list_n, o.list_n)
    assert np.array_equal(g.list_k, o.list_k)
    assert np.array_equal(np.sort(g.failures), np.sort(o.failures))
    if per_n:
        assert np.array_equal(g.per_n_k, o.per_n_k)


def test_prime_table(gpu, orc):
    # element by element against the oracle's Eratosthenes, and every
    # constant against its definition (numpy uint64 arithmetic is exact)
    from paper_2411_01964_gb300 import B
    n, largest = gpu.prime_count()
    want = orc.odd_primes(orc.isqrt(inputs.TABLE_MAX_HI - 1))
    assert n == len(want) and largest == int(want[-1])
    p, mu, inv, lim = B.sv_prime_table_copy(gpu.ctx)
    assert np.array_equal(p, want)
    p64 = p.astype(np.uint64)
    top = np.uint64(2 ** 64 - 1)
    assert np.array_equal(mu, top // (p64 * p64))                 # Barrett constant of p^2
    nd = len(inv)
    assert nd == int(np.searchsorted(p, 1 << 21))                 # every p < 2^21
    with np.errstate(over="ignore"):
        assert np.all(p64[:nd] * inv == np.uint64(1))             # p * p^-1 = 1 mod 2^64
    assert np.array_equal(lim, top // p64[:nd])


@pytest.mark.parametrize("lo,hi", [
    (0, 1), (0, 2), (1, 2), (0, 64), (1, 65), (2, 66), (63, 200), (3, 1 << 16),
    (12345, 12345 + 5 * (1 << 21) + 77),                       # several tiles + ragged tail
    ((1 << 40) - 999, (1 << 40) + 3 * (1 << 21) + 13),
    ((1 << 50) - (1 << 22) - 5, (1 << 50) + 3),
    (8, 9), (9, 10), (9 * 9 * 17, 9 * 9 * 17 + 1),             # single odd values, struck or not
])
def test_sieve_bitmap(gpu, orc, lo, hi):
    words = gpu.sieve_bitmap(lo, hi).cpu().numpy().view(np.uint32)
    bits, f0, cnt = unpack_bitmap(words, lo, hi)
    want = orc.sieve_odd(lo, hi)
    assert np.array_equal(bits[f0:f0 + cnt], want)
    assert not bits[:f0].any() and not bits[f0 + cnt:].any()


def test_C1_full_range_per_n(gpu, orc):
    lo, hi = inputs.C1
    g = gpu.verify_range(lo, hi, per_n=True)
    o = orc.verify_range(lo, hi, per_n=True)
    assert_same_range(g, o)
    want = tables.table3_records()
    rec = g.records()
    for m in range(1, 7):  # n_m < 2^24 for m <= 6
        assert rec[m] == want[m]


RANGES = [
    (3, 4), (3, 5), (0, 3), (4, 4), (1, 100), (3, 1000),
    ((1 << 40) + 1, (1 << 40) + 2),
    ((1 << 40) + 12345, (1 << 40) + 12345 + (1 << 23) + 777),
    ((1 << 50) - (1 << 36) + 1001, (1 << 50) - (1 << 36) + 1001 + (1 << 22) + 333),
    (6915752957 - (1 << 20), 6915752957 + (1 << 20)),          # contains Table 3's n_9
]


@pytest.mark.parametrize("lo,hi", RANGES)
def test_ranges_default_config(gpu, orc, lo, hi):
    g = gpu.verify_range(lo, hi, per_n=True)
    o = orc.verify_range(lo, hi, per_n=True)
    assert_same_range(g, o)


KNOBS = [
    dict(tile_log2=14, margin_log2=10),
    dict(tile_log2=14, margin_log2=6),          # kwin = 6: mink >= 7 go to the exact path
    dict(tile_log2=16, margin_log2=17, threads=256),
    dict(tile_log2=17, large_prime_min=64),     # nearly every prime through the buckets
    dict(tile_log2=18, threads=512, ctas_per_sm=2),
    dict(tile_log2=20, margin_log2=18),
    dict(tile_log2=15, record_k_threshold=3),   # long lists
    dict(stamp_primes=2),
    dict(stamp_primes=6, tile_log2=19, threads=512, ctas_per_sm=2, margin_log2=13),
    dict(stamp_primes=8, tile_log2=16, record_k_threshold=5),
    dict(mult_prime_log2=14),                   # nearly all bucket primes through their multipliers
    dict(mult_prime_log2=24, large_prime_min=4096),  # nearly all through one Barrett reduction each
]


@pytest.mark.parametrize("knobs", KNOBS, ids=lambda k: "-".join(f"{a}{b}" for a, b in k.items()))
def test_knobs_do_not_change_results(orc, knobs):
    with Verifier(max_hi=(1 << 50) + (1 << 24), **knobs) as v:
        for lo, hi in [(3, 1 << 22), ((1 << 40) + 7, (1 << 40) + 7 + (1 << 22) + 99),
                       ((1 << 50) - (1 << 22) - 11, (1 << 50) + 5)]:
            g = v.verify_range(lo, hi, per_n=True)
            o = orc.verify_range(lo, hi, per_n=True, list_k_threshold=v.config.record_k_threshold)
            assert_same_range(g, o)
            # without the per-n output (T >= 6: the lean scan and the ordered list)
            assert_same_range(v.verify_range(lo, hi), o, per_n=False)


@pytest.mark.parametrize("lo,hi", [((1 << 53) - (1 << 22) - 11, (1 << 53) + 5),
                                   ((1 << 56) + 12345, (1 << 56) + 12345 + (1 << 21) + 77)])
def test_ranges_above_2p50(orc, lo, hi):
    # beyond the paper's sweep: prime tables past 2^25 (2^28 at 2^56)
    with Verifier(max_hi=hi + 1) as v:
        assert_same_range(v.verify_range(lo, hi, per_n=True), orc.verify_range(lo, hi, per_n=True))
        assert_same_range(v.verify_range(lo, hi), orc.verify_range(lo, hi), per_n=False)


def test_small_buckets_overflow_and_retry(orc):
    # a bucket capacity far too small must be detected on the device and grown
    with Verifier(max_hi=1 << 51, tile_log2=18, large_prime_min=40, bucket_capacity=1) as v:
        lo, hi = (1 << 50) - (1 << 23), 1 << 50
        g = v.verify_range(lo, hi, per_n=True)
        assert_same_range(g, orc.verify_range(lo, hi, per_n=True))


@pytest.mark.parametrize("stage_cap", [1, 2, 0])
def test_ordered_list_and_its_fallback(orc, stage_cap):
    # lists come out of the device ascending (staged per tile, compacted);
    # a tile with more listed n than it may stage repeats the launch through
    # the unordered list path, with the same results
    with Verifier(max_hi=(1 << 50) + (1 << 24), tile_log2=16, list_stage_capacity=stage_cap) as v:
        for lo, hi in [(3, 1 << 22), ((1 << 40) + 7, (1 << 40) + 7 + (1 << 23) + 99)]:
            o = orc.verify_range(lo, hi)
            assert_same_range(v.verify_range(lo, hi), o, per_n=False)
            g = v.verify_range(lo, hi, list_cap=7)
            assert g.list_len == len(o.list_n) and np.array_equal(g.list_n, o.list_n[:7])


def test_list_capacity_truncation_is_deterministic(gpu, orc):
    lo, hi = (1 << 40), (1 << 40) + (1 << 24)
    o = orc.verify_range(lo, hi)
    g = gpu.verify_range(lo, hi, list_cap=5)
    assert g.list_len == len(o.list_n) > 5 and g.list_overflow
    assert np.array_equal(g.list_n, o.list_n[:5])


def test_points(gpu, orc):
    want = tables.table3_records()
    pts = [want[m] for m in sorted(want)]
    pts += [0, 1, 2, 3, 4, 5, 7, 9, 11, 13, 15, 1 << 40, (1 << 40) + 1]
    pts += inputs.random_points(1, 300, 2, 1 << 50)
    pts += inputs.random_points(2, 100, 2, 1 << 30)
    pts += inputs.crt_forced(5, 10, max_bits=50) + inputs.crt_forced(6, 10, max_bits=50)
    g = gpu.min_k(pts)
    o = orc.min_k(pts)
    assert np.array_equal(g, o)
    assert list(g[:12]) == [m + 1 for m in sorted(want)]


def test_points_above_2p50(orc):
    # the exact path with prime tables past 2^25: random points up to 2^57
    # and CRT-forced points with mink >= 9 (Remark in Sec. 2)
    pts = inputs.random_points(4, 40, 1 << 50, 1 << 57) + inputs.crt_forced(8, 12, seed=9, max_bits=57)
    with Verifier(max_hi=(1 << 57) + 1) as v:
        g = v.min_k(pts)
    o = orc.min_k(pts)
    assert np.array_equal(g, o)
    assert all(int(k) >= 9 for k in g[40:])


def test_points_device_entry(gpu, orc):
    import torch
    pts = inputs.random_points(9, 257, 2, 1 << 46)
    d_pts = torch.tensor(np.array(pts, dtype=np.uint64).view(np.int64), device="cuda")
    d_out = torch.zeros(len(pts), dtype=torch.uint8, device="cuda")
    gpu.min_k_device(d_pts, d_out)
    gpu.synchronize()
    assert np.array_equal(d_out.cpu().numpy(), orc.min_k(pts))


def test_device_resident_launch(gpu, orc):
    import torch
    lo, hi = (1 << 44) + 999, (1 << 44) + 999 + 3 * (1 << 21) + 55
    n = (hi - (lo | 1) + 1) // 2
    d = torch.full((n,), 77, dtype=torch.uint8, device="cuda")
    gpu.launch_range(lo, hi, d)
    g = gpu.fetch_range()
    o = orc.verify_range(lo, hi, per_n=True)
    g.per_n_k = d.cpu().numpy()
    assert_same_range(g, o)


def test_batch_matches_oracle_per_request(gpu, orc):
    reqs = inputs.batch_requests(7, 48)
    # keep the lengths modest for the oracle; keep the starts as drawn
    reqs = [(lo, lo + min(hi - lo, 1 << 21)) for lo, hi in reqs] + [(3, 3), (5, 4), (3, 100)]
    res = gpu.verify_batch([a for a, _ in reqs], [b for _, b in reqs], list_cap=4096)
    for (lo, hi), g in zip(reqs, res):
        o = orc.verify_range(lo, hi)
        assert_same_range(g, o, per_n=False)


def test_repeatable(gpu):
    lo, hi = (1 << 45) + 1, (1 << 45) + (1 << 24)
    a = gpu.verify_range(lo, hi, per_n=True)
    b = gpu.verify_range(lo, hi, per_n=True)
    assert a.hist == b.hist and np.array_equal(a.per_n_k, b.per_n_k)


def test_kernel_timing_selects_kernels():
    """Per-kernel event timing: a set of kernel ids times only those kernels.
    Timing the tile kernel alone keeps launch_range on its captured graph,
    whose event nodes get fresh events at every replay: three launches give
    three timings."""
    from paper_2411_01964_gb300 import binding as B
    lo, hi = (1 << 40) + 1, (1 << 40) + (1 << 28)
    with Verifier(max_hi=hi + 1) as v:
        B.sv_kernel_timing(v.ctx, ["tile"])
        for _ in range(3):
            v.launch_range(lo, hi)
            r = v.fetch_range()
        assert sum(r.hist) == r.n_odd
        ms, n = B.sv_kernel_time(v.ctx, B.KERNEL_IDS["tile"])
        assert n == 3 and ms > 0
        for name in ("init", "bucket_fill", "stragglers", "list_compact"):
            assert B.sv_kernel_time(v.ctx, B.KERNEL_IDS[name])[1] == 0, name
        B.sv_kernel_timing(v.ctx, True)
        v.launch_range(lo, hi)
        v.fetch_range()
        for name in ("init", "bucket_fill", "tile", "stragglers", "list_compact"):
            assert B.sv_kernel_time(v.ctx, B.KERNEL_IDS[name])[1] == 1, name
        B.sv_kernel_timing(v.ctx, False)


def test_pinned_list_buffers_take_the_direct_copy():
    """A single range's list is copied straight into page-locked caller
    buffers: the same histogram and the same ascending list (n, mink) as
    through pageable buffers, also when the caller has room for only a prefix
    (the smallest entries), and nothing is written past the caller's room."""
    from paper_2411_01964_gb300 import _ResultBuffers, binding as B
    lo, hi = (1 << 40) + 1, (1 << 40) + (1 << 30)
    with Verifier(max_hi=hi + 1) as v:
        for cap in (1 << 13, 16):
            ref = _ResultBuffers(cap, 64, None)
            B.check(B.sv_verify_range(v.ctx, lo, hi, ref.res), "pageable")
            pin = _ResultBuffers(cap + 8, 64, None, pinned=True)
            pin.list_n[:] = 7
            pin.res.list_cap = cap  # the last 8 entries lie past the caller's room
            B.check(B.sv_verify_range(v.ctx, lo, hi, pin.res), "pinned")
            a, b = ref.result(), pin.result()
            assert a.hist == b.hist and a.list_len == b.list_len and a.list_len > 16
            assert np.array_equal(a.list_n, b.list_n) and np.array_equal(a.list_k, b.list_k)
            assert len(b.list_n) == min(cap, b.list_len)
            assert (pin.list_n[cap:] == 7).all()


def test_batch_graph_replay_and_recapture(orc):
    """Consecutive batches replay one captured graph; a batch that needs larger
    buffers re-captures it.  Every result equals the oracle's."""
    with Verifier(max_hi=(1 << 50) + (1 << 28)) as v:
        b1 = inputs.batch_requests(7, 40)
        b1 = [(lo, lo + min(hi - lo, 1 << 20)) for lo, hi in b1]
        b2 = inputs.batch_requests(8, 40)
        b2 = [(lo, lo + min(hi - lo, 1 << 19)) for lo, hi in b2]
        b3 = b2[:5] + [((1 << 44) + 1, (1 << 44) + 1 + (1 << 26))]  # more tiles: new buffers
        for batch in (b1, b2, b1, b3):
            res = v.verify_batch([a for a, _ in batch], [b for _, b in batch], list_cap=4096)
            for (lo, hi), g in zip(batch, res):
                o = orc.verify_range(lo, hi)
                assert g.hist == o.hist and g.first_n == o.first_n
                assert np.array_equal(g.list_n, o.list_n)
        # device-resident form
        v.launch_batch([a for a, _ in b2], [b for _, b in b2])
        res = v.fetch_batch(list_cap=4096)
        for (lo, hi), g in zip(b2, res):
            assert g.hist == orc.verify_range(lo, hi).hist
