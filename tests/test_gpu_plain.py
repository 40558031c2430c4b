"""The plain (unfused) path: Algorithm 1 writes the bitmap to device memory
(bulk stores), Algorithm 2 reads it back (bulk loads).  Its results must be
the oracle's, element by element, for every range and launch shape, and equal
the fused path's at full size."""
import numpy as np
import pytest

from paper_2411_01964_gb300 import Verifier, inputs

pytestmark = pytest.mark.gpu


def assert_same_range(g, o, per_n=True):
    assert g.n_odd == o.n_odd
    assert g.hist == o.hist and g.first_n == o.first_n
    assert g.ksum == o.ksum and g.kmax == o.kmax
    assert np.array_equal(g.list_n, o.list_n) and np.array_equal(g.list_k, o.list_k)
    assert np.array_equal(np.sort(g.failures), np.sort(o.failures))
    if per_n:
        assert np.array_equal(g.per_n_k, o.per_n_k)


RANGES = [
    (3, 4), (0, 3), (4, 4), (1, 100), (3, 1000), (3, 8193),     # near 0: windows partly below 1
    (63, 200), (3, 1 << 16),
    ((1 << 40) + 1, (1 << 40) + 2),
    ((1 << 40) + 12345, (1 << 40) + 12345 + (1 << 23) + 777),  # several tiles, ragged tail
    ((1 << 50) - (1 << 36) + 1001, (1 << 50) - (1 << 36) + 1001 + (1 << 22) + 333),
    (6915752957 - (1 << 20), 6915752957 + (1 << 20)),          # contains Table 3's n_9
]


@pytest.mark.parametrize("lo,hi", RANGES)
def test_plain_ranges(gpu, orc, lo, hi):
    o = orc.verify_range(lo, hi, per_n=True)
    assert_same_range(gpu.verify_range_plain(lo, hi, per_n=True), o)
    assert_same_range(gpu.verify_range_plain(lo, hi), o, per_n=False)  # lean scan, ordered list


KNOBS = [
    dict(tile_log2=14, margin_log2=6),    # one margin word: bulk stores are not aligned, plain stores instead
    dict(tile_log2=15, margin_log2=7),    # two margin words
    dict(tile_log2=16, margin_log2=17, threads=256),
    dict(tile_log2=20, margin_log2=18),
    dict(tile_log2=17, record_k_threshold=3),
]


@pytest.mark.parametrize("knobs", KNOBS, ids=lambda k: "-".join(f"{a}{b}" for a, b in k.items()))
def test_plain_knobs(orc, knobs):
    with Verifier(max_hi=(1 << 50) + (1 << 24), **knobs) as v:
        for lo, hi in [(3, 1 << 22), ((1 << 40) + 7, (1 << 40) + 7 + (1 << 22) + 99),
                       ((1 << 50) - (1 << 22) - 11, (1 << 50) + 5)]:
            o = orc.verify_range(lo, hi, per_n=True, list_k_threshold=v.config.record_k_threshold)
            assert_same_range(v.verify_range_plain(lo, hi, per_n=True), o)
            assert_same_range(v.verify_range_plain(lo, hi), o, per_n=False)


def test_plain_device_resident_and_fused_agree(gpu, orc):
    import torch
    lo, hi = (1 << 44) + 999, (1 << 44) + 999 + 3 * (1 << 21) + 55
    n = (hi - (lo | 1) + 1) // 2
    d = torch.full((n,), 77, dtype=torch.uint8, device="cuda")
    gpu.launch_range_plain(lo, hi, d)
    g = gpu.fetch_range()
    g.per_n_k = d.cpu().numpy()
    assert_same_range(g, orc.verify_range(lo, hi, per_n=True))


@pytest.mark.parametrize("name", ["C2", "C3"])
def test_plain_full_config(gpu, orc, name):
    lo, hi = inputs.CONFIGS[name]
    gpu.launch_range_plain(lo, hi)
    plain = gpu.fetch_range(list_cap=1 << 20)
    o = orc.verify_range(lo, hi, list_cap=1 << 20)
    assert_same_range(plain, o, per_n=False)
    assert plain.list_len == len(o.list_n)


def test_sieve_bitmap_unaligned_buffer(gpu, orc):
    # an output 4 bytes past a 16-byte boundary takes the plain stores
    import torch
    from paper_2411_01964_gb300 import B
    lo, hi = (1 << 40) + 12345, (1 << 40) + 12345 + 3 * (1 << 21) + 77
    nw = B.sv_bitmap_words(lo, hi)
    buf = torch.zeros(nw + 4, dtype=torch.int32, device="cuda")
    assert B.sv_sieve_bitmap(gpu.ctx, lo, hi, buf.data_ptr() + 4) == B.SV_OK
    got = buf[1:nw + 1].cpu().numpy()
    assert np.array_equal(got, gpu.sieve_bitmap(lo, hi).cpu().numpy())
    bits = np.unpackbits(got.view(np.uint8), bitorder="little")
    first = lo | 1
    f0 = (first - 1) // 2 - 32 * (lo // 64)
    cnt = (hi - first + 1) // 2
    assert np.array_equal(bits[f0:f0 + cnt], orc.sieve_odd(lo, hi))


def test_bounded_wait_runs_out_and_the_context_stays_usable(orc):
    # the scan pass's wait for a window's bulk load is bounded; with the loads
    # left out on purpose (nothing in flight), every block gives up, the call
    # returns SV_ETIMEDOUT, and the next calls are correct
    from paper_2411_01964_gb300 import B
    lo, hi = (1 << 40) + 12345, (1 << 40) + 12345 + (1 << 23) + 777
    with Verifier(max_hi=1 << 41) as v:
        B.sv_inject_bulk_timeout(v.ctx, 1)
        with pytest.raises(B.SvError) as e:
            v.verify_range_plain(lo, hi)
        assert e.value.status == B.SV_ETIMEDOUT
        o = orc.verify_range(lo, hi, per_n=True)
        assert_same_range(v.verify_range_plain(lo, hi, per_n=True), o)
        assert_same_range(v.verify_range(lo, hi, per_n=True), o)
