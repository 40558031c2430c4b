"""Full-size workloads, in the benchmark's launch configuration, compared with
the oracle element by element.

C2 = [2^40, 2^40 + 2^34) (2^33 odd n) and C3 = [2^50 - 2^36, 2^50) (2^35 odd
n): the device-resident launch the benchmark times is compared, whole, with
the oracle's Algorithm 1 + Algorithm 2 over the same range (histogram, first
occurrences, sum and maximum of mink, the complete ascending list of n with
mink >= 6 and their exponents, failures).  The same range with a per-n output
must agree with it, and sampled per-n values and contiguous windows must equal
the oracle's.  C4 = the 4096 ranges of seed 7 at their drawn lengths, as one
batched graph launch, each range against the oracle.
"""
import numpy as np
import pytest

from paper_2411_01964_gb300 import inputs

pytestmark = pytest.mark.gpu


def odd_index_to_n(lo, i):
    return (max(lo, 3) | 1) + 2 * i


def assert_same(g, o):
    assert g.n_odd == o.n_odd
    assert g.hist == o.hist
    assert g.first_n == o.first_n
    assert g.ksum == o.ksum and g.kmax == o.kmax
    assert g.list_len == len(o.list_n)
    assert np.array_equal(g.list_n, o.list_n) and np.array_equal(g.list_k, o.list_k)
    assert g.fail_len == len(o.failures) and np.array_equal(g.failures, o.failures)


@pytest.mark.parametrize("name", ["C2", "C3"])
def test_full_config(gpu, orc, name):
    import torch
    lo, hi = inputs.CONFIGS[name]
    n_odd = (hi - (lo | 1) + 1) // 2

    # 1. the aggregate-only launch the benchmark times, whole, against the oracle
    gpu.launch_range(lo, hi)
    agg = gpu.fetch_range(list_cap=1 << 20)
    o = orc.verify_range(lo, hi, list_cap=1 << 20)
    assert not o.list_overflow
    assert_same(agg, o)
    assert sum(agg.hist) == n_odd and agg.fail_len == 0 and agg.kmax <= 13  # Theorem, Sec. 4

    # 2. the same range with a per-n output on the device
    per_n = torch.empty(n_odd, dtype=torch.uint8, device="cuda")
    gpu.launch_range(lo, hi, per_n)
    full = gpu.fetch_range(list_cap=1 << 20)
    assert_same(full, o)
    counts = np.zeros(256, dtype=np.int64)
    for c0 in range(0, n_odd, 1 << 30):
        counts += torch.bincount(per_n[c0:c0 + (1 << 30)].to(torch.int32), minlength=256).cpu().numpy()
    assert list(counts[1:64]) == o.hist[1:64] and counts[0] == 0 and counts[255] == 0

    # 3. sampled points against the definition (trial division)
    idx = np.array(inputs.random_points(17, 600, 0, 2 * n_odd), dtype=np.int64) // 2
    got = per_n[torch.tensor(idx, device="cuda")].cpu().numpy()
    pts = [odd_index_to_n(lo, int(i)) for i in idx]
    assert np.array_equal(got, orc.min_k(pts))

    # 4. contiguous windows of the per-n output against the oracle's
    for start in (0, n_odd // 2 + 12345, n_odd - (1 << 18)):
        a = odd_index_to_n(lo, start)
        b = a + 2 * (1 << 18)
        w = orc.verify_range(a, b, per_n=True)
        assert np.array_equal(per_n[start:start + (1 << 18)].cpu().numpy(), w.per_n_k)

    # 5. every listed n sits at its index of the per-n output with its mink
    li = torch.tensor(((o.list_n.astype(np.int64) - (lo | 1)) // 2), device="cuda")
    assert np.array_equal(per_n[li].cpu().numpy(), o.list_k)
    del per_n, li
    torch.cuda.empty_cache()


def test_full_batch_C4(orc):
    """All 4096 ranges of seed 7 at their drawn lengths (starts odd in
    [2^30, 2^50), lengths 2^10..2^28), as the benchmark launches them."""
    from paper_2411_01964_gb300 import Verifier
    reqs = inputs.batch_requests(7, 4096)
    with Verifier(max_hi=inputs.TABLE_MAX_HI) as v:
        v.launch_batch([a for a, _ in reqs], [b for _, b in reqs])
        res = v.fetch_batch(list_cap=4096, fail_cap=16)
    want = orc.verify_ranges(reqs)
    assert sum(r.n_odd for r in res) == sum(o.n_odd for o in want)
    for (lo, hi), g, o in zip(reqs, res, want):
        assert g.lo == lo and g.hi == hi
        assert_same(g, o)
