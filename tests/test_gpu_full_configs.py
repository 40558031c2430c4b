"""Full-size workloads in the benchmark's launch configuration, checked by
sampling against the oracle and by properties that hold at any size.

C2 = [2^40, 2^40 + 2^34) (2^33 odd n) and C3 = [2^50 - 2^36, 2^50) (2^35 odd
n) are too large for the oracle to redo in a test, so:
  * every odd n is accounted for (sum of the histogram = n_odd, no failures,
    mink <= 13 below 2^50 as the Theorem of Sec. 4 states);
  * the device-resident launch with a per-n output agrees with the
    aggregate-only launch the benchmark times;
  * sampled per-n values and contiguous sub-windows (start, middle, tail)
    equal the oracle's, and every listed n and every first occurrence has the
    exponent the oracle assigns to it by trial division;
  * the histogram fractions sit where Table 2's heuristic puts them.
"""
import numpy as np
import pytest

from paper_2411_01964_gb300 import inputs

pytestmark = pytest.mark.gpu

# Table 2 (Sec. 2): c_k - c_{k-1}, the heuristic probability that mink = k
TABLE2 = {1: 8.1056e-1, 2: 1.6530e-1, 3: 2.1980e-2, 4: 2.0092e-3, 5: 1.3216e-4, 6: 6.5857e-6}


def odd_index_to_n(lo, i):
    return (max(lo, 3) | 1) + 2 * i


@pytest.mark.parametrize("name", ["C2", "C3"])
def test_full_config(gpu, orc, name):
    import torch
    lo, hi = inputs.CONFIGS[name]
    n_odd = (hi - (lo | 1) + 1) // 2

    # 1. aggregate-only launch (what the benchmark times)
    gpu.launch_range(lo, hi)
    agg = gpu.fetch_range(list_cap=1 << 20)
    assert sum(agg.hist) == n_odd and agg.fail_len == 0
    assert agg.kmax <= 13
    assert agg.list_len == sum(agg.hist[6:]) == len(agg.list_n)
    for k, p in TABLE2.items():
        mean = n_odd * p
        assert abs(agg.hist[k] - mean) < 6 * mean ** 0.5 + 0.01 * mean, (k, agg.hist[k], mean)

    # 2. the same range with a per-n output on the device
    per_n = torch.empty(n_odd, dtype=torch.uint8, device="cuda")
    gpu.launch_range(lo, hi, per_n)
    full = gpu.fetch_range(list_cap=1 << 20)
    assert full.hist == agg.hist and full.first_n == agg.first_n
    assert np.array_equal(full.list_n, agg.list_n)
    counts = np.zeros(256, dtype=np.int64)
    for c0 in range(0, n_odd, 1 << 30):
        counts += torch.bincount(per_n[c0:c0 + (1 << 30)].to(torch.int32), minlength=256).cpu().numpy()
    assert list(counts[1:64]) == agg.hist[1:64] and counts[0] == 0 and counts[255] == 0

    # 3. sampled points against the definition (trial division)
    idx = np.array(inputs.random_points(17, 600, 0, 2 * n_odd), dtype=np.int64) // 2
    got = per_n[torch.tensor(idx, device="cuda")].cpu().numpy()
    pts = [odd_index_to_n(lo, int(i)) for i in idx]
    assert np.array_equal(got, orc.min_k(pts))

    # 4. contiguous windows against the oracle's range verification
    for start in (0, n_odd // 2 + 12345, n_odd - (1 << 18)):
        a = odd_index_to_n(lo, start)
        b = a + 2 * (1 << 18)
        o = orc.verify_range(a, b, per_n=True)
        assert np.array_equal(per_n[start:start + (1 << 18)].cpu().numpy(), o.per_n_k)

    # 5. listed n and first occurrences carry the oracle's exponent
    sample = agg.list_n[:: max(1, len(agg.list_n) // 48)][:48]
    ks = agg.list_k[:: max(1, len(agg.list_n) // 48)][:48]
    assert np.array_equal(orc.min_k(sample), ks)
    firsts = [(k, agg.first_n[k]) for k in range(1, 14) if agg.first_n[k] != (1 << 64) - 1]
    assert list(orc.min_k([n for _, n in firsts])) == [k for k, _ in firsts]
    del per_n
    torch.cuda.empty_cache()
