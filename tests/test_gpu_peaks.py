"""The microbenchmarks behind the rooflines (sv_measure_peaks): each probe must
report a positive rate no larger than the hardware can issue, so that a
fraction against it means something."""
import pytest

from paper_2411_01964_gb300 import B, Verifier

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_sane():
    with Verifier(max_hi=1 << 20) as v:
        pk = B.sv_measure_peaks(v.ctx)
    sms, mhz = pk["sms"], pk["sm_clock_max_mhz"]
    assert sms > 0 and mhz > 0
    lanes = sms * 128 * mhz * 1e6        # 128 integer lanes per SM and clock at most
    for name in ("int_alu_ops_per_s", "scan_mix_ops_per_s"):
        assert 0.05 * lanes < pk[name] <= 1.1 * lanes, (name, pk[name], lanes)
    assert 0 < pk["popc_per_s"] <= 1.1 * lanes
    # one shared-memory atomic instruction serves at most a warp per clock
    for name in ("smem_atomic_per_s", "smem_atomic_strike_per_s"):
        assert 0 < pk[name] <= 1.1 * sms * 32 * mhz * 1e6, (name, pk[name])
    # bank conflicts can only slow the atomics down
    assert pk["smem_atomic_strike_per_s"] <= 1.1 * pk["smem_atomic_per_s"]
