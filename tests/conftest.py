import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
for p in (ROOT, os.path.join(ROOT, "tests", "golden")):
    if p not in sys.path:
        sys.path.insert(0, p)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: runs the CUDA library on a GPU and compares it with the CPU oracle")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def gpu():
    """A library context with the prime table for every workload (hi <= 2^50 + 2^28)."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("gpu-marked test without a CUDA device")
    from paper_2411_01964_gb300 import Verifier
    from paper_2411_01964_gb300.inputs import TABLE_MAX_HI
    v = Verifier(max_hi=TABLE_MAX_HI)
    yield v
    v.close()
