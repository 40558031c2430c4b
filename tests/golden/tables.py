"""Readers for the values the paper prints (tests/golden/*.txt)."""
import os

_HERE = os.path.dirname(os.path.abspath(__file__))


def _pairs(name):
    out = {}
    with open(os.path.join(_HERE, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                a, b = line.split()
                out[int(a)] = int(b)
    return out


def table4_histogram():
    """{k: count} for odd 1 < n < 2^30 (Table 4)."""
    return _pairs("table4_histogram_below_2p30.txt")


def table3_records():
    """{m: smallest odd n with n - 2^1..n - 2^m all not squarefree} (Table 3)."""
    return _pairs("table3_records.txt")
