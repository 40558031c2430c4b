"""Splitting one range over several processes (one GPU each) and merging the
per-rank results exactly.

Disjoint sub-ranges are independent: each rank's tiles re-sieve their own
look-back margin, so no halo exchange is needed.  The only communication is
the final merge of small aggregates (Sec. 3 "Collecting the results"): sums of
the histograms, minima of the first occurrences, the maximum exponent, and the
union of the lists.  The merge is associative, so any split gives the result
of the unsplit range.
"""
from __future__ import annotations

import numpy as np

NO_N = (1 << 64) - 1


def shard_range(lo: int, hi: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous piece `rank` of [lo, hi) split into `world` pieces with even
    inner boundaries, so every odd n lands in exactly one piece."""
    if hi <= lo:
        return lo, lo
    span = hi - lo
    cuts = [lo + (span * r // world) for r in range(world + 1)]
    cuts = [cuts[0]] + [c & ~1 for c in cuts[1:-1]] + [cuts[-1]]
    a, b = cuts[rank], cuts[rank + 1]
    return a, max(a, b)


def merge_results(res, group=None) -> dict:
    """All-reduce one rank's range result (an object with hist, first_n,
    list_n, list_k, failures, n_odd) over torch.distributed; every rank gets
    the merged dict."""
    import torch
    import torch.distributed as dist

    hist = torch.tensor(np.asarray(res.hist, dtype=np.int64))
    dist.all_reduce(hist, op=dist.ReduceOp.SUM, group=group)
    # first occurrences: min over ranks (NO_N does not fit int64: map it to max)
    first = np.asarray([x if x != NO_N else (1 << 63) - 1 for x in res.first_n], dtype=np.int64)
    first_t = torch.tensor(first)
    dist.all_reduce(first_t, op=dist.ReduceOp.MIN, group=group)
    n_odd = torch.tensor([int(res.n_odd)], dtype=torch.int64)
    dist.all_reduce(n_odd, op=dist.ReduceOp.SUM, group=group)
    world = dist.get_world_size(group)
    lists = [None] * world
    dist.all_gather_object(lists, (np.asarray(res.list_n).tolist(), np.asarray(res.list_k).tolist(),
                                   np.asarray(res.failures).tolist()), group=group)
    pairs = sorted((n, k) for ln, lk, _ in lists for n, k in zip(ln, lk))
    fails = sorted(f for _, _, fl in lists for f in fl)
    h = [int(x) for x in hist.tolist()]
    return {
        "n_odd": int(n_odd.item()),
        "hist": h,
        "first_n": [int(x) if x != (1 << 63) - 1 else NO_N for x in first_t.tolist()],
        "ksum": sum(k * c for k, c in enumerate(h)),
        "kmax": max((k for k, c in enumerate(h) if c), default=0),
        "list_n": np.array([n for n, _ in pairs], dtype=np.uint64),
        "list_k": np.array([k for _, k in pairs], dtype=np.uint8),
        "failures": np.array(fails, dtype=np.uint64),
    }
