"""The multi-process path on CPU: two gloo ranks each verify their piece of a
range (the per-rank compute is the oracle here; on GPUs it is the library),
merge with torch.distributed, and must reproduce the unsplit range exactly.
A rank that fails before the merge makes the others fail fast, not hang."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2411_01964_gb300.shard import shard_range


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, lo, hi, q, fail_rank):
    import datetime

    import torch.distributed as dist

    import oracle
    from paper_2411_01964_gb300.shard import merge_results
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    try:
        if rank == fail_rank:
            raise RuntimeError("injected failure before the merge")
        a, b = shard_range(lo, hi, rank, world)
        r = oracle.verify_range(a, b, list_k_threshold=5, threads=2)
        m = merge_results(r)
        q.put((rank, "ok", m["hist"], m["first_n"], m["list_n"].tolist(), m["n_odd"]))
    except Exception as e:  # reported to the parent; the process exits
        q.put((rank, "error", repr(e), None, None, None))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def test_shard_boundaries_partition_odd_numbers():
    for lo, hi, w in [(3, 1000, 2), (3, 1001, 3), ((1 << 40) + 1, (1 << 40) + 12345, 4), (10, 11, 2)]:
        pieces = [shard_range(lo, hi, r, w) for r in range(w)]
        odds = [n for a, b in pieces for n in range(a | 1, b, 2) if n >= max(lo, 3)]
        assert odds == [n for n in range(max(lo, 3) | 1, hi, 2)]


def test_two_rank_merge_equals_single_range(orc):
    lo, hi = (1 << 38) + 7, (1 << 38) + 7 + (1 << 22) + 12
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, lo, hi, q, -1)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    want = orc.verify_range(lo, hi, list_k_threshold=5)
    for rank, status, hist, first, lst, n_odd in out:
        assert status == "ok", hist
        assert hist == want.hist and first == want.first_n and n_odd == want.n_odd
        assert np.array_equal(np.array(lst, dtype=np.uint64), want.list_n)


def test_failed_rank_does_not_hang_the_other():
    lo, hi = (1 << 30) + 1, (1 << 30) + (1 << 20)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, lo, hi, q, 1)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, status, *_ = q.get(timeout=120)
        out[rank] = status
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
            pytest.fail("a rank hung after its peer failed")
    assert out == {0: "error", 1: "error"}
