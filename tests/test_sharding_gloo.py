"""Shift-range sharding across ranks, on CPU with the gloo backend
(world size 2): the shard arithmetic and the single FP64 all-reduce give the
oracle's M2; a rank that fails before the collective is detected by the
other rank through the process-group timeout, with no GPU involved."""
import datetime
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2512_24685_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_ranges_cover_exactly():
    for d in (2, 7, 64, 1 << 20):
        for world in (1, 2, 3, 8):
            if world > d:
                continue
            spans = [shard.shard_range(d, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == d
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            sizes = [e - b for b, e in spans]
            assert max(sizes) - min(sizes) <= 1


def _worker(rank, world, port, N, seed, fail_rank, q):
    import torch.distributed as dist

    import oracle
    from paper_2512_24685_gb300 import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=6))
    psi = W.haar_state(N, seed)
    try:
        if rank == fail_rank:
            raise RuntimeError("injected failure before the collective")

        def partial(b, e):
            return oracle.sum4_xorfwht(psi, b, e), oracle.norm2(psi)
        S, n2 = shard.sum_sharded(N, partial)
        m2 = oracle.m2_from_sum(S, n2, N)
        q.put((rank, "ok", m2))
    except Exception as exc:  # reported to the parent
        q.put((rank, "error", repr(exc)))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run(world, N, seed, fail_rank=-1):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, N, seed, fail_rank, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    return sorted(out)


def test_two_rank_sharded_m2_matches_oracle():
    import oracle
    from paper_2512_24685_gb300 import workloads as W
    N = 7
    res = _run(2, N, 11)
    ref = oracle.m2(W.haar_state(N, 11))
    for rank, status, val in res:
        assert status == "ok", val
        assert abs(val - ref) < 1e-12


def test_failed_rank_is_detected_by_the_other():
    res = _run(2, 6, 12, fail_rank=1)
    by_rank = {r: (s, v) for r, s, v in res}
    assert by_rank[1][0] == "error" and "injected" in by_rank[1][1]
    assert by_rank[0][0] == "error"  # the collective did not complete
