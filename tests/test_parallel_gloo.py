"""The multi-GPU host logic with two CPU ranks over gloo: instance sharding
without overlap, max-over-ranks timing, the global best and the global
termination flag across ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2504_00987_gb300 import parallel


def test_shard_and_split():
    assert parallel.shard(4, 0, 1024) == (0, 1024)
    assert parallel.shard(4, 3, 1024) == (3072, 1024)
    ranges = [parallel.split_range(10, 4, r) for r in range(4)]
    assert ranges == [(0, 3), (3, 3), (6, 2), (8, 2)]
    covered = sorted(i for f, c in ranges for i in range(f, f + c))
    assert covered == list(range(10))
    with pytest.raises(ValueError):
        parallel.shard(2, 2, 10)
    with pytest.raises(ValueError):
        parallel.shard(2, 1, (1 << 31) + 1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first, count = parallel.shard(world, rank, 8)
        # rank 1 is the slow one and owns the best energy
        local_ms = [10.0 + 5.0 * rank, 3.0 - rank]
        mx = parallel.max_over_ranks(dist, local_ms)
        tot = parallel.sum_over_ranks(dist, [float(count)])
        E = 100 - 7 * rank
        best = parallel.best_over_ranks(dist, E, first + 3)
        out[rank] = (first, count, mx, tot, best)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][:2] == (0, 8) and res[1][:2] == (8, 8)
    for r in range(2):
        assert res[r][2] == [15.0, 3.0]
        assert res[r][3] == [16.0]
        assert res[r][4] == (93, 11)


def _glf_worker(rank, world, port, reach_at, out):
    """Rank r "reaches" the target in slice reach_at[r] (None: never), on the host."""
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ran = []

        def run_slice(i):
            ran.append(i)
            return reach_at[rank] is not None and i >= reach_at[rank]

        out[rank] = (parallel.run_until_any(dist, run_slice, 10), ran)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("reach_at,expect", [((None, 3), (4, True)), ((5, 2), (3, True)),
                                             ((None, None), (10, False))])
def test_glf_across_two_gloo_ranks(reach_at, expect):
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_glf_worker, args=(r, 2, port, reach_at, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):  # both ranks stop after the same slice, as soon as one reached
        assert res[r][0] == expect
        assert res[r][1] == list(range(expect[0]))


def test_glf_one_process():
    assert parallel.run_until_any(None, lambda i: i == 2, 5) == (3, True)
    assert parallel.run_until_any(None, lambda i: False, 5) == (5, False)
    with pytest.raises(ValueError):
        parallel.run_until_any(None, lambda i: False, -1)
