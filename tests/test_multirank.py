"""Replica aggregation of bench.py on two gloo ranks (CPU): max-over-ranks timing and the
whole-job rate; no collective touches the data path."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    r, w, lr = bench.dist_env()
    seconds = [1.5, 2.5][rank]
    mx = bench.max_over_ranks(seconds, w)
    rate = bench.whole_job_rate(10, w, mx)
    dist.barrier()
    q.put((r, w, lr, mx, rate))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for r, w, lr, mx, rate in out:
        assert w == 2 and lr == r
        assert mx == pytest.approx(2.5)
        assert rate == pytest.approx(20 / 2.5)


def test_single_rank_identity():
    import bench

    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.whole_job_rate(4, 1, 2.0) == 2.0
