"""The benchmark's multi-rank logic on CPU: two gloo ranks (one process per
rank, rendezvous on 127.0.0.1) agree on the max over ranks, and the
whole-job rate counts every rank's units over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = bench.dist_setup()
    ms = 10.0 + 5.0 * rank                      # rank 1 is the slow one
    mx = bench.reduce_max(ms, w, device="cpu")
    q.put((r, w, lr, mx, bench.whole_job_rate(1000.0, w, mx)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[3] == 15.0 for o in out)
    assert out[0][4] == pytest.approx(2 * 1000.0 / 0.015)


def test_single_rank_is_identity():
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == pytest.approx(5000.0)
